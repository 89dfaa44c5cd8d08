// ltne_reduce.cu -- FP64 reduction of the macroscopic fields to the
// observables (wall Nusselt numbers, mass, energy, extrema, means, the
// steady-state residual and a non-finite count).
//
// Two passes with a fixed summation order, so results are bitwise
// reproducible for a given lattice size: pass 1 writes one partial vector per
// block (RB columns x SEG rows) into a scratch buffer; pass 2 (one block)
// reduces the partials in block order.  Per-node terms are accumulated in
// the fields' precision over at most SEG nodes per thread (FP64 on GB300
// runs at a small fraction of the FP32 rate, so FP64 per node would make
// this pass compute-bound); every combination above that is FP64.
#include "ltne_internal.h"

namespace ltne {

namespace {

constexpr int RB = 256;  // threads per block in both passes
constexpr int SEG = 64;  // rows per pass-1 block

__device__ __forceinline__ double combine(int k, double a, double b) {
  return (k == A_MAXU || k == A_MAXDT) ? fmax(a, b) : a + b;
}

// Block-wide reduction of NACC accumulators per thread into acc of
// thread 0 (fixed shuffle and warp order).
__device__ void block_reduce(double (&acc)[NACC], double* sh /* [RB/32][NACC] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NACC; ++k) {
    double v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = combine(k, v, __shfl_down_sync(0xffffffffu, v, o));
    acc[k] = v;
  }
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NACC; ++k) sh[warp * NACC + k] = acc[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < RB / 32; ++w)
#pragma unroll
      for (int k = 0; k < NACC; ++k) acc[k] = combine(k, acc[k], sh[w * NACC + k]);
  }
}

// Pass 1.  Block (RB threads) covers RB consecutive columns and SEG rows;
// each thread walks its column down the segment (coalesced rows across the
// warp), accumulating in the fields' own precision C over at most SEG nodes,
// then everything from the per-thread partials upward is combined in FP64.
template <typename C>
__global__ void __launch_bounds__(RB) k_reduce_pass1(ReduceArgs a) {
  __shared__ double sh[(RB / 32) * NACC];
  C acc[NACC];
#pragma unroll
  for (int k = 0; k < NACC; ++k) acc[k] = C(0);
  const C* mac = static_cast<const C*>(a.mac);
  const C* phi_f = static_cast<const C*>(a.phi);
  C* prev = static_cast<C*>(a.prev);
  const int x = blockIdx.x * RB + threadIdx.x;
  const int y0 = blockIdx.y * SEG;
  const int y1 = min(y0 + SEG, a.ny);
  const C phi_u = C(a.phi_u), sigma = C(a.sigma);
  // Wall-flux stencil weights: q_hot = 1.5 T_h - 2 T(1,y) + 0.5 T(2,y),
  // q_cold = -1.5 T_c + 2 T(nx-2,y) - 0.5 T(nx-3,y), trapezoid rule in y.
  const C whot = (x == 1) ? C(-2) : (x == 2) ? C(0.5) : C(0);
  const C wcold = (x == a.nx - 2) ? C(2) : (x == a.nx - 3) ? C(-0.5) : C(0);
  if (x < a.nx) {
    for (int y = y0; y < y1; ++y) {
      const int64_t off = (int64_t)y * a.pitch + x;
      // deviations: rho - 1, ux, uy, T_f - T0, T_s - T0
      const C rho = mac[off], ux = mac[a.plane + off], uy = mac[2 * a.plane + off];
      const C Tf = mac[3 * a.plane + off], Ts = mac[4 * a.plane + off];
      const C phi = phi_f ? phi_f[off] : phi_u;
      const C wy = (y == 0 || y == a.ny - 1) ? C(0.5) : C(1);
      acc[A_NUF_H] += whot * wy * Tf;
      acc[A_NUS_H] += whot * wy * Ts;
      acc[A_NUF_C] += wcold * wy * Tf;
      acc[A_NUS_C] += wcold * wy * Ts;
      acc[A_MASS] += rho;
      // deviation part of phi T_f + (1-phi) sigma T_s; the T0 and Q parts
      // are restored from the porosity sum in FP64
      acc[A_ENERGY] += phi * Tf + (C(1) - phi) * sigma * Ts;
      acc[A_SUMPHI] += phi;
      const C u2 = ux * ux + uy * uy;
      acc[A_MAXU] = u2 > acc[A_MAXU] ? u2 : acc[A_MAXU];  // |u|^2, rooted in FP64
      const C dT = Tf > Ts ? Tf - Ts : Ts - Tf;
      acc[A_MAXDT] = dT > acc[A_MAXDT] ? dT : acc[A_MAXDT];
      acc[A_SUMTF] += Tf;
      acc[A_SUMTS] += Ts;
      const C pux = prev[off], puy = prev[a.plane + off];
      const C pTf = prev[2 * a.plane + off], pTs = prev[3 * a.plane + off];
      acc[A_DU2] += (ux - pux) * (ux - pux) + (uy - puy) * (uy - puy);
      acc[A_U2] += u2;
      acc[A_DTF2] += (Tf - pTf) * (Tf - pTf);
      acc[A_TF2] += Tf * Tf;
      acc[A_DTS2] += (Ts - pTs) * (Ts - pTs);
      acc[A_TS2] += Ts * Ts;
      if (!(isfinite(rho) && isfinite(ux) && isfinite(uy) && isfinite(Tf) && isfinite(Ts)))
        acc[A_BAD] += C(1);
      if (a.update_prev) {
        prev[off] = ux;
        prev[a.plane + off] = uy;
        prev[2 * a.plane + off] = Tf;
        prev[3 * a.plane + off] = Ts;
      }
    }
  }
  double dacc[NACC];
#pragma unroll
  for (int k = 0; k < NACC; ++k) dacc[k] = (double)acc[k];
  block_reduce(dacc, sh);
  if (threadIdx.x == 0) {
    const int64_t b = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
#pragma unroll
    for (int k = 0; k < NACC; ++k) a.partials[b * NACC + k] = dacc[k];
  }
}

__global__ void __launch_bounds__(RB) k_reduce_pass2(const double* __restrict__ partials,
                                                     int blocks, double* __restrict__ out) {
  __shared__ double sh[(RB / 32) * NACC];
  double acc[NACC];
#pragma unroll
  for (int k = 0; k < NACC; ++k) acc[k] = 0.0;
  for (int b = threadIdx.x; b < blocks; b += RB)
#pragma unroll
    for (int k = 0; k < NACC; ++k) acc[k] = combine(k, acc[k], partials[(int64_t)b * NACC + k]);
  block_reduce(acc, sh);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NACC; ++k) out[k] = acc[k];
}

}  // namespace

int reduce_blocks(int nx, int ny) {
  return ((nx + RB - 1) / RB) * ((ny + SEG - 1) / SEG);
}

cudaError_t launch_reduce(const ReduceArgs& a, cudaStream_t st) {
  dim3 grid((a.nx + RB - 1) / RB, (a.ny + SEG - 1) / SEG);
  if ((int)(grid.x * grid.y) != a.blocks) return cudaErrorInvalidValue;
  if (a.is_double)
    k_reduce_pass1<double><<<grid, RB, 0, st>>>(a);
  else
    k_reduce_pass1<float><<<grid, RB, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_reduce_pass2<<<1, RB, 0, st>>>(a.partials, a.blocks, a.out);
  return cudaGetLastError();
}

}  // namespace ltne
