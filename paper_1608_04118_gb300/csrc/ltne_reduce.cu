// ltne_reduce.cu -- FP64 reduction of the macroscopic fields to the
// observables (wall Nusselt numbers, mass, energy, extrema, means, the
// steady-state residual and a non-finite count).
//
// Two passes with a fixed summation order, so results are bitwise
// reproducible for a given lattice size: pass 1 (grid-stride, fixed grid)
// writes one partial vector per block into a scratch buffer; pass 2 (one
// block) reduces the partials in block order.
#include "ltne_internal.h"

namespace ltne {

namespace {

constexpr int RB = 256;  // threads per block in both passes

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

template <typename C>
__global__ void __launch_bounds__(RB) k_reduce_pass1(ReduceArgs a) {
  __shared__ double sh[(RB / 32) * NACC];
  double acc[NACC];
#pragma unroll
  for (int k = 0; k < NACC; ++k) acc[k] = 0.0;
  const C* mac = static_cast<const C*>(a.mac);
  const C* phi_f = static_cast<const C*>(a.phi);
  C* prev = static_cast<C*>(a.prev);
  const int64_t n_nodes = (int64_t)a.nx * a.ny;
  const int64_t stride = (int64_t)gridDim.x * RB;
  for (int64_t n = (int64_t)blockIdx.x * RB + threadIdx.x; n < n_nodes; n += stride) {
    const int y = (int)(n / a.nx), x = (int)(n - (int64_t)y * a.nx);
    const int64_t off = (int64_t)y * a.pitch + x;
    const double rho = mac[off], ux = mac[a.plane + off], uy = mac[2 * a.plane + off];
    const double Tf = mac[3 * a.plane + off], Ts = mac[4 * a.plane + off];
    const double phi = phi_f ? (double)phi_f[off] : a.phi_u;
    // Wall-flux stencil weights: q_hot = 1.5 T_h - 2 T(1,y) + 0.5 T(2,y),
    // q_cold = -1.5 T_c + 2 T(nx-2,y) - 0.5 T(nx-3,y); trapezoid in y.
    const double wy = (y == 0 || y == a.ny - 1) ? 0.5 : 1.0;
    if (x == 1) { acc[A_NUF_H] += -2.0 * wy * Tf; acc[A_NUS_H] += -2.0 * wy * Ts; }
    if (x == 2) { acc[A_NUF_H] += 0.5 * wy * Tf; acc[A_NUS_H] += 0.5 * wy * Ts; }
    if (x == a.nx - 2) { acc[A_NUF_C] += 2.0 * wy * Tf; acc[A_NUS_C] += 2.0 * wy * Ts; }
    if (x == a.nx - 3) { acc[A_NUF_C] += -0.5 * wy * Tf; acc[A_NUS_C] += -0.5 * wy * Ts; }
    acc[A_MASS] += rho;
    acc[A_ENERGY] += phi * Tf + (1.0 - phi) * a.sigma * Ts
                     - 0.5 * (phi * a.qf + (1.0 - phi) * a.sigma * a.qs);
    const double u2 = ux * ux + uy * uy;
    acc[A_MAXU] = fmax(acc[A_MAXU], sqrt(u2));
    acc[A_MAXDT] = fmax(acc[A_MAXDT], fabs(Tf - Ts));
    acc[A_SUMTF] += Tf;
    acc[A_SUMTS] += Ts;
    const double pux = prev[off], puy = prev[a.plane + off];
    const double pTf = prev[2 * a.plane + off], pTs = prev[3 * a.plane + off];
    acc[A_DU2] += (ux - pux) * (ux - pux) + (uy - puy) * (uy - puy);
    acc[A_U2] += u2;
    acc[A_DTF2] += (Tf - pTf) * (Tf - pTf);
    acc[A_TF2] += Tf * Tf;
    acc[A_DTS2] += (Ts - pTs) * (Ts - pTs);
    acc[A_TS2] += Ts * Ts;
    if (!(isfinite(rho) && isfinite(ux) && isfinite(uy) && isfinite(Tf) && isfinite(Ts)))
      acc[A_BAD] += 1.0;
    if (a.update_prev) {
      prev[off] = mac[a.plane + off];
      prev[a.plane + off] = mac[2 * a.plane + off];
      prev[2 * a.plane + off] = mac[3 * a.plane + off];
      prev[3 * a.plane + off] = mac[4 * a.plane + off];
    }
  }
  block_reduce(acc, sh);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NACC; ++k) a.partials[(int64_t)blockIdx.x * NACC + k] = acc[k];
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

int reduce_blocks(int64_t nodes) {
  int64_t b = (nodes + RB * 8 - 1) / (RB * 8);
  if (b < 1) b = 1;
  if (b > 1216) b = 1216;  // 8 blocks per SM on 152 SMs
  return (int)b;
}

cudaError_t launch_reduce(const ReduceArgs& a, cudaStream_t st) {
  if (a.is_double)
    k_reduce_pass1<double><<<a.blocks, RB, 0, st>>>(a);
  else
    k_reduce_pass1<float><<<a.blocks, RB, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_reduce_pass2<<<1, RB, 0, st>>>(a.partials, a.blocks, a.out);
  return cudaGetLastError();
}

}  // namespace ltne
