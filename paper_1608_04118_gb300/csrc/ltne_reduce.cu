// ltne_reduce.cu -- FP64 reduction of the macroscopic fields to the
// observables (wall Nusselt numbers, mass, energy, extrema, means, the
// steady-state residual and a non-finite count).
//
// Two passes with a fixed summation order, so results are bitwise
// reproducible for a given lattice size: pass 1 writes one partial vector per
// block (RB columns x seg rows) into a scratch buffer; pass 2 reduces the
// partials in block order.  FP64 on GB300 runs at a small fraction of the
// FP32 rate, so a thread of pass 1 sums its nodes' terms in the fields'
// precision over its column segment (seg <= 64 rows) and only the threads'
// sums are combined in FP64, through shared memory in a fixed order.  The
// wall-flux integrals of Nu touch four columns only: pass 2 forms them in
// FP64 from the first add while it combines the partials.  (Two-part FP32
// sums with error-free additions for every term of every node made pass 1
// bound by FP32 arithmetic, 0.32 ms at 4096^2.)
#include "ltne_internal.h"

namespace ltne {

namespace {

constexpr int RB = 256;  // threads per block in both passes
// Rows per pass-1 block: 64, 32 or 16, the longest that still gives 2048
// blocks (about three waves of the 4-5 blocks an SM holds: enough resident
// warps to keep the loads in flight, and a short last wave), within
// kReduceMaxBlocks.  (1024 blocks of 64 rows at 4096^2: 0.22 ms per call.)
int reduce_seg(int nx, int ny) {
  const int64_t cols = (nx + RB - 1) / RB;
  for (int seg = 64; seg >= 16; seg /= 2) {
    const int64_t b = cols * ((ny + seg - 1) / seg);
    if (b >= 2048 && b <= kReduceMaxBlocks) return seg;
  }
  for (int seg = 16; seg <= 64; seg *= 2)
    if (cols * ((ny + seg - 1) / seg) <= kReduceMaxBlocks) return seg;
  return 64;
}

__device__ __forceinline__ double cmax(double a, double b) { return fmax(a, b); }

template <typename C>
__device__ __forceinline__ C combine(int k, C a, C b) {
  return (k == A_MAXU || k == A_MAXDT) ? cmax(a, b) : a + b;
}

// Block-wide reduction of NACC accumulators per thread into acc of
// thread 0 (fixed shuffle and warp order).
__device__ void block_reduce(double (&acc)[NACC], double* sh /* [RB/32][NACC] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NACC; ++k) {
    double v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      v = combine<double>(k, v, __shfl_down_sync(0xffffffffu, v, o));
    acc[k] = v;
  }
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NACC; ++k) sh[warp * NACC + k] = acc[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < RB / 32; ++w)
#pragma unroll
      for (int k = 0; k < NACC; ++k) acc[k] = combine<double>(k, acc[k], sh[w * NACC + k]);
  }
}

static_assert(A_NUF_H == 0 && A_NUS_H == 1 && A_NUF_C == 2 && A_NUS_C == 3 && A_MASS == 4,
              "the Nu slots come first");

// Pass 1.  Block (RB threads) covers RB consecutive columns and seg rows;
// each thread walks its column down the segment (coalesced rows across the
// warp).  Rows go in groups of RU (4 in FP32, 2 in FP64, which holds twice
// the registers per value): all loads of a group are issued before any of
// its snapshot stores, so a thread keeps RU rows of loads in flight.
template <typename C>
__global__ void __launch_bounds__(RB) k_reduce_pass1(ReduceArgs a, int seg) {
  constexpr int RU = sizeof(C) == 4 ? 4 : 2;
  __shared__ double sh[NACC][RB];
  const int t = threadIdx.x;
  C acc[NACC];  // the thread's sums (slots from A_MASS on)
#pragma unroll
  for (int k = 0; k < NACC; ++k) acc[k] = C(0);
  const C* __restrict__ mac = static_cast<const C*>(a.mac);
  const C* __restrict__ phi_f = static_cast<const C*>(a.phi);
  C* __restrict__ prev = static_cast<C*>(a.prev);
  const int64_t pl = a.plane;
  const int x = blockIdx.x * RB + threadIdx.x;
  const int y0 = blockIdx.y * seg;
  const int y1 = min(y0 + seg, a.ny);
  const C phi_u = C(a.phi_u), sigma = C(a.sigma);
  if (x < a.nx) {
#pragma unroll 1
    for (int yg = y0; yg < y1; yg += RU) {
      // deviations: rho - 1, ux, uy, T_f - T0, T_s - T0; the previous
      // snapshot of ux, uy, T_f, T_s
      C rho[RU], ux[RU], uy[RU], Tf[RU], Ts[RU], phi[RU], pux[RU], puy[RU], pTf[RU], pTs[RU];
#pragma unroll
      for (int r = 0; r < RU; ++r) {
        const int y = min(yg + r, y1 - 1);  // a short last group re-reads its last row
        const int64_t off = (int64_t)y * a.pitch + x;
        rho[r] = mac[off];
        ux[r] = mac[pl + off];
        uy[r] = mac[2 * pl + off];
        Tf[r] = mac[3 * pl + off];
        Ts[r] = mac[4 * pl + off];
        phi[r] = phi_f ? phi_f[off] : phi_u;
        pux[r] = prev[off];
        puy[r] = prev[pl + off];
        pTf[r] = prev[2 * pl + off];
        pTs[r] = prev[3 * pl + off];
      }
#pragma unroll
      for (int r = 0; r < RU; ++r) {
        const int y = yg + r;
        if (y >= y1) break;
        acc[A_MASS] += rho[r];
        // deviation part of phi T_f + (1-phi) sigma T_s; the T0 and Q parts
        // are restored from the porosity sum in FP64
        acc[A_ENERGY] += phi[r] * Tf[r] + (C(1) - phi[r]) * sigma * Ts[r];
        acc[A_SUMPHI] += phi[r];
        const C u2 = ux[r] * ux[r] + uy[r] * uy[r];
        acc[A_MAXU] = u2 > acc[A_MAXU] ? u2 : acc[A_MAXU];  // |u|^2, rooted in FP64
        const C dT = Tf[r] > Ts[r] ? Tf[r] - Ts[r] : Ts[r] - Tf[r];
        acc[A_MAXDT] = dT > acc[A_MAXDT] ? dT : acc[A_MAXDT];
        acc[A_SUMTF] += Tf[r];
        acc[A_SUMTS] += Ts[r];
        acc[A_DU2] += (ux[r] - pux[r]) * (ux[r] - pux[r]) + (uy[r] - puy[r]) * (uy[r] - puy[r]);
        acc[A_U2] += u2;
        acc[A_DTF2] += (Tf[r] - pTf[r]) * (Tf[r] - pTf[r]);
        acc[A_TF2] += Tf[r] * Tf[r];
        acc[A_DTS2] += (Ts[r] - pTs[r]) * (Ts[r] - pTs[r]);
        acc[A_TS2] += Ts[r] * Ts[r];
        if (!(isfinite(rho[r]) && isfinite(ux[r]) && isfinite(uy[r]) && isfinite(Tf[r]) &&
              isfinite(Ts[r])))
          acc[A_BAD] += C(1);
      }
      if (a.update_prev) {
#pragma unroll
        for (int r = 0; r < RU; ++r) {
          const int y = yg + r;
          if (y >= y1) break;
          const int64_t off = (int64_t)y * a.pitch + x;
          prev[off] = ux[r];
          prev[pl + off] = uy[r];
          prev[2 * pl + off] = Tf[r];
          prev[3 * pl + off] = Ts[r];
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < NACC; ++k) sh[k][t] = (double)acc[k];  // the Nu slots stay 0
  // the block's threads in FP64, in a fixed order: eight column chunks of
  // 32 threads per accumulator, then the chunks
  __syncthreads();
  __shared__ double sh2[NACC][RB / 32];
  if (threadIdx.x < NACC * (RB / 32)) {
    const int k = threadIdx.x / (RB / 32), c = threadIdx.x % (RB / 32);
    double v = sh[k][c * 32];
    for (int i = 1; i < 32; ++i) v = combine<double>(k, v, sh[k][c * 32 + i]);
    sh2[k][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < NACC) {
    const int k = threadIdx.x;
    double v = sh2[k][0];
    for (int c = 1; c < RB / 32; ++c) v = combine<double>(k, v, sh2[k][c]);
    // accumulator-major: pass 2 reads each accumulator's partials contiguously
    const int64_t b = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    a.partials[(int64_t)k * a.blocks + b] = v;
  }
}

// Pass 2: block k forms accumulator k -- the partials of pass 1 in block
// order (contiguous, accumulator-major), or for the four Nu slots the
// wall-flux integral in FP64: q_hot = 1.5 T_h - 2 T(1,y) + 0.5 T(2,y) and
// q_cold = -1.5 T_c + 2 T(nx-2,y) - 0.5 T(nx-3,y) of one phase (their
// deviation parts; the wall terms are added on the host), trapezoid rule in
// y -- thread t taking rows or partials t, t + RB, ..., then the block tree.
template <typename C>
__global__ void __launch_bounds__(RB) k_reduce_pass2(ReduceArgs a) {
  __shared__ double sh[(RB / 32) * NACC];
  double acc[NACC];
#pragma unroll
  for (int k = 0; k < NACC; ++k) acc[k] = 0.0;
  const int k = blockIdx.x;
  double v = 0.0;
  if (k >= A_MASS) {
    const double* __restrict__ p = a.partials + (int64_t)k * a.blocks;
#pragma unroll 4
    for (int b = threadIdx.x; b < a.blocks; b += RB) v = combine<double>(k, v, p[b]);
  } else {
    const C* __restrict__ mac = static_cast<const C*>(a.mac);
    const C* __restrict__ T = mac + (k == A_NUF_H || k == A_NUF_C ? 3 : 4) * a.plane;
    const bool hot = k == A_NUF_H || k == A_NUS_H;
    const int c1 = hot ? 1 : a.nx - 2, c2 = hot ? 2 : a.nx - 3;
    const double w1 = hot ? -2.0 : 2.0, w2 = hot ? 0.5 : -0.5;
#pragma unroll 4
    for (int y = threadIdx.x; y < a.ny; y += RB) {
      const double wy = ((y == 0 && a.wall_lo) || (y == a.ny - 1 && a.wall_hi)) ? 0.5 : 1.0;
      const C* row = T + (int64_t)y * a.pitch;
      v += wy * (w1 * (double)row[c1] + w2 * (double)row[c2]);
    }
  }
  acc[k] = v;
  block_reduce(acc, sh);
  if (threadIdx.x == 0) a.out[k] = acc[k];
}

}  // namespace

int reduce_blocks(int nx, int ny) {
  const int seg = reduce_seg(nx, ny);
  return ((nx + RB - 1) / RB) * ((ny + seg - 1) / seg);
}

cudaError_t launch_reduce(const ReduceArgs& a, cudaStream_t st) {
  const int seg = reduce_seg(a.nx, a.ny);
  dim3 grid((a.nx + RB - 1) / RB, (a.ny + seg - 1) / seg);
  if ((int)(grid.x * grid.y) != a.blocks) return cudaErrorInvalidValue;
  if (a.is_double)
    k_reduce_pass1<double><<<grid, RB, 0, st>>>(a, seg);
  else
    k_reduce_pass1<float><<<grid, RB, 0, st>>>(a, seg);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (a.is_double)
    k_reduce_pass2<double><<<NACC, RB, 0, st>>>(a);
  else
    k_reduce_pass2<float><<<NACC, RB, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace ltne
