// ltne_reduce.cu -- FP64 reduction of the macroscopic fields to the
// observables (wall Nusselt numbers, mass, energy, extrema, means, the
// steady-state residual and a non-finite count).
//
// Two passes with a fixed summation order, so results are bitwise
// reproducible for a given lattice size: pass 1 writes one partial vector per
// block (RB columns x seg rows) into a scratch buffer; pass 2 reduces the
// partials in block order.  Per-node terms of FP32 fields are summed over at
// most seg nodes per thread and across the 32 threads of a warp as two-part
// FP32 sums (error-free additions, ltne_obs.cuh): FP64 on GB300 runs at a
// small fraction of the FP32 rate, so FP64 per node -- or a warp shuffle
// tree in FP64 in every block -- would make this pass compute-bound, while
// the two-part sums carry about 48 significant bits at FP32 speed; every
// combination above the warp, the warps of a block and the blocks, is FP64.
// This pass serves the states whose last step did not accumulate the
// observables itself (after set_fields, a checkpoint restore, the slab and
// adjoint paths, the batched form and the allocation-free entry point).
#include "ltne_obs.cuh"

namespace ltne {

namespace {

constexpr int RB = 256;  // threads per block in both passes
// Rows per pass-1 block: the smallest of 16, 32, 64 that keeps the block
// count within kReduceMaxBlocks (more, shorter blocks keep more loads in
// flight: 2048^2 with 64 rows gives 256 blocks, fewer than two per SM).
int reduce_seg(int nx, int ny) {
  const int cols = (nx + RB - 1) / RB;
  for (int seg = 16; seg < 64; seg *= 2)
    if ((int64_t)cols * ((ny + seg - 1) / seg) <= kReduceMaxBlocks) return seg;
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

// Pass 1.  Block (RB threads) covers RB consecutive columns and seg rows;
// each thread walks its column down the segment (coalesced rows across the
// warp) and accumulates its nodes' terms (obs_node) as two-part FP32 sums,
// then the warp, then the warps' partials in FP64 (obs_block_store).  Rows
// go in groups of RU (4 in FP32, 2 in FP64, which holds twice the
// registers per value): all loads of a group are issued before any of its
// snapshot stores, so a thread keeps RU rows of loads in flight.
template <typename C>
__global__ void __launch_bounds__(RB) k_reduce_pass1(ReduceArgs a, int seg) {
  constexpr int RU = sizeof(C) == 4 ? 4 : 2;
  ObsAcc<C> acc;
  obs_zero(acc);
  const C* __restrict__ mac = static_cast<const C*>(a.mac);
  const C* __restrict__ phi_f = static_cast<const C*>(a.phi);
  C* __restrict__ prev = static_cast<C*>(a.prev);
  const int64_t pl = a.plane;
  const int x = blockIdx.x * RB + threadIdx.x;
  const int y0 = blockIdx.y * seg;
  const int y1 = min(y0 + seg, a.ny);
  const C phi_u = C(a.phi_u), sigma = C(a.sigma);
  if (x < a.nx) {
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
        const C wy = ((y == 0 && a.wall_lo) || (y == a.ny - 1 && a.wall_hi)) ? C(0.5) : C(1);
        obs_node<C>(acc, rho[r], ux[r], uy[r], Tf[r], Ts[r], phi[r], sigma, pux[r], puy[r],
                    pTf[r], pTs[r], wy, x, a.nx);
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
  obs_block_store<C>(acc, a.partials);
}

// Block b combines partial vectors [b * chunk, min((b + 1) * chunk, blocks))
// into out[b] (fixed order: thread strides, then the block tree).
__global__ void __launch_bounds__(RB) k_reduce_pass2(const double* __restrict__ partials,
                                                     int64_t blocks, int64_t chunk,
                                                     double* __restrict__ out) {
  __shared__ double sh[(RB / 32) * NACC];
  double acc[NACC];
#pragma unroll
  for (int k = 0; k < NACC; ++k) acc[k] = 0.0;
  const int64_t b0 = (int64_t)blockIdx.x * chunk;
  const int64_t b1 = b0 + chunk < blocks ? b0 + chunk : blocks;
  for (int64_t b = b0 + threadIdx.x; b < b1; b += RB)
#pragma unroll
    for (int k = 0; k < NACC; ++k)
      acc[k] = combine<double>(k, acc[k], partials[b * NACC + k]);
  block_reduce(acc, sh);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NACC; ++k) out[(int64_t)blockIdx.x * NACC + k] = acc[k];
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
  k_reduce_pass2<<<1, RB, 0, st>>>(a.partials, a.blocks, a.blocks, a.out);
  return cudaGetLastError();
}

}  // namespace ltne
