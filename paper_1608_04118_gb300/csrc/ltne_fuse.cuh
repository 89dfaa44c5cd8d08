// ltne_fuse.cuh -- the observables' terms accumulated by the last time step
// of an ltne_step() call, which holds every node's macroscopic values in
// registers while it writes them to the field planes: ltne_observables()
// then only combines the per-block partials (and forms the Nu integrals from
// the four columns next to the walls), instead of reading the fields back.
//
// Per node: the same terms as the reduction pass of ltne_reduce.cu for the
// slots from A_MASS on (mass, energy, the maxima of |u|^2 and |T_f - T_s|,
// the sums and squares of the residual, a non-finite count, the porosity
// sum).  A thread sums its one or two nodes in the compute type; the block's
// threads are combined through shared memory, in chunks of 16 threads in the
// compute type (at most 32 nodes per FP32 sum) and the chunks in FP64, in a
// fixed order (bitwise reproducible for a given launch shape).
#pragma once

#include "ltne_internal.h"

namespace ltne {

constexpr int kFuseSlots = NACC - A_MASS;  // slots A_MASS .. NACC-1
constexpr int kFuseChunk = 16;             // threads summed in the compute type

template <typename C>
struct FuseAcc {
  C v[kFuseSlots];
};

template <typename C>
__device__ __forceinline__ void fuse_zero(FuseAcc<C>& a) {
#pragma unroll
  for (int j = 0; j < kFuseSlots; ++j) a.v[j] = C(0);
}

__host__ __device__ constexpr bool fuse_is_max(int j) {
  return j + A_MASS == A_MAXU || j + A_MASS == A_MAXDT;
}

// One node's terms: the deviations the field planes hold (drho .. dTs), the
// porosity, and the residual reference's u_x, u_y, T_f - T0, T_s - T0.
template <typename C>
__device__ __forceinline__ void fuse_node(FuseAcc<C>& a, C drho, C ux, C uy, C dTf, C dTs,
                                          C phi, C sigma, C pux, C puy, C pTf, C pTs) {
  const C u2 = ux * ux + uy * uy;
  const C dux = ux - pux, duy = uy - puy, dtf = dTf - pTf, dts = dTs - pTs;
  a.v[A_MASS - A_MASS] += drho;
  a.v[A_ENERGY - A_MASS] += phi * dTf + (C(1) - phi) * sigma * dTs;
  a.v[A_MAXU - A_MASS] = u2 > a.v[A_MAXU - A_MASS] ? u2 : a.v[A_MAXU - A_MASS];
  const C dT = dTf > dTs ? dTf - dTs : dTs - dTf;
  a.v[A_MAXDT - A_MASS] = dT > a.v[A_MAXDT - A_MASS] ? dT : a.v[A_MAXDT - A_MASS];
  a.v[A_SUMTF - A_MASS] += dTf;
  a.v[A_SUMTS - A_MASS] += dTs;
  a.v[A_DU2 - A_MASS] += dux * dux + duy * duy;
  a.v[A_U2 - A_MASS] += u2;
  a.v[A_DTF2 - A_MASS] += dtf * dtf;
  a.v[A_TF2 - A_MASS] += dTf * dTf;
  a.v[A_DTS2 - A_MASS] += dts * dts;
  a.v[A_TS2 - A_MASS] += dTs * dTs;
  if (!(isfinite(drho) && isfinite(ux) && isfinite(uy) && isfinite(dTf) && isfinite(dTs)))
    a.v[A_BAD - A_MASS] += C(1);
  a.v[A_SUMPHI - A_MASS] += phi;
}

// The block's partial vector into part (slot A_MASS + j of block b at
// (A_MASS + j) * blocks + b).  Every thread of the block calls it; at most
// 256 threads per block, a multiple of kFuseChunk.
template <typename C>
__device__ __forceinline__ void fuse_block_store(const FuseAcc<C>& a, double* __restrict__ part) {
  __shared__ C sh[kFuseSlots][256];
  __shared__ double sh2[kFuseSlots][256 / kFuseChunk];
  const int nt = blockDim.x * blockDim.y;
  const int t = threadIdx.x + blockDim.x * threadIdx.y;
  const int nchunks = nt / kFuseChunk;
#pragma unroll
  for (int j = 0; j < kFuseSlots; ++j) sh[j][t] = a.v[j];
  __syncthreads();
  if (t < kFuseSlots * nchunks) {
    const int j = t / nchunks, c = t % nchunks;
    const C* row = &sh[j][c * kFuseChunk];
    C v = row[0];
    if (fuse_is_max(j)) {
#pragma unroll
      for (int i = 1; i < kFuseChunk; ++i) v = row[i] > v ? row[i] : v;
    } else {
#pragma unroll
      for (int i = 1; i < kFuseChunk; ++i) v += row[i];
    }
    sh2[j][c] = (double)v;
  }
  __syncthreads();
  if (t < kFuseSlots) {
    double v = sh2[t][0];
    for (int c = 1; c < nchunks; ++c) v = fuse_is_max(t) ? fmax(v, sh2[t][c]) : v + sh2[t][c];
    const int64_t blocks = (int64_t)gridDim.x * gridDim.y;
    const int64_t b = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    part[(int64_t)(A_MASS + t) * blocks + b] = v;
  }
}

}  // namespace ltne
