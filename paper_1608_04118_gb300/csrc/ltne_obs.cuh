// ltne_obs.cuh -- per-node terms of the observables and their per-block
// combination, for the reduction pass of ltne_reduce.cu.
//
// Per node: the wall-flux stencils of Nu (second-order one-sided difference,
// trapezoid rule in y), mass, energy, the sums and squares of the residual,
// the maxima of |u|^2 and |T_f - T_s|, a non-finite count.  For FP32 fields
// a thread's terms and the 32 lanes of a warp are combined as unevaluated
// sums of two FP32 values (hi + lo, each addition and its renormalisation
// error-free by Knuth's TwoSum), so the warp sums carry about 48
// significant bits; from the warp partials upward every sum is FP64, in a
// fixed order (warps of a block, then blocks: bitwise reproducible for a
// given lattice).  FP64 fields accumulate in FP64 throughout.
#pragma once

#include "ltne_internal.h"

namespace ltne {

// Sum slots in accumulator order (the maxima A_MAXU, A_MAXDT are separate).
constexpr int kObsSums = NACC - 2;
__host__ __device__ constexpr int obs_slot(int j) { return j < A_MAXU ? j : j + 2; }

template <typename C>
struct ObsAcc {
  C s[kObsSums];  // sums, in the order of obs_slot()
  C lo[kObsSums]; // their low parts (FP32 compute only)
  C mu2, mdt;     // max |u|^2, max |T_f - T_s|
};

template <typename C>
__device__ __forceinline__ void obs_zero(ObsAcc<C>& a) {
#pragma unroll
  for (int j = 0; j < kObsSums; ++j) a.s[j] = a.lo[j] = C(0);
  a.mu2 = a.mdt = C(0);
}

// Error-free sum s + e = a + b (Knuth's TwoSum, six rounded operations,
// never contracted).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float ap = __fsub_rn(s, bp);
  e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

// (hi, lo) += x for an FP32 value x.  The renormalisation is a TwoSum too:
// sums that cancel (mass deviations, the wall fluxes) can leave |lo| above
// |s|, where the cheaper Fast2Sum would not be exact.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float x) {
  float s, e;
  two_sum(hi, x, s, e);
  two_sum(s, __fadd_rn(e, lo), hi, lo);
}
__device__ __forceinline__ void ff_add(double& hi, double&, double x) { hi += x; }

// (hi, lo) += (hi2, lo2).
__device__ __forceinline__ void ff_add2(float& hi, float& lo, float hi2, float lo2) {
  float s, e;
  two_sum(hi, hi2, s, e);
  two_sum(s, __fadd_rn(e, __fadd_rn(lo, lo2)), hi, lo);
}
__device__ __forceinline__ void ff_add2(double& hi, double&, double hi2, double) { hi += hi2; }

// One node's terms.  drho .. dTs are the deviations the macro planes hold;
// p* the previous snapshot's u_x, u_y, T_f - T0, T_s - T0; wy the node's
// trapezoid weight in y (1/2 on the cavity's bottom and top rows).
template <typename C>
__device__ __forceinline__ void obs_node(ObsAcc<C>& a, C drho, C ux, C uy, C dTf, C dTs, C phi,
                                         C sigma, C pux, C puy, C pTf, C pTs, C wy, int x,
                                         int nx) {
  const C whot = (x == 1) ? C(-2) : (x == 2) ? C(0.5) : C(0);
  const C wcold = (x == nx - 2) ? C(2) : (x == nx - 3) ? C(-0.5) : C(0);
  const C u2 = ux * ux + uy * uy;
  const C dux = ux - pux, duy = uy - puy, dtf = dTf - pTf, dts = dTs - pTs;
  C t[kObsSums];
  t[A_NUF_H] = whot * wy * dTf;
  t[A_NUS_H] = whot * wy * dTs;
  t[A_NUF_C] = wcold * wy * dTf;
  t[A_NUS_C] = wcold * wy * dTs;
  t[A_MASS] = drho;
  t[A_ENERGY] = phi * dTf + (C(1) - phi) * sigma * dTs;
  t[A_SUMTF - 2] = dTf;
  t[A_SUMTS - 2] = dTs;
  t[A_DU2 - 2] = dux * dux + duy * duy;
  t[A_U2 - 2] = u2;
  t[A_DTF2 - 2] = dtf * dtf;
  t[A_TF2 - 2] = dTf * dTf;
  t[A_DTS2 - 2] = dts * dts;
  t[A_TS2 - 2] = dTs * dTs;
  t[A_BAD - 2] = (isfinite(drho) && isfinite(ux) && isfinite(uy) && isfinite(dTf) &&
                  isfinite(dTs)) ? C(0) : C(1);
  t[A_SUMPHI - 2] = phi;
#pragma unroll
  for (int j = 0; j < kObsSums; ++j) ff_add(a.s[j], a.lo[j], t[j]);
  a.mu2 = u2 > a.mu2 ? u2 : a.mu2;
  const C dT = dTf > dTs ? dTf - dTs : dTs - dTf;
  a.mdt = dT > a.mdt ? dT : a.mdt;
}

// Reduce the block's accumulators and write its FP64 partial vector to
// partials[block].  Every thread of the block calls it.
template <typename C>
__device__ __forceinline__ void obs_block_store(ObsAcc<C>& a, double* __restrict__ partials) {
  __shared__ double sh[32][NACC];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int lane = tid & 31, warp = tid >> 5;
  const int nwarps = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
  for (int j = 0; j < kObsSums; ++j) {
    C hi = a.s[j], lo = a.lo[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const C h2 = __shfl_down_sync(0xffffffffu, hi, o);
      const C l2 = __shfl_down_sync(0xffffffffu, lo, o);
      ff_add2(hi, lo, h2, l2);
    }
    if (lane == 0) sh[warp][obs_slot(j)] = (double)hi + (double)lo;
  }
  C mu2 = a.mu2, mdt = a.mdt;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const C m1 = __shfl_down_sync(0xffffffffu, mu2, o);
    const C m2 = __shfl_down_sync(0xffffffffu, mdt, o);
    mu2 = m1 > mu2 ? m1 : mu2;
    mdt = m2 > mdt ? m2 : mdt;
  }
  if (lane == 0) {
    sh[warp][A_MAXU] = (double)mu2;
    sh[warp][A_MAXDT] = (double)mdt;
  }
  __syncthreads();
  if (tid < NACC) {
    const int k = tid;
    double v = sh[0][k];
    for (int w = 1; w < nwarps; ++w)
      v = (k == A_MAXU || k == A_MAXDT) ? fmax(v, sh[w][k]) : v + sh[w][k];
    const int64_t b = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    partials[b * NACC + k] = v;
  }
}

}  // namespace ltne
