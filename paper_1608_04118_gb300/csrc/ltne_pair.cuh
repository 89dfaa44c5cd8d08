// ltne_pair.cuh -- the time step with two neighbouring nodes per thread in
// paired FP32 arithmetic.
//
// sm_100 and later execute add, mul and fma on a pair of FP32 values as one
// instruction (PTX add/mul/fma.rn.f32x2).  A thread that owns the nodes
// (x, y) and (x + 1, y), x even, runs the same per-node physics as the
// one-node kernel (macros, collide, nee of ltne_node.cuh, instantiated for
// the pair type F2) and so issues about half the floating-point
// instructions per node.  The pair also shares memory instructions: the
// populations that stream along y or rest (i = 0, 2, 4 of both lattices)
// arrive as one aligned pair, the stores of all 19 are one aligned pair
// each, and the 16-bit forms convert both values with one instruction.
//
// Every value is rounded as by the scalar operations (each paired operation
// is the IEEE round-to-nearest operation on each lane), so the pair path is
// the same arithmetic; products that the scalar build contracts into FMAs
// may be contracted differently.  Pairs that contain a left/right wall node
// (or, with odd nx, only one node) take the one-node path.
#pragma once

#include "ltne_step_impl.cuh"

namespace ltne {

LTNE_HD float2 add2_(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
  return __fadd2_rn(a, b);
#else
  return make_float2(a.x + b.x, a.y + b.y);
#endif
}
LTNE_HD float2 mul2_(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
  return __fmul2_rn(a, b);
#else
  return make_float2(a.x * b.x, a.y * b.y);
#endif
}
LTNE_HD float2 fma2_(float2 a, float2 b, float2 c) {
#ifdef __CUDA_ARCH__
  return __ffma2_rn(a, b, c);
#else
  return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
#endif
}
LTNE_HD float2 neg2_(float2 a) { return make_float2(-a.x, -a.y); }

// Two FP32 lanes (lane x: the even node, lane y: the odd node).
struct F2 {
  float2 v;
  F2() = default;
  LTNE_HD explicit F2(double s) : v(make_float2((float)s, (float)s)) {}
  LTNE_HD F2(float a, float b) : v(make_float2(a, b)) {}
  LTNE_HD explicit F2(float2 a) : v(a) {}
};

// A product not yet rounded: a following + or - turns it into one fma.
struct P2 {
  float2 a, b;
  LTNE_HD operator F2() const { return F2(mul2_(a, b)); }
};

LTNE_HD F2 operator+(F2 x, F2 y) { return F2(add2_(x.v, y.v)); }
LTNE_HD F2 operator-(F2 x, F2 y) { return F2(add2_(x.v, neg2_(y.v))); }
LTNE_HD F2 operator-(F2 x) { return F2(neg2_(x.v)); }
LTNE_HD P2 operator*(F2 x, F2 y) { return P2{x.v, y.v}; }

LTNE_HD F2 operator+(P2 p, F2 c) { return F2(fma2_(p.a, p.b, c.v)); }
LTNE_HD F2 operator+(F2 c, P2 p) { return F2(fma2_(p.a, p.b, c.v)); }
LTNE_HD F2 operator-(F2 c, P2 p) { return F2(fma2_(neg2_(p.a), p.b, c.v)); }
LTNE_HD F2 operator-(P2 p, F2 c) { return F2(fma2_(p.a, p.b, neg2_(c.v))); }
LTNE_HD F2 operator+(P2 p, P2 q) { return F2(fma2_(p.a, p.b, F2(q).v)); }
LTNE_HD F2 operator-(P2 p, P2 q) { return F2(fma2_(neg2_(q.a), q.b, F2(p).v)); }
LTNE_HD P2 operator-(P2 p) { return P2{neg2_(p.a), p.b}; }
LTNE_HD P2 operator*(P2 p, F2 y) { return P2{F2(p).v, y.v}; }
LTNE_HD P2 operator*(F2 x, P2 p) { return P2{x.v, F2(p).v}; }
LTNE_HD P2 operator*(P2 p, P2 q) { return P2{F2(p).v, F2(q).v}; }

LTNE_HD F2& operator+=(F2& x, F2 y) { return x = x + y; }
LTNE_HD F2& operator+=(F2& x, P2 p) { return x = x + p; }
LTNE_HD F2& operator-=(F2& x, F2 y) { return x = x - y; }
LTNE_HD F2& operator-=(F2& x, P2 p) { return x = x - p; }

template <> LTNE_HD F2 cfma_<F2>(F2 a, F2 b, F2 c) { return F2(fma2_(a.v, b.v, c.v)); }
template <> LTNE_HD F2 rcp_<F2>(F2 x) { return F2(rcp_<float>(x.v.x), rcp_<float>(x.v.y)); }
template <> LTNE_HD F2 sqrt_<F2>(F2 x) { return F2(sqrt_<float>(x.v.x), sqrt_<float>(x.v.y)); }
template <> LTNE_HD F2 csqrt_<F2>(F2 x) { return F2(csqrt_<float>(x.v.x), csqrt_<float>(x.v.y)); }

// Eq. 52 per lane.
template <> LTNE_HD F2 hv_local_at<F2>(const NodeParams<F2>& P, F2 um) {
  NodeParams<float> q;
  q.hv_c = P.hv_c.v.x;
  return F2(hv_local_at<float>(q, um.v.x), hv_local_at<float>(q, um.v.y));
}

// Loads and stores of node pairs.  `p` points at the even node of a pair
// (an even element offset: pitch and plane are even, so pairs are aligned).
template <typename S> struct PairIO;

template <> struct PairIO<float> {
  static __device__ __forceinline__ F2 ld2(const float* p, float) {
    return F2(*reinterpret_cast<const float2*>(p));
  }
  static __device__ __forceinline__ F2 ld11(const float* a, const float* b, float) {
    return F2(*a, *b);
  }
  static __device__ __forceinline__ void st2(float* p, F2 v, float, uint32_t) {
    *reinterpret_cast<float2*>(p) = v.v;
  }
};

template <> struct PairIO<__half> {
  static __device__ __forceinline__ F2 ld2(const __half* p, float inv_scale) {
    const float2 w = __half22float2(*reinterpret_cast<const __half2*>(p));
    return F2(mul2_(w, make_float2(inv_scale, inv_scale)));
  }
  static __device__ __forceinline__ F2 ld11(const __half* a, const __half* b, float inv_scale) {
    return F2(mul2_(make_float2(__half2float(*a), __half2float(*b)),
                    make_float2(inv_scale, inv_scale)));
  }
  // Both lanes in one paired conversion with random bits: the rounding of
  // Codec<__half, float>::enc2 with the even node in the low half.
  static __device__ __forceinline__ void st2(__half* p, F2 v, float scale, uint32_t r) {
    const float2 w = mul2_(v.v, make_float2(scale, scale));
    uint32_t h;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(h) : "f"(w.y), "f"(w.x), "r"(r));
    *reinterpret_cast<uint32_t*>(p) = h;
  }
};

template <> struct PairIO<__nv_bfloat16> {
  static __device__ __forceinline__ F2 ld2(const __nv_bfloat16* p, float) {
    const uint32_t u = *reinterpret_cast<const uint32_t*>(p);
    return F2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
  }
  static __device__ __forceinline__ F2 ld11(const __nv_bfloat16* a, const __nv_bfloat16* b,
                                            float) {
    return F2(__bfloat162float(*a), __bfloat162float(*b));
  }
  // Both lanes in one paired conversion with random bits: the rounding of
  // Codec<__nv_bfloat16, float>::enc2 with the even node in the low half.
  static __device__ __forceinline__ void st2(__nv_bfloat16* p, F2 v, float, uint32_t r) {
    uint32_t h;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(h) : "f"(v.v.y), "f"(v.v.x), "r"(r));
    *reinterpret_cast<uint32_t*>(p) = h;
  }
};

template <typename S>
struct PairPops {
  // The 19 values streaming into the pair (x0, y), (x0 + 1, y): value i of a
  // node comes from x - e_i.  xm is the column left of x0 and xp the column
  // right of x0 + 1 (after wrapping); ym/yp the rows below/above y.
  static __device__ __forceinline__ void pull(const S* __restrict__ src, uint32_t pl, uint32_t pi,
                                              int x0, int xm, int xp, int y, int ym, int yp,
                                              float inv_scale, F2 (&f)[9], F2 (&gf)[5],
                                              F2 (&gs)[5]) {
    const uint32_t r0 = (uint32_t)y * pi, rm = (uint32_t)ym * pi, rp = (uint32_t)yp * pi;
    const uint32_t a = (uint32_t)x0, am = (uint32_t)xm, b = a + 1u, bp = (uint32_t)xp;
    // i = 0, 2, 4: aligned pairs at rows y, y - 1, y + 1
    // i = 1, 5, 8 (e_x = +1): lanes from columns xm and x0
    // i = 3, 6, 7 (e_x = -1): lanes from columns x0 + 1 and xp
    auto pair = [&](uint32_t k, uint32_t row) {
      return PairIO<S>::ld2(src + (k * pl + row + a), inv_scale);
    };
    auto left = [&](uint32_t k, uint32_t row) {
      const uint32_t q = k * pl + row;
      return PairIO<S>::ld11(src + (q + am), src + (q + a), inv_scale);
    };
    auto right = [&](uint32_t k, uint32_t row) {
      const uint32_t q = k * pl + row;
      return PairIO<S>::ld11(src + (q + b), src + (q + bp), inv_scale);
    };
    f[0] = pair(0, r0);
    f[1] = left(1, r0);
    f[2] = pair(2, rm);
    f[3] = right(3, r0);
    f[4] = pair(4, rp);
    f[5] = left(5, rm);
    f[6] = right(6, rm);
    f[7] = right(7, rp);
    f[8] = left(8, rp);
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      F2(&g)[5] = t == 0 ? gf : gs;
      const uint32_t k0 = t == 0 ? 9u : 14u;
      g[0] = pair(k0, r0);
      g[1] = left(k0 + 1, r0);
      g[2] = pair(k0 + 2, rm);
      g[3] = right(k0 + 3, r0);
      g[4] = pair(k0 + 4, rp);
    }
  }

  static __device__ __forceinline__ void store(S* __restrict__ dst, uint32_t pl, uint32_t off,
                                               float scale, const F2 (&f)[9], const F2 (&gf)[5],
                                               const F2 (&gs)[5], uint32_t seed_pair,
                                               uint32_t seed_step) {
    if constexpr (Codec<S, float>::kStochastic) {
      RandomBits rb(seed_pair, seed_step);
#pragma unroll
      for (int i = 0; i < 19; ++i) {
        const F2 v = i < 9 ? f[i] : (i < 14 ? gf[i - 9] : gs[i - 14]);
        PairIO<S>::st2(dst + ((uint32_t)i * pl + off), v, scale, rb.next());
      }
    } else {
#pragma unroll
      for (int i = 0; i < 19; ++i) {
        const F2 v = i < 9 ? f[i] : (i < 14 ? gf[i - 9] : gs[i - 14]);
        PairIO<S>::st2(dst + ((uint32_t)i * pl + off), v, scale, 0u);
      }
    }
  }
};

__device__ __forceinline__ F2 ld_f2(const float* __restrict__ p) {
  return F2(*reinterpret_cast<const float2*>(p));
}
__device__ __forceinline__ void st_f2(float* __restrict__ p, F2 v) {
  *reinterpret_cast<float2*>(p) = v.v;
}

// Everything after the pull for a pair at element offset off whose
// pre-collision values are in f, gf, gs: macroscopic values, collision,
// stores.  Shared by the pull from HBM and the pull from a staged tile.
template <typename S>
__device__ __forceinline__ void finish_pair(S* __restrict__ dst,
                                            const float* __restrict__ phi_field,
                                            float* __restrict__ mac, const NodeParams<F2>& P,
                                            const uint32_t off, const uint32_t pl,
                                            const float scale, const int write_macros,
                                            const uint32_t tick, const float* __restrict__ um_in,
                                            float* __restrict__ um_out, F2 (&f)[9], F2 (&gf)[5],
                                            F2 (&gs)[5]) {
  Medium<F2> md = phi_field ? medium_at<F2>(P, ld_f2(phi_field + off)) : P.um;
  if (P.hv_local) set_exchange<F2>(md, hv_local_at<F2>(P, ld_f2(um_in + off)));
  Macro<F2> m;
  macros<F2>(P, md, f, gf, gs, m);
  if (P.hv_local) st_f2(um_out + off, m.umag);
  if (write_macros) {
    st_f2(mac + off, m.drho);
    st_f2(mac + pl + off, m.ux);
    st_f2(mac + 2u * pl + off, m.uy);
    st_f2(mac + 3u * pl + off, m.dTf);
    st_f2(mac + 4u * pl + off, m.dTs);
  }
  collide<F2>(P, m, f, gf, gs);
  PairPops<S>::store(dst, pl, off, scale, f, gf, gs, off, tick);
}

// The pair (x0, y), (x0 + 1, y) when both nodes exist and neither is a
// left/right wall node: interior nodes, or both on a no-slip adiabatic row
// (same rebuild, from the row above or below).
template <typename S, int BC>
__device__ __forceinline__ void step_pair(const S* __restrict__ src, S* __restrict__ dst,
                                          const float* __restrict__ phi_field,
                                          float* __restrict__ mac, const NodeParams<F2>& P,
                                          const int x0, const int y, const int nx, const int ny,
                                          const uint32_t pi, const uint32_t pl, const float scale,
                                          const float inv_scale, const int write_macros,
                                          const uint32_t tick, const float* __restrict__ um_in,
                                          float* __restrict__ um_out) {
  int cy = y;
  bool wall_row = false;
  if (BC == BC_CAVITY || BC == BC_CHANNEL) {
    if (y == 0 || y == ny - 1) {
      wall_row = true;
      cy = (y == 0) ? 1 : ny - 2;
    }
  }
  int xm = x0 - 1, xp = x0 + 2, ym = cy - 1, yp = cy + 1;
  if (BC == BC_PERIODIC || BC == BC_CHANNEL) {
    xm = (x0 == 0) ? nx - 1 : xm;
    xp = (xp == nx) ? 0 : xp;
  }
  if (BC == BC_PERIODIC) {
    ym = (cy == 0) ? ny - 1 : ym;
    yp = (cy == ny - 1) ? 0 : yp;
  }
  F2 f[9], gf[5], gs[5];
  PairPops<S>::pull(src, pl, pi, x0, xm, xp, cy, ym, yp, inv_scale, f, gf, gs);

  const uint32_t off = (uint32_t)y * pi + (uint32_t)x0;
  if (BC != BC_PERIODIC && wall_row) {
    const uint32_t noff = (uint32_t)cy * pi + (uint32_t)x0;
    Medium<F2> mdn = phi_field ? medium_at<F2>(P, ld_f2(phi_field + noff)) : P.um;
    if (P.hv_local) set_exchange<F2>(mdn, hv_local_at<F2>(P, ld_f2(um_in + noff)));
    Macro<F2> mn;
    macros<F2>(P, mdn, f, gf, gs, mn);
    nee<F2>(P, mn, mn.dTf, mn.dTs, f, gf, gs);  // adiabatic: the neighbour's temperatures
  }
  finish_pair<S>(dst, phi_field, mac, P, off, pl, scale, write_macros, tick, um_in, um_out, f, gf,
                 gs);
}

// A cavity pair holding a left or right wall node (x0 = 0, or x0 + 1 =
// nx - 1).  The wall node is rebuilt from the interior node next to it,
// which is the pair's other node: both lanes pull around that node (one
// scalar pull, broadcast), its macroscopic values give the non-equilibrium
// extrapolation, and the lanes that are wall nodes take the rebuild -- the
// side wall node at its wall temperature, the other lane too on a
// bottom/top row (adiabatic: the neighbour's temperatures).  Then both
// lanes continue as any pair.  The same rebuild as the one-node step, in
// paired arithmetic, without the warp divergence of two one-node steps
// beside the pairs of the rest of the row.
template <typename S>
__device__ __forceinline__ void step_pair_side(const S* __restrict__ src, S* __restrict__ dst,
                                               const float* __restrict__ phi_field,
                                               float* __restrict__ mac, const NodeParams<F2>& P,
                                               const int x0, const int y, const int nx,
                                               const int ny, const uint32_t pi, const uint32_t pl,
                                               const float scale, const float inv_scale,
                                               const int write_macros, const uint32_t tick,
                                               const float* __restrict__ um_in,
                                               float* __restrict__ um_out) {
  const bool left = x0 == 0;
  const bool wall_row = y == 0 || y == ny - 1;
  const int cx = left ? 1 : nx - 2;
  const int cy = y == 0 ? 1 : (y == ny - 1 ? ny - 2 : y);
  float fs[9], gfs[5], gss[5];
  Pops<S, float>::pull(src, (int64_t)pi, (int64_t)pl, cx, cx - 1, cx + 1, cy, cy - 1, cy + 1,
                       inv_scale, fs, gfs, gss);
  F2 f[9], gf[5], gs[5];
#pragma unroll
  for (int i = 0; i < 9; ++i) f[i] = F2(fs[i], fs[i]);
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    gf[i] = F2(gfs[i], gfs[i]);
    gs[i] = F2(gss[i], gss[i]);
  }
  const uint32_t noff = (uint32_t)cy * pi + (uint32_t)cx;
  Medium<F2> mdn = P.um;
  if (phi_field) {
    const float pn = phi_field[noff];
    mdn = medium_at<F2>(P, F2(pn, pn));
  }
  if (P.hv_local) {
    const float un = um_in[noff];
    set_exchange<F2>(mdn, hv_local_at<F2>(P, F2(un, un)));
  }
  Macro<F2> mn;
  macros<F2>(P, mdn, f, gf, gs, mn);
  // wall temperatures: the side wall's in the wall lane, the neighbour's
  // (adiabatic rows) in the other
  const float side = left ? P.dT_hot.v.x : P.dT_cold.v.x;
  F2 twf = mn.dTf, tws = mn.dTs;
  if (left) {
    twf.v.x = side;
    tws.v.x = side;
  } else {
    twf.v.y = side;
    tws.v.y = side;
  }
  F2 rf[9], rgf[5], rgs[5];
#pragma unroll
  for (int i = 0; i < 9; ++i) rf[i] = f[i];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    rgf[i] = gf[i];
    rgs[i] = gs[i];
  }
  nee<F2>(P, mn, twf, tws, rf, rgf, rgs);
  const bool wx = left || wall_row, wy = !left || wall_row;
  auto pick = [&](F2 r, F2 v) { return F2(wx ? r.v.x : v.v.x, wy ? r.v.y : v.v.y); };
#pragma unroll
  for (int i = 0; i < 9; ++i) f[i] = pick(rf[i], f[i]);
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    gf[i] = pick(rgf[i], gf[i]);
    gs[i] = pick(rgs[i], gs[i]);
  }
  const uint32_t off = (uint32_t)y * pi + (uint32_t)x0;
  finish_pair<S>(dst, phi_field, mac, P, off, pl, scale, write_macros, tick, um_in, um_out, f, gf,
                 gs);
}

// Register budget of the pair kernel: blocks of at most 128 threads and at
// least 5 resident per SM, i.e. at most 102 registers (it compiles to 96
// without spilling) and 20 warps per SM.  Uncapped it takes about 110, and
// 256-thread blocks hold a finished warp's registers until the whole block
// is done; measured at 8192^2 FP16: 60.3 GLUPS with 32 x 4 blocks against
// 46.7 with 128 x 2 blocks uncapped.
constexpr int kPairMaxThreads = kPairBlockThreads;
constexpr int kPairMinBlocks = 5;

template <typename S, int BC>
__global__ void __launch_bounds__(kPairMaxThreads, kPairMinBlocks) k_step_pair(
    const S* __restrict__ src, S* __restrict__ dst, const float* __restrict__ phi_field,
    float* __restrict__ mac, const NodeParams<F2> P, const NodeParams<float> P1, const int nx,
    const int ny, const int64_t pitch, const int64_t plane, const float scale,
    const float inv_scale, const int write_macros, const uint32_t* __restrict__ tick_in,
    uint32_t* __restrict__ tick_out, const float* __restrict__ um_in, float* __restrict__ um_out) {
  grid_dep_wait();
  const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const uint32_t tick = read_tick<S, float>(tick_in, tick_out);
  if (x0 >= nx || y >= ny) return;
  const bool full = x0 + 1 < nx;
  const bool uniform = BC == BC_CAVITY ? (x0 > 0 && x0 + 2 < nx) : full;
  if (uniform) {
    step_pair<S, BC>(src, dst, phi_field, mac, P, x0, y, nx, ny, (uint32_t)pitch,
                     (uint32_t)plane, scale, inv_scale, write_macros, tick, um_in, um_out);
  } else if (BC == BC_CAVITY && full) {
    step_pair_side<S>(src, dst, phi_field, mac, P, x0, y, nx, ny, (uint32_t)pitch,
                      (uint32_t)plane, scale, inv_scale, write_macros, tick, um_in, um_out);
  } else {
    step_node<S, float, BC>(src, dst, phi_field, mac, P1, x0, y, nx, ny, pitch, plane, scale,
                            inv_scale, write_macros, tick, nullptr, um_in, um_out);
    if (full)
      step_node<S, float, BC>(src, dst, phi_field, mac, P1, x0 + 1, y, nx, ny, pitch, plane,
                              scale, inv_scale, write_macros, tick, nullptr, um_in, um_out);
  }
}

template <typename S>
cudaError_t launch_step_pair_t(const LatticeArgs& a, const NodeParams<double>& Pd, StepShape s,
                               cudaStream_t st) {
  if (s.bx * s.by > kPairMaxThreads) return cudaErrorInvalidValue;
  const NodeParams<F2> P = cast_params<F2>(Pd);
  const NodeParams<float> P1 = cast_params<float>(Pd);
  dim3 block(s.bx, s.by);
  const int pairs = (a.nx + 1) / 2;
  dim3 grid((pairs + s.bx - 1) / s.bx, (a.ny + s.by - 1) / s.by);
  const float scale = a.enc_scale, inv_scale = 1.0f / a.enc_scale;
  const S* src = static_cast<const S*>(a.src);
  S* dst = static_cast<S*>(a.dst);
  const float* phi = static_cast<const float*>(a.phi);
  float* mac = static_cast<float*>(a.mac);
  const float* um_in = static_cast<const float*>(a.um_in);
  float* um_out = static_cast<float*>(a.um_out);
  cudaError_t e;
#define LTNE_PAIR_LAUNCH(bc)                                                                   \
  e = launch_kernel(a.chained != 0, k_step_pair<S, bc>, grid, block, 0, st, src, dst, phi,     \
                    mac, P, P1, a.nx, a.ny, a.pitch, a.plane, scale, inv_scale,                \
                    a.write_macros, a.tick_in, a.tick_out, um_in, um_out)
  switch (a.bc) {
    case BC_CAVITY: LTNE_PAIR_LAUNCH(BC_CAVITY); break;
    case BC_PERIODIC: LTNE_PAIR_LAUNCH(BC_PERIODIC); break;
    case BC_CHANNEL: LTNE_PAIR_LAUNCH(BC_CHANNEL); break;
    default: return cudaErrorInvalidValue;
  }
#undef LTNE_PAIR_LAUNCH
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace ltne
