// ltne_step_impl.cuh -- fused collide-and-stream kernel of the
// three-distribution MRT-LB method (Liu & He, arXiv:1608.04118), templated
// on the population storage type S, the compute type C and the boundary
// mode.  Included once per storage type by step_<tag>.cu.
//
// Memory scheme: two population buffers (A-B) hold post-collision values.
// One thread owns one node and, in a single pass,
//   1. pulls the post-collision values of the previous step from x - e_i
//      (streaming, Eqs. 11, 34, 35), giving the pre-collision state S_n;
//      a wall node instead pulls around its interior neighbour and rebuilds
//      its populations by non-equilibrium extrapolation;
//   2. computes the macroscopic values (Eqs. 6, 18, 20-22, 43-46) and the
//      force (Eq. 5);
//   3. collides (Eqs. 10, 32, 33) and writes its 19 post-collision values.
// Per node and step this moves 19 reads + 19 writes of the storage type
// (+ one porosity read when the porosity varies per node); the macroscopic
// fields are written only on the last step of an ltne_step() call.
#pragma once

#include "ltne_internal.h"

namespace ltne {

template <typename C>
__host__ NodeParams<C> cast_params(const NodeParams<double>& d) {
  NodeParams<C> p;
  p.rho0 = C(d.rho0); p.T0 = C(d.T0);
  p.s_e = C(d.s_e); p.s_eps = C(d.s_eps); p.s_q = C(d.s_q); p.s_nu = C(d.s_nu);
  p.zeta_a = C(d.zeta_a); p.zeta_e = C(d.zeta_e); p.zeta_nu = C(d.zeta_nu);
  p.eta_a = C(d.eta_a); p.eta_e = C(d.eta_e); p.eta_nu = C(d.eta_nu);
  p.c3 = C(d.c3); p.wt0 = C(d.wt0); p.wt1 = C(d.wt1);
  p.gbeta = C(d.gbeta); p.ext_ax = C(d.ext_ax); p.ext_ay = C(d.ext_ay);
  p.phi_u = C(d.phi_u); p.hcoef = C(d.hcoef); p.sigma = C(d.sigma);
  p.qf = C(d.qf); p.qs = C(d.qs); p.dT_hot = C(d.dT_hot); p.dT_cold = C(d.dT_cold);
  p.nu_over_K = C(d.nu_over_K); p.inv_sqrtK = C(d.inv_sqrtK); p.Fconst = C(d.Fconst);
  p.erg_a = C(d.erg_a); p.erg_b = C(d.erg_b); p.erg_c = C(d.erg_c);
  p.kmode = d.kmode; p.fmode = d.fmode;
  p.um.phi = C(d.um.phi); p.um.inv_phi = C(d.um.inv_phi); p.um.a = C(d.um.a);
  p.um.b = C(d.um.b); p.um.inv_1d = C(d.um.inv_1d); p.um.c0 = C(d.um.c0);
  p.um.c1 = C(d.um.c1); p.um.l0 = C(d.um.l0); p.um.l1 = C(d.um.l1);
  p.um.inv_oms = C(d.um.inv_oms);
  p.hv_local = d.hv_local; p.hv_c = C(d.hv_c); p.tcorr = d.tcorr;
  return p;
}


template <typename S> __device__ __forceinline__ S bits_to(unsigned short b);
template <> __device__ __forceinline__ __half bits_to<__half>(unsigned short b) {
  return __ushort_as_half(b);
}
template <> __device__ __forceinline__ __nv_bfloat16 bits_to<__nv_bfloat16>(unsigned short b) {
  return __ushort_as_bfloat16(b);
}
template <> __device__ __forceinline__ float bits_to<float>(unsigned short) { return 0.0f; }
template <> __device__ __forceinline__ double bits_to<double>(unsigned short) { return 0.0; }

template <typename S, typename C>
struct Pops {
  // Loads the 19 post-collision values streaming into node (x, y):
  // value i of node (x, y) at the new step is value i of (x - ex_i, y - ey_i).
  // xm/xp and ym/yp are the columns/rows x-1, x+1, y-1, y+1 after wrapping.
  static __device__ __forceinline__ void pull(const S* __restrict__ src, int64_t pitch,
                                              int64_t plane, int x, int xm, int xp, int y,
                                              int ym, int yp, C inv_scale, C (&f)[9],
                                              C (&gf)[5], C (&gs)[5]) {
    // Element indices are 32-bit: 19 planes of a lattice stay below 2^32
    // elements (checked at create), so each access is one 32-bit add and one
    // wide multiply-add into the address.
    const uint32_t pl = (uint32_t)plane, pi = (uint32_t)pitch;
    const uint32_t r0 = (uint32_t)y * pi, rm = (uint32_t)ym * pi, rp = (uint32_t)yp * pi;
    const uint32_t ux = (uint32_t)x, uxm = (uint32_t)xm, uxp = (uint32_t)xp;
    // D2Q9 e_i (Eq. 8): 0 (0,0) 1 (1,0) 2 (0,1) 3 (-1,0) 4 (0,-1)
    //                   5 (1,1) 6 (-1,1) 7 (-1,-1) 8 (1,-1)
    const uint32_t so[9] = {r0 + ux, r0 + uxm, rm + ux, r0 + uxp, rp + ux,
                            rm + uxm, rm + uxp, rp + uxp, rp + uxm};
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = Codec<S, C>::dec(src[(uint32_t)i * pl + so[i]], inv_scale);
#pragma unroll
    for (int i = 0; i < 5; ++i)
      gf[i] = Codec<S, C>::dec(src[(uint32_t)(9 + i) * pl + so[i]], inv_scale);
#pragma unroll
    for (int i = 0; i < 5; ++i)
      gs[i] = Codec<S, C>::dec(src[(uint32_t)(14 + i) * pl + so[i]], inv_scale);
  }

  // Writes the 19 post-collision deviations of the node at offset off.
  // seed_node / seed_step key the stochastic rounding of the 16-bit forms.
  static __device__ __forceinline__ void store(S* __restrict__ dst, int64_t plane, uint32_t off,
                                               C scale, const C (&f)[9], const C (&gf)[5],
                                               const C (&gs)[5], uint32_t seed_node,
                                               uint32_t seed_step) {
    const uint32_t pl = (uint32_t)plane;
    if constexpr (Codec<S, C>::kStochastic) {
      // values 2k and 2k + 1 share one random word (low and high half) and
      // one paired conversion; value 18 takes the low half of the last word
      RandomBits rb(seed_node, seed_step);
      auto val = [&](int i) -> C { return i < 9 ? f[i] : (i < 14 ? gf[i - 9] : gs[i - 14]); };
#pragma unroll
      for (int i = 0; i < 19; i += 2) {
        const uint32_t d = Codec<S, C>::enc2(val(i), i + 1 < 19 ? val(i + 1) : C(0), scale,
                                             rb.next());
        dst[(uint32_t)i * pl + off] = bits_to<S>((unsigned short)(d & 0xffffu));
        if (i + 1 < 19) dst[(uint32_t)(i + 1) * pl + off] = bits_to<S>((unsigned short)(d >> 16));
      }
    } else {
#pragma unroll
      for (int i = 0; i < 9; ++i) dst[(uint32_t)i * pl + off] = Codec<S, C>::enc(f[i], scale, 0);
#pragma unroll
      for (int i = 0; i < 5; ++i)
        dst[(uint32_t)(9 + i) * pl + off] = Codec<S, C>::enc(gf[i], scale, 0);
#pragma unroll
      for (int i = 0; i < 5; ++i)
        dst[(uint32_t)(14 + i) * pl + off] = Codec<S, C>::enc(gs[i], scale, 0);
    }
  }
};

template <typename C>
__device__ __forceinline__ void store_macros(C* __restrict__ mac, int64_t plane, uint32_t off,
                                             const Macro<C>& m) {
  const uint32_t pl = (uint32_t)plane;
  mac[off] = m.drho;
  mac[pl + off] = m.ux;
  mac[2 * pl + off] = m.uy;
  mac[3 * pl + off] = m.dTf;
  mac[4 * pl + off] = m.dTs;
}

// One node (x, y) of one time step: pull, wall rebuild, macroscopic values,
// collision, store.  Shared by the single-lattice and the batched kernels.
template <typename S, typename C, int BC>
__device__ __forceinline__ void step_node(const S* __restrict__ src, S* __restrict__ dst,
                                          const C* __restrict__ phi_field, C* __restrict__ mac,
                                          const NodeParams<C>& P, const int x, const int y,
                                          const int nx, const int ny, const int64_t pitch,
                                          const int64_t plane, const C scale, const C inv_scale,
                                          const int write_macros, const uint32_t tick,
                                          C* __restrict__ pre_out = nullptr,
                                          const C* __restrict__ um_in = nullptr,
                                          C* __restrict__ um_out = nullptr,
                                          const int slab_walls = 0) {
  // Wall classification and the node whose neighbourhood is pulled.
  int cx = x, cy = y;
  int kind = -1;  // -1 interior, 0 hot wall, 1 cold wall, 2 adiabatic / no-slip row
  if (BC == BC_CAVITY || BC == BC_SLAB) {
    const bool ylo = (BC == BC_CAVITY || (slab_walls & SLAB_LO_WALL)) && y == 0;
    const bool yhi = (BC == BC_CAVITY || (slab_walls & SLAB_HI_WALL)) && y == ny - 1;
    if (x == 0 || x == nx - 1) {
      kind = (x == 0) ? 0 : 1;
      cx = (x == 0) ? 1 : nx - 2;
      if (ylo) cy = 1;
      else if (yhi) cy = ny - 2;
    } else if (ylo || yhi) {
      kind = 2;
      cy = ylo ? 1 : ny - 2;
    }
  } else if (BC == BC_CHANNEL) {
    if (y == 0 || y == ny - 1) {
      kind = 2;
      cy = (y == 0) ? 1 : ny - 2;
    }
  }
  int xm = cx - 1, xp = cx + 1, ym = cy - 1, yp = cy + 1;
  if (BC == BC_PERIODIC || BC == BC_CHANNEL) {
    xm = (cx == 0) ? nx - 1 : xm;
    xp = (cx == nx - 1) ? 0 : xp;
  }
  if (BC == BC_PERIODIC) {
    ym = (cy == 0) ? ny - 1 : ym;
    yp = (cy == ny - 1) ? 0 : yp;
  }

  C f[9], gf[5], gs[5];
  Pops<S, C>::pull(src, pitch, plane, cx, xm, xp, cy, ym, yp, inv_scale, f, gf, gs);

  const uint32_t off = (uint32_t)y * (uint32_t)pitch + (uint32_t)x;
  if (BC != BC_PERIODIC && kind >= 0) {
    const uint32_t noff = (uint32_t)cy * (uint32_t)pitch + (uint32_t)cx;
    Medium<C> mdn = phi_field ? medium_at<C>(P, phi_field[noff]) : P.um;
    if (P.hv_local) set_exchange<C>(mdn, hv_local_at<C>(P, um_in[noff]));
    Macro<C> mn;
    macros<C>(P, mdn, f, gf, gs, mn);
    C dTwf = mn.dTf, dTws = mn.dTs;  // adiabatic: the neighbour's temperature
    if (kind == 0) dTwf = dTws = P.dT_hot;
    if (kind == 1) dTwf = dTws = P.dT_cold;
    nee<C>(P, mn, dTwf, dTws, f, gf, gs);
  }
  if (pre_out) {  // record the pre-collision state (reverse-mode recomputation)
#pragma unroll
    for (int i = 0; i < 9; ++i) pre_out[(int64_t)i * plane + off] = f[i];
#pragma unroll
    for (int i = 0; i < 5; ++i) pre_out[(int64_t)(9 + i) * plane + off] = gf[i];
#pragma unroll
    for (int i = 0; i < 5; ++i) pre_out[(int64_t)(14 + i) * plane + off] = gs[i];
  }
  Medium<C> md = phi_field ? medium_at<C>(P, phi_field[off]) : P.um;
  if (P.hv_local) set_exchange<C>(md, hv_local_at<C>(P, um_in[off]));
  Macro<C> m;
  macros<C>(P, md, f, gf, gs, m);
  if (P.hv_local) um_out[off] = m.umag;  // u_m of Eq. 52 for the next state
  if (write_macros) store_macros<C>(mac, plane, off, m);
  collide<C>(P, m, f, gf, gs);
  Pops<S, C>::store(dst, plane, off, scale, f, gf, gs, (uint32_t)off, tick);
}

// Step counter of the stochastic rounding: every thread reads one slot and
// one thread writes the next value to the other (the slots alternate with
// the A-B buffers, so no slot is read and written by the same launch).
template <typename S, typename C>
__device__ __forceinline__ uint32_t read_tick(const uint32_t* __restrict__ tick_in,
                                              uint32_t* __restrict__ tick_out) {
  uint32_t tick = 0;
  if constexpr (Codec<S, C>::kStochastic) {
    tick = *tick_in;
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0)
      *tick_out = tick + 1u;
  }
  return tick;
}

template <typename S, typename C, int BC>
__global__ void __launch_bounds__(256) k_step(const S* __restrict__ src, S* __restrict__ dst,
                                              const C* __restrict__ phi_field,
                                              C* __restrict__ mac, const NodeParams<C> P,
                                              const int nx, const int ny, const int64_t pitch,
                                              const int64_t plane, const C scale,
                                              const C inv_scale, const int write_macros,
                                              const uint32_t* __restrict__ tick_in,
                                              uint32_t* __restrict__ tick_out,
                                              const C* __restrict__ um_in,
                                              C* __restrict__ um_out, const int slab_walls) {
  grid_dep_wait();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const uint32_t tick = read_tick<S, C>(tick_in, tick_out);
  if (x >= nx || y >= ny) return;
  if (BC == BC_SLAB && ((y == 0 && !(slab_walls & SLAB_LO_WALL)) ||
                        (y == ny - 1 && !(slab_walls & SLAB_HI_WALL))))
    return;  // a halo row: the neighbouring slab's values, read only
  step_node<S, C, BC>(src, dst, phi_field, mac, P, x, y, nx, ny, pitch, plane, scale, inv_scale,
                      write_macros, tick, nullptr, um_in, um_out, slab_walls);
}

// S_0 from the fields held in the macro planes (rho, ux, uy, Tf, Ts), then
// its macroscopic values (overwriting the planes) and its collision.
template <typename S, typename C>
__global__ void __launch_bounds__(256) k_init(S* __restrict__ dst,
                                              const C* __restrict__ phi_field,
                                              C* __restrict__ mac, const NodeParams<C> P,
                                              const int nx, const int ny, const int64_t pitch,
                                              const int64_t plane, const C scale,
                                              C* __restrict__ pre_out, C* __restrict__ um_out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= nx || y >= ny) return;
  const int64_t off = (int64_t)y * pitch + x;
  Medium<C> md = phi_field ? medium_at<C>(P, phi_field[off]) : P.um;
  if (P.hv_local) {  // u_m of S_0: the initial field's |u|
    const C ux = mac[plane + off], uy = mac[2 * plane + off];
    set_exchange<C>(md, hv_local_at<C>(P, sqrt_<C>(ux * ux + uy * uy)));
  }
  C f[9], gf[5], gs[5];
  equilibrium<C>(P, md.phi, mac[off], mac[plane + off], mac[2 * plane + off],
                 mac[3 * plane + off], mac[4 * plane + off], f, gf, gs);
  if (pre_out) {  // S_0, for reverse-mode recomputation
#pragma unroll
    for (int i = 0; i < 9; ++i) pre_out[(int64_t)i * plane + off] = f[i];
#pragma unroll
    for (int i = 0; i < 5; ++i) pre_out[(int64_t)(9 + i) * plane + off] = gf[i];
#pragma unroll
    for (int i = 0; i < 5; ++i) pre_out[(int64_t)(14 + i) * plane + off] = gs[i];
  }
  Macro<C> m;
  macros<C>(P, md, f, gf, gs, m);
  if (P.hv_local) um_out[off] = m.umag;
  store_macros<C>(mac, plane, off, m);
  collide<C>(P, m, f, gf, gs);
  Pops<S, C>::store(dst, plane, off, scale, f, gf, gs, (uint32_t)off, 0xffffffffu);
}

template <typename S, typename C>
cudaError_t launch_step_t(const LatticeArgs& a, const NodeParams<double>& Pd, StepShape s,
                          cudaStream_t st) {
  const NodeParams<C> P = cast_params<C>(Pd);
  dim3 block(s.bx, s.by);
  dim3 grid((a.nx + s.bx - 1) / s.bx, (a.ny + s.by - 1) / s.by);
  const C scale = C(a.enc_scale), inv_scale = C(1.0 / a.enc_scale);
  const S* src = static_cast<const S*>(a.src);
  S* dst = static_cast<S*>(a.dst);
  const C* phi = static_cast<const C*>(a.phi);
  C* mac = static_cast<C*>(a.mac);
  const C* um_in = static_cast<const C*>(a.um_in);
  C* um_out = static_cast<C*>(a.um_out);
  const bool ch = a.chained != 0;
  const dim3 g = grid, b = block;
  cudaError_t e;
#define LTNE_STEP_LAUNCH(bc, walls)                                                            \
  e = launch_kernel(ch, k_step<S, C, bc>, g, b, 0, st, src, dst, phi, mac, P, a.nx, a.ny,       \
                    a.pitch, a.plane, scale, inv_scale, a.write_macros, a.tick_in, a.tick_out,  \
                    um_in, um_out, walls)
  switch (a.bc) {
    case BC_CAVITY: LTNE_STEP_LAUNCH(BC_CAVITY, 0); break;
    case BC_PERIODIC: LTNE_STEP_LAUNCH(BC_PERIODIC, 0); break;
    case BC_CHANNEL: LTNE_STEP_LAUNCH(BC_CHANNEL, 0); break;
    case BC_SLAB: LTNE_STEP_LAUNCH(BC_SLAB, a.slab_walls); break;
    default:
      return cudaErrorInvalidValue;
  }
#undef LTNE_STEP_LAUNCH
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <typename S, typename C>
cudaError_t launch_init_t(const LatticeArgs& a, const NodeParams<double>& Pd, cudaStream_t st) {
  const NodeParams<C> P = cast_params<C>(Pd);
  dim3 block(128, 2);
  dim3 grid((a.nx + 127) / 128, (a.ny + 1) / 2);
  k_init<S, C><<<grid, block, 0, st>>>(static_cast<S*>(a.dst), static_cast<const C*>(a.phi),
                                       static_cast<C*>(a.mac), P, a.nx, a.ny, a.pitch, a.plane,
                                       C(a.enc_scale), static_cast<C*>(a.pre_out),
                                       static_cast<C*>(a.um_out));
  return cudaGetLastError();
}

}  // namespace ltne

#define LTNE_DEFINE_LAUNCHERS(tag, S, C)                                                        \
  namespace ltne {                                                                             \
  cudaError_t launch_step_##tag(const LatticeArgs& a, const NodeParams<double>& P,             \
                                StepShape s, cudaStream_t st) {                                \
    return launch_step_t<S, C>(a, P, s, st);                                                   \
  }                                                                                            \
  cudaError_t launch_init_##tag(const LatticeArgs& a, const NodeParams<double>& P,             \
                                cudaStream_t st) {                                             \
    return launch_init_t<S, C>(a, P, st);                                                      \
  }                                                                                            \
  }
