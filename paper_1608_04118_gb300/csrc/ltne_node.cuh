// ltne_node.cuh -- per-node physics of the three-distribution MRT-LB step
// (Liu & He, arXiv:1608.04118), in registers, for one lattice node.
//
// Every population is carried as a deviation from the rest equilibrium:
//   df_i = f_i - w_i rho0       (D2Q9, Eq. 8 and the weights below Eq. 24)
//   dg_i = g_i - w~_i T0        (D2Q5, weights below Eq. 31)
// The rest equilibrium has moments M(w rho0) = rho0 (1, -2, 1, 0, ..., 0)
// and N(w~ T0) = T0 (1, 0, 0, -4 + 5 varpi, 0), so the collision of Eq. 10
// and Eqs. 32-33 is applied to deviation moments unchanged except for the
// constant parts of m^eq_1, m^eq_2 and n^eq_3, which cancel.  Keeping the
// O(1) rest part out of the arithmetic is what lets FP32 (and the 16-bit
// storage forms) resolve velocities of O(1e-3).
//
// The moment transforms are closed forms of the products with M (Eq. 13)
// and N (Eq. 36); M^-1 = M^T diag(1/9,1/36,1/36,1/6,1/12,1/6,1/12,1/4,1/4)
// and N^-1 = N^T diag(1/5,1/2,1/2,1/20,1/4) follow from the row
// orthogonality of M and N.  No tensor cores: each is a few dozen adds.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace ltne {

// Lattice constants in compute type C, built from the paper's values.
template <typename C>
struct NodeParams {
  C rho0, T0;                       // deviation references
  C s_e, s_eps, s_q, s_nu;          // Eq. 17 (s_0 = s_3 = s_5 = 1)
  C zeta_a, zeta_e, zeta_nu;        // Eq. 39 (zeta_0 = 1)
  C eta_a, eta_e, eta_nu;           // Eq. 40 (eta_0 = 1)
  C c3;                             // -4 + 5 varpi (Eq. 37)
  C wt0, wt1;                       // w~_0 = 1 - varpi, w~_{1..4} = varpi/4
  C gbeta, ext_ax, ext_ay;          // Eq. 6 buoyancy (+ test acceleration)
  C phi_u;                          // uniform porosity
  C hcoef;                          // h_v / (rho c)_f
  C sigma;                          // (rho c)_s / (rho c)_f
  C qf, qs;                         // Q_f''', Q_s''' (Eq. 45)
  C dT_hot, dT_cold;                // wall temperatures minus T0
  // Medium (Eq. 7) as the two coefficients c0 = nu_f / K and
  // c1 = F_phi / sqrt(K) of Eqs. 5 and 22:
  //   Darcy K, constant F : c0 = nu_over_K, c1 = Fconst * inv_sqrtK
  //   Darcy K, Ergun F    : c1 = 1.75 / sqrt(150 phi^3) * inv_sqrtK
  //   Ergun K, Ergun F    : c0 = erg_a (1-phi)^2/phi^3, c1 = erg_b (1-phi)/phi^3
  //   Ergun K, constant F : c1 = erg_c (1-phi) / phi^(3/2)
  // with erg_a = 150 nu_f / d^2, erg_b = 1.75 / d, erg_c = Fconst sqrt(150) / d.
  C nu_over_K, inv_sqrtK, Fconst, erg_a, erg_b, erg_c;
  int kmode;                        // 0 Darcy, 1 Ergun
  int fmode;                        // 0 constant, 1 Ergun
};

template <typename C>
struct Macro {
  C rho, drho, ux, uy, umag;        // Eq. 18, Eq. 20
  C dTf, dTs;                       // Eqs. 43-44 (minus T0)
  C Fx, Fy;                         // Eq. 5
  C a, b;                           // h_v/(phi (rho c)_f), h_v/((1-phi)(rho c)_s)
  C phi, inv_phi;
};

template <typename C> __device__ __forceinline__ C csqrt_(C x);
template <> __device__ __forceinline__ float csqrt_<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double csqrt_<double>(double x) { return sqrt(x); }

// c0 = nu_f/K and c1 = F_phi/sqrt(K) at porosity phi (Eqs. 5, 7, 22).
template <typename C>
__device__ __forceinline__ void medium(const NodeParams<C>& P, C phi, C inv_phi, C& c0, C& c1) {
  if (P.kmode == 0) {
    c0 = P.nu_over_K;
    if (P.fmode == 0) {
      c1 = P.Fconst * P.inv_sqrtK;
    } else {
      c1 = C(1.75) / csqrt_<C>(C(150) * phi * phi * phi) * P.inv_sqrtK;
    }
  } else {
    C om = C(1) - phi;
    C ip3 = inv_phi * inv_phi * inv_phi;
    c0 = P.erg_a * om * om * ip3;
    if (P.fmode == 1) {
      c1 = P.erg_b * om * ip3;
    } else {
      c1 = P.erg_c * om * inv_phi / csqrt_<C>(phi);
    }
  }
}

// Macroscopic values of a node from its pre-collision deviations:
// temperatures by the explicit 2x2 solve (Eqs. 43-46), buoyancy (Eq. 6,
// gravity along -y), density (Eq. 18), velocity by the explicit root of the
// implicit Eq. 19 (Eqs. 20-22) and the total force (Eq. 5).
template <typename C>
__device__ __forceinline__ void macros(const NodeParams<C>& P, C phi, const C (&f)[9],
                                       const C (&gf)[5], const C (&gs)[5], Macro<C>& m) {
  m.phi = phi;
  m.inv_phi = C(1) / phi;
  m.a = P.hcoef * m.inv_phi;
  m.b = P.hcoef / ((C(1) - phi) * P.sigma);
  const C d0 = C(0.5) * m.a, d1 = C(0.5) * m.b;
  const C dAf = (gf[0] + gf[1] + gf[2] + gf[3] + gf[4]) + C(0.5) * P.qf;
  const C dAs = (gs[0] + gs[1] + gs[2] + gs[3] + gs[4]) + C(0.5) * P.qs;
  const C inv = C(1) / (C(1) + d0 + d1);
  m.dTf = ((C(1) + d1) * dAf + d0 * dAs) * inv;
  m.dTs = (d1 * dAf + (C(1) + d0) * dAs) * inv;
  const C Gx = P.ext_ax;
  const C Gy = P.gbeta * m.dTf + P.ext_ay;

  m.drho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
  m.rho = P.rho0 + m.drho;
  const C jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
  const C jy = (f[2] - f[4]) + (f[5] - f[7]) + (f[6] - f[8]);
  const C inv_rho = C(1) / m.rho;
  const C vx = jx * inv_rho + C(0.5) * phi * Gx;  // Eq. 21
  const C vy = jy * inv_rho + C(0.5) * phi * Gy;
  C c0, c1;
  medium<C>(P, phi, m.inv_phi, c0, c1);
  const C l0 = C(0.5) * (C(1) + C(0.5) * phi * c0);  // Eq. 22
  const C l1 = C(0.5) * phi * c1;
  const C vmag = csqrt_<C>(vx * vx + vy * vy);
  const C inv_den = C(1) / (l0 + csqrt_<C>(l0 * l0 + l1 * vmag));  // Eq. 20
  m.ux = vx * inv_den;
  m.uy = vy * inv_den;
  m.umag = vmag * inv_den;
  const C drag = c0 + c1 * m.umag;
  m.Fx = phi * (Gx - drag * m.ux);  // Eq. 5
  m.Fy = phi * (Gy - drag * m.uy);
}

// Collision of all three distributions, in place on the deviations.
// Flow: m* = m - Lambda (m - m^eq) + (I - Lambda/2) S~ (Eq. 10) with m^eq of
// Eq. 15 and S~ = M S for the porous forcing S_i = w_i rho [e_i.F/cs^2 +
// ((e_i.u)(e_i.F) - cs^2 u.F)/(phi cs^4)] (Eq. 16 is garbled in the text;
// this is the forcing whose moments are 0, rho F, rho (uF + Fu)/phi):
//   S~ = (0, 6 rho u.F/phi, -6 rho u.F/phi, rho Fx, -rho Fx, rho Fy,
//         -rho Fy, 2 rho (ux Fx - uy Fy)/phi, rho (ux Fy + uy Fx)/phi).
// Temperatures: n* = n - Q (n - n^eq) + (I - Q/2) Psi (Eqs. 32-33) with
// n^eq of Eqs. 37-38 and Psi = Sr (1, 0, 0, -4 + 5 varpi, 0) (Eqs. 29-31).
template <typename C>
__device__ __forceinline__ void collide(const NodeParams<C>& P, const Macro<C>& m, C (&f)[9],
                                        C (&gf)[5], C (&gs)[5]) {
  const C rho = m.rho, ux = m.ux, uy = m.uy, Fx = m.Fx, Fy = m.Fy, ip = m.inv_phi;
  // ---- flow: deviation moments M df
  const C sa = (f[1] + f[2]) + (f[3] + f[4]);
  const C sd = (f[5] + f[6]) + (f[7] + f[8]);
  const C m1 = C(-4) * f[0] - sa + C(2) * sd;
  const C m2 = C(4) * f[0] - C(2) * sa + sd;
  const C dx = (f[5] - f[6]) + (f[8] - f[7]);
  const C dy = (f[5] - f[7]) + (f[6] - f[8]);
  const C m4 = C(-2) * (f[1] - f[3]) + dx;
  const C m6 = C(-2) * (f[2] - f[4]) + dy;
  const C m7 = (f[1] - f[2]) + (f[3] - f[4]);
  const C m8 = (f[5] - f[6]) + (f[7] - f[8]);
  // equilibrium (deviation) moments, Eq. 15
  const C ru2 = C(3) * rho * (ux * ux + uy * uy) * ip;
  const C meq1 = C(-2) * m.drho + ru2;
  const C meq2 = m.drho - ru2;
  const C rux = rho * ux, ruy = rho * uy;
  const C meq7 = rho * (ux * ux - uy * uy) * ip;
  const C meq8 = rho * ux * uy * ip;
  // forcing moments
  const C rFx = rho * Fx, rFy = rho * Fy;
  const C S1 = C(6) * rho * (ux * Fx + uy * Fy) * ip;
  const C S7 = C(2) * rho * (ux * Fx - uy * Fy) * ip;
  const C S8 = rho * (ux * Fy + uy * Fx) * ip;
  // post-collision moments
  const C ms0 = m.drho;
  const C ms1 = m1 - P.s_e * (m1 - meq1) + (C(1) - C(0.5) * P.s_e) * S1;
  const C ms2 = m2 - P.s_eps * (m2 - meq2) - (C(1) - C(0.5) * P.s_eps) * S1;
  const C ms3 = rux + C(0.5) * rFx;  // s_3 = 1
  const C ms4 = m4 - P.s_q * (m4 + rux) - (C(1) - C(0.5) * P.s_q) * rFx;
  const C ms5 = ruy + C(0.5) * rFy;  // s_5 = 1
  const C ms6 = m6 - P.s_q * (m6 + ruy) - (C(1) - C(0.5) * P.s_q) * rFy;
  const C ms7 = m7 - P.s_nu * (m7 - meq7) + (C(1) - C(0.5) * P.s_nu) * S7;
  const C ms8 = m8 - P.s_nu * (m8 - meq8) + (C(1) - C(0.5) * P.s_nu) * S8;
  // df* = M^-1 m*
  const C r0 = ms0 * C(1.0 / 9.0), r1 = ms1 * C(1.0 / 36.0), r2 = ms2 * C(1.0 / 36.0);
  const C r3 = ms3 * C(1.0 / 6.0), r4 = ms4 * C(1.0 / 12.0);
  const C r5 = ms5 * C(1.0 / 6.0), r6 = ms6 * C(1.0 / 12.0);
  const C r7 = ms7 * C(0.25), r8 = ms8 * C(0.25);
  const C ax = r0 - r1 - C(2) * r2;  // common part of i = 1..4
  const C dg = r0 + C(2) * r1 + r2;  // common part of i = 5..8
  const C px = r3 - C(2) * r4, py = r5 - C(2) * r6;
  const C qx = r3 + r4, qy = r5 + r6;
  f[0] = r0 - C(4) * r1 + C(4) * r2;
  f[1] = ax + px + r7;
  f[2] = ax + py - r7;
  f[3] = ax - px + r7;
  f[4] = ax - py - r7;
  f[5] = dg + qx + qy + r8;
  f[6] = dg - qx + qy - r8;
  f[7] = dg - qx - qy + r8;
  f[8] = dg + qx - qy - r8;

  // ---- temperatures
  const C Srf = m.a * (m.dTs - m.dTf) + P.qf;  // Eq. 42
  const C Srs = m.b * (m.dTf - m.dTs) + P.qs;
  {
    const C Tf = P.T0 + m.dTf;
    const C n1 = gf[1] - gf[3], n2 = gf[2] - gf[4];
    const C n3 = C(-4) * gf[0] + ((gf[1] + gf[2]) + (gf[3] + gf[4]));
    const C n4 = (gf[1] - gf[2]) + (gf[3] - gf[4]);
    const C ns0 = m.dTf + C(0.5) * Srf;
    const C ns1 = n1 - P.zeta_a * (n1 - ux * Tf * ip);
    const C ns2 = n2 - P.zeta_a * (n2 - uy * Tf * ip);
    const C ns3 = n3 - P.zeta_e * (n3 - P.c3 * m.dTf) + (C(1) - C(0.5) * P.zeta_e) * P.c3 * Srf;
    const C ns4 = n4 - P.zeta_nu * n4;
    const C t0 = ns0 * C(0.2), t1 = ns1 * C(0.5), t2 = ns2 * C(0.5);
    const C t3 = ns3 * C(0.05), t4 = ns4 * C(0.25);
    gf[0] = t0 - C(4) * t3;
    gf[1] = t0 + t1 + t3 + t4;
    gf[2] = t0 + t2 + t3 - t4;
    gf[3] = t0 - t1 + t3 + t4;
    gf[4] = t0 - t2 + t3 - t4;
  }
  {
    const C n1 = gs[1] - gs[3], n2 = gs[2] - gs[4];
    const C n3 = C(-4) * gs[0] + ((gs[1] + gs[2]) + (gs[3] + gs[4]));
    const C n4 = (gs[1] - gs[2]) + (gs[3] - gs[4]);
    const C ns0 = m.dTs + C(0.5) * Srs;
    const C ns1 = n1 - P.eta_a * n1;
    const C ns2 = n2 - P.eta_a * n2;
    const C ns3 = n3 - P.eta_e * (n3 - P.c3 * m.dTs) + (C(1) - C(0.5) * P.eta_e) * P.c3 * Srs;
    const C ns4 = n4 - P.eta_nu * n4;
    const C t0 = ns0 * C(0.2), t1 = ns1 * C(0.5), t2 = ns2 * C(0.5);
    const C t3 = ns3 * C(0.05), t4 = ns4 * C(0.25);
    gs[0] = t0 - C(4) * t3;
    gs[1] = t0 + t1 + t3 + t4;
    gs[2] = t0 + t2 + t3 - t4;
    gs[3] = t0 - t1 + t3 + t4;
    gs[4] = t0 - t2 + t3 - t4;
  }
}

// Wall rebuild by non-equilibrium extrapolation from the interior
// neighbour n (values mn, populations in f/gf/gs on entry): on exit the
// arrays hold the wall node's populations
//   f_b  = w rho_n + (f_n - f^eq(rho_n, u_n, phi_n))        (u_wall = 0)
//   gf_b = w~ T_w  + (gf_n - g_f^eq(T_f,n, u_n, phi_n))      (Eq. 50)
//   gs_b = w~ T_w  + (gs_n - w~ T_s,n)                       (Eq. 51)
// dTwf, dTws are the wall temperatures minus T0 for the two phases.
template <typename C>
__device__ __forceinline__ void nee(const NodeParams<C>& P, const Macro<C>& mn, C dTwf, C dTws,
                                    C (&f)[9], C (&gf)[5], C (&gs)[5]) {
  const C ux = mn.ux, uy = mn.uy, ip = mn.inv_phi, rho = mn.rho;
  // f^eq(rho,u,phi) - w rho = w rho [3 e.u + 4.5 (e.u)^2/phi - 1.5 u^2/phi] (Eq. 24)
  const C q = C(1.5) * (ux * ux + uy * uy) * ip;
  const C w0 = C(4.0 / 9.0) * rho, w1 = C(1.0 / 9.0) * rho, w2 = C(1.0 / 36.0) * rho;
  f[0] -= w0 * (-q);
  const C e1 = ux, e2 = uy, e5 = ux + uy, e6 = uy - ux;
  f[1] -= w1 * (C(3) * e1 + C(4.5) * e1 * e1 * ip - q);
  f[2] -= w1 * (C(3) * e2 + C(4.5) * e2 * e2 * ip - q);
  f[3] -= w1 * (C(-3) * e1 + C(4.5) * e1 * e1 * ip - q);
  f[4] -= w1 * (C(-3) * e2 + C(4.5) * e2 * e2 * ip - q);
  f[5] -= w2 * (C(3) * e5 + C(4.5) * e5 * e5 * ip - q);
  f[6] -= w2 * (C(3) * e6 + C(4.5) * e6 * e6 * ip - q);
  f[7] -= w2 * (C(-3) * e5 + C(4.5) * e5 * e5 * ip - q);
  f[8] -= w2 * (C(-3) * e6 + C(4.5) * e6 * e6 * ip - q);
  // thermal: g_f^eq - w~ T = (e.u) T / (2 phi) for i = 1..4 (Eq. 50)
  const C Tf = P.T0 + mn.dTf;
  const C hx = C(0.5) * ux * Tf * ip, hy = C(0.5) * uy * Tf * ip;
  const C jf0 = P.wt0 * (dTwf - mn.dTf), jf1 = P.wt1 * (dTwf - mn.dTf);
  gf[0] += jf0;
  gf[1] += jf1 - hx;
  gf[2] += jf1 - hy;
  gf[3] += jf1 + hx;
  gf[4] += jf1 + hy;
  const C js0 = P.wt0 * (dTws - mn.dTs), js1 = P.wt1 * (dTws - mn.dTs);
  gs[0] += js0;
  gs[1] += js1;
  gs[2] += js1;
  gs[3] += js1;
  gs[4] += js1;
}

// Equilibrium deviations of given fields (Eqs. 24, 50, 51), for S_0.
template <typename C>
__device__ __forceinline__ void equilibrium(const NodeParams<C>& P, C phi, C rho, C ux, C uy,
                                            C Tf, C Ts, C (&f)[9], C (&gf)[5], C (&gs)[5]) {
  const C ip = C(1) / phi;
  const C drho = rho - P.rho0;
  const C q = C(1.5) * (ux * ux + uy * uy) * ip;
  const C w0 = C(4.0 / 9.0), w1 = C(1.0 / 9.0), w2 = C(1.0 / 36.0);
  const C e1 = ux, e2 = uy, e5 = ux + uy, e6 = uy - ux;
  f[0] = w0 * drho + w0 * rho * (-q);
  f[1] = w1 * drho + w1 * rho * (C(3) * e1 + C(4.5) * e1 * e1 * ip - q);
  f[2] = w1 * drho + w1 * rho * (C(3) * e2 + C(4.5) * e2 * e2 * ip - q);
  f[3] = w1 * drho + w1 * rho * (C(-3) * e1 + C(4.5) * e1 * e1 * ip - q);
  f[4] = w1 * drho + w1 * rho * (C(-3) * e2 + C(4.5) * e2 * e2 * ip - q);
  f[5] = w2 * drho + w2 * rho * (C(3) * e5 + C(4.5) * e5 * e5 * ip - q);
  f[6] = w2 * drho + w2 * rho * (C(3) * e6 + C(4.5) * e6 * e6 * ip - q);
  f[7] = w2 * drho + w2 * rho * (C(-3) * e5 + C(4.5) * e5 * e5 * ip - q);
  f[8] = w2 * drho + w2 * rho * (C(-3) * e6 + C(4.5) * e6 * e6 * ip - q);
  const C dTf = Tf - P.T0, dTs = Ts - P.T0;
  const C hx = C(0.5) * ux * Tf * ip, hy = C(0.5) * uy * Tf * ip;
  gf[0] = P.wt0 * dTf;
  gf[1] = P.wt1 * dTf + hx;
  gf[2] = P.wt1 * dTf + hy;
  gf[3] = P.wt1 * dTf - hx;
  gf[4] = P.wt1 * dTf - hy;
  gs[0] = P.wt0 * dTs;
  gs[1] = P.wt1 * dTs;
  gs[2] = P.wt1 * dTs;
  gs[3] = P.wt1 * dTs;
  gs[4] = P.wt1 * dTs;
}

// ---- storage codec: deviation <-> stored value
template <typename S, typename C> struct Codec;
template <> struct Codec<double, double> {
  static __device__ __forceinline__ double dec(double v, double) { return v; }
  static __device__ __forceinline__ double enc(double v, double) { return v; }
};
template <> struct Codec<float, float> {
  static __device__ __forceinline__ float dec(float v, float) { return v; }
  static __device__ __forceinline__ float enc(float v, float) { return v; }
};
template <> struct Codec<__half, float> {
  static __device__ __forceinline__ float dec(__half v, float inv_scale) {
    return __half2float(v) * inv_scale;
  }
  static __device__ __forceinline__ __half enc(float v, float scale) {
    return __float2half_rn(v * scale);
  }
};
template <> struct Codec<__nv_bfloat16, float> {
  static __device__ __forceinline__ float dec(__nv_bfloat16 v, float inv_scale) {
    return __bfloat162float(v) * inv_scale;
  }
  static __device__ __forceinline__ __nv_bfloat16 enc(float v, float scale) {
    return __float2bfloat16_rn(v * scale);
  }
};

}  // namespace ltne
