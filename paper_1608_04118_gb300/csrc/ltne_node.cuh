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

// Per-node functions compile for host and device (the host copies serve
// derivative checks of the reverse-mode functions).
#define LTNE_HD __host__ __device__ __forceinline__

namespace ltne {

// Porosity-dependent coefficients of one node: exchange coefficients of
// Eq. 42 (a = h_v/(phi (rho c)_f), b = h_v/((1-phi)(rho c)_s)), the factor
// 1/(1 + d0 + d1) of Eqs. 43-44 (Eq. 46: d0 = a/2, d1 = b/2), the medium
// coefficients c0 = nu_f/K and c1 = F_phi/sqrt(K) of Eqs. 5 and 7, and
// l0, l1 of Eq. 22.
template <typename C>
struct Medium {
  C phi, inv_phi, a, b, inv_1d, c0, c1, l0, l1;
  C inv_oms;  // 1 / ((1 - phi) sigma)
};

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
  Medium<C> um;                     // the coefficients at the uniform porosity
  // Local h_v of Eq. 52: h_v/(rho c)_f = hv_c |u_prev|^0.644 with
  // hv_c = 0.376 Pr^0.37 (D_p/nu_f)^0.644 alpha_f / D_p^2.
  int hv_local;
  C hv_c;
  int tcorr;  // correction term of Sec. 3.2 on (N C~ = (0, T_f F/phi, 0, 0))
};

template <typename C>
struct Macro {
  C rho, drho, ux, uy, umag;        // Eq. 18, Eq. 20
  C jx, jy;                         // sum_i e_i f_i (deviations carry no momentum)
  C sgf, sgs;                       // sum_i dg_i of both phases
  C dTf, dTs;                       // Eqs. 43-44 (minus T0)
  C Srf, Srs;                       // Eq. 42 source strengths
  C Fx, Fy;                         // Eq. 5
  C a, b;                           // h_v/(phi (rho c)_f), h_v/((1-phi)(rho c)_s)
  C phi, inv_phi;
};

template <typename C> LTNE_HD C cfma_(C a, C b, C c);
template <> LTNE_HD float cfma_<float>(float a, float b, float c) {
  return fmaf(a, b, c);
}
template <> LTNE_HD double cfma_<double>(double a, double b, double c) {
  return fma(a, b, c);
}

// x / d for a small integer d, given rc = RN(1/d): one residual correction
// (r = x - d q is exact in an FMA) removes the systematic bias that a plain
// product with the rounded reciprocal would add at every step -- in FP32,
// 6 RN(1/6) = 1 + 3e-8 would grow the momentum by that factor per step.
template <typename C>
LTNE_HD C div_small(C x, C d, C rc) {
  const C q = x * rc;
  const C r = cfma_<C>(-d, q, x);
  return cfma_<C>(r, rc, q);
}

// Reciprocal and square root of non-conserved quantities (porosity-derived
// coefficients, 1/rho and the velocity solve of Eq. 20).  FP32 uses the
// hardware approximations (about 1 ulp, no long IEEE expansion; errors in
// these quantities relax each step instead of accumulating); FP64 keeps the
// correctly rounded operations.
template <typename C> LTNE_HD C rcp_(C x);
template <> LTNE_HD double rcp_<double>(double x) { return 1.0 / x; }
template <> LTNE_HD float rcp_<float>(float x) {
#ifdef __CUDA_ARCH__
  return __fdividef(1.0f, x);
#else
  return 1.0f / x;
#endif
}
template <typename C> LTNE_HD C sqrt_(C x);
template <> LTNE_HD double sqrt_<double>(double x) { return sqrt(x); }
template <> LTNE_HD float sqrt_<float>(float x) {
#ifdef __CUDA_ARCH__
  return x > 0.0f ? x * rsqrtf(x) : 0.0f;
#else
  return sqrtf(x);
#endif
}

template <typename C> LTNE_HD C csqrt_(C x);
template <> LTNE_HD float csqrt_<float>(float x) { return sqrtf(x); }
template <> LTNE_HD double csqrt_<double>(double x) { return sqrt(x); }

// The coefficients at porosity phi (per-node porosity fields).
//   Darcy K, constant F : c0 = nu_over_K, c1 = Fconst * inv_sqrtK
//   Darcy K, Ergun F    : c1 = 1.75 / sqrt(150 phi^3) * inv_sqrtK
//   Ergun K, Ergun F    : c0 = erg_a (1-phi)^2/phi^3, c1 = erg_b (1-phi)/phi^3
//   Ergun K, constant F : c1 = erg_c (1-phi) / phi^(3/2)
template <typename C>
LTNE_HD Medium<C> medium_at(const NodeParams<C>& P, C phi) {
  Medium<C> md;
  md.phi = phi;
  md.inv_phi = rcp_<C>(phi);
  md.inv_oms = rcp_<C>((C(1) - phi) * P.sigma);
  md.a = P.hcoef * md.inv_phi;
  md.b = P.hcoef * md.inv_oms;
  md.inv_1d = rcp_<C>(C(1) + C(0.5) * md.a + C(0.5) * md.b);
  if (P.kmode == 0) {
    md.c0 = P.nu_over_K;
    if (P.fmode == 0) {
      md.c1 = P.Fconst * P.inv_sqrtK;
    } else {
      md.c1 = C(1.75) * rcp_<C>(sqrt_<C>(C(150) * phi * phi * phi)) * P.inv_sqrtK;
    }
  } else {
    const C om = C(1) - phi;
    const C ip3 = md.inv_phi * md.inv_phi * md.inv_phi;
    md.c0 = P.erg_a * om * om * ip3;
    if (P.fmode == 1) {
      md.c1 = P.erg_b * om * ip3;
    } else {
      md.c1 = P.erg_c * om * md.inv_phi * rcp_<C>(sqrt_<C>(phi));
    }
  }
  md.l0 = C(0.5) * (C(1) + C(0.5) * phi * md.c0);  // Eq. 22
  md.l1 = C(0.5) * phi * md.c1;
  return md;
}

// h_v / (rho c)_f from the correlation of Eq. 52 at a node whose previous
// velocity magnitude is um.
template <typename C>
LTNE_HD C hv_local_at(const NodeParams<C>& P, C um) {
  if (!(um > C(0))) return C(0);
#ifdef __CUDA_ARCH__
  return P.hv_c * exp2(C(0.644) * log2(um));
#else
  return P.hv_c * pow(um, C(0.644));
#endif
}

// The exchange-dependent coefficients of md with a node-local h_v.
template <typename C>
LTNE_HD void set_exchange(Medium<C>& md, C hv) {
  md.a = hv * md.inv_phi;
  md.b = hv * md.inv_oms;
  md.inv_1d = rcp_<C>(C(1) + C(0.5) * md.a + C(0.5) * md.b);
}

// Macroscopic values of a node from its pre-collision deviations:
// temperatures by the explicit 2x2 solve (Eqs. 43-46), buoyancy (Eq. 6,
// gravity along -y), density (Eq. 18), velocity by the explicit root of the
// implicit Eq. 19 (Eqs. 20-22) and the total force (Eq. 5).
template <typename C>
LTNE_HD void macros(const NodeParams<C>& P, const Medium<C>& md,
                                       const C (&f)[9], const C (&gf)[5], const C (&gs)[5],
                                       Macro<C>& m) {
  const C phi = md.phi;
  m.phi = phi;
  m.inv_phi = md.inv_phi;
  m.a = md.a;
  m.b = md.b;
  m.sgf = (gf[0] + gf[1]) + (gf[2] + gf[3]) + gf[4];
  m.sgs = (gs[0] + gs[1]) + (gs[2] + gs[3]) + gs[4];
  // Eqs. 43-44 solve T = sum g + Sr/2 (Eqs. 41-42).  They are evaluated
  // through the phase difference D = T_f - T_s = (A_f - A_s)/(1 + d0 + d1),
  // A = sum g + Q/2, so that each temperature is its population sum plus a
  // small exchange correction and no rounded factor multiplies the sum.
  const C D = ((m.sgf - m.sgs) + C(0.5) * (P.qf - P.qs)) * md.inv_1d;
  m.Srf = P.qf - m.a * D;
  m.Srs = P.qs + m.b * D;
  m.dTf = m.sgf + C(0.5) * m.Srf;
  m.dTs = m.sgs + C(0.5) * m.Srs;
  const C Gx = P.ext_ax;
  const C Gy = P.gbeta * m.dTf + P.ext_ay;

  m.drho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
  m.rho = P.rho0 + m.drho;
  m.jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
  m.jy = (f[2] - f[4]) + (f[5] - f[7]) + (f[6] - f[8]);
  const C inv_rho = rcp_<C>(m.rho);
  const C vx = m.jx * inv_rho + C(0.5) * phi * Gx;  // Eq. 21
  const C vy = m.jy * inv_rho + C(0.5) * phi * Gy;
  const C vmag = sqrt_<C>(vx * vx + vy * vy);
  const C inv_den = rcp_<C>(md.l0 + sqrt_<C>(md.l0 * md.l0 + md.l1 * vmag));  // Eq. 20
  m.ux = vx * inv_den;
  m.uy = vy * inv_den;
  m.umag = vmag * inv_den;
  const C drag = md.c0 + md.c1 * m.umag;
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
LTNE_HD void collide(const NodeParams<C>& P, const Macro<C>& m, C (&f)[9],
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
  const C rux = rho * ux, ruy = rho * uy;  // m^eq_3, m^eq_5 (Eq. 15)
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
  // s_3 = s_5 = 1: m*_3 = rho ux + rho Fx / 2 = j_x + rho Fx by Eq. 19, so
  // the momentum passes through exactly and only the force is added.
  const C ms3 = m.jx + rFx;
  const C ms4 = m4 - P.s_q * (m4 + rux) - (C(1) - C(0.5) * P.s_q) * rFx;
  const C ms5 = m.jy + rFy;
  const C ms6 = m6 - P.s_q * (m6 + ruy) - (C(1) - C(0.5) * P.s_q) * rFy;
  const C ms7 = m7 - P.s_nu * (m7 - meq7) + (C(1) - C(0.5) * P.s_nu) * S7;
  const C ms8 = m8 - P.s_nu * (m8 - meq8) + (C(1) - C(0.5) * P.s_nu) * S8;
  // df* = M^-1 m*
  const C r0 = div_small<C>(ms0, C(9), C(1.0 / 9.0));
  const C r1 = div_small<C>(ms1, C(36), C(1.0 / 36.0));
  const C r2 = div_small<C>(ms2, C(36), C(1.0 / 36.0));
  const C r3 = div_small<C>(ms3, C(6), C(1.0 / 6.0));
  const C r4 = div_small<C>(ms4, C(12), C(1.0 / 12.0));
  const C r5 = div_small<C>(ms5, C(6), C(1.0 / 6.0));
  const C r6 = div_small<C>(ms6, C(12), C(1.0 / 12.0));
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
  const C Srf = m.Srf, Srs = m.Srs;  // Eq. 42
  {
    const C Tf = P.T0 + m.dTf;
    const C n1 = gf[1] - gf[3], n2 = gf[2] - gf[4];
    const C n3 = C(-4) * gf[0] + ((gf[1] + gf[2]) + (gf[3] + gf[4]));
    const C n4 = (gf[1] - gf[2]) + (gf[3] - gf[4]);
    const C ns0 = m.sgf + Srf;  // = T_f + Sr_f / 2 (Eq. 41)
    C ns1 = n1 - P.zeta_a * (n1 - ux * Tf * ip);
    C ns2 = n2 - P.zeta_a * (n2 - uy * Tf * ip);
    if (P.tcorr) {
      // (I - Q/2) N C~ with C~_i = w~_i T_f (e_i.F)/(phi c_sT^2): only the
      // first-order moments are non-zero, T_f F/phi (sum_i w~_i e_i e_i = c_sT^2).
      const C cw = (C(1) - C(0.5) * P.zeta_a) * Tf * ip;
      ns1 += cw * Fx;
      ns2 += cw * Fy;
    }
    const C ns3 = n3 - P.zeta_e * (n3 - P.c3 * m.dTf) + (C(1) - C(0.5) * P.zeta_e) * P.c3 * Srf;
    const C ns4 = n4 - P.zeta_nu * n4;
    const C t0 = div_small<C>(ns0, C(5), C(0.2)), t1 = ns1 * C(0.5), t2 = ns2 * C(0.5);
    const C t3 = div_small<C>(ns3, C(20), C(0.05)), t4 = ns4 * C(0.25);
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
    const C ns0 = m.sgs + Srs;  // = T_s + Sr_s / 2
    const C ns1 = n1 - P.eta_a * n1;
    const C ns2 = n2 - P.eta_a * n2;
    const C ns3 = n3 - P.eta_e * (n3 - P.c3 * m.dTs) + (C(1) - C(0.5) * P.eta_e) * P.c3 * Srs;
    const C ns4 = n4 - P.eta_nu * n4;
    const C t0 = div_small<C>(ns0, C(5), C(0.2)), t1 = ns1 * C(0.5), t2 = ns2 * C(0.5);
    const C t3 = div_small<C>(ns3, C(20), C(0.05)), t4 = ns4 * C(0.25);
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
LTNE_HD void nee(const NodeParams<C>& P, const Macro<C>& mn, C dTwf, C dTws,
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
// drho = rho - rho0, dTf = T_f - T0, dTs = T_s - T0.
template <typename C>
LTNE_HD void equilibrium(const NodeParams<C>& P, C phi, C drho, C ux, C uy,
                                            C dTf, C dTs, C (&f)[9], C (&gf)[5], C (&gs)[5]) {
  const C ip = C(1) / phi;
  const C rho = P.rho0 + drho;
  const C Tf = P.T0 + dTf;
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
//
// The 16-bit forms round stochastically: a stored value is rounded up with
// probability equal to its distance from the value below, so the rounding
// error has zero mean.  Round-to-nearest would drop every per-step change
// smaller than half a unit in the last place, always in the same direction
// (stagnation), which at large lattices is most of the diffusion.  The random
// bits come from a counter-based stream keyed by (node, step); each value
// takes 16 of them.

// MurmurHash3's 32-bit finaliser (fmix32).
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

// A 32-bit linear congruential stream (Numerical Recipes' multiplier and
// increment) seeded from fmix32(node ^ fmix32(step)); each word is the state
// with its upper half folded onto the lower (x ^ (x >> 16)), so that the low
// bits, whose periods are short in the raw state, mix in the upper ones.
// Three instructions per word; the seed hash decorrelates nodes and steps.
struct RandomBits {
  uint32_t s;
  __device__ __forceinline__ RandomBits(uint32_t node, uint32_t step)
      : s(fmix32(node ^ fmix32(step * 0x9e3779b9u + 0x7f4a7c15u))) {}
  __device__ __forceinline__ uint32_t next() {
    s = s * 1664525u + 1013904223u;
    return s ^ (s >> 16);
  }
};

template <typename S, typename C> struct Codec;
template <> struct Codec<double, double> {
  static constexpr bool kStochastic = false;
  static __device__ __forceinline__ double dec(double v, double) { return v; }
  static __device__ __forceinline__ double enc(double v, double, uint32_t) { return v; }
};
template <> struct Codec<float, float> {
  static constexpr bool kStochastic = false;
  static __device__ __forceinline__ float dec(float v, float) { return v; }
  static __device__ __forceinline__ float enc(float v, float, uint32_t) { return v; }
};
template <> struct Codec<__half, float> {
  static constexpr bool kStochastic = true;
  static __device__ __forceinline__ float dec(__half v, float inv_scale) {
    return __half2float(v) * inv_scale;
  }
  // Two values at once by the paired conversion with random bits
  // (cvt.rs.f16x2.f32).  The deviations are scaled by 2^10 (exact) so that
  // values down to ~6e-8 stay in the normal FP16 range.  Each value gets 13
  // random bits added below its 10 kept fraction bits before truncation
  // (FP32 keeps 23): lo takes bits 0-12 of r and goes to the low half, hi
  // bits 16-28 and the high half; below the normal range the random bits
  // sit under the subnormal ulp.  Fewer random bits would quantise the
  // round-up probability, itself a bias for increments far below an ulp.
  static __device__ __forceinline__ uint32_t enc2(float lo, float hi, float scale, uint32_t r) {
    uint32_t d;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi * scale), "f"(lo * scale), "r"(r));
    return d;
  }
};
template <> struct Codec<__nv_bfloat16, float> {
  static constexpr bool kStochastic = true;
  static __device__ __forceinline__ float dec(__nv_bfloat16 v, float) {
    return __bfloat162float(v);
  }
  // Two values at once (cvt.rs.bf16x2.f32): BF16 is the top half of FP32;
  // 16 random bits are added below the kept ones and the result truncated,
  // lo with bits 0-15 of r (low half), hi with bits 16-31 (high half).
  static __device__ __forceinline__ uint32_t enc2(float lo, float hi, float, uint32_t r) {
    uint32_t d;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
    return d;
  }
};

}  // namespace ltne
