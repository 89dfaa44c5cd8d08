// ltne_adjoint.cuh -- reverse mode (transposed Jacobians) of the per-node
// functions of ltne_node.cuh, written by hand.  Each function recomputes the
// forward intermediates it needs from the same inputs as its forward
// counterpart and propagates adjoints ("_b") from outputs to inputs.
//
// Independent variables of the gradient: the node porosity phi (through the
// medium coefficients of Eq. 7, the exchange coefficients of Eq. 42 and the
// porous equilibria) and hcoef = h_v/(rho c)_f = H alpha_f/L^2 (Eq. 42); the
// Ergun particle diameter is held fixed.  |v| is differentiated as v/|v|,
// taken as zero at v = 0.
#pragma once

#include "ltne_node.cuh"

namespace ltne {

// Adjoints of the porosity-dependent coefficients (fields of Medium).
template <typename C>
struct MediumBar {
  C phi, inv_phi, a, b, inv_1d, c0, c1, l0, l1;
};

// Adjoints of the macroscopic values a collision or wall rebuild consumes.
template <typename C>
struct MacroBar {
  C drho, jx, jy, sgf, sgs, ux, uy, Fx, Fy, dTf, dTs, Srf, Srs, inv_phi;
};

template <typename C>
LTNE_HD void zero(MacroBar<C>& b) {
  b.drho = b.jx = b.jy = b.sgf = b.sgs = b.ux = b.uy = b.Fx = b.Fy = C(0);
  b.dTf = b.dTs = b.Srf = b.Srs = b.inv_phi = C(0);
}

template <typename C>
LTNE_HD void zero(MediumBar<C>& b) {
  b.phi = b.inv_phi = b.a = b.b = b.inv_1d = b.c0 = b.c1 = b.l0 = b.l1 = C(0);
}

// Medium coefficients -> (phi_b, hcoef_b).  Forward: medium_at().
// md: the node's coefficients, medium_at(P, phi).
template <typename C>
LTNE_HD void medium_adjoint(const NodeParams<C>& P, C phi, const Medium<C>& md,
                            const MediumBar<C>& mb, C& phi_b, C& hcoef_b) {
  C pb = mb.phi;
  // l0 = (1 + phi c0 / 2) / 2, l1 = phi c1 / 2
  pb += mb.l0 * C(0.25) * md.c0;
  const C c0_b = mb.c0 + mb.l0 * C(0.25) * phi;
  pb += mb.l1 * C(0.5) * md.c1;
  const C c1_b = mb.c1 + mb.l1 * C(0.5) * phi;
  // inv_1d = 1 / (1 + a/2 + b/2)
  const C t_b = -md.inv_1d * md.inv_1d * mb.inv_1d;
  const C a_b = mb.a + C(0.5) * t_b;
  const C b_b = mb.b + C(0.5) * t_b;
  // a = hcoef / phi, b = hcoef / ((1 - phi) sigma)
  const C om = C(1) - phi;
  hcoef_b += a_b * md.inv_phi + b_b * md.inv_oms;
  C ip_b = mb.inv_phi + a_b * P.hcoef;
  pb += b_b * P.hcoef * md.inv_oms * rcp_<C>(om);
  // c0(phi), c1(phi)
  const C ip = md.inv_phi;
  C dc0 = C(0), dc1 = C(0);
  if (P.kmode == 0) {
    if (P.fmode == 1) dc1 = C(-1.5) * md.c1 * ip;  // c1 ~ phi^(-3/2)
  } else {
    const C ip4 = ip * ip * ip * ip;
    dc0 = -P.erg_a * om * ip4 * (C(2) * phi + C(3) * om);
    if (P.fmode == 1) {
      dc1 = -P.erg_b * ip4 * (phi + C(3) * om);
    } else {
      dc1 = -P.erg_c * ip * ip * rcp_<C>(sqrt_<C>(phi)) * (phi + C(1.5) * om);
    }
  }
  pb += c0_b * dc0 + c1_b * dc1;
  // inv_phi = 1 / phi
  pb += -ip * ip * ip_b;
  phi_b += pb;
}

// Reverse of macros(): adds to the population adjoints and to the medium
// adjoints.
template <typename C>
LTNE_HD void macros_adjoint(const NodeParams<C>& P, const Medium<C>& md, const C (&f)[9],
                            const C (&gf)[5], const C (&gs)[5], const MacroBar<C>& in,
                            C (&f_b)[9], C (&gf_b)[5], C (&gs_b)[5], MediumBar<C>& mdb) {
  const C phi = md.phi;
  // ---- forward recomputation
  const C sgf = (gf[0] + gf[1]) + (gf[2] + gf[3]) + gf[4];
  const C sgs = (gs[0] + gs[1]) + (gs[2] + gs[3]) + gs[4];
  const C cq = C(0.5) * (P.qf - P.qs);
  const C D = ((sgf - sgs) + cq) * md.inv_1d;
  const C Srf = P.qf - md.a * D;
  const C dTf = sgf + C(0.5) * Srf;
  const C Gx = P.ext_ax, Gy = P.gbeta * dTf + P.ext_ay;
  const C drho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
  const C rho = P.rho0 + drho;
  const C jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
  const C jy = (f[2] - f[4]) + (f[5] - f[7]) + (f[6] - f[8]);
  const C ir = rcp_<C>(rho);
  const C vx = jx * ir + C(0.5) * phi * Gx;
  const C vy = jy * ir + C(0.5) * phi * Gy;
  const C vmag = sqrt_<C>(vx * vx + vy * vy);
  const C R = sqrt_<C>(md.l0 * md.l0 + md.l1 * vmag);
  const C id = rcp_<C>(md.l0 + R);
  const C ux = vx * id, uy = vy * id, umag = vmag * id;
  const C drag = md.c0 + md.c1 * umag;

  // ---- reverse
  C phi_b = C(0);
  C ux_b = in.ux, uy_b = in.uy;
  // F = phi (G - drag u)
  phi_b += in.Fx * (Gx - drag * ux) + in.Fy * (Gy - drag * uy);
  C Gy_b = phi * in.Fy;
  const C drag_b = -phi * (in.Fx * ux + in.Fy * uy);
  ux_b += -phi * drag * in.Fx;
  uy_b += -phi * drag * in.Fy;
  // drag = c0 + c1 |u|
  mdb.c0 += drag_b;
  mdb.c1 += drag_b * umag;
  const C umag_b = drag_b * md.c1;
  // u = v / den, |u| = |v| / den
  C vx_b = ux_b * id, vy_b = uy_b * id, vmag_b = umag_b * id;
  const C id_b = ux_b * vx + uy_b * vy + umag_b * vmag;
  const C den_b = -id * id * id_b;
  // den = l0 + R, R = sqrt(l0^2 + l1 |v|)
  mdb.l0 += den_b;
  if (R > C(0)) {
    const C hR = C(0.5) * den_b * rcp_<C>(R);
    mdb.l0 += hR * C(2) * md.l0;
    mdb.l1 += hR * vmag;
    vmag_b += hR * md.l1;
  }
  if (vmag > C(0)) {
    const C ivm = rcp_<C>(vmag);
    vx_b += vmag_b * vx * ivm;
    vy_b += vmag_b * vy * ivm;
  }
  // v = j / rho + phi G / 2
  C jx_b = in.jx + vx_b * ir;
  C jy_b = in.jy + vy_b * ir;
  const C ir_b = vx_b * jx + vy_b * jy;
  phi_b += C(0.5) * (vx_b * Gx + vy_b * Gy);
  Gy_b += C(0.5) * phi * vy_b;
  C drho_b = in.drho - ir * ir * ir_b;
  // Gy = gbeta dTf + ext
  C dTf_b = in.dTf + P.gbeta * Gy_b;
  C dTs_b = in.dTs;
  // dT = sum g + Sr / 2
  C sgf_b = in.sgf + dTf_b, sgs_b = in.sgs + dTs_b;
  const C Srf_b = in.Srf + C(0.5) * dTf_b;
  const C Srs_b = in.Srs + C(0.5) * dTs_b;
  // Srf = qf - a D, Srs = qs + b D
  mdb.a += -D * Srf_b;
  mdb.b += D * Srs_b;
  const C D_b = -md.a * Srf_b + md.b * Srs_b;
  // D = (sgf - sgs + cq) inv_1d
  sgf_b += D_b * md.inv_1d;
  sgs_b -= D_b * md.inv_1d;
  mdb.inv_1d += D_b * ((sgf - sgs) + cq);
  mdb.phi += phi_b;
  mdb.inv_phi += in.inv_phi;
  // sums over populations
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    gf_b[i] += sgf_b;
    gs_b[i] += sgs_b;
  }
  // e_i of Eq. 8: (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1)
  f_b[0] += drho_b;
  f_b[1] += drho_b + jx_b;
  f_b[2] += drho_b + jy_b;
  f_b[3] += drho_b - jx_b;
  f_b[4] += drho_b - jy_b;
  f_b[5] += drho_b + jx_b + jy_b;
  f_b[6] += drho_b - jx_b + jy_b;
  f_b[7] += drho_b - jx_b - jy_b;
  f_b[8] += drho_b + jx_b - jy_b;
}

// Reverse of collide(): given the adjoints of the 19 post-collision values
// (fo_b, gfo_b, gso_b), adds the adjoints of the 19 pre-collision values
// and of the medium coefficients.  (f, gf, gs) are the pre-collision values.
template <typename C>
LTNE_HD void collide_adjoint(const NodeParams<C>& P, const Medium<C>& md, const C (&f)[9],
                             const C (&gf)[5], const C (&gs)[5], const C (&fo_b)[9],
                             const C (&gfo_b)[5], const C (&gso_b)[5], C (&f_b)[9],
                             C (&gf_b)[5], C (&gs_b)[5], MediumBar<C>& mdb) {
  Macro<C> m;
  macros<C>(P, md, f, gf, gs, m);
  const C rho = m.rho, ux = m.ux, uy = m.uy, Fx = m.Fx, Fy = m.Fy, ip = m.inv_phi;
  MacroBar<C> mb;
  zero(mb);

  // ---- flow.  ms_b = D^-1 M fo_b (transpose of df* = M^T D^-1 m*).
  const C* A = fo_b;
  const C sa = (A[1] + A[2]) + (A[3] + A[4]);
  const C sd = (A[5] + A[6]) + (A[7] + A[8]);
  const C ax = (A[5] - A[6]) + (A[8] - A[7]);
  const C ay = (A[5] - A[7]) + (A[6] - A[8]);
  // divisions by the small integers of D as in the forward collision
  const C msb0 = div_small<C>(A[0] + sa + sd, C(9), C(1.0 / 9.0));
  const C msb1 = div_small<C>(C(-4) * A[0] - sa + C(2) * sd, C(36), C(1.0 / 36.0));
  const C msb2 = div_small<C>(C(4) * A[0] - C(2) * sa + sd, C(36), C(1.0 / 36.0));
  const C msb3 = div_small<C>((A[1] - A[3]) + ax, C(6), C(1.0 / 6.0));
  const C msb4 = div_small<C>(C(-2) * (A[1] - A[3]) + ax, C(12), C(1.0 / 12.0));
  const C msb5 = div_small<C>((A[2] - A[4]) + ay, C(6), C(1.0 / 6.0));
  const C msb6 = div_small<C>(C(-2) * (A[2] - A[4]) + ay, C(12), C(1.0 / 12.0));
  const C msb7 = ((A[1] - A[2]) + (A[3] - A[4])) * C(0.25);
  const C msb8 = ((A[5] - A[6]) + (A[7] - A[8])) * C(0.25);

  mb.drho += msb0;
  const C m1_b = (C(1) - P.s_e) * msb1;
  const C meq1_b = P.s_e * msb1;
  C S1_b = (C(1) - C(0.5) * P.s_e) * msb1;
  const C m2_b = (C(1) - P.s_eps) * msb2;
  const C meq2_b = P.s_eps * msb2;
  S1_b -= (C(1) - C(0.5) * P.s_eps) * msb2;
  mb.jx += msb3;
  C rFx_b = msb3;
  const C m4_b = (C(1) - P.s_q) * msb4;
  const C rux_b = -P.s_q * msb4;
  rFx_b -= (C(1) - C(0.5) * P.s_q) * msb4;
  mb.jy += msb5;
  C rFy_b = msb5;
  const C m6_b = (C(1) - P.s_q) * msb6;
  const C ruy_b = -P.s_q * msb6;
  rFy_b -= (C(1) - C(0.5) * P.s_q) * msb6;
  const C m7_b = (C(1) - P.s_nu) * msb7;
  const C meq7_b = P.s_nu * msb7;
  const C S7_b = (C(1) - C(0.5) * P.s_nu) * msb7;
  const C m8_b = (C(1) - P.s_nu) * msb8;
  const C meq8_b = P.s_nu * msb8;
  const C S8_b = (C(1) - C(0.5) * P.s_nu) * msb8;

  // equilibrium and forcing moments -> macroscopic values
  mb.drho += C(-2) * meq1_b + meq2_b;
  const C ru2_b = meq1_b - meq2_b;
  const C u2 = ux * ux + uy * uy;
  const C uF = ux * Fx + uy * Fy;
  const C uFm = ux * Fx - uy * Fy;
  const C uFx = ux * Fy + uy * Fx;
  const C rho_b = C(3) * u2 * ip * ru2_b + ux * rux_b + uy * ruy_b +
                  (ux * ux - uy * uy) * ip * meq7_b + ux * uy * ip * meq8_b + Fx * rFx_b +
                  Fy * rFy_b + C(6) * uF * ip * S1_b + C(2) * uFm * ip * S7_b +
                  uFx * ip * S8_b;
  const C rip = rho * ip;
  mb.ux += C(6) * rip * ux * ru2_b + rho * rux_b + C(2) * rip * ux * meq7_b + rip * uy * meq8_b +
           C(6) * rip * Fx * S1_b + C(2) * rip * Fx * S7_b + rip * Fy * S8_b;
  mb.uy += C(6) * rip * uy * ru2_b + rho * ruy_b - C(2) * rip * uy * meq7_b + rip * ux * meq8_b +
           C(6) * rip * Fy * S1_b - C(2) * rip * Fy * S7_b + rip * Fx * S8_b;
  mb.Fx += rho * rFx_b + C(6) * rip * ux * S1_b + C(2) * rip * ux * S7_b + rip * uy * S8_b;
  mb.Fy += rho * rFy_b + C(6) * rip * uy * S1_b - C(2) * rip * uy * S7_b + rip * ux * S8_b;
  mb.inv_phi += rho * (C(3) * u2 * ru2_b + (ux * ux - uy * uy) * meq7_b + ux * uy * meq8_b +
                       C(6) * uF * S1_b + C(2) * uFm * S7_b + uFx * S8_b);
  mb.drho += rho_b;
  // moment rows of M f (rows 1, 2, 4, 6, 7, 8 used directly): f_b += M^T m_b
  f_b[0] += C(-4) * m1_b + C(4) * m2_b;
  f_b[1] += -m1_b - C(2) * m2_b - C(2) * m4_b + m7_b;
  f_b[2] += -m1_b - C(2) * m2_b - C(2) * m6_b - m7_b;
  f_b[3] += -m1_b - C(2) * m2_b + C(2) * m4_b + m7_b;
  f_b[4] += -m1_b - C(2) * m2_b + C(2) * m6_b - m7_b;
  f_b[5] += C(2) * m1_b + m2_b + m4_b + m6_b + m8_b;
  f_b[6] += C(2) * m1_b + m2_b - m4_b + m6_b - m8_b;
  f_b[7] += C(2) * m1_b + m2_b - m4_b - m6_b + m8_b;
  f_b[8] += C(2) * m1_b + m2_b + m4_b - m6_b - m8_b;

  // ---- temperatures.  ns_b = D_N^-1 N go_b.
  {
    const C* B = gfo_b;
    const C nb0 = div_small<C>((B[0] + B[1]) + (B[2] + B[3]) + B[4], C(5), C(0.2));
    const C nb1 = (B[1] - B[3]) * C(0.5);
    const C nb2 = (B[2] - B[4]) * C(0.5);
    const C nb3 = div_small<C>(C(-4) * B[0] + ((B[1] + B[2]) + (B[3] + B[4])), C(20), C(0.05));
    const C nb4 = ((B[1] - B[2]) + (B[3] - B[4])) * C(0.25);
    const C Tf = P.T0 + m.dTf;
    mb.sgf += nb0;
    mb.Srf += nb0;
    const C n1_b = (C(1) - P.zeta_a) * nb1;
    const C n2_b = (C(1) - P.zeta_a) * nb2;
    mb.ux += P.zeta_a * Tf * ip * nb1;
    mb.uy += P.zeta_a * Tf * ip * nb2;
    mb.dTf += P.zeta_a * ip * (ux * nb1 + uy * nb2);
    mb.inv_phi += P.zeta_a * Tf * (ux * nb1 + uy * nb2);
    if (P.tcorr) {  // ns1 += cw Fx, ns2 += cw Fy, cw = (1 - zeta_a/2) T_f / phi
      const C c = C(1) - C(0.5) * P.zeta_a;
      mb.Fx += c * Tf * ip * nb1;
      mb.Fy += c * Tf * ip * nb2;
      mb.dTf += c * ip * (Fx * nb1 + Fy * nb2);
      mb.inv_phi += c * Tf * (Fx * nb1 + Fy * nb2);
    }
    const C n3_b = (C(1) - P.zeta_e) * nb3;
    mb.dTf += P.zeta_e * P.c3 * nb3;
    mb.Srf += (C(1) - C(0.5) * P.zeta_e) * P.c3 * nb3;
    const C n4_b = (C(1) - P.zeta_nu) * nb4;
    gf_b[0] += C(-4) * n3_b;
    gf_b[1] += n1_b + n3_b + n4_b;
    gf_b[2] += n2_b + n3_b - n4_b;
    gf_b[3] += -n1_b + n3_b + n4_b;
    gf_b[4] += -n2_b + n3_b - n4_b;
  }
  {
    const C* B = gso_b;
    const C nb0 = div_small<C>((B[0] + B[1]) + (B[2] + B[3]) + B[4], C(5), C(0.2));
    const C nb1 = (B[1] - B[3]) * C(0.5);
    const C nb2 = (B[2] - B[4]) * C(0.5);
    const C nb3 = div_small<C>(C(-4) * B[0] + ((B[1] + B[2]) + (B[3] + B[4])), C(20), C(0.05));
    const C nb4 = ((B[1] - B[2]) + (B[3] - B[4])) * C(0.25);
    mb.sgs += nb0;
    mb.Srs += nb0;
    const C n1_b = (C(1) - P.eta_a) * nb1;
    const C n2_b = (C(1) - P.eta_a) * nb2;
    const C n3_b = (C(1) - P.eta_e) * nb3;
    mb.dTs += P.eta_e * P.c3 * nb3;
    mb.Srs += (C(1) - C(0.5) * P.eta_e) * P.c3 * nb3;
    const C n4_b = (C(1) - P.eta_nu) * nb4;
    gs_b[0] += C(-4) * n3_b;
    gs_b[1] += n1_b + n3_b + n4_b;
    gs_b[2] += n2_b + n3_b - n4_b;
    gs_b[3] += -n1_b + n3_b + n4_b;
    gs_b[4] += -n2_b + n3_b - n4_b;
  }
  macros_adjoint<C>(P, md, f, gf, gs, mb, f_b, gf_b, gs_b, mdb);
}

// Reverse of nee(): (f, gf, gs) are the interior neighbour's post-stream
// values, (lf, lgf, lgs) the adjoints of the wall node's rebuilt values;
// adds to the neighbour's adjoints and medium adjoints.  isothermal: the
// wall temperature is imposed (else it is the neighbour's own, and those
// terms vanish identically).
template <typename C>
LTNE_HD void nee_adjoint(const NodeParams<C>& P, const Medium<C>& md, const C (&f)[9],
                         const C (&gf)[5], const C (&gs)[5], bool isothermal,
                         const C (&lf)[9], const C (&lgf)[5], const C (&lgs)[5], C (&f_b)[9],
                         C (&gf_b)[5], C (&gs_b)[5], MediumBar<C>& mdb) {
  Macro<C> m;
  macros<C>(P, md, f, gf, gs, m);
  const C ux = m.ux, uy = m.uy, ip = m.inv_phi, rho = m.rho;
  MacroBar<C> mb;
  zero(mb);
  const C u2 = ux * ux + uy * uy;
  // f_b = f_n - w_i rho P_i,  P_i = 3 e.u + 4.5 (e.u)^2 / phi - 1.5 u^2 / phi
  const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  const C w[9] = {C(4.0 / 9.0), C(1.0 / 9.0), C(1.0 / 9.0), C(1.0 / 9.0), C(1.0 / 9.0),
                  C(1.0 / 36.0), C(1.0 / 36.0), C(1.0 / 36.0), C(1.0 / 36.0)};
  C rho_b = C(0);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    f_b[i] += lf[i];
    const C eu = C(ex[i]) * ux + C(ey[i]) * uy;
    const C Pi = C(3) * eu + C(4.5) * eu * eu * ip - C(1.5) * u2 * ip;
    rho_b -= w[i] * Pi * lf[i];
    const C P_b = -w[i] * rho * lf[i];
    const C deu = C(3) + C(9) * eu * ip;
    mb.ux += P_b * (deu * C(ex[i]) - C(3) * ux * ip);
    mb.uy += P_b * (deu * C(ey[i]) - C(3) * uy * ip);
    mb.inv_phi += P_b * (C(4.5) * eu * eu - C(1.5) * u2);
  }
  mb.drho += rho_b;
  // g_f: + w~ (T_w - T_f,n) - (e_i.u) T_f,n / (2 phi)
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    gf_b[i] += lgf[i];
    gs_b[i] += lgs[i];
  }
  if (isothermal) {
    mb.dTf -= P.wt0 * lgf[0] + P.wt1 * ((lgf[1] + lgf[2]) + (lgf[3] + lgf[4]));
    mb.dTs -= P.wt0 * lgs[0] + P.wt1 * ((lgs[1] + lgs[2]) + (lgs[3] + lgs[4]));
  }
  const C hx_b = -lgf[1] + lgf[3], hy_b = -lgf[2] + lgf[4];
  const C Tf = P.T0 + m.dTf;
  mb.ux += C(0.5) * Tf * ip * hx_b;
  mb.uy += C(0.5) * Tf * ip * hy_b;
  mb.dTf += C(0.5) * ip * (ux * hx_b + uy * hy_b);
  mb.inv_phi += C(0.5) * Tf * (ux * hx_b + uy * hy_b);
  macros_adjoint<C>(P, md, f, gf, gs, mb, f_b, gf_b, gs_b, mdb);
}

}  // namespace ltne
