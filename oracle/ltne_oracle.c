/*
 * ltne_oracle.c -- plain FP64 CPU oracle for the three-distribution MRT
 * lattice Boltzmann time step of Liu & He (arXiv:1608.04118): a D2Q9
 * density distribution for generalized non-Darcy flow (Sec. 3.1) and two
 * D2Q5 temperature distributions for the fluid and solid phases under local
 * thermal non-equilibrium (Sec. 3.2).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library; the product path never
 * calls it.
 *
 * Shape, chosen to be checkable by eye against the paper rather than fast:
 *   - populations stored node-major (AoS): f[node*9 + i], g[node*5 + i];
 *   - moments by literal matrix-vector products with M (Eq. 13) and N
 *     (Eq. 36); M^-1 and N^-1 are formed numerically by Gauss-Jordan;
 *   - the forcing moments S~ are M times the velocity-space forcing S_i
 *     (Eq. 12), never a closed form;
 *   - push streaming into a second buffer (Eqs. 11, 34, 35);
 *   - one node loop per phase: collide, stream, then the wall rebuild.
 *
 * The same source is compiled twice: once with real_t = double (prefix
 * orc_) and once with real_t = double complex (prefix orc_cs_) so that the
 * complex-step derivative Im J(phi + i h e_k) / h gives exact gradients for
 * the adjoint checks.  |v| is written as sqrt(vx^2 + vy^2) so that it stays
 * analytic under the complex perturbation.
 *
 * State convention: the state S_n is the set of pre-collision populations
 * after streaming and the wall rebuild.  "Fields after n steps" are the
 * macroscopic values of S_n.  S_0 is the equilibrium of the initial fields.
 *
 * Readings of points where the paper is silent or garbled (all used below):
 *   R1  Eq. 16 is garbled in the source text; S~ is taken as M S with the
 *       porous Guo forcing S_i = w_i rho [e_i.F/cs^2 + ((e_i.u)(e_i.F)
 *       - cs^2 u.F)/(phi cs^4)], whose moments are 0, rho F and
 *       rho (uF + Fu)/phi.
 *   R2  gravity points along -y, so G = (0, g beta (T_f - T_0)).
 *   R3  the velocity scale is u_c = Ma c_s = sqrt(g beta dT L), L = ny - 1,
 *       nu_f = u_c L sqrt(Pr/Ra); Ma defaults to 0.1.
 *   R4  the non-equilibrium extrapolation walls ([56] in the paper, not
 *       defined there) overwrite every population of a wall node after
 *       streaming: equilibrium at the wall values plus the non-equilibrium
 *       part of the interior neighbour; corners belong to the isothermal
 *       columns and use the diagonal neighbour; on adiabatic rows the wall
 *       temperature is the neighbour's, phase by phase; u_wall = 0.
 *   R5  H is the constant H_v = h_v L^2 / k_f, so h_v/(rho c)_f = H alpha_f/L^2.
 *   R6  with the local correlation of Eq. 52 (hv_local), h_v/(rho c)_f =
 *       H_p alpha_f / D_p^2 with H_p = 0.376 Re^0.644 Pr^0.37 and
 *       Re = u_m D_p / nu_f, D_p = 0.0135 L; u_m, left undefined by the
 *       paper, is the node's |u| in the previous state (the initial field's
 *       |u| for S_0), so the temperature solve that precedes the velocity
 *       solve of a step stays explicit.
 */
#include <math.h>
#include <complex.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifdef ORC_COMPLEX
typedef double complex real_t;
#define ORC(name) orc_cs_##name
#define RSQRT(x) csqrt(x)
#define RE(x) creal(x)
#define IM(x) cimag(x)
#else
typedef double real_t;
#define ORC(name) orc_##name
#define RSQRT(x) sqrt(x)
#define RE(x) (x)
#define IM(x) (0.0)
#endif

/* Boundary modes (test-only modes besides the cavity of Sec. 4). */
#define ORC_BC_CAVITY 0
#define ORC_BC_PERIODIC 1
#define ORC_BC_CHANNEL 2

/* Problem statement in the paper's dimensionless groups (Sec. 2, Sec. 4). */
typedef struct orc_params {
  int32_t nx, ny;
  int32_t bc;
  int32_t ergun_K;      /* 0: K = Da L^2 everywhere; 1: Ergun K (Eq. 7)   */
  double Ra, Pr, Da, porosity, H, gamma_sf, sigma, J_e;
  double T_hot, T_cold, T_ref, Ma, F_phi, d_p, qf, qs;
  double s_e, s_eps, s_q, zeta_e, zeta_nu, eta_e, eta_nu, varpi;
  double ext_ax, ext_ay, nu_override;
  int32_t hv_local;     /* 1: h_v per node from Eq. 52 (reading R6 below)    */
  int32_t thermal_correction; /* 1: add the correction term of Sec. 3.2       */
  double Dp_over_L;     /* D_p / L of Eq. 52                                */
  double L_ref;         /* > 0: characteristic length L (else ny - 1); lets a
                           window of a larger cavity use that cavity's L  */
} orc_params;

/* Lattice data built once from the paper's definitions. */
typedef struct orc_lattice {
  int ex[9], ey[9];
  double w[9];
  double M[9][9], Minv[9][9];
  double N[5][5], Ninv[5][5];
} orc_lattice;

typedef struct orc_state {
  orc_params p;
  orc_lattice lat;
  int nn;
  double L, cs2, csT2, nu_f, nu_e, alpha_f, alpha_s, gbeta, d_ergun;
  double s[9], Qf[5], Qs[5];  /* relaxation matrices Eq. 17, 39, 40 (diagonals) */
  double wt[5];               /* thermal weights w~ (Sec. 3.2)                  */
  real_t H;
  real_t *phi, *K, *Fphi;     /* per node */
  real_t *hv;                 /* per node h_v / (rho c)_f                       */
  double *um, *um_next;       /* per node |u| of the previous state (Eq. 52)    */
  real_t *f, *gf, *gs;
  real_t *fn, *gfn, *gsn;
  long step;
} orc_state;

/* ---------------------------------------------------------------------- */
/* Lattice construction.                                                   */

/* Gauss-Jordan inverse of an n x n matrix with partial pivoting. */
static void invert(int n, const double* A, double* Ainv) {
  double a[9][18];
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < 2 * n; ++c)
      a[r][c] = (c < n) ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
    if (piv != col)
      for (int c = 0; c < 2 * n; ++c) {
        double t = a[col][c];
        a[col][c] = a[piv][c];
        a[piv][c] = t;
      }
    double d = a[col][col];
    for (int c = 0; c < 2 * n; ++c) a[col][c] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double m = a[r][col];
      if (m != 0.0)
        for (int c = 0; c < 2 * n; ++c) a[r][c] -= m * a[col][c];
    }
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) Ainv[r * n + c] = a[r][n + c];
}

static void build_lattice(orc_lattice* lat) {
  /* Eq. 8: i = 0 rest; i = 1..4 axis directions at angle (i-1) pi/2;
     i = 5..8 diagonals at angle (2i-9) pi/4 with length sqrt(2) (c = 1). */
  const double pi = 3.14159265358979323846;
  lat->ex[0] = lat->ey[0] = 0;
  for (int i = 1; i <= 4; ++i) {
    lat->ex[i] = (int)lround(cos((i - 1) * pi / 2));
    lat->ey[i] = (int)lround(sin((i - 1) * pi / 2));
  }
  for (int i = 5; i <= 8; ++i) {
    lat->ex[i] = (int)lround(sqrt(2.0) * cos((2 * i - 9) * pi / 4));
    lat->ey[i] = (int)lround(sqrt(2.0) * sin((2 * i - 9) * pi / 4));
  }
  /* Weights below Eq. 24. */
  lat->w[0] = 4.0 / 9.0;
  for (int i = 1; i <= 4; ++i) lat->w[i] = 1.0 / 9.0;
  for (int i = 5; i <= 8; ++i) lat->w[i] = 1.0 / 36.0;
  /* Eq. 13, as printed. */
  static const double M13[9][9] = {
      {1, 1, 1, 1, 1, 1, 1, 1, 1},
      {-4, -1, -1, -1, -1, 2, 2, 2, 2},
      {4, -2, -2, -2, -2, 1, 1, 1, 1},
      {0, 1, 0, -1, 0, 1, -1, -1, 1},
      {0, -2, 0, 2, 0, 1, -1, -1, 1},
      {0, 0, 1, 0, -1, 1, 1, -1, -1},
      {0, 0, -2, 0, 2, 1, 1, -1, -1},
      {0, 1, -1, 1, -1, 0, 0, 0, 0},
      {0, 0, 0, 0, 0, 1, -1, 1, -1}};
  /* Eq. 36, as printed. */
  static const double N36[5][5] = {
      {1, 1, 1, 1, 1},
      {0, 1, 0, -1, 0},
      {0, 0, 1, 0, -1},
      {-4, 1, 1, 1, 1},
      {0, 1, -1, 1, -1}};
  memcpy(lat->M, M13, sizeof(M13));
  memcpy(lat->N, N36, sizeof(N36));
  invert(9, &lat->M[0][0], &lat->Minv[0][0]);
  invert(5, &lat->N[0][0], &lat->Ninv[0][0]);
}

/* ---------------------------------------------------------------------- */
/* Parameter mapping: dimensionless groups (Sec. 2) to lattice units.      */

static void derive(orc_state* st, const double* phi_in) {
  const orc_params* p = &st->p;
  st->L = p->L_ref > 0 ? p->L_ref : (double)(p->ny - 1);
  st->cs2 = 1.0 / 3.0;                 /* c_s = c / sqrt(3), below Eq. 23 */
  st->csT2 = p->varpi / 2.0;           /* c_sT^2 = varpi c^2 / 2, Eq. 49   */
  double uc = p->Ma * sqrt(st->cs2);   /* reading R3 */
  double dT = p->T_hot - p->T_cold;
  st->gbeta = (p->Ra > 0 && dT != 0) ? uc * uc / (dT * st->L) : 0.0;
  if (p->nu_override > 0)
    st->nu_f = p->nu_override;
  else
    st->nu_f = uc * st->L * sqrt(p->Pr / p->Ra); /* Ra = g b dT L^3/(nu a) */
  st->alpha_f = st->nu_f / p->Pr;                /* Pr = nu_f / alpha_f    */
  st->nu_e = p->J_e * st->nu_f;                  /* J_e = nu_e / nu_f      */
  /* gamma_sf = k_s/k_f and sigma = (rho c)_s/(rho c)_f, so
     alpha_s / alpha_f = gamma_sf / sigma. */
  st->alpha_s = p->gamma_sf / p->sigma * st->alpha_f;
  double s_nu = 1.0 / (st->nu_e / st->cs2 + 0.5);        /* Eq. 23 */
  double zeta_a = 1.0 / (st->alpha_f / st->csT2 + 0.5);  /* Eq. 49 */
  double eta_a = 1.0 / (st->alpha_s / st->csT2 + 0.5);   /* Eq. 49 */
  /* Eq. 17 */
  double s[9] = {1, p->s_e, p->s_eps, 1, p->s_q, 1, p->s_q, s_nu, s_nu};
  memcpy(st->s, s, sizeof(s));
  /* Eqs. 39-40 */
  double Qf[5] = {1, zeta_a, zeta_a, p->zeta_e, p->zeta_nu};
  double Qs[5] = {1, eta_a, eta_a, p->eta_e, p->eta_nu};
  memcpy(st->Qf, Qf, sizeof(Qf));
  memcpy(st->Qs, Qs, sizeof(Qs));
  /* Thermal weights (below Eq. 31). */
  st->wt[0] = 1.0 - p->varpi;
  for (int i = 1; i < 5; ++i) st->wt[i] = p->varpi / 4.0;
  st->H = p->H;

  for (int n = 0; n < st->nn; ++n) st->phi[n] = phi_in ? phi_in[n] : p->porosity;
  /* Ergun particle diameter: fixed so that the mean of K / L^2 over the
     nodes equals Da (computed from the real parts; held fixed under
     complex perturbation). */
  st->d_ergun = 0.0;
  if (p->ergun_K) {
    if (p->d_p > 0) {
      st->d_ergun = p->d_p;
    } else {
      double acc = 0.0;
      for (int n = 0; n < st->nn; ++n) {
        double ph = RE(st->phi[n]);
        acc += ph * ph * ph / ((1 - ph) * (1 - ph));
      }
      acc /= st->nn;
      st->d_ergun = st->L * sqrt(150.0 * p->Da / acc);
    }
  }
}

/* Per-node permeability and Forchheimer coefficient, Eq. 7. */
static void node_medium(orc_state* st, int n) {
  const orc_params* p = &st->p;
  real_t ph = st->phi[n];
  if (p->ergun_K)
    st->K[n] = ph * ph * ph * st->d_ergun * st->d_ergun / (150.0 * (1 - ph) * (1 - ph));
  else
    st->K[n] = p->Da * st->L * st->L; /* Da = K / L^2 */
  if (p->F_phi >= 0)
    st->Fphi[n] = p->F_phi;
  else
    st->Fphi[n] = 1.75 / RSQRT(150.0 * ph * ph * ph);
}

/* ---------------------------------------------------------------------- */
/* Per-node physics.                                                       */

typedef struct node_macro {
  real_t rho, ux, uy, Tf, Ts, Gx, Gy, Fx, Fy, a, b;
} node_macro;

/* h_v / (rho c)_f at a node whose previous |u| is um (readings R5, R6). */
static real_t hv_of(const orc_state* st, double um) {
  const orc_params* p = &st->p;
  if (!p->hv_local) return st->H * st->alpha_f / (st->L * st->L);
  double Dp = p->Dp_over_L * st->L;
  double Re = um * Dp / st->nu_f;                               /* Eq. 52 */
  double Hp = 0.376 * pow(Re, 0.644) * pow(p->Pr, 0.37);
  return Hp * st->alpha_f / (Dp * Dp);
}

/* Interphase coefficients of Eq. 42: a = h_v/(phi (rho c)_f),
   b = h_v/((1-phi)(rho c)_s), with the node's h_v. */
static void exchange_coeffs(const orc_state* st, int n, real_t phi, real_t* a, real_t* b) {
  real_t hv_f = st->hv[n]; /* h_v / (rho c)_f */
  *a = hv_f / phi;
  *b = hv_f / ((1 - phi) * st->p.sigma);
}

/* Macroscopic values of a node from its pre-collision populations:
   the coupled temperature solve (Eqs. 43-46), buoyancy (Eq. 6, reading R2),
   density (Eq. 18), the explicit velocity (Eqs. 20-22) and the total force
   (Eq. 5). */
static void node_macros(const orc_state* st, int n, const real_t* f, const real_t* gf,
                        const real_t* gs, node_macro* m) {
  const orc_params* p = &st->p;
  const orc_lattice* lat = &st->lat;
  real_t phi = st->phi[n], K = st->K[n], Fphi = st->Fphi[n];
  exchange_coeffs(st, n, phi, &m->a, &m->b);
  real_t d0 = 0.5 * m->a, d1 = 0.5 * m->b; /* Eq. 46, dt = 1 */
  real_t sum_gf = 0, sum_gs = 0;
  for (int i = 0; i < 5; ++i) {
    sum_gf += gf[i];
    sum_gs += gs[i];
  }
  real_t Af = sum_gf + 0.5 * p->qf, As = sum_gs + 0.5 * p->qs;
  m->Tf = ((1 + d1) * Af + d0 * As) / (1 + d0 + d1); /* Eq. 43 */
  m->Ts = (d1 * Af + (1 + d0) * As) / (1 + d0 + d1); /* Eq. 44 */
  m->Gx = p->ext_ax;
  m->Gy = st->gbeta * (m->Tf - p->T_ref) + p->ext_ay;
  real_t rho = 0, jx = 0, jy = 0;
  for (int i = 0; i < 9; ++i) {
    rho += f[i];
    jx += lat->ex[i] * f[i];
    jy += lat->ey[i] * f[i];
  }
  m->rho = rho;
  real_t vx = jx / rho + 0.5 * phi * m->Gx; /* Eq. 21 */
  real_t vy = jy / rho + 0.5 * phi * m->Gy;
  real_t l0 = 0.5 * (1 + phi * 0.5 * st->nu_f / K); /* Eq. 22 */
  real_t l1 = phi * 0.5 * Fphi / RSQRT(K);
  real_t vmag = RSQRT(vx * vx + vy * vy);
  real_t den = l0 + RSQRT(l0 * l0 + l1 * vmag); /* Eq. 20 */
  m->ux = vx / den;
  m->uy = vy / den;
  real_t umag = RSQRT(m->ux * m->ux + m->uy * m->uy);
  /* Eq. 5 */
  m->Fx = -phi * st->nu_f / K * m->ux - phi * Fphi / RSQRT(K) * umag * m->ux + phi * m->Gx;
  m->Fy = -phi * st->nu_f / K * m->uy - phi * Fphi / RSQRT(K) * umag * m->uy + phi * m->Gy;
}

/* Eq. 24 */
static void feq(const orc_state* st, real_t rho, real_t ux, real_t uy, real_t phi, real_t out[9]) {
  const orc_lattice* lat = &st->lat;
  double cs2 = st->cs2;
  for (int i = 0; i < 9; ++i) {
    real_t eu = lat->ex[i] * ux + lat->ey[i] * uy;
    out[i] = lat->w[i] * rho *
             (1 + eu / cs2 + eu * eu / (2 * phi * cs2 * cs2) - (ux * ux + uy * uy) / (2 * phi * cs2));
  }
}

/* Eq. 50 */
static void gfeq(const orc_state* st, real_t T, real_t ux, real_t uy, real_t phi, real_t out[5]) {
  const orc_lattice* lat = &st->lat;
  out[0] = (1 - st->p.varpi) * T;
  for (int i = 1; i < 5; ++i)
    out[i] = 0.25 * st->p.varpi * T + 0.5 * (lat->ex[i] * ux + lat->ey[i] * uy) * T / phi;
}

/* Eq. 51 */
static void gseq(const orc_state* st, real_t T, real_t out[5]) {
  for (int i = 0; i < 5; ++i) out[i] = st->wt[i] * T;
}

/* Eq. 15 */
static void meq_moments(real_t rho, real_t ux, real_t uy, real_t phi, real_t out[9]) {
  real_t u2 = ux * ux + uy * uy;
  out[0] = rho;
  out[1] = -2 * rho + 3 * rho * u2 / phi;
  out[2] = rho - 3 * rho * u2 / phi;
  out[3] = rho * ux;
  out[4] = -rho * ux;
  out[5] = rho * uy;
  out[6] = -rho * uy;
  out[7] = rho * (ux * ux - uy * uy) / phi;
  out[8] = rho * ux * uy / phi;
}

/* Velocity-space forcing term S_i (reading R1). */
static void forcing_S(const orc_state* st, real_t rho, real_t ux, real_t uy, real_t Fx, real_t Fy,
                      real_t phi, real_t out[9]) {
  const orc_lattice* lat = &st->lat;
  double cs2 = st->cs2;
  for (int i = 0; i < 9; ++i) {
    real_t eF = lat->ex[i] * Fx + lat->ey[i] * Fy;
    real_t eu = lat->ex[i] * ux + lat->ey[i] * uy;
    real_t uF = ux * Fx + uy * Fy;
    out[i] = lat->w[i] * rho * (eF / cs2 + (eu * eF - cs2 * uF) / (phi * cs2 * cs2));
  }
}

static void matvec9(const double A[9][9], const real_t* x, real_t* y) {
  for (int r = 0; r < 9; ++r) {
    real_t acc = 0;
    for (int c = 0; c < 9; ++c) acc += A[r][c] * x[c];
    y[r] = acc;
  }
}

static void matvec5(const double A[5][5], const real_t* x, real_t* y) {
  for (int r = 0; r < 5; ++r) {
    real_t acc = 0;
    for (int c = 0; c < 5; ++c) acc += A[r][c] * x[c];
    y[r] = acc;
  }
}

/* One node's collision: Eq. 10 for f, Eqs. 32-33 for g_f and g_s, with
   the macroscopic values from node_macros. */
static void node_collide(const orc_state* st, int n, const real_t* f, const real_t* gf,
                         const real_t* gs, real_t* fo, real_t* gfo, real_t* gso, node_macro* mo,
                         real_t* Stilde_out, real_t* meq_out) {
  const orc_params* p = &st->p;
  const orc_lattice* lat = &st->lat;
  node_macro m;
  node_macros(st, n, f, gf, gs, &m);
  real_t phi = st->phi[n];

  /* Flow: m = M f, m^eq (Eq. 15), S~ = M S (Eq. 12), Eq. 10, f* = M^-1 m*. */
  real_t mom[9], meq[9], S[9], St[9], ms[9];
  matvec9(lat->M, f, mom);
  meq_moments(m.rho, m.ux, m.uy, phi, meq);
  forcing_S(st, m.rho, m.ux, m.uy, m.Fx, m.Fy, phi, S);
  matvec9(lat->M, S, St);
  for (int k = 0; k < 9; ++k)
    ms[k] = mom[k] - st->s[k] * (mom[k] - meq[k]) + (1 - 0.5 * st->s[k]) * St[k];
  matvec9(lat->Minv, ms, fo);

  /* Temperature sources (Eqs. 29-31, 42). */
  real_t Srf = m.a * (m.Ts - m.Tf) + p->qf;
  real_t Srs = m.b * (m.Tf - m.Ts) + p->qs;
  real_t psit_f[5], psit_s[5], psi_f[5], psi_s[5];
  for (int i = 0; i < 5; ++i) {
    psit_f[i] = st->wt[i] * Srf;
    psit_s[i] = st->wt[i] * Srs;
  }
  matvec5(lat->N, psit_f, psi_f);
  matvec5(lat->N, psit_s, psi_s);
  /* Fluid phase: Eq. 37 equilibrium moments, Eq. 32 collision. */
  real_t nf[5], nfeq[5], nfs[5];
  matvec5(lat->N, gf, nf);
  nfeq[0] = m.Tf;
  nfeq[1] = m.ux * m.Tf / phi;
  nfeq[2] = m.uy * m.Tf / phi;
  nfeq[3] = (-4 + 5 * p->varpi) * m.Tf;
  nfeq[4] = 0;
  for (int k = 0; k < 5; ++k)
    nfs[k] = nf[k] - st->Qf[k] * (nf[k] - nfeq[k]) + (1 - 0.5 * st->Qf[k]) * psi_f[k];
  if (p->thermal_correction) {
    /* Correction term of Sec. 3.2: dt (I - Q/2) C, C = N C~,
       C~_i = w~_i T_f (e_i.F) / (phi c_sT^2). */
    real_t Ct[5], Cm[5];
    for (int i = 0; i < 5; ++i)
      Ct[i] = st->wt[i] * m.Tf * (lat->ex[i] * m.Fx + lat->ey[i] * m.Fy) / (phi * st->csT2);
    matvec5(lat->N, Ct, Cm);
    for (int k = 0; k < 5; ++k) nfs[k] += (1 - 0.5 * st->Qf[k]) * Cm[k];
  }
  matvec5(lat->Ninv, nfs, gfo);
  /* Solid phase: Eq. 38 equilibrium moments, Eq. 33 collision. */
  real_t ns[5], nseq[5], nss[5];
  matvec5(lat->N, gs, ns);
  nseq[0] = m.Ts;
  nseq[1] = 0;
  nseq[2] = 0;
  nseq[3] = (-4 + 5 * p->varpi) * m.Ts;
  nseq[4] = 0;
  for (int k = 0; k < 5; ++k)
    nss[k] = ns[k] - st->Qs[k] * (ns[k] - nseq[k]) + (1 - 0.5 * st->Qs[k]) * psi_s[k];
  matvec5(lat->Ninv, nss, gso);

  if (mo) *mo = m;
  if (Stilde_out)
    for (int k = 0; k < 9; ++k) Stilde_out[k] = St[k];
  if (meq_out)
    for (int k = 0; k < 9; ++k) meq_out[k] = meq[k];
}

/* ---------------------------------------------------------------------- */
/* Whole-lattice phases.                                                    */

static int wrap(int i, int n) { return (i % n + n) % n; }

/* Wall rebuild (reading R4) on the post-stream buffers st->f, st->gf, st->gs. */
static void apply_walls(orc_state* st) {
  const orc_params* p = &st->p;
  int nx = p->nx, ny = p->ny;
  if (p->bc == ORC_BC_PERIODIC) return;
  /* Collect wall nodes with their interior neighbour and wall temperatures.
     The neighbour's values are read before any wall node is written; since
     every neighbour is an interior node, the order does not matter. */
  int nwall = 0;
  int* wb = malloc(sizeof(int) * 2 * (nx + ny));
  int* wn = malloc(sizeof(int) * 2 * (nx + ny));
  int* wkind = malloc(sizeof(int) * 2 * (nx + ny)); /* 0 hot, 1 cold, 2 adiabatic */
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      int on_x = (p->bc == ORC_BC_CAVITY) && (x == 0 || x == nx - 1);
      int on_y = (y == 0 || y == ny - 1);
      if (!on_x && !on_y) continue;
      int xn = x, yn = y, kind = 2;
      if (on_x) {
        xn = (x == 0) ? 1 : nx - 2;
        kind = (x == 0) ? 0 : 1;
        if (on_y) yn = (y == 0) ? 1 : ny - 2; /* corner: diagonal neighbour */
      } else {
        yn = (y == 0) ? 1 : ny - 2;
      }
      wb[nwall] = y * nx + x;
      wn[nwall] = yn * nx + xn;
      wkind[nwall] = kind;
      ++nwall;
    }
  real_t* nf = malloc(sizeof(real_t) * 19 * nwall);
#pragma omp parallel for
  for (int k = 0; k < nwall; ++k) {
    int b = wb[k], n = wn[k];
    node_macro m;
    node_macros(st, n, st->f + 9 * n, st->gf + 5 * n, st->gs + 5 * n, &m);
    real_t fe[9], gfe[5], gse[5];
    feq(st, m.rho, m.ux, m.uy, st->phi[n], fe);
    gfeq(st, m.Tf, m.ux, m.uy, st->phi[n], gfe);
    gseq(st, m.Ts, gse);
    real_t Twf, Tws;
    if (wkind[k] == 0) Twf = Tws = p->T_hot;
    else if (wkind[k] == 1) Twf = Tws = p->T_cold;
    else { Twf = m.Tf; Tws = m.Ts; }
    real_t* o = nf + 19 * k;
    for (int i = 0; i < 9; ++i) o[i] = st->lat.w[i] * m.rho + (st->f[9 * n + i] - fe[i]);
    for (int i = 0; i < 5; ++i) o[9 + i] = st->wt[i] * Twf + (st->gf[5 * n + i] - gfe[i]);
    for (int i = 0; i < 5; ++i) o[14 + i] = st->wt[i] * Tws + (st->gs[5 * n + i] - gse[i]);
    (void)b;
  }
  for (int k = 0; k < nwall; ++k) {
    int b = wb[k];
    for (int i = 0; i < 9; ++i) st->f[9 * b + i] = nf[19 * k + i];
    for (int i = 0; i < 5; ++i) st->gf[5 * b + i] = nf[19 * k + 9 + i];
    for (int i = 0; i < 5; ++i) st->gs[5 * b + i] = nf[19 * k + 14 + i];
  }
  free(nf);
  free(wb);
  free(wn);
  free(wkind);
}

/* ---------------------------------------------------------------------- */
/* Public API.                                                              */

orc_state* ORC(create)(const orc_params* p, const double* phi) {
  if (!p || p->nx < 3 || p->ny < 3) return NULL;
  orc_state* st = calloc(1, sizeof(orc_state));
  st->p = *p;
  st->nn = p->nx * p->ny;
  build_lattice(&st->lat);
  st->phi = malloc(sizeof(real_t) * st->nn);
  st->K = malloc(sizeof(real_t) * st->nn);
  st->Fphi = malloc(sizeof(real_t) * st->nn);
  st->f = calloc((size_t)st->nn * 9, sizeof(real_t));
  st->gf = calloc((size_t)st->nn * 5, sizeof(real_t));
  st->gs = calloc((size_t)st->nn * 5, sizeof(real_t));
  st->fn = calloc((size_t)st->nn * 9, sizeof(real_t));
  st->gfn = calloc((size_t)st->nn * 5, sizeof(real_t));
  st->gsn = calloc((size_t)st->nn * 5, sizeof(real_t));
  st->hv = calloc((size_t)st->nn, sizeof(real_t));
  st->um = calloc((size_t)st->nn, sizeof(double));
  st->um_next = calloc((size_t)st->nn, sizeof(double));
  derive(st, phi);
  for (int n = 0; n < st->nn; ++n) node_medium(st, n);
  return st;
}

void ORC(destroy)(orc_state* st) {
  if (!st) return;
  free(st->phi); free(st->K); free(st->Fphi);
  free(st->f); free(st->gf); free(st->gs);
  free(st->fn); free(st->gfn); free(st->gsn);
  free(st->hv); free(st->um); free(st->um_next);
  free(st);
}

/* S_0: equilibria (Eqs. 24, 50, 51) of the given fields; NULL arrays take
   rho = 1, u = 0, T = T_ref. */
void ORC(init)(orc_state* st, const double* rho, const double* ux, const double* uy,
               const double* Tf, const double* Ts) {
  for (int n = 0; n < st->nn; ++n) {
    real_t r = rho ? rho[n] : 1.0, vx = ux ? ux[n] : 0.0, vy = uy ? uy[n] : 0.0;
    real_t tf = Tf ? Tf[n] : st->p.T_ref, ts = Ts ? Ts[n] : st->p.T_ref;
    st->um[n] = sqrt(RE(vx) * RE(vx) + RE(vy) * RE(vy));
    st->hv[n] = hv_of(st, st->um[n]);
    feq(st, r, vx, vy, st->phi[n], st->f + 9 * n);
    gfeq(st, tf, vx, vy, st->phi[n], st->gf + 5 * n);
    gseq(st, ts, st->gs + 5 * n);
  }
  st->step = 0;
}

/* n time steps: collide every node, push-stream (Eqs. 11, 34, 35), then
   rebuild the walls. */
void ORC(step)(orc_state* st, long nsteps) {
  const orc_params* p = &st->p;
  int nx = p->nx, ny = p->ny;
  int px = (p->bc == ORC_BC_PERIODIC || p->bc == ORC_BC_CHANNEL);
  int py = (p->bc == ORC_BC_PERIODIC);
  for (long t = 0; t < nsteps; ++t) {
#pragma omp parallel for
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        int n = y * nx + x;
        real_t fo[9], gfo[5], gso[5];
        node_macro mo;
        node_collide(st, n, st->f + 9 * n, st->gf + 5 * n, st->gs + 5 * n, fo, gfo, gso, &mo,
                     NULL, NULL);
        st->um_next[n] = sqrt(RE(mo.ux) * RE(mo.ux) + RE(mo.uy) * RE(mo.uy));
        for (int i = 0; i < 9; ++i) {
          int tx = x + st->lat.ex[i], ty = y + st->lat.ey[i];
          if (px) tx = wrap(tx, nx);
          if (py) ty = wrap(ty, ny);
          if (tx < 0 || tx >= nx || ty < 0 || ty >= ny) continue; /* leaves the domain */
          st->fn[9 * (ty * nx + tx) + i] = fo[i];
        }
        for (int i = 0; i < 5; ++i) {
          int tx = x + st->lat.ex[i], ty = y + st->lat.ey[i];
          if (px) tx = wrap(tx, nx);
          if (py) ty = wrap(ty, ny);
          if (tx < 0 || tx >= nx || ty < 0 || ty >= ny) continue;
          st->gfn[5 * (ty * nx + tx) + i] = gfo[i];
          st->gsn[5 * (ty * nx + tx) + i] = gso[i];
        }
      }
    real_t* t1 = st->f; st->f = st->fn; st->fn = t1;
    real_t* t2 = st->gf; st->gf = st->gfn; st->gfn = t2;
    real_t* t3 = st->gs; st->gs = st->gsn; st->gsn = t3;
    if (p->hv_local) {
      /* the new state's temperature solves use |u| of the state just collided */
      double* t4 = st->um; st->um = st->um_next; st->um_next = t4;
      for (int n = 0; n < st->nn; ++n) st->hv[n] = hv_of(st, st->um[n]);
    }
    apply_walls(st);
    ++st->step;
  }
}

long ORC(get_step)(const orc_state* st) { return st->step; }

/* Macroscopic fields of the current state (real parts). */
void ORC(macros)(const orc_state* st, double* rho, double* ux, double* uy, double* Tf, double* Ts) {
#pragma omp parallel for
  for (int n = 0; n < st->nn; ++n) {
    node_macro m;
    node_macros(st, n, st->f + 9 * n, st->gf + 5 * n, st->gs + 5 * n, &m);
    if (rho) rho[n] = RE(m.rho);
    if (ux) ux[n] = RE(m.ux);
    if (uy) uy[n] = RE(m.uy);
    if (Tf) Tf[n] = RE(m.Tf);
    if (Ts) Ts[n] = RE(m.Ts);
  }
}

/* Wall heat fluxes (trapezoid over y of the second-order one-sided
   gradient; the wall column takes the imposed wall temperature), for one
   phase given its temperature field. Nu = (1/dT) * integral q dy. */
static real_t nusselt(const orc_state* st, const real_t* T, int hot) {
  const orc_params* p = &st->p;
  int nx = p->nx, ny = p->ny;
  real_t acc = 0;
  for (int y = 0; y < ny; ++y) {
    real_t q;
    if (hot)
      q = -(-3 * p->T_hot + 4 * T[y * nx + 1] - T[y * nx + 2]) / 2;
    else
      q = -(3 * p->T_cold - 4 * T[y * nx + nx - 2] + T[y * nx + nx - 3]) / 2;
    double wgt = (y == 0 || y == ny - 1) ? 0.5 : 1.0;
    acc += wgt * q;
  }
  return acc / (p->T_hot - p->T_cold);
}

/* Observables of the current state, out[12]:
   0 Nu_f,hot 1 Nu_s,hot 2 Nu_f,cold 3 Nu_s,cold 4 mass 5 energy (from
   populations) 6 max|u| 7 max|T_f - T_s| 8 mean T_f 9 mean T_s
   10 Fo = alpha_f t / L^2  11 number of non-finite macro values. */
void ORC(observables)(const orc_state* st, double* out) {
  int nn = st->nn;
  real_t* Tf = malloc(sizeof(real_t) * nn);
  real_t* Ts = malloc(sizeof(real_t) * nn);
  double mass = 0, energy = 0, maxu = 0, maxdT = 0, mTf = 0, mTs = 0, bad = 0;
  for (int n = 0; n < nn; ++n) {
    node_macro m;
    node_macros(st, n, st->f + 9 * n, st->gf + 5 * n, st->gs + 5 * n, &m);
    Tf[n] = m.Tf;
    Ts[n] = m.Ts;
    mass += RE(m.rho);
    double sgf = 0, sgs = 0;
    for (int i = 0; i < 5; ++i) {
      sgf += RE(st->gf[5 * n + i]);
      sgs += RE(st->gs[5 * n + i]);
    }
    double ph = RE(st->phi[n]);
    energy += ph * sgf + (1 - ph) * st->p.sigma * sgs;
    double um = sqrt(RE(m.ux) * RE(m.ux) + RE(m.uy) * RE(m.uy));
    if (um > maxu) maxu = um;
    double dT = fabs(RE(m.Tf) - RE(m.Ts));
    if (dT > maxdT) maxdT = dT;
    mTf += RE(m.Tf);
    mTs += RE(m.Ts);
    if (!isfinite(RE(m.rho)) || !isfinite(RE(m.ux)) || !isfinite(RE(m.uy)) ||
        !isfinite(RE(m.Tf)) || !isfinite(RE(m.Ts)))
      bad += 1;
  }
  int cav = (st->p.bc == ORC_BC_CAVITY);
  out[0] = cav ? RE(nusselt(st, Tf, 1)) : 0;
  out[1] = cav ? RE(nusselt(st, Ts, 1)) : 0;
  out[2] = cav ? RE(nusselt(st, Tf, 0)) : 0;
  out[3] = cav ? RE(nusselt(st, Ts, 0)) : 0;
  out[4] = mass;
  out[5] = energy;
  out[6] = maxu;
  out[7] = maxdT;
  out[8] = mTf / nn;
  out[9] = mTs / nn;
  out[10] = st->alpha_f * st->step / (st->L * st->L);
  out[11] = bad;
  free(Tf);
  free(Ts);
}

/* Objective of the gradient checks: J = (Nu_f,hot + Nu_s,hot) / 2 of the
   current state, real and imaginary parts. */
void ORC(objective)(const orc_state* st, double* re, double* im) {
  int nn = st->nn;
  real_t* Tf = malloc(sizeof(real_t) * nn);
  real_t* Ts = malloc(sizeof(real_t) * nn);
  for (int n = 0; n < nn; ++n) {
    node_macro m;
    node_macros(st, n, st->f + 9 * n, st->gf + 5 * n, st->gs + 5 * n, &m);
    Tf[n] = m.Tf;
    Ts[n] = m.Ts;
  }
  real_t J = 0.5 * (nusselt(st, Tf, 1) + nusselt(st, Ts, 1));
  *re = RE(J);
  *im = IM(J);
  free(Tf);
  free(Ts);
}

/* Populations of the current state, node-major (AoS) real parts. */
void ORC(get_pops)(const orc_state* st, double* f, double* gf, double* gs) {
  for (long k = 0; k < 9L * st->nn; ++k) f[k] = RE(st->f[k]);
  for (long k = 0; k < 5L * st->nn; ++k) {
    gf[k] = RE(st->gf[k]);
    gs[k] = RE(st->gs[k]);
  }
}

void ORC(set_pops)(orc_state* st, const double* f, const double* gf, const double* gs) {
  for (long k = 0; k < 9L * st->nn; ++k) st->f[k] = f[k];
  for (long k = 0; k < 5L * st->nn; ++k) {
    st->gf[k] = gf[k];
    st->gs[k] = gs[k];
  }
}

#ifdef ORC_COMPLEX
/* Complex-step perturbation: node >= 0 adds i*h to phi at that node (and
   updates its K and F_phi); node == -1 adds i*h to H. Call before init. */
void orc_cs_perturb(orc_state* st, int node, double h) {
  if (node < 0) {
    st->H += I * h;
  } else {
    st->phi[node] += I * h;
    node_medium(st, node);
  }
}
#else
/* Derived lattice parameters, out[16]: L, nu_f, nu_e, alpha_f, alpha_s,
   gbeta, s_nu, zeta_alpha, eta_alpha, d_ergun, csT2, hv/(rho c)_f,
   s_e, s_eps, s_q, cs2. */
void orc_derived(const orc_state* st, double* out) {
  out[0] = st->L; out[1] = st->nu_f; out[2] = st->nu_e; out[3] = st->alpha_f;
  out[4] = st->alpha_s; out[5] = st->gbeta; out[6] = st->s[7]; out[7] = st->Qf[1];
  out[8] = st->Qs[1]; out[9] = st->d_ergun; out[10] = st->csT2;
  out[11] = st->H * st->alpha_f / (st->L * st->L);
  out[12] = st->s[1]; out[13] = st->s[2]; out[14] = st->s[4]; out[15] = st->cs2;
}

/* Per-node medium: K and F_phi at every node. */
void orc_medium(const orc_state* st, double* K, double* Fphi) {
  for (int n = 0; n < st->nn; ++n) {
    K[n] = st->K[n];
    Fphi[n] = st->Fphi[n];
  }
}

/* Lattice tables: e (18 ints as doubles: ex then ey), w[9], M[81],
   Minv[81], N[25], Ninv[25]. */
void orc_lattice_tables(double* e, double* w, double* M, double* Minv, double* N, double* Ninv) {
  orc_lattice lat;
  build_lattice(&lat);
  for (int i = 0; i < 9; ++i) {
    e[i] = lat.ex[i];
    e[9 + i] = lat.ey[i];
    w[i] = lat.w[i];
  }
  memcpy(M, lat.M, sizeof(lat.M));
  memcpy(Minv, lat.Minv, sizeof(lat.Minv));
  memcpy(N, lat.N, sizeof(lat.N));
  memcpy(Ninv, lat.Ninv, sizeof(lat.Ninv));
}

/* One node in isolation (node index n of st supplies phi, K, F_phi):
   collides the given populations; macro[11] = rho, ux, uy, Tf, Ts, Gx, Gy,
   Fx, Fy, a, b; Stilde[9]; meq[9]. */
void orc_node(const orc_state* st, int n, const double* f, const double* gf, const double* gs,
              double* fo, double* gfo, double* gso, double* macro, double* Stilde, double* meq) {
  node_macro m;
  node_collide(st, n, f, gf, gs, fo, gfo, gso, &m, Stilde, meq);
  double v[11] = {m.rho, m.ux, m.uy, m.Tf, m.Ts, m.Gx, m.Gy, m.Fx, m.Fy, m.a, m.b};
  memcpy(macro, v, sizeof(v));
}

/* Equilibria of one node: feq[9] (Eq. 24), gfeq[5] (Eq. 50), gseq[5] (Eq. 51),
   meq[9] (Eq. 15); forcing S[9] (reading R1) for a given force. */
void orc_equilibria(const orc_state* st, double rho, double ux, double uy, double Tf, double Ts,
                    double phi, double Fx, double Fy, double* fe, double* gfe, double* gse,
                    double* me, double* S) {
  feq(st, rho, ux, uy, phi, fe);
  gfeq(st, Tf, ux, uy, phi, gfe);
  gseq(st, Ts, gse);
  meq_moments(rho, ux, uy, phi, me);
  forcing_S(st, rho, ux, uy, Fx, Fy, phi, S);
}

/* Ergun particle diameter that makes the mean of K / L^2 over the n given
   porosities equal Da (Eq. 7 with the mean Darcy number). */
double orc_ergun_diameter(const double* phi, long n, double L, double Da) {
  double acc = 0.0;
  for (long k = 0; k < n; ++k) acc += phi[k] * phi[k] * phi[k] / ((1 - phi[k]) * (1 - phi[k]));
  acc /= n;
  return L * sqrt(150.0 * Da / acc);
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the node loops from now on (n >= 1); for timing only. */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
#endif
