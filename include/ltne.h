/*
 * ltne.h -- C ABI of the GB300 (sm_103a) implementation of the
 * three-distribution MRT lattice Boltzmann time step of Liu & He,
 * "Multiple-relaxation-time lattice Boltzmann model for convection heat
 * transfer in porous media under local thermal non-equilibrium condition"
 * (arXiv:1608.04118).
 *
 * One time step advances, in one fused pass per lattice node,
 *   - the D2Q9 density distribution f of the generalized non-Darcy
 *     (Brinkman-Forchheimer) flow: Sec. 3.1, Eqs. 9-24;
 *   - the D2Q5 fluid-phase and solid-phase temperature distributions g_f,
 *     g_s with the interphase source terms and their (I - Q/2) treatment:
 *     Sec. 3.2, Eqs. 27-51;
 *   - the wall rebuild of the cavity of Sec. 4 (non-equilibrium
 *     extrapolation, which the paper cites but does not define: every
 *     population of a wall node is replaced after streaming by the
 *     equilibrium at the wall values plus the non-equilibrium part of the
 *     interior neighbour; corners use the diagonal neighbour and belong to
 *     the isothermal walls; adiabatic rows take the neighbour's temperature).
 *
 * Conventions shared by every entry point:
 *   - Every call returns an int status (LTNE_OK or an LTNE_ERR_* code) and
 *     never aborts; ltne_error_string() names the code.
 *   - Host arrays are row-major [ny][nx] doubles: x is horizontal (hot wall
 *     at x = 0, cold wall at x = nx-1), y is vertical (gravity along -y).
 *   - The caller owns all memory.  Device memory is one workspace buffer
 *     the caller allocates (e.g. a torch tensor) and binds with
 *     ltne_bind_workspace(); the handle holds only host-side metadata and
 *     the CUDA graphs it builds.  The library allocates no device memory.
 *   - All device work is enqueued on the stream given to ltne_create().
 *     Calls that return host data synchronise that stream.
 *   - A handle is not thread-safe; use one handle per stream.
 */
#ifndef LTNE_H
#define LTNE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum {
  LTNE_OK = 0,
  LTNE_ERR_INVALID_ARG = 1,   /* bad pointer, size or parameter value        */
  LTNE_ERR_UNSTABLE_TAU = 2,  /* a relaxation rate falls outside (0, 2)       */
  LTNE_ERR_CUDA = 3,          /* a CUDA runtime call failed                   */
  LTNE_ERR_NONFINITE = 4,     /* observables found NaN/Inf in the fields      */
  LTNE_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up           */
  LTNE_ERR_STATE = 6,         /* call out of order (e.g. no workspace bound)  */
  LTNE_ERR_WORKSPACE = 7      /* workspace missing, too small or misaligned   */
};

/* Population storage.  Compute is FP64 for LTNE_F64 and FP32 otherwise.
   Every form stores deviations from the rest equilibrium: f_i - w_i rho_0
   and g_i - w~_i T_0 (rho_0 = 1, T_0 = T_ref).  The 16-bit forms round
   stochastically, not to nearest: the FP32 deviation (times 2^10 for FP16,
   unscaled for BF16) gets random bits added below the kept fraction bits
   before truncation (the paired conversion with random bits of sm_100 and
   later), the bits drawn from a counter-based generator seeded by the node
   and the step, so a run is reproducible bit for bit. */
enum { LTNE_F64 = 0, LTNE_F32 = 1, LTNE_F16DEV = 2, LTNE_BF16DEV = 3 };

/* Boundary modes.  CAVITY is the problem of Sec. 4; the other two are test
   boxes: PERIODIC wraps both directions, CHANNEL wraps x and puts no-slip,
   adiabatic walls at y = 0 and y = ny-1. */
enum { LTNE_BC_CAVITY = 0, LTNE_BC_PERIODIC = 1, LTNE_BC_CHANNEL = 2 };

/* Permeability model: DARCY takes K = Da L^2 at every node; ERGUN takes
   Eq. 7, K = phi^3 d^2 / (150 (1-phi)^2), with d = d_p, or (d_p <= 0)
   with d fixed so that the mean of K / L^2 over the nodes equals Da. */
enum { LTNE_K_DARCY = 0, LTNE_K_ERGUN = 1 };

/* Problem statement.  The dimensionless groups follow Sec. 2 of the
   paper (Ra, Pr, Da, J_e, gamma_sf, sigma, H_v); relaxation rates and
   varpi default to the values of Sec. 4.  Lattice mapping (the paper
   leaves the velocity scale open): L = ny - 1, u_c = Ma c_s = sqrt(g beta
   dT L), nu_f = u_c L sqrt(Pr/Ra), alpha_f = nu_f/Pr, nu_e = J_e nu_f,
   alpha_s = (gamma_sf/sigma) alpha_f, s_nu from Eq. 23, zeta_alpha and
   eta_alpha from Eq. 49 with c_sT^2 = varpi/2, and h_v/(rho c)_f =
   H alpha_f / L^2. */
typedef struct ltne_params {
  int32_t nx, ny;          /* nodes including the wall nodes (>= 4 each)     */
  int32_t storage;         /* LTNE_F64 | LTNE_F32 | LTNE_F16DEV | LTNE_BF16DEV */
  int32_t bc;              /* LTNE_BC_*                                      */
  int32_t permeability;    /* LTNE_K_DARCY | LTNE_K_ERGUN                    */
  int32_t porosity_field;  /* 1: a per-node porosity is given to set_fields  */
  double Ra, Pr, Da;       /* Rayleigh, Prandtl, Darcy (mean Da for ERGUN)   */
  double porosity;         /* uniform porosity when porosity_field == 0      */
  double H;                /* H_v = h_v L^2 / k_f                            */
  double gamma_sf, sigma;  /* k_s/k_f, (rho c_p)_s/(rho c_p)_f               */
  double J_e;              /* nu_e / nu_f                                    */
  double T_hot, T_cold;    /* wall temperatures at x = 0 and x = nx-1        */
  double T_ref;            /* Boussinesq T_0 of Eq. 6, also the deviation
                              reference of the thermal populations          */
  double Ma;               /* u_c / c_s (default 0.1)                        */
  double F_phi;            /* < 0: Ergun F_phi = 1.75/sqrt(150 phi^3) (Eq. 7)
                              per node; >= 0: this constant                 */
  double d_p;              /* Ergun particle diameter (lattice units); <= 0:
                              derived from the mean Darcy number            */
  double qf, qs;           /* Q_f''', Q_s''' of Eq. 45 in lattice units      */
  double s_e, s_eps, s_q;  /* Eq. 17                                         */
  double zeta_e, zeta_nu;  /* Eq. 39                                         */
  double eta_e, eta_nu;    /* Eq. 40                                         */
  double varpi;            /* thermal weight parameter (Sec. 3.2), (0, 1)    */
  double ext_ax, ext_ay;   /* extra body acceleration added to G (tests)     */
  double nu_override;      /* > 0: nu_f in lattice units (needed for Ra = 0) */
  int32_t hv_local;        /* 1: h_v per node from the correlation of Eq. 52,
                              H_p = h_v D_p^2 / k_f = 0.376 Re^0.644 Pr^0.37,
                              Re = u_m D_p / nu_f, with u_m the node's |u| in
                              the previous state (the initial field's |u| for
                              the initial state; the paper leaves u_m and its
                              time level open); H is then unused.  Not
                              supported by the batched form or the adjoint. */
  int32_t thermal_correction; /* 1: add the correction term of Sec. 3.2,
                              dt N^-1 (I - Q/2) C with C = N C~ and
                              C~_i = w~_i T_f (e_i.F) / (phi c_sT^2), to the
                              fluid-phase equation (Eq. 27); the paper
                              neglects it (0, default).  Not supported by the
                              batched form. */
  double Dp_over_L;        /* D_p / L of Eq. 52 (Sec. 4: 0.0135)            */
} ltne_params;

/* Observables of the current state, reduced on the device in FP64.
   Nu: (1/dT) * trapezoid over y of q(y) = -(dT/dx) at the wall, with the
   second-order one-sided difference and the wall column at the imposed
   wall temperature (the paper plots but never defines Nu).  residual:
   max over {u, T_f, T_s} of ||X - X_prev|| / ||X|| against the previous
   ltne_observables() call (NaN on the first call).  energy:
   sum[phi T_f + (1-phi) sigma T_s] - sum[phi Q_f + (1-phi) sigma Q_s]/2,
   which equals sum[phi sum g_f + (1-phi) sigma sum g_s] because the
   interphase sources cancel. */
typedef struct ltne_obs {
  double Nu_f_hot, Nu_s_hot, Nu_f_cold, Nu_s_cold;
  double residual;
  double mass;             /* sum of rho                                     */
  double energy;
  double max_u;            /* max |u|                                        */
  double max_dT;           /* max |T_f - T_s|                                */
  double mean_Tf, mean_Ts;
  double Fo;               /* alpha_f t / L^2 (the Fo of Sec. 2, read as a
                              dimensionless time)                            */
  int64_t step;            /* steps taken since set_fields                   */
  int64_t nonfinite;       /* number of nodes with a non-finite field        */
} ltne_obs;

typedef struct ltne_handle ltne_handle;

/* Fill *p with the defaults (Sec. 4 rates, varpi = 2/5, J_e = sigma =
   gamma_sf = 1, Ma = 0.1, T_hot = 1, T_cold = 0, T_ref = 0.5, Ergun F_phi,
   FP32 storage, cavity, Darcy permeability). */
void ltne_default_params(ltne_params* p, int32_t nx, int32_t ny);

/* Validate *p, derive the lattice constants and create a handle bound to
   cuda_stream (a cudaStream_t; NULL = legacy default stream).  Errors:
   INVALID_ARG for sizes < 4, porosity outside (0,1), non-positive Pr,
   sigma, varpi outside (0,1) etc.; UNSTABLE_TAU if any relaxation rate is
   outside (0, 2).  No device memory is touched. */
int ltne_create(const ltne_params* p, void* cuda_stream, ltne_handle** out);

/* Bytes of device workspace the handle needs (populations in two
   buffers, porosity, macroscopic fields, reduction partials). */
size_t ltne_workspace_bytes(const ltne_handle* h);

/* Bind caller-owned device memory (>= ltne_workspace_bytes, 256-byte
   aligned).  The caller keeps it alive until ltne_destroy(). */
int ltne_bind_workspace(ltne_handle* h, void* device_ptr, size_t bytes);

/* Initial state S_0: equilibria of the given fields (Eqs. 24, 50, 51) at
   every node, walls included.  Host arrays of nx*ny doubles, row-major:
   porosity must be non-NULL iff porosity_field was set (values in (0,1));
   rho, ux, uy, T_f, T_s may be NULL (defaults rho = 1, u = 0, T = T_ref).
   Resets the step counter.  The arrays are read before the call returns
   (the device work after them may still be in flight).  INVALID_ARG for a
   porosity outside (0, 1) or a value that is not finite; the handle then
   has no fields (STATE) until a call succeeds. */
int ltne_set_fields(ltne_handle* h, const double* porosity, const double* rho,
                    const double* ux, const double* uy, const double* T_f,
                    const double* T_s);

/* Advance n >= 0 time steps (collision, streaming and walls per step),
   asynchronously on the handle's stream, replaying a cached CUDA graph of
   steps where it can. */
int ltne_step(ltne_handle* h, int64_t n);

/* Reduce the current fields to *out (synchronises the stream).  Returns
   LTNE_ERR_NONFINITE (with *out filled) if any field is NaN or Inf. */
int ltne_observables(ltne_handle* h, ltne_obs* out);

/* Copy the macroscopic fields of the current state to host arrays of
   nx*ny doubles (any pointer may be NULL).  Synchronises the stream. */
int ltne_get_fields(ltne_handle* h, double* rho, double* ux, double* uy, double* T_f,
                    double* T_s);

/* How ltne_set_fields and ltne_get_fields move whole fields between the
   caller's host arrays and the device (no counterpart in the paper).
   LTNE_HOST_IO_STAGED: host threads convert the values (absolute FP64 <->
   deviations in the compute type) through two pinned buffers that are
   copied while the other is converted; any GPU.  LTNE_HOST_IO_DIRECT:
   kernels read and write the caller's arrays themselves and convert on the
   device, for GPUs that reach pageable host memory through the host's page
   tables (GB300 with Grace memory over NVLink-C2C); ltne_set_fields then
   returns only after the arrays were read (the porosity kernel also forms
   the Ergun mean, in the summation order ltne_ergun_diameter takes), and
   ltne_get_fields writes directly only into
   page-locked arrays (pinned or registered; pageable ones are staged: a
   device write to a page the host never touched costs a host-serviced
   fault per page).  LTNE_HOST_IO_AUTO (the default): DIRECT where the
   device supports it, else STAGED.  Both forms give the same bits and the
   same errors.  ltne_set_host_io: INVALID_ARG for an unknown mode or for
   DIRECT on a device without that access.  ltne_get_host_io: the form in
   use (STAGED or DIRECT). */
#define LTNE_HOST_IO_AUTO 0
#define LTNE_HOST_IO_STAGED 1
#define LTNE_HOST_IO_DIRECT 2
int ltne_set_host_io(ltne_handle* h, int32_t mode);
int ltne_get_host_io(ltne_handle* h, int32_t* mode);

/* Checkpoint: size of the state blob, and copies of it to / from host
   memory.  The blob holds the populations, the macroscopic fields, the
   per-node porosity (if any), the previous |u| of the local h_v model (if
   on), the step and the Ergun diameter in use, so a handle created with the
   same parameters and restored from it continues bit for bit as if it had
   never stopped.  Synchronises the stream. */
size_t ltne_state_bytes(const ltne_handle* h);
int ltne_get_state(ltne_handle* h, void* host, size_t bytes);
int ltne_set_state(ltne_handle* h, const void* host, size_t bytes);

/* Number of step-kernel launches issued by this handle so far. */
int64_t ltne_launch_count(const ltne_handle* h);

/* Launch schedule of the step kernel (no counterpart in the paper, which
   prescribes no implementation): blocks of block_x x block_y threads
   (block_x a multiple of 32 in 32..256, block_x * block_y <= 256), each
   thread advancing nodes_per_thread = 1 node or 2 neighbouring nodes of a
   row in paired FP32 arithmetic (FP32, FP16 and BF16 storage only, and
   block_x * block_y <= 128).  The schedule changes no result beyond FP32
   rounding: the arithmetic per node is the same, and for a given
   nodes_per_thread the block shape changes no bit.  Defaults: 32 x 4 with
   two nodes per thread for FP16 / BF16 lattices of 2^20 nodes or more,
   128 x 1 with two for FP32 lattices of 2^22 nodes or more, 64 x 2 with
   one otherwise (and always for FP64).  May be called at any time between
   steps.
   LTNE_ERR_INVALID_ARG for other schedules. */
int ltne_set_schedule(ltne_handle* h, int32_t block_x, int32_t block_y,
                      int32_t nodes_per_thread);

/* Staged tiles (no counterpart in the paper): staged = 1 runs the step as
   the two-node kernel whose persistent blocks stream tiles of
   (2 block_x) x block_y nodes, with a halo of one row and 16 bytes of
   columns, from HBM into shared memory by the tensor memory accelerator,
   several tiles ahead, instead of loading each node's values directly
   (FP32, FP16, BF16 storage with cavity walls only; block shapes 32 x 4,
   64 x 2 or 32 x 2 threads, any other shape runs as 32 x 4).  Results are
   the same bits as the direct two-node schedule.  A staged step whose tile never
   arrives gives up after about a second and makes the next
   ltne_observables return LTNE_ERR_TIMEOUT.  staged = 0 (default) returns
   to the schedule.  LTNE_ERR_INVALID_ARG for other storage or walls. */
int ltne_set_staging(ltne_handle* h, int32_t staged);
int ltne_get_staging(const ltne_handle* h, int32_t* staged);

/* Row-slab decomposition on one device (no counterpart in the paper; the
   decomposition a multi-GPU run would use, checked here without a second
   GPU).  ltne_step_slabs advances the lattice n steps as nslabs slabs of
   consecutive rows, each with its own population buffers in `scratch`
   (caller-owned device memory of ltne_slab_scratch_bytes bytes, 256-byte
   aligned) and one halo row towards each neighbouring slab: after every
   step the slabs' boundary rows (all 19 planes) are copied into the
   neighbours' halo rows by device-to-device copies, then the computed rows
   and the macroscopic fields are gathered back into the handle.  The
   result is the same bits as ltne_step(h, n).  Cavity walls, FP32 or FP64
   storage, no local h_v, at least 2 rows per slab; otherwise
   ltne_slab_scratch_bytes returns 0 and ltne_step_slabs
   LTNE_ERR_INVALID_ARG.  Asynchronous on the handle's stream. */
size_t ltne_slab_scratch_bytes(const ltne_handle* h, int32_t nslabs);
int ltne_step_slabs(ltne_handle* h, int32_t nslabs, int64_t n, void* scratch, size_t bytes);

/* ------------------------------------------------------------------------
 * One row slab of the cavity per process (no counterpart in the paper,
 * which has no parallel code; its Sec. 1 notes the method's low
 * communication-to-computation ratio).  The lattice is cut into nslabs
 * slabs of consecutive rows; each process (typically one per GPU) creates a
 * slab handle for its own slab and, after every step, swaps the values that
 * stream across each cut with its neighbours through its own communicator
 * (NCCL, MPI, host-staged sockets ...).  With pull streaming a row reads
 * from the row below only the populations that stream up (e_y = +1: f_2,
 * f_5, f_6 and g_2 of both temperature lattices) and from the row above only
 * those that stream down (e_y = -1: f_4, f_7, f_8, g_4 of both): one message
 * of 5 x nx values per cut and direction and step.  Walls need no exchange
 * (the side walls lie in every slab, the bottom and top walls in the end
 * slabs).  The slabs' computed rows are the same bits as the undivided
 * lattice run with one node per thread (ltne_set_schedule(h, 64, 2, 1)).
 * Restrictions: cavity walls, FP32 or FP64 storage, no local h_v, at least 2
 * rows per slab; an Ergun permeability with a porosity field needs p->d_p > 0
 * (the diameter belongs to the whole field: ltne_ergun_diameter).
 * Sequence per process:
 *   ltne_create_slab -> ltne_workspace_bytes / ltne_bind_workspace ->
 *   ltne_set_fields (arrays of the LOCAL lattice: rows y0 - halo_lo ..
 *   y0 + rows - 1 + halo_hi of the cavity, nx per row; the halo rows take
 *   the neighbours' initial values) -> per step: ltne_step_slab ->
 *   exchange (send_lo -> the slab below's recv_hi, send_hi -> the slab
 *   above's recv_lo) -> ltne_halo_unpack.
 * ltne_step, ltne_observables, the adjoint, staging and two-node schedules
 * return LTNE_ERR_INVALID_ARG on a slab handle; ltne_get_fields returns the
 * local lattice (its halo rows hold no computed values); checkpoints work
 * per slab.
 * ---------------------------------------------------------------------- */

/* Slab `index` of `nslabs` of a cavity of ny rows: first row *y0, *rows
   rows (ny / nslabs, the first ny % nslabs slabs one more), and whether it
   has a halo row below / above (a neighbouring slab).  Any output pointer
   may be NULL.  INVALID_ARG unless 0 <= index < nslabs and ny / nslabs >= 2. */
int ltne_slab_rows(int32_t ny, int32_t nslabs, int32_t index, int32_t* y0, int32_t* rows,
                   int32_t* halo_lo, int32_t* halo_hi);

/* Handle for slab `index` of `nslabs` of the cavity *p (p->nx, p->ny and
   every other field describe the WHOLE cavity: the lattice constants,
   L = ny - 1 included, are the cavity's).  Errors as ltne_create, plus
   INVALID_ARG for the restrictions above. */
int ltne_create_slab(const ltne_params* p, int32_t nslabs, int32_t index, void* cuda_stream,
                     ltne_handle** out);

/* Device addresses of the four message buffers inside the bound workspace
   (NULL on a side without a neighbour) and their common size in bytes
   (5 x nx values of the storage type).  send_lo / send_hi: the values this
   slab gives the slab below / above, written by ltne_step_slab and
   ltne_halo_pack; recv_lo / recv_hi: where the caller puts what the slab
   below / above sent, read by ltne_halo_unpack.  The buffers hold, in this
   order, plane by plane (nx values each): below, f_4 f_7 f_8 g_f4 g_s4;
   above, f_2 f_5 f_6 g_f2 g_s2. */
int ltne_halo_buffers(ltne_handle* h, void** send_lo, void** send_hi, void** recv_lo,
                      void** recv_hi, size_t* bytes);

/* One time step of the slab's rows (the halo rows are read, not updated),
   then ltne_halo_pack.  write_macros = 1 also stores the macroscopic fields
   (needed before ltne_slab_accumulators or ltne_get_fields); 0 skips them.
   Asynchronous on the handle's stream: the send buffers are ready when the
   stream reaches this point. */
int ltne_step_slab(ltne_handle* h, int32_t write_macros);

/* Copy the current state's outgoing values into send_lo / send_hi (e.g.
   to fill the neighbours' halos right after ltne_set_fields or
   ltne_set_state), and the received values from recv_lo / recv_hi into the
   halo rows.  Asynchronous on the handle's stream. */
int ltne_halo_pack(ltne_handle* h);
int ltne_halo_unpack(ltne_handle* h);

/* The slab's share of the observables: LTNE_NACC FP64 accumulators of its
   computed rows (the wall-flux integrals take the trapezoid's half weight
   only at the cavity's bottom and top rows), as left by the last step with
   write_macros = 1.  Updates the slab's residual snapshot.  Synchronises. */
#define LTNE_NACC 18
int ltne_slab_accumulators(ltne_handle* h, double* acc, int32_t nacc);

/* acc <- acc combined with other (sums; the two maxima take the larger).
   Combining the slabs' vectors in slab order on every process gives every
   process the same bits. */
int ltne_accumulators_combine(double* acc, const double* other, int32_t nacc);

/* Observables of the whole cavity *p from its combined accumulators, after
   `step` steps; have_prev = 0 on the first reduction of a run (residual
   NaN), 1 after.  Returns LTNE_ERR_NONFINITE (with *out filled) if any
   node was non-finite.  Host only. */
int ltne_observables_from_accumulators(const ltne_params* p, int64_t step, int32_t have_prev,
                                       const double* acc, int32_t nacc, ltne_obs* out);

/* The Ergun particle diameter that makes the mean of K / L^2 over the n
   porosities equal Da (Eq. 7), with the arithmetic ltne_set_fields uses
   for d_p <= 0 (so a slab given it matches the undivided lattice bit for
   bit).  Host only. */
int ltne_ergun_diameter(const double* porosity, int64_t n, double L, double Da, double* d);

/* Self-check of the bounded wait of the staged step (no counterpart in the
   paper): one GPU thread waits, with at most `spins` polls, on an mbarrier
   phase that can never complete; *gave_up = 1 when the wait returned
   without it, as it must.  Allocates 4 bytes of device memory on the
   stream; synchronises it. */
int ltne_check_bounded_wait(void* cuda_stream, int32_t spins, int32_t* gave_up);
int ltne_get_schedule(const ltne_handle* h, int32_t* block_x, int32_t* block_y,
                      int32_t* nodes_per_thread);

/* ------------------------------------------------------------------------
 * Adjoint: gradients of J = (Nu_f,hot + Nu_s,hot) / 2 after n_steps steps
 * with respect to the per-node porosity and to H, by hand-written reverse
 * kernels of the time step (transposed collision, streaming and wall
 * rebuild of Sec. 3 / Sec. 4) with checkpoints every `segment` steps.  The
 * Ergun particle diameter derived from the porosity field is held fixed.
 * Restrictions: bc LTNE_BC_CAVITY, porosity_field = 1, storage LTNE_F32 or
 * LTNE_F64 (the gradient is computed in that precision), T_hot != T_cold,
 * and the fluid initially at rest (no initial velocity), which makes the
 * initial state independent of the porosity and of H.
 * ---------------------------------------------------------------------- */

/* Bytes of the adjoint workspace (caller-owned device memory): checkpoints
   of the pre-collision state at every segment start, `segment` recompute
   slots, adjoint and gradient buffers; about
   (ceil(n_steps/segment) + 2 segment + 6) * 19 planes of the compute type
   (two sets of recompute slots: one segment is reversed while the one
   before it is recomputed). */
size_t ltne_adjoint_workspace_bytes(const ltne_handle* h, int64_t n_steps, int32_t segment);

/* Register budget of the adjoint's transposed-collision kernel (no
   counterpart in the paper).  LTNE_ADJ_ONE_WAVE: every register the kernel
   wants (123 per thread in FP32), for lattices whose grid fits one wave of
   the device, where a reverse step's time is one thread's latency;
   LTNE_ADJ_CAPPED: registers capped at 64 so that 1024 threads share an SM
   (FP32; a few values spill to local memory), for larger
   lattices, where occupancy hides the latency.  LTNE_ADJ_AUTO (default)
   picks by the lattice size.  The two builds run the same code; they agree
   to rounding (under the cap the compiler may contract a different set of
   multiply-adds), and each is deterministic.  LTNE_ERR_INVALID_ARG for
   other values. */
#define LTNE_ADJ_AUTO 0
#define LTNE_ADJ_ONE_WAVE 1
#define LTNE_ADJ_CAPPED 2
int ltne_set_adjoint_schedule(ltne_handle* h, int32_t mode);
int ltne_get_adjoint_schedule(const ltne_handle* h, int32_t* mode);

/* Set the initial fields (as ltne_set_fields with u = 0; rho, T_f, T_s may
   be NULL), run n_steps >= 1 steps forward (the handle ends at step
   n_steps, exactly as after ltne_step), compute *J, and by the reverse
   sweep dJ/dphi into dJ_dphi (device, nx*ny values of the compute type,
   row-major, may be NULL) and dJ/dH into *dJ_dH.  adj_workspace: device,
   >= ltne_adjoint_workspace_bytes(), 256-byte aligned.  Synchronises the
   handle's stream.  Errors: INVALID_ARG (restrictions above, bad sizes),
   WORKSPACE, STATE (no workspace bound), CUDA. */
int ltne_adjoint(ltne_handle* h, const double* porosity, const double* rho, const double* T_f,
                 const double* T_s, int64_t n_steps, int32_t segment, void* adj_workspace,
                 size_t bytes, void* dJ_dphi, double* J, double* dJ_dH);

/* Observables of fields the caller holds on the device, allocating nothing.
   The paper has no counterpart: this serves callers that cannot allocate
   device memory at the moment they need a reduction -- a plug-in or monitor
   inside a host application that owns every device allocation and lends
   none to its guests, a thread from which the framework's allocator is not
   reachable, a real-time loop that must not allocate.  Those callers can
   neither size nor bind a workspace, so the reduction's per-block partial
   sums go to a fixed __device__ array inside this library (590 KB, held by
   every GPU that loads the library until the process exits).
   fields: device, FP32, five planes of nx*ny values with row pitch `pitch`
     (>= nx) elements and plane stride pitch*ny, holding rho - 1, u_x, u_y,
     T_f - T_ref, T_s - T_ref (the layout ltne_get_fields() values map to).
   porosity: device, FP32, one plane in the same layout, non-NULL iff
     p->porosity_field; otherwise p->porosity is used.
   step: reported in out->step and used for out->Fo.
   p: the problem statement (validated as by ltne_create; storage must not
     be LTNE_F64).  Results equal ltne_observables() on the same fields,
     except that no residual snapshot is kept: out->residual is NaN.
   Limit: ceil(nx/256) * ceil(ny/64) <= 4096 (e.g. any lattice up to
     8192 x 8192); larger lattices return LTNE_ERR_INVALID_ARG before any
     device work.
   The first call on each device asks the runtime for the array's device
   address (cudaGetSymbolAddress, with that device current), so make one
   call before any stream capture begins; a call that finds a different
   context current on the device (after cudaDeviceReset) asks again.  All
   calls share the array and it keeps the last call's contents (every slot
   a call reads is written by that call first): calls that overlap on the
   GPU -- on different streams, or on one stream while another thread also
   calls -- race and give wrong results.  The call copies the result back
   and synchronises `cuda_stream` before it returns. */
int ltne_observables_static(const ltne_params* p, const float* fields, int64_t pitch,
                            const float* porosity, int64_t step, void* cuda_stream,
                            ltne_obs* out);

/* Free the handle's host state and graphs (not the workspace). */
void ltne_destroy(ltne_handle* h);

/* Name of a status code. */
const char* ltne_error_string(int code);

/* ------------------------------------------------------------------------
 * Batched form: `count` independent cavities of uneven size and parameters
 * advanced together, one persistent launch per time step (replayed from a
 * captured CUDA graph).  The per-node method is exactly that of
 * ltne_step(); every cavity keeps its own walls (Sec. 4).  Restrictions:
 * storage LTNE_F32, bc LTNE_BC_CAVITY, uniform porosity per cavity
 * (porosity_field = 0).  Same ownership and stream rules as above.
 * ---------------------------------------------------------------------- */
typedef struct ltne_batch ltne_batch;

/* Validate and derive every cavity's constants from params[0..count-1].
   Errors as ltne_create, plus INVALID_ARG for a cavity outside the
   restrictions above. */
int ltne_batch_create(const ltne_params* params, int32_t count, void* cuda_stream,
                      ltne_batch** out);

/* Device workspace bytes (two population buffers for all cavities, macro
   and snapshot planes, reduction scratch, the cavity table and the largest
   tile list), and the total node count. */
size_t ltne_batch_workspace_bytes(const ltne_batch* b);
int64_t ltne_batch_nodes(const ltne_batch* b);

/* Bind caller-owned device memory (>= workspace bytes, 256-byte aligned);
   uploads the cavity table and the default schedule (128 x 2 tiles, one
   block per tile). */
int ltne_batch_bind_workspace(ltne_batch* b, void* device_ptr, size_t bytes);

/* Launch schedule: tiles of tile_x x tile_y nodes walked by `blocks`
   persistent blocks (0: one block per tile), each thread advancing
   nodes_per_thread = 1 node or 2 neighbouring nodes of a row (paired FP32
   arithmetic).  A block has tile_x / nodes_per_thread x tile_y threads:
   tile_x / nodes_per_thread in 32..256 and tile_y in 1..8, powers of two,
   64 to 256 threads per block (64 to 128 with two nodes per thread).
   Results do not depend on the schedule beyond FP32 contraction order
   (bitwise for a fixed nodes_per_thread). */
int ltne_batch_set_schedule(ltne_batch* b, int32_t tile_x, int32_t tile_y, int32_t blocks,
                            int32_t nodes_per_thread);

/* Every cavity at rest: rho = 1, u = 0, T_f = T_s = its T_ref (equilibrium
   populations, walls included).  Resets the step counter. */
int ltne_batch_set_fields(ltne_batch* b);

/* Advance all cavities n >= 0 steps, asynchronously on the stream. */
int ltne_batch_step(ltne_batch* b, int64_t n);

/* Observables of every cavity into out[0..count-1] (synchronises). */
int ltne_batch_observables(ltne_batch* b, ltne_obs* out);

/* Fields of cavity `index` into host arrays of nx*ny doubles (synchronises). */
int ltne_batch_get_fields(ltne_batch* b, int32_t index, double* rho, double* ux, double* uy,
                          double* T_f, double* T_s);

/* Number of step launches issued so far (one per time step). */
int64_t ltne_batch_launch_count(const ltne_batch* b);

void ltne_batch_destroy(ltne_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* LTNE_H */
