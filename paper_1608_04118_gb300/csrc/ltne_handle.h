// ltne_handle.h -- host state of one lattice handle (opaque to C callers),
// shared by the translation units that implement the ltne_* entry points.
// Kept apart from ltne_internal.h, which holds what the kernels see.
#pragma once

#include "ltne_internal.h"

// Host state of one lattice (opaque to C callers).
struct ltne_handle {
  ltne_params p;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t aux_stream = nullptr;  // the adjoint's recompute
  ltne::NodeParams<double> P{};
  ltne::StepShape shape;
  // derived lattice values
  double L = 0, nu_f = 0, alpha_f = 0, d_ergun = 0;
  // layout
  int64_t pitch = 0, plane = 0;
  size_t es = 0, ec = 0;  // storage / compute element sizes
  size_t off_pop[2] = {0, 0}, off_phi = 0, off_part = 0, off_out = 0;
  // two sets of the 5 macro planes: the current state's, and the snapshot
  // taken by the last ltne_observables call (the residual's reference)
  size_t off_mac[2] = {0, 0};
  size_t off_tick = 0;
  size_t off_um[2] = {0, 0};  // |u| planes (local h_v of Eq. 52)
  size_t ws_bytes = 0;
  char* ws = nullptr;
  int red_blocks = 1;
  // state
  int cur = 0;
  int64_t step = 0;
  bool fields_set = false;
  bool have_prev = false;
  int mcur = 0;             // macro set holding the current state's fields
  int msnap = -1;           // macro set holding the snapshot (-1: none yet)
  float enc_scale = 1.0f;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int64_t launches = 0;
  int32_t adj_sched = 0;  // LTNE_ADJ_*
  // two pinned host buffers that stage whole fields in and out (allocated
  // at the first set_fields / get_fields, freed by ltne_destroy), with an
  // event per buffer marking its last copy
  char* pin[2] = {nullptr, nullptr};
  cudaEvent_t pin_ev[2] = {nullptr, nullptr};
  size_t pin_bytes = 0;
  // host I/O form (LTNE_HOST_IO_*) and whether the device reaches pageable
  // host memory through the host's page tables (-1: not asked yet)
  int32_t host_io = LTNE_HOST_IO_AUTO;
  int direct_io = -1;
  // Row slab of a cavity advanced by one process (ltne_create_slab): the
  // local lattice is the slab's computed rows with a halo row towards each
  // neighbouring slab; p.ny counts the local rows, gny the cavity's.
  int slab = 0;
  int nslabs = 1, slab_index = 0;
  int gny = 0;             // rows of the whole cavity
  int g0 = 0, srows = 0;   // first global row computed here, rows computed
  int slo = 0, shi = 0;    // halo row below / above (0 or 1)
  size_t off_halo[4] = {0, 0, 0, 0};  // send below, send above, receive below, above
  // pinned landing place of the observables' accumulators and the device
  // error word (one asynchronous read-back per ltne_observables call)
  double* pin_obs = nullptr;
};

namespace ltne {
// The current state's macro planes.
inline char* mac_cur(const ltne_handle* h) { return h->ws + h->off_mac[h->mcur]; }
// The macro set the next write of the fields goes to: never the snapshot
// of the last observables call while the residual still needs it.
inline int mac_next(const ltne_handle* h) {
  return h->msnap == h->mcur ? (h->mcur ^ 1) : h->mcur;
}
// Initial state S_0 from host fields (ltne_set_fields); pre_out, if not
// null, also receives S_0 (compute type, population-plane layout).
int set_fields_impl(ltne_handle* h, const double* porosity, const double* rho, const double* ux,
                    const double* uy, const double* T_f, const double* T_s, void* pre_out);
// The handle's observables reduction into acc[NACC] (synchronises).
int reduce_handle(ltne_handle* h, double* acc);
// The same reduction, enqueued on the handle's stream only (the result in
// the workspace's output slot).
int reduce_launch(ltne_handle* h);
}  // namespace ltne
