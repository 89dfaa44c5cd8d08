// ltne_internal.h -- host-side declarations shared by the library's
// translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ltne.h"
#include "ltne_node.cuh"

namespace ltne {

// Boundary modes (values of LTNE_BC_*), and BC_SLAB: a row slab of a cavity
// (left/right walls; its first and last rows are either the cavity's
// bottom/top wall rows or halo rows holding the neighbouring slabs' values,
// which are read but not updated).
constexpr int BC_CAVITY = 0, BC_PERIODIC = 1, BC_CHANNEL = 2, BC_SLAB = 3;
constexpr int SLAB_LO_WALL = 1, SLAB_HI_WALL = 2;  // bits of slab_walls

// Geometry and buffers of one lattice as the kernels see it.  Populations
// are structure-of-arrays planes, index q*plane + y*pitch + x, in the order
// f_0..f_8, g_f0..g_f4, g_s0..g_s4.  Rows are padded to a multiple of 64
// elements and planes to a multiple of 256 bytes.
struct LatticeArgs {
  const void* src;   // post-collision populations of the last step
  void* dst;         // populations written by this step
  const void* phi;   // per-node porosity plane (compute type) or nullptr
  void* mac;         // 5 macro planes (rho-1, ux, uy, Tf-T0, Ts-T0; compute type)
  int nx, ny;
  int bc;            // LTNE_BC_*
  int write_macros;  // 1: also store the macroscopic fields of S_n
  int64_t pitch;     // elements per row
  int64_t plane;     // elements per plane
  float enc_scale;   // 16-bit storage scale (power of two)
  const uint32_t* tick_in;  // step counter slot read by this step (16-bit forms)
  uint32_t* tick_out;       // slot receiving the next step's counter
  void* pre_out;            // k_init: also record S_0 here (compute type), or nullptr
  const void* um_in;        // |u| plane of the previous state (local h_v), or nullptr
  void* um_out;             // |u| plane written for the next state
  int* err;                 // device error word: set by a bounded wait that gave up
  int slab_walls;           // BC_SLAB: which of the first / last rows are walls
  int chained;              // launch as a programmatic dependent of the stream's last kernel
};

// Programmatic dependent launch.  A kernel launched with programmatic
// stream serialisation is scheduled as the blocks of the kernel before it
// on the stream exit, before that grid's completion is signalled, and waits
// here for the completion (and its memory flush) before touching global
// memory; without the launch attribute the wait is a no-op.  Every thread
// of a kernel that may be launched so executes it before any global access
// or early return, so each grid completes only after its predecessor did.
// No kernel triggers its dependents early (griddepcontrol.launch_dependents):
// blocks of the next kernel parked on the SMs while a single-wave grid still
// runs made the adjoint's chain 6-20 % slower at 256 x 256.
__device__ __forceinline__ void grid_dep_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Launch k with the programmatic-serialisation attribute when `chained`.
template <typename... KArgs, typename... Args>
cudaError_t launch_kernel(bool chained, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem,
                          cudaStream_t s, Args... args) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = chained ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

// Launch configuration of the step kernel: a block of bx x by threads,
// each advancing one node or (pair = 1, FP32 arithmetic only, at most
// kPairBlockThreads threads per block) two neighbouring nodes of a row.
constexpr int kPairBlockThreads = 128;
struct StepShape {
  int bx = 64;
  int by = 2;
  int pair = 0;
  int tma = 0;  // two nodes per thread from TMA-staged tiles (cavity walls only)
};

// Per-storage-type launchers (one translation unit each).
#define LTNE_DECLARE_LAUNCHERS(tag)                                                            \
  cudaError_t launch_step_##tag(const LatticeArgs& a, const NodeParams<double>& P,             \
                                StepShape s, cudaStream_t st);                                 \
  cudaError_t launch_init_##tag(const LatticeArgs& a, const NodeParams<double>& P,             \
                                cudaStream_t st);
LTNE_DECLARE_LAUNCHERS(f64)
LTNE_DECLARE_LAUNCHERS(f32)
LTNE_DECLARE_LAUNCHERS(f16)
LTNE_DECLARE_LAUNCHERS(bf16)
#undef LTNE_DECLARE_LAUNCHERS

// Observables reduction (FP64): accumulator slots.
enum {
  A_NUF_H = 0, A_NUS_H, A_NUF_C, A_NUS_C, A_MASS, A_ENERGY, A_MAXU, A_MAXDT, A_SUMTF,
  A_SUMTS, A_DU2, A_U2, A_DTF2, A_TF2, A_DTS2, A_TS2, A_BAD, A_SUMPHI, NACC
};

struct ReduceArgs {
  const void* mac;   // 5 macro planes (deviations: rho-1, ux, uy, Tf-T0, Ts-T0)
  const void* phi;   // porosity plane or nullptr
  void* prev;        // 4 planes: ux, uy, Tf, Ts of the previous call
  double* partials;  // [blocks][NACC] scratch
  double* out;       // [NACC]
  int nx, ny;
  int64_t pitch, plane;
  double phi_u, sigma, qf, qs;
  int update_prev;
  int blocks;
  int is_double;     // macro planes hold doubles (else floats)
  // 1: the first / last reduced row is a wall row of the cavity (half
  // trapezoid weight in the wall-flux integrals); 0 for the inner edge of a
  // row slab
  int wall_lo = 1, wall_hi = 1;
};

cudaError_t launch_reduce(const ReduceArgs& a, cudaStream_t st);

// Halo rows of a row slab (ltne_slab.cu).  Pack: the populations of the
// slab's first computed row that stream down (e_y = -1: f_4, f_7, f_8,
// g_f4, g_s4) into send_lo, those of its last computed row that stream up
// (e_y = +1: f_2, f_5, f_6, g_f2, g_s2) into send_hi, 5 x nx values each.
// Unpack: recv_lo into the same five e_y = +1 planes of the halo row below,
// recv_hi into the e_y = -1 planes of the halo row above.  A null buffer
// skips its side.  Element size es (4 or 8 bytes).
cudaError_t launch_halo_pack(const void* pops, int64_t pitch, int64_t plane, int nx, int row_lo,
                             int row_hi, size_t es, void* send_lo, void* send_hi,
                             cudaStream_t st);
cudaError_t launch_halo_unpack(void* pops, int64_t pitch, int64_t plane, int nx, int halo_lo,
                               int halo_hi, size_t es, const void* recv_lo, const void* recv_hi,
                               cudaStream_t st);
// Whole fields between the caller's host arrays (row-major nx x ny, FP64,
// absolute values) and the device planes (deviations ref subtracted, compute
// type), moved by kernels that access the host arrays themselves
// (ltne_hostio.cu); for GPUs that reach pageable host memory through the
// host's page tables.  A null src / dst skips that plane.
struct HostPlanes {
  const double* src[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  double* dst[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  double ref[5] = {0, 0, 0, 0, 0};
};
cudaError_t launch_fields_to_host(const void* mac, bool dbl, int64_t plane, int64_t pitch, int nx,
                                  int ny, const HostPlanes& hp, cudaStream_t s);
cudaError_t launch_fields_from_host(void* mac, bool dbl, int64_t plane, int64_t pitch, int nx,
                                    int ny, const HostPlanes& hp, uint32_t* bad, cudaStream_t s);
// The porosity plane from the caller's host array; with erg_part, also the
// Ergun chunk sums of the field (kErgunChunk order below) into
// erg_part[0 .. ergun_chunks(n)).
cudaError_t launch_porosity_from_host(const double* phi, void* dst, bool dbl, int64_t pitch, int nx,
                                      int ny, double* erg_part, uint32_t* bad, cudaStream_t s);

// The Ergun mean of a porosity field, mean(phi^3 / (1 - phi)^2): with the
// Ergun permeability (Eq. 7) it fixes the particle diameter that makes the
// mean of K / L^2 equal to Da.  Its summation order is the same on the host
// (ergun_mean) and in the porosity kernel, so the diameter has the same bits
// whichever forms it: chunks of kErgunChunk consecutive values; in chunk c,
// lane l adds the terms of values c * kErgunChunk + kErgunLanes * j + l for
// j = 0, 1, ... in order; the lane sums combine by strides 16, 8, 4, 2, 1
// (sum l += sum l + stride); the chunk sums are added in order.
constexpr int kErgunLanes = 32, kErgunPerLane = 64, kErgunChunk = kErgunLanes * kErgunPerLane;
__host__ __device__ inline double ergun_term(double ph) {
  return ph * ph * ph / ((1.0 - ph) * (1.0 - ph));
}
inline int64_t ergun_chunks(int64_t n) { return (n + kErgunChunk - 1) / kErgunChunk; }
// Mean of phi^3 / (1 - phi)^2 over n porosities, in the order above.
double ergun_mean(const double* porosity, int64_t n);
// The same mean from the chunk sums.
double ergun_mean_of_chunks(const double* part, int64_t n);

// Host-side parameter mapping and observables (ltne_api.cu), shared with
// the batched form.
struct DerivedInfo {
  double L = 0, nu_f = 0, alpha_f = 0;
  double d_ergun = 0;  // Ergun particle diameter in use (0: Darcy permeability)
};
int validate_params(const ltne_params& p);
// erg_mean: the mean of phi^3 / (1 - phi)^2 over a per-node porosity field
// (nullptr: the uniform porosity's value); it fixes the Ergun diameter when
// none is given
int derive_params(const ltne_params& p, const double* erg_mean, NodeParams<double>& P,
                  DerivedInfo& info);
int finish_observables(const ltne_params& p, const DerivedInfo& info, int64_t step,
                       bool have_prev, const double* acc, ltne_obs* out);
int reduce_blocks(int nx, int ny);  // pass-1 blocks (= partial vectors)
// Pass-1 blocks stay within this count whenever rows of 64 allow it (every
// lattice up to 8192 x 8192): the size of the fixed partials array of the
// allocation-free observables.
constexpr int kReduceMaxBlocks = 4096;

}  // namespace ltne
