// ltne_adjoint.cu -- reverse-mode (adjoint) time stepping of the
// three-distribution MRT-LB method (Liu & He, arXiv:1608.04118) for
// gradients of J = (Nu_f,hot + Nu_s,hot)/2 at the final step with respect to
// the per-node porosity and to H.
//
// State: S_n = pre-collision populations after streaming and the wall
// rebuild.  One forward transition is S_{n+1} = W(Pull(Coll(S_n))), Coll the
// per-node collision (Eqs. 10, 32, 33 with Eqs. 5-7, 15, 37-46), Pull the
// streaming (Eqs. 11, 34, 35) and W the wall rebuild.  Its transpose, applied
// to the adjoint lambda_{n+1} of S_{n+1}:
//   R1 (wall fold): a wall node's populations are rebuilt from those of one
//      interior neighbour r by non-equilibrium extrapolation; the transposed rebuild Jacobian at r
//      maps the wall node's adjoint onto r.  The thread that computes a wall
//      node's adjoint applies it at once and stores the result in the wall
//      node's place (a wall node's own adjoint is never pulled).
//   R2 (grid kernel): the adjoint of Coll's output at y is gathered from
//      y + e_i (the transpose of a pull is a pull the other way; only
//      interior targets pulled; a target next to a wall adds the folds of its
//      wall nodes in a fixed order), then the transposed collision Jacobian at
//      S_n(y) gives lambda_n(y) and the porosity / h_v contributions.
// Gradients accumulate per node (porosity, and the h_v term reduced once in
// FP64 at the end; a fold's porosity term in its wall node's place of a
// separate plane, added to r once at the end), so the result is
// deterministic.
//
// Memory: sqrt(T)-style checkpointing.  The forward pass records S_a at the
// start of every segment of K steps; the reverse sweep recomputes each
// segment's S_{a+1..a+K} from its checkpoint into K slots, then walks back
// through it.  Total extra work: one forward pass, run on a second stream
// beside the reverse sweep of the segment after it.
#include <math.h>
#include <string.h>

#include "ltne.h"
#include "ltne_internal.h"
#include "ltne_handle.h"
#include "ltne_step_impl.cuh"
#include "ltne_adjoint.cuh"

using namespace ltne;

namespace {

constexpr int kRB = 256;

template <typename C>
__device__ __forceinline__ void load19(const C* __restrict__ b, int64_t plane, int64_t off,
                                       C (&f)[9], C (&gf)[5], C (&gs)[5]) {
#pragma unroll
  for (int i = 0; i < 9; ++i) f[i] = b[(int64_t)i * plane + off];
#pragma unroll
  for (int i = 0; i < 5; ++i) gf[i] = b[(int64_t)(9 + i) * plane + off];
#pragma unroll
  for (int i = 0; i < 5; ++i) gs[i] = b[(int64_t)(14 + i) * plane + off];
}

template <typename C>
__device__ __forceinline__ void store19(C* __restrict__ b, int64_t plane, int64_t off,
                                        const C (&f)[9], const C (&gf)[5], const C (&gs)[5]) {
#pragma unroll
  for (int i = 0; i < 9; ++i) b[(int64_t)i * plane + off] = f[i];
#pragma unroll
  for (int i = 0; i < 5; ++i) b[(int64_t)(9 + i) * plane + off] = gf[i];
#pragma unroll
  for (int i = 0; i < 5; ++i) b[(int64_t)(14 + i) * plane + off] = gs[i];
}

// Forward step that also records S_{n+1} (pre_out may be null).
template <typename C>
__global__ void __launch_bounds__(256) k_step_record(const C* __restrict__ src,
                                                     C* __restrict__ dst,
                                                     const C* __restrict__ phi,
                                                     C* __restrict__ mac, const NodeParams<C> P,
                                                     int nx, int ny, int64_t pitch,
                                                     int64_t plane, int write_macros,
                                                     C* __restrict__ pre_out) {
  grid_dep_wait();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= nx || y >= ny) return;
  step_node<C, C, BC_CAVITY>(src, dst, phi, mac, P, x, y, nx, ny, pitch, plane, C(1), C(1),
                             write_macros, 0u, pre_out);
}

// Post-collision values of a recorded pre-collision state.
template <typename C>
__global__ void __launch_bounds__(256) k_collide_pre(const C* __restrict__ pre,
                                                     C* __restrict__ dst,
                                                     const C* __restrict__ phi,
                                                     const NodeParams<C> P, int nx, int ny,
                                                     int64_t pitch, int64_t plane) {
  grid_dep_wait();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= nx || y >= ny) return;
  const int64_t off = (int64_t)y * pitch + x;
  C f[9], gf[5], gs[5];
  load19(pre, plane, off, f, gf, gs);
  const Medium<C> md = medium_at<C>(P, phi[off]);
  Macro<C> m;
  macros<C>(P, md, f, gf, gs, m);
  collide<C>(P, m, f, gf, gs);
  store19(dst, plane, off, f, gf, gs);
}

// R1 for a wall node: the interior node r its populations are rebuilt from
// (the isothermal columns own the corners) and that node's state.
template <typename C>
struct WallSource {
  C f[9], gf[5], gs[5];
  C phi;
  bool iso;
};

template <typename C>
__device__ __forceinline__ void load_wall_source(const C* __restrict__ S,
                                                 const C* __restrict__ phi, int x, int y, int nx,
                                                 int ny, int64_t pitch, int64_t plane,
                                                 WallSource<C>& w) {
  int rx = x, ry;
  if (x == 0 || x == nx - 1) {
    rx = (x == 0) ? 1 : nx - 2;
    ry = y < 1 ? 1 : (y > ny - 2 ? ny - 2 : y);
    w.iso = true;
  } else {
    ry = (y == 0) ? 1 : ny - 2;
    w.iso = false;
  }
  const int64_t roff = (int64_t)ry * pitch + rx;
  load19(S, plane, roff, w.f, w.gf, w.gs);
  w.phi = phi[roff];
}

// The wall node's adjoint (lf, lgf, lgs) through the transposed rebuild
// Jacobian at r: stored in the wall node's place of lam; the porosity term
// (for r) accumulates in the wall node's place of wphib, the h_v term in hv.
template <typename C>
__device__ __forceinline__ void fold_wall(const NodeParams<C>& P, const WallSource<C>& w,
                                          const C (&lf)[9], const C (&lgf)[5], const C (&lgs)[5],
                                          C* __restrict__ lam, C* __restrict__ wphib,
                                          int64_t plane, int64_t off, C& hv) {
  const Medium<C> md = medium_at<C>(P, w.phi);
  C cf[9] = {}, cgf[5] = {}, cgs[5] = {};
  MediumBar<C> mdb;
  zero(mdb);
  nee_adjoint<C>(P, md, w.f, w.gf, w.gs, w.iso, lf, lgf, lgs, cf, cgf, cgs, mdb);
  store19(lam, plane, off, cf, cgf, cgs);
  C pb = C(0), hb = C(0);
  medium_adjoint<C>(P, w.phi, md, mdb, pb, hb);
  wphib[off] += pb;
  hv += hb;
}

// Adds to the gathered adjoint q (pulled from y + e_i) the folds stored at
// the wall nodes of each target next to a wall: its side-column node, its
// bottom/top-row node, then the corner, in that order.
template <typename C>
__device__ __forceinline__ void add_wall_folds(const C* __restrict__ Lam, int x, int y, int nx,
                                               int ny, int64_t pitch, int64_t plane,
                                               C (&qf)[9], C (&qgf)[5], C (&qgs)[5]) {
  const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int tx = x + ex[i], ty = y + ey[i];
    if (tx < 1 || tx > nx - 2 || ty < 1 || ty > ny - 2) continue;
    const bool cx = tx == 1 || tx == nx - 2, cy = ty == 1 || ty == ny - 2;
    if (!cx && !cy) continue;
    const int wx = (tx == 1) ? 0 : nx - 1, wy = (ty == 1) ? 0 : ny - 1;
    int64_t wo[3];
    bool wv[3];
    wv[0] = cx;
    wo[0] = (int64_t)ty * pitch + wx;
    wv[1] = cy;
    wo[1] = (int64_t)wy * pitch + tx;
    wv[2] = cx && cy;
    wo[2] = (int64_t)wy * pitch + wx;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (!wv[k]) continue;
      qf[i] += Lam[(int64_t)i * plane + wo[k]];
      if (i < 5) {
        qgf[i] += Lam[(int64_t)(9 + i) * plane + wo[k]];
        qgs[i] += Lam[(int64_t)(14 + i) * plane + wo[k]];
      }
    }
  }
}

// lambda_N: J depends on S_N through the temperatures of columns 1 and 2
// (wall-flux stencil of the Nusselt numbers, trapezoid weights in y).  The
// end nodes of the two columns lie on the bottom and top walls: their
// adjoints are folded (R1) at once.
template <typename C>
__global__ void __launch_bounds__(256) k_adj_seed(const C* __restrict__ SN, C* __restrict__ lam,
                                                  const C* __restrict__ phi,
                                                  C* __restrict__ phib, C* __restrict__ hb,
                                                  C* __restrict__ wphib, const NodeParams<C> P,
                                                  int nx, int ny, int64_t pitch, int64_t plane,
                                                  C inv_dT) {
  grid_dep_wait();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * ny) return;
  const int y = t >> 1, x = 1 + (t & 1);
  const int64_t off = (int64_t)y * pitch + x;
  const C wy = (y == 0 || y == ny - 1) ? C(0.5) : C(1);
  // J = (1/2)(Nu_f + Nu_s), Nu = (1/dT) sum_y w_y (1.5 T_h - 2 T(1,y) + 0.5 T(2,y))
  const C dT_b = (x == 1) ? -wy * inv_dT : C(0.25) * wy * inv_dT;
  C f[9], gf[5], gs[5];
  load19(SN, plane, off, f, gf, gs);
  const C ph = phi[off];
  const Medium<C> md = medium_at<C>(P, ph);
  MacroBar<C> mb;
  zero(mb);
  mb.dTf = dT_b;
  mb.dTs = dT_b;
  C fb[9] = {}, gfb[5] = {}, gsb[5] = {};
  MediumBar<C> mdb;
  zero(mdb);
  macros_adjoint<C>(P, md, f, gf, gs, mb, fb, gfb, gsb, mdb);
  C pb = C(0), hv = C(0);
  if (y == 0 || y == ny - 1) {
    WallSource<C> w;
    load_wall_source(SN, phi, x, y, nx, ny, pitch, plane, w);
    fold_wall(P, w, fb, gfb, gsb, lam, wphib, plane, off, hv);
  } else {
    store19(lam, plane, off, fb, gfb, gsb);
  }
  medium_adjoint<C>(P, ph, md, mdb, pb, hv);
  phib[off] += pb;
  hb[off] += hv;
}

// R2: transposed streaming (gather from y + e_i) and transposed collision;
// a wall node's thread then folds its result (R1) unless S_n is the initial
// state (fold = 0), whose wall nodes were not rebuilt.  The fold raises the
// kernel's registers (123 against 73 without it, FP32).  Two builds of the
// same code: kCapped = false keeps them all (lattices that fit one wave,
// where the kernel's time is one thread's latency); kCapped = true caps them
// at 64, 1024 threads' worth per SM (FP32; larger lattices, where occupancy
// hides the latency), spilling a few values to local memory.
template <typename C, bool kCapped>
__global__ void __launch_bounds__(256, (kCapped && sizeof(C) == 4) ? 4 : 1)
    k_adj_main(const C* __restrict__ Lam,
                                                  C* __restrict__ lam_out,
                                                  const C* __restrict__ S,
                                                  const C* __restrict__ phi,
                                                  C* __restrict__ phib, C* __restrict__ hb,
                                                  C* __restrict__ wphib, const NodeParams<C> P,
                                                  int nx, int ny, int64_t pitch, int64_t plane,
                                                  int fold, const C* __restrict__ S_prev) {
  grid_dep_wait();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= nx || y >= ny) return;
  const int64_t off = (int64_t)y * pitch + x;
  // one-wave build: this node's gradient accumulators, read here so that
  // their latency is not the last link of the chain below (the capped build
  // keeps its registers for the chain and reads them at the end)
  C phib0 = C(0), hb0 = C(0);
  if (!kCapped) {
    phib0 = phib[off];
    hb0 = hb[off];
  }
  // the next reverse step's state, recomputed a whole segment ago and mostly
  // evicted to HBM by now: fetched into L2 while this step runs (one-wave
  // build only: on larger lattices, bound by HBM throughput, it cost 4 %)
  if (!kCapped && S_prev && (x & 7) == 0) {
#pragma unroll
    for (int i = 0; i < 19; ++i)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(S_prev + (int64_t)i * plane + off));
  }
  // e_i of Eq. 8
  const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  C qf[9], qgf[5], qgs[5];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int tx = x + ex[i], ty = y + ey[i];
    const bool pulled = tx >= 1 && tx <= nx - 2 && ty >= 1 && ty <= ny - 2;
    const int64_t toff = (int64_t)ty * pitch + tx;
    qf[i] = pulled ? Lam[(int64_t)i * plane + toff] : C(0);
    if (i < 5) {
      qgf[i] = pulled ? Lam[(int64_t)(9 + i) * plane + toff] : C(0);
      qgs[i] = pulled ? Lam[(int64_t)(14 + i) * plane + toff] : C(0);
    }
  }
  if (x <= 2 || x >= nx - 3 || y <= 2 || y >= ny - 3)
    add_wall_folds(Lam, x, y, nx, ny, pitch, plane, qf, qgf, qgs);
  const bool wall = fold && (x == 0 || x == nx - 1 || y == 0 || y == ny - 1);
  WallSource<C> w;
  if (wall) load_wall_source(S, phi, x, y, nx, ny, pitch, plane, w);
  C f[9], gf[5], gs[5];
  load19(S, plane, off, f, gf, gs);
  const C ph = phi[off];
  const Medium<C> md = medium_at<C>(P, ph);
  C fb[9] = {}, gfb[5] = {}, gsb[5] = {};
  MediumBar<C> mdb;
  zero(mdb);
  collide_adjoint<C>(P, md, f, gf, gs, qf, qgf, qgs, fb, gfb, gsb, mdb);
  C pb = C(0), hv = C(0);
  if (wall)
    fold_wall(P, w, fb, gfb, gsb, lam_out, wphib, plane, off, hv);
  else
    store19(lam_out, plane, off, fb, gfb, gsb);
  medium_adjoint<C>(P, ph, md, mdb, pb, hv);
  if (kCapped) {
    phib0 = phib[off];
    hb0 = hb[off];
  }
  phib[off] = phib0 + pb;
  hb[off] = hb0 + hv;
}

// The folds' porosity terms, kept in their wall nodes' places, added to the
// interior node each wall node was rebuilt from (side column, bottom/top
// row, corner: the order of the gather).
template <typename C>
__global__ void __launch_bounds__(256) k_add_wall_phib(C* __restrict__ phib,
                                                       const C* __restrict__ wphib, int nx,
                                                       int ny, int64_t pitch) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x < 1 || x > nx - 2 || y < 1 || y > ny - 2) return;
  const bool cx = x == 1 || x == nx - 2, cy = y == 1 || y == ny - 2;
  if (!cx && !cy) return;
  const int wx = (x == 1) ? 0 : nx - 1, wy = (y == 1) ? 0 : ny - 1;
  C acc = phib[(int64_t)y * pitch + x];
  if (cx) acc += wphib[(int64_t)y * pitch + wx];
  if (cy) acc += wphib[(int64_t)wy * pitch + x];
  if (cx && cy) acc += wphib[(int64_t)wy * pitch + wx];
  phib[(int64_t)y * pitch + x] = acc;
}

// FP64 sum of one plane (fixed grid and order: deterministic).
template <typename C>
__global__ void __launch_bounds__(kRB) k_sum_plane(const C* __restrict__ v, int nx, int ny,
                                                   int64_t pitch, double* __restrict__ part) {
  __shared__ double sh[kRB / 32];
  double acc = 0.0;
  const int64_t n = (int64_t)nx * ny;
  for (int64_t k = (int64_t)blockIdx.x * kRB + threadIdx.x; k < n; k += (int64_t)gridDim.x * kRB) {
    const int y = (int)(k / nx), x = (int)(k - (int64_t)y * nx);
    acc += (double)v[(int64_t)y * pitch + x];
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kRB / 32; ++w) s += sh[w];
    part[blockIdx.x] = s;
  }
}

__global__ void k_sum_partials(const double* __restrict__ part, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    *out = s;
  }
}

template <typename C>
__global__ void __launch_bounds__(256) k_copy19(const C* __restrict__ src, C* __restrict__ dst,
                                                int64_t n) {
  grid_dep_wait();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    dst[k] = src[k];
}

// A captured launch sequence whose first kernel's arguments are replaced
// before each replay (the only argument that changes between segments).
struct SegGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t root = nullptr;
  ~SegGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
  template <typename F>
  cudaError_t capture(cudaStream_t cap, F&& body) {
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const cudaError_t le = body(cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cap, &g);
    if (le != cudaSuccess || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return le != cudaSuccess ? le : e;
    }
    size_t nroot = 1;
    e = cudaGraphGetRootNodes(g, &root, &nroot);
    if (e == cudaSuccess && nroot != 1) e = cudaErrorInvalidValue;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      return e;
    }
    graph = g;
    return cudaSuccess;
  }
  // Replace the root kernel's arguments and launch.
  cudaError_t launch(void* func, dim3 grid, dim3 block, void** args, cudaStream_t st) {
    cudaKernelNodeParams kp = {};
    kp.func = func;
    kp.gridDim = grid;
    kp.blockDim = block;
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    kp.extra = nullptr;
    cudaError_t e = cudaGraphExecKernelNodeSetParams(exec, root, &kp);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
    return e;
  }
};

// Every kernel above waits in grid_dep_wait(): launched chained to its
// predecessor on the stream when that is one of them.
template <typename... KArgs, typename... Args>
cudaError_t launch_chained(bool chained, void (*k)(KArgs...), dim3 grid, dim3 block,
                           cudaStream_t s, Args... args) {
  return launch_kernel(chained, k, grid, block, 0, s, args...);
}

// Two events for a fork and a join between streams (no timing).
struct EventPair {
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaError_t create() {
    cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
    return e;
  }
  ~EventPair() {
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
  }
};

constexpr int kSumBlocks = 128;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct AdjLayout {
  int64_t nseg = 0;
  size_t p19 = 0, pl = 0;  // bytes of 19 planes, of one plane
  size_t ckpt = 0, slots = 0, seg0 = 0, pops = 0, lam = 0, phib = 0, hb = 0, wphib = 0, part = 0;
  size_t total = 0;
};

AdjLayout adj_layout(const ltne_handle* h, int64_t n_steps, int32_t segment) {
  AdjLayout L;
  const size_t A = 256;
  L.nseg = (n_steps + segment - 1) / segment;
  L.pl = align_up((size_t)h->plane * h->ec, A);
  L.p19 = 19 * L.pl;
  size_t off = 0;
  L.ckpt = off;
  off += (size_t)L.nseg * L.p19;
  L.slots = off;  // two sets: one being reversed, one being recomputed
  off += 2 * (size_t)segment * L.p19;
  L.seg0 = off;  // the segments' checkpoints copied for graph replay (two)
  off += 2 * L.p19;
  L.pops = off;
  off += 2 * L.p19;
  L.lam = off;
  off += 2 * L.p19;
  L.phib = off;
  off += L.pl;
  L.hb = off;
  off += L.pl;
  L.wphib = off;
  off += L.pl;
  L.part = off;
  off += align_up((kSumBlocks + 1) * sizeof(double), A);
  L.total = off;
  return L;
}

template <typename C>
int run_adjoint(ltne_handle* h, const double* porosity, const double* rho, const double* T_f,
                const double* T_s, int64_t N, int32_t K, char* ws, void* dJ_dphi, double* J,
                double* dJ_dH) {
  const AdjLayout L = adj_layout(h, N, K);
  const cudaStream_t st = h->stream;
  const int nx = h->p.nx, ny = h->p.ny;
  const int64_t pitch = h->pitch, plane = h->plane;
  // plane strides in elements: every buffer uses the population layout
  const int64_t pe = (int64_t)(L.pl / sizeof(C));
  auto buf19 = [&](size_t base, int64_t k) { return reinterpret_cast<C*>(ws + base + k * L.p19); };
  C* phib = reinterpret_cast<C*>(ws + L.phib);
  C* hb = reinterpret_cast<C*>(ws + L.hb);
  C* wphib = reinterpret_cast<C*>(ws + L.wphib);
  double* part = reinterpret_cast<double*>(ws + L.part);
  (void)pe;

  int rc = set_fields_impl(h, porosity, rho, nullptr, nullptr, T_f, T_s, buf19(L.ckpt, 0));
  if (rc != LTNE_OK) return rc;
  const NodeParams<C> P = cast_params<C>(h->P);
  const C* phi = reinterpret_cast<const C*>(h->ws + h->off_phi);
  C* mac = reinterpret_cast<C*>(mac_cur(h));  // set 0 after set_fields, no snapshot
  // 64 x 2 blocks: measured against 128 x 2, 128 x 1, 256 x 1, 32 x 4,
  // 64 x 1 and 32 x 2 (the recompute shares the SMs with the reverse sweep;
  // 256^2: 5,530 against 5,456 MLUPS with 128 x 2, 1024^2: 9,548 against
  // 9,131)
  const dim3 blk(64, 2), grd((nx + 63) / 64, (ny + 1) / 2);
  cudaError_t e = cudaSuccess;

  // ---- forward, recording S at the start of every segment.  Step n
  // produces S_{n+1}; it records when n + 1 is a multiple of K.  Runs of K
  // steps whose first step records (and whose last is not the final step)
  // replay a captured graph with the checkpoint pointer replaced.
  if (!h->cap_stream) {
    e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return LTNE_ERR_CUDA;
  }
  auto fwd_step = [&](cudaStream_t s_, int src_buf, int wm, C* rec, bool chained) {
    const C* src = reinterpret_cast<const C*>(h->ws + h->off_pop[src_buf]);
    C* dst = reinterpret_cast<C*>(h->ws + h->off_pop[src_buf ^ 1]);
    return launch_chained(chained, k_step_record<C>, grd, blk, s_, src, dst, phi, mac, P, nx, ny,
                          pitch, plane, wm, rec);
  };
  bool after_kernel = false;  // the stream's last operation is a kernel above
  SegGraph gf[2];
  int64_t n = 0;
  while (n < N && e == cudaSuccess) {
    const int64_t a = n + 1;
    const bool records = (a % K == 0) && a < N;
    if (records && K > 1 && n + K < N) {
      const int par = h->cur;
      if (!gf[par].exec)
        e = gf[par].capture(h->cap_stream, [&](cudaStream_t cs) {
          int b = par;
          cudaError_t le = cudaSuccess;
          for (int j = 0; j < K && le == cudaSuccess; ++j) {
            le = fwd_step(cs, b, 0, j == 0 ? buf19(L.ckpt, 1) : nullptr, j > 0);
            b ^= 1;
          }
          return le;
        });
      if (e != cudaSuccess) break;
      const C* src = reinterpret_cast<const C*>(h->ws + h->off_pop[par]);
      C* dst = reinterpret_cast<C*>(h->ws + h->off_pop[par ^ 1]);
      C* rec = buf19(L.ckpt, a / K);
      int wm = 0;
      int inx = nx, iny = ny;
      int64_t ipitch = pitch, iplane = plane;
      NodeParams<C> iP = P;
      const C* iphi = phi;
      C* imac = mac;
      void* args[] = {&src, &dst, &iphi, &imac, &iP, &inx, &iny, &ipitch, &iplane, &wm, &rec};
      e = gf[par].launch(reinterpret_cast<void*>(k_step_record<C>), grd, blk, args, st);
      after_kernel = false;
      if (K & 1) h->cur ^= 1;
      h->step += K;
      h->launches += K;
      n += K;
    } else {
      e = fwd_step(st, h->cur, n == N - 1 ? 1 : 0, records ? buf19(L.ckpt, a / K) : nullptr,
                   after_kernel);
      after_kernel = true;
      h->cur ^= 1;
      ++h->step;
      ++h->launches;
      ++n;
    }
  }
  if (e != cudaSuccess) return LTNE_ERR_CUDA;
  double acc[NACC];
  rc = reduce_handle(h, acc);
  if (rc != LTNE_OK) return rc;
  DerivedInfo info;
  info.L = h->L;
  info.nu_f = h->nu_f;
  info.alpha_f = h->alpha_f;
  ltne_obs ob;
  finish_observables(h->p, info, h->step, false, acc, &ob);
  h->have_prev = true;
  *J = 0.5 * (ob.Nu_f_hot + ob.Nu_s_hot);

  // ---- reverse
  e = cudaMemsetAsync(ws + L.lam, 0, 2 * L.p19, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ws + L.phib, 0, 3 * L.pl, st);  // phib, hb, wphib
  if (e != cudaSuccess) return LTNE_ERR_CUDA;
  after_kernel = false;
  C* lamL = buf19(L.lam, 0);
  C* lamO = buf19(L.lam, 1);
  const C inv_dT = C(1.0 / (h->p.T_hot - h->p.T_cold));
  const int64_t n19 = 19 * plane;
  bool capped = h->adj_sched == LTNE_ADJ_CAPPED;
  if (h->adj_sched == LTNE_ADJ_AUTO) {
    // all registers when the transposed-collision grid fits one wave
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adj_main<C, false>,
                                                        (int)(blk.x * blk.y), 0);
    if (e != cudaSuccess) return LTNE_ERR_CUDA;
    capped = (int64_t)grd.x * grd.y > (int64_t)sms * per_sm;
  }
  // Slot set q holds a segment's states: slot 0 (S_a, copied from its
  // checkpoint) and K recomputed slots.  The sweep reverses segment s from
  // one set while segment s - 1 is recomputed into the other on a second
  // stream: at small lattices every kernel is a single wave bound by one
  // thread's latency, and the two chains share the SMs.
  const dim3 cgrid(1216), cblk(256);
  auto slot = [&](int q, int64_t j) {
    return j == 0 ? buf19(L.seg0, q) : buf19(L.slots, (int64_t)q * K + j - 1);
  };
  // Copy of the checkpoint into slot 0 (a graph's root), then the recompute.
  auto recompute_body = [&](cudaStream_t s_, int64_t len, const C* ckpt, int q, bool chained) {
    cudaError_t le = launch_chained(chained, k_copy19<C>, cgrid, cblk, s_, ckpt, slot(q, 0), n19);
    C* p0 = buf19(L.pops, 0);
    C* p1 = buf19(L.pops, 1);
    if (le == cudaSuccess)
      le = launch_chained(true, k_collide_pre<C>, grd, blk, s_, (const C*)slot(q, 0), p0, phi, P,
                          nx, ny, pitch, plane);
    for (int64_t j = 1; j <= len && le == cudaSuccess; ++j) {
      le = launch_chained(true, k_step_record<C>, grd, blk, s_, (const C*)p0, p1, phi, mac, P,
                          nx, ny, pitch, plane, 0, slot(q, j));
      C* t = p0;
      p0 = p1;
      p1 = t;
    }
    return le;
  };
  // The reverse sweep over set q (the seed first on the last segment); the
  // segment that starts at step 0 does not fold its last adjoint (the
  // initial state's wall nodes were not rebuilt).
  auto reverse_body = [&](cudaStream_t s_, int64_t len, int q, bool seed, C*& lL, C*& lO,
                          bool chained, bool initial) {
    cudaError_t le = cudaSuccess;
    if (seed) {
      le = launch_chained(chained, k_adj_seed<C>, dim3((2 * ny + 255) / 256), dim3(256), s_,
                          (const C*)slot(q, len), lL, phi, phib, hb, wphib, P, nx, ny, pitch,
                          plane, inv_dT);
      chained = true;
    }
    for (int64_t j = len - 1; j >= 0 && le == cudaSuccess; --j) {
      const int fold = (initial && j == 0) ? 0 : 1;
      const C* pre = j > 0 ? slot(q, j - 1) : nullptr;
      if (capped)
        le = launch_chained(chained, k_adj_main<C, true>, grd, blk, s_, (const C*)lL, lO,
                            (const C*)slot(q, j), phi, phib, hb, wphib, P, nx, ny, pitch, plane,
                            fold, pre);
      else
        le = launch_chained(chained, k_adj_main<C, false>, grd, blk, s_, (const C*)lL, lO,
                            (const C*)slot(q, j), phi, phib, hb, wphib, P, nx, ny, pitch, plane,
                            fold, pre);
      chained = true;
      C* t = lL;
      lL = lO;
      lO = t;
    }
    return le;
  };
  if (!h->aux_stream) {
    e = cudaStreamCreateWithFlags(&h->aux_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return LTNE_ERR_CUDA;
  }
  EventPair ev;
  if (ev.create() != cudaSuccess) return LTNE_ERR_CUDA;
  const cudaStream_t st2 = h->aux_stream;
  // Reverse of segment s on `main_s` while segment s - 1 (if any) is
  // recomputed on `aux`, joined at the end.
  auto iteration = [&](cudaStream_t main_s, cudaStream_t aux, int64_t s, int q, C*& lL, C*& lO,
                       bool chained) {
    const int64_t a = s * K, len = ((a + K < N) ? a + K : N) - a;
    cudaError_t le = cudaSuccess;
    bool forked = false;
    if (s > 0) {
      le = cudaEventRecord(ev.fork, main_s);
      if (le == cudaSuccess) le = cudaStreamWaitEvent(aux, ev.fork, 0);
      forked = le == cudaSuccess;
      if (le == cudaSuccess) le = recompute_body(aux, K, buf19(L.ckpt, s - 1), q ^ 1, false);
      chained = false;
    }
    if (le == cudaSuccess)
      le = reverse_body(main_s, len, q, s == L.nseg - 1, lL, lO, chained, s == 0);
    if (forked) {  // the main stream waits for the recompute even after a failure
      cudaError_t je = cudaEventRecord(ev.join, aux);
      if (je == cudaSuccess) je = cudaStreamWaitEvent(main_s, ev.join, 0);
      if (le == cudaSuccess) le = je;
    }
    return le;
  };
  // Full segments other than the last and the first replay one captured
  // iteration per (slot set, adjoint-buffer parity); its root copies
  // segment s - 1's checkpoint into slot 0 of the other set, the only
  // argument that changes between replays.
  SegGraph gr[2][2];
  int q = 0;
  const int64_t last = L.nseg - 1;
  e = recompute_body(st, N - last * K, buf19(L.ckpt, last), q, after_kernel);
  after_kernel = true;
  for (int64_t s = last; s >= 0 && e == cudaSuccess; --s) {
    if (s != last && s > 0 && K > 1) {
      const int lp = (lamL == buf19(L.lam, 0)) ? 0 : 1;
      SegGraph& g = gr[q][lp];
      if (!g.exec)
        e = g.capture(h->cap_stream, [&](cudaStream_t cs) {
          C* seg_next = slot(q ^ 1, 0);
          k_copy19<C><<<cgrid, cblk, 0, cs>>>(buf19(L.ckpt, 0), seg_next, n19);
          cudaError_t le = cudaGetLastError();
          if (le == cudaSuccess) le = cudaEventRecord(ev.fork, cs);
          if (le == cudaSuccess) le = cudaStreamWaitEvent(st2, ev.fork, 0);
          const bool forked = le == cudaSuccess;
          // the recompute without its copy (the root)
          C* p0 = buf19(L.pops, 0);
          C* p1 = buf19(L.pops, 1);
          if (le == cudaSuccess)
            le = launch_chained(false, k_collide_pre<C>, grd, blk, st2, (const C*)seg_next, p0,
                                phi, P, nx, ny, pitch, plane);
          for (int64_t j = 1; j <= K && le == cudaSuccess; ++j) {
            le = launch_chained(true, k_step_record<C>, grd, blk, st2, (const C*)p0, p1, phi,
                                mac, P, nx, ny, pitch, plane, 0, slot(q ^ 1, j));
            C* t = p0;
            p0 = p1;
            p1 = t;
          }
          C* lL = buf19(L.lam, lp);
          C* lO = buf19(L.lam, lp ^ 1);
          if (le == cudaSuccess) le = reverse_body(cs, K, q, false, lL, lO, false, false);
          // rejoin the second stream even after a failed launch, so that the
          // capture can end and leave it usable
          if (forked) {
            cudaError_t je = cudaEventRecord(ev.join, st2);
            if (je == cudaSuccess) je = cudaStreamWaitEvent(cs, ev.join, 0);
            if (le == cudaSuccess) le = je;
          }
          return le;
        });
      if (e != cudaSuccess) break;
      const C* src = buf19(L.ckpt, s - 1);
      C* dst = slot(q ^ 1, 0);
      int64_t cnt = n19;
      void* args[] = {&src, &dst, &cnt};
      e = g.launch(reinterpret_cast<void*>(k_copy19<C>), cgrid, cblk, args, st);
      if (K & 1) {
        C* t = lamL;
        lamL = lamO;
        lamO = t;
      }
    } else {
      e = iteration(st, st2, s, q, lamL, lamO, after_kernel);
    }
    after_kernel = false;
    q ^= 1;
  }
  if (e != cudaSuccess) return LTNE_ERR_CUDA;
  // ---- outputs
  k_add_wall_phib<C><<<grd, blk, 0, st>>>(phib, wphib, nx, ny, pitch);
  k_sum_plane<C><<<kSumBlocks, kRB, 0, st>>>(hb, nx, ny, pitch, part);
  k_sum_partials<<<1, 32, 0, st>>>(part, kSumBlocks, part + kSumBlocks);
  e = cudaGetLastError();
  if (e == cudaSuccess && dJ_dphi)
    e = cudaMemcpy2DAsync(dJ_dphi, (size_t)nx * sizeof(C), phib, (size_t)pitch * sizeof(C),
                          (size_t)nx * sizeof(C), (size_t)ny, cudaMemcpyDeviceToDevice, st);
  double hsum = 0.0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&hsum, part + kSumBlocks, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return LTNE_ERR_CUDA;
  // h_v/(rho c)_f = H alpha_f / L^2
  *dJ_dH = hsum * h->alpha_f / (h->L * h->L);
  return LTNE_OK;
}

}  // namespace

extern "C" {

int ltne_set_adjoint_schedule(ltne_handle* h, int32_t mode) {
  if (!h || mode < LTNE_ADJ_AUTO || mode > LTNE_ADJ_CAPPED) return LTNE_ERR_INVALID_ARG;
  h->adj_sched = mode;
  return LTNE_OK;
}

int ltne_get_adjoint_schedule(const ltne_handle* h, int32_t* mode) {
  if (!h || !mode) return LTNE_ERR_INVALID_ARG;
  *mode = h->adj_sched;
  return LTNE_OK;
}

size_t ltne_adjoint_workspace_bytes(const ltne_handle* h, int64_t n_steps, int32_t segment) {
  if (!h || n_steps < 1 || segment < 1 || h->slab) return 0;
  return adj_layout(h, n_steps, segment).total;
}

int ltne_adjoint(ltne_handle* h, const double* porosity, const double* rho, const double* T_f,
                 const double* T_s, int64_t n_steps, int32_t segment, void* adj_workspace,
                 size_t bytes, void* dJ_dphi, double* J, double* dJ_dH) {
  if (!h || !porosity || !J || !dJ_dH || n_steps < 1 || segment < 1 || !adj_workspace ||
      h->slab)
    return LTNE_ERR_INVALID_ARG;
  if (!h->ws) return LTNE_ERR_STATE;
  const ltne_params& p = h->p;
  if (p.bc != LTNE_BC_CAVITY || !p.porosity_field || p.hv_local ||
      (p.storage != LTNE_F32 && p.storage != LTNE_F64) || p.T_hot == p.T_cold)
    return LTNE_ERR_INVALID_ARG;
  if (bytes < ltne_adjoint_workspace_bytes(h, n_steps, segment) ||
      (reinterpret_cast<uintptr_t>(adj_workspace) & 255u) != 0)
    return LTNE_ERR_WORKSPACE;
  char* ws = static_cast<char*>(adj_workspace);
  if (p.storage == LTNE_F64)
    return run_adjoint<double>(h, porosity, rho, T_f, T_s, n_steps, segment, ws, dJ_dphi, J,
                               dJ_dH);
  return run_adjoint<float>(h, porosity, rho, T_f, T_s, n_steps, segment, ws, dJ_dphi, J, dJ_dH);
}

}  // extern "C"
