// ltne_batch.cu -- batched form: many independent cavities of uneven size
// and parameters advanced by one persistent launch per time step, replayed
// from a captured CUDA graph.  The per-node work is the same step_node() as
// the single-lattice kernel (collision, streaming and walls of Liu & He's
// three-distribution MRT-LB method, arXiv:1608.04118).
//
// Work decomposition: every cavity is cut into tiles of TX x TY nodes; the
// tile list (cavity, origin and the cavity's geometry per tile) is built on
// the host for the schedule the autotuner picked.  Either one block per tile
// (k_batch_tile: the block reads its descriptor and the cavity constants
// straight from global memory) or a persistent grid whose blocks walk the
// list with a stride of the grid size, staging each tile's constants in
// shared memory (k_batch_step).  A thread updates NPT = 1 node, or NPT = 2
// neighbouring nodes in paired FP32 arithmetic (the two-node step of
// ltne_pair.cuh).  FP32 storage and arithmetic, uniform porosity per cavity.
#include <math.h>
#include <string.h>

#include <vector>

#include "ltne.h"
#include "ltne_internal.h"
#include "ltne_pair.cuh"

using namespace ltne;

namespace {

constexpr int kGraphSteps = 32;

// A cavity's constants for the one-node step (P) and, lane-broadcast, for
// the two-node step (P2).
struct BatchConst {
  NodeParams<float> P;
  NodeParams<F2> P2;
};

struct BatchCavity {
  int32_t nx, ny;
  int64_t pitch, plane;
  int64_t pop_off;  // element offset of the cavity's 19 planes in either buffer
  int64_t mac_off;  // element offset of its 5 macro planes
  int64_t prev_off; // element offset of its 4 residual snapshot planes
  BatchConst K;
};

static_assert(sizeof(NodeParams<float>) % sizeof(uint32_t) == 0, "NodeParams<float> layout");
static_assert(sizeof(BatchConst) % sizeof(uint32_t) == 0, "BatchConst layout");
constexpr int kMinBlockThreads = 64;  // every schedule has at least this many

// One tile of the list: its cavity, origin, and the cavity geometry a tile
// needs (copied from the cavity table, so that a block reads one descriptor
// and can issue its population loads without a dependent second lookup).
struct TileDesc {
  int32_t c, x0, y0, nx, ny, pad;
  int64_t pitch, plane, pop_off, mac_off;
};

// The step of the nodes a thread owns in tile d: one node, or a pair of
// neighbouring nodes (two-node step where both are off the side walls).
template <int NPT>
__device__ __forceinline__ void tile_nodes(const float* __restrict__ src, float* __restrict__ dst,
                                           float* __restrict__ mac, const TileDesc& d,
                                           const BatchConst& K, int lx, int ly,
                                           int write_macros) {
  const float* s = src + d.pop_off;
  float* o = dst + d.pop_off;
  float* m = mac + d.mac_off;
  const int y = d.y0 + ly;
  if constexpr (NPT == 1) {
    const int x = d.x0 + lx;
    if (x < d.nx && y < d.ny)
      step_node<float, float, BC_CAVITY>(s, o, nullptr, m, K.P, x, y, d.nx, d.ny, d.pitch,
                                         d.plane, 1.0f, 1.0f, write_macros, 0u);
  } else {
    const int x0 = d.x0 + 2 * lx;
    if (x0 < d.nx && y < d.ny) {
      if (x0 > 0 && x0 + 2 < d.nx) {
        step_pair<float, BC_CAVITY>(s, o, nullptr, m, K.P2, x0, y, d.nx, d.ny,
                                    (uint32_t)d.pitch, (uint32_t)d.plane, 1.0f, 1.0f,
                                    write_macros, 0u, nullptr, nullptr);
      } else if (x0 + 1 < d.nx) {  // a wall column in the pair
        step_pair_side<float>(s, o, nullptr, m, K.P2, x0, y, d.nx, d.ny, (uint32_t)d.pitch,
                              (uint32_t)d.plane, 1.0f, 1.0f, write_macros, 0u, nullptr,
                              nullptr);
      } else {  // the last node of an odd row
        step_node<float, float, BC_CAVITY>(s, o, nullptr, m, K.P, x0, y, d.nx, d.ny, d.pitch,
                                           d.plane, 1.0f, 1.0f, write_macros, 0u);
      }
    }
  }
}

// One block per tile: the block reads its descriptor and takes the cavity
// constants straight from the cavity table (uniform loads through the
// read-only cache), with no staging and no barrier.
template <int NPT>
__global__ void __launch_bounds__(NPT == 1 ? 256 : kPairMaxThreads, NPT == 1 ? 4 : kPairMinBlocks)
    k_batch_tile(const float* __restrict__ src, float* __restrict__ dst, float* __restrict__ mac,
                 const BatchCavity* __restrict__ cav, const TileDesc* __restrict__ tiles,
                 int tx_log2, int write_macros) {
  const TileDesc d = tiles[blockIdx.x];
  const int tid = threadIdx.x;
  tile_nodes<NPT>(src, dst, mac, d, cav[d.c].K, tid & ((1 << tx_log2) - 1), tid >> tx_log2,
                  write_macros);
}

// Persistent form: a grid of `blocks` blocks walks the tile list with a
// stride of the grid size (round-robin, so block loads differ by at most
// one tile), each tile exactly as in k_batch_tile.
template <int NPT>
__global__ void __launch_bounds__(NPT == 1 ? 256 : kPairMaxThreads, NPT == 1 ? 4 : kPairMinBlocks)
    k_batch_step(const float* __restrict__ src, float* __restrict__ dst, float* __restrict__ mac,
                 const BatchCavity* __restrict__ cav, const TileDesc* __restrict__ tiles,
                 int ntiles, int tx_log2, int write_macros) {
  const int tid = threadIdx.x;
  const int lx = tid & ((1 << tx_log2) - 1), ly = tid >> tx_log2;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const TileDesc d = tiles[t];
    tile_nodes<NPT>(src, dst, mac, d, cav[d.c].K, lx, ly, write_macros);
  }
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int fail_cuda(cudaError_t e) {
  if (e == cudaSuccess) return LTNE_OK;
  cudaGetLastError();
  return LTNE_ERR_CUDA;
}

}  // namespace

struct ltne_batch {
  int count = 0;
  std::vector<ltne_params> p;
  std::vector<DerivedInfo> info;
  std::vector<NodeParams<double>> Pd;
  std::vector<BatchCavity> cav;
  std::vector<bool> have_prev;
  cudaStream_t stream = nullptr, cap_stream = nullptr;
  // layout (bytes)
  int64_t pop_elems = 0, mac_elems = 0, prev_elems = 0, max_tiles = 0;
  int max_red_blocks = 1;
  size_t off_pop[2] = {0, 0}, off_mac = 0, off_prev = 0, off_part = 0, off_out = 0, off_cav = 0,
         off_tiles = 0, ws_bytes = 0;
  char* ws = nullptr;
  // schedule
  int tx = 128, ty = 2, blocks = 0, npt = 1;
  int64_t ntiles = 0;
  bool schedule_uploaded = false;
  // state
  int cur = 0;
  int64_t step = 0, launches = 0, nodes = 0;
  bool fields_set = false;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
};

namespace {

int64_t count_tiles(const ltne_batch* b, int tx, int ty) {
  int64_t n = 0;
  for (const auto& c : b->cav) n += (int64_t)((c.nx + tx - 1) / tx) * ((c.ny + ty - 1) / ty);
  return n;
}

// Tiles of tx x ty nodes, npt nodes per thread: tx / npt threads across
// (32..256, a power of two), ty in 1..8 (a power of two), 64 to 256 threads
// per block (64 to 128 with two nodes per thread).
bool valid_shape(int tx, int ty, int npt) {
  if (npt != 1 && npt != 2) return false;
  const int txt = tx / npt;
  if (tx % npt != 0 || txt < 32 || txt > 256 || (txt & (txt - 1)) != 0) return false;
  if (ty < 1 || ty > 8 || (ty & (ty - 1)) != 0) return false;
  const int threads = txt * ty;
  return threads >= kMinBlockThreads && threads <= (npt == 1 ? 256 : kPairMaxThreads);
}

void drop_graphs(ltne_batch* b) {
  for (auto& g : b->graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

int upload_schedule(ltne_batch* b) {
  std::vector<TileDesc> tl;
  tl.reserve((size_t)count_tiles(b, b->tx, b->ty));
  for (int c = 0; c < b->count; ++c) {
    const BatchCavity& cv = b->cav[c];
    for (int y0 = 0; y0 < cv.ny; y0 += b->ty)
      for (int x0 = 0; x0 < cv.nx; x0 += b->tx)
        tl.push_back(TileDesc{c, x0, y0, cv.nx, cv.ny, 0, cv.pitch, cv.plane, cv.pop_off,
                              cv.mac_off});
  }
  b->ntiles = (int64_t)tl.size();
  if (b->ntiles > b->max_tiles) return LTNE_ERR_INVALID_ARG;
  cudaError_t e = cudaMemcpyAsync(b->ws + b->off_tiles, tl.data(), tl.size() * sizeof(TileDesc),
                                  cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return fail_cuda(e);
  b->schedule_uploaded = true;
  drop_graphs(b);
  return LTNE_OK;
}

cudaError_t launch_batch_step(ltne_batch* b, int src_buf, int write_macros, cudaStream_t st) {
  const int txt = b->tx / b->npt;  // threads across a tile
  const int threads = txt * b->ty;
  const int64_t grid64 = b->blocks > 0 ? (int64_t)b->blocks : b->ntiles;
  const int grid = (int)(grid64 < 1 ? 1 : (grid64 > (1 << 30) ? (1 << 30) : grid64));
  int tx_log2 = 0;
  while ((1 << tx_log2) < txt) ++tx_log2;
  const float* src = reinterpret_cast<const float*>(b->ws + b->off_pop[src_buf]);
  float* dst = reinterpret_cast<float*>(b->ws + b->off_pop[src_buf ^ 1]);
  float* mac = reinterpret_cast<float*>(b->ws + b->off_mac);
  const BatchCavity* cav = reinterpret_cast<const BatchCavity*>(b->ws + b->off_cav);
  const TileDesc* tiles = reinterpret_cast<const TileDesc*>(b->ws + b->off_tiles);
  if (b->blocks == 0) {  // one block per tile
    if (b->npt == 2)
      k_batch_tile<2><<<grid, threads, 0, st>>>(src, dst, mac, cav, tiles, tx_log2, write_macros);
    else
      k_batch_tile<1><<<grid, threads, 0, st>>>(src, dst, mac, cav, tiles, tx_log2, write_macros);
  } else if (b->npt == 2) {
    k_batch_step<2><<<grid, threads, 0, st>>>(src, dst, mac, cav, tiles, (int)b->ntiles, tx_log2,
                                              write_macros);
  } else {
    k_batch_step<1><<<grid, threads, 0, st>>>(src, dst, mac, cav, tiles, (int)b->ntiles, tx_log2,
                                              write_macros);
  }
  return cudaGetLastError();
}

cudaError_t build_graph(ltne_batch* b, int parity) {
  cudaError_t e;
  if (!b->cap_stream) {
    e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
  }
  e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  int s = parity;
  cudaError_t le = cudaSuccess;
  for (int k = 0; k < kGraphSteps && le == cudaSuccess; ++k) {
    le = launch_batch_step(b, s, 0, b->cap_stream);
    s ^= 1;
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(b->cap_stream, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return le;
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(&b->graph[parity], g, 0);
  cudaGraphDestroy(g);
  return e;
}

}  // namespace

extern "C" {

int ltne_batch_create(const ltne_params* params, int32_t count, void* cuda_stream,
                      ltne_batch** out) {
  if (!params || !out || count < 1) return LTNE_ERR_INVALID_ARG;
  *out = nullptr;
  ltne_batch* b = new ltne_batch();
  b->count = count;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->p.assign(params, params + count);
  b->info.resize(count);
  b->Pd.resize(count);
  b->cav.resize(count);
  b->have_prev.assign(count, false);
  int64_t pop = 0, mac = 0, prev = 0;
  for (int c = 0; c < count; ++c) {
    const ltne_params& p = b->p[c];
    int rc = validate_params(p);
    if (rc == LTNE_OK &&
        (p.storage != LTNE_F32 || p.bc != LTNE_BC_CAVITY || p.porosity_field || p.hv_local ||
         p.thermal_correction))
      rc = LTNE_ERR_INVALID_ARG;  // the batched form is FP32 cavities with uniform porosity
    if (rc == LTNE_OK) rc = derive_params(p, nullptr, b->Pd[c], b->info[c]);
    if (rc != LTNE_OK) {
      delete b;
      return rc;
    }
    BatchCavity& cv = b->cav[c];
    cv.nx = p.nx;
    cv.ny = p.ny;
    cv.pitch = (int64_t)align_up((size_t)p.nx, 32);  // 128-byte rows
    cv.plane = cv.pitch * p.ny;
    cv.pop_off = pop;
    cv.mac_off = mac;
    cv.prev_off = prev;
    cv.K.P = cast_params<float>(b->Pd[c]);
    cv.K.P2 = cast_params<F2>(b->Pd[c]);
    pop += 19 * cv.plane;
    mac += 5 * cv.plane;
    prev += 4 * cv.plane;
    b->nodes += (int64_t)p.nx * p.ny;
    const int rb = reduce_blocks(p.nx, p.ny);
    if (rb > b->max_red_blocks) b->max_red_blocks = rb;
  }
  b->pop_elems = pop;
  b->mac_elems = mac;
  b->prev_elems = prev;
  // capacity of the tile list: the largest count over every allowed shape
  for (int npt = 1; npt <= 2; ++npt)
    for (int tx = 32; tx <= 512; tx *= 2)
      for (int ty = 1; ty <= 8; ty *= 2)
        if (valid_shape(tx, ty, npt)) {
          const int64_t t = count_tiles(b, tx, ty);
          if (t > b->max_tiles) b->max_tiles = t;
        }
  const size_t A = 256;
  size_t off = 0;
  for (int k = 0; k < 2; ++k) {
    b->off_pop[k] = off;
    off = align_up(off + (size_t)pop * sizeof(float), A);
  }
  b->off_mac = off;
  off = align_up(off + (size_t)mac * sizeof(float), A);
  b->off_prev = off;
  off = align_up(off + (size_t)prev * sizeof(float), A);
  b->off_part = off;
  off = align_up(off + (size_t)b->max_red_blocks * NACC * sizeof(double), A);
  b->off_out = off;
  off = align_up(off + (size_t)count * NACC * sizeof(double), A);
  b->off_cav = off;
  off = align_up(off + (size_t)count * sizeof(BatchCavity), A);
  b->off_tiles = off;
  off = align_up(off + (size_t)b->max_tiles * sizeof(TileDesc), A);
  b->ws_bytes = off;
  *out = b;
  return LTNE_OK;
}

size_t ltne_batch_workspace_bytes(const ltne_batch* b) { return b ? b->ws_bytes : 0; }

int64_t ltne_batch_nodes(const ltne_batch* b) { return b ? b->nodes : 0; }

int ltne_batch_bind_workspace(ltne_batch* b, void* device_ptr, size_t bytes) {
  if (!b || !device_ptr) return LTNE_ERR_INVALID_ARG;
  if (bytes < b->ws_bytes || (reinterpret_cast<uintptr_t>(device_ptr) & 255u) != 0)
    return LTNE_ERR_WORKSPACE;
  drop_graphs(b);
  b->ws = static_cast<char*>(device_ptr);
  b->fields_set = false;
  b->schedule_uploaded = false;
  cudaError_t e = cudaMemcpyAsync(b->ws + b->off_cav, b->cav.data(),
                                  b->cav.size() * sizeof(BatchCavity), cudaMemcpyHostToDevice,
                                  b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return fail_cuda(e);
  return upload_schedule(b);
}

int ltne_batch_set_schedule(ltne_batch* b, int32_t tile_x, int32_t tile_y, int32_t blocks,
                            int32_t nodes_per_thread) {
  if (!b || !valid_shape(tile_x, tile_y, nodes_per_thread) || blocks < 0)
    return LTNE_ERR_INVALID_ARG;
  if (!b->ws) return LTNE_ERR_STATE;
  b->tx = tile_x;
  b->ty = tile_y;
  b->blocks = blocks;
  b->npt = nodes_per_thread;
  return upload_schedule(b);
}

int ltne_batch_set_fields(ltne_batch* b) {
  if (!b) return LTNE_ERR_INVALID_ARG;
  if (!b->ws || !b->schedule_uploaded) return LTNE_ERR_STATE;
  // Rest state (rho = 1, u = 0, T = T_ref): all deviations zero.
  cudaError_t e = cudaMemsetAsync(b->ws + b->off_pop[0], 0, b->off_part - b->off_pop[0], b->stream);
  if (e != cudaSuccess) return fail_cuda(e);
  for (int c = 0; c < b->count && e == cudaSuccess; ++c) {
    const BatchCavity& cv = b->cav[c];
    LatticeArgs a{};
    a.src = nullptr;
    a.dst = b->ws + b->off_pop[0] + cv.pop_off * sizeof(float);
    a.phi = nullptr;
    a.mac = b->ws + b->off_mac + cv.mac_off * sizeof(float);
    a.nx = cv.nx;
    a.ny = cv.ny;
    a.bc = LTNE_BC_CAVITY;
    a.write_macros = 1;
    a.pitch = cv.pitch;
    a.plane = cv.plane;
    a.enc_scale = 1.0f;
    a.tick_in = nullptr;
    a.tick_out = nullptr;
    a.pre_out = nullptr;
    a.um_in = nullptr;
    a.um_out = nullptr;
    e = launch_init_f32(a, b->Pd[c], b->stream);
  }
  if (e != cudaSuccess) return fail_cuda(e);
  b->cur = 0;
  b->step = 0;
  b->fields_set = true;
  b->have_prev.assign(b->count, false);
  return LTNE_OK;
}

int ltne_batch_step(ltne_batch* b, int64_t n) {
  if (!b || n < 0) return LTNE_ERR_INVALID_ARG;
  if (!b->ws || !b->fields_set) return LTNE_ERR_STATE;
  if (n == 0) return LTNE_OK;
  int64_t plain = n - 1;
  cudaError_t e;
  while (plain >= kGraphSteps) {
    if (!b->graph[b->cur]) {
      e = build_graph(b, b->cur);
      if (e != cudaSuccess) return fail_cuda(e);
    }
    e = cudaGraphLaunch(b->graph[b->cur], b->stream);
    if (e != cudaSuccess) return fail_cuda(e);
    plain -= kGraphSteps;
    b->step += kGraphSteps;
    b->launches += kGraphSteps;
  }
  for (; plain > 0; --plain) {
    e = launch_batch_step(b, b->cur, 0, b->stream);
    if (e != cudaSuccess) return fail_cuda(e);
    b->cur ^= 1;
    ++b->step;
    ++b->launches;
  }
  e = launch_batch_step(b, b->cur, 1, b->stream);
  if (e != cudaSuccess) return fail_cuda(e);
  b->cur ^= 1;
  ++b->step;
  ++b->launches;
  return LTNE_OK;
}

int ltne_batch_observables(ltne_batch* b, ltne_obs* out) {
  if (!b || !out) return LTNE_ERR_INVALID_ARG;
  if (!b->ws || !b->fields_set) return LTNE_ERR_STATE;
  cudaError_t e = cudaSuccess;
  for (int c = 0; c < b->count && e == cudaSuccess; ++c) {
    const BatchCavity& cv = b->cav[c];
    ReduceArgs a;
    a.mac = b->ws + b->off_mac + cv.mac_off * sizeof(float);
    a.phi = nullptr;
    a.prev = b->ws + b->off_prev + cv.prev_off * sizeof(float);
    a.partials = reinterpret_cast<double*>(b->ws + b->off_part);  // reused in stream order
    a.out = reinterpret_cast<double*>(b->ws + b->off_out) + (size_t)c * NACC;
    a.nx = cv.nx;
    a.ny = cv.ny;
    a.pitch = cv.pitch;
    a.plane = cv.plane;
    a.phi_u = b->p[c].porosity;
    a.sigma = b->p[c].sigma;
    a.qf = b->p[c].qf;
    a.qs = b->p[c].qs;
    a.update_prev = 1;
    a.blocks = reduce_blocks(cv.nx, cv.ny);
    a.is_double = 0;
    e = launch_reduce(a, b->stream);
  }
  if (e != cudaSuccess) return fail_cuda(e);
  std::vector<double> acc((size_t)b->count * NACC);
  e = cudaMemcpyAsync(acc.data(), b->ws + b->off_out, acc.size() * sizeof(double),
                      cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return fail_cuda(e);
  int rc = LTNE_OK;
  for (int c = 0; c < b->count; ++c) {
    const int r = finish_observables(b->p[c], b->info[c], b->step, b->have_prev[c],
                                     acc.data() + (size_t)c * NACC, out + c);
    b->have_prev[c] = true;
    if (r != LTNE_OK) rc = r;
  }
  return rc;
}

int ltne_batch_get_fields(ltne_batch* b, int32_t index, double* rho, double* ux, double* uy,
                          double* T_f, double* T_s) {
  if (!b || index < 0 || index >= b->count) return LTNE_ERR_INVALID_ARG;
  if (!b->ws || !b->fields_set) return LTNE_ERR_STATE;
  const BatchCavity& cv = b->cav[index];
  const int64_t n = (int64_t)cv.nx * cv.ny;
  double* dst[5] = {rho, ux, uy, T_f, T_s};
  const double T0 = b->p[index].T_ref;
  std::vector<float> tmp((size_t)n);
  for (int k = 0; k < 5; ++k) {
    if (!dst[k]) continue;
    const char* srcp = b->ws + b->off_mac + (cv.mac_off + (int64_t)k * cv.plane) * sizeof(float);
    cudaError_t e = cudaMemcpy2DAsync(tmp.data(), (size_t)cv.nx * sizeof(float), srcp,
                                      (size_t)cv.pitch * sizeof(float),
                                      (size_t)cv.nx * sizeof(float), (size_t)cv.ny,
                                      cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return fail_cuda(e);
    const double ref = (k == 0) ? 1.0 : (k >= 3 ? T0 : 0.0);  // planes hold deviations
    for (int64_t i = 0; i < n; ++i) dst[k][i] = ref + (double)tmp[(size_t)i];
  }
  return LTNE_OK;
}

int64_t ltne_batch_launch_count(const ltne_batch* b) { return b ? b->launches : 0; }

void ltne_batch_destroy(ltne_batch* b) {
  if (!b) return;
  drop_graphs(b);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b;
}

}  // extern "C"
