// ltne_tma.cuh -- the two-node time step with the population tiles staged
// in shared memory by the tensor memory accelerator (TMA), for cavity
// lattices.
//
// A persistent block walks tiles of W = 2 TX nodes x H = TY rows.  For each
// tile one thread asks the TMA for a single 3-D box of all 19 population
// planes covering the tile plus a one-row and A-column halo (A = 16 bytes
// of the storage type, so that every box starts on a 16-byte boundary);
// the box lands in one of LTNE_TMA_STAGES shared-memory stages and arrives
// on that stage's mbarrier.  While the block computes tile k, the boxes of
// the next tiles stream into the other stages, so the HBM latency is meant
// to be hidden by the copy engine instead of by resident warps (the
// two-node step holds about 96 registers per thread, 20 warps per SM).  Interior pairs pull
// their 19 values from the staged box and then run exactly the code of the
// direct-load two-node kernel (finish_pair), so both kernels give the same
// bits; pairs on a wall row or next to a wall column take the direct-load
// path.  Rows and columns outside the lattice arrive as zeros (TMA
// out-of-bounds fill) and are never used by interior pairs.
//
// Every wait on an mbarrier is bounded: after kWaitSpins polls the block
// records an error flag, waits once more (bounded) for its copies in flight,
// and leaves; the host reports LTNE_ERR_TIMEOUT on the next observables call.
// A copy can be neither cancelled nor waited for without limit, so if that
// second wait gives up too, the block leaves with copies still in flight,
// which may land in shared memory given to a later block of the same
// launch: the error flag is already set, and the state of such a step is
// reported invalid and must be discarded.
#pragma once

#include <cuda.h>

#include <mutex>

#include "ltne_pair.cuh"

namespace ltne {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

constexpr int kWaitSpins = 1 << 22;  // about a second of polling with back-off

// Waits for the phase with the given parity of an mbarrier; false if it has
// not completed after `spins` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          int spins = kWaitSpins) {
  for (int i = 0; i < spins; ++i) {
    if (mbar_test(bar, parity)) return true;
    if (i >= 32) __nanosleep(64);
  }
  return false;
}

// One TMA load of a 3-D box at (x, y, z) of the tensor map into shared
// memory at dst, completing on bar.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

// Geometry of a staged tile for storage type S, a TX x TY block and NS
// stages.
template <typename S, int TX, int TY, int NS>
struct TileBox {
  static constexpr int A = 16 / (int)sizeof(S);  // halo columns (16 bytes)
  static constexpr int W = 2 * TX, H = TY;       // nodes of the tile
  static constexpr int BW = W + 2 * A, BH = H + 2;
  static constexpr int kPlane = BW * BH;          // elements per staged plane
  static constexpr int kBytes = 19 * kPlane * (int)sizeof(S);
  static constexpr int kStride = (kBytes + 127) / 128 * 128;  // stage stride (TMA: 128-B aligned)
  static constexpr int kSmem = NS * kStride + 8 * NS;         // stages + one mbarrier each
};

// The 19 values streaming into the interior pair whose even node sits at
// column c, row r of the staged box (value i from (x - e_i, y - e_i)).
template <typename S, int BW, int kPlane>
__device__ __forceinline__ void pull_staged(const S* __restrict__ sb, int r, int c, float inv_scale,
                                            F2 (&f)[9], F2 (&gf)[5], F2 (&gs)[5]) {
  auto at = [&](int k, int row, int col) { return sb + k * kPlane + row * BW + col; };
  auto pair = [&](int k, int row) { return PairIO<S>::ld2(at(k, row, c), inv_scale); };
  auto left = [&](int k, int row) {
    return PairIO<S>::ld11(at(k, row, c - 1), at(k, row, c), inv_scale);
  };
  auto right = [&](int k, int row) {
    return PairIO<S>::ld11(at(k, row, c + 1), at(k, row, c + 2), inv_scale);
  };
  // rows: r - 1 holds y - 1 (values streaming up, e_y = +1), r + 1 holds y + 1
  f[0] = pair(0, r);
  f[1] = left(1, r);
  f[2] = pair(2, r - 1);
  f[3] = right(3, r);
  f[4] = pair(4, r + 1);
  f[5] = left(5, r - 1);
  f[6] = right(6, r - 1);
  f[7] = right(7, r + 1);
  f[8] = left(8, r + 1);
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    F2(&g)[5] = t == 0 ? gf : gs;
    const int k0 = t == 0 ? 9 : 14;
    g[0] = pair(k0, r);
    g[1] = left(k0 + 1, r);
    g[2] = pair(k0 + 2, r - 1);
    g[3] = right(k0 + 3, r);
    g[4] = pair(k0 + 4, r + 1);
  }
}

template <typename S, int TX, int TY, int NS>
__global__ void __launch_bounds__(TX * TY, kPairMinBlocks) k_step_tma(
    const __grid_constant__ CUtensorMap tmap, const S* __restrict__ src, S* __restrict__ dst,
    const float* __restrict__ phi_field, float* __restrict__ mac, const NodeParams<F2> P,
    const NodeParams<float> P1, const int nx, const int ny, const int64_t pitch,
    const int64_t plane, const float scale, const float inv_scale, const int write_macros,
    const uint32_t* __restrict__ tick_in, uint32_t* __restrict__ tick_out,
    const float* __restrict__ um_in, float* __restrict__ um_out, int* __restrict__ err) {
  using B = TileBox<S, TX, TY, NS>;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + NS * B::kStride);
  const uint32_t tick = read_tick<S, float>(tick_in, tick_out);
  const int tid = threadIdx.y * TX + threadIdx.x;
  const int tiles_x = (nx + B::W - 1) / B::W;
  const int ntiles = tiles_x * ((ny + B::H - 1) / B::H);
  const uint32_t pi = (uint32_t)pitch, pl = (uint32_t)plane;
  if (tid == 0) {
    for (int i = 0; i < NS; ++i) mbar_init(&bar[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int tile, int stage) {  // thread 0 only
    const int x0 = (tile % tiles_x) * B::W, y0 = (tile / tiles_x) * B::H;
    mbar_expect_tx(&bar[stage], (uint32_t)B::kBytes);
    tma_load_3d(smem + stage * B::kStride, &tmap, &bar[stage], x0 - B::A, y0 - 1, 0);
  };
  // the block's j-th tile is blockIdx.x + j gridDim.x, staged in stage j % NS;
  // the first NS - 1 are requested up front, then one more per tile
  if (tid == 0)
    for (int j = 0; j < NS - 1; ++j) {
      const int tj = blockIdx.x + j * gridDim.x;
      if (tj < ntiles) issue(tj, j);
    }
  int t = blockIdx.x;
  for (int k = 0; t < ntiles; ++k, t += gridDim.x) {
    const int s = k % NS;
    const uint32_t parity = (uint32_t)((k / NS) & 1);
    const bool ok = mbar_wait(&bar[s], parity);
    // every thread has also finished the previous tile: its stage is free
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicExch(err, 1);
        // the copies in flight: this tile's and those of the next NS - 2
        for (int j = 0; j < NS - 1; ++j) {
          const int kj = k + j;
          if (blockIdx.x + kj * gridDim.x < ntiles)
            mbar_wait(&bar[kj % NS], (uint32_t)((kj / NS) & 1));
        }
      }
      return;
    }
    const int tn = t + (NS - 1) * gridDim.x;
    if (tn < ntiles && tid == 0) issue(tn, (k + NS - 1) % NS);
    const int x0 = (t % tiles_x) * B::W + 2 * (int)threadIdx.x;
    const int y = (t / tiles_x) * B::H + (int)threadIdx.y;
    if (x0 >= nx || y >= ny) continue;
    const bool interior = x0 > 0 && x0 + 2 < nx && y > 0 && y < ny - 1;
    if (interior) {
      const S* sb = reinterpret_cast<const S*>(smem + s * B::kStride);
      F2 f[9], gf[5], gs[5];
      pull_staged<S, B::BW, B::kPlane>(sb, (int)threadIdx.y + 1, B::A + 2 * (int)threadIdx.x,
                                       inv_scale, f, gf, gs);
      finish_pair<S>(dst, phi_field, mac, P, (uint32_t)y * pi + (uint32_t)x0, pl, scale,
                     write_macros, tick, um_in, um_out, f, gf, gs);
    } else if (x0 > 0 && x0 + 2 < nx) {  // both nodes on a wall row
      step_pair<S, BC_CAVITY>(src, dst, phi_field, mac, P, x0, y, nx, ny, pi, pl, scale,
                              inv_scale, write_macros, tick, um_in, um_out);
    } else if (x0 + 1 < nx) {  // a wall column in the pair
      step_pair_side<S>(src, dst, phi_field, mac, P, x0, y, nx, ny, pi, pl, scale, inv_scale,
                        write_macros, tick, um_in, um_out);
    } else {  // the last node of an odd row
      step_node<S, float, BC_CAVITY>(src, dst, phi_field, mac, P1, x0, y, nx, ny, pitch, plane,
                                     scale, inv_scale, write_macros, tick, nullptr, um_in, um_out);
    }
  }
}

// cuTensorMapEncodeTiled from the driver, fetched once through the runtime.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiledFn encode_tiled_fn() {
  // initialised once, thread-safely (function-local static)
  static const EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeTiledFn>(p);
    return static_cast<EncodeTiledFn>(nullptr);
  }();
  return fn;
}

// Launch facts of one staged-kernel instantiation on one device: the
// dynamic shared memory attribute is set and the occupancy and SM count
// are queried once per device, under a lock (host threads may launch on
// several devices at once).
struct TmaLaunchInfo {
  int blocks_per_sm = 0, sms = 0;
};
constexpr int kTmaMaxDevices = 64;

// Tensor map of a population buffer: dims (pitch, ny, 19 planes) of the
// storage type, box (BW, BH, 19), zeros outside.
template <typename S, int TX, int TY>
cudaError_t make_tile_map(CUtensorMap* map, const void* base, int64_t pitch, int ny,
                          int64_t plane) {
  using B = TileBox<S, TX, TY, 1>;
  EncodeTiledFn fn = encode_tiled_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[3] = {(cuuint64_t)pitch, (cuuint64_t)ny, 19};
  const cuuint64_t strides[2] = {(cuuint64_t)pitch * sizeof(S), (cuuint64_t)plane * sizeof(S)};
  const cuuint32_t box[3] = {(cuuint32_t)B::BW, (cuuint32_t)B::BH, 19};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUtensorMapDataType dt = sizeof(S) == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16
                                                : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const CUresult r = fn(map, dt, 3, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Pipeline depth of the staged kernel (tiles requested ahead: stages - 1).
// Measured at 8192^2 FP16 with 32 x 4 blocks: 2 stages 47.9 GLUPS, 3 stages
// 39.8, 4 stages 34.5 (each stage costs resident blocks); the direct-load
// two-node kernel runs at 60.3, so staging is off by default.
#ifndef LTNE_TMA_STAGES
#define LTNE_TMA_STAGES 2
#endif

template <typename S, int TX, int TY>
cudaError_t launch_tma_shape(const LatticeArgs& a, const NodeParams<double>& Pd,
                             cudaStream_t st) {
  constexpr int NS = LTNE_TMA_STAGES;
  using B = TileBox<S, TX, TY, NS>;
  CUtensorMap map;
  cudaError_t e = make_tile_map<S, TX, TY>(&map, a.src, a.pitch, a.ny, a.plane);
  if (e != cudaSuccess) return e;
  static TmaLaunchInfo info[kTmaMaxDevices];
  static std::mutex mu;
  int dev = 0, blocks_per_sm = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kTmaMaxDevices)
    return cudaErrorInvalidDevice;
  {
    std::lock_guard<std::mutex> lock(mu);
    TmaLaunchInfo& li = info[dev];
    if (!li.blocks_per_sm) {
      int nb = 0, n_sm = 0;
      if (cudaFuncSetAttribute(k_step_tma<S, TX, TY, NS>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               B::kSmem) != cudaSuccess ||
          cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_tma<S, TX, TY, NS>, TX * TY,
                                                        B::kSmem) != cudaSuccess ||
          nb < 1)
        return cudaErrorInvalidConfiguration;
      li.sms = n_sm;
      li.blocks_per_sm = nb;
    }
    blocks_per_sm = li.blocks_per_sm;
    sms = li.sms;
  }
  const int ntiles = ((a.nx + B::W - 1) / B::W) * ((a.ny + B::H - 1) / B::H);
  const int grid = ntiles < blocks_per_sm * sms ? ntiles : blocks_per_sm * sms;
  const NodeParams<F2> P = cast_params<F2>(Pd);
  const NodeParams<float> P1 = cast_params<float>(Pd);
  k_step_tma<S, TX, TY, NS><<<grid, dim3(TX, TY), B::kSmem, st>>>(
      map, static_cast<const S*>(a.src), static_cast<S*>(a.dst),
      static_cast<const float*>(a.phi), static_cast<float*>(a.mac), P, P1, a.nx, a.ny, a.pitch,
      a.plane, a.enc_scale, 1.0f / a.enc_scale, a.write_macros, a.tick_in, a.tick_out,
      static_cast<const float*>(a.um_in), static_cast<float*>(a.um_out), a.err);
  return cudaGetLastError();
}

// The staged kernel's tile follows the schedule's block shape: 32 x 4,
// 64 x 2 or 32 x 2 threads (any other shape runs as 32 x 4).
template <typename S>
cudaError_t launch_step_tma_t(const LatticeArgs& a, const NodeParams<double>& Pd, StepShape s,
                              cudaStream_t st) {
  if (a.bc != BC_CAVITY || !a.err) return cudaErrorInvalidValue;
  if (s.bx == 64 && s.by == 2) return launch_tma_shape<S, 64, 2>(a, Pd, st);
  if (s.bx == 32 && s.by == 2) return launch_tma_shape<S, 32, 2>(a, Pd, st);
  return launch_tma_shape<S, 32, 4>(a, Pd, st);
}

}  // namespace ltne

// Launchers of a storage type with FP32 arithmetic: the schedule picks one
// or two nodes per thread, and the staged or the direct-load two-node form.
#define LTNE_DEFINE_FLOAT_LAUNCHERS(tag, S)                                                     \
  namespace ltne {                                                                             \
  cudaError_t launch_step_##tag(const LatticeArgs& a, const NodeParams<double>& P,             \
                                StepShape s, cudaStream_t st) {                                \
    return s.tma    ? launch_step_tma_t<S>(a, P, s, st)                                       \
           : s.pair ? launch_step_pair_t<S>(a, P, s, st)                                      \
                    : launch_step_t<S, float>(a, P, s, st);                                   \
  }                                                                                            \
  cudaError_t launch_init_##tag(const LatticeArgs& a, const NodeParams<double>& P,             \
                                cudaStream_t st) {                                             \
    return launch_init_t<S, float>(a, P, st);                                                  \
  }                                                                                            \
  }
