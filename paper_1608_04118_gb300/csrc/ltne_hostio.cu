// ltne_hostio.cu -- the fields moved between the caller's host arrays and
// the device planes by kernels that read and write the host arrays
// themselves (no counterpart in the paper).  On a GPU that reaches pageable
// host memory through the host's page tables (Grace's memory over
// NVLink-C2C on GB300), one pass does what the staged path does in three:
// the conversion between the host's absolute FP64 values and the device's
// deviations in the compute type, the checks, and the transfer.  Each
// element is converted exactly as the staged path's host loops convert it
// (one FP64 subtraction or addition, then round to nearest), so both paths
// give the same bits.
#include "ltne_internal.h"

namespace ltne {
namespace {

constexpr int kHioThreads = 256;

dim3 hio_grid(int nx, int ny) {
  return dim3((unsigned)((nx + kHioThreads - 1) / kHioThreads), (unsigned)(ny < 65535 ? ny : 65535));
}

// dst[k][y * nx + x] = ref[k] + mac plane k at (x, y), for every given k
template <typename C>
__global__ void __launch_bounds__(kHioThreads)
    k_fields_to_host(const C* __restrict__ mac, int64_t plane, int64_t pitch, int nx, int ny,
                     HostPlanes hp) {
  const int x = blockIdx.x * kHioThreads + threadIdx.x;
  if (x >= nx) return;
  for (int y = blockIdx.y; y < ny; y += gridDim.y) {
    const int64_t off = (int64_t)y * pitch + x, i = (int64_t)y * nx + x;
#pragma unroll
    for (int k = 0; k < 5; ++k)
      if (hp.dst[k]) hp.dst[k][i] = hp.ref[k] + (double)mac[(int64_t)k * plane + off];
  }
}

// mac plane k at (x, y) = src[k][y * nx + x] - ref[k] in the compute type,
// for every given k; bit 0 of *bad set on a value that is not finite
template <typename C>
__global__ void __launch_bounds__(kHioThreads)
    k_fields_from_host(C* __restrict__ mac, int64_t plane, int64_t pitch, int nx, int ny,
                       HostPlanes hp, uint32_t* __restrict__ bad) {
  const int x = blockIdx.x * kHioThreads + threadIdx.x;
  if (x >= nx) return;
  bool ok = true;
  for (int y = blockIdx.y; y < ny; y += gridDim.y) {
    const int64_t off = (int64_t)y * pitch + x, i = (int64_t)y * nx + x;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      if (!hp.src[k]) continue;
      const double v = hp.src[k][i] - hp.ref[k];
      ok = ok && isfinite(v);
      mac[(int64_t)k * plane + off] = (C)v;
    }
  }
  if (!ok) atomicOr(bad, 1u);
}

// The porosity plane (compute type) from the host array, one warp per
// chunk of kErgunChunk consecutive values (lane l takes values l, l + 32,
// ...: coalesced reads); bit 0 of *bad set on a value outside (0, 1).  With
// part, the chunk's Ergun sum in the order ergun_mean takes on the host:
// each lane's terms in order, then the lanes by strides 16, 8, 4, 2, 1.
constexpr int kPorWarps = kHioThreads / 32;

template <typename C>
__global__ void __launch_bounds__(kHioThreads)
    k_porosity_from_host(const double* __restrict__ phi, C* __restrict__ dst, int64_t pitch,
                         int nx, int64_t n, int64_t chunks, double* __restrict__ part,
                         uint32_t* __restrict__ bad) {
  static_assert(kErgunLanes == 32, "one warp per chunk");
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * kPorWarps;
  bool ok = true;
  for (int64_t c = (int64_t)blockIdx.x * kPorWarps + (threadIdx.x >> 5); c < chunks; c += nwarps) {
    int64_t i = c * kErgunChunk + lane;
    int64_t y = i / nx;
    int64_t x = i - y * nx;
    double s = 0.0;
#pragma unroll 8
    for (int j = 0; j < kErgunPerLane; ++j) {
      if (i < n) {
        const double v = phi[i];
        ok = ok && v > 0.0 && v < 1.0;  // false for NaN too
        dst[y * pitch + x] = (C)v;
        if (part) s += ergun_term(v);
      }
      i += kErgunLanes;
      x += kErgunLanes;
      while (x >= nx) {
        x -= nx;
        ++y;
      }
    }
    if (part) {  // uniform over the warp
      for (int o = kErgunLanes / 2; o >= 1; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) part[c] = s;
    }
  }
  if (!ok) atomicOr(bad, 1u);
}

}  // namespace

cudaError_t launch_fields_to_host(const void* mac, bool dbl, int64_t plane, int64_t pitch, int nx,
                                  int ny, const HostPlanes& hp, cudaStream_t s) {
  const dim3 g = hio_grid(nx, ny);
  if (dbl)
    k_fields_to_host<double><<<g, kHioThreads, 0, s>>>(static_cast<const double*>(mac), plane,
                                                       pitch, nx, ny, hp);
  else
    k_fields_to_host<float><<<g, kHioThreads, 0, s>>>(static_cast<const float*>(mac), plane,
                                                      pitch, nx, ny, hp);
  return cudaGetLastError();
}

cudaError_t launch_fields_from_host(void* mac, bool dbl, int64_t plane, int64_t pitch, int nx,
                                    int ny, const HostPlanes& hp, uint32_t* bad, cudaStream_t s) {
  const dim3 g = hio_grid(nx, ny);
  if (dbl)
    k_fields_from_host<double><<<g, kHioThreads, 0, s>>>(static_cast<double*>(mac), plane, pitch,
                                                         nx, ny, hp, bad);
  else
    k_fields_from_host<float><<<g, kHioThreads, 0, s>>>(static_cast<float*>(mac), plane, pitch,
                                                        nx, ny, hp, bad);
  return cudaGetLastError();
}

cudaError_t launch_porosity_from_host(const double* phi, void* dst, bool dbl, int64_t pitch, int nx,
                                      int ny, double* erg_part, uint32_t* bad, cudaStream_t s) {
  const int64_t n = (int64_t)nx * ny, chunks = ergun_chunks(n);
  const unsigned blocks = (unsigned)((chunks + kPorWarps - 1) / kPorWarps);
  if (dbl)
    k_porosity_from_host<double><<<blocks, kHioThreads, 0, s>>>(
        phi, static_cast<double*>(dst), pitch, nx, n, chunks, erg_part, bad);
  else
    k_porosity_from_host<float><<<blocks, kHioThreads, 0, s>>>(
        phi, static_cast<float*>(dst), pitch, nx, n, chunks, erg_part, bad);
  return cudaGetLastError();
}

}  // namespace ltne
