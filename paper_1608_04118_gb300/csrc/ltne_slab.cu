// ltne_slab.cu -- halo rows of a row slab of the cavity, for a lattice
// split across processes (one slab per process or device).
//
// With pull streaming, a node of row y gathers population i from row
// y - e_y,i.  A slab that owns rows [g0, g0 + rows) therefore reads, from
// the row below it, only the populations that stream up (e_y = +1: f_2,
// f_5, f_6 of Eq. 8's D2Q9 set and g_2 of both D2Q5 sets, Eqs. 34-35) and,
// from the row above it, only those that stream down (e_y = -1: f_4, f_7,
// f_8, g_4 of both).  After every step each slab hands its first computed
// row's downward five and its last computed row's upward five to its
// neighbours: 5 x nx values per cut and direction.  The kernels here copy
// those values between the population planes and contiguous message
// buffers that the caller's communicator moves.
#include "ltne_internal.h"

namespace ltne {

namespace {

// Population planes (f_0..f_8, g_f0..g_f4, g_s0..g_s4) that cross a cut.
__constant__ int kUpPlanes[5] = {2, 5, 6, 11, 16};    // e_y = +1
__constant__ int kDownPlanes[5] = {4, 7, 8, 13, 18};  // e_y = -1

// One thread per (message value): blockIdx.y = 0 handles the lower side,
// 1 the upper side; value v = k * nx + x of the message is plane k's column x.
template <typename T>
__global__ void k_halo_pack(const T* __restrict__ pops, int64_t pitch, int64_t plane, int nx,
                            int row_lo, int row_hi, T* __restrict__ send_lo,
                            T* __restrict__ send_hi) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= 5 * nx) return;
  const int k = v / nx, x = v - k * nx;
  if (blockIdx.y == 0) {
    if (send_lo) send_lo[v] = pops[kDownPlanes[k] * plane + (int64_t)row_lo * pitch + x];
  } else {
    if (send_hi) send_hi[v] = pops[kUpPlanes[k] * plane + (int64_t)row_hi * pitch + x];
  }
}

template <typename T>
__global__ void k_halo_unpack(T* __restrict__ pops, int64_t pitch, int64_t plane, int nx,
                              int halo_lo, int halo_hi, const T* __restrict__ recv_lo,
                              const T* __restrict__ recv_hi) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= 5 * nx) return;
  const int k = v / nx, x = v - k * nx;
  if (blockIdx.y == 0) {
    if (recv_lo) pops[kUpPlanes[k] * plane + (int64_t)halo_lo * pitch + x] = recv_lo[v];
  } else {
    if (recv_hi) pops[kDownPlanes[k] * plane + (int64_t)halo_hi * pitch + x] = recv_hi[v];
  }
}

constexpr int kHaloThreads = 256;

}  // namespace

cudaError_t launch_halo_pack(const void* pops, int64_t pitch, int64_t plane, int nx, int row_lo,
                             int row_hi, size_t es, void* send_lo, void* send_hi,
                             cudaStream_t st) {
  if (!send_lo && !send_hi) return cudaSuccess;
  const dim3 grid((5 * nx + kHaloThreads - 1) / kHaloThreads, 2);
  if (es == 8)
    k_halo_pack<double><<<grid, kHaloThreads, 0, st>>>(
        static_cast<const double*>(pops), pitch, plane, nx, row_lo, row_hi,
        static_cast<double*>(send_lo), static_cast<double*>(send_hi));
  else if (es == 4)
    k_halo_pack<float><<<grid, kHaloThreads, 0, st>>>(
        static_cast<const float*>(pops), pitch, plane, nx, row_lo, row_hi,
        static_cast<float*>(send_lo), static_cast<float*>(send_hi));
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_halo_unpack(void* pops, int64_t pitch, int64_t plane, int nx, int halo_lo,
                               int halo_hi, size_t es, const void* recv_lo, const void* recv_hi,
                               cudaStream_t st) {
  if (!recv_lo && !recv_hi) return cudaSuccess;
  const dim3 grid((5 * nx + kHaloThreads - 1) / kHaloThreads, 2);
  if (es == 8)
    k_halo_unpack<double><<<grid, kHaloThreads, 0, st>>>(
        static_cast<double*>(pops), pitch, plane, nx, halo_lo, halo_hi,
        static_cast<const double*>(recv_lo), static_cast<const double*>(recv_hi));
  else if (es == 4)
    k_halo_unpack<float><<<grid, kHaloThreads, 0, st>>>(
        static_cast<float*>(pops), pitch, plane, nx, halo_lo, halo_hi,
        static_cast<const float*>(recv_lo), static_cast<const float*>(recv_hi));
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace ltne
