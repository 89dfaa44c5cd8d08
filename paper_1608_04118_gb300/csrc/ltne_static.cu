// ltne_static.cu -- observables of caller-held fields with no memory
// allocation at all: the reduction's per-block partial sums live in a fixed
// device array defined in this file instead of in a caller-provided
// workspace.
//
// Who needs it: code that can hand over field buffers but cannot allocate
// device memory when it wants a reduction -- a monitor running inside CUDA
// graph capture (allocation is not permitted while capturing), a host
// framework whose allocator is not reachable from the calling thread, or a
// real-time loop where an allocation (and the device synchronisation it may
// imply) is not acceptable.
#include <mutex>

#include "ltne.h"
#include "ltne_internal.h"

using namespace ltne;

namespace {

// Largest pass-1 grid served: 4096 blocks of 256 columns x 16 to 64 rows,
// i.e. any lattice with ceil(nx/256) * ceil(ny/64) <= 4096 (8192 x 8192 fits).
constexpr int kMaxBlocks = kReduceMaxBlocks;

// Reduction scratch: kMaxBlocks partial vectors, then one result vector.
// 4097 x 18 doubles = 590 KB, held by every GPU that loads the library.
__device__ __align__(256) double g_reduce_scratch[(kMaxBlocks + 1) * NACC];

// Device address of g_reduce_scratch per device ordinal.  In host code the
// symbol's name is only a stand-in: its device address must be asked for,
// with the device current, before a kernel may be given it.
constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

cudaError_t scratch_for_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_reduce_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int ltne_observables_static(const ltne_params* p, const float* fields, int64_t pitch,
                                       const float* porosity, int64_t step, void* cuda_stream,
                                       ltne_obs* out) {
  if (!p || !fields || !out || pitch < p->nx) return LTNE_ERR_INVALID_ARG;
  int rc = validate_params(*p);
  if (rc != LTNE_OK) return rc;
  if (p->storage == LTNE_F64) return LTNE_ERR_INVALID_ARG;  // FP32 fields only
  if ((porosity != nullptr) != (p->porosity_field != 0)) return LTNE_ERR_INVALID_ARG;
  const int blocks = reduce_blocks(p->nx, p->ny);
  if (blocks > kMaxBlocks) return LTNE_ERR_INVALID_ARG;  // beyond the fixed scratch
  NodeParams<double> P;
  DerivedInfo info;
  rc = derive_params(*p, nullptr, P, info);
  if (rc != LTNE_OK) return rc;
  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LTNE_ERR_CUDA;
  }
  const cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int64_t plane = pitch * p->ny;
  ReduceArgs a;
  a.mac = fields;
  a.phi = porosity;
  // No residual snapshot here: the "previous" planes are the current u, T_f,
  // T_s planes themselves (differences zero) and nothing is written back.
  a.prev = const_cast<float*>(fields) + plane;
  a.partials = scratch;                 // every slot in use is written by pass 1
  a.out = scratch + (size_t)kMaxBlocks * NACC;  // written by pass 2
  a.nx = p->nx;
  a.ny = p->ny;
  a.pitch = pitch;
  a.plane = plane;
  a.phi_u = p->porosity;
  a.sigma = p->sigma;
  a.qf = p->qf;
  a.qs = p->qs;
  a.update_prev = 0;
  a.blocks = blocks;
  a.is_double = 0;
  e = launch_reduce(a, st);
  double acc[NACC];
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(acc, a.out, sizeof(acc), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LTNE_ERR_CUDA;
  }
  return finish_observables(*p, info, step, false, acc, out);
}
