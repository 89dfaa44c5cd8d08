// ltne_static.cu -- observables of caller-held fields with no memory
// allocation at all: the reduction's per-block partial sums live in a fixed
// device array defined in this file instead of in a caller-provided
// workspace.
//
// Who needs it: code that can hand over field buffers but cannot allocate
// device memory when it wants a reduction -- a plug-in or monitor inside a
// host application that owns every device allocation and offers none to its
// guests, a thread from which the framework's allocator is not reachable, or
// a real-time loop where an allocation (and the device synchronisation it
// may imply) is not acceptable.
#include <mutex>

#include <cuda.h>

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
// with the device current, before a kernel may be given it.  The address
// belongs to the device's current (primary) context; after a
// cudaDeviceReset() the next call finds a new context and asks again, so a
// cached address never outlives the context it came from.
constexpr int kMaxDevices = 64;
struct ScratchSlot {
  unsigned long long ctx_id = 0;  // unique id of the context the address is for
  double* ptr = nullptr;
};
ScratchSlot g_scratch[kMaxDevices];
std::mutex g_scratch_mu;

// cuCtxGetCurrent and cuCtxGetId from the driver, fetched through the
// runtime (no link-time dependence on the driver library).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

template <typename Fn>
Fn driver_fn(const char* name) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    return reinterpret_cast<Fn>(p);
  return nullptr;
}

// Unique id of the calling thread's current context; 0 when none is
// current yet (the runtime creates the primary context on its first call
// that needs one).
cudaError_t current_context_id(unsigned long long* id) {
  static const CtxGetCurrentFn get_current = driver_fn<CtxGetCurrentFn>("cuCtxGetCurrent");
  static const CtxGetIdFn get_id = driver_fn<CtxGetIdFn>("cuCtxGetId");
  if (!get_current || !get_id) return cudaErrorNotSupported;
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  *id = 0;
  if (!ctx) return cudaSuccess;
  return get_id(ctx, id) == CUDA_SUCCESS ? cudaSuccess : cudaErrorDeviceUninitialized;
}

cudaError_t scratch_for_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  unsigned long long id = 0;
  e = current_context_id(&id);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  ScratchSlot& slot = g_scratch[dev];
  if (!slot.ptr || id == 0 || slot.ctx_id != id) {
    // first call on this device, or a context the cached address is not
    // from: ask the runtime (which makes the primary context current if no
    // context was), then record the context it answered for
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_reduce_scratch);
    if (e != cudaSuccess) return e;
    e = current_context_id(&id);
    if (e != cudaSuccess) return e;
    if (id == 0) return cudaErrorDeviceUninitialized;
    slot.ptr = static_cast<double*>(p);
    slot.ctx_id = id;
  }
  *out = slot.ptr;
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
