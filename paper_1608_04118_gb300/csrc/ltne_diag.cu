// ltne_diag.cu -- a self-check of the bounded mbarrier wait used by the
// staged step (ltne_check_bounded_wait in include/ltne.h).
#include "ltne.h"
#include "ltne_tma.cuh"

namespace {

// One thread initialises an mbarrier that expects two arrivals, arrives
// once, and waits (bounded) for a phase that therefore never completes.
__global__ void k_wait_gives_up(int spins, int* gave_up) {
  __shared__ uint64_t bar;
  ltne::mbar_init(&bar, 2);
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(ltne::smem_addr(&bar))
               : "memory");
  *gave_up = ltne::mbar_wait(&bar, 0u, spins) ? 0 : 1;
}

}  // namespace

extern "C" int ltne_check_bounded_wait(void* cuda_stream, int32_t spins, int32_t* gave_up) {
  if (!gave_up || spins < 1) return LTNE_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int* d = nullptr;
  cudaError_t e = cudaMallocAsync(&d, sizeof(int), st);
  if (e == cudaSuccess) {
    k_wait_gives_up<<<1, 1, 0, st>>>(spins, d);
    e = cudaGetLastError();
  }
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (d) cudaFreeAsync(d, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LTNE_ERR_CUDA;
  }
  *gave_up = h;
  return LTNE_OK;
}
