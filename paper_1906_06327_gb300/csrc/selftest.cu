// selftest.cu -- a check of the bounded device waits used by the TMA tile
// passes (tiles_xy.cu, tiles_line.cu): one CTA arms an mbarrier for 16
// bytes that no copy will ever deliver and waits on it with the same
// bounded wait as the tile passes.  The wait must give up by itself and the
// kernel must return normally, leaving the context usable.
#include <cstdint>

#include "../../include/rotgp.h"
#include "common.cuh"
#include "tma.cuh"

namespace rotgp {

__global__ void k_wait_selftest(int* status, long long* cycles) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
    mbar_expect_tx(&bar, 16);  // one arrival now; 16 bytes that never come
  }
  __syncthreads();
  const long long t0 = clock64();
  const bool done = mbar_wait(&bar, 0);
  if (threadIdx.x == 0) {
    *status = done ? 0 : 1;
    *cycles = clock64() - t0;
  }
}

}  // namespace rotgp

extern "C" int rotgp_check_bounded_wait(void* stream, double* seconds) {
  using namespace rotgp;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* d = nullptr;
  cudaError_t e = cudaMalloc(&d, 16);
  if (e != cudaSuccess) return ROTGP_ENOMEM;
  int status = -1;
  long long cyc = 0;
  int rate_khz = 0, dev = 0;
  e = cudaMemsetAsync(d, 0xff, 16, s);
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 32, 0, s>>>(d, reinterpret_cast<long long*>(d + 2));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, d, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&cyc, d + 2, sizeof(long long), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&rate_khz, cudaDevAttrClockRate, dev);
  cudaFree(d);
  if (e != cudaSuccess) return ROTGP_ECUDA;
  if (seconds) *seconds = rate_khz > 0 ? (double)cyc / (rate_khz * 1e3) : -1.0;
  // the wait is expected to give up: that is the only passing outcome
  return status == 1 ? ROTGP_OK : ROTGP_ECUDA;
}
