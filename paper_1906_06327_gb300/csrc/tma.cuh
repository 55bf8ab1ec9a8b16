// tma.cuh -- tensor-memory-accelerator loads and shared-memory barriers
// (inline PTX, sm_100 family) for the tile kernels of tiles_xy.cu and
// tiles_line.cu, plus the host-side tensor-map encoder.
//
// A CTA's thread 0 initialises an mbarrier, arms it with the byte count of
// the box, and issues cp.async.bulk.tensor; the box lands in shared memory
// (elements outside the tensor read as zero) and completes the barrier's
// transaction count.  Every thread then waits on the barrier's phase with a
// bounded wait: after ~2 s of device time it gives up and reports a timeout
// instead of waiting forever.
#pragma once

#include <cuda.h>
#include <cstdint>

namespace rotgp {

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

// make initialised barriers visible to the async (TMA) proxy
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// As mbar_try_wait, but a thread whose phase is not complete is suspended
// in hardware until it completes or `ns` nanoseconds pass (no polling loop
// competing for issue slots while a TMA load is in flight).
__device__ __forceinline__ bool mbar_try_wait_for(uint64_t* bar, unsigned parity, unsigned ns) {
  unsigned ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of the barrier; false after ~2 s of device time
// (or 2^26 suspended waits of at most 0.1 ms each).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  for (int i = 0; i < (1 << 26); ++i) {
    if (mbar_try_wait_for(bar, parity, 100000u)) return true;
    if (clock64() - t0 > 4000000000LL) break;
  }
  return false;
}

// 3-D tiled TMA load of the box at element coordinates (c0, c1, c2) into
// shared memory (16-byte aligned start in c0 is the caller's duty).
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
      : "memory");
}

// L2 cache policies for loads: evict_first for data read once in whole
// lines (the state the y and z sweeps stream through, so that it does not
// push the sweep's output, read by the next sweep, out of L2), evict_last
// for small tables read by every sweep.  The row (x) sweep's boxes read
// parts of lines and keep the normal policy.
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// tma_load_3d with an L2 cache policy
__device__ __forceinline__ void tma_load_3d_hint(void* dst, const CUtensorMap* map, int c0, int c1,
                                                 int c2, uint64_t* bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      ".L2::cache_hint [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar)),
      "l"(policy)
      : "memory");
}

// 2-D tiled TMA load of the box at element coordinates (c0, c1).
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_addr(bar))
      : "memory");
}

// 3-D tiled TMA store of the box at (c0, c1, c2) from shared memory (bulk
// async-group of the issuing thread; elements outside the tensor are not
// written).  The writing threads fence their shared-memory stores to the
// async proxy and synchronise before the issuing thread calls this.
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, int c0, int c1, int c2,
                                             const void* src) {
  asm volatile(
      "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(src))
      : "memory");
}
// tma_load_2d with an L2 cache policy
__device__ __forceinline__ void tma_load_2d_hint(void* dst, const CUtensorMap* map, int c0, int c1,
                                                 uint64_t* bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      ".L2::cache_hint [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}

// 2-D tiled TMA store of the box at (c0, c1) from shared memory.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int c0, int c1,
                                             const void* src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(c0), "r"(c1), "r"(smem_addr(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// until at most N of this thread's bulk groups still read shared memory
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
// until all of this thread's bulk groups are complete
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Host: encode a 2-D float32 tensor map over the rows of a complex-float
// state (nrows rows of nx points; dimension 0 counts floats) with the box
// (floats, rows).  Same return convention as encode_state_map.
// swizzle_bytes: 0 (none), 64 or 128 (16-byte units of each box row of that
// many bytes are permuted by the row's shared-memory address bits 7.. as the
// tensor map's 64B / 128B swizzle modes define).
int encode_rows_map(CUtensorMap* map, void* base, int nx, long long nrows, unsigned box0,
                    unsigned box1, int swizzle_bytes = 0);

// Host: encode a 3-D float32 tensor map over a complex-float state of
// nx x ny x nz points (x fastest; dimension 0 counts floats, 2 per point)
// with the given box (floats, rows, planes).  Returns a CUDA driver status
// (0 = success); -1 if the encoder entry point is unavailable.
int encode_state_map(CUtensorMap* map, void* base, int nx, int ny, int nz, unsigned box0,
                     unsigned box1, unsigned box2);

}  // namespace rotgp
