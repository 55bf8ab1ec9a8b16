// sweep_common.cuh -- device helpers shared by the line-sweep kernels
// (sweep_x.cu, sweep_s.cu) of one split step (Sec. 2).
//
// Line solver.  Each line's tridiagonal system (Eqs. eqD.11/eq5) has
// coefficients constant along the line and is solved by the Thomas
// algorithm, folded into
//   forward   d'_p = a0 psi_p + am psi_{p-1} + ap psi_{p+1} + al d'_{p-1}
//   backward  x_p  = d'_p + be x_{p+1}
// (coef5 in common.cuh).  One lane owns V lines and walks a segment of them
// chunk by chunk (C points per chunk): the forward carry d' passes exactly
// from chunk to chunk, and the back substitution of chunk q-1 starts H
// points into chunk q from x = 0.  Both recurrences are strictly contracting
// (|al| and |be| per point are at most the "decay" factor), so a carry
// truncated H points away changes the result by decay^H relative, which the
// host keeps below 1e-9 (float) or 1e-17 (double).  Lines longer than one
// segment are split: a segment's forward sweep starts `warm` chunks early
// from d' = 0 and its last back substitution looks H points into the next
// segment.  Near the line start (p < lt) and in a ragged last chunk the
// coefficients come from the table; everywhere else from registers.
//
// Memory.  Each sweep reads the state once and writes it once into the
// other ping-pong buffer.  Chunks stream through an R-slot shared-memory ring
// per warp with cp.async; a chunk copy also brings the first point of the
// next chunk (the stencil's right neighbour), so a chunk can be solved as
// soon as its own copy lands while up to R-1 later chunks are in flight.
#pragma once

#include "common.cuh"

namespace rotgp {

template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
  unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  if (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(src), "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
// wait until the oldest outstanding chunk of an R-slot ring (R = 3 or 4) has landed
__device__ __forceinline__ void ring_wait(int R) {
  if (R == 3)
    cp_async_wait<1>();
  else
    cp_async_wait<2>();
}

// Dynamic shared memory of this launch, in bytes.
__device__ __forceinline__ unsigned dynamic_smem_bytes() {
  unsigned r;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
  return r;
}

__device__ __forceinline__ float exp_t(float v) { return expf(v); }
__device__ __forceinline__ double exp_t(double v) { return exp(v); }
__device__ __forceinline__ void sincos_t(float v, float* s, float* c) { sincosf(v, s, c); }
__device__ __forceinline__ void sincos_t(double v, double* s, double* c) { sincos(v, s, c); }

template <class T>
__device__ __forceinline__ cpx<T> zero() { return mk<T>(0, 0); }

// a * b + c for complex numbers
template <class T>
__device__ __forceinline__ cpx<T> cfma(cpx<T> a, cpx<T> b, cpx<T> c) {
  return mk<T>(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

// One forward step d' = a0 pc + am pm + ap pn + al d', summed as two
// independent halves so that only the last complex FMA waits on d'.
template <class T>
__device__ __forceinline__ cpx<T> fwd(const coef5<T>& k, cpx<T> pm, cpx<T> pc, cpx<T> pn,
                                      cpx<T> d) {
  const cpx<T> s1 = cfma(k.am, pm, k.a0 * pc);
  const cpx<T> s2 = cfma(k.ap, pn, s1);
  return cfma(k.al, d, s2);
}

// Coefficients of position p: registers in the converged interior, the
// table near the line start and in a ragged last chunk.
template <class T, bool FAST>
__device__ __forceinline__ const coef5<T>& coef_at(const coef5<T>* crow, const coef5<T>& cinf,
                                                   int p, int lt) {
  return FAST ? cinf : crow[min(p, lt)];
}

// Unroll factor of the per-point loops.
template <int C>
struct unroll_of {
  static constexpr int value = C <= 16 ? C : 8;
};

template <bool B>
struct bool_tag {
  static constexpr bool value = B;
};

// V complex numbers of adjacent lines, moved as one 8- or 16-byte unit.
template <class T, int V>
struct __align__(V * sizeof(cpx<T>)) pack {
  cpx<T> v[V];
};

}  // namespace rotgp
