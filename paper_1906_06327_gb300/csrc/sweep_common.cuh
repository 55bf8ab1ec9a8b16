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
//
// The one-line-per-lane TMA forms of complex float (k_sweep_x1t,
// k_sweep_s1t) use the same chunking with the unfolded solve of the same
// system (A y = psi, psi' = 2y - psi: weights m2, al, be, no neighbour
// points), TMA box loads and stores through R + 1 slots per warp, persistent
// warps and programmatic launch; they serve imaginary time, while real time
// keeps the folded form above (it holds the CN map's norm to rounding).
#pragma once

#include "common.cuh"
#include <cstdint>

namespace rotgp {

// Dynamic shared-memory opt-in of a kernel on the current device (sweep_s.cu):
// `bytes`, or all the device allows beside the kernel's static shared memory.
cudaError_t allow_smem_bytes(const void* fn, int bytes);
cudaError_t allow_smem(const void* fn);

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

// The real-time H1 factor exp(-i theta) as 1 + c1 - i s1 with
// c1 = cos(theta) - 1 = -2 sin^2(theta/2) and s1 = sin(theta) =
// 2 sin(theta/2) cos(theta/2), both to full relative precision.  Rounding
// cos(theta) itself near 1 (to 1 exactly when theta is small) leaves a
// modulus error of up to half an ulp of 1 that has the same sign on every
// point of a plane of nearly equal potential, which makes the real-time norm
// drift by ~1e-8 per step in complex float; with c1 and s1 the modulus is one
// to about theta^2 times the rounding.
template <class T>
__device__ __forceinline__ void rot_t(T theta, T* c1, T* s1) {
  T sh, ch;
  sincos_t(theta * (T)0.5, &sh, &ch);
  *c1 = -(T)2 * sh * sh;
  *s1 = (T)2 * sh * ch;
}
// v exp(-i theta) = v + (c1 v - i s1 v)
__device__ __forceinline__ float2 rotate_f(float2 v, float c1, float s1) {
  return make_float2(fmaf(c1, v.x, fmaf(s1, v.y, v.x)), fmaf(c1, v.y, fmaf(-s1, v.x, v.y)));
}

// A point advanced by the real-time H1 substep, held as its value before the
// substep and the substep's increment: v exp(-i theta) = v + dl, dl = c1 v -
// i s1 v.  The sum v + dl rounded on its own loses the second-order part of
// dl (c1 v, ~theta^2/2 of v) wherever it is below half an ulp of that
// component, which happens each time a component of the rotating v passes
// an extremum; the loss always enlarges |v + dl|, and with Delta ~ 1e-4 the
// complex-float norm climbed ~1e-8 per step.  The folded forward step
// (fwd_inc) therefore adds dl to the rest of the CN sum, which is of order
// kappa |v|, and the raw value last: one rounding whose discarded part is
// no longer biased.
template <class T>
struct hpt {
  cpx<T> v, dl;
};
template <class T>
__device__ __forceinline__ hpt<T> rot_inc(cpx<T> v, T c1, T s1) {
  return {v, mk<T>(fma(c1, v.x, s1 * v.y), fma(c1, v.y, -(s1 * v.x)))};
}
// the advanced value, rounded (neighbours in the CN sum, where the rounding
// is weighted by the small off-diagonal coefficients)
template <class T>
__device__ __forceinline__ cpx<T> hw(const hpt<T>& p) {
  return mk<T>(p.v.x + p.dl.x, p.v.y + p.dl.y);
}

template <class T>
__device__ __forceinline__ cpx<T> zero() { return mk<T>(0, 0); }

// a * b + c for complex numbers
template <class T>
__device__ __forceinline__ cpx<T> cfma(cpx<T> a, cpx<T> b, cpx<T> c) {
  return mk<T>(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

// Summation order of the folded recurrences.  Each step adds terms of
// order kappa |psi| to one term of order |psi| (pc in the forward step, d'
// in the backward one).  Rounded into the large term one FMA at a time,
// every term costs a rounding at the scale of |psi|, and these roundings
// leave a small systematic gain of norm (measured ~2e-9 per real-time step
// on a vortex lattice in complex float, eight roundings per point in the
// forward step); the small terms are therefore summed first and the large
// one is added once.
//
// One forward step d' = pc + (a0 pc + am pm + ap pn + al d').
template <class T>
__device__ __forceinline__ cpx<T> fwd(const coef5<T>& k, cpx<T> pm, cpx<T> pc, cpx<T> pn,
                                      cpx<T> d) {
  const cpx<T> s = cfma(k.ap, pn, cfma(k.am, pm, mk<T>(fma(k.a0.x, pc.x, -(k.a0.y * pc.y)),
                                                       fma(k.a0.x, pc.y, k.a0.y * pc.x))));
  const cpx<T> t = cfma(k.al, d, s);
  return mk<T>(pc.x + t.x, pc.y + t.y);
}
// One backward step x = d' + be x.
template <class T>
__device__ __forceinline__ cpx<T> bwd(const cpx<T>& be, cpx<T> x, cpx<T> d) {
  const cpx<T> t = mk<T>(fma(be.x, x.x, -(be.y * x.y)), fma(be.x, x.y, be.y * x.x));
  return mk<T>(d.x + t.x, d.y + t.y);
}

// The forward step with the centre point as value + H1 increment:
// d' = v + (dl + a0 (v + dl) + am pm + ap pn + al d').
template <class T>
__device__ __forceinline__ cpx<T> fwd_inc(const coef5<T>& k, cpx<T> pm, const hpt<T>& pc,
                                          cpx<T> pn, cpx<T> d) {
  cpx<T> s = cfma(k.a0, hw(pc), pc.dl);
  s = cfma(k.am, pm, s);
  s = cfma(k.ap, pn, s);
  s = cfma(k.al, d, s);
  return mk<T>(pc.v.x + s.x, pc.v.y + s.y);
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

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Per-thread sum of |x|^2: Kahan-compensated in float, plain in double.
template <class T>
struct acc_t {
  T s = 0, c = 0;
  __device__ __forceinline__ void add(T v) {
    T y = v - c;
    T t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
template <>
struct acc_t<double> {
  double s = 0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double value() const { return s; }
};

// Block sum of v -> per-block partial; the last block to finish sums the
// partials in block order (deterministic), sets the norm, the pending scale
// (1/sqrt(norm) in imaginary time, 1 in real time) and the non-finite flag.
template <class A>
static __device__ void norm_epilogue(double v, const A& a) {
  __shared__ double ws[32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned nblocks = gridDim.x;
  v = warp_sum(v);
  if (lane == 0) ws[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int w = 0; w < nw; ++w) s += ws[w];
    a.partials[blockIdx.x] = s;
    __threadfence();
    unsigned t = atomicAdd(a.counter, 1u);
    last = (t == nblocks - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0;
  for (unsigned i = threadIdx.x; i < nblocks; i += blockDim.x) s += __ldcg(&a.partials[i]);
  s = warp_sum(s);
  __syncthreads();
  if (lane == 0) ws[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0;
    for (int w = 0; w < nw; ++w) tot += ws[w];
    double n = tot * a.vol;
    *a.norm_out = n;
    if (!(n > 0.0) || !isfinite(n)) {
      atomicOr(a.flags, 1);
      *a.scale_out = 1.0;
    } else {
      *a.scale_out = a.imag ? 1.0 / sqrt(n) : 1.0;
    }
    *a.counter = 0u;
  }
}

// ---------------------------------------------------------------- packed FP32x2
// Two lines solved by one lane in complex float are held in split form: the
// real parts of both lines in one float2 and the imaginary parts in another,
// so that every complex multiply-add of the two lines is four packed FP32x2
// FMAs (__ffma2_rn) instead of eight scalar ones.
struct c2 {
  float2 re, im;
};
// a complex coefficient of the two lines, split, with negated imaginary parts
struct k2 {
  float2 x, y, ny;
};
struct coef2 {
  k2 a0, am, ap, al, be;
};

__device__ __forceinline__ k2 make_k2(cpx<float> a, cpx<float> b) {
  k2 k;
  k.x = make_float2(a.x, b.x);
  k.y = make_float2(a.y, b.y);
  k.ny = make_float2(-a.y, -b.y);
  return k;
}
__device__ __forceinline__ coef2 make_coef2(const coef5<float>& u, const coef5<float>& v) {
  coef2 c;
  c.a0 = make_k2(u.a0, v.a0);
  c.am = make_k2(u.am, v.am);
  c.ap = make_k2(u.ap, v.ap);
  c.al = make_k2(u.al, v.al);
  c.be = make_k2(u.be, v.be);
  return c;
}
// k * b
__device__ __forceinline__ c2 kmul2(const k2& k, const c2& b) {
  c2 r;
  r.re = __ffma2_rn(k.ny, b.im, __fmul2_rn(k.x, b.re));
  r.im = __ffma2_rn(k.y, b.re, __fmul2_rn(k.x, b.im));
  return r;
}
// k * b + c
__device__ __forceinline__ c2 kfma2(const k2& k, const c2& b, const c2& c) {
  c2 r;
  r.re = __ffma2_rn(k.ny, b.im, __ffma2_rn(k.x, b.re, c.re));
  r.im = __ffma2_rn(k.y, b.re, __ffma2_rn(k.x, b.im, c.im));
  return r;
}
// forward step of both lines, small terms first (see fwd):
// d' = pc + (a0 pc + am pm + ap pn + al d')
__device__ __forceinline__ c2 fwd2(const coef2& k, const c2& pm, const c2& pc, const c2& pn,
                                   const c2& d) {
  c2 s = kfma2(k.al, d, kfma2(k.ap, pn, kfma2(k.am, pm, kmul2(k.a0, pc))));
  s.re = __fadd2_rn(pc.re, s.re);
  s.im = __fadd2_rn(pc.im, s.im);
  return s;
}
// ... with the centre point as value pv + real-time H1 increment pdl (see
// hpt): d' = pv + (pdl + a0 (pv + pdl) + am pm + ap pn + al d')
__device__ __forceinline__ c2 fwd2_inc(const coef2& k, const c2& pm, const c2& pv,
                                       const c2& pdl, const c2& pn, const c2& d) {
  c2 w;
  w.re = __fadd2_rn(pv.re, pdl.re);
  w.im = __fadd2_rn(pv.im, pdl.im);
  c2 s = kfma2(k.al, d, kfma2(k.ap, pn, kfma2(k.am, pm, kfma2(k.a0, w, pdl))));
  s.re = __fadd2_rn(pv.re, s.re);
  s.im = __fadd2_rn(pv.im, s.im);
  return s;
}
// backward step of both lines: x = d' + be x
__device__ __forceinline__ c2 bwd2(const k2& be, const c2& x, const c2& d) {
  c2 t = kmul2(be, x);
  t.re = __fadd2_rn(d.re, t.re);
  t.im = __fadd2_rn(d.im, t.im);
  return t;
}
__device__ __forceinline__ c2 zero2() {
  c2 r;
  r.re = make_float2(0.f, 0.f);
  r.im = make_float2(0.f, 0.f);
  return r;
}
// two interleaved complex numbers (line 0, line 1) <-> split form
__device__ __forceinline__ c2 split2(const float4& t) {
  c2 r;
  r.re = make_float2(t.x, t.z);
  r.im = make_float2(t.y, t.w);
  return r;
}
__device__ __forceinline__ float4 join2(const c2& c) {
  return make_float4(c.re.x, c.im.x, c.re.y, c.im.y);
}
// split form stored as one float4 (re0, re1, im0, im1)
__device__ __forceinline__ float4 pack_split(const c2& c) {
  return make_float4(c.re.x, c.re.y, c.im.x, c.im.y);
}
__device__ __forceinline__ c2 unpack_split(const float4& t) {
  c2 r;
  r.re = make_float2(t.x, t.y);
  r.im = make_float2(t.z, t.w);
  return r;
}

// ---------------------------------------------------------------- stencil form
// Table row of output position p of a line with N points and B end rows at
// each end: rows r < B are the left end (position r; row 0, the zero edge,
// has no weights), row B the interior, row B + 1 + e the right end
// (position N - 1 - e).
__device__ __forceinline__ int stencil_row(int p, int N, int B) {
  return p < B ? p : (p >= N - B ? B + 1 + (N - 1 - p) : B);
}

// Complex multiply-accumulate on the interleaved (re, im) layout: with
// w = wr + i wi, a += (wr, wr) * v and b += (wi, wi) * v; the sum is then
// (a.x - b.y, a.y + b.x).  Two independent packed FP32x2 chains, and the
// operands are used as they are stored.
struct cacc {
  float2 a, b;
};
__device__ __forceinline__ cacc cacc_zero() {
  cacc c;
  c.a = make_float2(0.f, 0.f);
  c.b = make_float2(0.f, 0.f);
  return c;
}
__device__ __forceinline__ void cmac(cacc& c, const float2& wr, const float2& wi,
                                     const float2& v) {
  c.a = __ffma2_rn(wr, v, c.a);
  c.b = __ffma2_rn(wi, v, c.b);
}
__device__ __forceinline__ float2 cfin(const cacc& c) {
  return make_float2(c.a.x - c.b.y, c.a.y + c.b.x);
}
// Unfolded-form weights of positions p0 .. p0 + C - 1 of line li from the
// planes of stream_args::coefT (entries past the table length are the
// converged ones).  The loads of a chunk are issued together, ahead of the
// recurrence that would otherwise wait on each in turn; the lanes of a warp
// read consecutive lines, so every load is one or two contiguous segments.
// The loads carry an L2 policy (evict_last: the planes are read by every
// sweep, between which the state streams through L2).
__device__ __forceinline__ float2 coef_plane(const float2* tab, int tl, int lt, int f, int p,
                                             int li, uint64_t pol) {
  const float2* a = tab + ((size_t)f * (lt + 1) + min(p, lt)) * tl + li;
  float2 v;
  asm volatile("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
               : "=f"(v.x), "=f"(v.y)
               : "l"(a), "l"(pol));
  return v;
}
template <int C>
__device__ __forceinline__ void table_fwd(const float2* tab, int tl, int lt, int li, int p0,
                                          uint64_t pol, float2 (&m2)[C], float2 (&al)[C]) {
#pragma unroll
  for (int r = 0; r < C; ++r) {
    m2[r] = coef_plane(tab, tl, lt, 0, p0 + r, li, pol);
    al[r] = coef_plane(tab, tl, lt, 1, p0 + r, li, pol);
  }
}
template <int C>
__device__ __forceinline__ void table_be(const float2* tab, int tl, int lt, int li, int p0,
                                         uint64_t pol, float2 (&be)[C]) {
#pragma unroll
  for (int r = 0; r < C; ++r) be[r] = coef_plane(tab, tl, lt, 2, p0 + r, li, pol);
}

// a complex weight as the two duplicated pairs (wr, wr), (wi, wi)
__device__ __forceinline__ void wsplit(const float2& w, float2& wr, float2& wi) {
  wr = make_float2(w.x, w.x);
  wi = make_float2(w.y, w.y);
}

}  // namespace rotgp
