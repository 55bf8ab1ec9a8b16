// sweep_s.cu -- the strided line sweeps of one split step: H3 along y
// (Eq. eq3, "performed similarly" to Eq. eqD.9) and the z sweep of the 3D
// "identical prescription", with the norm of the state reduced in the last
// sweep of a step; and the per-line coefficient tables of every sweep.
//
// y and z lines are strided: lane = adjacent columns, so every copy of a
// warp covers 32*V consecutive points, each lane keeps its own column in a
// [point][lane] slab of the ring (no bank conflicts, no cross-lane sharing)
// and stores its results straight to global memory, coalesced.  The solver
// and the ring are described in sweep_common.cuh.
#include "sweep_common.cuh"
#include "tma.cuh"

namespace rotgp {

// --------------------------------------------------------------- tables
// Thomas multipliers of one line, m_1 = 1/A0, c'_1 = A+ m_1,
// m_p = 1/(A0 - A- c'_{p-1}), c'_p = A+ m_p, folded into coef5 entries
// p = 1..lt (computed in double); entry 0 is zero.
struct dcx {
  double x, y;
};
__device__ __forceinline__ dcx dmul(dcx a, dcx b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ dcx dsub(dcx a, dcx b) { return {a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ dcx dinv(dcx a) {
  const double r = 1.0 / (a.x * a.x + a.y * a.y);
  return {a.x * r, -a.y * r};
}
template <class T>
__device__ __forceinline__ cpx<T> dcast(dcx a) { return mk<T>((T)a.x, (T)a.y); }

template <class T>
__global__ void k_tables(coef5<T>* tab, int nlines, int lt, axis_coef co) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nlines) return;
  const double u = co.u0 + (double)l * co.du;
  const dcx kap{co.kap_re, co.kap_im}, tau{co.tau_re * u, co.tau_im * u};
  const dcx one{1.0, 0.0};
  const dcx a0{1.0 + 2.0 * kap.x, 2.0 * kap.y};
  const dcx am = dsub(tau, kap), ap{-kap.x - tau.x, -kap.y - tau.y};
  const dcx diag = dsub(one, {2.0 * kap.x, 2.0 * kap.y});
  const dcx kmt = dsub(kap, tau), kpt{kap.x + tau.x, kap.y + tau.y};
  coef5<T>* t = tab + (size_t)l * (lt + 1);
  t[0].a0 = t[0].am = t[0].ap = t[0].al = t[0].be = zero<T>();
  dcx c{0.0, 0.0};
  for (int p = 1; p <= lt; ++p) {
    const dcx m = dinv(dsub(a0, dmul(am, c)));
    c = dmul(ap, m);
    t[p].a0 = dcast<T>(dmul(m, diag));
    t[p].am = dcast<T>(dmul(m, kmt));
    t[p].ap = dcast<T>(dmul(m, kpt));
    const dcx mam = dmul(m, am);
    t[p].al = dcast<T>({-mam.x, -mam.y});
    t[p].be = dcast<T>({-c.x, -c.y});
  }
}

// --------------------------------------------------------------- y / z sweeps
// Forward sweep over one chunk slot (C+1 packs, stride 32 between points):
// psi -> d' in place for the first C points.
template <class T, int V, int C, bool FAST>
__device__ __forceinline__ void strided_forward(pack<T, V>* s0, cpx<T> (&pm)[V], cpx<T> (&d)[V],
                                                const coef5<T>* const (&crow)[V],
                                                const coef5<T> (&cinf)[V], int p0, int lt) {
  pack<T, V> cur = s0[0];
#pragma unroll(unroll_of<C>::value)
  for (int r = 0; r < C; ++r) {
    const pack<T, V> nx = s0[(r + 1) * 32];
    pack<T, V> o;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      d[v] = fwd(coef_at<T, FAST>(crow[v], cinf[v], p0 + r, lt), pm[v], cur.v[v], nx.v[v], d[v]);
      pm[v] = cur.v[v];
      o.v[v] = d[v];
    }
    s0[r * 32] = o;
    cur = nx;
  }
}

template <class T, int V, int C, bool REDUCE>
__global__ void __launch_bounds__(128) k_sweep_strided(const stream_args a) {
  using E = cpx<T>;
  using Pk = pack<T, V>;
  constexpr int SLOT = (C + 1) * 32;  // packs per ring slot
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int R = a.ring;
  // a launch whose shared memory does not match this instantiation flags an
  // error and does nothing (uniform over the block)
  if (R < 3 || R > 4 ||
      dynamic_smem_bytes() < (blockDim.x >> 5) * (unsigned)(R * SLOT) * (unsigned)sizeof(Pk)) {
    if (threadIdx.x == 0) atomicOr(a.flags, 2);
    return;
  }
  Pk* ring = reinterpret_cast<Pk*>(smem_raw) + (size_t)wib * R * SLOT;
  const long long ngroups = (a.nlines + 32 * V - 1) / (32 * V);
  const long long wg = (long long)blockIdx.x * (blockDim.x >> 5) + wib;
  acc_t<T> acc;
  if (wg < ngroups * a.nseg) {
    const long long g = wg % ngroups;
    const int sg = (int)(wg / ngroups);
    const long long c0 = (g * 32 + lane) * V;
    const bool active = c0 < a.nlines;
    const long long base = active ? (c0 / a.nx) * a.outer + (c0 % a.nx) : 0;
    const E* in = static_cast<const E*>(a.in) + base;
    E* out = static_cast<E*>(a.out) + base;
    const int N = a.len, nch = (N + C - 1) / C, lt = a.lt;
    const int qo0 = sg * a.seg_chunks, qo1 = min(nch, qo0 + a.seg_chunks);
    const int qa = max(0, qo0 - a.warm), qb = min(nch, qo1 + 1);
    const coef5<T>* crow[V];
    coef5<T> cinf[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int li = (a.coef_mode == 1 && active) ? (int)((c0 + v) % a.nx) : 0;
      crow[v] = static_cast<const coef5<T>*>(a.coef) + (size_t)li * (lt + 1);
      cinf[v] = crow[v][lt];
    }
    auto slot = [&](int q) { return ring + (size_t)(q % R) * SLOT + lane; };
    // copy points q*C .. q*C + C of this lane's lines (zero past the line)
    auto issue = [&](int q) {
      if (q < qb) {
        Pk* s = slot(q);
#pragma unroll
        for (int r = 0; r <= C; ++r) {
          const int p = q * C + r;
          if (active && p < N)
            cp_async<sizeof(Pk)>(&s[r * 32], in + (long long)p * a.stride);
          else
            s[r * 32] = Pk{};
        }
      }
      cp_async_commit();
    };
    for (int i = 0; i < R - 1; ++i) issue(qa + i);
    E pm[V], d[V];
#pragma unroll
    for (int v = 0; v < V; ++v) pm[v] = d[v] = zero<T>();
    for (int q = qa; q <= qb; ++q) {
      if (q < qb) {
        ring_wait(R);
        if (q * C >= lt && (q + 1) * C <= N)
          strided_forward<T, V, C, true>(slot(q), pm, d, crow, cinf, q * C, lt);
        else
          strided_forward<T, V, C, false>(slot(q), pm, d, crow, cinf, q * C, lt);
      }
      const int qq = q - 1;
      if (qq >= qo0 && qq < qo1) {
        E x[V];
#pragma unroll
        for (int v = 0; v < V; ++v) x[v] = zero<T>();
        // H points of look-ahead into chunk q (truncated start), or the exact
        // start at the last unknown N-1 when the line ends first
        const int la = min(a.halo, N - q * C);
        const Pk* sq = slot(q);
        for (int h = la - 1; h >= 0; --h) {
          const Pk t = sq[h * 32];
#pragma unroll
          for (int v = 0; v < V; ++v) {
            const E be = crow[v][min(q * C + h, lt)].be;
            x[v] = cfma(be, x[v], t.v[v]);
          }
        }
        const Pk* sp = slot(qq);
        const bool fast = qq * C >= lt && q * C <= N;
        auto back = [&](auto fast_tag) {
          constexpr bool FAST = decltype(fast_tag)::value;
#pragma unroll(unroll_of<C>::value)
          for (int r = C - 1; r >= 0; --r) {
            const int p = qq * C + r;
            if (!FAST && p >= N) continue;
            const Pk t = sp[r * 32];
            Pk o;
#pragma unroll
            for (int v = 0; v < V; ++v) {
              x[v] = cfma(coef_at<T, FAST>(crow[v], cinf[v], p, lt).be, x[v], t.v[v]);
              o.v[v] = x[v];
              if (REDUCE) acc.add(abs2(x[v]));
            }
            if (active) *reinterpret_cast<Pk*>(out + (long long)p * a.stride) = o;
          }
        };
        if (fast)
          back(bool_tag<true>{});
        else
          back(bool_tag<false>{});
      }
      issue(q + R - 1);
    }
    cp_async_wait<0>();
  }
  if (REDUCE) norm_epilogue(acc.value(), a);
}

// Complex float, two lines per lane: the same pipeline with the two lines in
// split form (packed FP32x2 arithmetic, sweep_common.cuh); d' is kept in the
// ring in split form and joined back to interleaved complex on the store.
template <int C, bool FAST>
__device__ __forceinline__ void strided_forward2(float4* s0, c2& pm, c2& d,
                                                 const coef5<float>* const (&crow)[2],
                                                 const coef2& cf, int p0, int lt) {
  // stage the chunk (and the next point) in registers first: the solve then
  // never waits on a shared load queued behind its own stores
  float4 w[C + 1];
#pragma unroll
  for (int r = 0; r <= C; ++r) w[r] = s0[r * 32];
  c2 cur = split2(w[0]);
#pragma unroll
  for (int r = 0; r < C; ++r) {
    const c2 nx = split2(w[r + 1]);
    coef2 k;
    if (FAST) {
      k = cf;
    } else {
      const int i = min(p0 + r, lt);
      k = make_coef2(crow[0][i], crow[1][i]);
    }
    d = fwd2(k, pm, cur, nx, d);
    pm = cur;
    w[r] = pack_split(d);
    cur = nx;
  }
#pragma unroll
  for (int r = 0; r < C; ++r) s0[r * 32] = w[r];
}

// RING: slots of the chunk ring (3 or 4), a compile-time constant so that
// slot indices are cheap.
template <int C, bool REDUCE, int RING>
__global__ void __launch_bounds__(128) k_sweep_strided2(const stream_args a) {
  using E = cpx<float>;
  constexpr int SLOT = (C + 1) * 32;  // float4 (two complex) per slot
  constexpr int R = RING;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  if (a.ring != R ||
      dynamic_smem_bytes() < (blockDim.x >> 5) * (unsigned)(R * SLOT) * 16u) {
    if (threadIdx.x == 0) atomicOr(a.flags, 2);
    return;
  }
  float4* ring = reinterpret_cast<float4*>(smem_raw) + (size_t)wib * R * SLOT;
  const long long ngroups = (a.nlines + 63) / 64;
  const long long wg = (long long)blockIdx.x * (blockDim.x >> 5) + wib;
  acc_t<float> acc;
  if (wg < ngroups * a.nseg) {
    const long long g = wg % ngroups;
    const int sg = (int)(wg / ngroups);
    const long long c0 = (g * 32 + lane) * 2;
    const bool active = c0 < a.nlines;
    const long long base = active ? (c0 / a.nx) * a.outer + (c0 % a.nx) : 0;
    const E* in = static_cast<const E*>(a.in) + base;
    E* out = static_cast<E*>(a.out) + base;
    const int N = a.len, nch = (N + C - 1) / C, lt = a.lt;
    const int qo0 = sg * a.seg_chunks, qo1 = min(nch, qo0 + a.seg_chunks);
    const int qa = max(0, qo0 - a.warm), qb = min(nch, qo1 + 1);
    const coef5<float>* crow[2];
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int li = (a.coef_mode == 1 && active) ? (int)((c0 + v) % a.nx) : 0;
      crow[v] = static_cast<const coef5<float>*>(a.coef) + (size_t)li * (lt + 1);
    }
    const coef2 cf = make_coef2(crow[0][lt], crow[1][lt]);
    auto slot = [&](int q) { return ring + (size_t)(q % R) * SLOT + lane; };
    auto issue = [&](int q) {
      if (q < qb) {
        float4* sl = slot(q);
#pragma unroll
        for (int r = 0; r <= C; ++r) {
          const int p = q * C + r;
          if (active && p < N)
            cp_async<16>(&sl[r * 32], in + (long long)p * a.stride);
          else
            sl[r * 32] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      cp_async_commit();
    };
    for (int i = 0; i < R - 1; ++i) issue(qa + i);
    c2 pm = zero2(), d = zero2();
    for (int q = qa; q <= qb; ++q) {
      if (q < qb) {
        if (R == 3)
          cp_async_wait<1>();
        else
          cp_async_wait<2>();
        if (q * C >= lt && (q + 1) * C <= N)
          strided_forward2<C, true>(slot(q), pm, d, crow, cf, q * C, lt);
        else
          strided_forward2<C, false>(slot(q), pm, d, crow, cf, q * C, lt);
      }
      const int qq = q - 1;
      if (qq >= qo0 && qq < qo1) {
        c2 x = zero2();
        const int la = min(a.halo, N - q * C);
        const float4* sq = slot(q);
        const bool la_fast = q * C >= lt;
#pragma unroll
        for (int h = C - 1; h >= 0; --h) {
          if (h >= la) continue;  // the halo is at most one chunk
          k2 be = cf.be;
          if (!la_fast) {
            const int i = min(q * C + h, lt);
            be = make_k2(crow[0][i].be, crow[1][i].be);
          }
          x = kfma2(be, x, unpack_split(sq[h * 32]));
        }
        const float4* sp = slot(qq);
        const bool fast = qq * C >= lt && q * C <= N;
        auto back = [&](auto fast_tag) {
          constexpr bool FAST = decltype(fast_tag)::value;
          float4 w[C];
#pragma unroll
          for (int r = 0; r < C; ++r) w[r] = sp[r * 32];
#pragma unroll
          for (int r = C - 1; r >= 0; --r) {
            const int p = qq * C + r;
            if (!FAST && p >= N) continue;
            k2 be;
            if (FAST) {
              be = cf.be;
            } else {
              const int i = min(p, lt);
              be = make_k2(crow[0][i].be, crow[1][i].be);
            }
            x = kfma2(be, x, unpack_split(w[r]));
            if (REDUCE) {
              const float2 n2 = __ffma2_rn(x.im, x.im, __fmul2_rn(x.re, x.re));
              acc.add(n2.x + n2.y);
            }
            if (active) *reinterpret_cast<float4*>(out + (long long)p * a.stride) = join2(x);
          }
        };
        if (fast)
          back(bool_tag<true>{});
        else
          back(bool_tag<false>{});
      }
      issue(q + R - 1);
    }
    cp_async_wait<0>();
  }
  if (REDUCE) norm_epilogue(acc.value(), a);
}

// --------------------------------------------------------------- launchers
cudaError_t launch_tables(bool fp64, void* table, int nlines, int lt, const axis_coef& co,
                          cudaStream_t s) {
  const int threads = 128, blocks = (nlines + threads - 1) / threads;
  if (fp64)
    k_tables<double><<<blocks, threads, 0, s>>>(static_cast<coef5<double>*>(table), nlines, lt, co);
  else
    k_tables<float><<<blocks, threads, 0, s>>>(static_cast<coef5<float>*>(table), nlines, lt, co);
  return cudaGetLastError();
}

size_t sweep_smem_per_warp(bool fp64, bool x_sweep, int V, int C, int R) {
  const size_t e = fp64 ? 16 : 8;
  if (x_sweep) return (size_t)R * (32 * V) * (fp64 ? C + 1 : C + 2) * e;
  return (size_t)R * (C + 1) * 32 * V * e;
}

cudaError_t allow_smem(const void* fn, bool* done) {
  if (*done) return cudaSuccess;
  int dev = 0, optin = 0;
  cudaFuncAttributes fa{};
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess) *done = true;
  return e;
}

template <class T, int V, int C>
static cudaError_t dispatch_s(bool reduce, const stream_args& a, const sweep_shape& sh,
                              cudaStream_t s) {
  static bool done[2] = {false, false};
  auto fn = reduce ? k_sweep_strided<T, V, C, true> : k_sweep_strided<T, V, C, false>;
  cudaError_t e = allow_smem((const void*)fn, &done[reduce ? 1 : 0]);
  if (e != cudaSuccess) return e;
  fn<<<(unsigned)sh.blocks, 32 * sh.warps_per_block, sh.smem, s>>>(a);
  return cudaGetLastError();
}

template <int C>
static cudaError_t dispatch_s2(bool reduce, const stream_args& a, const sweep_shape& sh,
                               cudaStream_t s) {
  static bool done[4] = {false, false, false, false};
  if (sh.R != 3 && sh.R != 4) return cudaErrorInvalidValue;
  auto fn = sh.R == 3 ? (reduce ? k_sweep_strided2<C, true, 3> : k_sweep_strided2<C, false, 3>)
                      : (reduce ? k_sweep_strided2<C, true, 4> : k_sweep_strided2<C, false, 4>);
  cudaError_t e = allow_smem((const void*)fn, &done[(sh.R == 4 ? 2 : 0) + (reduce ? 1 : 0)]);
  if (e != cudaSuccess) return e;
  fn<<<(unsigned)sh.blocks, 32 * sh.warps_per_block, sh.smem, s>>>(a);
  return cudaGetLastError();
}

// Every (precision, V, C) combination the host can choose is instantiated
// here; anything else is rejected before a launch.
// One line per lane, complex float, chunks by TMA (the strided counterpart
// of k_sweep_x1t).  A warp owns 32 consecutive x of one transverse position
// (z for y lines, AX = 1; y for z lines, AX = 2): one line position of its
// 32 lines is 256 contiguous bytes, so each chunk of C + 1 positions is one
// 3-D TMA box landing as [position][lane] (conflict-free 8-byte shared
// reads), and every output position is one coalesced 256-byte store straight
// from registers.  Arithmetic on the interleaved (re, im) layout with two
// packed-FP32x2 accumulators, as in k_sweep_x1t.
template <int C, bool REDUCE, int RING, int AX>
__global__ void __launch_bounds__(128) k_sweep_s1t(const __grid_constant__ CUtensorMap map,
                                                   const stream_args a) {
  constexpr int R = RING;
  constexpr int SLOT = (C + 1) * 32;  // float2 per slot
  static_assert((SLOT * 8) % 128 == 0, "TMA slots");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[4 * 4];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  if (a.ring != R || blockDim.x > 128 ||
      dynamic_smem_bytes() < (blockDim.x >> 5) * (unsigned)(R * SLOT * 8) + 128u) {
    if (threadIdx.x == 0) atomicOr(a.flags, 2);
    return;
  }
  unsigned char* sbase = smem_raw + ((128 - (smem_addr(smem_raw) & 127)) & 127);
  float2* ring = reinterpret_cast<float2*>(sbase) + (size_t)wib * R * SLOT;
  uint64_t* bar = bars + wib * 4;
  const int tiles_x = (a.nx + 31) / 32;
  const int nt = (int)(a.nlines / a.nx);  // transverse positions
  const long long ngroups = (long long)tiles_x * nt;
  const long long wg = (long long)blockIdx.x * (blockDim.x >> 5) + wib;
  acc_t<float> acc;
  if (wg < ngroups * a.nseg) {
    const long long g = wg % ngroups;
    const int sg = (int)(wg / ngroups);
    const int gx = (int)(g % tiles_x), gt = (int)(g / tiles_x);
    const int x = 32 * gx + lane;
    const bool act = x < a.nx;
    const int N = a.len, nch = (N + C - 1) / C, lt = a.lt;
    const int qo0 = sg * a.seg_chunks, qo1 = min(nch, qo0 + a.seg_chunks);
    const int qa = max(0, qo0 - a.warm), qb = min(nch, qo1 + 1);
    const long long base = (long long)gt * a.outer + x;  // the line's point 0
    float2* out = static_cast<float2*>(a.out) + (act ? base : 0);
    const coef5<float>* crow = static_cast<const coef5<float>*>(a.coef) +
                               (size_t)(a.coef_mode == 1 && act ? x : 0) * (lt + 1);
    float2 A0R, A0I, AMR, AMI, APR, API, ALR, ALI, BER, BEI;
    {
      const coef5<float> cf = crow[lt];
      wsplit(make_float2(cf.a0.x, cf.a0.y), A0R, A0I);
      wsplit(make_float2(cf.am.x, cf.am.y), AMR, AMI);
      wsplit(make_float2(cf.ap.x, cf.ap.y), APR, API);
      wsplit(make_float2(cf.al.x, cf.al.y), ALR, ALI);
      wsplit(make_float2(cf.be.x, cf.be.y), BER, BEI);
    }
    auto fwd_fast = [&](float2 pm, float2 pc, float2 pn, float2 d) -> float2 {
      float2 A = __fmul2_rn(A0R, pc), B = __fmul2_rn(A0I, pc);
      A = __ffma2_rn(AMR, pm, A);
      B = __ffma2_rn(AMI, pm, B);
      A = __ffma2_rn(APR, pn, A);
      B = __ffma2_rn(API, pn, B);
      A = __ffma2_rn(ALR, d, A);
      B = __ffma2_rn(ALI, d, B);
      return make_float2(A.x - B.y, A.y + B.x);
    };
    auto fwd_tab = [&](int p, float2 pm, float2 pc, float2 pn, float2 d) -> float2 {
      const coef5<float> k = crow[min(p, lt)];
      cacc c = cacc_zero();
      float2 wr, wi;
      wsplit(make_float2(k.a0.x, k.a0.y), wr, wi);
      cmac(c, wr, wi, pc);
      wsplit(make_float2(k.am.x, k.am.y), wr, wi);
      cmac(c, wr, wi, pm);
      wsplit(make_float2(k.ap.x, k.ap.y), wr, wi);
      cmac(c, wr, wi, pn);
      wsplit(make_float2(k.al.x, k.al.y), wr, wi);
      cmac(c, wr, wi, d);
      return cfin(c);
    };
    auto bstep = [&](float2 br, float2 bi, float2 xx, float2 dp) -> float2 {
      const float2 A = __ffma2_rn(br, xx, dp), B = __fmul2_rn(bi, xx);
      return make_float2(A.x - B.y, A.y + B.x);
    };
    auto be_at = [&](int p, float2& br, float2& bi) {
      const coef5<float> k = crow[min(p, lt)];
      wsplit(make_float2(k.be.x, k.be.y), br, bi);
    };
    auto slot = [&](int q) { return ring + (size_t)((q - qa) % R) * SLOT + lane; };
    auto issue = [&](int q) {
      if (q < qb && lane == 0) {
        const int sl = (q - qa) % R;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bar[sl], (unsigned)(SLOT * 8));
        if (AX == 1)
          tma_load_3d(ring + (size_t)sl * SLOT, &map, 64 * gx, q * C, gt, &bar[sl]);
        else
          tma_load_3d(ring + (size_t)sl * SLOT, &map, 64 * gx, gt, q * C, &bar[sl]);
      }
    };
    if (lane == 0) {
      for (int i = 0; i < R; ++i) mbar_init(&bar[i], 1);
      mbar_fence_init();
    }
    __syncwarp();
    for (int i = 0; i < R - 1; ++i) issue(qa + i);
    float2 pm = make_float2(0.f, 0.f), d = make_float2(0.f, 0.f);
    bool good = true;
    for (int q = qa; q <= qb && good; ++q) {
      if (q < qb) {
        if (!__all_sync(0xffffffffu,
                        mbar_wait(&bar[(q - qa) % R], (unsigned)(((q - qa) / R) & 1)))) {
          for (int r = q + 1; r < min(q + R - 1, qb); ++r)
            mbar_wait(&bar[(r - qa) % R], (unsigned)(((r - qa) / R) & 1));
          if (lane == 0) atomicOr(a.flags, 4);
          good = false;
          break;
        }
        float2* sp = slot(q);
        const int p0 = q * C;
        float2 w[C + 1];
#pragma unroll
        for (int r = 0; r <= C; ++r) w[r] = sp[r * 32];
        if (p0 >= lt && p0 + C <= N) {
#pragma unroll
          for (int r = 0; r < C; ++r) {
            const float2 pc = w[r];
            d = fwd_fast(pm, pc, w[r + 1], d);
            pm = pc;
            sp[r * 32] = d;
          }
        } else {
#pragma unroll
          for (int r = 0; r < C; ++r) {
            const float2 pc = w[r];
            d = fwd_tab(p0 + r, pm, pc, w[r + 1], d);
            pm = pc;
            sp[r * 32] = d;
          }
        }
      }
      const int qq = q - 1;
      if (qq >= qo0 && qq < qo1) {
        float2 xx = make_float2(0.f, 0.f);
        const int la = min(a.halo, N - q * C);
        const float2* sq = slot(q);
        const bool la_fast = q * C >= lt;
#pragma unroll
        for (int h = C - 1; h >= 0; --h) {
          if (h >= la) continue;  // the halo is at most one chunk
          float2 br = BER, bi = BEI;
          if (!la_fast) be_at(q * C + h, br, bi);
          xx = bstep(br, bi, xx, sq[h * 32]);
        }
        const float2* sp = slot(qq);
        const int p0 = qq * C;
        float2 w[C];
#pragma unroll
        for (int r = 0; r < C; ++r) w[r] = sp[r * 32];
        const bool fast = p0 >= lt && q * C <= N;
#pragma unroll
        for (int r = C - 1; r >= 0; --r) {
          const int p = p0 + r;
          if (!fast && p >= N) continue;
          float2 br = BER, bi = BEI;
          if (!fast) be_at(p, br, bi);
          xx = bstep(br, bi, xx, w[r]);
          if (act) out[(long long)p * a.stride] = xx;
          if (REDUCE) acc.add(fmaf(xx.x, xx.x, xx.y * xx.y));
        }
      }
      __syncwarp();
      issue(q + R - 1);
    }
  }
  if (REDUCE) norm_epilogue(acc.value(), a);
}

template <int C, int R, int AX>
static cudaError_t dispatch_s1t(bool reduce, const stream_args& a, const sweep_shape& sh,
                                const void* map, cudaStream_t s) {
  static bool done[2] = {false, false};
  if (sh.warps_per_block > 4) return cudaErrorInvalidValue;
  const CUtensorMap& m = *static_cast<const CUtensorMap*>(map);
  auto fn = reduce ? k_sweep_s1t<C, true, R, AX> : k_sweep_s1t<C, false, R, AX>;
  cudaError_t e = allow_smem((const void*)fn, &done[reduce ? 1 : 0]);
  if (e != cudaSuccess) return e;
  const long long groups = (long long)((a.nx + 31) / 32) * (a.nlines / a.nx);
  const unsigned blocks =
      (unsigned)((groups * a.nseg + sh.warps_per_block - 1) / sh.warps_per_block);
  fn<<<blocks, 32 * sh.warps_per_block, sh.smem + 128, s>>>(m, a);
  return cudaGetLastError();
}

long long strided1_blocks(long long nlines, int nx, int nseg) {
  return (long long)((nx + 31) / 32) * (nlines / nx) * nseg;
}

cudaError_t launch_sweep_strided(bool fp64, bool reduce, const stream_args& a,
                                 const sweep_shape& sh, const void* map, int axis,
                                 cudaStream_t s) {
  if (!fp64 && sh.V == 1 && (sh.C == 8 || sh.C == 16) && map) {
    // one line per lane through TMA (the host passes the box map of this axis and C)
#define ROTGP_S1(CC, RR)                                                             \
  if (sh.C == CC && sh.R == RR)                                                      \
    return axis == 1 ? dispatch_s1t<CC, RR, 1>(reduce, a, sh, map, s)                \
                     : dispatch_s1t<CC, RR, 2>(reduce, a, sh, map, s);
    ROTGP_S1(8, 3)
    ROTGP_S1(8, 4)
    ROTGP_S1(16, 3)
    ROTGP_S1(16, 4)
#undef ROTGP_S1
    return cudaErrorInvalidValue;
  }
  if (fp64) {
    if (sh.V == 1 && sh.C == 16) return dispatch_s<double, 1, 16>(reduce, a, sh, s);
    if (sh.V == 1 && sh.C == 64) return dispatch_s<double, 1, 64>(reduce, a, sh, s);
    return cudaErrorInvalidValue;
  }
  if (sh.V == 2 && sh.C == 8) return dispatch_s2<8>(reduce, a, sh, s);
  if (sh.V == 2 && sh.C == 16) return dispatch_s2<16>(reduce, a, sh, s);
  if (sh.V == 1 && sh.C == 16) return dispatch_s<float, 1, 16>(reduce, a, sh, s);
  if (sh.V == 1 && sh.C == 64) return dispatch_s<float, 1, 64>(reduce, a, sh, s);
  return cudaErrorInvalidValue;
}

}  // namespace rotgp
