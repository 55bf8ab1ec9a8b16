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
#include <algorithm>
#include <map>
#include <set>
#include <mutex>
#include <tuple>

#include "sweep_common.cuh"
#include "tma.cuh"

namespace rotgp {

// --------------------------------------------------------------- tables
// Thomas multipliers of one line, m_1 = 1/A0, c'_1 = A+ m_1,
// m_p = 1/(A0 - A- c'_{p-1}), c'_p = A+ m_p, folded into coef5 entries
// p = 1..lt (computed in double, a0 as its difference from 1); entry 0 is
// zero.
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
__global__ void k_tables(coef5<T>* tab, float2* tabT, int nlines, int lt, axis_coef co) {
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
  t[0].a0 = t[0].am = t[0].ap = t[0].al = t[0].be = t[0].m2 = zero<T>();
  dcx c{0.0, 0.0};
  for (int p = 1; p <= lt; ++p) {
    const dcx m = dinv(dsub(a0, dmul(am, c)));
    c = dmul(ap, m);
    const dcx md = dmul(m, diag);
    t[p].a0 = dcast<T>({md.x - 1.0, md.y});
    t[p].am = dcast<T>(dmul(m, kmt));
    t[p].ap = dcast<T>(dmul(m, kpt));
    const dcx mam = dmul(m, am);
    t[p].al = dcast<T>({-mam.x, -mam.y});
    t[p].be = dcast<T>({-c.x, -c.y});
    t[p].m2 = dcast<T>({2.0 * m.x, 2.0 * m.y});
  }
  if (tabT) {
    const size_t P = (size_t)(lt + 1) * nlines;
    for (int p = 0; p <= lt; ++p) {
      const size_t i = (size_t)p * nlines + l;
      tabT[i] = make_float2((float)t[p].m2.x, (float)t[p].m2.y);
      tabT[P + i] = make_float2((float)t[p].al.x, (float)t[p].al.y);
      tabT[2 * P + i] = make_float2((float)t[p].be.x, (float)t[p].be.y);
    }
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
            x[v] = bwd(be, x[v], t.v[v]);
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
              x[v] = bwd(coef_at<T, FAST>(crow[v], cinf[v], p, lt).be, x[v], t.v[v]);
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
          x = bwd2(be, x, unpack_split(sq[h * 32]));
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
            x = bwd2(be, x, unpack_split(w[r]));
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
cudaError_t launch_tables(bool fp64, void* table, void* tableT, int nlines, int lt,
                          const axis_coef& co, cudaStream_t s) {
  const int threads = 128, blocks = (nlines + threads - 1) / threads;
  if (fp64)
    k_tables<double><<<blocks, threads, 0, s>>>(static_cast<coef5<double>*>(table), nullptr,
                                                nlines, lt, co);
  else
    k_tables<float><<<blocks, threads, 0, s>>>(static_cast<coef5<float>*>(table),
                                               static_cast<float2*>(tableT), nlines, lt, co);
  return cudaGetLastError();
}

size_t s1t_smem_per_warp(int C, int R) { return (size_t)(R + 1) * C * 32 * 8; }

size_t sweep_smem_per_warp(bool fp64, bool x_sweep, int V, int C, int R) {
  const size_t e = fp64 ? 16 : 8;
  if (x_sweep) {
    const size_t chunked = (size_t)R * (32 * V) * (fp64 ? C + 1 : C + 2) * e;
    // one row per lane in complex float: the TMA form, R + 1 slots of 32 x C
    if (!fp64 && V == 1 && (C == 8 || C == 16))
      return std::max(chunked, (size_t)(R + 1) * 32 * C * 8);
    return chunked;
  }
  const size_t chunked = (size_t)R * (C + 1) * 32 * V * e;
  // one line per lane in complex float: the TMA form may serve it
  if (!fp64 && V == 1 && (C == 8 || C == 16)) return std::max(chunked, s1t_smem_per_warp(C, R));
  return chunked;
}

// Grid of a kernel whose warps take work units round-robin: W warps per
// block (at most max_warps, and no more than the units per SM, so that the units
// spread over every SM) and as many blocks as are resident at once, at most
// one per W units.  One launch wave of long-lived warps replaces a block per
// unit (block launches and, in the last sweep, norm partials per block).
cudaError_t resident_grid(const void* fn, long long units, size_t smem_per_warp, size_t extra,
                          int max_warps, int* warps, unsigned* blocks) {
  int dev = 0, sms = 0, nb = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  // launch shapes are asked for every sweep launch: remember them
  static std::mutex mu;
  static std::map<std::tuple<const void*, long long, size_t, size_t, int, int>,
                  std::pair<int, unsigned>>
      memo;
  const auto key = std::make_tuple(fn, units, smem_per_warp, extra, max_warps, dev);
  {
    std::lock_guard<std::mutex> lk(mu);
    const auto it = memo.find(key);
    if (it != memo.end()) {
      *warps = it->second.first;
      *blocks = it->second.second;
      return cudaSuccess;
    }
  }
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  int W = (int)std::min<long long>(max_warps, std::max<long long>(1, (units + sms - 1) / sms));
  for (; W >= 1; --W) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, 32 * W, smem_per_warp * W + extra);
    if (e != cudaSuccess) return e;
    if (nb >= 1) break;
  }
  if (W < 1) return cudaErrorInvalidConfiguration;
  *warps = W;
  *blocks = (unsigned)std::max<long long>(
      1, std::min<long long>((units + W - 1) / W, (long long)sms * nb));
  std::lock_guard<std::mutex> lk(mu);
  memo[key] = {*warps, *blocks};
  return cudaSuccess;
}

// Opt a kernel in to at least `bytes` of dynamic shared memory (bytes < 0:
// all that the device allows beside its static shared memory) on the current
// device.  The attribute belongs to the kernel on that device; it is only
// ever raised (a launch with fewer bytes stays valid), so a context on a
// second device in the same process sets its own and launches of one kernel
// with different tile sizes never undo each other.
cudaError_t allow_smem_bytes(const void* fn, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> opted;  // (kernel, device) -> bytes
  const auto key = std::make_pair(fn, dev);
  std::lock_guard<std::mutex> lk(mu);
  const auto it = opted.find(key);
  if (bytes >= 0 && it != opted.end() && it->second >= bytes) return cudaSuccess;
  if (bytes < 0) {
    if (it != opted.end() && it->second == -1) return cudaSuccess;
    int optin = 0;
    cudaFuncAttributes fa{};
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess) opted[key] = -1;  // the maximum: covers every request
    return e;
  }
  if (it != opted.end() && it->second == -1) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) opted[key] = bytes;
  return e;
}

cudaError_t allow_smem(const void* fn) { return allow_smem_bytes(fn, -1); }

template <class T, int V, int C>
static cudaError_t dispatch_s(bool reduce, const stream_args& a, const sweep_shape& sh,
                              cudaStream_t s) {
  auto fn = reduce ? k_sweep_strided<T, V, C, true> : k_sweep_strided<T, V, C, false>;
  cudaError_t e = allow_smem((const void*)fn);
  if (e != cudaSuccess) return e;
  fn<<<(unsigned)sh.blocks, 32 * sh.warps_per_block, sh.smem, s>>>(a);
  return cudaGetLastError();
}

template <int C>
static cudaError_t dispatch_s2(bool reduce, const stream_args& a, const sweep_shape& sh,
                               cudaStream_t s) {
  if (sh.R != 3 && sh.R != 4) return cudaErrorInvalidValue;
  auto fn = sh.R == 3 ? (reduce ? k_sweep_strided2<C, true, 3> : k_sweep_strided2<C, false, 3>)
                      : (reduce ? k_sweep_strided2<C, true, 4> : k_sweep_strided2<C, false, 4>);
  cudaError_t e = allow_smem((const void*)fn);
  if (e != cudaSuccess) return e;
  fn<<<(unsigned)sh.blocks, 32 * sh.warps_per_block, sh.smem, s>>>(a);
  return cudaGetLastError();
}

// Every (precision, V, C) combination the host can choose is instantiated
// here; anything else is rejected before a launch.
// One line per lane, complex float, TMA in and out.  A warp owns 32
// consecutive x of one transverse position (z for y lines, AX = 1; y for z
// lines, AX = 2): one line position of its 32 lines is 256 contiguous bytes,
// so a chunk of C positions is one 3-D TMA box landing as [position][lane]
// (conflict-free 8-byte shared reads), and the finished chunk leaves the
// same slot as one TMA box store.
//
// The step is solved unfolded: with A y = psi, psi' = 2y - psi, so
//   forward   d_p = m2_p psi_p + al_p d_{p-1}          (m2 = 2 m)
//   backward  z_p = d_p + be_p z_{p+1},   psi'_p = z_p - psi_p
// (two complex multiply-adds forward, one back, and no neighbour points).
// d of a chunk stays in registers until the chunk's back substitution one
// chunk later, which starts from a truncated carry: the next chunk back-
// substituted from zero at its end (C >= H points, error below decay^H).
// The ring holds R + 1 slots: R - 1 chunk loads in flight ahead of the
// forward sweep, the chunk being back-substituted, and one more whose store
// may still be reading shared memory.  Arithmetic on the interleaved
// (re, im) layout with packed FP32x2 (cacc form, sweep_common.cuh).
template <int C, bool REDUCE, int RING, int AX>
__global__ void __launch_bounds__(C == 8 ? 512 : 256) k_sweep_s1t(const __grid_constant__ CUtensorMap map,
                                                   const __grid_constant__ CUtensorMap omap,
                                                   const stream_args a) {
  constexpr int NS = RING + 1;        // slots per warp
  constexpr int SLOT = C * 32;        // float2 per slot
  static_assert((SLOT * 8) % 128 == 0 && NS <= 8, "TMA slots");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[16 * 8];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  if (a.ring != RING || blockDim.x > (C == 8 ? 512u : 256u) ||
      dynamic_smem_bytes() < (blockDim.x >> 5) * (unsigned)(NS * SLOT * 8) + 128u) {
    if (threadIdx.x == 0) atomicOr(a.flags, 2);
    return;
  }
  unsigned char* sbase = smem_raw + ((128 - (smem_addr(smem_raw) & 127)) & 127);
  float2* ring = reinterpret_cast<float2*>(sbase) + (size_t)wib * NS * SLOT;
  uint64_t* bar = bars + wib * 8;
  const int tiles_x = (a.nx + 31) / 32;
  const int nt = (int)(a.nlines / a.nx);  // transverse positions
  const long long ngroups = (long long)tiles_x * nt;
  acc_t<float> acc;
  if (lane == 0) {
    for (int i = 0; i < NS; ++i) mbar_init(&bar[i], 1);
    mbar_fence_init();
  }
  __syncwarp();
  // launched programmatically: the next sweep's blocks may be scheduled as
  // SMs free up; the previous kernel's state and pending scale are complete
  // and visible past this wait, and nothing above touched global memory
  griddep_launch_dependents();
  griddep_wait();
  const uint64_t pol_first = l2_evict_first(), pol_last = l2_evict_last();
  unsigned ph = 0;  // phase parity of every slot's barrier, kept from unit to unit
  bool good = true;
  // units (a patch of 32 lines and one segment of them) in a fixed
  // round-robin order over the resident warps
  const long long nunits = ngroups * a.nseg;
  const long long wstride = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long wg = (long long)blockIdx.x * (blockDim.x >> 5) + wib; wg < nunits && good;
       wg += wstride) {
    const long long g = wg % ngroups;
    const int sg = (int)(wg / ngroups);
    const int gx = (int)(g % tiles_x), gt = (int)(g / tiles_x);
    const int x = 32 * gx + lane;
    const bool act = x < a.nx;
    const int N = a.len, nch = (N + C - 1) / C, lt = a.lt;
    const int qo0 = sg * a.seg_chunks, qo1 = min(nch, qo0 + a.seg_chunks);
    const int qa = max(0, qo0 - a.warm), qb = min(nch, qo1 + 1);
    const int li = a.coef_mode == 1 && act ? x : 0;  // the line's coefficient line
    const float2* tab = a.coefT;
    const int tl = a.tlines;
    float2 M2R, M2I, ALR, ALI, BER, BEI;
    wsplit(coef_plane(tab, tl, lt, 0, lt, li, pol_last), M2R, M2I);
    wsplit(coef_plane(tab, tl, lt, 1, lt, li, pol_last), ALR, ALI);
    wsplit(coef_plane(tab, tl, lt, 2, lt, li, pol_last), BER, BEI);
    const float2 NEG1 = make_float2(-1.f, -1.f);
    // d_p = m2 psi_p + al d_{p-1}
    auto fwd = [](float2 mr, float2 mi, float2 lr, float2 li, float2 psi, float2 d) -> float2 {
      float2 A = __fmul2_rn(mr, psi), B = __fmul2_rn(mi, psi);
      A = __ffma2_rn(lr, d, A);
      B = __ffma2_rn(li, d, B);
      return make_float2(A.x - B.y, A.y + B.x);
    };
    // z_p = d_p + be z_{p+1}
    auto bstep = [](float2 br, float2 bi, float2 z, float2 dp) -> float2 {
      const float2 A = __ffma2_rn(br, z, dp), B = __fmul2_rn(bi, z);
      return make_float2(A.x - B.y, A.y + B.x);
    };
    auto coords = [&](int q, int& c1, int& c2) {
      c1 = AX == 1 ? q * C : gt;
      c2 = AX == 1 ? gt : q * C;
    };
    auto issue = [&](int q, int sl) {  // lane 0
      int c1, c2;
      coords(q, c1, c2);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(&bar[sl], (unsigned)(SLOT * 8));
      tma_load_3d_hint(ring + (size_t)sl * SLOT, &map, 64 * gx, c1, c2, &bar[sl],
                       pol_first);
    };
    if (lane == 0) {
      bulk_wait_read<0>();  // the previous unit's stores have left their slots
      for (int q = qa; q < min(qa + RING - 1, qb); ++q) issue(q, q - qa);
    }
    __syncwarp();
    float2 d = make_float2(0.f, 0.f);
    int sq = 0;  // slot of chunk q
    // forward over chunk q into cur[], back substitution and store of chunk
    // q - 1 from prv[], then the load of chunk q + R - 1 (into chunk q - 2's slot)
    auto step = [&](int q, float2 (&cur)[C], float2 (&prv)[C]) -> bool {
      if (q < qb) {
        if (!__all_sync(0xffffffffu, mbar_wait(&bar[sq], (ph >> sq) & 1u))) {
          int s = sq;
          for (int r = q + 1; r < min(q + RING - 1, qb); ++r) {
            s = s + 1 == NS ? 0 : s + 1;
            mbar_wait(&bar[s], (ph >> s) & 1u);
          }
          if (lane == 0) atomicOr(a.flags, 4);
          return false;
        }
        ph ^= 1u << sq;
        const float2* sp = ring + (size_t)sq * SLOT + lane;
        const int p0 = q * C;
        if (p0 >= lt && p0 + C <= N) {
#pragma unroll
          for (int r = 0; r < C; ++r) {
            d = fwd(M2R, M2I, ALR, ALI, sp[r * 32], d);
            cur[r] = d;
          }
        } else {
          float2 km[C], kl[C];
          table_fwd<C>(tab, tl, lt, li, p0, pol_last, km, kl);
#pragma unroll
          for (int r = 0; r < C; ++r) {
            float2 mr, mi, lr, li;
            wsplit(km[r], mr, mi);
            wsplit(kl[r], lr, li);
            d = fwd(mr, mi, lr, li, sp[r * 32], d);
            cur[r] = d;
          }
        }
      }
      const int qq = q - 1;
      bool stored = false;
      if (qq >= qo0 && qq < qo1) {
        float2 z = make_float2(0.f, 0.f);
        if (q < qb) {
          const int p0 = q * C;
          if (p0 >= lt && p0 + C <= N) {
#pragma unroll
            for (int h = C - 1; h >= 0; --h) z = bstep(BER, BEI, z, cur[h]);
          } else {
            float2 kb[C];
            table_be<C>(tab, tl, lt, li, p0, pol_last, kb);
#pragma unroll
            for (int h = C - 1; h >= 0; --h)
              if (p0 + h < N) {
                float2 br, bi;
                wsplit(kb[h], br, bi);
                z = bstep(br, bi, z, cur[h]);
              }
          }
        }
        const int sl = sq == 0 ? NS - 1 : sq - 1;
        float2* sp = ring + (size_t)sl * SLOT + lane;
        const int p0 = qq * C;
        float2 n2 = make_float2(0.f, 0.f);
        if (p0 >= lt && p0 + C <= N) {
#pragma unroll
          for (int r = C - 1; r >= 0; --r) {
            z = bstep(BER, BEI, z, prv[r]);
            const float2 o = __ffma2_rn(NEG1, sp[r * 32], z);
            sp[r * 32] = o;
            if (REDUCE) n2 = __ffma2_rn(o, o, n2);
          }
        } else {
          float2 kb[C];
          table_be<C>(tab, tl, lt, li, p0, pol_last, kb);
#pragma unroll
          for (int r = C - 1; r >= 0; --r)
            if (p0 + r < N) {
              float2 br, bi;
              wsplit(kb[r], br, bi);
              z = bstep(br, bi, z, prv[r]);
              const float2 o = __ffma2_rn(NEG1, sp[r * 32], z);
              sp[r * 32] = o;
              if (REDUCE) n2 = __ffma2_rn(o, o, n2);
            }
        }
        if (REDUCE && act) acc.add(n2.x + n2.y);
        // the chunk's results are in its slot: one box store (columns past
        // N_x and points past N are clipped by the tensor map)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          int c1, c2;
          coords(qq, c1, c2);
          tma_store_3d(&omap, 64 * gx, c1, c2, ring + (size_t)sl * SLOT);
          bulk_commit();
        }
        stored = true;
      }
      // refill the slot of chunk q - 2: every lane left it before the
      // previous step's store; its own store is the older of at most two
      if (lane == 0 && q + RING - 1 < qb) {
        if (stored)
          bulk_wait_read<1>();
        else
          bulk_wait_read<0>();
        int sl = sq + NS - 2;
        if (sl >= NS) sl -= NS;
        issue(q + RING - 1, sl);
      }
      __syncwarp();
      sq = sq + 1 == NS ? 0 : sq + 1;
      return true;
    };
    float2 dA[C], dB[C];
#pragma unroll
    for (int r = 0; r < C; ++r) dA[r] = dB[r] = make_float2(0.f, 0.f);
    for (int q = qa; q <= qb; q += 2) {
      if (!step(q, dA, dB)) {
        good = false;
        break;
      }
      if (q + 1 > qb) break;
      if (!step(q + 1, dB, dA)) {
        good = false;
        break;
      }
    }
  }
  if (lane == 0) bulk_wait_all();
  if (REDUCE) norm_epilogue(acc.value(), a);
}

template <int C, int R, int AX>
static cudaError_t dispatch_s1t(bool reduce, const stream_args& a, const sweep_shape& sh,
                                const void* map, const void* omap, cudaStream_t s) {
  const CUtensorMap& m = *static_cast<const CUtensorMap*>(map);
  const CUtensorMap& om = *static_cast<const CUtensorMap*>(omap);
  auto fn = reduce ? k_sweep_s1t<C, true, R, AX> : k_sweep_s1t<C, false, R, AX>;
  cudaError_t e = allow_smem((const void*)fn);
  if (e != cudaSuccess) return e;
  const long long units = (long long)((a.nx + 31) / 32) * (a.nlines / a.nx) * a.nseg;
  int W = 1;
  unsigned blocks = 0;
  e = resident_grid((const void*)fn, units, s1t_smem_per_warp(C, R), 128, C == 8 ? 16 : 8, &W,
                    &blocks);
  if (e != cudaSuccess) return e;
  return launch_programmatic(fn, blocks, 32 * W, s1t_smem_per_warp(C, R) * W + 128, s, m, om, a);
}

long long strided1_blocks(long long nlines, int nx, int nseg) {
  return (long long)((nx + 31) / 32) * (nlines / nx) * nseg;
}

cudaError_t launch_sweep_strided(bool fp64, bool reduce, const stream_args& a,
                                 const sweep_shape& sh, const void* map, const void* omap,
                                 int axis, cudaStream_t s) {
  if (!fp64 && sh.V == 1 && (sh.C == 8 || sh.C == 16) && map && omap) {
    // one line per lane through TMA (the host passes the box map of this axis and C)
#define ROTGP_S1(CC, RR)                                                             \
  if (sh.C == CC && sh.R == RR)                                                      \
    return axis == 1 ? dispatch_s1t<CC, RR, 1>(reduce, a, sh, map, omap, s)          \
                     : dispatch_s1t<CC, RR, 2>(reduce, a, sh, map, omap, s);
    ROTGP_S1(8, 3)
    ROTGP_S1(8, 4)
    ROTGP_S1(8, 5)
    ROTGP_S1(8, 6)
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
