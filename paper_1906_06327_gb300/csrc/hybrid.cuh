// hybrid.cuh -- the tile step of the exact partition-method line solve
// (hybrid.cu describes the method): shared by the single-context sweep
// kernels (hybrid.cu) and the persistent multi-instance step (batch_kernel.cu).
#pragma once

#include <cooperative_groups.h>

#include "sweep_common.cuh"

namespace cg = cooperative_groups;

namespace rotgp {

namespace hyb {

constexpr int kHL = 16;                 // lines per tile
constexpr int kHS = 16;                 // sub-segments per line in one CTA (a half-warp)
constexpr int kHThreads = kHL * kHS;    // 256

template <class T>
__device__ __forceinline__ cpx<T> cmad(cpx<T> a, cpx<T> b, cpx<T> c) {
  return mk<T>(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

// Products with every rounding spelled out as fused multiply-adds, so that
// each kernel that inlines the tile step computes the same bits (no room for
// the compiler to contract differently from one kernel to another).
template <class T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
  return mk<T>(fma(a.x, b.x, -(a.y * b.y)), fma(a.x, b.y, a.y * b.x));
}
template <class T>
__device__ __forceinline__ T sq(cpx<T> a) {
  return fma(a.x, a.x, a.y * a.y);
}
template <class T>
__device__ __forceinline__ cpx<T> rscale(T s, cpx<T> a) {
  return mk<T>(s * a.x, s * a.y);
}

// z^n for n >= 0 by repeated squaring
template <class T>
__device__ __forceinline__ cpx<T> cpow_n(cpx<T> z, int n) {
  cpx<T> r = mk<T>(1, 0);
  while (n > 0) {
    if (n & 1) r = cmul(r, z);
    z = cmul(z, z);
    n >>= 1;
  }
  return r;
}

}  // namespace hyb
using namespace hyb;

struct hybrid_args {
  stream_args s;
  int cs;     // CTAs per line group (cluster size)
  int pc;     // positions per CTA (kHS * lsub)
  int lsub;   // positions per thread
  int vec;    // 1: 16-byte global accesses of two complex floats
  long long ngroups;
};

// One tile of the exact line solve: lines [16 grp, 16 grp + 16) of an axis
// (or 16 consecutive x at one transverse position), positions
// [rank pc, (rank + 1) pc) of them, read from a.in and written to a.out;
// H1 with the pending scale J.scale applied on the way in (x sweep).  Called
// by every thread of the block (and of the cluster, cs > 1) with the same job.
// Returns this thread's sum of |psi'|^2 over its points (REDUCE).
struct hybrid_job {
  long long grp;   // line group
  int rank;        // position block (CTA of the cluster)
  int cs, pc, lsub, vec;
  double scale;    // pending renormalisation (x sweep)
};

template <class T>
__device__ __forceinline__ cpx<T> ldcg_c(const cpx<T>* p) {
  cpx<T> v;
  v.x = __ldcg(&p->x);
  v.y = __ldcg(&p->y);
  return v;
}

// shuffles within the kHS lanes that hold the sub-segments of one line
template <class T>
__device__ __forceinline__ cpx<T> shfl_up_seg(cpx<T> v, int off) {
  return mk<T>(__shfl_up_sync(0xffffffffu, v.x, off, kHS),
               __shfl_up_sync(0xffffffffu, v.y, off, kHS));
}
template <class T>
__device__ __forceinline__ cpx<T> shfl_down_seg(cpx<T> v, int off) {
  return mk<T>(__shfl_down_sync(0xffffffffu, v.x, off, kHS),
               __shfl_down_sync(0xffffffffu, v.y, off, kHS));
}

template <int V>
struct int_tag {
  static constexpr int value = V;
};

template <class T, int AX, bool H1, bool IMAG, bool REDUCE>
__device__ __forceinline__ double hybrid_tile(const stream_args& a, const hybrid_job& J,
                                              unsigned char* smem_raw) {
  using E = cpx<T>;
  E* tile = reinterpret_cast<E*>(smem_raw);
  // per-line summaries of the sub-segments ([line][sub-segment], padded)
  __shared__ E sG[kHL][kHS + 1], sD[kHL][kHS + 1];
  // per-line totals of this CTA, read by the other CTAs of the cluster
  __shared__ E xG[kHL], xD[kHL], xB[kHL], xX[kHL];
  // H1: the y and z part of the potential of each line
  __shared__ T hv[kHL];

  cg::cluster_group cluster = cg::this_cluster();
  const int cs = J.cs, pc = J.pc, lsub = J.lsub, rank = J.rank;
  // a tile of whole lines (cs = 1) runs without a cluster: no cluster
  // barrier and no remote shared memory then
  auto csync = [&]() {
    if (cs > 1)
      cluster.sync();
    else
      __syncthreads();
  };
  const long long grp = J.grp;
  const int W = pc + 4;          // tile positions incl. 2 halo points either side
  const int N = a.len, lt = a.lt;
  const int p0 = rank * pc;      // first position of this CTA
  const int tid = threadIdx.x;
  const E* in = static_cast<const E*>(a.in);
  E* out = static_cast<E*>(a.out);
  __syncthreads();  // a previous tile of this block has left the shared memory

  // lines of the group: x lines are rows (j, k) -> row = grp * 16 + l;
  // y/z lines are 16 consecutive x at transverse position t
  const int tiles_x = (a.nx + kHL - 1) / kHL;
  const long long nrows = a.nlines;
  const long long t_pos = AX == 0 ? 0 : grp / tiles_x;
  const int x0l = AX == 0 ? 0 : (int)(grp % tiles_x) * kHL;
  auto line_ok = [&](int l) -> bool {
    return AX == 0 ? grp * kHL + l < nrows : x0l + l < a.nx;
  };
  // global index of (line l, position p)
  auto gidx = [&](int l, int p) -> long long {
    if (AX == 0) return (grp * kHL + l) * (long long)N + p;
    return t_pos * a.outer + x0l + l + (long long)p * a.stride;
  };
  // tile element (line l, tile position e), position p = p0 - 2 + e
  auto el = [&](int l, int e) -> E& {
    return AX == 0 ? tile[l * W + e] : tile[e * kHL + l];
  };

  // ---- load the tile (zeros outside the grid and past the line end), ep
  // complex numbers per copy
  auto load = [&](auto ep_tag) {
    constexpr int ep = decltype(ep_tag)::value;
    if (AX == 0) {
      for (int l = 0; l < kHL; ++l) {
        const bool ok = line_ok(l);
        const E* src = in + (grp * kHL + l) * (long long)N;
        E* dst = tile + l * W;
        for (int c = tid; c < W / ep; c += kHThreads) {
          const int e = c * ep, p = p0 - 2 + e;
          if (ok && p >= 0 && p + ep <= N) {
            cp_async<ep * sizeof(E)>(dst + e, src + p);
          } else {
#pragma unroll
            for (int q = 0; q < ep; ++q)
              dst[e + q] = (ok && p + q >= 0 && p + q < N) ? ldcg_c(src + p + q) : zero<T>();
          }
        }
      }
    } else {
      constexpr int per = kHL / ep;  // copies per tile position
      for (int u = tid; u < W * per; u += kHThreads) {
        const int e = u / per, l = (u % per) * ep, p = p0 - 2 + e;
        E* dst = &el(l, e);
        if (p >= 0 && p < N && line_ok(l + ep - 1)) {
          cp_async<ep * sizeof(E)>(dst, in + gidx(l, p));
        } else {
#pragma unroll
          for (int q = 0; q < ep; ++q)
            dst[q] = (line_ok(l + q) && p >= 0 && p < N) ? ldcg_c(in + gidx(l + q, p)) : zero<T>();
        }
      }
    }
  };
  if (sizeof(T) == 4 && J.vec)
    load(int_tag<2>{});
  else
    load(int_tag<1>{});
  if (H1 && tid < kHL) {
    const long long r = grp * kHL + tid;
    const int j = (int)(r % a.ny), kz = (int)(r / a.ny);
    const T y = (T)(a.y0 + (double)j * a.hy), z = (T)(a.z0 + (double)kz * a.hz);
    hv[tid] = fma((T)a.hnu2 * y, y, (T)a.hlam2 * z * z);
  }
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();

  // ---- H1 with the pending renormalisation (x sweep): psi <- s psi, then
  // exp(-Delta (V + g|psi|^2)) or exp(-i Delta (V + g|psi|^2)) (Eq. eq1).
  // Imaginary time advances the tile in place.  Real time leaves it as
  // loaded: each forward pass forms every point as value + increment (hpt)
  // when it reaches it.
  constexpr bool RT = H1 && !IMAG;
  const T h_s = (T)J.scale, h_gg = (T)a.g, h_dt = (T)a.dt;
  const T h_hg2 = (T)a.hgam2, h_xs = (T)a.x0, h_hx = (T)a.hx;
  if (H1 && IMAG) {
    const T s = (T)J.scale, hg2 = (T)a.hgam2, gg = (T)a.g, dt = (T)a.dt;
    const T xs = (T)a.x0, hx = (T)a.hx;
    for (int l = 0; l < kHL; ++l) {
      const T vyz = hv[l];
      E* row = tile + l * W;
      for (int e = tid; e < W; e += kHThreads) {
        const T x = fma((T)(p0 - 2 + e), hx, xs);
        E v = rscale(s, row[e]);
        const T en = fma(gg, sq(v), fma(hg2 * x, x, vyz));
        row[e] = rscale(exp_t(-dt * en), v);
      }
    }
    __syncthreads();
  }

  // ---- this thread's line and sub-segment
  const int l = AX == 0 ? tid / kHS : tid % kHL;
  const int k = AX == 0 ? tid % kHS : tid / kHL;
  const int pb = p0 + k * lsub;                      // first position
  const int nv = max(0, min(lsub, N - pb));          // positions inside the line
  const int it = max(0, min(nv, lt - pb));           // of them with a table entry
  const int eb = 2 + k * lsub;                       // its tile position
  int li = 0;                                        // coefficient line
  if (AX == 0) li = line_ok(l) ? (int)((grp * kHL + l) % a.ny) : 0;
  if (AX == 1) li = line_ok(l) ? x0l + l : 0;
  const coef5<T>* crow = static_cast<const coef5<T>*>(a.coef) + (size_t)li * (lt + 1);
  const coef5<T> cinf = crow[lt];
  // the scan threads: a half-warp over the sub-segments of one line
  const int l2 = tid / kHS, k2 = tid % kHS;

  // real time: the loaded value u of tile position e of this thread's line,
  // scaled and advanced
  auto rt_at = [&](E u, int e) -> hpt<T> {
    const T x = fma((T)(p0 - 2 + e), h_hx, h_xs);
    const E v = rscale(h_s, u);
    const T en = fma(h_gg, sq(v), fma(h_hg2 * x, x, hv[AX == 0 ? l : 0]));
    T c1, s1;
    rot_t(h_dt * en, &c1, &s1);
    return rot_inc(v, c1, s1);
  };
  auto rt = [&](int e) -> hpt<T> { return rt_at(el(l, e), e); };

  // ---- F1: local forward from a zero carry; summary (prod al, d at the end)
  const E left = el(l, eb - 1), right = el(l, eb + nv);
  if constexpr (RT) {
    E d = zero<T>(), G = mk<T>(1, 0);
    E pm = hw(rt_at(left, eb - 1));
    hpt<T> pc = rt(eb);
    int i = 0;
    for (; i < it; ++i) {
      const hpt<T> pn = i + 1 < nv ? rt(eb + i + 1) : rt_at(right, eb + nv);
      d = fwd_inc(crow[pb + i], pm, pc, hw(pn), d);
      G = cmul(crow[pb + i].al, G);
      pm = hw(pc);
      pc = pn;
    }
#pragma unroll 2
    for (; i < nv; ++i) {
      const hpt<T> pn = i + 1 < nv ? rt(eb + i + 1) : rt_at(right, eb + nv);
      d = fwd_inc(cinf, pm, pc, hw(pn), d);
      pm = hw(pc);
      pc = pn;
    }
    if (nv > it) G = cmul(G, cpow_n(cinf.al, nv - it));
    sG[l][k] = G;
    sD[l][k] = d;
  } else {
    E d = zero<T>(), G = mk<T>(1, 0);
    E pm = left, pcur = el(l, eb);
    int i = 0;
    for (; i < it; ++i) {
      const coef5<T> c = crow[pb + i];
      const E pn = el(l, eb + i + 1);
      d = fwd(c, pm, pcur, pn, d);
      G = cmul(c.al, G);
      pm = pcur;
      pcur = pn;
    }
#pragma unroll 4
    for (; i < nv; ++i) {
      const E pn = el(l, eb + i + 1);
      d = fwd(cinf, pm, pcur, pn, d);
      pm = pcur;
      pcur = pn;
    }
    if (nv > it) G = cmul(G, cpow_n(cinf.al, nv - it));
    sG[l][k] = G;
    sD[l][k] = d;
  }
  __syncthreads();
  // reduced system, forward: affine prefix over the sub-segments of a line
  // (log-depth scan in a half-warp), the CTA total to the cluster, and the true d
  // before every sub-segment
  {
    E g = sG[l2][k2], dd = sD[l2][k2];
#pragma unroll
    for (int off = 1; off < kHS; off <<= 1) {
      const E gp = shfl_up_seg(g, off), dp = shfl_up_seg(dd, off);
      if (k2 >= off) {
        dd = cmad(g, dp, dd);
        g = cmul(g, gp);
      }
    }
    if (k2 == kHS - 1) {
      xG[l2] = g;
      xD[l2] = dd;
    }
    csync();
    E cin = zero<T>();
    if (cs > 1) {
      E rg[8], rd[8];
#pragma unroll
      for (int r = 0; r < 8; ++r)
        if (r < rank) {
          rg[r] = cluster.map_shared_rank(xG, r)[l2];
          rd[r] = cluster.map_shared_rank(xD, r)[l2];
        }
#pragma unroll
      for (int r = 0; r < 8; ++r)
        if (r < rank) cin = cmad(rg[r], cin, rd[r]);
    }
    const E gq = shfl_up_seg(g, 1), dq = shfl_up_seg(dd, 1);
    sD[l2][k2] = k2 == 0 ? cin : cmad(gq, cin, dq);
  }
  __syncthreads();

  // ---- F2: forward from the true carry; d overwrites psi in the tile
  if constexpr (RT) {
    // the neighbours outside the sub-segment come from the values read
    // before the barrier: the adjacent sub-segments overwrite them in this
    // pass (inside it, the read of eb + i + 1 precedes the store at eb + i + 1)
    E d = sD[l][k];
    E pm = hw(rt_at(left, eb - 1));
    hpt<T> pc = rt(eb);
    const hpt<T> rend = rt_at(right, eb + nv);
    int i = 0;
    for (; i < it; ++i) {
      const hpt<T> pn = i + 1 < nv ? rt(eb + i + 1) : rend;
      d = fwd_inc(crow[pb + i], pm, pc, hw(pn), d);
      el(l, eb + i) = d;
      pm = hw(pc);
      pc = pn;
    }
#pragma unroll 2
    for (; i < nv; ++i) {
      const hpt<T> pn = i + 1 < nv ? rt(eb + i + 1) : rend;
      d = fwd_inc(cinf, pm, pc, hw(pn), d);
      el(l, eb + i) = d;
      pm = hw(pc);
      pc = pn;
    }
  } else {
    E d = sD[l][k];
    E pm = left, pcur = el(l, eb);
    int i = 0;
    for (; i < it; ++i) {
      const coef5<T> c = crow[pb + i];
      const E pn = i + 1 < nv ? el(l, eb + i + 1) : right;
      d = fwd(c, pm, pcur, pn, d);
      el(l, eb + i) = d;
      pm = pcur;
      pcur = pn;
    }
#pragma unroll 4
    for (; i < nv; ++i) {
      const E pn = i + 1 < nv ? el(l, eb + i + 1) : right;
      d = fwd(cinf, pm, pcur, pn, d);
      el(l, eb + i) = d;
      pm = pcur;
      pcur = pn;
    }
  }
  // ---- B1: local backward from a zero carry; summary (prod be, x at the start)
  {
    E x = zero<T>(), B = mk<T>(1, 0);
    int i = nv - 1;
#pragma unroll 4
    for (; i >= it; --i) x = bwd(cinf.be, x, el(l, eb + i));
    if (nv > it) B = cpow_n(cinf.be, nv - it);
    for (; i >= 0; --i) {
      const coef5<T> c = crow[pb + i];
      x = bwd(c.be, x, el(l, eb + i));
      B = cmul(c.be, B);
    }
    __syncthreads();  // every thread has read its forward carry
    sG[l][k] = B;
    sD[l][k] = x;
  }
  __syncthreads();
  // reduced system, backward: affine suffix over the sub-segments, the CTA
  // total to the cluster, and the true x after every sub-segment
  {
    E b = sG[l2][k2], xx = sD[l2][k2];
#pragma unroll
    for (int off = 1; off < kHS; off <<= 1) {
      const E bn = shfl_down_seg(b, off), xn = shfl_down_seg(xx, off);
      if (k2 + off < kHS) {
        xx = cmad(b, xn, xx);
        b = cmul(b, bn);
      }
    }
    if (k2 == 0) {
      xB[l2] = b;
      xX[l2] = xx;
    }
    csync();
    E cin = zero<T>();
    if (cs > 1) {
      E rb[8], rx[8];
#pragma unroll
      for (int r = 0; r < 8; ++r)
        if (r > rank && r < cs) {
          rb[r] = cluster.map_shared_rank(xB, r)[l2];
          rx[r] = cluster.map_shared_rank(xX, r)[l2];
        }
#pragma unroll
      for (int r = 7; r >= 0; --r)
        if (r > rank && r < cs) cin = cmad(rb[r], cin, rx[r]);
    }
    const E bq = shfl_down_seg(b, 1), xq = shfl_down_seg(xx, 1);
    sD[l2][k2] = k2 == kHS - 1 ? cin : cmad(bq, cin, xq);
  }
  // every CTA's remote reads are done before any CTA moves on (and exits)
  csync();

  // ---- B2: backward from the true carry; x overwrites d in the tile
  acc_t<T> acc;
  {
    E x = sD[l][k];
    int i = nv - 1;
#pragma unroll 4
    for (; i >= it; --i) {
      x = bwd(cinf.be, x, el(l, eb + i));
      el(l, eb + i) = x;
      if (REDUCE) acc.add(sq(x));
    }
    for (; i >= 0; --i) {
      const coef5<T> c = crow[pb + i];
      x = bwd(c.be, x, el(l, eb + i));
      el(l, eb + i) = x;
      if (REDUCE) acc.add(sq(x));
    }
  }
  __syncthreads();

  // ---- store the tile's own positions
  auto store = [&](auto ep_tag) {
    constexpr int ep = decltype(ep_tag)::value;
    if (AX == 0) {
      for (int ln = 0; ln < kHL; ++ln) {
        if (!line_ok(ln)) continue;
        E* dst = out + (grp * kHL + ln) * (long long)N;
        const E* row = tile + ln * W;
        for (int c = tid; c < pc / ep; c += kHThreads) {
          const int e = 2 + c * ep, p = p0 - 2 + e;
          if (p >= N) continue;
          if (ep == 2 && p + 1 < N) {
            *reinterpret_cast<float4*>(dst + p) = *reinterpret_cast<const float4*>(row + e);
          } else {
#pragma unroll
            for (int q = 0; q < ep; ++q)
              if (p + q < N) dst[p + q] = row[e + q];
          }
        }
      }
    } else {
      constexpr int per = kHL / ep;
      for (int u = tid; u < pc * per; u += kHThreads) {
        const int e = 2 + u / per, ln = (u % per) * ep, p = p0 - 2 + e;
        if (p >= N) continue;
        if (ep == 2 && line_ok(ln + 1)) {
          *reinterpret_cast<float4*>(out + gidx(ln, p)) =
              *reinterpret_cast<const float4*>(&el(ln, e));
        } else {
#pragma unroll
          for (int q = 0; q < ep; ++q)
            if (line_ok(ln + q)) out[gidx(ln + q, p)] = el(ln + q, e);
        }
      }
    }
  };
  if (sizeof(T) == 4 && J.vec)
    store(int_tag<2>{});
  else
    store(int_tag<1>{});
  return REDUCE ? acc.value() : 0.0;
}

}  // namespace rotgp
