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
constexpr int kHS = 16;                 // sub-segments per line in one CTA
constexpr int kHThreads = kHL * kHS;    // 256

template <class T>
__device__ __forceinline__ cpx<T> cmad(cpx<T> a, cpx<T> b, cpx<T> c) {
  return mk<T>(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

// z^n for n >= 0 by repeated squaring
template <class T>
__device__ __forceinline__ cpx<T> cpow_n(cpx<T> z, int n) {
  cpx<T> r = mk<T>(1, 0);
  while (n > 0) {
    if (n & 1) r = r * z;
    z = z * z;
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

template <class T, int AX, bool H1, bool IMAG, bool REDUCE>
__device__ __forceinline__ double hybrid_tile(const stream_args& a, const hybrid_job& J,
                                              unsigned char* smem_raw) {
  using E = cpx<T>;
  E* tile = reinterpret_cast<E*>(smem_raw);
  // per-line summaries of the sub-segments ([line][sub-segment], padded)
  __shared__ E sG[kHL][kHS + 1], sD[kHL][kHS + 1];
  // per-line totals of this CTA, read by the other CTAs of the cluster
  __shared__ E xG[kHL], xD[kHL], xB[kHL], xX[kHL];

  cg::cluster_group cluster = cg::this_cluster();
  const int cs = J.cs, pc = J.pc, lsub = J.lsub;
  // a tile of whole lines (cs = 1) is launched without a cluster: no cluster
  // barrier and no remote shared memory then
  auto csync = [&]() {
    if (cs > 1)
      cluster.sync();
    else
      __syncthreads();
  };
  const int rank = J.rank;
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

  // ---- load the tile (zeros outside the grid and past the line end)
  {
    constexpr int EPv = sizeof(T) == 4 ? 2 : 1;
    const bool vec = sizeof(T) == 4 && J.vec;
    const int ep = vec ? EPv : 1;
    if (AX == 0) {
      const int per = W / ep;  // copies per line (W even)
      for (int u = tid; u < kHL * per; u += kHThreads) {
        const int l = u / per, e = (u % per) * ep, p = p0 - 2 + e;
        E* dst = &el(l, e);
        if (line_ok(l) && p >= 0 && p + ep <= N) {
          if (vec)
            cp_async<16>(dst, in + gidx(l, p));
          else
            cp_async<sizeof(E)>(dst, in + gidx(l, p));
        } else {
          for (int q = 0; q < ep; ++q)
            dst[q] = (line_ok(l) && p + q >= 0 && p + q < N) ? ldcg_c(in + gidx(l, p + q)) : zero<T>();
        }
      }
    } else {
      const int per = kHL / ep;  // copies per tile position
      for (int u = tid; u < W * per; u += kHThreads) {
        const int e = u / per, l = (u % per) * ep, p = p0 - 2 + e;
        E* dst = &el(l, e);
        if (p >= 0 && p < N && line_ok(l + ep - 1)) {
          if (vec)
            cp_async<16>(dst, in + gidx(l, p));
          else
            cp_async<sizeof(E)>(dst, in + gidx(l, p));
        } else {
          for (int q = 0; q < ep; ++q)
            dst[q] = (line_ok(l + q) && p >= 0 && p < N) ? ldcg_c(in + gidx(l + q, p)) : zero<T>();
        }
      }
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
  }

  // ---- H1 with the pending renormalisation (x sweep): psi <- s psi, then
  // exp(-Delta (V + g|psi|^2)) or exp(-i Delta (V + g|psi|^2)) (Eq. eq1)
  if (H1) {
    const T s = (T)J.scale, hg2 = (T)a.hgam2, gg = (T)a.g, dt = (T)a.dt;
    for (int u = tid; u < kHL * W; u += kHThreads) {
      const int l = u / W, e = u % W, p = p0 - 2 + e;
      const long long r = grp * kHL + l;
      const int j = (int)(r % a.ny), k = (int)(r / a.ny);
      const T x = (T)(a.x0 + (double)p * a.hx);
      const T y = (T)(a.y0 + (double)j * a.hy), z = (T)(a.z0 + (double)k * a.hz);
      E v = s * el(l, e);
      const T en = hg2 * x * x + ((T)a.hnu2 * y * y + (T)a.hlam2 * z * z) + gg * abs2(v);
      if (IMAG) {
        v = exp_t(-dt * en) * v;
      } else {
        T sn, cn;
        sincos_t(dt * en, &sn, &cn);
        v = v * mk<T>(cn, -sn);
      }
      el(l, e) = v;
    }
    __syncthreads();
  }

  // ---- this thread's line and sub-segment
  const int l = AX == 0 ? tid / kHS : tid % kHL;
  const int k = AX == 0 ? tid % kHS : tid / kHL;
  const int pb = p0 + k * lsub;                      // first position
  const int nv = max(0, min(lsub, N - pb));          // positions inside the line
  const int eb = 2 + k * lsub;                       // its tile position
  int li = 0;                                        // coefficient line
  if (AX == 0) li = line_ok(l) ? (int)((grp * kHL + l) % a.ny) : 0;
  if (AX == 1) li = line_ok(l) ? x0l + l : 0;
  const coef5<T>* crow = static_cast<const coef5<T>*>(a.coef) + (size_t)li * (lt + 1);
  const coef5<T> cinf = crow[lt];
  auto coef = [&](int p) -> coef5<T> { return p >= lt ? cinf : crow[p]; };

  // ---- F1: local forward from a zero carry; summary (prod al, d at the end)
  const E left = el(l, eb - 1), right = el(l, eb + nv);
  {
    E d = zero<T>(), G = mk<T>(1, 0);
    int nin = 0;
    E pm = left, pcur = el(l, eb);
    for (int i = 0; i < nv; ++i) {
      const int p = pb + i;
      const E pn = i + 1 < nv ? el(l, eb + i + 1) : right;
      const coef5<T> c = coef(p);
      d = cmad(c.al, d, cmad(c.ap, pn, cmad(c.am, pm, c.a0 * pcur)));
      if (p < lt)
        G = c.al * G;
      else
        ++nin;
      pm = pcur;
      pcur = pn;
    }
    if (nin) G = G * cpow_n(cinf.al, nin);
    sG[l][k] = G;
    sD[l][k] = d;
  }
  __syncthreads();
  // reduced system, forward: the true d before every sub-segment
  if (tid < kHL) {
    const int ln = tid;
    E Gc = mk<T>(1, 0), Dc = zero<T>();
    for (int q = 0; q < kHS; ++q) {
      Dc = cmad(sG[ln][q], Dc, sD[ln][q]);
      Gc = sG[ln][q] * Gc;
    }
    xG[ln] = Gc;
    xD[ln] = Dc;
  }
  csync();
  if (tid < kHL) {
    const int ln = tid;
    E carry = zero<T>();
    for (int r = 0; r < rank; ++r) {
      const E* rg = cluster.map_shared_rank(xG, r);
      const E* rd = cluster.map_shared_rank(xD, r);
      carry = cmad(rg[ln], carry, rd[ln]);
    }
    for (int q = 0; q < kHS; ++q) {
      const E dq = sD[ln][q];
      sD[ln][q] = carry;
      carry = cmad(sG[ln][q], carry, dq);
    }
  }
  __syncthreads();

  // ---- F2: forward from the true carry; d overwrites psi in the tile
  {
    E d = sD[l][k];
    E pm = left, pcur = el(l, eb);
    for (int i = 0; i < nv; ++i) {
      const int p = pb + i;
      const E pn = i + 1 < nv ? el(l, eb + i + 1) : right;
      const coef5<T> c = coef(p);
      d = cmad(c.al, d, cmad(c.ap, pn, cmad(c.am, pm, c.a0 * pcur)));
      el(l, eb + i) = d;
      pm = pcur;
      pcur = pn;
    }
  }
  // ---- B1: local backward from a zero carry; summary (prod be, x at the start)
  {
    E x = zero<T>(), B = mk<T>(1, 0);
    int nin = 0;
    for (int i = nv - 1; i >= 0; --i) {
      const int p = pb + i;
      const coef5<T> c = coef(p);
      x = cmad(c.be, x, el(l, eb + i));
      if (p < lt)
        B = c.be * B;
      else
        ++nin;
    }
    if (nin) B = B * cpow_n(cinf.be, nin);
    __syncthreads();  // every thread has read its sD carry before sG/sD are reused
    sG[l][k] = B;
    sD[l][k] = x;
  }
  __syncthreads();
  // reduced system, backward: the true x after every sub-segment
  if (tid < kHL) {
    const int ln = tid;
    E Bc = mk<T>(1, 0), Xc = zero<T>();
    for (int q = kHS - 1; q >= 0; --q) {
      Xc = cmad(sG[ln][q], Xc, sD[ln][q]);
      Bc = sG[ln][q] * Bc;
    }
    xB[ln] = Bc;
    xX[ln] = Xc;
  }
  csync();
  if (tid < kHL) {
    const int ln = tid;
    E carry = zero<T>();
    for (int r = cs - 1; r > rank; --r) {
      const E* rb = cluster.map_shared_rank(xB, r);
      const E* rx = cluster.map_shared_rank(xX, r);
      carry = cmad(rb[ln], carry, rx[ln]);
    }
    for (int q = kHS - 1; q >= 0; --q) {
      const E xq = sD[ln][q];
      sD[ln][q] = carry;
      carry = cmad(sG[ln][q], carry, xq);
    }
  }
  // every CTA's remote reads are done before any CTA moves on (and exits)
  csync();

  // ---- B2: backward from the true carry; x overwrites d in the tile
  acc_t<T> acc;
  {
    E x = sD[l][k];
    for (int i = nv - 1; i >= 0; --i) {
      const int p = pb + i;
      const coef5<T> c = coef(p);
      x = cmad(c.be, x, el(l, eb + i));
      el(l, eb + i) = x;
      if (REDUCE) acc.add(abs2(x));
    }
  }
  __syncthreads();

  // ---- store the tile's own positions
  {
    const bool vec = sizeof(T) == 4 && J.vec;
    const int ep = vec ? 2 : 1;
    if (AX == 0) {
      const int per = pc / ep;
      for (int u = tid; u < kHL * per; u += kHThreads) {
        const int ln = u / per, e = 2 + (u % per) * ep, p = p0 - 2 + e;
        if (!line_ok(ln) || p >= N) continue;
        if (vec && p + 1 < N) {
          *reinterpret_cast<float4*>(out + gidx(ln, p)) = *reinterpret_cast<const float4*>(&el(ln, e));
        } else {
          for (int q = 0; q < ep && p + q < N; ++q) out[gidx(ln, p + q)] = el(ln, e + q);
        }
      }
    } else {
      const int per = kHL / ep;
      for (int u = tid; u < pc * per; u += kHThreads) {
        const int e = 2 + u / per, ln = (u % per) * ep, p = p0 - 2 + e;
        if (p >= N) continue;
        if (vec && line_ok(ln + 1)) {
          *reinterpret_cast<float4*>(out + gidx(ln, p)) = *reinterpret_cast<const float4*>(&el(ln, e));
        } else {
          for (int q = 0; q < ep; ++q)
            if (line_ok(ln + q)) out[gidx(ln + q, p)] = el(ln + q, e);
        }
      }
    }
  }
  return REDUCE ? acc.value() : 0.0;
}

}  // namespace rotgp
