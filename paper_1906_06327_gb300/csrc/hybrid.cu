// hybrid.cu -- exact line solves of one Crank-Nicolson sweep (Sec. 2, the
// tridiagonal systems of Eqs. eqD.11/eq5) by a partition method, for lines
// that the chunked solver of sweep_x.cu / sweep_s.cu serves badly or not at
// all: long lines whose Thomas carries decay slowly (Delta/h^2 large, so the
// truncation halo H of the chunked solver grows past its chunk) and lines
// whose carries decay too slowly for any truncation.
//
// Method.  The folded Thomas recurrences of one line (coef5 in common.cuh),
//   forward   d_p = a0 psi_p + am psi_{p-1} + ap psi_{p+1} + al_p d_{p-1}
//   backward  x_p = d_p + be_p x_{p+1},
// are affine maps of their carries.  A line is cut into segments; each
// segment runs both recurrences locally from a zero carry and reports its
// affine summary, the product of its multipliers and its local end value
// (forward: G = prod al, D = d at the segment end; backward: B = prod be,
// X = x at the segment start).  The true carry into every segment follows by
// composing the summaries of the segments before it (forward) or after it
// (backward), which is the reduced system of the partition method, solved
// here by direct composition; the segments then rerun their recurrences from
// the true carries.  Nothing is truncated: the result is the Thomas solution
// of the whole line up to rounding, whatever the decay of the carries.
//
// Layout.  A CTA of 256 threads holds a tile of 16 lines x pc positions (+2
// halo positions either side) in shared memory; thread (line l, sub-segment
// k) owns lsub = pc/16 consecutive positions of line l.  A line longer than
// one tile is spread over a cluster of cs CTAs (cs = 1, 2, 4 or 8), CTA r
// holding positions [r pc, (r+1) pc); the CTAs exchange their per-line
// summaries through distributed shared memory.  x lines (contiguous rows) sit
// in the tile as [line][position] with an even pitch and an odd lsub, so the
// 32 threads of a warp (2 lines x 16 sub-segments) touch distinct banks; y
// and z lines (16 consecutive x at one transverse position, 128 contiguous
// bytes per position in complex float) sit as [position][line], a warp being
// 16 lines x 2 sub-segments.  Each point is read from and written to global
// memory once per sweep; H1 (with the pending renormalisation) is applied to
// the tile as it lands in the x sweep; the last sweep of a step reduces the
// norm.  The same kernel serves both propagation modes (the table of the mode
// is passed) and both precisions.
#include <cooperative_groups.h>

#include "sweep_common.cuh"

namespace cg = cooperative_groups;

namespace rotgp {

namespace {

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

}  // namespace

struct hybrid_args {
  stream_args s;
  int cs;     // CTAs per line group (cluster size)
  int pc;     // positions per CTA (kHS * lsub)
  int lsub;   // positions per thread
  int vec;    // 1: 16-byte global accesses of two complex floats
  long long ngroups;
};

template <class T, int AX, bool H1, bool IMAG, bool REDUCE>
__global__ void __launch_bounds__(kHThreads) k_line_hybrid(const hybrid_args ha) {
  using E = cpx<T>;
  const stream_args& a = ha.s;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  E* tile = reinterpret_cast<E*>(smem_raw);
  // per-line summaries of the sub-segments ([line][sub-segment], padded)
  __shared__ E sG[kHL][kHS + 1], sD[kHL][kHS + 1];
  // per-line totals of this CTA, read by the other CTAs of the cluster
  __shared__ E xG[kHL], xD[kHL], xB[kHL], xX[kHL];

  cg::cluster_group cluster = cg::this_cluster();
  const int cs = ha.cs, pc = ha.pc, lsub = ha.lsub;
  // a tile of whole lines (cs = 1) is launched without a cluster: no cluster
  // barrier and no remote shared memory then
  auto csync = [&]() {
    if (cs > 1)
      cluster.sync();
    else
      __syncthreads();
  };
  const int rank = (int)(blockIdx.x % (unsigned)cs);
  const long long grp = blockIdx.x / (unsigned)cs;
  const int W = pc + 4;          // tile positions incl. 2 halo points either side
  const int N = a.len, lt = a.lt;
  const int p0 = rank * pc;      // first position of this CTA
  const int tid = threadIdx.x;
  const E* in = static_cast<const E*>(a.in);
  E* out = static_cast<E*>(a.out);

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
    const bool vec = sizeof(T) == 4 && ha.vec;
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
            dst[q] = (line_ok(l) && p + q >= 0 && p + q < N) ? in[gidx(l, p + q)] : zero<T>();
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
            dst[q] = (line_ok(l + q) && p >= 0 && p < N) ? in[gidx(l + q, p)] : zero<T>();
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
    const T s = (T)(*a.scale), hg2 = (T)a.hgam2, gg = (T)a.g, dt = (T)a.dt;
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
    const bool vec = sizeof(T) == 4 && ha.vec;
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
  if (REDUCE) norm_epilogue(acc.value(), a);
}

namespace {

thread_local const char* g_hybrid_stage = "";

template <class T, int AX, bool H1, bool IMAG, bool REDUCE>
cudaError_t launch_h(const hybrid_args& ha, cudaStream_t s) {
  auto fn = k_line_hybrid<T, AX, H1, IMAG, REDUCE>;
  const size_t smem = (size_t)kHL * (ha.pc + 4) * sizeof(cpx<T>);
  g_hybrid_stage = "an earlier runtime call";
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  g_hybrid_stage = "shared-memory opt-in";
  e = allow_smem_bytes((const void*)fn, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)(ha.ngroups * ha.cs);
  if (ha.cs == 1) {
    g_hybrid_stage = "launch";
    fn<<<blocks, kHThreads, smem, s>>>(ha);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(kHThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)ha.cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  g_hybrid_stage = "cluster launch";
  return cudaLaunchKernelEx(&cfg, fn, ha);
}

template <class T, int AX>
cudaError_t launch_h_ax(bool imag, bool reduce, const hybrid_args& ha, cudaStream_t s) {
  if (AX == 0) {
    // H1 is fused into the x sweep (never the last sweep of a step)
    return imag ? launch_h<T, 0, true, true, false>(ha, s)
                : launch_h<T, 0, true, false, false>(ha, s);
  }
  return reduce ? launch_h<T, AX, false, false, true>(ha, s)
                : launch_h<T, AX, false, false, false>(ha, s);
}

}  // namespace

// Tile of a cluster of cs CTAs over lines of N points: lsub positions per
// thread (odd for x lines: bank spread), pc = 16 lsub per CTA; returns the
// tile's shared-memory bytes.
size_t hybrid_tile(int N, int axis, bool fp64, int cs, int* pc, int* lsub) {
  const int per = (N + cs - 1) / cs;
  int ls = (per + kHS - 1) / kHS;
  if (axis == 0 && ls % 2 == 0) ++ls;
  *lsub = ls;
  *pc = kHS * ls;
  return (size_t)kHL * (*pc + 4) * (fp64 ? 16 : 8);
}

// Tile shape of the hybrid solve of lines of N points: the smallest cluster
// (1, 2, 4 or 8 CTAs) whose tiles fit in max_bytes of shared memory each.
// Returns false when no cluster of at most 8 CTAs is enough.
bool hybrid_shape(int N, int axis, bool fp64, size_t max_bytes, int* cs, int* pc, int* lsub) {
  for (int c = 1; c <= 8; c *= 2) {
    if (hybrid_tile(N, axis, fp64, c, pc, lsub) <= max_bytes) {
      *cs = c;
      return true;
    }
  }
  return false;
}

size_t hybrid_smem_bytes(int pc, bool fp64) { return (size_t)kHL * (pc + 4) * (fp64 ? 16 : 8); }

long long hybrid_groups(int axis, long long nlines, int nx) {
  if (axis == 0) return (nlines + kHL - 1) / kHL;
  return (long long)((nx + kHL - 1) / kHL) * (nlines / nx);
}

// Number of clusters of this shape that fit on the device at once (0: the
// shape cannot be launched).
int hybrid_max_clusters(bool fp64, int axis, int cs, int pc) {
  const void* fn = nullptr;
  if (fp64)
    fn = axis == 0 ? (const void*)k_line_hybrid<double, 0, true, true, false>
                   : (const void*)k_line_hybrid<double, 1, false, false, true>;
  else
    fn = axis == 0 ? (const void*)k_line_hybrid<float, 0, true, true, false>
                   : (const void*)k_line_hybrid<float, 1, false, false, true>;
  const size_t smem = hybrid_smem_bytes(pc, fp64);
  cudaError_t e = allow_smem_bytes(fn, (int)smem);
  if (e != cudaSuccess) {
    g_hybrid_stage = cudaGetErrorString(e);
    cudaGetLastError();
    return 0;
  }
  if (cs == 1) {
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kHThreads, smem);
    if (e != cudaSuccess) {
      g_hybrid_stage = cudaGetErrorString(e);
      cudaGetLastError();
      return 0;
    }
    if (nb < 1) g_hybrid_stage = "no resident block";
    return nb;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(cs * 64));
  cfg.blockDim = dim3(kHThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  e = cudaOccupancyMaxActiveClusters(&n, fn, &cfg);
  if (e != cudaSuccess) {
    g_hybrid_stage = cudaGetErrorString(e);
    cudaGetLastError();
    return 0;
  }
  if (n < 1) g_hybrid_stage = "no resident cluster";
  return n;
}

const char* hybrid_launch_stage() { return g_hybrid_stage; }

cudaError_t launch_line_hybrid(bool fp64, bool imag, bool reduce, int axis, const stream_args& a,
                               int cs, int pc, int lsub, cudaStream_t s) {
  hybrid_args ha{};
  ha.s = a;
  ha.cs = cs;
  ha.pc = pc;
  ha.lsub = lsub;
  // 16-byte accesses: complex float with even rows (x) or even x extent (y, z)
  ha.vec = !fp64 && a.nx % 2 == 0;
  ha.ngroups = hybrid_groups(axis, a.nlines, a.nx);
  if (fp64) {
    if (axis == 0) return launch_h_ax<double, 0>(imag, reduce, ha, s);
    if (axis == 1) return launch_h_ax<double, 1>(imag, reduce, ha, s);
    return launch_h_ax<double, 2>(imag, reduce, ha, s);
  }
  if (axis == 0) return launch_h_ax<float, 0>(imag, reduce, ha, s);
  if (axis == 1) return launch_h_ax<float, 1>(imag, reduce, ha, s);
  return launch_h_ax<float, 2>(imag, reduce, ha, s);
}

}  // namespace rotgp
