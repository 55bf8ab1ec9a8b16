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
// 16 lines x 2 sub-segments.  The affine scans over a line's sub-segments run
// in a half-warp with shuffles (32 sub-segments per line in a full warp
// measured slower on GB300: 3.0e10 against 3.3e10 site-updates/s on the 4096^2
// state, 241 against 196 us per persistent batch step).  Each point is read from and written to global
// memory once per sweep; H1 (with the pending renormalisation) is applied to
// the tile as it lands in the x sweep; the last sweep of a step reduces the
// norm.  The same kernel serves both propagation modes (the table of the mode
// is passed) and both precisions.
#include "hybrid.cuh"



namespace rotgp {

template <class T, int AX, bool H1, bool IMAG, bool REDUCE>
__global__ void __launch_bounds__(kHThreads, sizeof(T) == 4 ? 2 : 1) k_line_hybrid(const hybrid_args ha) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  hybrid_job J;
  J.cs = ha.cs;
  J.pc = ha.pc;
  J.lsub = ha.lsub;
  J.vec = ha.vec;
  J.rank = (int)(blockIdx.x % (unsigned)ha.cs);
  J.grp = blockIdx.x / (unsigned)ha.cs;
  J.scale = H1 ? *ha.s.scale : 1.0;
  const double v = hybrid_tile<T, AX, H1, IMAG, REDUCE>(ha.s, J, smem_raw);
  if (REDUCE) norm_epilogue(v, ha.s);
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
