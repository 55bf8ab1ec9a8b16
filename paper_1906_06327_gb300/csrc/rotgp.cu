// rotgp.cu -- host side of the C ABI declared in include/rotgp.h: context
// lifetime, solver sizing, launch plans of one split step (Sec. 2: H1 fused
// into the x sweep, then the y sweep and, in 3D, the z sweep, with the norm
// reduced in the last sweep), observables, state I/O and kernel timing.
#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "../../include/rotgp.h"
#include "common.cuh"
#include "tma.cuh"

using namespace rotgp;

namespace {

thread_local std::string g_create_error;

constexpr int kMaxHalo = 64;
constexpr int kMaxTable = 512;

enum KernelId {
  K_SWEEP_X, K_SWEEP_Y, K_SWEEP_Z, K_OBS, K_VMOM, K_VCOUNT, K_NORM, K_INIT, K_IO, K_TABLES,
  K_XY, K_COUNT
};
const char* kKernelNames[K_COUNT] = {"sweep_x_h1",  "sweep_y",        "sweep_z",
                                     "observables", "vortex_moments", "vortex_count",
                                     "norm",        "init_analytic",  "pack_unpack",
                                     "tables",      "xy_pass_h1"};

struct AxisPlan {
  int nlines = 0;       // lines with distinct coefficients (table rows)
  axis_coef co[2];      // [mode] 0 = real, 1 = imaginary
  void* table[2] = {nullptr, nullptr};
  void* tableT[2] = {nullptr, nullptr};  // complex float: [m2, al, be][lt + 1][nlines]
  // launch plan of this axis' sweep
  long long lines = 0;  // lines solved per sweep
  int len = 0;          // points per line
  int nseg = 1, seg_chunks = 1, warm = 1;
  sweep_shape sh{};
  // real-time launch plan when sh is a one-line-per-lane TMA (unfolded)
  // shape: that form rounds 2 A^-1 psi before subtracting psi, which doubles
  // the effect of the rounded weights and drifts the real-time norm; real
  // time keeps the folded two-lines-per-lane form
  struct {
    bool set = false;
    int nseg = 1, seg_chunks = 1, warm = 1;
    sweep_shape sh{};
  } rt;
  // banded-inverse stencil (complex float): taps K, end rows B, weights [mode]
  bool stencil_ok = false;  // stencil form available for this axis
  bool use_stencil = false;
  int sK = 0, sB = 0;
  int lsegs = 1;  // segments per line of the stencil line pass (y, z)
  void* wtab[2] = {nullptr, nullptr};
  // exact partition-method solve (hybrid.cu): clusters of hcs CTAs, each a
  // tile of 16 lines x hpc positions, hlsub positions per thread
  bool hyb_ok = false;
  bool use_hybrid = false;
  std::string hyb_why;  // why no tile shape was found
  int hcs = 1, hpc = 0, hlsub = 0;
};

struct ProfRec {
  int kid;
  cudaEvent_t a, b;
};

}  // namespace

struct rotgp_ctx {
  rotgp_grid grid{};
  rotgp_phys phys{};
  int prec = ROTGP_FP32;
  bool fp64 = false;
  cudaStream_t stream = nullptr;
  int nx = 0, ny = 0, nz = 1;  // stored points
  long long sites = 0;
  size_t elem = 8;
  double x0 = 0, y0 = 0, z0 = 0, vol = 1;
  // solver sizing
  int halo = 2, lt = 8;
  double decay = 0;
  bool chunk_ok = true;  // carries decay fast enough for the chunked solver
  // device memory
  void* psi[2] = {nullptr, nullptr};
  int cur = 0;
  void* staging = nullptr;
  size_t staging_bytes = 0;
  double* dR = nullptr;
  AxisPlan axis[3];
  // tile passes (complex float): H1 + x + y in one pass over each plane
  // (fuse_xy), and the y/z stencil sweeps; TMA maps per state buffer
  bool maps_ok = false;
  bool fuse_ok = false, fuse_xy = false;
  bool x_tma = true;  // Thomas x sweep loads its chunks with TMA (when the maps exist)
  long long plan_version = 0;  // bumped whenever launches or tables change
  CUtensorMap map_xy[2], map_y[2], map_z[2];
  bool xpass_ok = false;  // x sweep alone in stencil form through TMA tiles
  CUtensorMap map_xp[2];
  // rows maps of the Thomas x sweep's TMA chunk loads: [buffer][C = 8, 16]
  bool xmaps_ok = false;
  CUtensorMap map_x[2][2];
  // ... and of its one-row-per-lane form: boxes of 32 rows, [buffer][C = 8, 16]
  CUtensorMap map_x1[2][2];
  // one-line-per-lane y/z Thomas sweeps: boxes of 32 lines x (C + 1) positions,
  // [buffer][axis - 1][C = 8, 16]
  bool smaps_ok = false;
  CUtensorMap map_s1[2][2][2];
  double* partials = nullptr;
  size_t partial_doubles = 0;
  unsigned* counter = nullptr;
  double* scalars = nullptr;  // [0] scale, [1] norm, [2..2+NOBS) obs, [+2] moments
  int* iflags = nullptr;      // [0] flags, [1] vortex count
  double* h_obs = nullptr;    // pinned: NOBS doubles + 2 ints
  size_t device_bytes = 0;
  long long steps = 0;
  std::string err;
  // profiling
  bool prof = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  double bytes_per_launch[K_COUNT] = {0};
  int sm_count = 148;
  int smem_optin = 232448;

  double* d_scale() { return scalars; }
  double* d_norm() { return scalars + 1; }
  double* d_obs() { return scalars + 2; }
  double* d_moments() { return scalars + 2 + NOBS; }
  int* d_flags() { return iflags; }
  int* d_count() { return iflags + 1; }
};

namespace {

int fail(rotgp_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c)
    c->err = buf;
  else
    g_create_error = buf;
  return code;
}

int cuda_fail(rotgp_ctx* c, cudaError_t e, const char* what) {
  return fail(c, ROTGP_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

using cd = std::complex<double>;

// Coefficients of Eqs. eqD.11/eq5 for one axis and mode (see axis_coef):
// kappa = (i Delta | Delta)/(4 h^2); tau_unit multiplies the line's
// coordinate: x lines (u = y_j): real -Delta Omega/(4h), imaginary
// +i Delta Omega/(4h); y lines (u = x_i): the negatives (Omega y -> -Omega x);
// z lines: 0.
axis_coef make_coef(int axis, int imag, double h, double dt, double omega, double u0, double du) {
  axis_coef co{};
  const cd idt = imag ? cd(dt, 0) : cd(0, dt);
  const cd kap = idt / (4.0 * h * h);
  cd tau_unit(0, 0);
  const cd dplain = idt / cd(0, 1);  // Delta in real time, -i Delta in imaginary time
  if (axis == 0) tau_unit = -dplain * omega / (4.0 * h);
  if (axis == 1) tau_unit = dplain * omega / (4.0 * h);
  co.kap_re = kap.real();
  co.kap_im = kap.imag();
  co.tau_re = tau_unit.real();
  co.tau_im = tau_unit.imag();
  co.u0 = u0;
  co.du = du;
  return co;
}

// Worst-case carry decay and multiplier-table length over the lines of an
// axis: iterate c'_p = A+ / (A0 - A- c'_{p-1}) to its fixed point c* (to
// within 1e-15 relative, the rounding level of the iteration itself), then
// forward decay |A- m*|, backward decay |c*|.  *converged turns false when a
// line does not get there within kMaxTable points.
void size_axis(const axis_coef& co, int nlines, double* decay, int* lt, bool* converged) {
  for (int l = 0; l < nlines; ++l) {
    const double u = co.u0 + l * co.du;
    const cd kap(co.kap_re, co.kap_im), tau = cd(co.tau_re, co.tau_im) * u;
    const cd a0 = 1.0 + 2.0 * kap, am = -kap + tau, ap = -kap - tau;
    cd c(0, 0), m(0, 0);
    int p = 1;
    for (; p <= kMaxTable; ++p) {
      m = 1.0 / (a0 - am * c);
      const cd cn = ap * m;
      const bool conv = std::abs(cn - c) <= 1e-15 * std::abs(cn);
      c = cn;
      if (conv) break;
    }
    if (p > kMaxTable) *converged = false;
    *lt = std::max(*lt, std::min(p + 1, kMaxTable));
    *decay = std::max(*decay, std::max(std::abs(am * m), std::abs(c)));
  }
}

double nlines_u0(const rotgp_ctx* c, int axis) {
  return axis == 0 ? c->y0 : (axis == 1 ? c->x0 : 0.0);
}
double nlines_du(const rotgp_ctx* c, int axis) {
  return axis == 0 ? c->grid.h[1] : (axis == 1 ? c->grid.h[0] : 0.0);
}

// Size the line solver for the current physics (both modes).  A halo above
// kMaxHalo leaves only the exact partition solve (hybrid.cu), which needs the
// table of every line to reach its fixed point (the Toeplitz interior).
int plan_solver(rotgp_ctx* c, int* halo, int* lt, double* decay, bool* chunk_ok) {
  double dec = 0;
  int tl = 2;
  bool conv = true;
  for (int a = 0; a < c->grid.dim; ++a) {
    const int nl = a == 0 ? c->ny : (a == 1 ? c->nx : 1);
    for (int mode = 0; mode < 2; ++mode) {
      axis_coef co = make_coef(a, mode, c->grid.h[a], c->phys.dt, c->phys.omega,
                               nlines_u0(c, a), nlines_du(c, a));
      size_axis(co, nl, &dec, &tl, &conv);
    }
  }
  if (!(dec < 1.0) || !std::isfinite(dec))
    return fail(c, ROTGP_EUNSUPPORTED, "line carry does not decay (factor %g)", dec);
  const double tol = c->fp64 ? 1e-17 : 1e-9;
  int H = dec <= 0 ? 1 : (int)std::ceil(std::log(tol) / std::log(dec)) + 1;
  H = std::max(H, 2);
  *chunk_ok = H <= kMaxHalo;
  if (!*chunk_ok) {
    if (!conv)
      return fail(c, ROTGP_EUNSUPPORTED,
                  "line coefficients do not reach their fixed point within %d points "
                  "(carry decay factor %.4f): Delta/h^2 too large",
                  kMaxTable, dec);
    H = kMaxHalo;
  }
  *halo = H;
  *lt = tl;
  *decay = dec;
  return ROTGP_OK;
}

// Rows of W = 2 A^{-1} - I for a short line of m unknowns with the
// coefficients of line u of an axis (double, Thomas solves column by
// column): W[p][j] for p, j = 1..m, stored row-major in w (size (m+1)^2).
void short_line_w(const axis_coef& co, double u, int m, std::vector<cd>& w) {
  const cd kap(co.kap_re, co.kap_im), tau = cd(co.tau_re, co.tau_im) * u;
  const cd a0 = 1.0 + 2.0 * kap, am = -kap + tau, ap = -kap - tau;
  std::vector<cd> c(m + 2), mm(m + 2), d(m + 2);
  c[0] = 0.0;
  for (int i = 1; i <= m; ++i) {
    mm[i] = 1.0 / (a0 - am * c[i - 1]);
    c[i] = ap * mm[i];
  }
  w.assign((size_t)(m + 1) * (m + 1), 0.0);
  for (int j = 1; j <= m; ++j) {
    d[0] = 0.0;
    for (int i = 1; i <= m; ++i) d[i] = ((i == j ? 1.0 : 0.0) - am * d[i - 1]) * mm[i];
    for (int i = m - 1; i >= 1; --i) d[i] = d[i] - c[i] * d[i + 1];
    for (int i = 1; i <= m; ++i) w[(size_t)i * (m + 1) + j] = 2.0 * d[i] - (i == j ? 1.0 : 0.0);
  }
}

// Stencil size of one axis (both modes, worst line): the smallest K in
// {4, 6, 8} whose dropped taps are below 2e-10 of the largest weight, and
// the number B of rows at each line end that differ from the interior row
// by more than 1e-10 of it.  Returns false when no built K is enough.
bool plan_stencil(rotgp_ctx* c, int a, int* K_out, int* B_out) {
  const int N = a == 0 ? c->nx : (a == 1 ? c->ny : c->nz);
  const int nl = a == 0 ? c->ny : (a == 1 ? c->nx : 1);
  const int m = 84;  // short line: interior row at 42, far from both ends
  int K = 0, B = 0;
  std::vector<cd> w;
  for (int mode = 0; mode < 2; ++mode) {
    const axis_coef co = make_coef(a, mode, c->grid.h[a], c->phys.dt, c->phys.omega,
                                   nlines_u0(c, a), nlines_du(c, a));
    for (int l : {0, nl - 1, nl / 2}) {
      short_line_w(co, co.u0 + l * co.du, m, w);
      auto W = [&](int i, int j) { return w[(size_t)i * (m + 1) + j]; };
      const int mid = m / 2;
      const double w0 = std::abs(W(mid, mid));
      int k = 0;
      for (int kk : {4, 6, 8}) {
        if (std::abs(W(mid, mid - kk - 1)) <= 2e-10 * w0 && std::abs(W(mid, mid + kk + 1)) <= 2e-10 * w0) {
          k = kk;
          break;
        }
      }
      if (!k) return false;
      K = std::max(K, k);
      // first row from each end that equals the interior row within 1e-10
      for (int e = 1; e < mid - 8; ++e) {
        double dl = 0, dr = 0;
        for (int t = -8; t <= 8; ++t) {
          const cd ref = W(mid, mid + t);
          if (e + t >= 1) dl = std::max(dl, std::abs(W(e, e + t) - ref));
          if (m + 1 - e + t <= m && m + 1 - e + t >= 1)
            dr = std::max(dr, std::abs(W(m + 1 - e, m + 1 - e + t) - ref));
        }
        if (dl <= 1e-10 * w0 && dr <= 1e-10 * w0) {
          B = std::max(B, e);
          break;
        }
        if (e == mid - 9) return false;
      }
    }
  }
  B = std::max(B, K + 1);
  if (N < 2 * B + 2) return false;
  *K_out = K;
  *B_out = B;
  return true;
}

// Set the launch shape of axis a: V lines per lane, chunk C, R ring slots,
// wpb warps per block, nseg segments per line; recompute blocks and shared
// memory.  Only shapes with an instantiated kernel are accepted.
int set_shape(rotgp_ctx* c, int a, int V, int C, int R, int wpb, long long nseg) {
  AxisPlan& ap = c->axis[a];
  const bool x = a == 0;
  const size_t limit = (size_t)c->smem_optin - 1024;
  // the x sweep also has a one-row-per-lane TMA form for complex float rows
  // of 16-byte multiples, chunk 8 or 16
  const bool x1t = !c->fp64 && V == 1 && (C == 8 || C == 16) && c->nx % 2 == 0;
  if (!sweep_shape_built(c->fp64, V, C) && !x1t)
    return fail(c, ROTGP_EINVAL, "no sweep kernel for %d lines per lane and chunk %d", V, C);
  if (V == 2 && !x && c->nx % 2 != 0)
    return fail(c, ROTGP_EINVAL, "two lines per lane in y/z sweeps need an even N_x");
  if (C < c->halo) return fail(c, ROTGP_EINVAL, "chunk %d shorter than the halo %d", C, c->halo);
  // the one-line-per-lane TMA forms with chunk 8 also take 5 or 6 slots
  const bool deep = !c->fp64 && V == 1 && C == 8 && c->nx % 2 == 0 &&
                    (x ? c->xmaps_ok && c->x_tma : c->smaps_ok);
  if (R != 3 && R != 4 && !(deep && (R == 5 || R == 6)))
    return fail(c, ROTGP_EINVAL, "ring must have 3 or 4 slots (5 or 6 in the TMA forms, chunk 8)");
  const size_t per_warp = sweep_smem_per_warp(c->fp64, x, V, C, R);
  if (per_warp * wpb > limit) return fail(c, ROTGP_EINVAL, "launch shape exceeds shared memory");
  const int nch = (ap.len + C - 1) / C;
  nseg = std::max<long long>(1, std::min<long long>(nseg, nch));
  ap.seg_chunks = (int)((nch + nseg - 1) / nseg);
  ap.nseg = (nch + ap.seg_chunks - 1) / ap.seg_chunks;
  ap.warm = (c->halo + 1 + C - 1) / C;
  ap.sh.V = V;
  ap.sh.C = C;
  ap.sh.R = R;
  ap.sh.vec16 = c->fp64 || (x && c->nx % 2 == 0);
  ap.sh.warps_per_block = wpb;
  ap.sh.smem = per_warp * wpb;
  const long long groups = (ap.lines + 32 * V - 1) / (32 * V);
  ap.sh.blocks = (groups * ap.nseg + wpb - 1) / wpb;
  return ROTGP_OK;
}

// Default shape of the one-line-per-lane TMA sweeps (complex float, once
// their tensor maps exist): chunks of 8, a 5-slot ring, and segments so that
// the 32-line units come to about 14 per SM (one wave of persistent warps).
void lean_defaults(rotgp_ctx* c) {
  if (c->fp64 || c->halo > 8) return;
  for (int a = 0; a < c->grid.dim; ++a) {
    AxisPlan& ap = c->axis[a];
    if (!(a == 0 ? c->xmaps_ok && c->x_tma : c->smaps_ok)) continue;
    const AxisPlan keep = ap;
    const long long groups = (ap.lines + 31) / 32, nch = (ap.len + 7) / 8;
    const long long nseg = std::max<long long>(
        1, std::min<long long>(nch, (14LL * c->sm_count + groups / 2) / groups));
    if (set_shape(c, a, 1, 8, 5, 1, nseg) != ROTGP_OK) ap = keep;
  }
}

// Default launch plan of every sweep: complex float solves two lines per
// lane in chunks of 8 (16 if the halo is longer), double one line in chunks
// of 16 (64); a 3-slot ring; one warp per block, so that blocks of ~15 KB
// pack each SM densely; and enough segments per line for about one wave of
// resident warps.  Where the TMA maps exist, complex float takes the
// one-line-per-lane forms instead (lean_defaults).
int plan_axes(rotgp_ctx* c) {
  const size_t sm_bytes = 228 * 1024;
  for (int a = 0; a < c->grid.dim; ++a) {
    AxisPlan& ap = c->axis[a];
    const bool x = a == 0;
    ap.len = a == 0 ? c->nx : (a == 1 ? c->ny : c->nz);
    ap.lines = a == 0 ? (long long)c->ny * c->nz
                      : (a == 1 ? (long long)c->nx * c->nz : (long long)c->nx * c->ny);
    // exact partition solve: tiles of at most ~100 KB (two or three CTAs per
    // SM), else up to ~200 KB, in clusters of at most 8 CTAs
    ap.hyb_ok = false;
    ap.hyb_why = "line too long for a cluster of 8 tiles";
    for (size_t budget : {(size_t)100 * 1024, (size_t)200 * 1024}) {
      int cs = 0, pc = 0, ls = 0;
      if (budget > (size_t)c->smem_optin - 16 * 1024) break;
      if (!hybrid_shape(ap.len, a, c->fp64, budget, &cs, &pc, &ls)) continue;
      if (hybrid_max_clusters(c->fp64, a, cs, pc) < 1) {
        char buf[160];
        snprintf(buf, sizeof buf, "%d CTAs of tile %d: %s", cs, pc, hybrid_launch_stage());
        ap.hyb_why = buf;
        continue;
      }
      ap.hyb_ok = true;
      ap.hcs = cs;
      ap.hpc = pc;
      ap.hlsub = ls;
      break;
    }
    if (!c->chunk_ok) {
      // carries too slow for any truncation: the exact solve on every axis
      if (!ap.hyb_ok)
        return fail(c, ROTGP_EUNSUPPORTED,
                    "carry decay %.4f needs the exact line solve, which has no tile shape "
                    "for %d points per line",
                    c->decay, ap.len);
      ap.use_hybrid = true;
      ap.use_stencil = false;
      ap.stencil_ok = false;
      continue;
    }
    int V = 1, C = c->halo <= 16 ? 16 : 64;
    if (!c->fp64 && c->halo <= 16 && (x || c->nx % 2 == 0)) {
      V = 2;
      C = c->halo <= 8 ? 8 : 16;
    }
    const int R = 3;
    const size_t per_warp = sweep_smem_per_warp(c->fp64, x, V, C, R);
    const long long resident =
        std::max<long long>(1, std::min<long long>(32, (long long)(sm_bytes / (per_warp + 1024))));
    const long long target = resident * c->sm_count;
    const long long groups = (ap.lines + 32 * V - 1) / (32 * V);
    int rc = set_shape(c, a, V, C, R, 1, std::max<long long>(1, target / groups));
    if (rc) return rc == ROTGP_EINVAL ? fail(c, ROTGP_EUNSUPPORTED, "%s", c->err.c_str()) : rc;
    // this folded plan also serves real-time steps whenever a one-line-per-
    // lane TMA (unfolded) shape is chosen for the axis later
    ap.rt.set = true;
    ap.rt.nseg = ap.nseg;
    ap.rt.seg_chunks = ap.seg_chunks;
    ap.rt.warm = ap.warm;
    ap.rt.sh = ap.sh;
    // banded-inverse stencil: complex float, even N_x (TMA rows of 16-byte
    // multiples; the separate x-stencil kernel also wants N_x % 4 == 0)
    int K = 0, B = 0;
    const bool sized = ap.wtab[0] != nullptr;  // tables already allocated
    ap.stencil_ok = !c->fp64 && c->nx % 2 == 0 && plan_stencil(c, a, &K, &B);
    if (sized) {
      // keep the allocated size; a larger K or B than needed is only more exact
      ap.stencil_ok = ap.stencil_ok && K <= ap.sK && B <= ap.sB;
      ap.use_stencil = ap.use_stencil && ap.stencil_ok;
      continue;
    }
    if (ap.stencil_ok) {
      ap.sK = K;
      ap.sB = B;
      if (!x) {
        // line pass: enough segments for ~24 resident warps per SM, each
        // segment at least 16 points
        const long long nt = a == 1 ? c->nz : c->ny;
        const long long warps = ((c->nx + 31) / 32) * ((nt + 1) / 2) * 2;
        const long long want = (24LL * c->sm_count + warps - 1) / warps;
        ap.lsegs = (int)std::max(1LL, std::min(want, (long long)std::min(8, ap.len / 16)));
      }
    }
    // default: the Thomas form (the stencil and fused forms are selected by
    // rotgp_set_solver or rotgp_autotune), except that complex-float lines
    // too long-range for the chunk-8/16 forms take the exact partition solve
    ap.use_stencil = false;
    ap.use_hybrid = !c->fp64 && c->halo > 16 && ap.hyb_ok;
  }
  // one pass for H1, x and y: both axes in stencil form with one reach K
  // (the larger of the two; a longer stencil is only more exact)
  AxisPlan &ax = c->axis[0], &ay = c->axis[1];
  if (!c->chunk_ok) {
    c->fuse_ok = c->fuse_xy = false;
    return ROTGP_OK;
  }
  if (!ax.wtab[0] && ax.stencil_ok && ay.stencil_ok) {
    const int K = std::max(ax.sK, ay.sK);
    ax.sK = ay.sK = K;
    c->fuse_ok = tile_k_built(K);
    c->fuse_xy = false;
  }
  c->fuse_ok = c->fuse_ok && ax.stencil_ok && ay.stencil_ok;
  lean_defaults(c);
  c->fuse_xy = c->fuse_xy && c->fuse_ok;
  return ROTGP_OK;
}

// Launch shape of the xy pass: one CTA per (tile, range of z planes), the
// ranges as long as one wave of resident CTAs allows (2D: one CTA per tile).
void xy_shape(const rotgp_ctx* c, int* tiles_x, int* tiles_y, int* zchunk, unsigned* blocks) {
  int TX, TY, R, WX;
  const int K = c->axis[0].sK;
  xy_tile_geometry(K, &TX, &TY, &R, &WX);
  *tiles_x = (c->nx + TX - 1) / TX;
  *tiles_y = (c->ny + TY - 1) / TY;
  const long long txy = (long long)*tiles_x * *tiles_y;
  // occupancy of the most demanding instantiation (real time, with norm)
  const long long resident =
      (long long)xy_pass_ctas_per_sm(K, false, c->grid.dim == 2) * c->sm_count;
  const int chunks = (int)std::max<long long>(1, std::min<long long>(c->nz, resident / txy));
  *zchunk = (c->nz + chunks - 1) / chunks;
  *blocks = (unsigned)(txy * ((c->nz + *zchunk - 1) / *zchunk));
}
// Launch shape of the x pass: as the xy pass, tiles of 32 rows x 64 points.
void x_shape(const rotgp_ctx* c, int* tiles_x, int* tiles_y, int* zchunk, unsigned* blocks) {
  *tiles_x = (c->nx + 63) / 64;
  *tiles_y = (c->ny + 31) / 32;
  const long long txy = (long long)*tiles_x * *tiles_y;
  const long long resident = (long long)x_pass_ctas_per_sm(c->axis[0].sK) * c->sm_count;
  const int chunks = (int)std::max<long long>(1, std::min<long long>(c->nz, resident / txy));
  *zchunk = (c->nz + chunks - 1) / chunks;
  *blocks = (unsigned)(txy * ((c->nz + *zchunk - 1) / *zchunk));
}

unsigned xy_blocks(const rotgp_ctx* c) {
  int tx, ty, zc;
  unsigned b;
  xy_shape(c, &tx, &ty, &zc, &b);
  return b;
}
// line pass: patches of 32 x line_rows() lines times segments per line
int line_seg_len(const rotgp_ctx* c, int axis) {
  const AxisPlan& ap = c->axis[axis];
  return (ap.len + ap.lsegs - 1) / ap.lsegs;
}
unsigned line_blocks(const rotgp_ctx* c, int axis) {
  const int nt = axis == 1 ? c->nz : c->ny, rows = line_rows();
  const int L = line_seg_len(c, axis);
  return (unsigned)(((c->nx + 31) / 32) * ((nt + rows - 1) / rows) *
                    ((c->axis[axis].len + L - 1) / L));
}
constexpr int kMaxLineSegs = 8;

// Driver entry point of the tensor-map encoder, looked up once.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// TMA maps of both state buffers for the tile passes; without them the
// stencil form of y and z and the fused x-y pass are switched off.
void build_maps(rotgp_ctx* c) {
  c->maps_ok = false;
  bool ok = !c->fp64 && c->nx % 2 == 0;
  for (int b = 0; b < 2 && ok; ++b) {
    if (c->fuse_ok) {
      int TX, TY, R, WX;
      xy_tile_geometry(c->axis[0].sK, &TX, &TY, &R, &WX);
      ok = ok && encode_state_map(&c->map_xy[b], c->psi[b], c->nx, c->ny, c->nz, 2 * WX, R, 1) == 0;
    }
    const unsigned rows = (unsigned)line_rows();
    ok = ok && encode_state_map(&c->map_y[b], c->psi[b], c->nx, c->ny, c->nz, 64, 8, rows) == 0;
    ok = ok && encode_state_map(&c->map_z[b], c->psi[b], c->nx, c->ny, c->nz, 64, rows, 8) == 0;
  }
  // the y and z Thomas sweeps, one line per lane
  c->smaps_ok = !c->fp64 && c->nx % 2 == 0;
  for (int b = 0; b < 2 && c->smaps_ok; ++b)
    for (int ax = 1; ax < c->grid.dim && c->smaps_ok; ++ax)
      for (int ci = 0; ci < 2 && c->smaps_ok; ++ci) {
        const unsigned pts = ci == 0 ? 8 : 16;
        c->smaps_ok = encode_state_map(&c->map_s1[b][ax - 1][ci], c->psi[b], c->nx, c->ny,
                                       c->nz, 64, ax == 1 ? pts : 1, ax == 1 ? 1 : pts) == 0;
      }
  // the x sweep alone in stencil form: boxes of 32 rows x (64 + 2K + 2) points
  c->xpass_ok = !c->fp64 && c->nx % 2 == 0 && c->axis[0].stencil_ok && tile_k_built(c->axis[0].sK);
  for (int b = 0; b < 2 && c->xpass_ok; ++b)
    c->xpass_ok = encode_state_map(&c->map_xp[b], c->psi[b], c->nx, c->ny, c->nz,
                                   2 * (64 + 2 * c->axis[0].sK + 2), 32, 1) == 0;
  // the Thomas x sweep: boxes of 64 rows x (C + 2) points (two rows per
  // lane) and swizzled boxes of 32 rows x C points (one row per lane)
  c->xmaps_ok = !c->fp64 && c->nx % 2 == 0;
  for (int b = 0; b < 2 && c->xmaps_ok; ++b)
    for (int ci = 0; ci < 2 && c->xmaps_ok; ++ci) {
      const int C = ci == 0 ? 8 : 16;
      c->xmaps_ok = encode_rows_map(&c->map_x[b][ci], c->psi[b], c->nx,
                                    (long long)c->ny * c->nz, 2 * (C + 2), 64) == 0 &&
                    encode_rows_map(&c->map_x1[b][ci], c->psi[b], c->nx,
                                    (long long)c->ny * c->nz, 2 * C, 32, 8 * C) == 0;
    }
  c->maps_ok = ok;
  if (!ok) {
    c->fuse_ok = c->fuse_xy = false;
    for (int a = 1; a < c->grid.dim; ++a) c->axis[a].stencil_ok = c->axis[a].use_stencil = false;
  }
  for (int a = 1; a < c->grid.dim; ++a)
    if (!tile_k_built(c->axis[a].sK)) c->axis[a].stencil_ok = c->axis[a].use_stencil = false;
}

int reduce_blocks(const rotgp_ctx* c, long long n) {
  long long b = (n + 255) / 256;
  const long long cap = (long long)c->sm_count * 8;
  return (int)std::max(1LL, std::min(b, cap));
}

// --------------------------------------------------------------- profiling
cudaEvent_t take_event(rotgp_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

struct Timed {
  rotgp_ctx* c;
  int kid;
  cudaEvent_t a = nullptr;
  Timed(rotgp_ctx* cc, int k) : c(cc), kid(k) {
    if (c->prof) {
      a = take_event(c);
      cudaEventRecord(a, c->stream);
    }
  }
  ~Timed() {
    if (c->prof) {
      cudaEvent_t b = take_event(c);
      cudaEventRecord(b, c->stream);
      c->recs.push_back({kid, a, b});
    }
  }
};

int build_tables(rotgp_ctx* c) {
  for (int a = 0; a < c->grid.dim; ++a) {
    AxisPlan& ap = c->axis[a];
    for (int mode = 0; mode < 2; ++mode) {
      ap.co[mode] = make_coef(a, mode, c->grid.h[a], c->phys.dt, c->phys.omega,
                              nlines_u0(c, a), nlines_du(c, a));
      Timed t(c, K_TABLES);
      cudaError_t e = launch_tables(c->fp64, ap.table[mode], ap.tableT[mode], ap.nlines, c->lt,
                                    ap.co[mode], c->stream);
      if (e == cudaSuccess && ap.stencil_ok && ap.wtab[mode])
        e = launch_stencil_tables(ap.wtab[mode], ap.nlines, ap.sK, ap.sB,
                                  2 * ap.sB + 2 * ap.sK + 8, ap.co[mode], c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "table kernel");
    }
  }
  return ROTGP_OK;
}

// --------------------------------------------------------------- one step
tile_args make_tile_args(rotgp_ctx* c, bool imag) {
  tile_args t{};
  const int mode = imag ? 1 : 0;
  t.out = c->psi[1 - c->cur];
  t.wx = c->axis[0].wtab[mode];
  t.wy = c->axis[1].wtab[mode];
  t.wz = c->grid.dim == 3 ? c->axis[2].wtab[mode] : nullptr;
  t.nx = c->nx;
  t.ny = c->ny;
  t.nz = c->nz;
  t.bx = c->axis[0].sB;
  t.by = c->axis[1].sB;
  t.bz = c->grid.dim == 3 ? c->axis[2].sB : 0;
  t.dt = (float)c->phys.dt;
  t.g = (float)c->phys.g;
  t.hgam2 = (float)(0.5 * c->phys.gamma * c->phys.gamma);
  t.hnu2 = (float)(0.5 * c->phys.nu * c->phys.nu);
  t.hlam2 = c->grid.dim == 3 ? (float)(0.5 * c->phys.lambda * c->phys.lambda) : 0.f;
  t.x0 = (float)c->x0;
  t.hx = (float)c->grid.h[0];
  t.y0 = (float)c->y0;
  t.hy = (float)c->grid.h[1];
  t.z0 = (float)c->z0;
  t.hz = c->grid.dim == 3 ? (float)c->grid.h[2] : 0.f;
  t.scale = c->d_scale();
  t.vol = c->vol;
  t.imag = imag ? 1 : 0;
  t.partials = c->partials;
  t.counter = c->counter;
  t.scale_out = c->d_scale();
  t.norm_out = c->d_norm();
  t.flags = c->d_flags();
  return t;
}

// H1, x and y sweeps in one pass (the whole step in 2D)
int xy_pass(rotgp_ctx* c, bool imag) {
  tile_args t = make_tile_args(c, imag);
  unsigned blocks;
  xy_shape(c, &t.tiles_x, &t.tiles_y, &t.zchunk, &blocks);
  cudaError_t e;
  {
    Timed tm(c, K_XY);
    e = launch_xy_pass(imag, c->grid.dim == 2, c->axis[0].sK, &c->map_xy[c->cur], t, blocks,
                       c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "xy pass launch");
  c->cur = 1 - c->cur;
  return ROTGP_OK;
}

int sweep(rotgp_ctx* c, int axis, bool imag, bool last) {
  const int mode = imag ? 1 : 0;
  AxisPlan ap = c->axis[axis];
  if (!imag && !c->fp64 && ap.sh.V == 1 && (ap.sh.C == 8 || ap.sh.C == 16) && ap.rt.set &&
      (axis == 0 ? c->xmaps_ok && c->x_tma : c->smaps_ok)) {
    ap.nseg = ap.rt.nseg;
    ap.seg_chunks = ap.rt.seg_chunks;
    ap.warm = ap.rt.warm;
    ap.sh = ap.rt.sh;
  }
  stream_args a{};
  a.in = c->psi[c->cur];
  a.out = c->psi[1 - c->cur];
  a.coef = ap.table[mode];
  a.coefT = static_cast<const float2*>(ap.tableT[mode]);
  a.tlines = ap.nlines;
  a.len = ap.len;
  a.lt = c->lt;
  a.nseg = ap.nseg;
  a.seg_chunks = ap.seg_chunks;
  a.warm = ap.warm;
  a.halo = c->halo;
  a.ring = ap.sh.R;
  a.nlines = ap.lines;
  a.nx = c->nx;
  a.ny = c->ny;
  a.vol = c->vol;
  a.imag = imag ? 1 : 0;
  a.partials = c->partials;
  a.counter = c->counter;
  a.scale_out = c->d_scale();
  a.norm_out = c->d_norm();
  a.flags = c->d_flags();
  a.wtab = ap.wtab[mode];
  a.taps_k = ap.sK;
  a.brows = ap.sB;
  cudaError_t e;
  if (ap.use_hybrid) {
    // exact partition solve, every precision and mode (H1 fused into x)
    a.coef_mode = axis == 0 ? 2 : (axis == 1 ? 1 : 0);
    a.stride = axis == 1 ? (long long)c->nx : (long long)c->nx * c->ny;
    a.outer = axis == 1 ? (long long)c->nx * c->ny : (long long)c->nx;
    a.dt = c->phys.dt;
    a.g = c->phys.g;
    a.hgam2 = 0.5 * c->phys.gamma * c->phys.gamma;
    a.hnu2 = 0.5 * c->phys.nu * c->phys.nu;
    a.hlam2 = c->grid.dim == 3 ? 0.5 * c->phys.lambda * c->phys.lambda : 0.0;
    a.x0 = c->x0;
    a.hx = c->grid.h[0];
    a.y0 = c->y0;
    a.hy = c->grid.h[1];
    a.z0 = c->z0;
    a.hz = c->grid.dim == 3 ? c->grid.h[2] : 0.0;
    a.scale = c->d_scale();
    Timed t(c, axis == 0 ? K_SWEEP_X : (axis == 1 ? K_SWEEP_Y : K_SWEEP_Z));
    e = launch_line_hybrid(c->fp64, imag, last, axis, a, ap.hcs, ap.hpc, ap.hlsub, c->stream);
    if (e != cudaSuccess)
      return fail(c, ROTGP_ECUDA, "hybrid sweep of axis %d (%s, %d CTAs per line, tile %d): %s",
                  axis, hybrid_launch_stage(), ap.hcs, ap.hpc, cudaGetErrorString(e));
    c->cur = 1 - c->cur;
    return ROTGP_OK;
  }
  if (axis == 0) {
    a.coef_mode = 2;
    a.dt = c->phys.dt;
    a.g = c->phys.g;
    a.hgam2 = 0.5 * c->phys.gamma * c->phys.gamma;
    a.hnu2 = 0.5 * c->phys.nu * c->phys.nu;
    a.hlam2 = c->grid.dim == 3 ? 0.5 * c->phys.lambda * c->phys.lambda : 0.0;
    a.x0 = c->x0;
    a.hx = c->grid.h[0];
    a.y0 = c->y0;
    a.hy = c->grid.h[1];
    a.z0 = c->z0;
    a.hz = c->grid.dim == 3 ? c->grid.h[2] : 0.0;
    a.scale = c->d_scale();
    Timed t(c, K_SWEEP_X);
    if (ap.use_stencil && imag && c->xpass_ok) {
      tile_args ta = make_tile_args(c, imag);
      unsigned blocks;
      x_shape(c, &ta.tiles_x, &ta.tiles_y, &ta.zchunk, &blocks);
      e = launch_x_pass(imag, ap.sK, &c->map_xp[c->cur], ta, blocks, c->stream);
    } else if (ap.use_stencil && imag && c->nx % 4 == 0) {
      const long long warps = ((ap.lines + 1) / 2) * ((ap.len + 127) / 128);
      e = launch_stencil_x(imag, a, warps, c->stream);
    } else {
      const void *xm = nullptr, *om = nullptr;
      if (c->xmaps_ok && c->x_tma && ap.sh.vec16 && (ap.sh.C == 8 || ap.sh.C == 16)) {
        const int ci = ap.sh.C == 8 ? 0 : 1;
        xm = ap.sh.V == 2 ? &c->map_x[c->cur][ci] : &c->map_x1[c->cur][ci];
        om = ap.sh.V == 2 ? nullptr : &c->map_x1[1 - c->cur][ci];
      }
      e = launch_sweep_x(c->fp64, imag, a, ap.sh, xm, om, c->stream);
    }
  } else {
    a.stride = axis == 1 ? (long long)c->nx : (long long)c->nx * c->ny;
    a.outer = axis == 1 ? (long long)c->nx * c->ny : (long long)c->nx;
    a.coef_mode = axis == 1 ? 1 : 0;
    Timed t(c, axis == 1 ? K_SWEEP_Y : K_SWEEP_Z);
    if (ap.use_stencil && imag) {
      tile_args ta = make_tile_args(c, imag);
      ta.tiles_x = (c->nx + 31) / 32;
      ta.tiles_y = ((axis == 1 ? c->nz : c->ny) + line_rows() - 1) / line_rows();
      ta.seg_len = line_seg_len(c, axis);
      e = launch_line_pass(axis, last, ap.sK, axis == 1 ? &c->map_y[c->cur] : &c->map_z[c->cur],
                           ta, line_blocks(c, axis), c->stream);
    } else {
      const void *sm = nullptr, *om = nullptr;
      if (c->smaps_ok && ap.sh.V == 1 && (ap.sh.C == 8 || ap.sh.C == 16)) {
        sm = &c->map_s1[c->cur][axis - 1][ap.sh.C == 8 ? 0 : 1];
        om = &c->map_s1[1 - c->cur][axis - 1][ap.sh.C == 8 ? 0 : 1];
      }
      e = launch_sweep_strided(c->fp64, last, a, ap.sh, sm, om, axis, c->stream);
    }
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "sweep launch");
  c->cur = 1 - c->cur;
  return ROTGP_OK;
}

int run_steps(rotgp_ctx* c, long long n, bool imag) {
  if (!c) return ROTGP_EINVAL;
  if (n < 0) return fail(c, ROTGP_EINVAL, "negative step count");
  for (long long s = 0; s < n; ++s) {
    for (int a = 0; a < c->grid.dim; ++a) {
      int rc;
      // the stencil and fused forms serve imaginary time; real-time steps
      // keep the folded Thomas form, whose near-unit diagonal factor is
      // stored as its difference from 1 so that the rounded CN map stays
      // unitary to ~1e-10 per sweep (the stencil's rounded central weight,
      // close to 1 itself, would not)
      if (a == 0 && c->fuse_xy && imag) {
        rc = xy_pass(c, imag);
        ++a;  // the y sweep is part of the pass
      } else {
        rc = sweep(c, a, imag, a == c->grid.dim - 1);
      }
      if (rc) return rc;
    }
    ++c->steps;
  }
  return ROTGP_OK;
}

int check_flags(rotgp_ctx* c) {
  int flags = 0;
  cudaError_t e = cudaMemcpyAsync(&flags, c->d_flags(), sizeof(int), cudaMemcpyDeviceToHost,
                                  c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "synchronise");
  if (flags & 2) return fail(c, ROTGP_ECUDA, "a sweep kernel was launched with a shape it was not built for");
  if (flags & 4) return fail(c, ROTGP_ETIMEOUT, "a tile pass gave up waiting for its TMA load");
  if (flags & 1) return fail(c, ROTGP_ENONFINITE, "non-finite or zero norm in a reduction");
  return ROTGP_OK;
}

bool finite_phys(const rotgp_phys* p) {
  const double v[6] = {p->gamma, p->nu, p->lambda, p->g, p->omega, p->dt};
  for (double x : v)
    if (!std::isfinite(x)) return false;
  return p->dt > 0;
}

void release(rotgp_ctx* c) {
  for (void*& p : c->psi) cudaFree(p), p = nullptr;
  cudaFree(c->staging);
  cudaFree(c->dR);
  for (auto& ap : c->axis) {
    for (void*& t : ap.table) cudaFree(t), t = nullptr;
    for (void*& t : ap.wtab) cudaFree(t), t = nullptr;
  }
  cudaFree(c->partials);
  cudaFree(c->counter);
  cudaFree(c->scalars);
  cudaFree(c->iflags);
  if (c->h_obs) cudaFreeHost(c->h_obs);
  for (auto& r : c->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : c->pool) cudaEventDestroy(e);
}

int dev_alloc(rotgp_ctx* c, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(c, ROTGP_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  }
  c->device_bytes += bytes;
  return ROTGP_OK;
}

}  // namespace

namespace rotgp {
int encode_rows_map(CUtensorMap* map, void* base, int nx, long long nrows, unsigned box0,
                    unsigned box1, int swizzle_bytes) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
  if (!fn) return -1;
  const cuuint64_t dims[2] = {2ull * (cuuint64_t)nx, (cuuint64_t)nrows};
  const cuuint64_t strides[1] = {8ull * (cuuint64_t)nx};
  const cuuint32_t box[2] = {box0, box1};
  const cuuint32_t estr[2] = {1, 1};
  const CUtensorMapSwizzle sw = swizzle_bytes == 128  ? CU_TENSOR_MAP_SWIZZLE_128B
                                : swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                      : CU_TENSOR_MAP_SWIZZLE_NONE;
  if (swizzle_bytes != 0 && box0 * 4u != (unsigned)swizzle_bytes) return -1;
  return (int)fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

int encode_state_map(CUtensorMap* map, void* base, int nx, int ny, int nz, unsigned box0,
                     unsigned box1, unsigned box2) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
  if (!fn) return -1;
  const cuuint64_t dims[3] = {2ull * (cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {8ull * (cuuint64_t)nx, 8ull * (cuuint64_t)nx * (cuuint64_t)ny};
  const cuuint32_t box[3] = {box0, box1, box2};
  const cuuint32_t estr[3] = {1, 1, 1};
  return (int)fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

int ctx_buffer(const rotgp_ctx* c) { return c->cur; }
void ctx_set_buffer(rotgp_ctx* c, int cur) { c->cur = cur; }
long long ctx_steps(const rotgp_ctx* c) { return c->steps; }
long long ctx_plan_version(const rotgp_ctx* c) { return c->plan_version; }
void ctx_add_steps(rotgp_ctx* c, long long n) { c->steps += n; }
void ctx_get_view(const rotgp_ctx* c, ctx_view* v) {
  v->dim = c->grid.dim;
  v->fp64 = c->fp64 ? 1 : 0;
  v->nx = c->nx;
  v->ny = c->ny;
  v->lt = c->lt;
  v->cur = c->cur;
  v->psi[0] = c->psi[0];
  v->psi[1] = c->psi[1];
  for (int a = 0; a < 2; ++a)
    for (int m = 0; m < 2; ++m) v->table[a][m] = c->axis[a].table[m];
  v->scale = c->scalars;
  v->norm = c->scalars + 1;
  v->flags = c->iflags;
  v->dt = c->phys.dt;
  v->g = c->phys.g;
  v->gamma = c->phys.gamma;
  v->nu = c->phys.nu;
  v->x0 = c->x0;
  v->y0 = c->y0;
  v->hx = c->grid.h[0];
  v->hy = c->grid.h[1];
  v->vol = c->vol;
}

// Message returned by rotgp_last_error(NULL) on this thread.
void set_thread_error(const char* msg) { g_create_error = msg ? msg : ""; }
}  // namespace rotgp

namespace {

// Eq. fun into the current buffer (phase_mode as k_init_analytic), then the
// norm and the pending scale 1/sqrt(norm).
int init_state(rotgp_ctx* c, int function, int phase_mode, const double* phase_R,
               unsigned long long seed, double d_xy, double d_z) {
  if (function != 0 && function != 1) return fail(c, ROTGP_EINVAL, "function must be 0 or 1");
  if (!(d_xy > 0) || (c->grid.dim == 3 && !(d_z > 0)))
    return fail(c, ROTGP_EINVAL, "widths must be positive");
  cudaError_t e = cudaSuccess;
  if (phase_mode == 1) {
    e = cudaMemcpyAsync(c->dR, phase_R, (size_t)(c->nx + 1) * (c->ny + 1) * 8,
                        cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "copy phase field");
  }
  {
    Timed t(c, K_INIT);
    e = launch_init_analytic(c->fp64, c->psi[c->cur], c->nx, c->ny, c->nz, c->grid.dim, c->x0,
                             c->grid.h[0], c->y0, c->grid.h[1], c->z0,
                             c->grid.dim == 3 ? c->grid.h[2] : 0.0, function, phase_mode,
                             phase_mode == 1 ? c->dR : nullptr, seed, d_xy, d_z, c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
  if ((e = cudaMemsetAsync(c->iflags, 0, sizeof(int), c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "reset flags");
  {
    Timed t(c, K_NORM);
    e = launch_norm(c->fp64, c->psi[c->cur], c->sites, c->vol, 1, c->partials, c->counter,
                    c->d_scale(), c->d_norm(), c->d_flags(), reduce_blocks(c, c->sites), 256,
                    c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "norm kernel");
  c->steps = 0;
  return check_flags(c);  // also releases phase_R
}

}  // namespace

// =============================================================== C ABI
extern "C" {

const char* rotgp_last_error(const rotgp_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

int rotgp_create(const rotgp_grid* grid, const rotgp_phys* phys, int precision, void* stream,
                 rotgp_ctx** out) {
  g_create_error.clear();
  if (!grid || !phys || !out) return fail(nullptr, ROTGP_EINVAL, "null argument");
  *out = nullptr;
  if (grid->dim != 2 && grid->dim != 3) return fail(nullptr, ROTGP_EINVAL, "dim must be 2 or 3");
  for (int a = 0; a < grid->dim; ++a) {
    if (grid->n[a] < 4) return fail(nullptr, ROTGP_EINVAL, "n[%d] = %d < 4", a, grid->n[a]);
    if (!(grid->h[a] > 0) || !std::isfinite(grid->h[a]))
      return fail(nullptr, ROTGP_EINVAL, "h[%d] must be positive", a);
  }
  if (precision != ROTGP_FP32 && precision != ROTGP_FP64)
    return fail(nullptr, ROTGP_EINVAL, "precision must be ROTGP_FP32 or ROTGP_FP64");
  if (!finite_phys(phys)) return fail(nullptr, ROTGP_EINVAL, "physics must be finite, dt > 0");
  const long long pts = (long long)grid->n[0] * grid->n[1] * (grid->dim == 3 ? grid->n[2] : 1);
  if (pts > (1LL << 34)) return fail(nullptr, ROTGP_EINVAL, "grid too large");

  rotgp_ctx* c = new (std::nothrow) rotgp_ctx();
  if (!c) return fail(nullptr, ROTGP_ENOMEM, "host allocation failed");
  c->grid = *grid;
  c->phys = *phys;
  c->prec = precision;
  c->fp64 = precision == ROTGP_FP64;
  c->elem = c->fp64 ? 16 : 8;
  c->stream = static_cast<cudaStream_t>(stream);
  c->nx = grid->n[0];
  c->ny = grid->n[1];
  c->nz = grid->dim == 3 ? grid->n[2] : 1;
  c->sites = pts;
  c->x0 = -0.5 * grid->n[0] * grid->h[0];
  c->y0 = -0.5 * grid->n[1] * grid->h[1];
  c->z0 = grid->dim == 3 ? -0.5 * grid->n[2] * grid->h[2] : 0.0;
  c->vol = grid->h[0] * grid->h[1] * (grid->dim == 3 ? grid->h[2] : 1.0);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) {
    int rc = fail(nullptr, ROTGP_ECUDA, "no usable CUDA device: %s", cudaGetErrorString(e));
    delete c;
    return rc;
  }
  // the decay factor is needed by plan_axes' messages
  int rc = plan_solver(c, &c->halo, &c->lt, &c->decay, &c->chunk_ok);
  if (!rc) rc = plan_axes(c);
  if (rc) {
    g_create_error = c->err;
    delete c;
    return rc;
  }
  c->axis[0].nlines = c->ny;
  c->axis[1].nlines = c->nx;
  c->axis[2].nlines = 1;
  // reduction scratch: the largest per-block partial count of any reduction
  size_t pd = (size_t)reduce_blocks(c, c->sites) * NQ;
  {
    // largest block count any launch shape of the last sweep can take:
    // one warp per block, one line per lane, one segment per chunk
    const AxisPlan& last = c->axis[grid->dim - 1];
    const long long nch = (last.len + 7) / 8;
    pd = std::max(pd, (size_t)(((last.lines + 31) / 32) * nch));
    // the one-line-per-lane form groups lines by 32 consecutive x
    pd = std::max(pd, (size_t)strided1_blocks(last.lines, c->nx, (int)nch));
  }
  pd = std::max(pd, (size_t)reduce_blocks(c, (long long)c->nx * c->ny) * 3);
  {
    // the exact partition solve of the last axis: one block per tile
    const int la = grid->dim - 1;
    const AxisPlan& last = c->axis[la];
    if (last.hyb_ok)
      pd = std::max(pd, (size_t)(hybrid_groups(la, last.lines, c->nx) * 8));
  }
  c->partial_doubles = pd;
  c->staging_bytes = (size_t)(grid->n[0] + 1) * (grid->n[1] + 1) *
                     (grid->dim == 3 ? grid->n[2] + 1 : 1) * 16;
  // (also the autotuner's copy of the state and its pending scale)
  c->staging_bytes = std::max(c->staging_bytes, (size_t)pts * (c->fp64 ? 16 : 8) + 64);
  const size_t state = (size_t)c->sites * c->elem;
  const size_t tab_elem = c->fp64 ? sizeof(coef5<double>) : sizeof(coef5<float>);
  rc = dev_alloc(c, &c->psi[0], state);
  if (!rc) rc = dev_alloc(c, &c->psi[1], state);
  if (!rc) rc = dev_alloc(c, &c->staging, c->staging_bytes);
  if (!rc) rc = dev_alloc(c, (void**)&c->dR, (size_t)(grid->n[0] + 1) * (grid->n[1] + 1) * 8);
  for (int a = 0; a < grid->dim && !rc; ++a)
    for (int m = 0; m < 2 && !rc; ++m)
      rc = dev_alloc(c, &c->axis[a].table[m], (size_t)c->axis[a].nlines * (c->lt + 1) * tab_elem);
  for (int a = 0; a < grid->dim && !rc && !c->fp64; ++a)
    for (int m = 0; m < 2 && !rc; ++m)
      rc = dev_alloc(c, &c->axis[a].tableT[m],
                     (size_t)3 * c->axis[a].nlines * (c->lt + 1) * sizeof(float2));
  for (int a = 0; a < grid->dim && !rc; ++a) {
    AxisPlan& ap = c->axis[a];
    if (!ap.stencil_ok) continue;
    const size_t bytes = (size_t)ap.nlines * (2 * ap.sB + 1) * (2 * ap.sK + 1) * sizeof(cpx<float>);
    for (int m = 0; m < 2 && !rc; ++m) rc = dev_alloc(c, &ap.wtab[m], bytes);
  }
  if (!rc) {
    // the tile passes reduce the norm in their own blocks
    if (c->fuse_ok && grid->dim == 2)
      c->partial_doubles = std::max(c->partial_doubles, (size_t)xy_blocks(c));
    const int la = grid->dim - 1;
    if (c->axis[la].stencil_ok && tile_k_built(c->axis[la].sK)) {
      const int keep = c->axis[la].lsegs;
      c->axis[la].lsegs = kMaxLineSegs;
      c->partial_doubles = std::max(c->partial_doubles, (size_t)line_blocks(c, la));
      c->axis[la].lsegs = keep;
    }
  }
  if (!rc) rc = dev_alloc(c, (void**)&c->partials, c->partial_doubles * sizeof(double));
  if (!rc) rc = dev_alloc(c, (void**)&c->counter, sizeof(unsigned));
  if (!rc) rc = dev_alloc(c, (void**)&c->scalars, (2 + NOBS + 2) * sizeof(double));
  if (!rc) rc = dev_alloc(c, (void**)&c->iflags, 2 * sizeof(int));
  if (!rc && cudaMallocHost((void**)&c->h_obs, (NOBS + 2) * sizeof(double)) != cudaSuccess)
    rc = fail(c, ROTGP_ENOMEM, "pinned host allocation failed");
  if (!rc) {
    e = cudaMemsetAsync(c->psi[0], 0, state, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->psi[1], 0, state, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->counter, 0, sizeof(unsigned), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->iflags, 0, 2 * sizeof(int), c->stream);
    if (e == cudaSuccess) e = launch_set_scalar(c->d_scale(), 1.0, c->stream);
    if (e != cudaSuccess) rc = cuda_fail(c, e, "initialise buffers");
  }
  if (!rc) build_maps(c);
  if (!rc) lean_defaults(c);
  if (!rc) rc = build_tables(c);
  if (!rc) {
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) rc = cuda_fail(c, e, "create");
  }
  if (rc) {
    g_create_error = c->err;
    release(c);
    delete c;
    return rc;
  }
  // algorithmic bytes per launch: one read + one write of the state per sweep
  c->bytes_per_launch[K_SWEEP_X] = 2.0 * state;
  c->bytes_per_launch[K_SWEEP_Y] = 2.0 * state;
  c->bytes_per_launch[K_SWEEP_Z] = 2.0 * state;
  c->bytes_per_launch[K_XY] = 2.0 * state;
  c->bytes_per_launch[K_OBS] = 1.0 * state;
  *out = c;
  return ROTGP_OK;
}

void rotgp_destroy(rotgp_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  release(ctx);
  delete ctx;
}

int rotgp_set_phys(rotgp_ctx* c, const rotgp_phys* phys) {
  if (!c || !phys) return ROTGP_EINVAL;
  ++c->plan_version;
  if (!finite_phys(phys)) return fail(c, ROTGP_EINVAL, "physics must be finite, dt > 0");
  const rotgp_phys old = c->phys;
  c->phys = *phys;
  int halo = 0, lt = 0;
  double dec = 0;
  bool chunk_ok = true;
  const bool old_chunk_ok = c->chunk_ok;
  int rc = plan_solver(c, &halo, &lt, &dec, &chunk_ok);
  if (!rc && chunk_ok != old_chunk_ok) {
    // switch between the chunked and the exact-only plans
    c->chunk_ok = chunk_ok;
    const int old_h = c->halo;
    c->halo = std::max(halo, c->halo);
    rc = lt > c->lt ? fail(c, ROTGP_EUNSUPPORTED,
                           "new physics needs %d table entries (context has %d)", lt, c->lt)
                    : plan_axes(c);
    if (rc) {
      c->chunk_ok = old_chunk_ok;
      c->halo = old_h;
      c->phys = old;
      plan_axes(c);
      return rc;
    }
    c->decay = std::max(c->decay, dec);
    return build_tables(c);
  }
  if (!rc && lt > c->lt) {
    // tables were sized at create; a longer table needs more memory
    rc = fail(c, ROTGP_EUNSUPPORTED, "new physics needs %d table entries (context has %d)", lt,
              c->lt);
  }
  if (!rc && halo > c->halo) {
    const int old_h = c->halo;
    c->halo = halo;
    rc = plan_axes(c);
    if (!rc && (size_t)c->axis[c->grid.dim - 1].sh.blocks > c->partial_doubles)
      rc = fail(c, ROTGP_EUNSUPPORTED, "new physics needs a larger reduction buffer");
    if (rc) {
      c->halo = old_h;
      plan_axes(c);
    }
  }
  if (rc) {
    c->phys = old;
    return rc;
  }
  if (halo <= c->halo) {
    // re-check the stencil sizes against the new physics (plan_axes keeps
    // the allocated K and B and falls back to the Thomas form if they are
    // no longer enough)
    const int keep_h = c->halo;
    rc = plan_axes(c);
    c->halo = keep_h;
    if (rc) {
      c->phys = old;
      return rc;
    }
  }
  c->decay = std::max(c->decay, dec);
  return build_tables(c);
}

int rotgp_set_omega(rotgp_ctx* c, double omega) {
  if (!c) return ROTGP_EINVAL;
  rotgp_phys p = c->phys;
  p.omega = omega;
  return rotgp_set_phys(c, &p);
}

int rotgp_init_analytic(rotgp_ctx* c, int function, int random_phase, unsigned long long seed,
                        double d_xy, double d_z) {
  if (!c) return ROTGP_EINVAL;
  return init_state(c, function, random_phase ? 2 : 0, nullptr, seed, d_xy, d_z);
}

int rotgp_init_analytic_field(rotgp_ctx* c, int function, const double* phase_R, double d_xy,
                              double d_z) {
  if (!c) return ROTGP_EINVAL;
  return init_state(c, function, phase_R ? 1 : 0, phase_R, 0ull, d_xy, d_z);
}

int rotgp_set_psi(rotgp_ctx* c, const void* src, int src_on_device, int src_is_fp64,
                  int normalise) {
  if (!c || !src) return c ? fail(c, ROTGP_EINVAL, "null source") : ROTGP_EINVAL;
  const size_t pts = c->staging_bytes / 16;
  const size_t bytes = pts * (src_is_fp64 ? 16 : 8);
  const void* from = src;
  cudaError_t e = cudaSuccess;
  if (!src_on_device) {
    e = cudaMemcpyAsync(c->staging, src, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "copy state to device");
    from = c->staging;
  }
  {
    Timed t(c, K_IO);
    e = launch_pack(c->fp64, src_is_fp64 != 0, from, c->psi[c->cur], c->nx, c->ny, c->nz,
                    c->grid.dim, c->d_scale(), c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "pack kernel");
  if ((e = cudaMemsetAsync(c->iflags, 0, sizeof(int), c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "reset flags");
  if (normalise) {
    // the norm and the pending scale 1/sqrt(norm), as after an imaginary-time step
    Timed t(c, K_NORM);
    e = launch_norm(c->fp64, c->psi[c->cur], c->sites, c->vol, 1, c->partials, c->counter,
                    c->d_scale(), c->d_norm(), c->d_flags(), reduce_blocks(c, c->sites), 256,
                    c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "norm kernel");
  }
  c->steps = 0;
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "set_psi");
  return normalise ? check_flags(c) : ROTGP_OK;
}

int rotgp_get_psi(rotgp_ctx* c, void* dst, int dst_on_device, int dst_is_fp64) {
  if (!c || !dst) return c ? fail(c, ROTGP_EINVAL, "null destination") : ROTGP_EINVAL;
  const size_t pts = c->staging_bytes / 16;
  const size_t bytes = pts * (dst_is_fp64 ? 16 : 8);
  void* to = dst_on_device ? dst : c->staging;
  cudaError_t e;
  {
    Timed t(c, K_IO);
    e = launch_unpack(c->fp64, dst_is_fp64 != 0, c->psi[c->cur], to, c->nx, c->ny, c->nz,
                      c->grid.dim, c->d_scale(), c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "unpack kernel");
  if (!dst_on_device) {
    e = cudaMemcpyAsync(dst, c->staging, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "copy state to host");
  }
  return check_flags(c);
}

int rotgp_column_density(rotgp_ctx* c, double* dst, int dst_on_device) {
  if (!c || !dst) return c ? fail(c, ROTGP_EINVAL, "null destination") : ROTGP_EINVAL;
  const size_t n = (size_t)(c->nx + 1) * (c->ny + 1);
  double* to = dst_on_device ? dst : reinterpret_cast<double*>(c->staging);
  cudaError_t e;
  {
    Timed t(c, K_IO);
    e = launch_column_density(c->fp64, c->psi[c->cur], to, c->nx, c->ny, c->nz,
                              c->grid.dim == 3 ? c->grid.h[2] : 1.0, c->d_scale(), c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "column density kernel");
  if (!dst_on_device) {
    e = cudaMemcpyAsync(dst, c->staging, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "copy column density");
  }
  return check_flags(c);
}

int rotgp_step_imag(rotgp_ctx* c, long long n) { return run_steps(c, n, true); }
int rotgp_step_real(rotgp_ctx* c, long long n) { return run_steps(c, n, false); }

int rotgp_step_schedule(rotgp_ctx* c, long long n, int imag, const double* omega) {
  if (!c) return ROTGP_EINVAL;
  if (n < 0) return fail(c, ROTGP_EINVAL, "negative step count");
  if (n == 0) return ROTGP_OK;
  if (!omega) return fail(c, ROTGP_EINVAL, "null schedule");
  ++c->plan_version;
  // the solver was sized for the context's Omega: the largest |Omega| of the
  // schedule has the slowest carries and must fit the same halo and tables
  double big = std::fabs(c->phys.omega);
  for (long long k = 0; k < n; ++k) {
    if (!std::isfinite(omega[k])) return fail(c, ROTGP_EINVAL, "non-finite Omega at step %lld", k);
    big = std::max(big, std::fabs(omega[k]));
  }
  {
    const rotgp_phys keep = c->phys;
    c->phys.omega = big;
    int halo = 0, lt = 0;
    double dec = 0;
    bool ck = true;
    int rc = plan_solver(c, &halo, &lt, &dec, &ck);
    c->phys = keep;
    if (rc) return rc;
    if (lt > c->lt || (ck && halo > c->halo) || ck != c->chunk_ok)
      return fail(c, ROTGP_EUNSUPPORTED,
                  "|Omega| = %g needs a larger line-solver plan than the context's; create the "
                  "context (or rotgp_set_phys) with the largest |Omega| of the schedule",
                  big);
  }
  const int mode = imag ? 1 : 0;
  for (long long k = 0; k < n; ++k) {
    if (omega[k] != c->phys.omega) {
      // the x and y tables of this mode (z lines carry no rotation term)
      c->phys.omega = omega[k];
      for (int a = 0; a < 2; ++a) {
        AxisPlan& ap = c->axis[a];
        ap.co[mode] = make_coef(a, mode, c->grid.h[a], c->phys.dt, c->phys.omega,
                                nlines_u0(c, a), nlines_du(c, a));
        Timed t(c, K_TABLES);
        cudaError_t e = launch_tables(c->fp64, ap.table[mode], ap.tableT[mode], ap.nlines, c->lt,
                                      ap.co[mode], c->stream);
        if (e == cudaSuccess && ap.stencil_ok && ap.wtab[mode])
          e = launch_stencil_tables(ap.wtab[mode], ap.nlines, ap.sK, ap.sB,
                                    2 * ap.sB + 2 * ap.sK + 8, ap.co[mode], c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "table kernel");
      }
    }
    const int rc = run_steps(c, 1, imag != 0);
    if (rc) return rc;
  }
  // the other mode's tables follow the final Omega too
  return build_tables(c);
}

int rotgp_observables(rotgp_ctx* c, rotgp_obs* out) {
  if (!c || !out) return c ? fail(c, ROTGP_EINVAL, "null output") : ROTGP_EINVAL;
  obs_args a{};
  a.psi = c->psi[c->cur];
  a.nx = c->nx;
  a.ny = c->ny;
  a.nz = c->nz;
  a.dim = c->grid.dim;
  a.hx = c->grid.h[0];
  a.hy = c->grid.h[1];
  a.hz = c->grid.dim == 3 ? c->grid.h[2] : 0.0;
  a.x0 = c->x0;
  a.y0 = c->y0;
  a.z0 = c->z0;
  a.hgam2 = 0.5 * c->phys.gamma * c->phys.gamma;
  a.hnu2 = 0.5 * c->phys.nu * c->phys.nu;
  a.hlam2 = c->grid.dim == 3 ? 0.5 * c->phys.lambda * c->phys.lambda : 0.0;
  a.g = c->phys.g;
  a.omega = c->phys.omega;
  a.scale = c->d_scale();
  a.partials = c->partials;
  a.counter = c->counter;
  a.result = c->d_obs();
  cudaError_t e;
  {
    // work items of 32 x 8 columns and a z range: split z until there are
    // about reduce_blocks() items (at least 16 planes each), at most that
    // many blocks (the partials buffer), items taken grid-stride
    const long long tiles = (long long)((c->nx + 31) / 32) * ((c->ny + 7) / 8);
    const long long want = reduce_blocks(c, c->sites);
    const int nz = c->grid.dim == 3 ? c->nz : 1;
    const long long zparts =
        std::max(1LL, std::min<long long>((want + tiles - 1) / tiles, nz / 16));
    a.zchunk = (int)((nz + zparts - 1) / zparts);
    const long long items = tiles * ((nz + a.zchunk - 1) / a.zchunk);
    const int blocks = (int)std::min(items, want);
    Timed t(c, K_OBS);
    e = launch_observables(c->fp64, a, blocks, 256, c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "observables kernel");
  vort_args v{};
  v.psi = c->psi[c->cur];
  v.nx = c->nx;
  v.ny = c->ny;
  v.nz = c->nz;
  v.dim = c->grid.dim;
  v.kplane = c->grid.dim == 3 ? c->grid.n[2] / 2 : 0;
  v.hx = c->grid.h[0];
  v.hy = c->grid.h[1];
  v.x0 = c->x0;
  v.y0 = c->y0;
  v.partials = c->partials;
  v.counter = c->counter;
  v.moments = c->d_moments();
  v.count = c->d_count();
  const int vb = reduce_blocks(c, (long long)c->nx * c->ny);
  {
    Timed t(c, K_VMOM);
    e = launch_vortex_moments(c->fp64, v, vb, 256, c->stream);
  }
  if (e == cudaSuccess) {
    Timed t(c, K_VCOUNT);
    e = launch_vortex_count(c->fp64, v, vb, 256, c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "vortex kernels");
  e = cudaMemcpyAsync(c->h_obs, c->d_obs(), NOBS * sizeof(double), cudaMemcpyDeviceToHost,
                      c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->h_obs + NOBS, c->d_count(), sizeof(int), cudaMemcpyDeviceToHost,
                        c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "copy observables");
  int rc = check_flags(c);
  if (rc) return rc;
  const double* r = c->h_obs;
  out->norm = r[0];
  out->mu = r[1];
  out->energy = r[2];
  out->mu_c = r[3];
  out->energy_c = r[4];
  out->rms_x = r[5];
  out->rms_y = r[6];
  out->rms_z = r[7];
  out->rms_r = r[8];
  out->max_density = r[9];
  out->mu4 = r[10];
  out->energy4 = r[11];
  int cnt = 0;
  std::memcpy(&cnt, c->h_obs + NOBS, sizeof(int));
  out->vortices = cnt;
  out->step = c->steps;
  out->flags = c->phys.omega >= std::min(c->phys.gamma, c->phys.nu) ? 1 : 0;
  return ROTGP_OK;
}

int rotgp_sync(rotgp_ctx* c) {
  if (!c) return ROTGP_EINVAL;
  return check_flags(c);
}

int rotgp_info(const rotgp_ctx* c, rotgp_solver_info* out) {
  if (!c || !out) return ROTGP_EINVAL;
  out->precision = c->prec;
  out->halo = c->halo;
  for (int a = 0; a < 3; ++a) {
    const bool on = a < c->grid.dim;
    out->chunk[a] = on ? c->axis[a].sh.C : 0;
    out->segments[a] =
        on ? (c->axis[a].use_hybrid ? c->axis[a].hcs
                                    : (a >= 1 && c->axis[a].use_stencil ? c->axis[a].lsegs
                                                                        : c->axis[a].nseg))
           : 0;
    out->lines_per_lane[a] = on ? c->axis[a].sh.V : 0;
    out->ring[a] = on ? c->axis[a].sh.R : 0;
    out->stencil_taps[a] = on && c->axis[a].use_stencil ? 2 * c->axis[a].sK + 1 : 0;
    out->warps_per_block[a] = on ? c->axis[a].sh.warps_per_block : 0;
    out->hybrid_cluster[a] = on && c->axis[a].use_hybrid ? c->axis[a].hcs : 0;
  }
  out->table_len = c->lt;
  out->fused_xy = c->fuse_xy ? 1 : 0;
  out->decay = c->decay;
  out->device_bytes = c->device_bytes;
  return ROTGP_OK;
}

int rotgp_tune(rotgp_ctx* c, int axis, int lines_per_lane, int chunk, int ring,
               int warps_per_block, int segments) {
  if (!c) return ROTGP_EINVAL;
  ++c->plan_version;
  if (axis >= 1 && axis < c->grid.dim && c->axis[axis].use_stencil) {
    // stencil form of a y or z sweep: only the segment count applies
    if (segments < 1 || segments > kMaxLineSegs || segments > c->axis[axis].len / 8)
      return fail(c, ROTGP_EINVAL, "segments must be 1..%d and leave >= 8 points each",
                  kMaxLineSegs);
    c->axis[axis].lsegs = segments;
    return ROTGP_OK;
  }
  if (axis < 0 || axis >= c->grid.dim) return fail(c, ROTGP_EINVAL, "axis out of range");
  if (c->axis[axis].use_hybrid) {
    // exact partition solve: only the segment count applies, as the number
    // of CTAs (one cluster) that share each line
    AxisPlan& ap = c->axis[axis];
    if (segments != 1 && segments != 2 && segments != 4 && segments != 8)
      return fail(c, ROTGP_EINVAL, "the exact solve splits a line over 1, 2, 4 or 8 CTAs");
    int pc = 0, ls = 0;
    const size_t bytes = hybrid_tile(ap.len, axis, c->fp64, segments, &pc, &ls);
    if (bytes > (size_t)c->smem_optin - 16 * 1024 ||
        hybrid_max_clusters(c->fp64, axis, segments, pc) < 1)
      return fail(c, ROTGP_EINVAL, "a line of %d points does not fit %d CTAs", ap.len, segments);
    if (axis == c->grid.dim - 1 &&
        (size_t)(hybrid_groups(axis, ap.lines, c->nx) * segments) > c->partial_doubles)
      return fail(c, ROTGP_EINVAL, "%d CTAs per line exceed the reduction buffer", segments);
    ap.hcs = segments;
    ap.hpc = pc;
    ap.hlsub = ls;
    return ROTGP_OK;
  }
  if (warps_per_block < 1 || warps_per_block > 8)
    return fail(c, ROTGP_EINVAL, "warps_per_block must be 1..8");
  if (segments < 1) return fail(c, ROTGP_EINVAL, "segments must be >= 1");
  const AxisPlan keep = c->axis[axis];
  int rc = set_shape(c, axis, lines_per_lane, chunk, ring, warps_per_block, segments);
  if (rc) {
    c->axis[axis] = keep;
    return rc;
  }
  return ROTGP_OK;
}

int rotgp_set_solver(rotgp_ctx* c, int axis, int solver) {
  if (!c) return ROTGP_EINVAL;
  ++c->plan_version;
  if (axis < 0 || axis >= c->grid.dim) return fail(c, ROTGP_EINVAL, "axis out of range");
  if (solver != ROTGP_SOLVER_THOMAS && solver != ROTGP_SOLVER_STENCIL &&
      solver != ROTGP_SOLVER_FUSED && solver != ROTGP_SOLVER_HYBRID)
    return fail(c, ROTGP_EINVAL, "unknown solver %d", solver);
  AxisPlan& ap = c->axis[axis];
  if (solver == ROTGP_SOLVER_HYBRID) {
    if (!ap.hyb_ok)
      return fail(c, ROTGP_EUNSUPPORTED, "no exact line-solve tile for axis %d (%s)", axis,
                  ap.hyb_why.c_str());
    ap.use_hybrid = true;
    ap.use_stencil = false;
    if (axis <= 1) c->fuse_xy = false;
    return ROTGP_OK;
  }
  if (!c->chunk_ok)
    return fail(c, ROTGP_EUNSUPPORTED,
                "the line carries decay too slowly for any form but the exact solve");
  if (solver == ROTGP_SOLVER_FUSED) {
    if (axis > 1) return fail(c, ROTGP_EINVAL, "the fused pass covers the x and y sweeps only");
    if (!c->fuse_ok)
      return fail(c, ROTGP_EUNSUPPORTED, "no fused x-y pass for this context");
    c->axis[0].use_stencil = c->axis[1].use_stencil = true;
    c->axis[0].use_hybrid = c->axis[1].use_hybrid = false;
    c->fuse_xy = true;
    return ROTGP_OK;
  }
  if (solver == ROTGP_SOLVER_STENCIL &&
      (!ap.stencil_ok || (axis == 0 && c->nx % 4 != 0 && !c->xpass_ok)))
    return fail(c, ROTGP_EUNSUPPORTED, "no stencil form for axis %d of this context", axis);
  ap.use_stencil = solver == ROTGP_SOLVER_STENCIL;
  ap.use_hybrid = false;
  if (axis <= 1) c->fuse_xy = false;
  return ROTGP_OK;
}

int rotgp_autotune(rotgp_ctx* c, int steps, int* choice) {
  if (!c) return ROTGP_EINVAL;
  ++c->plan_version;
  if (steps < 1) return fail(c, ROTGP_EINVAL, "steps must be >= 1");
  const int dim = c->grid.dim;
  // candidate forms: bit a = axis a in stencil form, bit 3 = fused x-y pass,
  // bit 4 + a = axis a in the exact partition solve
  std::vector<int> cand;
  for (int m = 0; m < (1 << dim); ++m) {
    bool ok = true;
    for (int a = 0; a < dim; ++a)
      if ((m >> a) & 1)
        ok = ok && c->axis[a].stencil_ok && (a != 0 || c->nx % 4 == 0 || c->xpass_ok);
    if (ok) cand.push_back(m);
  }
  if (c->fuse_ok) {
    cand.push_back(8 | 3);
    if (dim == 3 && c->axis[2].stencil_ok) cand.push_back(8 | 7);
  }
  {
    // each candidate again with any of its Thomas axes in the exact solve
    const size_t nbase = cand.size();
    for (size_t i = 0; i < nbase; ++i)
      for (int h = 1; h < (1 << dim); ++h) {
        bool ok = true;
        for (int a = 0; a < dim; ++a)
          if ((h >> a) & 1)
            ok = ok && c->axis[a].hyb_ok && !((cand[i] >> a) & 1) &&
                 !((cand[i] & 8) && a <= 1);
        if (ok) cand.push_back(cand[i] | (h << 4));
      }
    if (!c->chunk_ok) cand.assign(1, ((1 << dim) - 1) << 4);
  }
  auto apply = [&](int m) {
    c->fuse_xy = (m & 8) != 0;
    for (int a = 0; a < dim; ++a) {
      c->axis[a].use_stencil = ((m >> a) & 1) != 0;
      c->axis[a].use_hybrid = ((m >> (4 + a)) & 1) != 0;
    }
  };
  // save the state, its pending scale and the counters
  const size_t state = (size_t)c->sites * c->elem;
  const int cur0 = c->cur;
  const long long steps0 = c->steps;
  const bool prof0 = c->prof;
  c->prof = false;
  double* saved_scale = reinterpret_cast<double*>(static_cast<char*>(c->staging) + state);
  cudaError_t e = cudaMemcpyAsync(c->staging, c->psi[cur0], state, cudaMemcpyDeviceToDevice,
                                  c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(saved_scale, c->d_scale(), sizeof(double), cudaMemcpyDeviceToDevice,
                        c->stream);
  auto restore = [&]() {
    c->cur = cur0;
    c->steps = steps0;
    cudaError_t r = cudaMemcpyAsync(c->psi[cur0], c->staging, state, cudaMemcpyDeviceToDevice,
                                    c->stream);
    if (r == cudaSuccess)
      r = cudaMemcpyAsync(c->d_scale(), saved_scale, sizeof(double), cudaMemcpyDeviceToDevice,
                          c->stream);
    return r;
  };
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  int best = 0, rc = ROTGP_OK;
  float best_ms = 0;
  // the current form and shapes: the faster of two timed repeats
  auto time_current = [&](float* ms) -> bool {
    if ((e = restore()) != cudaSuccess) return false;
    if ((rc = run_steps(c, 1, true))) return false;
    *ms = 0;
    for (int rep = 0; rep < 2; ++rep) {
      float t = 0;
      if ((e = cudaEventRecord(ev[0], c->stream)) != cudaSuccess) return false;
      if ((rc = run_steps(c, steps, true))) return false;
      if ((e = cudaEventRecord(ev[1], c->stream)) != cudaSuccess) return false;
      if ((e = cudaEventSynchronize(ev[1])) != cudaSuccess) return false;
      if ((e = cudaEventElapsedTime(&t, ev[0], ev[1])) != cudaSuccess) return false;
      *ms = rep == 0 ? t : std::min(*ms, t);
    }
    return true;
  };
  for (size_t i = 0; i < cand.size() && e == cudaSuccess && !rc; ++i) {
    apply(cand[i]);
    float ms = 0;
    if (!time_current(&ms)) break;
    if (i == 0 || ms < best_ms) {
      best_ms = ms;
      best = cand[i];
    }
  }
  apply(best);
  // then the launch shapes of the Thomas sweeps (chunk, ring, segments: the
  // number of warps decides how many waves of resident warps a launch takes)
  for (int ax = 0; ax < dim && e == cudaSuccess && !rc; ++ax) {
    AxisPlan& ap = c->axis[ax];
    if (ap.use_stencil || ap.use_hybrid || (ax <= 1 && c->fuse_xy)) continue;
    // lines per lane, chunk length and segment count together (they decide
    // the warp count and the warm-up overhead jointly), then the ring depth
    for (int phase = 0; phase < 2 && e == cudaSuccess && !rc; ++phase) {
      const AxisPlan keep = ap;
      AxisPlan best_plan = keep;
      std::vector<std::array<int, 4>> shapes;  // {V, C, R, segments}
      if (phase == 0) {
        for (int V : {1, 2}) {
          const bool lean_ok = !c->fp64 && (ax == 0 ? c->xmaps_ok : c->smaps_ok);
          if (V != keep.sh.V && !lean_ok) continue;
          for (int C : {8, 16, 64})
            for (int sg : {1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64}) {
              if (sg > (ap.len + C - 1) / C) continue;
              shapes.push_back({V, C, keep.sh.R, sg});
            }
        }
      } else {
        for (int R : {3, 4, 5, 6}) shapes.push_back({keep.sh.V, keep.sh.C, R, keep.nseg});
      }
      for (const auto& sh : shapes) {
        if (sh[0] == keep.sh.V && sh[1] == keep.sh.C && sh[2] == keep.sh.R && sh[3] == keep.nseg)
          continue;
        const bool x1t = sh[0] == 1 && (sh[1] == 8 || sh[1] == 16) &&
                         (ax == 0 ? c->xmaps_ok : c->smaps_ok);
        if (!sweep_shape_built(c->fp64, sh[0], sh[1]) && !x1t) continue;
        if (set_shape(c, ax, sh[0], sh[1], sh[2], keep.sh.warps_per_block, sh[3]) != ROTGP_OK ||
            ap.nseg != sh[3] || ((size_t)ap.sh.blocks > c->partial_doubles && ax == dim - 1)) {
          ap = keep;
          continue;
        }
        float ms = 0;
        if (!time_current(&ms)) break;
        if (ms < best_ms) {
          best_ms = ms;
          best_plan = ap;
        }
        ap = keep;
      }
      ap = best_plan;
    }
  }
  // and the segment count of each y/z sweep in stencil form
  for (int ax = 1; ax < dim && e == cudaSuccess && !rc; ++ax) {
    AxisPlan& ap = c->axis[ax];
    if (!ap.use_stencil) continue;
    int best_s = ap.lsegs;
    for (int sg : {1, 2, 4, 8}) {
      if (sg == best_s || sg > ap.len / 16) continue;
      const int keep = ap.lsegs;
      ap.lsegs = sg;
      float ms = 0;
      if (!time_current(&ms)) break;
      if (ms < best_ms) {
        best_ms = ms;
        best_s = sg;
      }
      ap.lsegs = keep;
    }
    ap.lsegs = best_s;
  }
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  const cudaError_t er = restore();
  c->prof = prof0;
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_fail(c, e, "autotune");
  if (er != cudaSuccess) return cuda_fail(c, er, "autotune restore");
  if (choice) *choice = best;
  return check_flags(c);
}

int rotgp_profile_enable(rotgp_ctx* c, int on) {
  if (!c) return ROTGP_EINVAL;
  c->prof = on != 0;
  return ROTGP_OK;
}

int rotgp_profile_read(rotgp_ctx* c, rotgp_kstat* out, int max, int* count) {
  if (!c || (!out && max > 0)) return ROTGP_EINVAL;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "profile sync");
  long long n[K_COUNT] = {0};
  double ms[K_COUNT] = {0};
  for (auto& r : c->recs) {
    float t = 0;
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
      n[r.kid] += 1;
      ms[r.kid] += t;
    }
    c->pool.push_back(r.a);
    c->pool.push_back(r.b);
  }
  c->recs.clear();
  int k = 0;
  for (int id = 0; id < K_COUNT; ++id) {
    if (!n[id]) continue;
    if (k < max) {
      std::memset(&out[k], 0, sizeof(rotgp_kstat));
      std::snprintf(out[k].name, sizeof out[k].name, "%s", kKernelNames[id]);
      out[k].launches = n[id];
      out[k].total_ms = ms[id];
      out[k].bytes_per_launch = c->bytes_per_launch[id];
    }
    ++k;
  }
  if (count) *count = std::min(k, max);
  return ROTGP_OK;
}

}  // extern "C"
