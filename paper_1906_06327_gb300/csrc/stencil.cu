// stencil.cu -- the complex-float Crank-Nicolson sweeps in banded-inverse
// form.
//
// For one line, the CN substep of Eq. eqD.9 is A psi' = E psi with the
// tridiagonal A of Eqs. eqD.11/eq5 and E its explicit counterpart (diagonal
// 1 - 2 kappa, off-diagonals -A- and -A+).  E = 2 I - A exactly, so
//     psi' = (2 A^{-1} - I) psi = W psi.
// A is strictly diagonally dominant, so the entries of W decay
// geometrically away from the diagonal (by the carry-decay factor per
// point, ~1e-2 on the workloads here): W is banded to within a relative
// 1e-9 with K points on either side.  Away from the ends of the line its
// rows are the same for every point (A is Toeplitz); B rows at each end
// differ.  Each line's weights -- the interior row and the 2B end rows --
// are computed here from the exact inverse of a short line (Thomas solves
// in double), and the sweep becomes a (2K+1)-tap complex stencil: every
// output point is independent, loads are coalesced, and two lines are
// processed per lane in packed FP32x2 arithmetic.  The result equals the
// Thomas solve up to the truncated tail (bounded by the host) and float
// rounding.
//
// This file holds the weight tables and the x sweep on its own (used when
// the y sweep is not in stencil form): a warp stages two rows of 128 + 2K
// points in shared memory with the pending scale and the H1 substep (Eq.
// eq1) applied once per point, and each lane produces 4 consecutive points
// of both rows.  The y and z sweeps (tiles_line.cu) and the fused H1 + x + y
// pass (tiles_xy.cu) use the same tables.
#include <algorithm>

#include "sweep_common.cuh"

namespace rotgp {

// ----------------------------------------------------------------- weights
namespace {
constexpr int kMaxSmall = 96;  // unknowns of the short line used for the weights
}

// Thread per coefficient line.  The short line has m unknowns (positions
// 1..m); W = 2 A^{-1} - I column by column (A y = e_j by the Thomas
// algorithm).  Table rows: r < B left end (position r, row 0 = the zero
// edge), r = B interior (the middle of the short line), r = B + 1 + e the
// right end (position N - 1 - e); tap k multiplies the point p - K + k.
__global__ void k_stencil_tables(cpx<float>* wtab, int nlines, int K, int B, int m,
                                 axis_coef co) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nlines || m > kMaxSmall) return;
  const int S = 2 * K + 1, NR = 2 * B + 1;
  const double u = co.u0 + (double)l * co.du;
  const double kr = co.kap_re, ki = co.kap_im;
  const double tr = co.tau_re * u, ti = co.tau_im * u;
  const double a0r = 1.0 + 2.0 * kr, a0i = 2.0 * ki;
  const double amr = -kr + tr, ami = -ki + ti;
  const double apr = -kr - tr, api = -ki - ti;
  cpx<float>* T = wtab + (size_t)l * NR * S;
  for (int i = 0; i < NR * S; ++i) T[i] = mk<float>(0.f, 0.f);
  // Thomas multipliers m_i = 1/(A0 - A- c_{i-1}), c_i = A+ m_i
  double cr[kMaxSmall + 1], ci[kMaxSmall + 1], mr[kMaxSmall + 1], mi[kMaxSmall + 1];
  double dr[kMaxSmall + 2], di[kMaxSmall + 2];
  cr[0] = ci[0] = 0.0;
  for (int i = 1; i <= m; ++i) {
    const double xr = a0r - (amr * cr[i - 1] - ami * ci[i - 1]);
    const double xi = a0i - (amr * ci[i - 1] + ami * cr[i - 1]);
    const double inv = 1.0 / (xr * xr + xi * xi);
    mr[i] = xr * inv;
    mi[i] = -xi * inv;
    cr[i] = apr * mr[i] - api * mi[i];
    ci[i] = apr * mi[i] + api * mr[i];
  }
  const int pmid = B + K + 4;
  for (int j = 1; j <= m; ++j) {
    // forward: d_i = (delta_ij - A- d_{i-1}) m_i
    dr[0] = di[0] = 0.0;
    for (int i = 1; i <= m; ++i) {
      const double br = (i == j ? 1.0 : 0.0) - (amr * dr[i - 1] - ami * di[i - 1]);
      const double bi = -(amr * di[i - 1] + ami * dr[i - 1]);
      dr[i] = br * mr[i] - bi * mi[i];
      di[i] = br * mi[i] + bi * mr[i];
    }
    // back substitution in place: y_i = d_i - c_i y_{i+1}
    for (int i = m - 1; i >= 1; --i) {
      const double yr = dr[i] - (cr[i] * dr[i + 1] - ci[i] * di[i + 1]);
      const double yi = di[i] - (cr[i] * di[i + 1] + ci[i] * dr[i + 1]);
      dr[i] = yr;
      di[i] = yi;
    }
    for (int r = 0; r < NR; ++r) {
      const int p = r < B ? r : (r == B ? pmid : m - (r - B - 1));
      if (p < 1) continue;
      const int k = j - p + K;
      if (k < 0 || k >= S) continue;
      T[r * S + k] = mk<float>((float)(2.0 * dr[p] - (p == j ? 1.0 : 0.0)), (float)(2.0 * di[p]));
    }
  }
}

cudaError_t launch_stencil_tables(void* wtab, int nlines, int K, int B, int m,
                                  const axis_coef& co, cudaStream_t s) {
  if (m > kMaxSmall) return cudaErrorInvalidValue;
  const int threads = 64, blocks = (nlines + threads - 1) / threads;
  k_stencil_tables<<<blocks, threads, 0, s>>>(static_cast<cpx<float>*>(wtab), nlines, K, B, m, co);
  return cudaGetLastError();
}

// Weights of two lines at table row r, tap k, as a split coefficient.
__device__ __forceinline__ k2 wpair(const cpx<float>* w0, const cpx<float>* w1, int S, int r,
                                    int k) {
  return make_k2(w0[r * S + k], w1[r * S + k]);
}

// ----------------------------------------------------------------- x
// A task is two rows x 128 output points.  Each lane loads its four points
// of both rows (and, at the warp's ends, the K-point halos), applies the
// pending scale and H1 once per point into a small shared staging row, and
// produces four consecutive points of both rows from its 4 + 2K window.
template <int K>
struct xstencil_layout {
  static constexpr int TW = 128;                // output points per row and task
  static constexpr int WIN = TW + 2 * K;        // staged points
  static constexpr int SP = WIN + WIN / 8 + 1;  // staging, one pad unit per 8
};

template <int K, bool IMAG>
__global__ void __launch_bounds__(128) k_stencil_x(const stream_args a) {
  using E = cpx<float>;
  using LY = xstencil_layout<K>;
  constexpr int S = 2 * K + 1, TW = LY::TW, SP = LY::SP;
  __shared__ float4 stage[4][SP];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nrows = (int)a.nlines;
  const int N = a.len, B = a.brows, NR = 2 * B + 1;
  const int npairs = (nrows + 1) / 2;
  const int ntiles = (N + TW - 1) / TW;
  const int t = blockIdx.x * (blockDim.x >> 5) + wib;
  if (t >= npairs * ntiles) return;  // whole warp; no block barrier below
  const int pair = t / ntiles;
  const int x0 = (t - pair * ntiles) * TW;
  const int r0 = 2 * pair, r1 = r0 + 1;
  const bool act1 = r1 < nrows;
  const E* in = static_cast<const E*>(a.in);
  E* out = static_cast<E*>(a.out);
  const E* row0 = in + (size_t)r0 * N;
  const E* row1 = in + (size_t)(act1 ? r1 : r0) * N;
  // loads first: the lane's points x0 + 4 lane .. + 3 (two 16-byte copies per
  // row) and, for the first and last K/2 lanes, one halo copy per row
  const int pl = x0 + 4 * lane;
  float4 u[4], hv[2];
  const bool in_line = pl < N;  // N is a multiple of 4
  u[0] = in_line ? *reinterpret_cast<const float4*>(row0 + pl) : make_float4(0.f, 0.f, 0.f, 0.f);
  u[1] = in_line ? *reinterpret_cast<const float4*>(row0 + pl + 2) : make_float4(0.f, 0.f, 0.f, 0.f);
  u[2] = in_line && act1 ? *reinterpret_cast<const float4*>(row1 + pl) : make_float4(0.f, 0.f, 0.f, 0.f);
  u[3] = in_line && act1 ? *reinterpret_cast<const float4*>(row1 + pl + 2) : make_float4(0.f, 0.f, 0.f, 0.f);
  int ph = -1;  // halo pair start of this lane (even), or -1
  if (lane < K / 2) ph = x0 - K + 2 * lane;
  if (lane >= 32 - K / 2) ph = x0 + TW + 2 * (lane - (32 - K / 2));
  const bool hin = ph >= 0 && ph < N;
  hv[0] = hin ? *reinterpret_cast<const float4*>(row0 + ph) : make_float4(0.f, 0.f, 0.f, 0.f);
  hv[1] = hin && act1 ? *reinterpret_cast<const float4*>(row1 + ph) : make_float4(0.f, 0.f, 0.f, 0.f);

  const int k0 = r0 / a.ny, j0 = r0 - k0 * a.ny;
  const int k1 = act1 ? r1 / a.ny : k0, j1 = act1 ? r1 - k1 * a.ny : j0;
  const E* w0 = static_cast<const E*>(a.wtab) + (size_t)j0 * NR * S;
  const E* w1 = static_cast<const E*>(a.wtab) + (size_t)j1 * NR * S;
  float2 VYZ;
  {
    const float ya = (float)(a.y0 + (double)j0 * a.hy), za = (float)(a.z0 + (double)k0 * a.hz);
    const float yb = (float)(a.y0 + (double)j1 * a.hy), zb = (float)(a.z0 + (double)k1 * a.hz);
    VYZ = make_float2((float)a.hnu2 * ya * ya + (float)a.hlam2 * za * za,
                      (float)a.hnu2 * yb * yb + (float)a.hlam2 * zb * zb);
  }
  const float s = (float)(*a.scale), hg2 = (float)a.hgam2, dt = (float)a.dt;
  const float2 S2 = make_float2(s, s), G2 = make_float2((float)a.g, (float)a.g);
  const float xs = (float)a.x0, hx = (float)a.hx;
  // point p of both rows (re/im of row 0 and row 1), scaled and advanced by H1
  auto h1 = [&](float2 a0, float2 a1, int p) -> c2 {
    c2 v = zero2();
    if (p >= 1 && p < N) {
      v.re = __fmul2_rn(S2, make_float2(a0.x, a1.x));
      v.im = __fmul2_rn(S2, make_float2(a0.y, a1.y));
      const float x = xs + (float)p * hx;
      const float vx = hg2 * x * x;
      const float2 dens = __ffma2_rn(v.im, v.im, __fmul2_rn(v.re, v.re));
      const float2 en = __ffma2_rn(G2, dens, __fadd2_rn(VYZ, make_float2(vx, vx)));
      if (IMAG) {
        const float2 f = make_float2(__expf(-dt * en.x), __expf(-dt * en.y));
        v.re = __fmul2_rn(f, v.re);
        v.im = __fmul2_rn(f, v.im);
      } else {
        float2 s1, c1;
        rot_t(dt * en.x, &c1.x, &s1.x);
        rot_t(dt * en.y, &c1.y, &s1.y);
        const float2 re = __ffma2_rn(c1, v.re, __ffma2_rn(s1, v.im, v.re));
        v.im = __ffma2_rn(c1, v.im, __ffma2_rn(make_float2(-s1.x, -s1.y), v.re, v.im));
        v.re = re;
      }
    }
    return v;
  };
  float4* st = stage[wib];
  auto put_stage = [&](int i, const c2& v) { st[i + i / 8] = pack_split(v); };
  // staged index i <-> point x0 - K + i
  {
    const int i0 = 4 * lane + K;
    put_stage(i0 + 0, h1(make_float2(u[0].x, u[0].y), make_float2(u[2].x, u[2].y), pl + 0));
    put_stage(i0 + 1, h1(make_float2(u[0].z, u[0].w), make_float2(u[2].z, u[2].w), pl + 1));
    put_stage(i0 + 2, h1(make_float2(u[1].x, u[1].y), make_float2(u[3].x, u[3].y), pl + 2));
    put_stage(i0 + 3, h1(make_float2(u[1].z, u[1].w), make_float2(u[3].z, u[3].w), pl + 3));
    if (ph >= 0 || lane < K / 2 || lane >= 32 - K / 2) {
      if (lane < K / 2 || lane >= 32 - K / 2) {
        const int ih = ph - (x0 - K);
        put_stage(ih, h1(make_float2(hv[0].x, hv[0].y), make_float2(hv[1].x, hv[1].y), ph));
        put_stage(ih + 1, h1(make_float2(hv[0].z, hv[0].w), make_float2(hv[1].z, hv[1].w), ph + 1));
      }
    }
  }
  __syncwarp();
  c2 win[4 + 2 * K];
#pragma unroll
  for (int i = 0; i < 4 + 2 * K; ++i) {
    const int idx = 4 * lane + i;
    win[i] = unpack_split(st[idx + idx / 8]);
  }
  c2 res[4];
  if (pl >= B && pl + 3 < N - B) {
    k2 w[S];
#pragma unroll
    for (int kk = 0; kk < S; ++kk) w[kk] = wpair(w0, w1, S, B, kk);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      c2 x = kmul2(w[0], win[m]);
#pragma unroll
      for (int kk = 1; kk < S; ++kk) x = kfma2(w[kk], win[m + kk], x);
      res[m] = x;
    }
  } else {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int p = pl + m;
      c2 x = zero2();
      if (p < N) {
        const int row = stencil_row(p, N, B);
#pragma unroll
        for (int kk = 0; kk < S; ++kk) x = kfma2(wpair(w0, w1, S, row, kk), win[m + kk], x);
      }
      res[m] = x;
    }
  }
  if (in_line) {
    float4* o0 = reinterpret_cast<float4*>(out + (size_t)r0 * N + pl);
    o0[0] = make_float4(res[0].re.x, res[0].im.x, res[1].re.x, res[1].im.x);
    o0[1] = make_float4(res[2].re.x, res[2].im.x, res[3].re.x, res[3].im.x);
    if (act1) {
      float4* o1 = reinterpret_cast<float4*>(out + (size_t)r1 * N + pl);
      o1[0] = make_float4(res[0].re.y, res[0].im.y, res[1].re.y, res[1].im.y);
      o1[1] = make_float4(res[2].re.y, res[2].im.y, res[3].re.y, res[3].im.y);
    }
  }
}

// ----------------------------------------------------------------- launchers
cudaError_t launch_stencil_x(bool imag, const stream_args& a, long long /*warps*/,
                             cudaStream_t s) {
  const long long tasks = ((a.nlines + 1) / 2) * ((a.len + 127) / 128);
  const unsigned blocks = (unsigned)((tasks + 3) / 4);
#define ROTGP_SX(KK)                                                              \
  if (a.taps_k == KK) {                                                           \
    if (imag)                                                                     \
      k_stencil_x<KK, true><<<blocks, 128, 0, s>>>(a);                            \
    else                                                                          \
      k_stencil_x<KK, false><<<blocks, 128, 0, s>>>(a);                           \
    return cudaGetLastError();                                                    \
  }
  ROTGP_SX(4)
  ROTGP_SX(6)
  ROTGP_SX(8)
#undef ROTGP_SX
  return cudaErrorInvalidValue;
}

}  // namespace rotgp
