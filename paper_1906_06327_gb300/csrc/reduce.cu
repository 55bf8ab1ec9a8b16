// reduce.cu -- the read-only reductions over a state: the observables of
// Sec. 2 (norm, real-part mu and E of Eqs. e2dr/e3dr, complex forms of
// Eqs. e2d/e3d, rms sizes), the vortex count diagnostic, and the plain norm
// used after loading a state.
//
// Every reduction is one pass over the state: each thread accumulates its
// sites in registers, blocks reduce with warp shuffles and write one partial
// per block, and the last block to finish (atomic ticket) combines the
// partials in block order, so results are deterministic run to run.  The
// pending imaginary-time scale is applied as the state is read.
#include "common.cuh"

namespace rotgp {

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double wmax(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// Reduce q[0..NV) over the block (entry NV-1 with max if MAXLAST), store the
// block partial, and return true in the block that finishes last (whose
// threads must then combine the partials).
template <int NV, bool MAXLAST>
__device__ bool block_partials(double* q, double* partials, unsigned* counter) {
  __shared__ double ws[32][NV];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double x = (MAXLAST && v == NV - 1) ? wmax(q[v]) : wsum(q[v]);
    if (lane == 0) ws[warp][v] = x;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    const int v = threadIdx.x;
    double s = 0;
    for (int w = 0; w < nw; ++w) s = (MAXLAST && v == NV - 1) ? fmax(s, ws[w][v]) : s + ws[w][v];
    partials[(size_t)blockIdx.x * NV + v] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  return last;
}

// In the last block: thread v < NV sums partial v over all blocks in order.
// Combine the partials of all blocks into fin[0..NV) (shared), in the last
// block: thread t sums blocks t, t + blockDim, ... in order, then warps and
// the block reduce in a fixed order (deterministic run to run).  Every
// thread of the block must call it.
template <int NV, bool MAXLAST>
__device__ void combine_all(const double* partials, double* fin) {
  __shared__ double red[32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const bool mx = MAXLAST && v == NV - 1;
    double s = 0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
      const double x = __ldcg(&partials[(size_t)b * NV + v]);
      s = mx ? fmax(s, x) : s + x;
    }
    s = mx ? wmax(s) : wsum(s);
    if (lane == 0) red[warp][v] = s;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    const bool mx = MAXLAST && (int)threadIdx.x == NV - 1;
    double s = 0;
    for (int w = 0; w < nw; ++w) s = mx ? fmax(s, red[w][threadIdx.x]) : s + red[w][threadIdx.x];
    fin[threadIdx.x] = s;
  }
  __syncthreads();
}

// ------------------------------------------------------------ observables
// Per interior site (edges are zero and contribute nothing), with the
// 3-point Laplacian lap and central differences D of the CN sweeps:
//   q0 |psi|^2   q1 psi_R^2   q2 psi_I^2
//   q3 psi_R (-lap psi_R/2 + V psi_R + Omega (y D_x psi_I - x D_y psi_I))
//   q4 g |psi|^2 psi_R^2
//   q5, q6  the same two for the state rotated by -i (R <- I, I <- -R)
//   q7 Re psi^* (-lap/2 + V - Omega L_z) psi, L_z = i (y D_x - x D_y)
//   q8 g |psi|^4   q9..q11  x^2, y^2, z^2 times |psi|^2
//   q12 as q7 with fourth-order central differences (Laplacian
//       (-f2 + 16 f1 - 30 f0 + 16 f-1 - f-2)/(12 h^2), first derivative
//       (-f2 + 8 f1 - 8 f-1 + f-2)/(12 h); points beyond the grid are zero)
//   q13 max |psi|^2
// The state is read once: a block owns tiles of 32 x 8 columns (x, y) and a
// range of z; each thread walks its column in z with the five points z-2 ..
// z+2 in registers, and the plane z is staged in shared memory with a halo
// of 2 in x and y for the x and y differences (a star stencil: no corners).
// Work items (tile, z range) are taken grid-stride.
constexpr int kObsTX = 32, kObsTY = 8;

// fused multiply-add in the working precision
__device__ __forceinline__ float fmat(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmat(double a, double b, double c) { return fma(a, b, c); }

// Per-thread running sums of the observables: Kahan-compensated in float
// (the error of a sum of n terms stays at float rounding instead of growing
// with n), plain in double.
template <class T>
struct obs_acc {
  T s[NQ], c[NQ];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int v = 0; v < NQ; ++v) s[v] = c[v] = 0;
  }
  template <int V>
  __device__ __forceinline__ void add(T x) {
    const T y = x - c[V];
    const T t = s[V] + y;
    c[V] = (t - s[V]) - y;
    s[V] = t;
  }
  __device__ __forceinline__ double value(int v) const { return (double)s[v] - (double)c[v]; }
};
template <>
struct obs_acc<double> {
  double s[NQ];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int v = 0; v < NQ; ++v) s[v] = 0;
  }
  template <int V>
  __device__ __forceinline__ void add(double x) { s[V] += x; }
  __device__ __forceinline__ double value(int v) const { return s[v]; }
};

template <class T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k_observables(const obs_args a) {
  using C = cpx<T>;
  constexpr int TX = kObsTX, TY = kObsTY, WX = TX + 4, WY = TY + 4;
  __shared__ C tile[2][WY][WX];
  const C* psi = static_cast<const C*>(a.psi);
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const long long plane = (long long)nx * ny;
  const T s = (T)(*a.scale);
  const T ihx2 = (T)(1.0 / (a.hx * a.hx)), ihy2 = (T)(1.0 / (a.hy * a.hy));
  const T ihz2 = a.dim == 3 ? (T)(1.0 / (a.hz * a.hz)) : (T)0;
  const T i2hx = (T)(0.5 / a.hx), i2hy = (T)(0.5 / a.hy);
  const T om = (T)a.omega, g = (T)a.g;
  const T c12x = ihx2 / (T)12, c12y = ihy2 / (T)12, c12z = ihz2 / (T)12;
  const T i12hx = (T)(0.5 / a.hx / 6.0), i12hy = (T)(0.5 / a.hy / 6.0);
  // coordinates and potential constants in the working precision, once:
  // no conversion from double inside the site loops
  const T x0 = (T)a.x0, y0 = (T)a.y0, z0 = (T)a.z0, hx = (T)a.hx, hy = (T)a.hy;
  const T hz = a.dim == 3 ? (T)a.hz : (T)0;
  const T hgam2 = (T)a.hgam2, hnu2 = (T)a.hnu2, hlam2 = (T)a.hlam2;
  const bool d3 = a.dim == 3;
  const T l0 = (T)2 * (ihx2 + ihy2 + ihz2), l04 = (T)30 * (c12x + c12y + c12z);
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int tiles_x = (nx + TX - 1) / TX, tiles_y = (ny + TY - 1) / TY;
  const int zlen = a.zchunk, zparts = (nz + zlen - 1) / zlen;
  const long long items = (long long)tiles_x * tiles_y * zparts;
  // a point of the state (scaled), zero outside the stored grid
  auto at = [&](int i, int j, int k) -> C {
    if (i < 0 || i >= nx || j < 0 || j >= ny || k < 0 || k >= nz) return mk<T>(0, 0);
    return s * psi[(long long)k * plane + (long long)j * nx + i];
  };
  // per-thread sums in the working precision (compensated in float),
  // promoted to double for the block and grid reduction
  obs_acc<T> t;
  t.zero();
  T dmax = 0;
  int buf = 0;
  for (long long it = blockIdx.x; it < items; it += gridDim.x) {
    const int zp_ = (int)(it % zparts);
    const long long tt = it / zparts;
    const int bx = (int)(tt % tiles_x), by = (int)(tt / tiles_x);
    const int i = bx * TX + tx, j = by * TY + ty;
    const int k0 = zp_ * zlen, k1 = min(nz, k0 + zlen);
    const T x = x0 + (T)i * hx;
    const T y = y0 + (T)j * hy;
    const T xxv = hgam2 * x * x + hnu2 * y * y;
    const T x2 = x * x, y2 = y * y;
    const T yh = y * i2hx, xh = x * i2hy, y12 = y * i12hx, x12 = x * i12hy;
    T kf = (T)k0;  // the plane index as a number, advanced per plane
    // the column's window z-2 .. z+2
    C w[5];
#pragma unroll
    for (int d = 0; d < 5; ++d) w[d] = at(i, j, k0 - 2 + d);
    // this thread's halo points of a plane (at most one in x, one in y)
    const bool hxl = tx < 2, hxr = tx >= TX - 2, hyl = ty < 2, hyr = ty >= TY - 2;
    const int hxi = hxl ? bx * TX - 2 + tx : bx * TX + tx + 2;
    const int hyj = hyl ? by * TY - 2 + ty : by * TY + ty + 2;
    auto halo_x = [&](int k) { return (hxl || hxr) ? at(hxi, j, k) : mk<T>(0, 0); };
    auto halo_y = [&](int k) { return (hyl || hyr) ? at(i, hyj, k) : mk<T>(0, 0); };
    C hxv = halo_x(k0), hyv = halo_y(k0);
    for (int k = k0; k < k1; ++k) {
      // the next plane's points are requested before this plane is used
      const C wn = at(i, j, k + 3);
      const C hxn = k + 1 < k1 ? halo_x(k + 1) : mk<T>(0, 0);
      const C hyn = k + 1 < k1 ? halo_y(k + 1) : mk<T>(0, 0);
      // stage the plane: centre from the window, halo strips
      tile[buf][ty + 2][tx + 2] = w[2];
      if (hxl) tile[buf][ty + 2][tx] = hxv;
      if (hxr) tile[buf][ty + 2][tx + 4] = hxv;
      if (hyl) tile[buf][ty][tx + 2] = hyv;
      if (hyr) tile[buf][ty + 4][tx + 2] = hyv;
      __syncthreads();
      const bool interior = i >= 1 && i < nx && j >= 1 && j < ny && (!d3 || k >= 1);
      if (interior) {
        // the same terms with the sums and differences of each axis formed
        // once (in 2D the z points are zero and ihz2 = 0)
        const C c = w[2];
        const C xp = tile[buf][ty + 2][tx + 3], xm = tile[buf][ty + 2][tx + 1];
        const C xp2 = tile[buf][ty + 2][tx + 4], xm2 = tile[buf][ty + 2][tx];
        const C yp = tile[buf][ty + 3][tx + 2], ym = tile[buf][ty + 1][tx + 2];
        const C yp2 = tile[buf][ty + 4][tx + 2], ym2 = tile[buf][ty][tx + 2];
        const C zp = w[3], zm = w[1], zp2 = w[4], zm2 = w[0];
        const T z = z0 + kf * hz;
        const T V = xxv + hlam2 * z * z;
        const C sx = xp + xm, sy = yp + ym, sz = zp + zm;    // neighbour sums
        const C ex = xp2 + xm2, ey = yp2 + ym2, ez = zp2 + zm2;
        const C dx = xp - xm, dy = yp - ym;                  // central differences
        const C fx = xp2 - xm2, fy = yp2 - ym2;
        const T re = c.x, im = c.y, dens = fmat(re, re, im * im);
        // -lap/2 + V and the rotation term, 3-point and 5-point forms;
        // L_z psi / i = y D_x psi - x D_y psi
        const T lapr = fmat(ihx2, sx.x, fmat(ihy2, sy.x, fmat(ihz2, sz.x, -l0 * re)));
        const T lapi = fmat(ihx2, sx.y, fmat(ihy2, sy.y, fmat(ihz2, sz.y, -l0 * im)));
        const T lzr = fmat(yh, dx.x, -xh * dy.x), lzi = fmat(yh, dx.y, -xh * dy.y);
        const T hr = fmat((T)-0.5, lapr, fmat(V, re, om * lzi));
        const T hi = fmat((T)-0.5, lapi, fmat(V, im, -om * lzr));
        const T l4r = fmat(c12x, fmat((T)16, sx.x, -ex.x),
                           fmat(c12y, fmat((T)16, sy.x, -ey.x),
                                fmat(c12z, fmat((T)16, sz.x, -ez.x), -l04 * re)));
        const T l4i = fmat(c12x, fmat((T)16, sx.y, -ex.y),
                           fmat(c12y, fmat((T)16, sy.y, -ey.y),
                                fmat(c12z, fmat((T)16, sz.y, -ez.y), -l04 * im)));
        const T z4r = fmat(y12, fmat((T)8, dx.x, -fx.x), -x12 * fmat((T)8, dy.x, -fy.x));
        const T z4i = fmat(y12, fmat((T)8, dx.y, -fx.y), -x12 * fmat((T)8, dy.y, -fy.y));
        const T h4r = fmat((T)-0.5, l4r, fmat(V, re, om * z4i));
        const T h4i = fmat((T)-0.5, l4i, fmat(V, im, -om * z4r));
        const T gd = g * dens;
        const T e3 = re * hr, e5 = im * hi;
        t.template add<0>(dens);
        t.template add<1>(re * re);
        t.template add<2>(im * im);
        t.template add<3>(e3);
        t.template add<4>(gd * re * re);
        t.template add<5>(e5);
        t.template add<6>(gd * im * im);
        // q7, the complex-form energy density, is q3 + q5 site by site
        t.template add<7>(e3 + e5);
        t.template add<8>(gd * dens);
        t.template add<9>(x2 * dens);
        t.template add<10>(y2 * dens);
        t.template add<11>(z * z * dens);
        t.template add<12>(fmat(re, h4r, im * h4i));
        dmax = dmax > dens ? dmax : dens;
      }
#pragma unroll
      for (int d = 0; d < 4; ++d) w[d] = w[d + 1];
      w[4] = wn;
      hxv = hxn;
      hyv = hyn;
      kf += (T)1;
      buf ^= 1;  // the other buffer is free: every thread is past this plane's barrier
    }
    __syncthreads();  // the next item restages both buffers
  }
  double q[NQ];
#pragma unroll
  for (int v = 0; v < NQ; ++v) q[v] = t.value(v);
  q[13] = (double)dmax;
  if (!block_partials<NQ, true>(q, a.partials, a.counter)) return;
  __shared__ double fin[NQ];
  __threadfence();
  combine_all<NQ, true>(a.partials, fin);
  if (threadIdx.x == 0) {
    double vol = a.hx * a.hy * (a.dim == 3 ? a.hz : 1.0);
    const bool rot = fin[1] < 1e-3 * fin[0];
    const double lin = rot ? fin[5] : fin[3], nl = rot ? fin[6] : fin[4];
    const double den = rot ? fin[2] : fin[1];
    double* r = a.result;
    r[0] = vol * fin[0];
    r[1] = (lin + nl) / den;
    r[2] = (lin + 0.5 * nl) / den;
    r[3] = (fin[7] + fin[8]) / fin[0];
    r[4] = (fin[7] + 0.5 * fin[8]) / fin[0];
    r[5] = sqrt(fin[9] / fin[0]);
    r[6] = sqrt(fin[10] / fin[0]);
    r[7] = a.dim == 3 ? sqrt(fin[11] / fin[0]) : 0.0;
    r[8] = sqrt((fin[9] + fin[10] + fin[11]) / fin[0]);
    r[9] = fin[13];
    r[10] = (fin[12] + fin[8]) / fin[0];
    r[11] = (fin[12] + 0.5 * fin[8]) / fin[0];
    *a.counter = 0u;
  }
}

// ------------------------------------------------------------ vortex count
// Pass 1: density moments of the plane k = kplane (double): sum rho,
// sum x^2 rho, sum y^2 rho -> R_x^2 = 6 <x^2>, R_y^2 = 6 <y^2>.
template <class T>
__global__ void __launch_bounds__(256) k_vort_moments(const vort_args a) {
  using C = cpx<T>;
  const C* pl = static_cast<const C*>(a.psi) + (size_t)a.kplane * a.nx * a.ny;
  const long long n = (long long)a.nx * a.ny;
  double q[3] = {0, 0, 0};
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % a.nx), j = (int)(idx / a.nx);
    const C c = pl[idx];
    const double d = (double)c.x * c.x + (double)c.y * c.y;
    const double x = a.x0 + i * a.hx, y = a.y0 + j * a.hy;
    q[0] += d;
    q[1] += x * x * d;
    q[2] += y * y * d;
  }
  if (!block_partials<3, false>(q, a.partials, a.counter)) return;
  __shared__ double fin[3];
  __threadfence();
  combine_all<3, false>(a.partials, fin);
  if (threadIdx.x == 0) {
    a.moments[0] = fin[0] > 0 ? 6.0 * fin[1] / fin[0] : 0.0;
    a.moments[1] = fin[0] > 0 ? 6.0 * fin[2] / fin[0] : 0.0;
    *a.count = 0;
    *a.counter = 0u;
  }
}

__device__ __forceinline__ float atan2_t(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double atan2_t(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ int round_half_away(float v) { return (int)roundf(v); }
__device__ __forceinline__ int round_half_away(double v) { return (int)round(v); }

// Pass 2: one thread per plaquette (i,j)..(i+1,j+1) touching no edge and
// centred inside 0.9 of the ellipse: winding = round(sum of
// arg(psi_b conj(psi_a)) around the loop / 2 pi), computed in T.
template <class T>
__global__ void __launch_bounds__(256) k_vort_count(const vort_args a) {
  using C = cpx<T>;
  const C* pl = static_cast<const C*>(a.psi) + (size_t)a.kplane * a.nx * a.ny;
  const double rx2 = a.moments[0], ry2 = a.moments[1];
  const long long n = (long long)a.nx * a.ny;
  int cnt = 0;
  if (rx2 > 0 && ry2 > 0) {
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
      const int i = (int)(idx % a.nx), j = (int)(idx / a.nx);
      // corners i..i+1 must avoid both edges 0 and N (N = nx implicit)
      if (i < 1 || j < 1 || i + 1 > a.nx - 1 || j + 1 > a.ny - 1) continue;
      const double xc = a.x0 + i * a.hx + 0.5 * a.hx, yc = a.y0 + j * a.hy + 0.5 * a.hy;
      if (!(xc * xc / rx2 + yc * yc / ry2 < 0.81)) continue;
      C q[4] = {pl[idx], pl[idx + 1], pl[idx + 1 + a.nx], pl[idx + a.nx]};
      T w = 0;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const C u = q[(t + 1) & 3], v = q[t];
        const T pr = u.x * v.x + u.y * v.y;
        const T pim = u.y * v.x - u.x * v.y;
        w += atan2_t(pim, pr);
      }
      const int wn = round_half_away(w / (T)6.28318530717958647692);
      cnt += wn < 0 ? -wn : wn;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(a.count, cnt);
}

// ------------------------------------------------------------ plain norm
template <class T>
__global__ void __launch_bounds__(256) k_norm(const void* psi_v, long long n, double vol,
                                              int imag_scale, double* partials,
                                              unsigned* counter, double* scale_out,
                                              double* norm_out, int* flags) {
  const cpx<T>* psi = static_cast<const cpx<T>*>(psi_v);
  double q[1] = {0.0};
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x)
    q[0] += (double)abs2(psi[idx]);
  if (!block_partials<1, false>(q, partials, counter)) return;
  __threadfence();
  __shared__ double fin1[1];
  combine_all<1, false>(partials, fin1);
  if (threadIdx.x == 0) {
    const double nrm = fin1[0] * vol;
    *norm_out = nrm;
    if (!(nrm > 0.0) || !isfinite(nrm)) {
      atomicOr(flags, 1);
      *scale_out = 1.0;
    } else {
      *scale_out = imag_scale ? 1.0 / sqrt(nrm) : 1.0;
    }
    *counter = 0u;
  }
}

// ------------------------------------------------------------ launchers
cudaError_t launch_observables(bool fp64, const obs_args& a, int blocks, int threads,
                               cudaStream_t s) {
  if (fp64)
    k_observables<double><<<blocks, threads, 0, s>>>(a);
  else
    k_observables<float><<<blocks, threads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_vortex_moments(bool fp64, const vort_args& a, int blocks, int threads,
                                  cudaStream_t s) {
  if (fp64)
    k_vort_moments<double><<<blocks, threads, 0, s>>>(a);
  else
    k_vort_moments<float><<<blocks, threads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_vortex_count(bool fp64, const vort_args& a, int blocks, int threads,
                                cudaStream_t s) {
  if (fp64)
    k_vort_count<double><<<blocks, threads, 0, s>>>(a);
  else
    k_vort_count<float><<<blocks, threads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_norm(bool fp64, const void* psi, long long nsites, double vol, int imag_scale,
                        double* partials, unsigned int* counter, double* scale_out,
                        double* norm_out, int* flags, int blocks, int threads, cudaStream_t s) {
  if (fp64)
    k_norm<double><<<blocks, threads, 0, s>>>(psi, nsites, vol, imag_scale, partials, counter,
                                              scale_out, norm_out, flags);
  else
    k_norm<float><<<blocks, threads, 0, s>>>(psi, nsites, vol, imag_scale, partials, counter,
                                             scale_out, norm_out, flags);
  return cudaGetLastError();
}

}  // namespace rotgp
