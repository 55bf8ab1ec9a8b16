// sweeps.cu -- the Crank-Nicolson line sweeps of one split step (Sec. 2):
// H1 (Eq. eq1) fused into the x sweep (H2, Eqs. eqD.9/eqD.11/eq5), the y
// sweep (H3, "performed similarly") and the z sweep (3D), plus the
// per-line LU multiplier tables they read.
//
// Line solver.  Every line's tridiagonal matrix is constant along the line
// (A-, A0, A+ depend only on the line's rotation coordinate) and strictly
// diagonally dominant, so the influence of the right-hand side decays
// geometrically along the Thomas recurrences: a forward carry is multiplied
// by |A- m*| and a backward carry by |c*| per point.  A line of N points is
// therefore cut into chunks of C output points, and each chunk re-solves
// H extra points on either side, starting its forward sweep from d' = 0 and
// its back substitution from x = d'; H is chosen on the host so that
// decay^H is far below the rounding of the working precision.  The LU
// multipliers m_p, c'_p are exact table entries for p < L (L = table_len)
// and the converged Toeplitz values beyond.  This gives N/C independent
// work items per line with no grid-wide synchronisation, at the cost of
// (C + 2H)/C recurrence work; the loaded halo points come from L2.
//
// Memory: every sweep reads the state once and writes it once (ping-pong
// buffers, so that halos read by one chunk are never overwritten by
// another).  x lines are contiguous: a warp stages 32 rows x (C + 2H + 2)
// points in shared memory with cp.async (coalesced along x), then each lane
// runs the recurrences of one row from shared memory (odd row pitch: no bank
// conflicts), and the warp stores the C results coalesced.  y and z lines
// are strided: lane = adjacent column, so each cp.async of a warp covers
// 32 consecutive points; each thread keeps its column in a [point][lane]
// shared-memory slab and stores its results straight to global memory.
#include "common.cuh"

namespace rotgp {

// --------------------------------------------------------------- helpers
__device__ __forceinline__ void cp_async_elem(cpx<float>* dst, const cpx<float>* src) {
  unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_elem(cpx<double>* dst, const cpx<double>* src) {
  unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

__device__ __forceinline__ float exp_t(float v) { return expf(v); }
__device__ __forceinline__ double exp_t(double v) { return exp(v); }
__device__ __forceinline__ void sincos_t(float v, float* s, float* c) { sincosf(v, s, c); }
__device__ __forceinline__ void sincos_t(double v, double* s, double* c) { sincos(v, s, c); }

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
__device__ void norm_epilogue(double v, const sweep_args& a) {
  __shared__ double ws[32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned nblocks = gridDim.x * gridDim.y;
  const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
  v = warp_sum(v);
  if (lane == 0) ws[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int w = 0; w < nw; ++w) s += ws[w];
    a.partials[bid] = s;
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

// --------------------------------------------------------------- tables
// Thomas forward multipliers of one line (Eq. eq5 coefficients, see
// axis_coef): m_1 = 1/A0, c'_1 = A+ m_1, m_p = 1/(A0 - A- c'_{p-1}),
// c'_p = A+ m_p, for p = 1..lt, computed in double.
template <class T>
__global__ void k_tables(lu_entry<T>* tab, int nlines, int lt, axis_coef co) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nlines) return;
  const double u = co.u0 + (double)l * co.du;
  const double kr = co.kap_re, ki = co.kap_im;
  const double tr = co.tau_re * u, ti = co.tau_im * u;
  const double a0r = 1.0 + 2.0 * kr, a0i = 2.0 * ki;
  const double amr = -kr + tr, ami = -ki + ti;
  const double apr = -kr - tr, api = -ki - ti;
  lu_entry<T>* t = tab + (size_t)l * (lt + 1);
  t[0].c = mk<T>(0, 0);
  t[0].m = mk<T>(0, 0);
  double cr = 0.0, ci = 0.0;
  for (int p = 1; p <= lt; ++p) {
    const double dr = a0r - (amr * cr - ami * ci);
    const double di = a0i - (amr * ci + ami * cr);
    const double inv = 1.0 / (dr * dr + di * di);
    const double mr = dr * inv, mi = -di * inv;
    const double ncr = apr * mr - api * mi, nci = apr * mi + api * mr;
    t[p].c = mk<T>((T)ncr, (T)nci);
    t[p].m = mk<T>((T)mr, (T)mi);
    cr = ncr;
    ci = nci;
  }
}

// --------------------------------------------------------------- x sweep
template <class T, bool IMAG, bool H1>
__global__ void __launch_bounds__(128) k_sweep_x(const sweep_args a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using C = cpx<T>;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  const int H = a.halo, CH = a.chunk, W = CH + 2 * H + 2, P = a.pitch;
  C* tile = reinterpret_cast<C*>(smem_raw) + (size_t)warp * 32 * P;
  const long long rows = (long long)a.ny * a.nz;
  const long long tile_id = (long long)blockIdx.x * nwarps + warp;
  const long long rg = tile_id / a.nchunks;
  const int q = (int)(tile_id - rg * a.nchunks);
  const long long row0 = rg * 32;
  if (row0 >= rows) return;  // whole warp; no block-level barrier below
  const int nx = a.nx;
  const int x0 = q * CH;
  const int ps = x0 - H - 1;  // position of tile element 0
  const C* in = static_cast<const C*>(a.in);
  C* out = static_cast<C*>(a.out);
  const int nr = (int)min(32LL, rows - row0);

  for (int r = 0; r < nr; ++r) {
    const C* src = in + (row0 + r) * nx;
    for (int e = lane; e < W; e += 32) {
      const int p = ps + e;
      if (p >= 0 && p < nx)
        cp_async_elem(&tile[r * P + e], &src[p]);
      else
        tile[r * P + e] = mk<T>(0, 0);
    }
  }
  cp_async_wait_all();
  __syncwarp();

  if (lane < nr) {
    const long long row = row0 + lane;
    const int j = (int)(row % a.ny);
    const int k = (int)(row / a.ny);
    const T u = (T)(a.co.u0 + (double)j * a.co.du);
    const C kap = mk<T>((T)a.co.kap_re, (T)a.co.kap_im);
    const C tau = mk<T>((T)a.co.tau_re * u, (T)a.co.tau_im * u);
    const C am = tau - kap;
    const lu_entry<T>* tab = static_cast<const lu_entry<T>*>(a.table) + (size_t)j * (a.lt + 1);
    const lu_entry<T> inf = tab[a.lt];
    T s = 1, vyz = 0, hg2 = 0, g = 0, dt = 0, xs = 0, hx = 0;
    if (H1) {
      const T y = (T)(a.y0 + (double)j * a.hy);
      const T z = (T)(a.z0 + (double)k * a.hz);
      vyz = (T)a.hnu2 * y * y + (T)a.hlam2 * z * z;
      hg2 = (T)a.hgam2;
      g = (T)a.g;
      dt = (T)a.dt;
      s = (T)(*a.scale);
      xs = (T)a.x0;
      hx = (T)a.hx;
    }
    C* t = tile + lane * P;
    // psi at tile element e, after the pending scale and the H1 substep;
    // zero outside the unknowns 1..nx-1
    auto fetch = [&](int e) -> C {
      const int p = ps + e;
      C v = t[e];
      if (p < 1 || p >= nx) return mk<T>(0, 0);
      if (H1) {
        v = s * v;
        const T x = xs + (T)p * hx;
        const T en = hg2 * x * x + vyz + g * abs2(v);
        if (IMAG) {
          v = exp_t(-dt * en) * v;
        } else {
          T sn, cs;
          sincos_t(dt * en, &sn, &cs);
          v = v * mk<T>(cs, -sn);
        }
      }
      return v;
    };
    C wm = fetch(0), w0 = fetch(1), d = mk<T>(0, 0);
    for (int e = 1; e <= W - 2; ++e) {
      const int p = ps + e;
      const C wp = fetch(e + 1);
      if (p >= 1 && p < nx) {
        const C b = w0 + kap * (wp - (T)2 * w0 + wm) + tau * (wp - wm);
        const C m = p < a.lt ? tab[p].m : inf.m;
        d = (b - am * d) * m;
      } else {
        d = mk<T>(0, 0);
      }
      t[e] = d;
      wm = w0;
      w0 = wp;
    }
    C xn = mk<T>(0, 0);
    for (int e = W - 2; e >= H + 1; --e) {
      const int p = ps + e;
      C xv = mk<T>(0, 0);
      if (p >= 1 && p < nx) {
        const C c = p < a.lt ? tab[p].c : inf.c;
        xv = t[e] - c * xn;
      }
      t[e] = xv;
      xn = xv;
    }
  }
  __syncwarp();
  for (int r = 0; r < nr; ++r) {
    C* dst = out + (row0 + r) * nx;
    for (int e = lane; e < CH; e += 32) {
      const int p = x0 + e;
      if (p < nx) dst[p] = tile[r * P + H + 1 + e];
    }
  }
}

// --------------------------------------------------------------- y / z sweeps
template <class T>
__global__ void __launch_bounds__(256) k_sweep_strided(const sweep_args a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using C = cpx<T>;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int H = a.halo, CH = a.chunk, W = CH + 2 * H + 2;
  C* t = reinterpret_cast<C*>(smem_raw) + (size_t)w * W * 32 + lane;
  const long long c = (long long)blockIdx.x * 32 + lane;
  const int q = blockIdx.y * (blockDim.x >> 5) + w;
  const bool active = c < a.ncols && q < a.nchunks;
  const int N = a.len;
  const int x0 = q * CH, ps = x0 - H - 1;
  acc_t<T> acc;
  if (active) {
    const long long base = (c / a.nx) * a.outer + (c % a.nx);
    const C* in = static_cast<const C*>(a.in) + base;
    C* out = static_cast<C*>(a.out) + base;
    for (int e = 0; e < W; ++e) {
      const int p = ps + e;
      if (p >= 0 && p < N)
        cp_async_elem(&t[e * 32], &in[(long long)p * a.stride]);
      else
        t[e * 32] = mk<T>(0, 0);
    }
    cp_async_wait_all();  // each thread reads only its own column

    const int line = a.tab_mod ? (int)(c % a.nx) : 0;
    const T u = (T)(a.co.u0 + (double)line * a.co.du);
    const C kap = mk<T>((T)a.co.kap_re, (T)a.co.kap_im);
    const C tau = mk<T>((T)a.co.tau_re * u, (T)a.co.tau_im * u);
    const C am = tau - kap;
    const lu_entry<T>* tab = static_cast<const lu_entry<T>*>(a.table) + (size_t)line * (a.lt + 1);
    const lu_entry<T> inf = tab[a.lt];
    auto fetch = [&](int e) -> C {
      const int p = ps + e;
      return (p < 1 || p >= N) ? mk<T>(0, 0) : t[e * 32];
    };
    C wm = fetch(0), w0 = fetch(1), d = mk<T>(0, 0);
    for (int e = 1; e <= W - 2; ++e) {
      const int p = ps + e;
      const C wp = fetch(e + 1);
      if (p >= 1 && p < N) {
        const C b = w0 + kap * (wp - (T)2 * w0 + wm) + tau * (wp - wm);
        const C m = p < a.lt ? tab[p].m : inf.m;
        d = (b - am * d) * m;
      } else {
        d = mk<T>(0, 0);
      }
      t[e * 32] = d;
      wm = w0;
      w0 = wp;
    }
    C xn = mk<T>(0, 0);
    for (int e = W - 2; e >= H + 1; --e) {
      const int p = ps + e;
      C xv = mk<T>(0, 0);
      if (p >= 1 && p < N) {
        const C cc = p < a.lt ? tab[p].c : inf.c;
        xv = t[e * 32] - cc * xn;
      }
      xn = xv;
      if (e <= H + CH && p < N) {
        out[(long long)p * a.stride] = xv;
        acc.add(abs2(xv));
      }
    }
  }
  if (a.reduce) norm_epilogue(acc.value(), a);
}

// --------------------------------------------------------------- launchers
cudaError_t launch_tables(bool fp64, void* table, int nlines, int lt, const axis_coef& co,
                          cudaStream_t s) {
  const int threads = 128, blocks = (nlines + threads - 1) / threads;
  if (fp64)
    k_tables<double><<<blocks, threads, 0, s>>>(static_cast<lu_entry<double>*>(table), nlines,
                                                lt, co);
  else
    k_tables<float><<<blocks, threads, 0, s>>>(static_cast<lu_entry<float>*>(table), nlines,
                                               lt, co);
  return cudaGetLastError();
}

// Allow each kernel the device's opt-in shared memory (minus its static
// shared memory) once per process.
static cudaError_t allow_smem(const void* fn, bool* done) {
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

cudaError_t launch_sweep_x(bool fp64, bool imag, const sweep_args& a, int blocks, int threads,
                           size_t smem, cudaStream_t s) {
#define ROTGP_LX(T, IM, HH)                                                    \
  do {                                                                         \
    static bool done = false;                                                  \
    cudaError_t e_ = allow_smem((const void*)k_sweep_x<T, IM, HH>, &done);     \
    if (e_ != cudaSuccess) return e_;                                          \
    k_sweep_x<T, IM, HH><<<blocks, threads, smem, s>>>(a);                     \
  } while (0)
  if (fp64) {
    if (a.h1) {
      if (imag) ROTGP_LX(double, true, true); else ROTGP_LX(double, false, true);
    } else {
      ROTGP_LX(double, true, false);
    }
  } else {
    if (a.h1) {
      if (imag) ROTGP_LX(float, true, true); else ROTGP_LX(float, false, true);
    } else {
      ROTGP_LX(float, true, false);
    }
  }
#undef ROTGP_LX
  return cudaGetLastError();
}

cudaError_t launch_sweep_strided(bool fp64, const sweep_args& a, int blocks, int cols_per_block,
                                 int chunks_per_block, size_t smem, cudaStream_t s) {
  (void)cols_per_block;
  dim3 grid((unsigned)blocks, (unsigned)((a.nchunks + chunks_per_block - 1) / chunks_per_block));
  const int threads = 32 * chunks_per_block;
  if (fp64) {
    static bool done = false;
    cudaError_t e = allow_smem((const void*)k_sweep_strided<double>, &done);
    if (e != cudaSuccess) return e;
    k_sweep_strided<double><<<grid, threads, smem, s>>>(a);
  } else {
    static bool done = false;
    cudaError_t e = allow_smem((const void*)k_sweep_strided<float>, &done);
    if (e != cudaSuccess) return e;
    k_sweep_strided<float><<<grid, threads, smem, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace rotgp
