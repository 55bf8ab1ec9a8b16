// noalloc.cu -- observables of a caller-owned device wave function with no
// device-memory allocation at all.
//
// Some callers cannot call cudaMalloc: code whose device memory is owned by
// another allocator (a framework's caching allocator that must stay the only
// owner of the device heap), code running under a fixed memory budget
// reserved up front, and monitoring loops that must not add the implicit
// device synchronisation that cudaMalloc/cudaFree can bring.  For them this
// file offers rotgp_observables_noalloc: the same reduction as
// rotgp_observables, reading the wave function in the ABI layout straight
// from the caller's device buffer, with its scratch (per-block partial sums,
// result slots and the last-block ticket) in one file-scope device array.
//
// That array is part of the library image: every GPU that loads the library
// holds it (about 448 KiB) until the process exits.  All calls share it and it
// keeps the last call's contents; the ticket counter is cleared by every
// call before its kernel runs.  Calls whose work overlaps on the GPU (for
// example on two streams at once) race on the array and must be ordered by
// the caller.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/rotgp.h"
#include "common.cuh"

namespace rotgp {
void set_thread_error(const char* msg);  // rotgp.cu: message for rotgp_last_error(NULL)
}

namespace {

using namespace rotgp;

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 4096;               // per-block partial-sum slots
constexpr long long kPointsPerBlock = 8192;    // grid points one block reduces
constexpr long long kMaxPoints = kMaxBlocks * kPointsPerBlock;  // 33,554,432
constexpr int kResult = kMaxBlocks * NQ;       // offset of the NOBS results
constexpr int kTicket = kResult + NOBS;        // offset of the ticket counter
constexpr int kScratchDoubles = kTicket + 2;   // 57,358 doubles, about 448 KiB

}  // namespace

// The scratch.  In host code this name is only a handle for
// cudaGetSymbolAddress, never a device address.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

namespace {

__device__ __forceinline__ double nsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double nmax(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// The observables reduction over a wave function of (N_x+1)(N_y+1)[(N_z+1)]
// points, edges included, x fastest (the ABI layout).  Edge points are taken
// as zero.  Per interior site it accumulates the same sums as the context's
// reduction (reduce.cu): |psi|^2, psi_R^2, psi_I^2, the real-part energy
// terms for psi and for the state rotated by -i, the complex-form terms, the
// second moments and the maximum density; block b reduces points
// [b * 8192, (b + 1) * 8192) and the last block combines the partials in
// block order.
template <class T>
__global__ void __launch_bounds__(kThreads) k_observables_noalloc(
    const cpx<T>* psi, int nx, int ny, int nz, int dim, double hx, double hy, double hz,
    double x0, double y0, double z0, double hgam2, double hnu2, double hlam2, double gd,
    double omega, double* scratch) {
  using C = cpx<T>;
  const long long px = nx + 1, py = ny + 1, pz = dim == 3 ? nz + 1 : 1;
  const long long npts = px * py * pz;
  const T ihx2 = (T)(1.0 / (hx * hx)), ihy2 = (T)(1.0 / (hy * hy));
  const T ihz2 = dim == 3 ? (T)(1.0 / (hz * hz)) : (T)0;
  const T i2hx = (T)(0.5 / hx), i2hy = (T)(0.5 / hy);
  const T om = (T)omega, g = (T)gd;
  auto edge = [&](long long i, long long j, long long k) {
    return i <= 0 || i >= nx || j <= 0 || j >= ny || (dim == 3 && (k <= 0 || k >= nz));
  };
  auto at = [&](long long i, long long j, long long k) -> C {
    return edge(i, j, k) ? mk<T>(0, 0) : psi[(k * py + j) * px + i];
  };
  double q[NQ];
#pragma unroll
  for (int v = 0; v < NQ; ++v) q[v] = 0.0;
  const long long lo = (long long)blockIdx.x * kPointsPerBlock;
  const long long hi = min(npts, lo + kPointsPerBlock);
  for (long long idx = lo + threadIdx.x; idx < hi; idx += kThreads) {
    const long long i = idx % px, j = (idx / px) % py, k = idx / (px * py);
    if (edge(i, j, k)) continue;
    const T x = (T)(x0 + (double)i * hx), y = (T)(y0 + (double)j * hy);
    const T z = dim == 3 ? (T)(z0 + (double)k * hz) : (T)0;
    const T V = (T)hgam2 * x * x + (T)hnu2 * y * y + (T)hlam2 * z * z;
    const C c = psi[idx];
    const C xp = at(i + 1, j, k), xm = at(i - 1, j, k);
    const C yp = at(i, j + 1, k), ym = at(i, j - 1, k);
    C lap = ihx2 * (xp + xm - (T)2 * c) + ihy2 * (yp + ym - (T)2 * c);
    if (dim == 3) lap = lap + ihz2 * (at(i, j, k + 1) + at(i, j, k - 1) - (T)2 * c);
    const C dx = i2hx * (xp - xm), dy = i2hy * (yp - ym);
    const T re = c.x, im = c.y, dens = re * re + im * im;
    const T hr = (T)-0.5 * lap.x + V * re + om * (y * dx.y - x * dy.y);
    const T hi_ = (T)-0.5 * lap.y + V * im + om * (-(y * dx.x) + x * dy.x);
    const C lz = y * dx - x * dy;
    const C hlin = mk<T>((T)-0.5 * lap.x + V * c.x + om * lz.y, (T)-0.5 * lap.y + V * c.y - om * lz.x);
    q[0] += (double)dens;
    q[1] += (double)(re * re);
    q[2] += (double)(im * im);
    q[3] += (double)(re * hr);
    q[4] += (double)(g * dens * re * re);
    q[5] += (double)(im * hi_);
    q[6] += (double)(g * dens * im * im);
    q[7] += (double)(re * hlin.x + im * hlin.y);
    q[8] += (double)(g * dens * dens);
    q[9] += (double)(x * x * dens);
    q[10] += (double)(y * y * dens);
    q[11] += (double)(z * z * dens);
    {
      // fourth-order central differences (points beyond the grid are zero)
      const C xp2 = at(i + 2, j, k), xm2 = at(i - 2, j, k);
      const C yp2 = at(i, j + 2, k), ym2 = at(i, j - 2, k);
      C lap4 = (ihx2 / (T)12) * ((T)16 * (xp + xm) - xp2 - xm2 - (T)30 * c) +
               (ihy2 / (T)12) * ((T)16 * (yp + ym) - yp2 - ym2 - (T)30 * c);
      if (dim == 3)
        lap4 = lap4 + (ihz2 / (T)12) * ((T)16 * (at(i, j, k + 1) + at(i, j, k - 1)) -
                                        at(i, j, k + 2) - at(i, j, k - 2) - (T)30 * c);
      const C dx4 = (i2hx / (T)6) * ((T)8 * (xp - xm) - xp2 + xm2);
      const C dy4 = (i2hy / (T)6) * ((T)8 * (yp - ym) - yp2 + ym2);
      const C lz4 = y * dx4 - x * dy4;
      q[12] += (double)(re * ((T)-0.5 * lap4.x + V * c.x + om * lz4.y) +
                        im * ((T)-0.5 * lap4.y + V * c.y - om * lz4.x));
    }
    q[13] = fmax(q[13], (double)dens);
  }
  __shared__ double ws[kThreads / 32][NQ];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < NQ; ++v) {
    const double t = v == NQ - 1 ? nmax(q[v]) : nsum(q[v]);
    if (lane == 0) ws[warp][v] = t;
  }
  __syncthreads();
  double* partials = scratch;
  double* result = scratch + kResult;
  unsigned* ticket = reinterpret_cast<unsigned*>(scratch + kTicket);
  if (threadIdx.x < NQ) {
    double s = 0;
    for (int w = 0; w < kThreads / 32; ++w)
      s = threadIdx.x == NQ - 1 ? fmax(s, ws[w][threadIdx.x]) : s + ws[w][threadIdx.x];
    partials[(size_t)blockIdx.x * NQ + threadIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  // every thread sums a fixed strided subset of the blocks, then the warps
  // and the block combine in a fixed order (deterministic)
  __shared__ double fin[NQ];
#pragma unroll
  for (int v = 0; v < NQ; ++v) {
    double s = 0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += kThreads) {
      const double x = __ldcg(&partials[(size_t)b * NQ + v]);
      s = v == NQ - 1 ? fmax(s, x) : s + x;
    }
    s = v == NQ - 1 ? nmax(s) : nsum(s);
    if (lane == 0) ws[warp][v] = s;
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    double s = 0;
    for (int w = 0; w < kThreads / 32; ++w)
      s = threadIdx.x == NQ - 1 ? fmax(s, ws[w][threadIdx.x]) : s + ws[w][threadIdx.x];
    fin[threadIdx.x] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double vol = hx * hy * (dim == 3 ? hz : 1.0);
    const bool rot = fin[1] < 1e-3 * fin[0];
    const double lin = rot ? fin[5] : fin[3], nl = rot ? fin[6] : fin[4];
    const double den = rot ? fin[2] : fin[1];
    result[0] = vol * fin[0];
    result[1] = (lin + nl) / den;
    result[2] = (lin + 0.5 * nl) / den;
    result[3] = (fin[7] + fin[8]) / fin[0];
    result[4] = (fin[7] + 0.5 * fin[8]) / fin[0];
    result[5] = sqrt(fin[9] / fin[0]);
    result[6] = sqrt(fin[10] / fin[0]);
    result[7] = dim == 3 ? sqrt(fin[11] / fin[0]) : 0.0;
    result[8] = sqrt((fin[9] + fin[10] + fin[11]) / fin[0]);
    result[9] = fin[13];
    result[10] = (fin[12] + fin[8]) / fin[0];
    result[11] = (fin[12] + 0.5 * fin[8]) / fin[0];
    *ticket = 0u;
  }
}

std::mutex g_setup_mutex;
double* g_scratch_ptr[256] = {nullptr};

int fail_msg(int code, const char* fmt, long long a = 0, long long b = 0) {
  char buf[256];
  std::snprintf(buf, sizeof buf, fmt, a, b);
  set_thread_error(buf);
  return code;
}

}  // namespace

extern "C" int rotgp_observables_noalloc(const rotgp_grid* grid, const rotgp_phys* phys,
                                         int precision, const void* psi_device, void* stream,
                                         rotgp_obs* out) {
  if (!grid || !phys || !psi_device || !out)
    return fail_msg(ROTGP_EINVAL, "rotgp_observables_noalloc: null argument");
  if (grid->dim != 2 && grid->dim != 3)
    return fail_msg(ROTGP_EINVAL, "rotgp_observables_noalloc: dim must be 2 or 3");
  for (int a = 0; a < grid->dim; ++a)
    if (grid->n[a] < 4 || !(grid->h[a] > 0))
      return fail_msg(ROTGP_EINVAL, "rotgp_observables_noalloc: n >= 4 and h > 0 required");
  if (precision != ROTGP_FP32 && precision != ROTGP_FP64)
    return fail_msg(ROTGP_EINVAL, "rotgp_observables_noalloc: bad precision");
  long long pts = 1;
  for (int a = 0; a < grid->dim; ++a) pts *= (long long)grid->n[a] + 1;
  if (pts > kMaxPoints)
    return fail_msg(ROTGP_EINVAL,
                    "rotgp_observables_noalloc: the grid has %lld points; without allocation "
                    "at most %lld fit the fixed scratch",
                    pts, kMaxPoints);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 256)
    return fail_msg(ROTGP_ECUDA, "rotgp_observables_noalloc: no current CUDA device");
  double* scratch = nullptr;
  {
    // once per device, with that device current: the scratch's device address
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) {
        set_thread_error(cudaGetErrorString(e));
        return ROTGP_ECUDA;
      }
      g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_scratch_ptr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the last-block ticket must start at zero
  e = cudaMemsetAsync(scratch + kTicket, 0, sizeof(double), s);
  if (e != cudaSuccess) {
    set_thread_error(cudaGetErrorString(e));
    return ROTGP_ECUDA;
  }
  const int nz = grid->dim == 3 ? grid->n[2] : 1;
  const int blocks = (int)((pts + kPointsPerBlock - 1) / kPointsPerBlock);
  const double x0 = -0.5 * grid->n[0] * grid->h[0], y0 = -0.5 * grid->n[1] * grid->h[1];
  const double z0 = grid->dim == 3 ? -0.5 * grid->n[2] * grid->h[2] : 0.0;
  const double hz = grid->dim == 3 ? grid->h[2] : 0.0;
  const double hl2 = grid->dim == 3 ? 0.5 * phys->lambda * phys->lambda : 0.0;
  if (precision == ROTGP_FP64)
    k_observables_noalloc<double><<<blocks, kThreads, 0, s>>>(
        static_cast<const cpx<double>*>(psi_device), grid->n[0], grid->n[1], nz, grid->dim,
        grid->h[0], grid->h[1], hz, x0, y0, z0, 0.5 * phys->gamma * phys->gamma,
        0.5 * phys->nu * phys->nu, hl2, phys->g, phys->omega, scratch);
  else
    k_observables_noalloc<float><<<blocks, kThreads, 0, s>>>(
        static_cast<const cpx<float>*>(psi_device), grid->n[0], grid->n[1], nz, grid->dim,
        grid->h[0], grid->h[1], hz, x0, y0, z0, 0.5 * phys->gamma * phys->gamma,
        0.5 * phys->nu * phys->nu, hl2, phys->g, phys->omega, scratch);
  e = cudaGetLastError();
  double res[NOBS];
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(res, scratch + kResult, sizeof res, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_thread_error(cudaGetErrorString(e));
    return ROTGP_ECUDA;
  }
  std::memset(out, 0, sizeof *out);
  out->norm = res[0];
  out->mu = res[1];
  out->energy = res[2];
  out->mu_c = res[3];
  out->energy_c = res[4];
  out->rms_x = res[5];
  out->rms_y = res[6];
  out->rms_z = res[7];
  out->rms_r = res[8];
  out->max_density = res[9];
  out->mu4 = res[10];
  out->energy4 = res[11];
  out->step = 0;
  out->vortices = -1;
  out->flags = phys->omega >= (phys->gamma < phys->nu ? phys->gamma : phys->nu) ? 1 : 0;
  return ROTGP_OK;
}
