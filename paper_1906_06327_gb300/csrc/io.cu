// io.cu -- states in and out of a context: the analytic initial state of
// Eq. fun, and conversion between the ABI layout ((N+1)^d points with both
// edges, float or double) and the device layout (N^d points, index 0 edge
// stored as zero, index N edge implicit) with the pending scale applied.
#include "common.cuh"

namespace rotgp {

// Eq. fun: psi = (x + i y)/sqrt(pi d^2) exp(-(x^2+y^2)/(2 d^2)) e^{2 pi i R}
// [3D: * (pi d_z^2)^(-1/4) exp(-z^2/(2 d_z^2))]; function 0: (x + i y) -> 1.
// Evaluated in double, stored in T.  R(x_i, y_j) is the number of the point
// n = j (N_x + 1) + i of the (N_x+1)(N_y+1) plane: read from the table R
// (phase_mode 1) or drawn from SplitMix64(seed) (phase_mode 2); phase_mode 0
// leaves the phase out.
template <class T>
__global__ void k_init_analytic(cpx<T>* psi, int nx, int ny, int nz, int dim, double x0,
                                double hx, double y0, double hy, double z0, double hz,
                                int function, int phase_mode, const double* R,
                                unsigned long long seed, double d_xy, double d_z) {
  const long long n = (long long)nx * ny * nz;
  const double kPi = 3.14159265358979323846;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % nx), j = (int)((idx / nx) % ny), k = (int)(idx / ((long long)nx * ny));
    if (i == 0 || j == 0 || (dim == 3 && k == 0)) {
      psi[idx] = mk<T>(0, 0);
      continue;
    }
    const double x = x0 + i * hx, y = y0 + j * hy;
    double pr = 1.0, pi = 0.0;
    if (function) {
      pr = x;
      pi = y;
    }
    double amp = exp(-(x * x + y * y) / (2.0 * d_xy * d_xy)) / sqrt(kPi * d_xy * d_xy);
    if (dim == 3) {
      const double z = z0 + k * hz;
      amp *= pow(kPi * d_z * d_z, -0.25) * exp(-z * z / (2.0 * d_z * d_z));
    }
    double sn = 0.0, cs = 1.0;
    const unsigned long long pn = (unsigned long long)j * (nx + 1) + i;
    if (phase_mode == 1) sincos(2.0 * kPi * R[pn], &sn, &cs);
    if (phase_mode == 2) sincos(2.0 * kPi * splitmix64_unit(seed, pn), &sn, &cs);
    psi[idx] = mk<T>((T)(amp * (pr * cs - pi * sn)), (T)(amp * (pr * sn + pi * cs)));
  }
}

// ABI layout -> device layout; resets the pending scale to 1.
template <class TS, class TD>
__global__ void k_pack(const cpx<TS>* src, cpx<TD>* psi, int nx, int ny, int nz, int dim,
                       double* scale) {
  const long long n = (long long)nx * ny * nz;
  const long long px = nx + 1, py = ny + 1;
  if (blockIdx.x == 0 && threadIdx.x == 0) *scale = 1.0;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long i = idx % nx, j = (idx / nx) % ny, k = idx / ((long long)nx * ny);
    if (i == 0 || j == 0 || (dim == 3 && k == 0)) {
      psi[idx] = mk<TD>(0, 0);
      continue;
    }
    const cpx<TS> v = src[(k * py + j) * px + i];
    psi[idx] = mk<TD>((TD)v.x, (TD)v.y);
  }
}

// Device layout -> ABI layout, multiplying by the pending scale (in double)
// and writing zeros on both edges of every axis.
template <class TS, class TD>
__global__ void k_unpack(const cpx<TS>* psi, cpx<TD>* dst, int nx, int ny, int nz, int dim,
                         const double* scale) {
  const long long px = nx + 1, py = ny + 1, pz = dim == 3 ? nz + 1 : 1;
  const long long n = px * py * pz;
  const double s = *scale;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long i = idx % px, j = (idx / px) % py, k = idx / (px * py);
    const bool edge = i == 0 || i == nx || j == 0 || j == ny || (dim == 3 && (k == 0 || k == nz));
    if (edge) {
      dst[idx] = mk<TD>(0, 0);
      continue;
    }
    const cpx<TS> v = psi[(k * ny + j) * nx + i];
    dst[idx] = mk<TD>((TD)(s * (double)v.x), (TD)(s * (double)v.y));
  }
}

__global__ void k_set_scalar(double* p, double v) { *p = v; }

// The density integrated along z (the paper's reduced 2D density of a 3D
// state, Sec. 3): out[j][i] = h_z sum_k |s psi(i, j, k)|^2 on the
// (N_x+1)(N_y+1) plane, edges zero; in 2D the density itself.
template <class T>
__global__ void k_column_density(const cpx<T>* psi, double* out, int nx, int ny, int nz,
                                 double hz, const double* scale) {
  const long long px = nx + 1, n = px * (ny + 1);
  const double s2 = (*scale) * (*scale);
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long i = idx % px, j = idx / px;
    double acc = 0.0;
    if (i > 0 && i < nx && j > 0 && j < ny)
      for (int k = 0; k < nz; ++k) {
        const cpx<T> v = psi[((long long)k * ny + j) * nx + i];
        acc += (double)v.x * v.x + (double)v.y * v.y;
      }
    out[idx] = s2 * acc * hz;
  }
}

static int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 65536) b = 65536;
  if (b < 1) b = 1;
  return (int)b;
}

cudaError_t launch_init_analytic(bool fp64, void* psi, int nx, int ny, int nz, int dim,
                                 double x0, double hx, double y0, double hy, double z0,
                                 double hz, int function, int phase_mode, const double* R,
                                 unsigned long long seed, double d_xy, double d_z,
                                 cudaStream_t s) {
  const int threads = 256, blocks = grid_for((long long)nx * ny * nz, threads);
  if (fp64)
    k_init_analytic<double><<<blocks, threads, 0, s>>>(static_cast<cpx<double>*>(psi), nx, ny,
                                                       nz, dim, x0, hx, y0, hy, z0, hz,
                                                       function, phase_mode, R, seed, d_xy, d_z);
  else
    k_init_analytic<float><<<blocks, threads, 0, s>>>(static_cast<cpx<float>*>(psi), nx, ny, nz,
                                                      dim, x0, hx, y0, hy, z0, hz, function,
                                                      phase_mode, R, seed, d_xy, d_z);
  return cudaGetLastError();
}

cudaError_t launch_pack(bool fp64_store, bool fp64_src, const void* src, void* psi, int nx,
                        int ny, int nz, int dim, double* scale, cudaStream_t s) {
  const int threads = 256, blocks = grid_for((long long)nx * ny * nz, threads);
#define ROTGP_PK(TS, TD)                                                                   \
  k_pack<TS, TD><<<blocks, threads, 0, s>>>(static_cast<const cpx<TS>*>(src),             \
                                            static_cast<cpx<TD>*>(psi), nx, ny, nz, dim, scale)
  if (fp64_src) {
    if (fp64_store) ROTGP_PK(double, double); else ROTGP_PK(double, float);
  } else {
    if (fp64_store) ROTGP_PK(float, double); else ROTGP_PK(float, float);
  }
#undef ROTGP_PK
  return cudaGetLastError();
}

cudaError_t launch_unpack(bool fp64_store, bool fp64_dst, const void* psi, void* dst, int nx,
                          int ny, int nz, int dim, const double* scale, cudaStream_t s) {
  const long long pts = (long long)(nx + 1) * (ny + 1) * (dim == 3 ? nz + 1 : 1);
  const int threads = 256, blocks = grid_for(pts, threads);
#define ROTGP_UP(TS, TD)                                                                   \
  k_unpack<TS, TD><<<blocks, threads, 0, s>>>(static_cast<const cpx<TS>*>(psi),           \
                                              static_cast<cpx<TD>*>(dst), nx, ny, nz, dim, scale)
  if (fp64_store) {
    if (fp64_dst) ROTGP_UP(double, double); else ROTGP_UP(double, float);
  } else {
    if (fp64_dst) ROTGP_UP(float, double); else ROTGP_UP(float, float);
  }
#undef ROTGP_UP
  return cudaGetLastError();
}

cudaError_t launch_column_density(bool fp64, const void* psi, double* out, int nx, int ny,
                                  int nz, double hz, const double* scale, cudaStream_t s) {
  const int threads = 256, blocks = grid_for((long long)(nx + 1) * (ny + 1), threads);
  if (fp64)
    k_column_density<double><<<blocks, threads, 0, s>>>(static_cast<const cpx<double>*>(psi), out,
                                                        nx, ny, nz, hz, scale);
  else
    k_column_density<float><<<blocks, threads, 0, s>>>(static_cast<const cpx<float>*>(psi), out,
                                                       nx, ny, nz, hz, scale);
  return cudaGetLastError();
}

cudaError_t launch_set_scalar(double* p, double v, cudaStream_t s) {
  k_set_scalar<<<1, 1, 0, s>>>(p, v);
  return cudaGetLastError();
}

}  // namespace rotgp
