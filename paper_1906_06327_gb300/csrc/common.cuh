// common.cuh -- shared device types and launcher declarations of the rotgp
// CUDA library (split-step Crank-Nicolson for the rotating GP equation).
//
// Device layout of a state: N_x * N_y [* N_z] complex points, x fastest;
// index 0 along every axis is the zero Dirichlet edge and is stored (always
// 0); index N (the other edge) is implicit and never stored, so every line
// holds N points and the N-1 unknowns sit at indices 1..N-1.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rotgp {

template <class T>
struct __align__(2 * sizeof(T)) cpx {
  T x, y;
};

template <class T>
__host__ __device__ __forceinline__ cpx<T> mk(T a, T b) {
  cpx<T> r;
  r.x = a;
  r.y = b;
  return r;
}
template <class T>
__device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <class T>
__device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <class T>
__device__ __forceinline__ cpx<T> operator*(cpx<T> a, cpx<T> b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <class T>
__device__ __forceinline__ cpx<T> operator*(T s, cpx<T> a) { return mk(s * a.x, s * a.y); }
template <class T>
__device__ __forceinline__ T abs2(cpx<T> a) { return a.x * a.x + a.y * a.y; }

// One entry of a line's LU multiplier table: for the unknown at index p,
// m_p = 1 / (A0 - A- c'_{p-1}) and c'_p = A+ m_p (Thomas forward sweep).
template <class T>
struct __align__(4 * sizeof(T)) lu_entry {
  cpx<T> c, m;
};

// Coefficients of one sweep axis in one propagation mode.  For a line with
// rotation coordinate u (y_j for x lines, x_i for y lines, 0 for z lines):
//   kappa   (i Delta or Delta) / (4 h^2)
//   tau     tau_unit * u
//   A0 = 1 + 2 kappa,  A- = -kappa + tau,  A+ = -kappa - tau
//   b_p = psi_p + kappa (psi_{p+1} - 2 psi_p + psi_{p-1}) + tau (psi_{p+1} - psi_{p-1})
struct axis_coef {
  double kap_re, kap_im;
  double tau_re, tau_im;  // tau_unit
  double u0, du;          // u of line l is u0 + l du
};

// Arguments of a sweep kernel (both x and strided variants).
struct sweep_args {
  const void* in;
  void* out;
  const void* table;  // lu_entry<T>[nlines_tab][lt + 1]
  int nx, ny, nz;     // stored points per axis (nz = 1 in 2D)
  int len;            // line length N_a (stored points)
  long long stride;   // element stride along the line
  long long ncols;    // number of lines
  long long outer;    // strided: base(c) = (c / nx) * outer + c % nx
  int chunk, halo, lt, nchunks, pitch;
  axis_coef co;
  int tab_mod;        // table line index = (line index for coef) ; see kernels
  // H1 fused into the x sweep
  int h1;
  double dt;          // Delta
  double g;
  double hgam2, hnu2, hlam2;  // gamma^2/2, nu^2/2, lambda^2/2
  double x0, hx, y0, hy, z0, hz;  // coordinates: x_i = x0 + i hx etc.
  const double* scale;  // pending scale applied at load (x sweep)
  // norm epilogue of the last sweep
  int reduce;
  double vol;         // h_x h_y [h_z]
  int imag;
  double* partials;   // per-block partial sums
  unsigned int* counter;
  double* scale_out;  // new pending scale
  double* norm_out;
  int* flags;         // bit 0: non-finite norm
};

struct obs_args {
  const void* psi;
  int nx, ny, nz, dim;
  double hx, hy, hz, x0, y0, z0;
  double hgam2, hnu2, hlam2, g, omega;
  const double* scale;
  double* partials;
  unsigned int* counter;
  double* result;  // NOBS doubles
};

enum { NQ = 13 };   // partial sums per block in the observables reduction
enum { NOBS = 10 }; // norm, mu, E, mu_c, E_c, rms_x, rms_y, rms_z, rms_r, max

struct vort_args {
  const void* psi;
  int nx, ny, nz, dim, kplane;
  double hx, hy, x0, y0;
  double* partials;
  unsigned int* counter;
  double* moments;  // rx2, ry2
  int* count;
};

// ---- launchers (one per translation unit group); return cudaGetLastError
cudaError_t launch_tables(bool fp64, void* table, int nlines, int lt, const axis_coef& co,
                          cudaStream_t s);
cudaError_t launch_sweep_x(bool fp64, bool imag, const sweep_args& a, int blocks, int threads,
                           size_t smem, cudaStream_t s);
cudaError_t launch_sweep_strided(bool fp64, const sweep_args& a, int blocks, int cols_per_block,
                                 int chunks_per_block, size_t smem, cudaStream_t s);
cudaError_t launch_observables(bool fp64, const obs_args& a, int blocks, int threads,
                               cudaStream_t s);
cudaError_t launch_vortex_moments(bool fp64, const vort_args& a, int blocks, int threads,
                                  cudaStream_t s);
cudaError_t launch_vortex_count(bool fp64, const vort_args& a, int blocks, int threads,
                                cudaStream_t s);
cudaError_t launch_norm(bool fp64, const void* psi, long long nsites, double vol, int imag_scale,
                        double* partials, unsigned int* counter, double* scale_out,
                        double* norm_out, int* flags, int blocks, int threads, cudaStream_t s);
cudaError_t launch_init_analytic(bool fp64, void* psi, int nx, int ny, int nz, int dim,
                                 double x0, double hx, double y0, double hy, double z0,
                                 double hz, int function, const double* R, double d_xy,
                                 double d_z, cudaStream_t s);
cudaError_t launch_pack(bool fp64_store, bool fp64_src, const void* src, void* psi, int nx,
                        int ny, int nz, int dim, double* scale, cudaStream_t s);
cudaError_t launch_unpack(bool fp64_store, bool fp64_dst, const void* psi, void* dst, int nx,
                          int ny, int nz, int dim, const double* scale, cudaStream_t s);
cudaError_t launch_set_scalar(double* p, double v, cudaStream_t s);

}  // namespace rotgp
