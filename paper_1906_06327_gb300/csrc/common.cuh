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

struct rotgp_ctx;

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

// Folded Thomas coefficients of one unknown p of one line (Eqs. eqD.11/eq5):
// with m_p = 1/(A0 - A- c'_{p-1}) and c'_p = A+ m_p,
//   forward   d'_p = (1 + a0) psi_p + am psi_{p-1} + ap psi_{p+1} + al d'_{p-1}
//             a0 = m_p (1 - 2 kappa) - 1, am = m_p (kappa - tau), ap = m_p (kappa + tau),
//             al = -m_p A-
//   backward  x_p = d'_p + be x_{p+1},  be = -c'_p.
// The diagonal factor m_p (1 - 2 kappa) is close to 1 and is kept as its
// difference from 1: rounded to float itself it would carry an error of up
// to half an ulp of 1, the same on every interior point of every line, and
// the real-time CN map would then gain or lose ~1e-8 of norm per sweep;
// stored as the difference the rounding is that many times smaller.
// m2 = 2 m_p serves the unfolded form of the same solve (psi' = 2y - psi
// with A y = psi): d_p = m2 psi_p + al d_{p-1}, z_p = d_p + be z_{p+1},
// psi'_p = z_p - psi_p.
// Entry 0 is all zero (the Dirichlet edge); entries past the table length
// equal the last one (the Toeplitz fixed point).
template <class T>
struct __align__(16) coef5 {
  cpx<T> a0, am, ap, al, be, m2;
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

// Arguments of a streaming line-sweep kernel.  A sweep solves nlines lines
// of len points; each warp owns 32*V lines (V per lane) and one segment of
// seg_chunks chunks of C points of them.
struct stream_args {
  const void* in;
  void* out;
  const void* coef;   // coef5<T>[coefficient lines][lt + 1]
  // the same unfolded-form weights of complex float as three planes
  // [m2, al, be][lt + 1][coefficient lines] (consecutive lines contiguous)
  const float2* coefT;
  int tlines;         // coefficient lines
  int len;            // N: stored points per line
  int lt;             // index of the converged table entry
  int nseg, seg_chunks, warm, halo;
  int ring;           // slots of the per-warp chunk ring (3 or 4)
  long long nlines;
  // strided lines (y, z): line c starts at (c / nx) * outer + c % nx, step stride
  int nx, ny;
  long long stride, outer;
  int coef_mode;      // 0: one coefficient line (z); 1: c % nx (y); 2: row % ny (x)
  // H1 substep fused into the x sweep
  double dt, g, hgam2, hnu2, hlam2;
  double x0, hx, y0, hy, z0, hz;
  const double* scale;  // pending renormalisation applied as the state is read
  // banded-inverse stencil sweeps (complex float): weights [line][2B+1][2K+1]
  const void* wtab;
  int taps_k;         // K: taps reach K points either side
  int brows;          // B: rows with their own weights at each line end
  int tile_rows;      // x stencil: row pairs per warp task
  // norm reduction in the last sweep of a step
  double vol;
  int imag;
  double* partials;
  unsigned int* counter;
  double* scale_out;
  double* norm_out;
  int* flags;
};

// Random number n of the SplitMix64 stream seeded with `seed` (Steele, Lea
// and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
// the counter state seed + (n + 1) * 0x9E3779B97F4A7C15 passed through the
// generator's output mix (two xor-shift-multiply rounds and a final
// xor-shift), all modulo 2^64; its top 53 bits scaled by 2^-53 give a double
// in [0, 1).  Counter based, so every grid point draws its own number.
#ifdef __CUDACC__
__device__ __forceinline__ double splitmix64_unit(unsigned long long seed, unsigned long long n) {
  unsigned long long z = seed + (n + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}
#endif

// Tile passes (tiles_xy.cu, tiles_line.cu), complex float only.
struct tile_args {
  void* out;             // the other state buffer
  const void* wx;        // banded-inverse weights, [line][2B+1][2K+1] complex float
  const void* wy;
  const void* wz;
  int nx, ny, nz;        // stored points per axis
  int bx, by, bz;        // end rows with their own weights, per axis
  int tiles_x, tiles_y;  // xy pass: tiles per plane; line pass: patches across the lines
  int zchunk;            // xy pass: z planes per CTA
  int seg_len;           // line pass: outputs per line segment
  // H1 substep and the pending scale (xy pass)
  float dt, g, hgam2, hnu2, hlam2;
  float x0, hx, y0, hy, z0, hz;
  const double* scale;
  // norm reduction in the last pass of a step
  double vol;
  int imag;
  double* partials;
  unsigned int* counter;
  double* scale_out;
  double* norm_out;
  int* flags;            // bit 0 non-finite norm, bit 2 TMA wait timed out
};

struct obs_args {
  const void* psi;
  int nx, ny, nz, dim;
  double hx, hy, hz, x0, y0, z0;
  double hgam2, hnu2, hlam2, g, omega;
  const double* scale;
  int zchunk;          // z planes per work item (tiles of 32 x 8 columns)
  double* partials;
  unsigned int* counter;
  double* result;  // NOBS doubles
};

enum { NQ = 14 };   // partial sums per block in the observables reduction (last: a max)
enum { NOBS = 12 }; // norm, mu, E, mu_c, E_c, rms_x, rms_y, rms_z, rms_r, max, mu4, E4

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
// Launch shape of one sweep, chosen on the host.
struct sweep_shape {
  int V;          // lines per lane (1 or 2)
  int C;          // chunk length (8, 16 or 64)
  int R;          // ring slots (3 or 4)
  bool vec16;     // x sweep: 16-byte copies (even row length)
  int warps_per_block;
  long long blocks;
  size_t smem;
};

// tableT: the planes of stream_args::coefT (complex float only), or null
cudaError_t launch_tables(bool fp64, void* table, void* tableT, int nlines, int lt,
                          const axis_coef& co, cudaStream_t s);
// map: rows TMA map of the input buffer or null; omap: the swizzled
// one-row-per-lane map of the output buffer (that form only) or null
cudaError_t launch_sweep_x(bool fp64, bool imag, const stream_args& a, const sweep_shape& sh,
                           const void* map, const void* omap, cudaStream_t s);
// map / omap: one-line-per-lane TMA box maps (C points along the line) of
// the input and output buffers, or null
cudaError_t launch_sweep_strided(bool fp64, bool reduce, const stream_args& a,
                                 const sweep_shape& sh, const void* map, const void* omap,
                                 int axis, cudaStream_t s);
// blocks of the one-line-per-lane strided form with one warp per block
long long strided1_blocks(long long nlines, int nx, int nseg);
// Exact partition-method line solve of one sweep (hybrid.cu): axis 0 (x,
// with H1 and the pending scale fused in), 1 (y) or 2 (z); clusters of cs
// CTAs, each a tile of 16 lines x pc positions, lsub positions per thread;
// reduce: the norm epilogue of the last sweep of a step.
cudaError_t launch_line_hybrid(bool fp64, bool imag, bool reduce, int axis, const stream_args& a,
                               int cs, int pc, int lsub, cudaStream_t s);
// tile shape for lines of N points within max_bytes of shared memory per CTA
bool hybrid_shape(int N, int axis, bool fp64, size_t max_bytes, int* cs, int* pc, int* lsub);
// the tile of a given cluster size; returns its shared-memory bytes
size_t hybrid_tile(int N, int axis, bool fp64, int cs, int* pc, int* lsub);
// line groups (tiles of 16 lines) of an axis
long long hybrid_groups(int axis, long long nlines, int nx);
// clusters of that shape resident at once on the current device (0: none)
int hybrid_max_clusters(bool fp64, int axis, int cs, int pc);
// the host step of the last hybrid launch on this thread (error messages)
const char* hybrid_launch_stage();
size_t sweep_smem_per_warp(bool fp64, bool x_sweep, int V, int C, int R);
// Launch with programmatic stream serialization: the kernel's blocks may be
// scheduled while the previous kernel in the stream finishes; the kernel
// itself waits (griddep_wait) for the previous kernel's writes before it
// touches global memory.
template <class... P, class... A>
cudaError_t launch_programmatic(void (*fn)(P...), unsigned blocks, unsigned threads, size_t smem,
                                cudaStream_t s, A&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fn, static_cast<A&&>(args)...);
}
#ifdef __CUDACC__
// the kernel side: allow the next kernel's blocks to launch; wait for the
// previous kernel's completion and memory (a no-op without a dependency)
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
#endif

// persistent grid of a warp-per-unit kernel (sweep_s.cu)
cudaError_t resident_grid(const void* fn, long long units, size_t smem_per_warp, size_t extra,
                          int max_warps, int* warps, unsigned* blocks);
// banded-inverse stencil form of the complex-float sweeps (stencil.cu)
cudaError_t launch_stencil_tables(void* wtab, int nlines, int K, int B, int m,
                                  const axis_coef& co, cudaStream_t s);
cudaError_t launch_stencil_x(bool imag, const stream_args& a, long long warps, cudaStream_t s);
inline bool stencil_k_built(int K) { return K == 4 || K == 6 || K == 8; }
// Tile passes.  xy_tile_geometry gives the host the xy tile of stencil
// reach K (TX x TY outputs, R rows and WX points per staged row);
// line_rows the transverse rows of a line-pass CTA (32 x line_rows lines);
// launch_* return cudaErrorInvalidValue for an unbuilt K (tile_k_built).
bool tile_k_built(int K);
unsigned xy_pass_smem(int K);  // dynamic shared memory of one xy-pass CTA
int xy_pass_ctas_per_sm(int K, bool imag, bool reduce);  // resident CTAs per SM
// x sweep alone in stencil form (tiles of 32 rows x 64 points): map with box
// {2 (64 + 2K + 2), 32, 1}
int x_pass_ctas_per_sm(int K);
cudaError_t launch_x_pass(bool imag, int K, const void* map, const tile_args& a, unsigned blocks,
                          cudaStream_t s);
void xy_tile_geometry(int K, int* TX, int* TY, int* R, int* WX);
int line_rows();
cudaError_t launch_xy_pass(bool imag, bool reduce, int K, const void* map, const tile_args& a,
                           unsigned blocks, cudaStream_t s);
cudaError_t launch_line_pass(int axis, bool reduce, int K, const void* map, const tile_args& a,
                             unsigned blocks, cudaStream_t s);
// Is (precision, V, C) one of the instantiated sweep kernels?
inline bool sweep_shape_built(bool fp64, int V, int C) {
  if (fp64) return V == 1 && (C == 16 || C == 64);
  return (V == 2 && (C == 8 || C == 16)) || (V == 1 && (C == 16 || C == 64));
}
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
                                 double hz, int function, int phase_mode, const double* R,
                                 unsigned long long seed, double d_xy, double d_z,
                                 cudaStream_t s);
cudaError_t launch_pack(bool fp64_store, bool fp64_src, const void* src, void* psi, int nx,
                        int ny, int nz, int dim, double* scale, cudaStream_t s);
cudaError_t launch_unpack(bool fp64_store, bool fp64_dst, const void* psi, void* dst, int nx,
                          int ny, int nz, int dim, const double* scale, cudaStream_t s);
cudaError_t launch_set_scalar(double* p, double v, cudaStream_t s);
cudaError_t launch_column_density(bool fp64, const void* psi, double* out, int nx, int ny,
                                  int nz, double hz, const double* scale, cudaStream_t s);

// Context bookkeeping for graph replay (batch.cu): which ping-pong buffer
// holds the state, and the step counter.
int ctx_buffer(const rotgp_ctx* c);
void ctx_set_buffer(rotgp_ctx* c, int cur);
long long ctx_steps(const rotgp_ctx* c);
long long ctx_plan_version(const rotgp_ctx* c);
void ctx_add_steps(rotgp_ctx* c, long long n);
// What a multi-instance kernel needs of one 2D context (batch.cu).
struct ctx_view {
  int dim, fp64, nx, ny, lt, cur;
  void* psi[2];
  const void* table[2][2];  // [axis][mode] coef5 tables
  double* scale;            // pending renormalisation (device)
  double* norm;             // last norm (device)
  int* flags;               // device flags word
  double dt, g, gamma, nu, x0, y0, hx, hy, vol;
};
void ctx_get_view(const rotgp_ctx* c, ctx_view* v);
// The persistent multi-instance step (batch_kernel.cu): device scratch owned
// by a batch, a fit check, one cooperative launch of nsteps split steps of the
// active instances, and the launch's flags word (bit 3: barrier timeout).
struct batch_dev;
void batch_kernel_free(batch_dev* d);
bool batch_kernel_fits(const ctx_view* v, int count, size_t smem_limit, const char** why);
cudaError_t batch_kernel_run(batch_dev** d, const ctx_view* v, int count, const int* active,
                             int nact, long long nsteps, bool imag, cudaStream_t s);
cudaError_t batch_kernel_flags(batch_dev* d, cudaStream_t s, int* flags);

}  // namespace rotgp
