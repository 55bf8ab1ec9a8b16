/*
 * rotgp_oracle.c -- plain, slow FP64 CPU oracle of the split-step
 * Crank-Nicolson (CN) scheme for the rotating Gross-Pitaevskii equation of
 * Kumar, Loncar, Muruganandam, Adhikari and Balaz, "C and Fortran OpenMP
 * programs for rotating Bose-Einstein condensates" (Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness authority that the
 * CUDA path is compared against.  Only tests/, the smoke check and the CPU
 * baseline leg of bench.py may load it.  It shares no code with the CUDA
 * library and must never be used as a fallback for it.
 *
 * Everything is double precision complex (C99 <complex.h>), single threaded,
 * and follows the paper's notation and order of operations:
 *
 *   grid      x_i = -N_x h_x / 2 + i h_x, i = 0..N_x (Sec. 2, below Eq. eqD.9),
 *             likewise y_j, z_k.  The arrays hold all (N+1)^d points, edges
 *             included, x fastest: psi[(k (N_y+1) + j)(N_x+1) + i].
 *             psi = 0 on every edge (Dirichlet; the paper's "proper boundary
 *             conditions").
 *   one step  H1 (analytic pointwise, Eq. eq1), then H2 (CN along x, Eq. eq2,
 *             discretised as Eq. eqD.9 with the tridiagonal coefficients of
 *             Eqs. eqD.11/eq5), then H3 (CN along y, Eq. eq3, "performed
 *             similarly"), then in 3D a plain CN sweep along z.  Imaginary time
 *             is the substitution i*Delta -> Delta in the same formulas, and is
 *             followed by renormalisation to unit norm.
 *
 * Parity pins: dense-LU line solves, closed-form Toeplitz eigenpairs, a
 * dense-matrix brute-force step on tiny grids built from the operators of
 * Eqs. eq1-eq3, harmonic ground energies, the 2 - Omega one-vortex energy,
 * real-time norm conservation and the Omega = 0 reduction (tests/).
 * The real-part energy formula at g != 0 beyond these is "parity unpinned".
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)

/* Physical parameters, in the paper's dimensionless units (Eqs. 3d / 2d). */
typedef struct {
  double gamma, nu, lambda; /* trap anisotropies along x, y, z          */
  double g;                 /* g_2D in 2D, g_3D in 3D                   */
  double omega;             /* rotation frequency Omega                 */
  double dt;                /* time step Delta                          */
} orc_phys;

typedef struct {
  int dim;    /* 2 or 3 */
  int n[3];   /* numbers of intervals N_x, N_y, N_z (points are N+1) */
  double h[3];
} orc_grid;

static int grid_ok(const orc_grid* G) {
  if (G->dim != 2 && G->dim != 3) return 0;
  for (int a = 0; a < G->dim; ++a)
    if (G->n[a] < 2 || !(G->h[a] > 0.0)) return 0;
  return 1;
}

static long long npts(const orc_grid* G, int a) {
  return a < G->dim ? (long long)G->n[a] + 1 : 1;
}

static long long total_points(const orc_grid* G) {
  return npts(G, 0) * npts(G, 1) * npts(G, 2);
}

/* Grid coordinate of index i along axis a (Sec. 2: x_i = -N_x h_x/2 + i h_x). */
static double coord(const orc_grid* G, int a, long long i) {
  return -0.5 * (double)G->n[a] * G->h[a] + (double)i * G->h[a];
}

static long long idx3(const orc_grid* G, long long i, long long j, long long k) {
  return (k * npts(G, 1) + j) * npts(G, 0) + i;
}

static int is_edge(const orc_grid* G, long long i, long long j, long long k) {
  if (i == 0 || i == G->n[0]) return 1;
  if (j == 0 || j == G->n[1]) return 1;
  if (G->dim == 3 && (k == 0 || k == G->n[2])) return 1;
  return 0;
}

/* "i Delta" of the real-time formulas, or its imaginary-time replacement
 * Delta (Sec. 2: imaginary time replaces i Delta -> Delta). */
static cplx i_delta(const orc_phys* P, int imag) {
  return imag ? (cplx)P->dt : I * P->dt;
}

/* ------------------------------------------------------------------------ */
/* Thomas algorithm (textbook Gaussian elimination of a tridiagonal system).
 * Solves  am x_{i-1} + a0 x_i + ap x_{i+1} = b_i,  i = 0..m-1, with
 * x_{-1} = x_m = 0, for constant coefficients (am, a0, ap) along the line.
 * Forward: c'_0 = ap/a0, d'_0 = b_0/a0, then c'_i = ap/(a0 - am c'_{i-1}),
 * d'_i = (b_i - am d'_{i-1})/(a0 - am c'_{i-1}).
 * Back substitution: x_{m-1} = d'_{m-1}, x_i = d'_i - c'_i x_{i+1}. */
int orc_thomas(int m, cplx am, cplx a0, cplx ap, const cplx* b, cplx* x) {
  if (m < 1) return ORC_EINVAL;
  cplx* cp = (cplx*)malloc(sizeof(cplx) * (size_t)m);
  cplx* dp = (cplx*)malloc(sizeof(cplx) * (size_t)m);
  if (!cp || !dp) { free(cp); free(dp); return ORC_ENOMEM; }
  cp[0] = ap / a0;
  dp[0] = b[0] / a0;
  for (int i = 1; i < m; ++i) {
    cplx den = a0 - am * cp[i - 1];
    cp[i] = ap / den;
    dp[i] = (b[i] - am * dp[i - 1]) / den;
  }
  x[m - 1] = dp[m - 1];
  for (int i = m - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
  free(cp);
  free(dp);
  return ORC_OK;
}

/* ctypes-friendly wrapper: coefficients and vectors as interleaved doubles. */
int orc_thomas_d(int m, const double* am, const double* a0, const double* ap,
                 const double* b, double* x) {
  return orc_thomas(m, am[0] + I * am[1], a0[0] + I * a0[1],
                    ap[0] + I * ap[1], (const cplx*)b, (cplx*)x);
}

/* ------------------------------------------------------------------------ */
/* H1 substep (Eq. eq1), exact pointwise solution:
 *   real time      psi <- exp(-i Delta (V + g|psi|^2)) psi
 *   imaginary time psi <- exp(-Delta (V + g|psi|^2)) psi
 * with V = (gamma^2 x^2 + nu^2 y^2 [+ lambda^2 z^2]) / 2 and |psi|^2 the
 * value before the substep.  Written as exp(-[i Delta] H1) psi. */
static void apply_h1(const orc_grid* G, const orc_phys* P, int imag, cplx* psi) {
  const cplx idt = i_delta(P, imag);
  for (long long k = 0; k < npts(G, 2); ++k)
    for (long long j = 0; j < npts(G, 1); ++j)
      for (long long i = 0; i < npts(G, 0); ++i) {
        long long p = idx3(G, i, j, k);
        if (is_edge(G, i, j, k)) { psi[p] = 0.0; continue; }
        double x = coord(G, 0, i), y = coord(G, 1, j);
        double V = 0.5 * (P->gamma * P->gamma * x * x + P->nu * P->nu * y * y);
        if (G->dim == 3) {
          double z = coord(G, 2, k);
          V += 0.5 * P->lambda * P->lambda * z * z;
        }
        double dens = creal(psi[p]) * creal(psi[p]) + cimag(psi[p]) * cimag(psi[p]);
        psi[p] = cexp(-idt * (V + P->g * dens)) * psi[p];
      }
}

/* ------------------------------------------------------------------------ */
/* One CN sweep along axis a (0 = x: H2, 1 = y: H3, 2 = z).
 *
 * x-sweep, per line (y_j[, z_k]), Eqs. eqD.11 and eq5, real time:
 *   A0 = 1 + i Delta/(2 h^2)
 *   A- = -(i Delta/(4h)) (1/h - i Omega y_j)
 *   A+ = -(i Delta/(4h)) (1/h + i Omega y_j)
 *   b_i = (i Delta/(4h^2)) (psi_{i+1} - 2 psi_i + psi_{i-1})
 *         - (Delta Omega y_j/(4h)) (psi_{i+1} - psi_{i-1}) + psi_i
 * Imaginary time replaces i Delta -> Delta everywhere (so the plain "Delta"
 * in b becomes Delta / i).
 * y-sweep: H3 = -(1/2) d^2/dy^2 + i Omega x d/dy differs from
 * H2 = -(1/2) d^2/dx^2 - i Omega y d/dx by the replacement Omega y_j ->
 * -Omega x_i ("performed similarly").
 * z-sweep: the same with no rotation term (the 3D "identical prescription").
 * Edge points stay zero; each line's N-1 interior unknowns are solved with
 * the Thomas algorithm above. */
static int sweep_axis(const orc_grid* G, const orc_phys* P, int imag, int a,
                      cplx* psi) {
  const cplx idt = i_delta(P, imag);
  const cplx dt_plain = idt / I; /* "Delta" of the real-time b_i */
  const double h = G->h[a];
  const int N = G->n[a];
  const int m = N - 1;
  cplx* b = (cplx*)malloc(sizeof(cplx) * (size_t)(N + 1));
  cplx* line = (cplx*)malloc(sizeof(cplx) * (size_t)(N + 1));
  cplx* x = (cplx*)malloc(sizeof(cplx) * (size_t)(N + 1));
  if (!b || !line || !x) { free(b); free(line); free(x); return ORC_ENOMEM; }

  long long stride = 1;
  for (int q = 0; q < a; ++q) stride *= npts(G, q);
  /* the two other axes */
  int o1 = (a == 0) ? 1 : 0;
  int o2 = (a == 2) ? 1 : 2;
  long long n1 = npts(G, o1), n2 = npts(G, o2);

  const cplx A0 = 1.0 + idt / (2.0 * h * h);
  for (long long u2 = 0; u2 < n2; ++u2) {
    for (long long u1 = 0; u1 < n1; ++u1) {
      long long ii[3] = {0, 0, 0};
      ii[o1] = u1;
      ii[o2] = u2;
      /* skip lines lying on an edge of another axis: they are identically 0 */
      if (o1 < G->dim && (u1 == 0 || u1 == G->n[o1])) continue;
      if (o2 < G->dim && (u2 == 0 || u2 == G->n[o2])) continue;
      /* rotation coordinate of this line: Omega y_j (x-sweep),
       * -Omega x_i (y-sweep), 0 (z-sweep) */
      double rot = 0.0;
      if (a == 0) rot = P->omega * coord(G, 1, ii[1]);
      if (a == 1) rot = -P->omega * coord(G, 0, ii[0]);
      const cplx Am = -(idt / (4.0 * h)) * (1.0 / h - I * rot);
      const cplx Ap = -(idt / (4.0 * h)) * (1.0 / h + I * rot);
      long long base = idx3(G, ii[0], ii[1], ii[2]);
      for (int i = 0; i <= N; ++i) line[i] = psi[base + (long long)i * stride];
      line[0] = 0.0;
      line[N] = 0.0;
      for (int i = 1; i < N; ++i) {
        b[i - 1] = (idt / (4.0 * h * h)) * (line[i + 1] - 2.0 * line[i] + line[i - 1])
                   - (dt_plain * rot / (4.0 * h)) * (line[i + 1] - line[i - 1])
                   + line[i];
      }
      int rc = orc_thomas(m, Am, A0, Ap, b, x);
      if (rc) { free(b); free(line); free(x); return rc; }
      psi[base] = 0.0;
      for (int i = 1; i < N; ++i) psi[base + (long long)i * stride] = x[i - 1];
      psi[base + (long long)N * stride] = 0.0;
    }
  }
  free(b);
  free(line);
  free(x);
  return ORC_OK;
}

/* Discrete norm h_x h_y [h_z] sum |psi|^2 (trapezoid rule; the edge terms
 * vanish because psi = 0 there).  Normalisation condition of Eqs. 3d / 2d. */
static double norm_of(const orc_grid* G, const cplx* psi) {
  double s = 0.0;
  long long T = total_points(G);
  for (long long p = 0; p < T; ++p)
    s += creal(psi[p]) * creal(psi[p]) + cimag(psi[p]) * cimag(psi[p]);
  double vol = 1.0;
  for (int a = 0; a < G->dim; ++a) vol *= G->h[a];
  return s * vol;
}

static void scale(const orc_grid* G, cplx* psi, double s) {
  long long T = total_points(G);
  for (long long p = 0; p < T; ++p) psi[p] *= s;
}

static int unpack(int dim, const int* n, const double* h, const double* phys,
                  orc_grid* G, orc_phys* P) {
  memset(G, 0, sizeof(*G));
  G->dim = dim;
  for (int a = 0; a < 3; ++a) {
    G->n[a] = a < dim ? n[a] : 0;
    G->h[a] = a < dim ? h[a] : 0.0;
  }
  if (P) {
    P->gamma = phys[0];
    P->nu = phys[1];
    P->lambda = phys[2];
    P->g = phys[3];
    P->omega = phys[4];
    P->dt = phys[5];
  }
  return grid_ok(G) ? ORC_OK : ORC_EINVAL;
}

/* ------------------------------------------------------------------------ */
/* Public entry points (interleaved re/im double arrays of (N+1)^d points). */

/* One substep only: which = 0 (H1), 1 (x-sweep), 2 (y-sweep), 3 (z-sweep). */
int orc_substep(int dim, const int* n, const double* h, const double* phys,
                int imag, int which, double* psi_d) {
  orc_grid G;
  orc_phys P;
  if (unpack(dim, n, h, phys, &G, &P)) return ORC_EINVAL;
  cplx* psi = (cplx*)psi_d;
  if (which == 0) { apply_h1(&G, &P, imag, psi); return ORC_OK; }
  if (which < 1 || which > dim) return ORC_EINVAL;
  return sweep_axis(&G, &P, imag, which - 1, psi);
}

/* nsteps full split steps: H1, x, y[, z]; in imaginary time each full step
 * ends with psi <- psi / sqrt(norm).  Returns the last discrete norm (before
 * renormalisation) in *last_norm if non-NULL. */
int orc_steps(int dim, const int* n, const double* h, const double* phys,
              int imag, long long nsteps, double* psi_d, double* last_norm) {
  orc_grid G;
  orc_phys P;
  if (unpack(dim, n, h, phys, &G, &P)) return ORC_EINVAL;
  cplx* psi = (cplx*)psi_d;
  double nrm = norm_of(&G, psi);
  for (long long s = 0; s < nsteps; ++s) {
    apply_h1(&G, &P, imag, psi);
    for (int a = 0; a < G.dim; ++a) {
      int rc = sweep_axis(&G, &P, imag, a, psi);
      if (rc) return rc;
    }
    nrm = norm_of(&G, psi);
    if (imag) scale(&G, psi, 1.0 / sqrt(nrm));
  }
  if (last_norm) *last_norm = nrm;
  return ORC_OK;
}

double orc_norm(int dim, const int* n, const double* h, const double* psi_d) {
  orc_grid G;
  if (unpack(dim, n, h, NULL, &G, NULL)) return NAN;
  return norm_of(&G, (const cplx*)psi_d);
}

/* ------------------------------------------------------------------------ */
/* Initial state, Eq. fun:
 *   psi(x,y) = (x + i y)/sqrt(pi d_xy^2) exp(-(x^2+y^2)/(2 d_xy^2)
 *              + 2 pi i R(x,y)),
 *   3D:  phi = psi(x,y) (pi d_z^2)^{-1/4} exp(-z^2/(2 d_z^2)),
 * function = 0 selects the Gaussian variant ((x + i y) -> 1).  R holds the
 * random numbers in [0,1) on the (N_x+1)(N_y+1) plane (x fastest), or NULL
 * for no random phase; R depends on (x, y) only.  Edges are zeroed; if
 * normalize != 0 the state is scaled to unit discrete norm. */
int orc_init_analytic(int dim, const int* n, const double* h, int function,
                      const double* R, double d_xy, double d_z, int normalize,
                      double* psi_d) {
  orc_grid G;
  if (unpack(dim, n, h, NULL, &G, NULL)) return ORC_EINVAL;
  cplx* psi = (cplx*)psi_d;
  const double pi = 3.14159265358979323846;
  for (long long k = 0; k < npts(&G, 2); ++k)
    for (long long j = 0; j < npts(&G, 1); ++j)
      for (long long i = 0; i < npts(&G, 0); ++i) {
        long long p = idx3(&G, i, j, k);
        if (is_edge(&G, i, j, k)) { psi[p] = 0.0; continue; }
        double x = coord(&G, 0, i), y = coord(&G, 1, j);
        cplx pre = function ? (x + I * y) : (cplx)1.0;
        double r = R ? R[j * npts(&G, 0) + i] : 0.0;
        cplx v = pre / sqrt(pi * d_xy * d_xy) *
                 cexp(-(x * x + y * y) / (2.0 * d_xy * d_xy) + 2.0 * pi * I * r);
        if (G.dim == 3) {
          double z = coord(&G, 2, k);
          v *= pow(pi * d_z * d_z, -0.25) * exp(-z * z / (2.0 * d_z * d_z));
        }
        psi[p] = v;
      }
  if (normalize) scale(&G, psi, 1.0 / sqrt(norm_of(&G, psi)));
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Observables.
 * Discrete operators are the ones of the CN sweeps: 3-point Laplacian
 * lap = sum_a (psi_{+a} - 2 psi + psi_{-a})/h_a^2 and central differences
 * D_a psi = (psi_{+a} - psi_{-a})/(2 h_a).
 *
 * Real-part forms, Eqs. e2dr / e3dr (alpha = 1: mu, alpha = 1/2: E), with the
 * kinetic term read as -(1/2) psi_R lap psi_R (integration by parts of
 * +(1/2)(grad psi_R)^2; the printed minus sign is taken as a misprint):
 *   [ sum psi_R(-lap psi_R/2 + V psi_R + Omega (y D_x - x D_y) psi_I)
 *     + alpha g sum |psi|^2 psi_R^2 ] / sum psi_R^2.
 * If sum psi_R^2 < 1e-3 sum |psi|^2 the global phase is first rotated by
 * -i (psi_R <- psi_I, psi_I <- -psi_R) so that the quotient is well posed.
 * Complex forms, Eqs. e2d / e3d: with H_lin = -lap/2 + V - Omega L_z,
 * L_z = i (y D_x - x D_y),
 *   mu_c = Re sum psi^* (H_lin + g|psi|^2) psi / sum|psi|^2,
 *   E_c  = Re sum psi^* (H_lin + g|psi|^2/2) psi / sum|psi|^2.
 * rms_a = sqrt(sum a^2 |psi|^2 / sum |psi|^2), rms_r = sqrt(<x^2>+<y^2>[+<z^2>]).
 * out[] = {norm, mu, E, mu_c, E_c, rms_x, rms_y, rms_z, rms_r, max |psi|^2}. */
/* psi at (i, j, k), zero outside the stored grid (the Dirichlet edges
 * extended by zero), for the five-point stencils below. */
static cplx at_or_zero(const orc_grid* G, const cplx* psi, long long i, long long j,
                       long long k) {
  if (i < 0 || i >= npts(G, 0) || j < 0 || j >= npts(G, 1) || k < 0 || k >= npts(G, 2))
    return 0.0;
  return psi[idx3(G, i, j, k)];
}

/* Observables.  out[0..9] as listed in rotgp_obs; out[10], out[11]: mu and
 * E in the complex form with fourth-order central differences for the
 * derivatives (Laplacian (-f2 + 16 f1 - 30 f0 + 16 f-1 - f-2)/(12 h^2),
 * first derivative (-f2 + 8 f1 - 8 f-1 + f-2)/(12 h)) -- the accuracy at
 * which the paper's Table 1 energies are evaluated. */
int orc_observables(int dim, const int* n, const double* h, const double* phys,
                    const double* psi_d, double* out) {
  orc_grid G;
  orc_phys P;
  if (unpack(dim, n, h, phys, &G, &P)) return ORC_EINVAL;
  const cplx* psi = (const cplx*)psi_d;
  double s_abs2 = 0, s_r2 = 0, s_i2 = 0;
  double lin_r = 0, nl_r = 0;   /* real-part sums for psi_R                */
  double lin_i = 0, nl_i = 0;   /* same for the phase-rotated state        */
  double lin_c = 0, nl_c = 0;   /* complex-form sums                       */
  double sx2 = 0, sy2 = 0, sz2 = 0, dmax = 0;
  double lin_4 = 0;             /* complex form, fourth-order differences  */
  const long long sx = 1, sy = npts(&G, 0), sz = npts(&G, 0) * npts(&G, 1);
  for (long long k = 0; k < npts(&G, 2); ++k)
    for (long long j = 0; j < npts(&G, 1); ++j)
      for (long long i = 0; i < npts(&G, 0); ++i) {
        if (is_edge(&G, i, j, k)) continue;
        long long p = idx3(&G, i, j, k);
        double x = coord(&G, 0, i), y = coord(&G, 1, j), z = 0.0;
        double V = 0.5 * (P.gamma * P.gamma * x * x + P.nu * P.nu * y * y);
        if (G.dim == 3) {
          z = coord(&G, 2, k);
          V += 0.5 * P.lambda * P.lambda * z * z;
        }
        cplx c = psi[p];
        cplx lap = (psi[p + sx] - 2.0 * c + psi[p - sx]) / (G.h[0] * G.h[0]) +
                   (psi[p + sy] - 2.0 * c + psi[p - sy]) / (G.h[1] * G.h[1]);
        if (G.dim == 3) lap += (psi[p + sz] - 2.0 * c + psi[p - sz]) / (G.h[2] * G.h[2]);
        cplx dx = (psi[p + sx] - psi[p - sx]) / (2.0 * G.h[0]);
        cplx dy = (psi[p + sy] - psi[p - sy]) / (2.0 * G.h[1]);
        double re = creal(c), im = cimag(c);
        double dens = re * re + im * im;
        /* psi_R terms: -lap_R/2 + V psi_R + Omega (y D_x psi_I - x D_y psi_I) */
        double hr = -0.5 * creal(lap) + V * re + P.omega * (y * cimag(dx) - x * cimag(dy));
        /* rotated state (psi_R' = psi_I, psi_I' = -psi_R) */
        double hi = -0.5 * cimag(lap) + V * im + P.omega * (-(y * creal(dx)) + x * creal(dy));
        lin_r += re * hr;
        nl_r += P.g * dens * re * re;
        lin_i += im * hi;
        nl_i += P.g * dens * im * im;
        cplx Lz = I * (y * dx - x * dy);
        cplx Hlin = -0.5 * lap + V * c - P.omega * Lz;
        lin_c += creal(conj(c) * Hlin);
        /* fourth order: f(+-1), f(+-2) along each axis */
        cplx lap4 = 0.0, d4[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < G.dim; ++a) {
          const long long di = a == 0, dj = a == 1, dk = a == 2;
          cplx p1 = at_or_zero(&G, psi, i + di, j + dj, k + dk);
          cplx m1 = at_or_zero(&G, psi, i - di, j - dj, k - dk);
          cplx p2 = at_or_zero(&G, psi, i + 2 * di, j + 2 * dj, k + 2 * dk);
          cplx m2 = at_or_zero(&G, psi, i - 2 * di, j - 2 * dj, k - 2 * dk);
          lap4 += (-p2 + 16.0 * p1 - 30.0 * c + 16.0 * m1 - m2) / (12.0 * G.h[a] * G.h[a]);
          d4[a] = (-p2 + 8.0 * p1 - 8.0 * m1 + m2) / (12.0 * G.h[a]);
        }
        cplx Lz4 = I * (y * d4[0] - x * d4[1]);
        lin_4 += creal(conj(c) * (-0.5 * lap4 + V * c - P.omega * Lz4));
        nl_c += P.g * dens * dens;
        s_abs2 += dens;
        s_r2 += re * re;
        s_i2 += im * im;
        sx2 += x * x * dens;
        sy2 += y * y * dens;
        sz2 += z * z * dens;
        if (dens > dmax) dmax = dens;
      }
  double vol = 1.0;
  for (int a = 0; a < G.dim; ++a) vol *= G.h[a];
  int rotate = s_r2 < 1e-3 * s_abs2;
  double lin = rotate ? lin_i : lin_r, nl = rotate ? nl_i : nl_r;
  double den = rotate ? s_i2 : s_r2;
  out[0] = vol * s_abs2;
  out[1] = (lin + nl) / den;
  out[2] = (lin + 0.5 * nl) / den;
  out[3] = (lin_c + nl_c) / s_abs2;
  out[4] = (lin_c + 0.5 * nl_c) / s_abs2;
  out[5] = sqrt(sx2 / s_abs2);
  out[6] = sqrt(sy2 / s_abs2);
  out[7] = G.dim == 3 ? sqrt(sz2 / s_abs2) : 0.0;
  out[8] = sqrt((sx2 + sy2 + sz2) / s_abs2);
  out[9] = dmax;
  out[10] = (lin_4 + nl_c) / s_abs2;
  out[11] = (lin_4 + 0.5 * nl_c) / s_abs2;
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Vortex count (a diagnostic; the paper counts vortices in density plots).
 * On the x-y plane (3D: the plane k = N_z/2, i.e. z = 0 for even N_z):
 *  1. Condensate ellipse from the plane's density moments (FP64):
 *     R_x^2 = 6 <x^2>, R_y^2 = 6 <y^2>, the Thomas-Fermi radii of a density
 *     n ~ 1 - x^2/R_x^2 - y^2/R_y^2 (for which <x^2> = R_x^2/6).
 *  2. For every plaquette (i,j),(i+1,j),(i+1,j+1),(i,j+1) that touches no
 *     domain edge and whose centre lies inside 0.9 of that ellipse, sum the
 *     phase increments arg(psi_b conj(psi_a)) in (-pi, pi] around the loop;
 *     the winding number is round(sum / 2 pi) (half away from zero).
 * Returns sum |winding|.  The ellipse keeps out the "ghost" windings of the
 * nearly empty halo without masking the (near-zero density) vortex cores.
 * A core sitting exactly on a grid node (psi = 0 there) is not detected.
 * fp32_decision != 0 computes the windings in single precision (float
 * products, atan2f, float sums), as a single-precision kernel does; the
 * ellipse test stays in double. */
int orc_vortex_count(int dim, const int* n, const double* h, const double* psi_d,
                     int fp32_decision) {
  orc_grid G;
  if (unpack(dim, n, h, NULL, &G, NULL)) return ORC_EINVAL;
  const cplx* psi = (const cplx*)psi_d;
  long long k = G.dim == 3 ? G.n[2] / 2 : 0;
  long long nx = npts(&G, 0), ny = npts(&G, 1);
  const double two_pi = 6.28318530717958647692;
  double s0 = 0, sx = 0, sy = 0;
  for (long long j = 0; j < ny; ++j)
    for (long long i = 0; i < nx; ++i) {
      cplx c = psi[idx3(&G, i, j, k)];
      double d = creal(c) * creal(c) + cimag(c) * cimag(c);
      double x = coord(&G, 0, i), y = coord(&G, 1, j);
      s0 += d;
      sx += x * x * d;
      sy += y * y * d;
    }
  if (!(s0 > 0.0)) return 0;
  double rx2 = 6.0 * sx / s0, ry2 = 6.0 * sy / s0;
  int count = 0;
  for (long long j = 1; j + 2 < ny; ++j)
    for (long long i = 1; i + 2 < nx; ++i) {
      double xc = coord(&G, 0, i) + 0.5 * G.h[0];
      double yc = coord(&G, 1, j) + 0.5 * G.h[1];
      if (!(xc * xc / rx2 + yc * yc / ry2 < 0.81)) continue;
      cplx q[4] = {psi[idx3(&G, i, j, k)], psi[idx3(&G, i + 1, j, k)],
                   psi[idx3(&G, i + 1, j + 1, k)], psi[idx3(&G, i, j + 1, k)]};
      int wn;
      if (!fp32_decision) {
        double w = 0.0;
        for (int t = 0; t < 4; ++t) w += carg(q[(t + 1) & 3] * conj(q[t]));
        wn = (int)lround(w / two_pi);
      } else {
        float re[4], im[4];
        for (int t = 0; t < 4; ++t) {
          re[t] = (float)creal(q[t]);
          im[t] = (float)cimag(q[t]);
        }
        float w = 0.0f;
        for (int t = 0; t < 4; ++t) {
          int u = (t + 1) & 3; /* arg(q_u conj(q_t)) */
          float pr = re[u] * re[t] + im[u] * im[t];
          float pim = im[u] * re[t] - re[u] * im[t];
          w += atan2f(pim, pr);
        }
        wn = (int)lroundf(w / (float)two_pi);
      }
      count += wn < 0 ? -wn : wn;
    }
  return count;
}
