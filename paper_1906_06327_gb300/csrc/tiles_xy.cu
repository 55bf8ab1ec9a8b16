// tiles_xy.cu -- the H1 substep and the x and y sweeps of one split step
// (Sec. 2, Eqs. eq1 and eqD.9-eqD.11/eq5) in a single pass over the state,
// complex float.
//
// Each sweep is applied in its banded-inverse form psi' = W psi with
// W = 2 A^{-1} - I truncated to K points on either side (stencil.cu derives
// the weights).  A sweep then only needs the K neighbours of a point along
// its axis, so H1, the x sweep and the y sweep of a tile of TX x TY points
// need the tile plus K-point halos in x and y of the state before the step,
// and nothing else:
//
//   1. one TMA load brings the (TY + 2K) x (TX + 2K') haloed tile of one z
//      plane into shared memory (points outside the grid read as zero; K' is
//      K rounded up to even so that the box starts on a 16-byte boundary).
//      CTAs are persistent (a few per SM, tiles taken round-robin) and
//      double-buffer the tiles: the next tile's load is in flight while the
//      current one is computed;
//   2. the x stencil runs on all TY + 2K rows (the halo rows are needed by
//      the y stencil): a lane owns one row and a warp a strip of 16
//      outputs; the lane reads its 16 + 2K window, applies the pending
//      renormalisation and H1 (Eq. eq1) to it in registers (neighbouring
//      strips recompute the 2K halo points), and writes 16 outputs;
//   3. the y stencil runs down the TX columns of the TY output rows, M
//      outputs per thread from a register window, and the result is stored
//      to the other state buffer.  In 2D this completes the step and the
//      block also reduces the norm of what it stored.
//
// The halo points are recomputed by neighbouring tiles and strips (H1 on
// (TY + 2K) x 4 (16 + 2K) points and the x stencil on TY + 2K rows per
// TX x TY outputs); in exchange the state crosses HBM once per pass instead
// of once per sweep.
#include "sweep_common.cuh"
#include "tma.cuh"

namespace rotgp {

template <int K>
struct xy_geom {
  static constexpr int TX = 64;                        // outputs per tile row
  static constexpr int KP = (K + 1) & ~1;              // x halo as loaded
  static constexpr int TY = ((32 - 2 * K) / 4) * 4;    // output rows per tile
  static constexpr int M = TY / 4;                     // y outputs per thread
  static constexpr int R = TY + 2 * K;                 // rows loaded (<= 32)
  static constexpr int WX = TX + 2 * KP + 2;           // complex per staged row (+2: banks)
  static constexpr int PX = TX + 2;                    // complex per x-output row (+2: banks)
  static constexpr unsigned BYTES = (unsigned)(R * WX * 8);  // one staged tile (x128 B)
  static constexpr unsigned SMEM = 2 * BYTES + R * PX * 8 + 128;
  static_assert(R <= 32 && TY % 4 == 0 && WX % 2 == 0 && BYTES % 128 == 0, "tile geometry");
};

// pending scale and H1 on one point held in registers; vxyz is its trap
// potential
template <bool IMAG>
__device__ __forceinline__ float2 h1_point(float2 v, float s, float vxyz, float g, float dt) {
  v.x *= s;
  v.y *= s;
  const float e = fmaf(g, fmaf(v.x, v.x, v.y * v.y), vxyz);
  if (IMAG) {
    const float f = __expf(-dt * e);
    return make_float2(f * v.x, f * v.y);
  } else {
    float c1, s1;
    rot_t(dt * e, &c1, &s1);
    return rotate_f(v, c1, s1);
  }
}

// One CTA per (x-y tile, range of z planes): the tile position is fixed, so
// each lane's x weights (its row) stay in registers for the whole range, and
// so do its y weights (its column) when K = 4 (longer stencils reload them
// per plane from L1: both sets would not fit).  Planes are double-buffered:
// the TMA load of the next plane is in flight while the current one is
// computed.
template <int K, bool IMAG, bool REDUCE>
__global__ void __launch_bounds__(128) k_xy_pass(const __grid_constant__ CUtensorMap map,
                                                 const tile_args a) {
  using G = xy_geom<K>;
  constexpr int S = 2 * K + 1;
  constexpr int XS = 16;          // x outputs of one warp's strip
  constexpr int NWIN = XS + 2 * K;
  static_assert(G::KP == K, "x halo must start on a 16-byte boundary");
  extern __shared__ __align__(128) unsigned char dsm[];
  unsigned char* base = dsm + ((128 - (smem_addr(dsm) & 127)) & 127);
  auto raw = [&](int bf) { return reinterpret_cast<float2*>(base + bf * G::BYTES); };
  float2* xo = reinterpret_cast<float2*>(base + 2 * G::BYTES);
  __shared__ __align__(8) uint64_t bar[2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tiles_xy = a.tiles_x * a.tiles_y;
  const int txy = blockIdx.x % tiles_xy;
  const int zb = (blockIdx.x / tiles_xy) * a.zchunk;
  const int ze = min(a.nz, zb + a.zchunk);
  const int x0 = (txy % a.tiles_x) * G::TX, y0 = (txy / a.tiles_x) * G::TY;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](int z, int bf) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&bar[bf], G::BYTES);
    tma_load_3d(raw(bf), &map, 2 * (x0 - K), y0 - K, z, &bar[bf]);
  };
  if (tid == 0 && zb < ze) issue(zb, 0);
  // x stage: lane = tile row r, warp = strip of 16 outputs
  const int r = lane;
  const float2* wxl = static_cast<const float2*>(a.wx) +
                      (size_t)min(max(y0 - K + r, 0), a.ny - 1) * (2 * a.bx + 1) * S;
  float2 XR[S], XI[S];
#pragma unroll
  for (int t = 0; t < S; ++t) wsplit(wxl[a.bx * S + t], XR[t], XI[t]);
  const int xq0 = x0 + XS * warp;  // first output of the strip
  const bool x_fast = xq0 >= a.bx && xq0 + XS - 1 < a.nx - a.bx;
  const float yc = a.y0 + (float)(y0 - K + r) * a.hy;
  const float vy = a.hnu2 * yc * yc;
  const float xw = a.x0 + (float)(xq0 - K) * a.hx;  // x of window point 0
  // y stage: lane = column (two column halves), groups of M rows
  const int cx = 32 * (warp & 1) + lane;
  const int x = x0 + cx;
  const float2* wyl =
      static_cast<const float2*>(a.wy) + (size_t)min(x, a.nx - 1) * (2 * a.by + 1) * S;
  constexpr bool YREG = K <= 4;
  float2 YR[YREG ? S : 1], YI[YREG ? S : 1];
  if (YREG) {
#pragma unroll
    for (int t = 0; t < S; ++t) wsplit(wyl[a.by * S + t], YR[t], YI[t]);
  }
  const float sc = (float)(*a.scale);
  acc_t<float> acc;
  bool good = true;
  int k = 0;
  for (int z = zb; z < ze; ++k, ++z) {
    const int bf = k & 1;
    // the other buffer's last reader (the x stage of the previous plane)
    // finished before the previous barrier
    if (tid == 0 && z + 1 < ze) issue(z + 1, bf ^ 1);
    if (!__syncthreads_and(mbar_wait(&bar[bf], (k >> 1) & 1))) {
      good = false;
      break;
    }
    // ---- x stage with the pending scale and H1 applied to the window
    if (r < G::R) {
      const float zc = a.z0 + (float)z * a.hz;
      const float vyz = fmaf(a.hlam2, zc * zc, vy);
      const float4* src = reinterpret_cast<const float4*>(raw(bf) + r * G::WX + XS * warp);
      float2 v[NWIN];
#pragma unroll
      for (int i = 0; i < NWIN / 2; ++i) {
        const float4 q = src[i];
        v[2 * i] = make_float2(q.x, q.y);
        v[2 * i + 1] = make_float2(q.z, q.w);
      }
#pragma unroll
      for (int t = 0; t < NWIN; ++t) {
        const float xc = fmaf((float)t, a.hx, xw);
        v[t] = h1_point<IMAG>(v[t], sc, fmaf(a.hgam2, xc * xc, vyz), a.g, a.dt);
      }
      float4* dst = reinterpret_cast<float4*>(xo + r * G::PX + XS * warp);
      if (x_fast) {
#pragma unroll
        for (int m = 0; m < XS; m += 2) {
          cacc c0 = cacc_zero(), c1 = cacc_zero();
#pragma unroll
          for (int t = 0; t < S; ++t) {
            cmac(c0, XR[t], XI[t], v[m + t]);
            cmac(c1, XR[t], XI[t], v[m + 1 + t]);
          }
          const float2 o0 = cfin(c0), o1 = cfin(c1);
          dst[m / 2] = make_float4(o0.x, o0.y, o1.x, o1.y);
        }
      } else {
#pragma unroll
        for (int m = 0; m < XS; m += 2) {
          float2 o[2];
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int xo_ = xq0 + m + e;
            const float2* wr = wxl + stencil_row(min(xo_, a.nx - 1), a.nx, a.bx) * S;
            cacc c = cacc_zero();
#pragma unroll
            for (int t = 0; t < S; ++t) {
              float2 pr, pi;
              wsplit(wr[t], pr, pi);
              cmac(c, pr, pi, v[m + e + t]);
            }
            o[e] = xo_ < a.nx ? cfin(c) : make_float2(0.f, 0.f);
          }
          dst[m / 2] = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
        }
      }
    }
    __syncthreads();
    // ---- y stage
    {
      float2* out = static_cast<float2*>(a.out) + (size_t)z * a.ny * a.nx + x;
      for (int gq = warp >> 1; gq < 4; gq += 2) {
        const int yg = y0 + gq * G::M;
        const float2* col = xo + gq * G::M * G::PX + cx;
        float2 win[G::M + 2 * K];
#pragma unroll
        for (int i = 0; i < G::M + 2 * K; ++i) win[i] = col[i * G::PX];
        float2 o[G::M];
        if (yg >= a.by && yg + G::M - 1 < a.ny - a.by) {
          float2 QR[S], QI[S];
#pragma unroll
          for (int t = 0; t < S; ++t) {
            if (YREG) {
              QR[t] = YR[YREG ? t : 0];
              QI[t] = YI[YREG ? t : 0];
            } else {
              wsplit(wyl[a.by * S + t], QR[t], QI[t]);
            }
          }
#pragma unroll
          for (int m = 0; m < G::M; ++m) {
            cacc c = cacc_zero();
#pragma unroll
            for (int t = 0; t < S; ++t) cmac(c, QR[t], QI[t], win[m + t]);
            o[m] = cfin(c);
          }
        } else {
#pragma unroll
          for (int m = 0; m < G::M; ++m) {
            const int y = yg + m;
            const float2* wr = wyl + stencil_row(min(y, a.ny - 1), a.ny, a.by) * S;
            cacc c = cacc_zero();
#pragma unroll
            for (int t = 0; t < S; ++t) {
              float2 pr, pi;
              wsplit(wr[t], pr, pi);
              cmac(c, pr, pi, win[m + t]);
            }
            o[m] = cfin(c);
          }
        }
        if (x < a.nx) {
#pragma unroll
          for (int m = 0; m < G::M; ++m) {
            const int y = yg + m;
            if (y < a.ny) {
              out[(size_t)y * a.nx] = o[m];
              if (REDUCE) acc.add(fmaf(o[m].x, o[m].x, o[m].y * o[m].y));
            }
          }
        }
      }
    }
    // the next plane's first barrier orders these reads of xo before the
    // next x stage writes it
  }
  if (!good) {
    // let the prefetch in flight (if any) land before the CTA leaves
    if (zb + k + 1 < ze) mbar_wait(&bar[(k & 1) ^ 1], ((k + 1) >> 1) & 1);
    if (tid == 0) atomicOr(a.flags, 4);
  }
  if (REDUCE) norm_epilogue(acc.value(), a);
}

// ------------------------------------------------------------ x sweep alone
// The x sweep (with the pending scale and H1) in stencil form when the y
// sweep is not fused with it: tiles of 32 rows x 64 points of one plane
// with the K-point x halo, staged by one TMA load (double-buffered along
// the CTA's z range); lane = row, warp = strip of 16 outputs, H1 applied to
// the strip's window in registers; the results are written back into the
// staged tile and copied out row by row (coalesced).  No y halo rows.
template <int K>
struct x_geom {
  static constexpr int TX = 64, ROWS = 32;
  static constexpr int WX = TX + 2 * K + 2;  // complex per staged row (+2: banks)
  static constexpr unsigned BYTES = (unsigned)(ROWS * WX * 8);
  static constexpr unsigned SMEM = 2 * BYTES + 128;
  static_assert(K % 2 == 0 && BYTES % 128 == 0, "x tile geometry");
};

template <int K, bool IMAG>
__global__ void __launch_bounds__(128) k_x_pass(const __grid_constant__ CUtensorMap map,
                                                const tile_args a) {
  using G = x_geom<K>;
  constexpr int S = 2 * K + 1;
  constexpr int XS = 16;
  constexpr int NWIN = XS + 2 * K;
  extern __shared__ __align__(128) unsigned char dsm[];
  unsigned char* base = dsm + ((128 - (smem_addr(dsm) & 127)) & 127);
  auto raw = [&](int bf) { return reinterpret_cast<float2*>(base + bf * G::BYTES); };
  __shared__ __align__(8) uint64_t bar[2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tiles_xy = a.tiles_x * a.tiles_y;
  const int txy = blockIdx.x % tiles_xy;
  const int zb = (blockIdx.x / tiles_xy) * a.zchunk;
  const int ze = min(a.nz, zb + a.zchunk);
  const int x0 = (txy % a.tiles_x) * G::TX, y0 = (txy / a.tiles_x) * G::ROWS;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](int z, int bf) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&bar[bf], G::BYTES);
    tma_load_3d(raw(bf), &map, 2 * (x0 - K), y0, z, &bar[bf]);
  };
  if (tid == 0 && zb < ze) issue(zb, 0);
  const int y = y0 + lane;
  const float2* wxl = static_cast<const float2*>(a.wx) +
                      (size_t)min(y, a.ny - 1) * (2 * a.bx + 1) * S;
  float2 XR[S], XI[S];
#pragma unroll
  for (int t = 0; t < S; ++t) wsplit(wxl[a.bx * S + t], XR[t], XI[t]);
  const int xq0 = x0 + XS * warp;
  const bool x_fast = xq0 >= a.bx && xq0 + XS - 1 < a.nx - a.bx;
  const float yc = a.y0 + (float)y * a.hy;
  const float vy = a.hnu2 * yc * yc;
  const float xw = a.x0 + (float)(xq0 - K) * a.hx;
  const float sc = (float)(*a.scale);
  bool good = true;
  int k = 0;
  for (int z = zb; z < ze; ++k, ++z) {
    const int bf = k & 1;
    if (!__syncthreads_and(mbar_wait(&bar[bf], (k >> 1) & 1))) {
      good = false;
      break;
    }
    // prefetch the next plane into the other buffer: its last reader (the
    // copy-out of the previous plane) finished before the barrier above
    if (tid == 0 && z + 1 < ze) issue(z + 1, bf ^ 1);
    const float zc = a.z0 + (float)z * a.hz;
    const float vyz = fmaf(a.hlam2, zc * zc, vy);
    const float4* src = reinterpret_cast<const float4*>(raw(bf) + lane * G::WX + XS * warp);
    float2 v[NWIN];
#pragma unroll
    for (int i = 0; i < NWIN / 2; ++i) {
      const float4 q = src[i];
      v[2 * i] = make_float2(q.x, q.y);
      v[2 * i + 1] = make_float2(q.z, q.w);
    }
#pragma unroll
    for (int t = 0; t < NWIN; ++t) {
      const float xc = fmaf((float)t, a.hx, xw);
      v[t] = h1_point<IMAG>(v[t], sc, fmaf(a.hgam2, xc * xc, vyz), a.g, a.dt);
    }
    float4 res[XS / 2];
#pragma unroll
    for (int m = 0; m < XS; m += 2) {
      float2 o[2];
      if (x_fast) {
        cacc c0 = cacc_zero(), c1 = cacc_zero();
#pragma unroll
        for (int t = 0; t < S; ++t) {
          cmac(c0, XR[t], XI[t], v[m + t]);
          cmac(c1, XR[t], XI[t], v[m + 1 + t]);
        }
        o[0] = cfin(c0);
        o[1] = cfin(c1);
      } else {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int xo_ = xq0 + m + e;
          const float2* wr = wxl + stencil_row(min(xo_, a.nx - 1), a.nx, a.bx) * S;
          cacc c = cacc_zero();
#pragma unroll
          for (int t = 0; t < S; ++t) {
            float2 pr, pi;
            wsplit(wr[t], pr, pi);
            cmac(c, pr, pi, v[m + e + t]);
          }
          o[e] = cfin(c);
        }
      }
      res[m / 2] = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
    }
    // every warp has read its window: the results go into the tile's
    // interior (row pitch WX, conflict-free for lane = row), and the whole
    // tile is then copied out row by row (32 lanes = 512 contiguous bytes)
    __syncthreads();
    {
      float4* dst = reinterpret_cast<float4*>(raw(bf) + lane * G::WX + K + XS * warp);
#pragma unroll
      for (int i = 0; i < XS / 2; ++i) dst[i] = res[i];
    }
    __syncthreads();
    {
      constexpr int PR = G::TX / 2;  // float4 (two points) per output row
      float2* outp = static_cast<float2*>(a.out) + (size_t)z * a.ny * a.nx;
#pragma unroll
      for (int i = 0; i < G::ROWS * PR / 128; ++i) {
        const int t = i * 128 + tid, rr = t / PR, cc = t % PR;
        const int yy = y0 + rr, xx = x0 + 2 * cc;
        if (yy < a.ny && xx < a.nx)
          *reinterpret_cast<float4*>(outp + (size_t)yy * a.nx + xx) =
              *reinterpret_cast<const float4*>(raw(bf) + rr * G::WX + K + 2 * cc);
      }
    }
  }
  if (!good && tid == 0) atomicOr(a.flags, 4);  // no prefetch was issued for this plane
}

bool tile_k_built(int K) { return K == 4 || K == 6 || K == 8; }

void xy_tile_geometry(int K, int* TX, int* TY, int* R, int* WX) {
  const int KP = (K + 1) & ~1;
  *TX = 64;
  *TY = ((32 - 2 * K) / 4) * 4;
  *R = *TY + 2 * K;
  *WX = 64 + 2 * KP + 2;
}

// opt an instantiation in to its dynamic shared memory, once per device
template <int K, bool IMAG, bool REDUCE>
cudaError_t xy_allow_smem() {
  return allow_smem_bytes((const void*)k_xy_pass<K, IMAG, REDUCE>, (int)xy_geom<K>::SMEM);
}

template <int K, bool IMAG, bool REDUCE>
int xy_ctas_k() {
  int n = 0;
  if (xy_allow_smem<K, IMAG, REDUCE>() != cudaSuccess) return 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_xy_pass<K, IMAG, REDUCE>, 128,
                                                    xy_geom<K>::SMEM) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

int xy_pass_ctas_per_sm(int K, bool imag, bool reduce) {
#define ROTGP_XO(KK)                                                     \
  if (K == KK) {                                                         \
    if (imag && reduce) return xy_ctas_k<KK, true, true>();              \
    if (imag) return xy_ctas_k<KK, true, false>();                       \
    if (reduce) return xy_ctas_k<KK, false, true>();                     \
    return xy_ctas_k<KK, false, false>();                                \
  }
  ROTGP_XO(4)
  ROTGP_XO(6)
  ROTGP_XO(8)
#undef ROTGP_XO
  return 1;
}

template <int K, bool IMAG, bool REDUCE>
cudaError_t launch_xy_k(const CUtensorMap& m, const tile_args& a, unsigned blocks,
                        cudaStream_t s) {
  using G = xy_geom<K>;
  const cudaError_t e = xy_allow_smem<K, IMAG, REDUCE>();
  if (e != cudaSuccess) return e;
  k_xy_pass<K, IMAG, REDUCE><<<blocks, 128, G::SMEM, s>>>(m, a);
  return cudaGetLastError();
}

template <int K, bool IMAG>
cudaError_t x_allow_smem() {
  return allow_smem_bytes((const void*)k_x_pass<K, IMAG>, (int)x_geom<K>::SMEM);
}

int x_pass_ctas_per_sm(int K) {
  int n = 0;
#define ROTGP_XC(KK)                                                                     \
  if (K == KK) {                                                                         \
    if (x_allow_smem<KK, false>() != cudaSuccess ||                                      \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_x_pass<KK, false>, 128,      \
                                                      x_geom<KK>::SMEM) != cudaSuccess)  \
      return 1;                                                                          \
    return n > 0 ? n : 1;                                                                \
  }
  ROTGP_XC(4)
  ROTGP_XC(6)
  ROTGP_XC(8)
#undef ROTGP_XC
  return 1;
}

cudaError_t launch_x_pass(bool imag, int K, const void* map, const tile_args& a, unsigned blocks,
                          cudaStream_t s) {
  const CUtensorMap& m = *static_cast<const CUtensorMap*>(map);
#define ROTGP_XP(KK)                                                                   \
  if (K == KK) {                                                                       \
    cudaError_t e = imag ? x_allow_smem<KK, true>() : x_allow_smem<KK, false>();       \
    if (e != cudaSuccess) return e;                                                    \
    if (imag)                                                                          \
      k_x_pass<KK, true><<<blocks, 128, x_geom<KK>::SMEM, s>>>(m, a);                  \
    else                                                                               \
      k_x_pass<KK, false><<<blocks, 128, x_geom<KK>::SMEM, s>>>(m, a);                 \
    return cudaGetLastError();                                                         \
  }
  ROTGP_XP(4)
  ROTGP_XP(6)
  ROTGP_XP(8)
#undef ROTGP_XP
  return cudaErrorInvalidValue;
}

unsigned xy_pass_smem(int K) {
  return K == 4 ? xy_geom<4>::SMEM : K == 6 ? xy_geom<6>::SMEM : xy_geom<8>::SMEM;
}

cudaError_t launch_xy_pass(bool imag, bool reduce, int K, const void* map, const tile_args& a,
                           unsigned blocks, cudaStream_t s) {
  const CUtensorMap& m = *static_cast<const CUtensorMap*>(map);
#define ROTGP_XY(KK)                                                             \
  if (K == KK) {                                                                 \
    if (imag && reduce) return launch_xy_k<KK, true, true>(m, a, blocks, s);     \
    if (imag) return launch_xy_k<KK, true, false>(m, a, blocks, s);              \
    if (reduce) return launch_xy_k<KK, false, true>(m, a, blocks, s);            \
    return launch_xy_k<KK, false, false>(m, a, blocks, s);                       \
  }
  ROTGP_XY(4)
  ROTGP_XY(6)
  ROTGP_XY(8)
#undef ROTGP_XY
  return cudaErrorInvalidValue;
}

}  // namespace rotgp
