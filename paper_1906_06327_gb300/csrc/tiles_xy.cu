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
//   2. the pending renormalisation and H1 (Eq. eq1) are applied once per
//      point, in place;
//   3. the x stencil runs on all TY + 2K rows (the halo rows are needed by
//      the y stencil), one row per lane, four outputs per step;
//   4. the y stencil runs down the TX columns of the TY output rows, M
//      outputs per thread from a register window, and the result is stored
//      to the other state buffer.  In 2D this completes the step and the
//      block also reduces the norm of what it stored.
//
// The halo points are recomputed by neighbouring tiles (H1 on (TY+2K) x
// (TX+2K') points and the x stencil on TY + 2K rows per TY output rows); in
// exchange the state crosses HBM once per pass instead of once per sweep.
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

// pending scale and H1 on two adjacent points (re, im, re, im); va, vb are
// their trap potentials
template <bool IMAG>
__device__ __forceinline__ float4 h1_pair(float4 v, float s, float va, float vb, float g,
                                          float dt) {
  v.x *= s;
  v.y *= s;
  v.z *= s;
  v.w *= s;
  const float ea = fmaf(g, fmaf(v.x, v.x, v.y * v.y), va);
  const float eb = fmaf(g, fmaf(v.z, v.z, v.w * v.w), vb);
  if (IMAG) {
    const float fa = __expf(-dt * ea), fb = __expf(-dt * eb);
    return make_float4(fa * v.x, fa * v.y, fb * v.z, fb * v.w);
  } else {
    float sa, ca, sb, cb;
    sincosf(dt * ea, &sa, &ca);
    sincosf(dt * eb, &sb, &cb);
    return make_float4(fmaf(ca, v.x, sa * v.y), fmaf(ca, v.y, -sa * v.x), fmaf(cb, v.z, sb * v.w),
                       fmaf(cb, v.w, -sb * v.z));
  }
}

// one output of a stencil with table weights w (2K+1 taps) over inputs in[0..2K]
template <int K>
__device__ __forceinline__ float2 stencil_slow(const float2* w, const float2* in, int step) {
  cacc c = cacc_zero();
#pragma unroll 1
  for (int t = 0; t <= 2 * K; ++t) {
    float2 wr, wi;
    wsplit(w[t], wr, wi);
    cmac(c, wr, wi, in[t * step]);
  }
  return cfin(c);
}

template <int K, bool IMAG, bool REDUCE>
__global__ void __launch_bounds__(128) k_xy_pass(const __grid_constant__ CUtensorMap map,
                                                 const tile_args a) {
  using G = xy_geom<K>;
  constexpr int S = 2 * K + 1;
  // dynamic shared memory: two staged tiles, then the x-stage output
  extern __shared__ __align__(128) unsigned char dsm[];
  unsigned char* base = dsm + ((128 - (smem_addr(dsm) & 127)) & 127);
  auto raw = [&](int bf) { return reinterpret_cast<float2*>(base + bf * G::BYTES); };
  float2* xo = reinterpret_cast<float2*>(base + 2 * G::BYTES);
  __shared__ __align__(8) uint64_t bar[2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per_plane = a.tiles_x * a.tiles_y;
  const int ntiles = per_plane * a.nz;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  // thread 0: start the TMA load of tile t into buffer bf
  auto issue = [&](int t, int bf) {
    const int tx = t % a.tiles_x, ty = (t / a.tiles_x) % a.tiles_y, z = t / per_plane;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&bar[bf], G::BYTES);
    tma_load_3d(raw(bf), &map, 2 * (tx * G::TX - G::KP), ty * G::TY - K, z, &bar[bf]);
  };
  int t = blockIdx.x;
  if (tid == 0 && t < ntiles) issue(t, 0);
  acc_t<float> acc;
  bool good = true;
  int k = 0;
  for (; t < ntiles; ++k, t += gridDim.x) {
    const int bf = k & 1;
    // prefetch the next tile into the other buffer: its last reader (the x
    // stage of the previous tile) finished before the previous barrier
    if (tid == 0 && t + (int)gridDim.x < ntiles) issue(t + gridDim.x, bf ^ 1);
    const int tx = t % a.tiles_x, ty = (t / a.tiles_x) % a.tiles_y, z = t / per_plane;
    const int x0 = tx * G::TX, y0 = ty * G::TY;
    // x weights of this lane's row (interior row), while the tile lands
    const int r = lane;
    const int jx = min(max(y0 - K + r, 0), a.ny - 1);
    const float2* wxl = static_cast<const float2*>(a.wx) + (size_t)jx * (2 * a.bx + 1) * S;
    float2 WR[S], WI[S];
#pragma unroll
    for (int q = 0; q < S; ++q) wsplit(wxl[a.bx * S + q], WR[q], WI[q]);
    if (!__syncthreads_and(mbar_wait(&bar[bf], (k >> 1) & 1))) {
      good = false;
      break;
    }
    float2* tile = raw(bf);
    // ---- 2. pending scale and H1, in place
    {
      const float s = (float)(*a.scale);
      const float zc = a.z0 + (float)z * a.hz;
      const float vz = a.hlam2 * zc * zc;
      constexpr int HALF = G::WX / 2;
      for (int u = tid; u < G::R * HALF; u += 128) {
        const int rr = u / HALF;
        const int i = 2 * (u - rr * HALF);
        float4* p = reinterpret_cast<float4*>(tile + rr * G::WX + i);
        const float yc = a.y0 + (float)(y0 - K + rr) * a.hy;
        const float xa = a.x0 + (float)(x0 - G::KP + i) * a.hx;
        const float xb = xa + a.hx;
        const float vyz = fmaf(a.hnu2, yc * yc, vz);
        *p = h1_pair<IMAG>(*p, s, fmaf(a.hgam2, xa * xa, vyz), fmaf(a.hgam2, xb * xb, vyz), a.g,
                           a.dt);
      }
    }
    __syncthreads();
    // ---- 3. x stencil on every loaded row: lane = row, warp = quads of 4 outputs
    if (r < G::R) {
      constexpr int NW = (4 + 2 * G::KP) / 2;  // float4 of the window
      constexpr int OFF = G::KP - K;
      const float2* row = tile + r * G::WX;
      float2* orow = xo + r * G::PX;
      for (int q = warp; q < G::TX / 4; q += 4) {
        const int xq = x0 + 4 * q;
        float2 o[4];
        if (xq >= a.bx && xq + 3 < a.nx - a.bx) {
          const float4* src = reinterpret_cast<const float4*>(row + 4 * q);
          float4 wv[NW];
#pragma unroll
          for (int i = 0; i < NW; ++i) wv[i] = src[i];
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            cacc c = cacc_zero();
#pragma unroll
            for (int j = 0; j < S; ++j) {
              const int i = OFF + m + j;
              const float4 w4 = wv[i >> 1];
              cmac(c, WR[j], WI[j], (i & 1) ? make_float2(w4.z, w4.w) : make_float2(w4.x, w4.y));
            }
            o[m] = cfin(c);
          }
        } else {
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const int x = xq + m;
            o[m] = make_float2(0.f, 0.f);
            if (x < a.nx)
              o[m] = stencil_slow<K>(wxl + stencil_row(x, a.nx, a.bx) * S, row + 4 * q + OFF + m, 1);
          }
        }
        float4* dst = reinterpret_cast<float4*>(orow + 4 * q);
        dst[0] = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
        dst[1] = make_float4(o[2].x, o[2].y, o[3].x, o[3].y);
      }
    }
    __syncthreads();
    // ---- 4. y stencil: lane = column (two column halves), M rows per group
    {
      const int cx = 32 * (warp & 1) + lane;
      const int x = x0 + cx;
      const float2* wyl =
          static_cast<const float2*>(a.wy) + (size_t)min(x, a.nx - 1) * (2 * a.by + 1) * S;
#pragma unroll
      for (int q = 0; q < S; ++q) wsplit(wyl[a.by * S + q], WR[q], WI[q]);
      float2* out = static_cast<float2*>(a.out) + (size_t)z * a.ny * a.nx + x;
      for (int gq = warp >> 1; gq < 4; gq += 2) {
        const int yg = y0 + gq * G::M;
        const float2* col = xo + gq * G::M * G::PX + cx;
        float2 o[G::M];
        if (yg >= a.by && yg + G::M - 1 < a.ny - a.by) {
          float2 win[G::M + 2 * K];
#pragma unroll
          for (int i = 0; i < G::M + 2 * K; ++i) win[i] = col[i * G::PX];
#pragma unroll
          for (int m = 0; m < G::M; ++m) {
            cacc c = cacc_zero();
#pragma unroll
            for (int j = 0; j < S; ++j) cmac(c, WR[j], WI[j], win[m + j]);
            o[m] = cfin(c);
          }
        } else {
#pragma unroll
          for (int m = 0; m < G::M; ++m) {
            const int y = yg + m;
            o[m] = make_float2(0.f, 0.f);
            if (y < a.ny)
              o[m] = stencil_slow<K>(wyl + stencil_row(y, a.ny, a.by) * S, col + m * G::PX, G::PX);
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
    // the next iteration's first barrier orders these reads of xo before
    // the next x stage writes it
  }
  if (!good) {
    // let the prefetch in flight (if any) land before the CTA leaves
    if (t + (int)gridDim.x < ntiles) mbar_wait(&bar[(k & 1) ^ 1], ((k + 1) >> 1) & 1);
    if (tid == 0) atomicOr(a.flags, 4);
  }
  if (REDUCE) norm_epilogue(acc.value(), a);
}

bool tile_k_built(int K) { return K == 4 || K == 6 || K == 8; }

void xy_tile_geometry(int K, int* TX, int* TY, int* R, int* WX) {
  const int KP = (K + 1) & ~1;
  *TX = 64;
  *TY = ((32 - 2 * K) / 4) * 4;
  *R = *TY + 2 * K;
  *WX = 64 + 2 * KP + 2;
}

template <int K, bool IMAG, bool REDUCE>
cudaError_t launch_xy_k(const CUtensorMap& m, const tile_args& a, unsigned blocks,
                        cudaStream_t s) {
  using G = xy_geom<K>;
  // opt this instantiation in to its dynamic shared memory, once
  static const cudaError_t e = cudaFuncSetAttribute(
      k_xy_pass<K, IMAG, REDUCE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
  if (e != cudaSuccess) return e;
  k_xy_pass<K, IMAG, REDUCE><<<blocks, 128, G::SMEM, s>>>(m, a);
  return cudaGetLastError();
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
