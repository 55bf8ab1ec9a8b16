// tiles_line.cu -- a y or z sweep of one split step (Sec. 2, Eqs. eqD.9-
// eqD.11/eq5) in banded-inverse form (psi' = W psi, W = 2 A^{-1} - I
// truncated to K points either side; stencil.cu derives the weights),
// complex float, for lines that are strided in memory.
//
// A CTA of two warps owns a patch of 32 x 2 lines (32 consecutive x, 2
// consecutive positions of the other transverse axis) and one segment of
// them (the whole lines, or a part with K-point halos read from the
// neighbouring segments when more warps are wanted), which it streams
// through an 8-slot ring of TMA boxes of 8 line positions each (4 KB):
// the box of positions 8b - K .. 8b + 7 - K lands in slot b % 8 while the
// CTA works on earlier boxes, and a slot is refilled as soon as both warps
// are done with it, so up to seven boxes per CTA are in flight.  A warp's
// 32 lanes are the 32 x values of one transverse row: every shared-memory
// read and global store of a warp is 256 contiguous bytes.  Each thread
// carries the last 2K positions of its line in registers from box to box
// and produces a box's eight outputs together (sixteen independent FMA
// chains; boxes at a line end take per-position weights).  In 3D the z
// sweep is the last of the step and also reduces the norm.
#include "sweep_common.cuh"
#include "tma.cuh"

namespace rotgp {

namespace {
constexpr int kRows = 2;                       // transverse rows per CTA (one per warp)
constexpr int kBox = 8;                        // line positions per TMA box
constexpr int kSlots = 8;                      // ring slots
constexpr int kSlot = kBox * kRows * 32;       // complex points per slot
constexpr unsigned kBoxBytes = kSlot * 8;      // 4 KB
}  // namespace

// AX = 1: y lines (transverse rows are z); AX = 2: z lines (rows are y).
template <int K, int AX, bool REDUCE>
__global__ void __launch_bounds__(64) k_line_pass(const __grid_constant__ CUtensorMap map,
                                                  const tile_args a) {
  constexpr int S = 2 * K + 1;
  __shared__ __align__(128) float2 ring[kSlots * kSlot];
  __shared__ __align__(8) uint64_t full[kSlots];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int px = blockIdx.x % a.tiles_x, pt = (blockIdx.x / a.tiles_x) % a.tiles_y;
  const int sg = blockIdx.x / (a.tiles_x * a.tiles_y);  // segment of the lines
  const int N = AX == 2 ? a.nz : a.ny;
  const int NT = AX == 2 ? a.ny : a.nz;
  const int B = AX == 2 ? a.bz : a.by;
  const int x = 32 * px + lane, t2 = kRows * pt + w;
  // outputs sb .. se-1 of this segment, from positions sb-K .. se-1+K
  const int sb = sg * a.seg_len, se = min(N, sb + a.seg_len);
  const int nb = (se - sb + 2 * K + kBox - 1) / kBox;
  if (tid == 0) {
#pragma unroll
    for (int i = 0; i < kSlots; ++i) mbar_init(&full[i], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](int b) {
    const int c = sb + kBox * b - K;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&full[b % kSlots], kBoxBytes);
    if (AX == 2)
      tma_load_3d(ring + (b % kSlots) * kSlot, &map, 64 * px, kRows * pt, c, &full[b % kSlots]);
    else
      tma_load_3d(ring + (b % kSlots) * kSlot, &map, 64 * px, c, kRows * pt, &full[b % kSlots]);
  };
  if (tid == 0)
    for (int b = 0; b < min(kSlots, nb); ++b) issue(b);
  const float2* wl = static_cast<const float2*>(AX == 2 ? a.wz : a.wy) +
                     (AX == 2 ? 0 : (size_t)min(x, a.nx - 1) * (2 * B + 1) * S);
  float2 WR[S], WI[S];
#pragma unroll
  for (int t = 0; t < S; ++t) wsplit(wl[B * S + t], WR[t], WI[t]);
  const bool store_ok = x < a.nx && t2 < NT;
  float2* out = static_cast<float2*>(a.out) + x +
                (AX == 2 ? (size_t)t2 * a.nx : (size_t)t2 * a.ny * a.nx);
  const size_t ostep = AX == 2 ? (size_t)a.ny * a.nx : (size_t)a.nx;
  acc_t<float> acc;
  // win[t]: staged positions 8b - 2K + t (t < 2K) before box b is read;
  // u[]: those followed by the box's 8 positions, so that output j of the
  // box (position 8b - 2K + j) uses u[j .. j + 2K]
  float2 win[2 * K];
#pragma unroll
  for (int t = 0; t < 2 * K; ++t) win[t] = make_float2(0.f, 0.f);
  bool good = true;
  int b = 0;
  for (; b < nb; ++b) {
    const int slot = b % kSlots;
    good = mbar_wait(&full[slot], (b / kSlots) & 1);
    const float2* sl = ring + slot * kSlot;
    float2 u[2 * K + kBox];
#pragma unroll
    for (int t = 0; t < 2 * K; ++t) u[t] = win[t];
#pragma unroll
    for (int j = 0; j < kBox; ++j)
      u[2 * K + j] = sl[(AX == 2 ? j * kRows + w : w * kBox + j) * 32 + lane];
    const int s0 = sb + kBox * b - 2 * K;  // output position of j = 0
    float2 r[kBox];
    if (s0 >= B && s0 + kBox <= N - B) {
      // interior box: eight independent outputs, no branches
#pragma unroll
      for (int j = 0; j < kBox; ++j) {
        cacc c = cacc_zero();
#pragma unroll
        for (int t = 0; t < S; ++t) cmac(c, WR[t], WI[t], u[j + t]);
        r[j] = cfin(c);
      }
    } else {
      // a line end (or the ramp-up before the first output): per-output rows
#pragma unroll
      for (int j = 0; j < kBox; ++j) {
        const int s = s0 + j;
        const float2* wr = wl + stencil_row(min(max(s, 0), N - 1), N, B) * S;
        cacc c = cacc_zero();
#pragma unroll
        for (int t = 0; t < S; ++t) {
          float2 pr, pi;
          wsplit(wr[t], pr, pi);
          cmac(c, pr, pi, u[j + t]);
        }
        r[j] = cfin(c);
      }
    }
#pragma unroll
    for (int j = 0; j < kBox; ++j) {
      const int s = s0 + j;
      if (store_ok && s >= sb && s < se) {
        out[(size_t)s * ostep] = r[j];
        if (REDUCE) acc.add(fmaf(r[j].x, r[j].x, r[j].y * r[j].y));
      }
    }
#pragma unroll
    for (int t = 0; t < 2 * K; ++t) win[t] = u[kBox + t];
    // both warps are done with this slot: refill it
    if (!__syncthreads_and(good)) break;
    if (tid == 0 && b + kSlots < nb) issue(b + kSlots);
  }
  if (b < nb) {
    // a wait ran out: let the boxes still in flight land before leaving
    for (int i = b + 1; i < min(b + kSlots, nb); ++i) mbar_wait(&full[i % kSlots], (i / kSlots) & 1);
    if (tid == 0) atomicOr(a.flags, 4);
  }
  if (REDUCE) norm_epilogue(acc.value(), a);
}

int line_rows() { return kRows; }

cudaError_t launch_line_pass(int axis, bool reduce, int K, const void* map, const tile_args& a,
                             unsigned blocks, cudaStream_t s) {
  const CUtensorMap& m = *static_cast<const CUtensorMap*>(map);
  if (axis != 1 && axis != 2) return cudaErrorInvalidValue;
#define ROTGP_LP(KK)                                                             \
  if (K == KK) {                                                                 \
    if (axis == 2 && reduce)                                                     \
      k_line_pass<KK, 2, true><<<blocks, 64, 0, s>>>(m, a);                     \
    else if (axis == 2)                                                          \
      k_line_pass<KK, 2, false><<<blocks, 64, 0, s>>>(m, a);                    \
    else if (reduce)                                                             \
      k_line_pass<KK, 1, true><<<blocks, 64, 0, s>>>(m, a);                     \
    else                                                                         \
      k_line_pass<KK, 1, false><<<blocks, 64, 0, s>>>(m, a);                    \
    return cudaGetLastError();                                                   \
  }
  ROTGP_LP(4)
  ROTGP_LP(6)
  ROTGP_LP(8)
#undef ROTGP_LP
  return cudaErrorInvalidValue;
}

}  // namespace rotgp
