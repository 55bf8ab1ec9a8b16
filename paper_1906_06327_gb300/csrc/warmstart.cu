// warmstart.cu -- the learned warm start: a convolutional encoder-decoder
// that proposes an initial wave function for a rotating run from its
// parameters (Omega, g, nu), standing in for the paper's practice (Sec. 1,
// Sec. 3) of starting a fast-rotating imaginary-time run from a converged
// lattice computed beforehand at a lower Omega.  Its proposal only seeds
// imaginary-time propagation, which decides the converged state.
//
// Network (every convolution 3 x 3, stride 1, zero padding 1, channels last):
//   input  6 planes on the G x G grid of the run: the Thomas-Fermi amplitude
//          of the rotating anisotropic trap, x / L, y / L, Omega, g / 1000,
//          (nu - 1) / 0.1 (features_kernel)
//   e0 = relu(conv0(in)), e1 = relu(conv1(e0))                 G,   6->32->32
//   e2 = relu(conv2(pool(e1))), e3 = relu(conv3(e2))           G/2, 32->64->64
//   e4 = relu(conv4(pool(e3))), e5 = relu(conv5(e4))           G/4, 64->128->128
//   b6 = relu(conv6(pool(e5))), b7 = relu(conv7(b6))           G/8, 128->128->128
//   d8 = relu(conv8(up(b7) + e5))                              G/4, 128->64
//   d9 = relu(conv9(up(d8) + e3))                              G/2, 64->32
//   d10 = relu(conv10(up(d9) + e1)), out = conv11(d10)         G,   32->32->2
// (pool = 2 x 2 mean, up = nearest doubling), 684,642 parameters.  out holds
// 2 L psi (real, imaginary parts) on the grid's points 0 .. G-1 of each
// axis (point G, the far edge, is zero).
//
// Precision: weights and activations are stored in bfloat16; every
// convolution, pooling and reduction accumulates in float; weight gradients,
// activation gradients and the Adam state are float, with a float master
// copy of the weights from which the bfloat16 copy is refreshed after every
// update.  The convolution kernels stage an 18 x 18 input patch and the
// weights of 8 input x 32 output channels in shared memory; one thread
// computes the 32 output channels of one pixel of a 16 x 16 tile.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/rotgp.h"
#include "common.cuh"

namespace {

using bf16 = __nv_bfloat16;
using rotgp::splitmix64_unit;

constexpr int kWsCin = 6;
constexpr int kWsLayers = 12;
constexpr int kWsC[kWsLayers][2] = {{kWsCin, 32}, {32, 32},  {32, 64},   {64, 64},
                                    {64, 128},    {128, 128}, {128, 128}, {128, 128},
                                    {128, 64},    {64, 32},   {32, 32},   {32, 2}};
// grid divisor of each layer (G / div)
constexpr int kWsDiv[kWsLayers] = {1, 1, 2, 2, 4, 4, 8, 8, 4, 2, 1, 1};

constexpr int kTile = 16;   // output pixels per tile side
constexpr int kCi = 8;      // input channels per staged chunk
constexpr int kCo = 32;     // output channels per block

__device__ __forceinline__ float ld_act(const bf16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ float ld_act(const float* p) { return *p; }

// ---------------------------------------------------------------- conv
// Forward or backward-data convolution of a [B][H][W][Ci] tensor with 3 x 3
// weights.  Forward: out[., co] = sum_{k, ci} in[p + off_k, ci] w[k][ci][co]
// + bias.  Backward data (BWD): the input is the layer's output gradient dY
// (masked by mask > 0 when mask is given: the ReLU of that layer), and
// out[., ci] = sum_{k, co} dZ[p - off_k, co] w[k][ci][co], i.e. the forward
// form with the flipped kernel and swapped channel roles.  ACC: add into out.
template <class TIn, class TOut, bool BWD>
__global__ void __launch_bounds__(256) k_conv(const TIn* __restrict__ in,
                                              const bf16* __restrict__ mask,
                                              const bf16* __restrict__ w,
                                              const float* __restrict__ bias, TOut* out, int B,
                                              int H, int W, int Ci, int Co, int relu, int acc) {
  __shared__ float sin_[kCi][kTile + 2][kTile + 2];  // channel-major: no bank conflicts
  __shared__ __align__(16) float sw[9][kCi][kCo];
  const int tiles_x = (W + kTile - 1) / kTile, tiles_y = (H + kTile - 1) / kTile;
  const int cob = blockIdx.y * kCo;
  int t = blockIdx.x;
  const int tx = t % tiles_x;
  t /= tiles_x;
  const int ty = t % tiles_y;
  const int b = t / tiles_y;
  const int px = threadIdx.x % kTile, py = threadIdx.x / kTile;
  const int x = tx * kTile + px, y = ty * kTile + py;
  float accv[kCo];
#pragma unroll
  for (int c = 0; c < kCo; ++c) accv[c] = 0.f;
  for (int c0 = 0; c0 < Ci; c0 += kCi) {
    __syncthreads();
    // input patch with a halo of one pixel (zeros outside the image)
    for (int u = threadIdx.x; u < (kTile + 2) * (kTile + 2) * kCi; u += 256) {
      const int c = u % kCi, q = u / kCi, qx = q % (kTile + 2), qy = q / (kTile + 2);
      const int gx = tx * kTile + qx - 1, gy = ty * kTile + qy - 1, gc = c0 + c;
      float v = 0.f;
      if (gx >= 0 && gx < W && gy >= 0 && gy < H && gc < Ci) {
        const size_t i = (((size_t)b * H + gy) * W + gx) * Ci + gc;
        v = ld_act(in + i);
        if (BWD && mask && !(__bfloat162float(mask[i]) > 0.f)) v = 0.f;
      }
      sin_[c][qy][qx] = v;
    }
    // weights of this chunk: forward w[k][ci][co]; backward w[8-k][co][ci]
    for (int u = threadIdx.x; u < 9 * kCi * kCo; u += 256) {
      const int co = u % kCo, c = (u / kCo) % kCi, k = u / (kCo * kCi);
      const int gc = c0 + c, go = cob + co;
      float v = 0.f;
      if (gc < Ci && go < Co) {
        // the layer's weight tensor is [9][layer Ci][layer Co]
        v = BWD ? __bfloat162float(w[((size_t)(8 - k) * Co + go) * Ci + gc])
                : __bfloat162float(w[((size_t)k * Ci + gc) * Co + go]);
      }
      sw[k][c][co] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int ky = k / 3, kx = k % 3;
#pragma unroll
      for (int c = 0; c < kCi; ++c) {
        const float v = sin_[c][py + ky][px + kx];
        const float4* wr = reinterpret_cast<const float4*>(&sw[k][c][0]);
#pragma unroll
        for (int q = 0; q < kCo / 4; ++q) {
          const float4 ww = wr[q];
          accv[4 * q + 0] = fmaf(v, ww.x, accv[4 * q + 0]);
          accv[4 * q + 1] = fmaf(v, ww.y, accv[4 * q + 1]);
          accv[4 * q + 2] = fmaf(v, ww.z, accv[4 * q + 2]);
          accv[4 * q + 3] = fmaf(v, ww.w, accv[4 * q + 3]);
        }
      }
    }
  }
  if (x >= W || y >= H) return;
  const size_t o = (((size_t)b * H + y) * W + x) * Co;
#pragma unroll
  for (int c = 0; c < kCo; ++c) {
    const int go = cob + c;
    if (go >= Co) break;
    float v = accv[c] + (bias ? bias[go] : 0.f);
    if (relu) v = fmaxf(v, 0.f);
    if (acc) v += (float)out[o + go];
    out[o + go] = (TOut)v;
  }
}

// Weight and bias gradients of a convolution: dW[k][ci][co] += sum over
// pixels of X[p + off_k, ci] dZ[p, co], db[co] += sum dZ[p, co], with
// dZ = dY masked by the ReLU of the layer's output.  A block takes 8 input
// x 32 output channels and a run of 16 x 16 tiles of one image; its sums go
// to the gradient with one atomic add per weight.
__global__ void __launch_bounds__(256) k_conv_wgrad(const bf16* __restrict__ X,
                                                    const float* __restrict__ dY,
                                                    const bf16* __restrict__ Yout, int relu,
                                                    float* dW, float* db, int B, int H, int W,
                                                    int Ci, int Co, int tiles_per_block) {
  __shared__ float sx[kTile + 2][kTile + 2][kCi];
  __shared__ float sz[kTile * kTile][kCo + 1];
  const int tiles_x = (W + kTile - 1) / kTile, tiles_y = (H + kTile - 1) / kTile;
  const int ntiles = tiles_x * tiles_y;
  const int runs = (ntiles + tiles_per_block - 1) / tiles_per_block;
  const int c0 = blockIdx.y * kCi, cob = blockIdx.z * kCo;
  const int b = blockIdx.x / runs, run = blockIdx.x % runs;
  const int ci = threadIdx.x / kCo, co = threadIdx.x % kCo;  // 8 x 32 threads
  float acc[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] = 0.f;
  float bacc = 0.f;
  for (int tt = run * tiles_per_block; tt < min(ntiles, (run + 1) * tiles_per_block); ++tt) {
    const int tx = tt % tiles_x, ty = tt / tiles_x;
    __syncthreads();
    for (int u = threadIdx.x; u < (kTile + 2) * (kTile + 2) * kCi; u += 256) {
      const int c = u % kCi, q = u / kCi, qx = q % (kTile + 2), qy = q / (kTile + 2);
      const int gx = tx * kTile + qx - 1, gy = ty * kTile + qy - 1, gc = c0 + c;
      float v = 0.f;
      if (gx >= 0 && gx < W && gy >= 0 && gy < H && gc < Ci)
        v = __bfloat162float(X[(((size_t)b * H + gy) * W + gx) * Ci + gc]);
      sx[qy][qx][c] = v;
    }
    for (int u = threadIdx.x; u < kTile * kTile * kCo; u += 256) {
      const int c = u % kCo, q = u / kCo, qx = q % kTile, qy = q / kTile;
      const int gx = tx * kTile + qx, gy = ty * kTile + qy, go = cob + c;
      float v = 0.f;
      if (gx < W && gy < H && go < Co) {
        const size_t i = (((size_t)b * H + gy) * W + gx) * Co + go;
        v = dY[i];
        if (relu && !(__bfloat162float(Yout[i]) > 0.f)) v = 0.f;
      }
      sz[q][c] = v;
    }
    __syncthreads();
    for (int q = 0; q < kTile * kTile; ++q) {
      const int qx = q % kTile, qy = q / kTile;
      const float dz = sz[q][co];
#pragma unroll
      for (int k = 0; k < 9; ++k) acc[k] = fmaf(sx[qy + k / 3][qx + k % 3][ci], dz, acc[k]);
      if (ci == 0) bacc += dz;
    }
  }
  const int gc = c0 + ci, go = cob + co;
  if (gc < Ci && go < Co) {
#pragma unroll
    for (int k = 0; k < 9; ++k) atomicAdd(&dW[((size_t)k * Ci + gc) * Co + go], acc[k]);
    // the bias gradient once, from the blocks of the first input-channel chunk
    if (ci == 0 && blockIdx.y == 0) atomicAdd(&db[go], bacc);
  }
}

// ---------------------------------------------------------------- glue
// out = mean of each 2 x 2 block of in ([B][2h][2w][C] -> [B][h][w][C])
__global__ void k_pool(const bf16* in, bf16* out, int B, int h, int w, int C) {
  const size_t n = (size_t)B * h * w * C;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    size_t r = i / C;
    const int x = (int)(r % w);
    r /= w;
    const int y = (int)(r % h);
    const int b = (int)(r / h);
    const size_t W2 = 2 * (size_t)w;
    const size_t base = (((size_t)b * 2 * h + 2 * y) * W2 + 2 * x) * C + c;
    const float s = __bfloat162float(in[base]) + __bfloat162float(in[base + C]) +
                    __bfloat162float(in[base + W2 * C]) + __bfloat162float(in[base + W2 * C + C]);
    out[i] = __float2bfloat16(0.25f * s);
  }
}
// gin[2x2 block] += gout / 4
__global__ void k_pool_bwd(const float* gout, float* gin, int B, int h, int w, int C) {
  const size_t n = (size_t)B * h * w * C;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    size_t r = i / C;
    const int x = (int)(r % w);
    r /= w;
    const int y = (int)(r % h);
    const int b = (int)(r / h);
    const size_t W2 = 2 * (size_t)w;
    const size_t base = (((size_t)b * 2 * h + 2 * y) * W2 + 2 * x) * C + c;
    const float g = 0.25f * gout[i];
    gin[base] += g;
    gin[base + C] += g;
    gin[base + W2 * C] += g;
    gin[base + W2 * C + C] += g;
  }
}
// out = up(a) + skip ([B][h][w][C] doubled, plus [B][2h][2w][C])
__global__ void k_up_add(const bf16* a, const bf16* skip, bf16* out, int B, int h, int w, int C) {
  const size_t n = (size_t)B * 4 * h * w * C;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    size_t r = i / C;
    const int x = (int)(r % (2 * w));
    r /= 2 * w;
    const int y = (int)(r % (2 * h));
    const int b = (int)(r / (2 * h));
    const float v = __bfloat162float(a[(((size_t)b * h + y / 2) * w + x / 2) * C + c]) +
                    __bfloat162float(skip[i]);
    out[i] = __float2bfloat16(v);
  }
}
// ga = sum of each 2 x 2 block of g; gskip = g (the skip's gradient starts here)
__global__ void k_up_add_bwd(const float* g, float* ga, float* gskip, int B, int h, int w, int C) {
  const size_t n = (size_t)B * h * w * C;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    size_t r = i / C;
    const int x = (int)(r % w);
    r /= w;
    const int y = (int)(r % h);
    const int b = (int)(r / h);
    const size_t W2 = 2 * (size_t)w;
    const size_t base = (((size_t)b * 2 * h + 2 * y) * W2 + 2 * x) * C + c;
    ga[i] = g[base] + g[base + C] + g[base + W2 * C] + g[base + W2 * C + C];
  }
  const size_t n4 = 4 * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4;
       i += (size_t)gridDim.x * blockDim.x)
    gskip[i] = g[i];
}

// Loss sum((y - t)^2) into per-block partials and its gradient 2 (y - t) / n.
__global__ void k_mse(const float* y, const float* t, float* dy, double* part, size_t n) {
  __shared__ double ws[8];
  double s = 0;
  const float inv = 2.0f / (float)n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    s += (double)d * d;
    dy[i] = inv * d;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += ws[i];
    part[blockIdx.x] = tot;
  }
}

// Adam on the float master weights, then their bfloat16 copy.
__global__ void k_adam(float* p, bf16* pb, const float* g, float* m, float* v, size_t n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
    const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
    m[i] = mi;
    v[i] = vi;
    const float w = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = w;
    pb[i] = __float2bfloat16(w);
  }
}

__global__ void k_to_bf16(const float* in, bf16* out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16(in[i]);
}

// Input planes of run i (Omega, g, nu = prm[3i..3i+2]) on the G x G points
// x_j = -L + j h of both axes (h = 2 L / G): the Thomas-Fermi amplitude of
// the rotating trap, sqrt(max(0, mu - (gx^2 x^2 + gy^2 y^2) / 2) / g) with
// the centrifugally reduced frequencies gx^2 = 1 - Omega^2, gy^2 = nu^2 -
// Omega^2 and mu = sqrt(g gx gy / pi) (unit norm), scaled by 2 L; then x / L,
// y / L, Omega, g / 1000, (nu - 1) / 0.1.
__global__ void k_features(const double* prm, bf16* out, int n, int G, double L) {
  const size_t tot = (size_t)n * G * G;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < tot;
       i += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(i % G), k = (int)((i / G) % G), r = (int)(i / ((size_t)G * G));
    const double om = prm[3 * r], g = prm[3 * r + 1], nu = prm[3 * r + 2];
    const double h = 2.0 * L / G, x = -L + j * h, y = -L + k * h;
    const double gx2 = fmax(1.0 - om * om, 1e-3), gy2 = fmax(nu * nu - om * om, 1e-3);
    const double mu = sqrt(g * sqrt(gx2 * gy2) / 3.14159265358979323846);
    const double n_tf = fmax(0.0, mu - 0.5 * (gx2 * x * x + gy2 * y * y)) / g;
    bf16* o = out + i * kWsCin;
    o[0] = __float2bfloat16((float)(2.0 * L * sqrt(n_tf)));
    o[1] = __float2bfloat16((float)(x / L));
    o[2] = __float2bfloat16((float)(y / L));
    o[3] = __float2bfloat16((float)om);
    o[4] = __float2bfloat16((float)(g / 1000.0));
    o[5] = __float2bfloat16((float)((nu - 1.0) / 0.1));
  }
}

// Network output (2 L psi on G x G points) -> ABI wave function of run i:
// (G+1) x (G+1) complex double, psi = out / (2 L), the far edge zero; with
// rp != 0 multiplied by the random phase exp(2 pi i R) of Eq. fun, R drawn
// from SplitMix64(seed) for point n = k (G + 1) + j as rotgp_init_analytic
// draws it.
__global__ void k_out_to_psi(const float* y, double* psi, int n, int G, double L, int rp,
                             unsigned long long seed) {
  const size_t P = (size_t)(G + 1) * (G + 1), tot = (size_t)n * P;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < tot;
       i += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(i / P);
    const size_t q = i % P;
    const int j = (int)(q % (G + 1)), k = (int)(q / (G + 1));
    double re = 0, im = 0;
    if (j < G && k < G && j > 0 && k > 0) {
      const float* v = y + (((size_t)r * G + k) * G + j) * 2;
      re = v[0] / (2.0 * L);
      im = v[1] / (2.0 * L);
      if (rp) {
        double sn, cs;
        sincos(2.0 * 3.14159265358979323846 * splitmix64_unit(seed, q), &sn, &cs);
        const double a = re * cs - im * sn;
        im = re * sn + im * cs;
        re = a;
      }
    }
    psi[2 * i] = re;
    psi[2 * i + 1] = im;
  }
}

// ABI wave functions ((G+1)^2 complex double) -> targets 2 L psi on G x G.
__global__ void k_psi_to_target(const double* psi, float* t, int n, int G, double L) {
  const size_t tot = (size_t)n * G * G;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < tot;
       i += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(i % G), k = (int)((i / G) % G), r = (int)(i / ((size_t)G * G));
    const double* v = psi + 2 * (((size_t)r * (G + 1) + k) * (G + 1) + j);
    t[2 * i] = (float)(2.0 * L * v[0]);
    t[2 * i + 1] = (float)(2.0 * L * v[1]);
  }
}

int blocks_for(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 152 * 16); }

}  // namespace

// ---------------------------------------------------------------- context
struct rotgp_ws {
  int G = 0, maxb = 0;
  cudaStream_t s = nullptr;
  size_t np = 0;
  std::vector<size_t> woff, boff;  // offsets of each layer's weights and bias
  float* p = nullptr;              // float master
  bf16* pb = nullptr;              // bfloat16 copy (weights; biases read as float master)
  float *g = nullptr, *m = nullptr, *v = nullptr;
  long long t = 0;                 // Adam step
  double* dprm = nullptr;          // run parameters (3 per run)
  bf16* x = nullptr;               // input planes
  bf16* act[kWsLayers] = {};       // layer outputs (the last one unused)
  bf16 *p1 = nullptr, *p2 = nullptr, *p3 = nullptr;  // pooled
  bf16 *s8 = nullptr, *s9 = nullptr, *s10 = nullptr; // up + skip sums
  float* y = nullptr;              // network output
  float* tgt = nullptr;            // targets
  float *gA = nullptr, *gB = nullptr, *gS1 = nullptr, *gS2 = nullptr, *gS3 = nullptr;
  double* part = nullptr;
  double* dpsi = nullptr;          // ABI wave functions (in or out)
  std::string err;
  size_t bytes = 0;
};

namespace {

thread_local std::string g_ws_error;

int wfail(rotgp_ws* w, int code, const char* msg, cudaError_t e = cudaSuccess) {
  std::string m = msg;
  if (e != cudaSuccess) m += std::string(": ") + cudaGetErrorString(e);
  if (w)
    w->err = m;
  else
    g_ws_error = m;
  return code;
}

template <class P>
cudaError_t walloc(rotgp_ws* w, P** p, size_t n) {
  w->bytes += n * sizeof(P);
  return cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(P));
}

size_t plane(const rotgp_ws* w, int layer, int c) {
  const size_t d = (size_t)w->G / kWsDiv[layer];
  return (size_t)w->maxb * d * d * c;
}

template <class TIn, class TOut, bool BWD>
cudaError_t conv(rotgp_ws* w, const TIn* in, const bf16* mask, int layer, TOut* out, int B,
                 int relu, int acc) {
  const int d = w->G / kWsDiv[layer];
  const int Ci = BWD ? kWsC[layer][1] : kWsC[layer][0];
  const int Co = BWD ? kWsC[layer][0] : kWsC[layer][1];
  const int tiles = ((d + kTile - 1) / kTile) * ((d + kTile - 1) / kTile);
  dim3 grid((unsigned)(tiles * B), (unsigned)((Co + kCo - 1) / kCo));
  const float* bias = BWD ? nullptr : w->p + w->boff[layer];
  k_conv<TIn, TOut, BWD><<<grid, 256, 0, w->s>>>(in, mask, w->pb + w->woff[layer], bias, out, B,
                                                 d, d, Ci, Co, relu, acc);
  return cudaGetLastError();
}

cudaError_t wgrad(rotgp_ws* w, const bf16* X, const float* dY, const bf16* Yout, int layer,
                  int B) {
  const int d = w->G / kWsDiv[layer];
  const int Ci = kWsC[layer][0], Co = kWsC[layer][1];
  const int tiles = ((d + kTile - 1) / kTile) * ((d + kTile - 1) / kTile);
  const int tpb = std::max(1, std::min(tiles, 8));
  const int runs = (tiles + tpb - 1) / tpb;
  dim3 grid((unsigned)(B * runs), (unsigned)((Ci + kCi - 1) / kCi), (unsigned)((Co + kCo - 1) / kCo));
  k_conv_wgrad<<<grid, 256, 0, w->s>>>(X, dY, Yout, layer < kWsLayers - 1 ? 1 : 0,
                                       w->g + w->woff[layer], w->g + w->boff[layer], B, d, d, Ci,
                                       Co, tpb);
  return cudaGetLastError();
}

// Forward pass of B runs whose input planes are in w->x; output in w->y.
cudaError_t forward(rotgp_ws* w, int B) {
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  const int G = w->G;
  chk(conv<bf16, bf16, false>(w, w->x, nullptr, 0, w->act[0], B, 1, 0));
  chk(conv<bf16, bf16, false>(w, w->act[0], nullptr, 1, w->act[1], B, 1, 0));
  k_pool<<<blocks_for((size_t)B * G * G / 4 * 32), 256, 0, w->s>>>(w->act[1], w->p1, B, G / 2, G / 2, 32);
  chk(conv<bf16, bf16, false>(w, w->p1, nullptr, 2, w->act[2], B, 1, 0));
  chk(conv<bf16, bf16, false>(w, w->act[2], nullptr, 3, w->act[3], B, 1, 0));
  k_pool<<<blocks_for((size_t)B * G * G / 16 * 64), 256, 0, w->s>>>(w->act[3], w->p2, B, G / 4, G / 4, 64);
  chk(conv<bf16, bf16, false>(w, w->p2, nullptr, 4, w->act[4], B, 1, 0));
  chk(conv<bf16, bf16, false>(w, w->act[4], nullptr, 5, w->act[5], B, 1, 0));
  k_pool<<<blocks_for((size_t)B * G * G / 64 * 128), 256, 0, w->s>>>(w->act[5], w->p3, B, G / 8, G / 8, 128);
  chk(conv<bf16, bf16, false>(w, w->p3, nullptr, 6, w->act[6], B, 1, 0));
  chk(conv<bf16, bf16, false>(w, w->act[6], nullptr, 7, w->act[7], B, 1, 0));
  k_up_add<<<blocks_for((size_t)B * G * G / 16 * 128), 256, 0, w->s>>>(w->act[7], w->act[5], w->s8, B, G / 8, G / 8, 128);
  chk(conv<bf16, bf16, false>(w, w->s8, nullptr, 8, w->act[8], B, 1, 0));
  k_up_add<<<blocks_for((size_t)B * G * G / 4 * 64), 256, 0, w->s>>>(w->act[8], w->act[3], w->s9, B, G / 4, G / 4, 64);
  chk(conv<bf16, bf16, false>(w, w->s9, nullptr, 9, w->act[9], B, 1, 0));
  k_up_add<<<blocks_for((size_t)B * G * G * 32), 256, 0, w->s>>>(w->act[9], w->act[1], w->s10, B, G / 2, G / 2, 32);
  chk(conv<bf16, bf16, false>(w, w->s10, nullptr, 10, w->act[10], B, 1, 0));
  chk(conv<bf16, float, false>(w, w->act[10], nullptr, 11, w->y, B, 0, 0));
  chk(cudaGetLastError());
  return e;
}

// Backward pass from dL/dy in w->gA (float, [B][G][G][2]); weight gradients
// accumulate into w->g (zeroed by the caller).
cudaError_t backward(rotgp_ws* w, int B) {
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  const int G = w->G;
  float *gA = w->gA, *gB = w->gB;
  // layer 11 (linear): dW from d10 and dy; d(d10) = conv^T(dy)
  chk(wgrad(w, w->act[10], gA, nullptr, 11, B));
  chk(conv<float, float, true>(w, gA, nullptr, 11, gB, B, 0, 0));
  // layer 10: input s10 = up(d9) + e1
  chk(wgrad(w, w->s10, gB, w->act[10], 10, B));
  chk(conv<float, float, true>(w, gB, w->act[10], 10, gA, B, 0, 0));  // gA = d(s10)
  k_up_add_bwd<<<blocks_for((size_t)B * G * G / 4 * 32), 256, 0, w->s>>>(gA, gB, w->gS1, B, G / 2, G / 2, 32);
  // gB = d(d9); layer 9: input s9 = up(d8) + e3
  chk(wgrad(w, w->s9, gB, w->act[9], 9, B));
  chk(conv<float, float, true>(w, gB, w->act[9], 9, gA, B, 0, 0));    // gA = d(s9)
  k_up_add_bwd<<<blocks_for((size_t)B * G * G / 16 * 64), 256, 0, w->s>>>(gA, gB, w->gS2, B, G / 4, G / 4, 64);
  // gB = d(d8); layer 8: input s8 = up(b7) + e5
  chk(wgrad(w, w->s8, gB, w->act[8], 8, B));
  chk(conv<float, float, true>(w, gB, w->act[8], 8, gA, B, 0, 0));    // gA = d(s8)
  k_up_add_bwd<<<blocks_for((size_t)B * G * G / 64 * 128), 256, 0, w->s>>>(gA, gB, w->gS3, B, G / 8, G / 8, 128);
  // gB = d(b7); layer 7
  chk(wgrad(w, w->act[6], gB, w->act[7], 7, B));
  chk(conv<float, float, true>(w, gB, w->act[7], 7, gA, B, 0, 0));    // gA = d(b6)
  // layer 6: input pool(e5)
  chk(wgrad(w, w->p3, gA, w->act[6], 6, B));
  chk(conv<float, float, true>(w, gA, w->act[6], 6, gB, B, 0, 0));    // gB = d(p3)
  k_pool_bwd<<<blocks_for((size_t)B * G * G / 64 * 128), 256, 0, w->s>>>(gB, w->gS3, B, G / 8, G / 8, 128);
  // gS3 = d(e5); layer 5
  chk(wgrad(w, w->act[4], w->gS3, w->act[5], 5, B));
  chk(conv<float, float, true>(w, w->gS3, w->act[5], 5, gA, B, 0, 0)); // gA = d(e4)
  chk(wgrad(w, w->p2, gA, w->act[4], 4, B));
  chk(conv<float, float, true>(w, gA, w->act[4], 4, gB, B, 0, 0));    // gB = d(p2)
  k_pool_bwd<<<blocks_for((size_t)B * G * G / 16 * 64), 256, 0, w->s>>>(gB, w->gS2, B, G / 4, G / 4, 64);
  // gS2 = d(e3); layer 3
  chk(wgrad(w, w->act[2], w->gS2, w->act[3], 3, B));
  chk(conv<float, float, true>(w, w->gS2, w->act[3], 3, gA, B, 0, 0)); // gA = d(e2)
  chk(wgrad(w, w->p1, gA, w->act[2], 2, B));
  chk(conv<float, float, true>(w, gA, w->act[2], 2, gB, B, 0, 0));    // gB = d(p1)
  k_pool_bwd<<<blocks_for((size_t)B * G * G / 4 * 32), 256, 0, w->s>>>(gB, w->gS1, B, G / 2, G / 2, 32);
  // gS1 = d(e1); layer 1
  chk(wgrad(w, w->act[0], w->gS1, w->act[1], 1, B));
  chk(conv<float, float, true>(w, w->gS1, w->act[1], 1, gA, B, 0, 0)); // gA = d(e0)
  chk(wgrad(w, w->x, gA, w->act[0], 0, B));
  chk(cudaGetLastError());
  return e;
}

int check_batch(rotgp_ws* w, int n) {
  if (!w) return ROTGP_EINVAL;
  if (n < 1 || n > w->maxb) return wfail(w, ROTGP_EINVAL, "batch size out of range");
  return ROTGP_OK;
}

// parameters of n runs (host, 3 n doubles: Omega, g, nu) -> input planes
int load_features(rotgp_ws* w, int n, const double* prm, double L) {
  cudaError_t e = cudaMemcpyAsync(w->dprm, prm, 3 * n * sizeof(double), cudaMemcpyHostToDevice, w->s);
  if (e != cudaSuccess) return wfail(w, ROTGP_ECUDA, "copy parameters", e);
  k_features<<<blocks_for((size_t)n * w->G * w->G), 256, 0, w->s>>>(w->dprm, w->x, n, w->G, L);
  e = cudaGetLastError();
  return e == cudaSuccess ? ROTGP_OK : wfail(w, ROTGP_ECUDA, "features kernel", e);
}

// targets from n ABI wave functions (host or device, complex double)
int load_targets(rotgp_ws* w, int n, const double* psi, int on_device, double L) {
  const size_t P = (size_t)(w->G + 1) * (w->G + 1) * 2 * n;
  const double* src = psi;
  if (!on_device) {
    cudaError_t e = cudaMemcpyAsync(w->dpsi, psi, P * sizeof(double), cudaMemcpyHostToDevice, w->s);
    if (e != cudaSuccess) return wfail(w, ROTGP_ECUDA, "copy targets", e);
    src = w->dpsi;
  }
  k_psi_to_target<<<blocks_for((size_t)n * w->G * w->G), 256, 0, w->s>>>(src, w->tgt, n, w->G, L);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ROTGP_OK : wfail(w, ROTGP_ECUDA, "target kernel", e);
}

// loss and gradients of n runs (features and targets loaded); loss to host
int loss_and_grad(rotgp_ws* w, int n, double* loss) {
  cudaError_t e = forward(w, n);
  const size_t ny = (size_t)n * w->G * w->G * 2;
  const int nb = 256;
  if (e == cudaSuccess) {
    k_mse<<<nb, 256, 0, w->s>>>(w->y, w->tgt, w->gA, w->part, ny);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(w->g, 0, w->np * sizeof(float), w->s);
  if (e == cudaSuccess) e = backward(w, n);
  double parts[256];
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(parts, w->part, sizeof parts, cudaMemcpyDeviceToHost, w->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(w->s);
  if (e != cudaSuccess) return wfail(w, ROTGP_ECUDA, "network pass", e);
  double s = 0;
  for (double x : parts) s += x;
  if (loss) *loss = s / (double)ny;
  return ROTGP_OK;
}

}  // namespace

// =============================================================== C ABI
extern "C" {

long long rotgp_ws_param_count(void) {
  long long n = 0;
  for (const auto& c : kWsC) n += 9LL * c[0] * c[1] + c[1];
  return n;
}

const char* rotgp_ws_last_error(const rotgp_ws* w) { return w ? w->err.c_str() : g_ws_error.c_str(); }

void rotgp_ws_destroy(rotgp_ws* w) {
  if (!w) return;
  cudaStreamSynchronize(w->s);
  void* ptrs[] = {w->p, w->pb, w->g, w->m, w->v, w->dprm, w->x, w->p1, w->p2, w->p3, w->s8,
                  w->s9, w->s10, w->y, w->tgt, w->gA, w->gB, w->gS1, w->gS2, w->gS3, w->part,
                  w->dpsi};
  for (void* p : ptrs) cudaFree(p);
  for (auto* a : w->act) cudaFree(a);
  delete w;
}

int rotgp_ws_create(int grid, int max_batch, void* stream, rotgp_ws** out) {
  g_ws_error.clear();
  if (!out) return wfail(nullptr, ROTGP_EINVAL, "null output");
  *out = nullptr;
  if (grid < 16 || grid % 16 != 0 || grid > 1024)
    return wfail(nullptr, ROTGP_EINVAL, "grid must be a multiple of 16 in [16, 1024]");
  if (max_batch < 1 || max_batch > 4096) return wfail(nullptr, ROTGP_EINVAL, "max_batch out of range");
  rotgp_ws* w = new (std::nothrow) rotgp_ws();
  if (!w) return wfail(nullptr, ROTGP_ENOMEM, "host allocation failed");
  w->G = grid;
  w->maxb = max_batch;
  w->s = static_cast<cudaStream_t>(stream);
  size_t off = 0;
  for (const auto& c : kWsC) {
    w->woff.push_back(off);
    off += 9 * (size_t)c[0] * c[1];
    w->boff.push_back(off);
    off += c[1];
  }
  w->np = off;
  const size_t G2 = (size_t)grid * grid * max_batch;
  cudaError_t e = walloc(w, &w->p, w->np);
  if (e == cudaSuccess) e = walloc(w, &w->pb, w->np);
  if (e == cudaSuccess) e = walloc(w, &w->g, w->np);
  if (e == cudaSuccess) e = walloc(w, &w->m, w->np);
  if (e == cudaSuccess) e = walloc(w, &w->v, w->np);
  if (e == cudaSuccess) e = walloc(w, &w->dprm, 3 * (size_t)max_batch);
  if (e == cudaSuccess) e = walloc(w, &w->x, G2 * kWsCin);
  for (int l = 0; l < kWsLayers && e == cudaSuccess; ++l)
    e = walloc(w, &w->act[l], plane(w, l, kWsC[l][1]));
  if (e == cudaSuccess) e = walloc(w, &w->p1, G2 / 4 * 32);
  if (e == cudaSuccess) e = walloc(w, &w->p2, G2 / 16 * 64);
  if (e == cudaSuccess) e = walloc(w, &w->p3, G2 / 64 * 128);
  if (e == cudaSuccess) e = walloc(w, &w->s8, G2 / 16 * 128);
  if (e == cudaSuccess) e = walloc(w, &w->s9, G2 / 4 * 64);
  if (e == cudaSuccess) e = walloc(w, &w->s10, G2 * 32);
  if (e == cudaSuccess) e = walloc(w, &w->y, G2 * 2);
  if (e == cudaSuccess) e = walloc(w, &w->tgt, G2 * 2);
  if (e == cudaSuccess) e = walloc(w, &w->gA, G2 * 32);
  if (e == cudaSuccess) e = walloc(w, &w->gB, G2 * 32);
  if (e == cudaSuccess) e = walloc(w, &w->gS1, G2 * 32);
  if (e == cudaSuccess) e = walloc(w, &w->gS2, G2 / 4 * 64);
  if (e == cudaSuccess) e = walloc(w, &w->gS3, G2 / 16 * 128);
  if (e == cudaSuccess) e = walloc(w, &w->part, 256);
  if (e == cudaSuccess) e = walloc(w, &w->dpsi, (size_t)(grid + 1) * (grid + 1) * 2 * max_batch);
  if (e == cudaSuccess) e = cudaMemsetAsync(w->m, 0, w->np * sizeof(float), w->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(w->v, 0, w->np * sizeof(float), w->s);
  if (e != cudaSuccess) {
    const int rc = wfail(nullptr, e == cudaErrorMemoryAllocation ? ROTGP_ENOMEM : ROTGP_ECUDA,
                         "network buffers", e);
    rotgp_ws_destroy(w);
    return rc;
  }
  *out = w;
  return ROTGP_OK;
}

int rotgp_ws_set_params(rotgp_ws* w, const float* params) {
  if (!w || !params) return w ? wfail(w, ROTGP_EINVAL, "null parameters") : ROTGP_EINVAL;
  cudaError_t e = cudaMemcpyAsync(w->p, params, w->np * sizeof(float), cudaMemcpyHostToDevice, w->s);
  if (e == cudaSuccess) {
    k_to_bf16<<<blocks_for(w->np), 256, 0, w->s>>>(w->p, w->pb, w->np);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(w->m, 0, w->np * sizeof(float), w->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(w->v, 0, w->np * sizeof(float), w->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(w->s);
  w->t = 0;
  return e == cudaSuccess ? ROTGP_OK : wfail(w, ROTGP_ECUDA, "set parameters", e);
}

int rotgp_ws_get_params(rotgp_ws* w, float* params) {
  if (!w || !params) return w ? wfail(w, ROTGP_EINVAL, "null parameters") : ROTGP_EINVAL;
  cudaError_t e = cudaMemcpyAsync(params, w->p, w->np * sizeof(float), cudaMemcpyDeviceToHost, w->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(w->s);
  return e == cudaSuccess ? ROTGP_OK : wfail(w, ROTGP_ECUDA, "get parameters", e);
}

int rotgp_ws_propose(rotgp_ws* w, int n, const double* prm, double half_width, int random_phase,
                     unsigned long long seed, void* psi, int psi_on_device) {
  int rc = check_batch(w, n);
  if (rc) return rc;
  if (!prm || !psi || !(half_width > 0)) return wfail(w, ROTGP_EINVAL, "bad arguments");
  if ((rc = load_features(w, n, prm, half_width))) return rc;
  cudaError_t e = forward(w, n);
  double* dst = psi_on_device ? static_cast<double*>(psi) : w->dpsi;
  if (e == cudaSuccess) {
    k_out_to_psi<<<blocks_for((size_t)n * (w->G + 1) * (w->G + 1)), 256, 0, w->s>>>(
        w->y, dst, n, w->G, half_width, random_phase ? 1 : 0, seed);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !psi_on_device)
    e = cudaMemcpyAsync(psi, w->dpsi, (size_t)n * (w->G + 1) * (w->G + 1) * 2 * sizeof(double),
                        cudaMemcpyDeviceToHost, w->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(w->s);
  return e == cudaSuccess ? ROTGP_OK : wfail(w, ROTGP_ECUDA, "propose", e);
}

int rotgp_ws_gradients(rotgp_ws* w, int n, const void* inputs, const float* targets, double* loss,
                       float* grads) {
  int rc = check_batch(w, n);
  if (rc) return rc;
  if (!inputs || !targets) return wfail(w, ROTGP_EINVAL, "null inputs or targets");
  const size_t G2 = (size_t)n * w->G * w->G;
  // input planes as float on the host -> bfloat16 on the device
  float* tmp = nullptr;
  cudaError_t e = cudaMalloc((void**)&tmp, G2 * kWsCin * sizeof(float));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(tmp, inputs, G2 * kWsCin * sizeof(float), cudaMemcpyHostToDevice, w->s);
  if (e == cudaSuccess) {
    k_to_bf16<<<blocks_for(G2 * kWsCin), 256, 0, w->s>>>(tmp, w->x, G2 * kWsCin);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w->tgt, targets, G2 * 2 * sizeof(float), cudaMemcpyHostToDevice, w->s);
  if (e != cudaSuccess) {
    cudaFree(tmp);
    return wfail(w, ROTGP_ECUDA, "gradient inputs", e);
  }
  rc = loss_and_grad(w, n, loss);
  cudaFree(tmp);
  if (rc) return rc;
  if (grads) {
    e = cudaMemcpy(grads, w->g, w->np * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return wfail(w, ROTGP_ECUDA, "copy gradients", e);
  }
  return ROTGP_OK;
}

int rotgp_ws_train_step(rotgp_ws* w, int n, const double* prm, double half_width,
                        const void* psi, int psi_on_device, float lr, double* loss) {
  int rc = check_batch(w, n);
  if (rc) return rc;
  if (!prm || !psi || !(half_width > 0) || !(lr > 0))
    return wfail(w, ROTGP_EINVAL, "bad arguments");
  if ((rc = load_features(w, n, prm, half_width))) return rc;
  if ((rc = load_targets(w, n, static_cast<const double*>(psi), psi_on_device, half_width)))
    return rc;
  if ((rc = loss_and_grad(w, n, loss))) return rc;
  ++w->t;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)w->t), c2 = 1.f - powf(b2, (float)w->t);
  k_adam<<<blocks_for(w->np), 256, 0, w->s>>>(w->p, w->pb, w->g, w->m, w->v, w->np, lr, b1, b2,
                                              1e-8f, c1, c2);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ROTGP_OK : wfail(w, ROTGP_ECUDA, "optimiser step", e);
}

}  // extern "C"
