// batch_kernel.cu -- many 2D condensates advanced by ONE persistent kernel
// launch for a whole block of split steps (the batched workload: instances of
// uneven grid sizes and differing Omega, g and trap anisotropy).
//
// Each split step of every instance is the exact line solve of hybrid.cuh on
// whole lines (one CTA per tile of 16 lines, no cluster): phase X runs H1 and
// the x sweep of every tile of every active instance, phase Y the y sweep and
// each tile's share of the norm.  The CTAs of one cooperative launch take the
// tiles of a phase from a fixed work list (tile w goes to CTA w mod grid) and
// meet at a grid barrier between phases; nothing returns to the host between
// steps.  The barrier is a counter and a generation word in global memory:
// each CTA waits for the generation to move for at most about 2 s of device
// time, after which it sets a flag and leaves (every other CTA leaves at its
// next barrier), so a stalled launch ends with ROTGP_ETIMEOUT on the host
// instead of hanging.
//
// The imaginary-time renormalisation of a step (Sec. 2) is read by the next
// step's X tiles from the instance's Y-tile partial sums, which every X tile
// combines in the same fixed order, so all tiles of an instance apply the
// same scale; the order is the one of the single-context sweep's norm
// reduction, and the tile solves are the same code, so an instance advanced
// here equals, bit for bit, the same instance advanced alone with the exact
// line solve on whole lines.
#include <algorithm>
#include <vector>

#include "hybrid.cuh"

namespace rotgp {

namespace {

// One instance as the kernel sees it.
struct binst {
  void* psi[2];
  const void* tab[2][2];  // [axis][mode] coef5 tables
  double* scale;          // the context's pending scale and norm
  double* norm;
  int* flags;
  int nx, ny, lt, cur;
  int pcx, lsx, pcy, lsy;  // whole-line tile shapes of the x and y sweeps
  int ytile0, ytiles;      // this instance's slots of the norm partials
  int vec;
  double dt, g, hgam2, hnu2, x0, hx, y0, hy, vol;
};

struct bwork {
  int inst, grp;
};

struct batch_args {
  const binst* inst;
  int ninst;
  const bwork* xw;
  int nxw;
  const bwork* yw;
  int nyw;
  double* partials;  // one per y tile of every instance
  unsigned* bar;     // grid barrier: [0] arrivals, [1] generation
  int* bflags;       // bit 3: a barrier wait gave up
  long long nsteps;
};

// Wait until every CTA of the launch has arrived; false if the wait gave up
// (after ~2 s of device time, or when another CTA already gave up).
__device__ bool grid_barrier(unsigned* bar, int* bflags) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u) + 1u;
    int good = 1;
    if (arrived == gridDim.x) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == gen) {
        if (*(volatile int*)bflags & 8) {
          good = 0;
          break;
        }
        if (clock64() - t0 > 4000000000LL) {
          atomicOr(bflags, 8);
          good = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// Block sum of v in the order of the single-context norm reduction (warp
// sums, then the warps in order); the value is returned to thread 0.
__device__ double block_sum(double v) {
  __shared__ double ws[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) ws[warp] = v;
  __syncthreads();
  double s = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < nw; ++w) s += ws[w];
  return s;
}

// Sum of an instance's y-tile partials, as the last block of the
// single-context reduction combines its blocks' partials; every thread
// receives it.
__device__ double partials_sum(const double* p, int n) {
  __shared__ double ws[32];
  __shared__ double tot;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double s = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += __ldcg(&p[i]);
  s = warp_sum(s);
  __syncthreads();
  if (lane == 0) ws[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < nw; ++w) t += ws[w];
    tot = t;
  }
  __syncthreads();
  return tot;
}

template <class T, bool IMAG>
__global__ void __launch_bounds__(kHThreads, sizeof(T) == 4 ? 2 : 1) k_batch_steps(const batch_args b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (long long step = 0; step < b.nsteps; ++step) {
    // ---- phase X: H1 (with the pending scale) and the x sweep
    for (int w = blockIdx.x; w < b.nxw; w += gridDim.x) {
      const bwork wk = b.xw[w];
      const binst& I = b.inst[wk.inst];
      double scale = 1.0;
      if (step == 0) {
        scale = *I.scale;
      } else if (IMAG) {
        const double n = partials_sum(b.partials + I.ytile0, I.ytiles) * I.vol;
        scale = (n > 0.0 && isfinite(n)) ? 1.0 / sqrt(n) : 1.0;
      }
      stream_args a{};
      a.in = I.psi[I.cur];
      a.out = I.psi[1 - I.cur];
      a.coef = I.tab[0][IMAG ? 1 : 0];
      a.len = I.nx;
      a.lt = I.lt;
      a.nlines = I.ny;
      a.nx = I.nx;
      a.ny = I.ny;
      a.dt = I.dt;
      a.g = I.g;
      a.hgam2 = I.hgam2;
      a.hnu2 = I.hnu2;
      a.hlam2 = 0.0;
      a.x0 = I.x0;
      a.hx = I.hx;
      a.y0 = I.y0;
      a.hy = I.hy;
      a.z0 = 0.0;
      a.hz = 0.0;
      hybrid_job J;
      J.grp = wk.grp;
      J.rank = 0;
      J.cs = 1;
      J.pc = I.pcx;
      J.lsub = I.lsx;
      J.vec = I.vec;
      J.scale = scale;
      hybrid_tile<T, 0, true, IMAG, false>(a, J, smem_raw);
    }
    if (!grid_barrier(b.bar, b.bflags)) return;
    // ---- phase Y: the y sweep and each tile's part of the norm
    for (int w = blockIdx.x; w < b.nyw; w += gridDim.x) {
      const bwork wk = b.yw[w];
      const binst& I = b.inst[wk.inst];
      stream_args a{};
      a.in = I.psi[1 - I.cur];
      a.out = I.psi[I.cur];
      a.coef = I.tab[1][IMAG ? 1 : 0];
      a.len = I.ny;
      a.lt = I.lt;
      a.nlines = I.nx;
      a.nx = I.nx;
      a.ny = I.ny;
      a.stride = I.nx;
      a.outer = (long long)I.nx * I.ny;
      hybrid_job J;
      J.grp = wk.grp;
      J.rank = 0;
      J.cs = 1;
      J.pc = I.pcy;
      J.lsub = I.lsy;
      J.vec = I.vec;
      J.scale = 1.0;
      const double v = hybrid_tile<T, 1, false, false, true>(a, J, smem_raw);
      const double bs = block_sum(v);
      if (threadIdx.x == 0) b.partials[I.ytile0 + wk.grp] = bs;
    }
    if (!grid_barrier(b.bar, b.bflags)) return;
  }
  // ---- each instance's norm and pending scale, as the single context keeps them
  for (int i = blockIdx.x; i < b.ninst; i += gridDim.x) {
    const binst& I = b.inst[i];
    const double n = partials_sum(b.partials + I.ytile0, I.ytiles) * I.vol;
    if (threadIdx.x == 0) {
      *I.norm = n;
      if (!(n > 0.0) || !isfinite(n)) {
        atomicOr(I.flags, 1);
        *I.scale = 1.0;
      } else {
        *I.scale = IMAG ? 1.0 / sqrt(n) : 1.0;
      }
    }
    __syncthreads();
  }
}

}  // namespace

// Device scratch of the persistent step, owned by a batch.
struct batch_dev {
  binst* inst = nullptr;
  bwork* work = nullptr;
  double* partials = nullptr;
  unsigned* bar = nullptr;  // [0..1] barrier, then the flags word
  size_t inst_cap = 0, work_cap = 0, part_cap = 0;
  std::vector<binst> h_inst;
  std::vector<bwork> h_work;
};

void batch_kernel_free(batch_dev* d) {
  if (!d) return;
  cudaFree(d->inst);
  cudaFree(d->work);
  cudaFree(d->partials);
  cudaFree(d->bar);
  delete d;
}

namespace {

template <class P>
cudaError_t grow(P** p, size_t* cap, size_t want) {
  if (want <= *cap && *p) return cudaSuccess;
  cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  const cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(want, 1) * sizeof(P));
  if (e == cudaSuccess) *cap = std::max<size_t>(want, 1);
  return e;
}

template <class T, bool IMAG>
cudaError_t launch_k(const batch_args& b, size_t smem, int work_max, cudaStream_t s) {
  auto fn = k_batch_steps<T, IMAG>;
  cudaError_t e = allow_smem_bytes((const void*)fn, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kHThreads, smem)) !=
      cudaSuccess)
    return e;
  if (per < 1) return cudaErrorInvalidConfiguration;
  // every CTA must be resident at once (grid barrier): at most one wave
  const int grid = std::max(1, std::min(per * sms, work_max));
  void* args[] = {const_cast<batch_args*>(&b)};
  return cudaLaunchCooperativeKernel((const void*)fn, dim3(grid), dim3(kHThreads), args, smem, s);
}

}  // namespace

// Whole-line tiles of every instance must fit one CTA's shared memory.
bool batch_kernel_fits(const ctx_view* v, int count, size_t smem_limit, const char** why) {
  for (int i = 0; i < count; ++i) {
    if (v[i].dim != 2) {
      *why = "the persistent batch step serves 2D instances";
      return false;
    }
    if (v[i].fp64 != v[0].fp64) {
      *why = "instances of one precision";
      return false;
    }
    int pc = 0, ls = 0;
    if (hybrid_tile(v[i].nx, 0, v[i].fp64, 1, &pc, &ls) > smem_limit ||
        hybrid_tile(v[i].ny, 1, v[i].fp64, 1, &pc, &ls) > smem_limit) {
      *why = "an instance's lines do not fit one CTA's shared memory";
      return false;
    }
  }
  return true;
}

cudaError_t batch_kernel_run(batch_dev** dp, const ctx_view* v, int count, const int* active,
                             int nact, long long nsteps, bool imag, cudaStream_t s) {
  if (!*dp) *dp = new batch_dev();
  batch_dev& d = **dp;
  const bool fp64 = v[0].fp64 != 0;
  d.h_inst.assign(count, binst{});
  int parts = 0;
  size_t smem = 0;
  for (int i = 0; i < count; ++i) {
    binst& I = d.h_inst[i];
    I.psi[0] = v[i].psi[0];
    I.psi[1] = v[i].psi[1];
    for (int a = 0; a < 2; ++a)
      for (int m = 0; m < 2; ++m) I.tab[a][m] = v[i].table[a][m];
    I.scale = v[i].scale;
    I.norm = v[i].norm;
    I.flags = v[i].flags;
    I.nx = v[i].nx;
    I.ny = v[i].ny;
    I.lt = v[i].lt;
    I.cur = v[i].cur;
    smem = std::max(smem, hybrid_tile(I.nx, 0, fp64, 1, &I.pcx, &I.lsx));
    smem = std::max(smem, hybrid_tile(I.ny, 1, fp64, 1, &I.pcy, &I.lsy));
    I.ytile0 = parts;
    I.ytiles = (int)hybrid_groups(1, I.nx, I.nx);
    parts += I.ytiles;
    I.vec = (!fp64 && I.nx % 2 == 0) ? 1 : 0;
    I.dt = v[i].dt;
    I.g = v[i].g;
    I.hgam2 = 0.5 * v[i].gamma * v[i].gamma;
    I.hnu2 = 0.5 * v[i].nu * v[i].nu;
    I.x0 = v[i].x0;
    I.hx = v[i].hx;
    I.y0 = v[i].y0;
    I.hy = v[i].hy;
    I.vol = v[i].vol;
  }
  // work lists of the active instances: all x tiles, then all y tiles
  d.h_work.clear();
  for (int k = 0; k < nact; ++k) {
    const int i = active[k];
    const int g = (int)hybrid_groups(0, d.h_inst[i].ny, d.h_inst[i].nx);
    for (int t = 0; t < g; ++t) d.h_work.push_back({i, t});
  }
  const int nxw = (int)d.h_work.size();
  for (int k = 0; k < nact; ++k) {
    const int i = active[k];
    for (int t = 0; t < d.h_inst[i].ytiles; ++t) d.h_work.push_back({i, t});
  }
  const int nyw = (int)d.h_work.size() - nxw;
  cudaError_t e = grow(&d.inst, &d.inst_cap, (size_t)count);
  if (e == cudaSuccess) e = grow(&d.work, &d.work_cap, d.h_work.size());
  if (e == cudaSuccess) e = grow(&d.partials, &d.part_cap, (size_t)parts);
  if (e == cudaSuccess && !d.bar) e = cudaMalloc((void**)&d.bar, 4 * sizeof(unsigned));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d.inst, d.h_inst.data(), count * sizeof(binst), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d.work, d.h_work.data(), d.h_work.size() * sizeof(bwork),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.bar, 0, 4 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  batch_args b{};
  b.inst = d.inst;
  b.ninst = count;
  b.xw = d.work;
  b.nxw = nxw;
  b.yw = d.work + nxw;
  b.nyw = nyw;
  b.partials = d.partials;
  b.bar = d.bar;
  b.bflags = reinterpret_cast<int*>(d.bar + 2);
  b.nsteps = nsteps;
  const int work_max = std::max(std::max(nxw, nyw), count);
  if (fp64)
    return imag ? launch_k<double, true>(b, smem, work_max, s)
                : launch_k<double, false>(b, smem, work_max, s);
  return imag ? launch_k<float, true>(b, smem, work_max, s)
              : launch_k<float, false>(b, smem, work_max, s);
}

// The flags word of the last launch (bit 3: a grid-barrier wait gave up);
// synchronises the stream.
cudaError_t batch_kernel_flags(batch_dev* d, cudaStream_t s, int* flags) {
  *flags = 0;
  if (!d || !d->bar) return cudaSuccess;
  cudaError_t e = cudaMemcpyAsync(flags, d->bar + 2, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

}  // namespace rotgp
