// batch.cu -- many independent condensates advanced together (the batched
// workload: instances of uneven grid sizes and differing Omega, g and trap
// anisotropy).
//
// Each instance is a full rotgp context on a stream of its own.  Three ways
// to run a block of steps of the active instances:
//  - ROTGP_BATCH_PERSISTENT: one cooperative kernel (batch_kernel.cu) takes
//    every tile of every active 2D instance, phase by phase, with grid
//    barriers between phases, for the whole block of steps;
//  - ROTGP_BATCH_GRAPH: the instances' own kernels, captured once into a CUDA
//    graph that forks from the caller's stream into the instance streams and
//    joins back, replayed as one graph launch;
//  - ROTGP_BATCH_DIRECT: the same kernels launched directly, forked and joined
//    the same way.  Convergence (imaginary time) is checked
// between graph launches: every `check_every` steps each active instance's
// mu is compared with its value one check earlier; an instance is converged
// when the relative change is below the tolerance and its vortex count did
// not change, and later graphs leave it out.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/rotgp.h"
#include "common.cuh"

// A captured block of steps: valid for the instances' buffer parity at
// capture time (the kernels' buffer pointers are part of the graph).
struct BatchGraph {
  std::vector<int> set;
  long long steps = 0;
  bool imag = true;
  std::vector<int> cur0, cur1;  // state buffer of each instance before / after
  std::vector<long long> plan;  // each instance's plan version at capture
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

struct rotgp_batch {
  std::vector<rotgp_ctx*> ctx;
  std::vector<cudaStream_t> streams;  // one per instance
  std::vector<cudaEvent_t> done;      // join events, one per instance
  cudaEvent_t fork = nullptr, user_ev = nullptr;
  cudaStream_t user = nullptr;        // the caller's stream
  cudaStream_t stream = nullptr;      // the batch's own (graphs are captured on it)
  std::vector<BatchGraph> graphs;     // at most two live (the two buffer parities)
  long long graph_launches = 0;
  rotgp::batch_dev* dev = nullptr;    // scratch of the persistent step
  std::string err;
};

namespace {

thread_local std::string g_batch_error;

int bfail(rotgp_batch* b, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (b)
    b->err = buf;
  else
    g_batch_error = buf;
  return code;
}

void drop_graph(rotgp_batch* b) {
  for (auto& g : b->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
  }
  b->graphs.clear();
}

int run_set_inner(rotgp_batch* b, const std::vector<int>& set, long long n, bool imag,
                  int mode);

// Run n steps of the instances in `set` (mode: ROTGP_BATCH_*), ordered after
// the caller's stream and before its next work.
int run_set(rotgp_batch* b, const std::vector<int>& set, long long n, bool imag, int mode) {
  if (set.empty() || n == 0) return ROTGP_OK;
  cudaError_t e = cudaEventRecord(b->user_ev, b->user);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->user_ev, 0);
  if (e != cudaSuccess) return bfail(b, ROTGP_ECUDA, "order: %s", cudaGetErrorString(e));
  const int rc = run_set_inner(b, set, n, imag, mode);
  e = cudaEventRecord(b->user_ev, b->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->user, b->user_ev, 0);
  if (!rc && e != cudaSuccess) return bfail(b, ROTGP_ECUDA, "order: %s", cudaGetErrorString(e));
  return rc;
}

int run_set_inner(rotgp_batch* b, const std::vector<int>& set, long long n, bool imag,
                  int mode) {
  cudaError_t e;
  // work already queued on the instance streams (table rebuilds of
  // rotgp_set_phys, state I/O) comes first
  for (int i : set) {
    if ((e = cudaEventRecord(b->done[i], b->streams[i])) != cudaSuccess ||
        (e = cudaStreamWaitEvent(b->stream, b->done[i], 0)) != cudaSuccess)
      return bfail(b, ROTGP_ECUDA, "order: %s", cudaGetErrorString(e));
  }
  if (mode == ROTGP_BATCH_PERSISTENT) {
    const int count = (int)b->ctx.size();
    std::vector<rotgp::ctx_view> v(count);
    for (int i = 0; i < count; ++i) rotgp::ctx_get_view(b->ctx[i], &v[i]);
    const char* why = "";
    if (!rotgp::batch_kernel_fits(v.data(), count, 200 * 1024, &why))
      return bfail(b, ROTGP_EUNSUPPORTED, "persistent batch step: %s", why);
    e = rotgp::batch_kernel_run(&b->dev, v.data(), count, set.data(), (int)set.size(), n, imag,
                                b->stream);
    if (e != cudaSuccess)
      return bfail(b, ROTGP_ECUDA, "persistent batch launch: %s", cudaGetErrorString(e));
    for (int i : set) rotgp::ctx_add_steps(b->ctx[i], n);
    // later work of the instances (observables, I/O) follows the launch
    if ((e = cudaEventRecord(b->fork, b->stream)) != cudaSuccess)
      return bfail(b, ROTGP_ECUDA, "order: %s", cudaGetErrorString(e));
    for (int i : set)
      if ((e = cudaStreamWaitEvent(b->streams[i], b->fork, 0)) != cudaSuccess)
        return bfail(b, ROTGP_ECUDA, "order: %s", cudaGetErrorString(e));
    return ROTGP_OK;
  }
  if (mode != ROTGP_BATCH_GRAPH) {
    if ((e = cudaEventRecord(b->fork, b->stream)) != cudaSuccess)
      return bfail(b, ROTGP_ECUDA, "fork: %s", cudaGetErrorString(e));
    for (int i : set) {
      if ((e = cudaStreamWaitEvent(b->streams[i], b->fork, 0)) != cudaSuccess)
        return bfail(b, ROTGP_ECUDA, "fork: %s", cudaGetErrorString(e));
      const int rc = imag ? rotgp_step_imag(b->ctx[i], n) : rotgp_step_real(b->ctx[i], n);
      if (rc) return bfail(b, rc, "instance %d: %s", i, rotgp_last_error(b->ctx[i]));
      if ((e = cudaEventRecord(b->done[i], b->streams[i])) != cudaSuccess ||
          (e = cudaStreamWaitEvent(b->stream, b->done[i], 0)) != cudaSuccess)
        return bfail(b, ROTGP_ECUDA, "join: %s", cudaGetErrorString(e));
    }
    return ROTGP_OK;
  }
  std::vector<int> cur(set.size());
  std::vector<long long> plan(set.size());
  for (size_t k = 0; k < set.size(); ++k) {
    cur[k] = rotgp::ctx_buffer(b->ctx[set[k]]);
    plan[k] = rotgp::ctx_plan_version(b->ctx[set[k]]);
  }
  BatchGraph* g = nullptr;
  for (auto& x : b->graphs)
    if (x.set == set && x.steps == n && x.imag == imag && x.cur0 == cur && x.plan == plan) g = &x;
  if (g) {
    // replay: the graph advances the states as captured
    for (size_t k = 0; k < set.size(); ++k) {
      rotgp::ctx_set_buffer(b->ctx[set[k]], g->cur1[k]);
      rotgp::ctx_add_steps(b->ctx[set[k]], n);
    }
  } else {
    if (b->graphs.size() >= 2) drop_graph(b);
    // capture: fork from the caller's stream into each instance stream, n
    // steps per instance, join back.  Capturing advances each context's
    // buffer index and step counter as if the steps ran; the launch below
    // runs them.
    std::vector<long long> steps0(set.size());
    for (size_t k = 0; k < set.size(); ++k) steps0[k] = rotgp::ctx_steps(b->ctx[set[k]]);
    BatchGraph ng;
    ng.set = set;
    ng.steps = n;
    ng.imag = imag;
    ng.cur0 = cur;
    ng.plan = plan;
    if ((e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return bfail(b, ROTGP_ECUDA, "begin capture: %s", cudaGetErrorString(e));
    int rc = ROTGP_OK;
    e = cudaEventRecord(b->fork, b->stream);
    for (int i : set) {
      if (e != cudaSuccess || rc) break;
      e = cudaStreamWaitEvent(b->streams[i], b->fork, 0);
      if (e == cudaSuccess) {
        rc = imag ? rotgp_step_imag(b->ctx[i], n) : rotgp_step_real(b->ctx[i], n);
        if (rc) bfail(b, rc, "instance %d: %s", i, rotgp_last_error(b->ctx[i]));
      }
      if (e == cudaSuccess && !rc) e = cudaEventRecord(b->done[i], b->streams[i]);
      if (e == cudaSuccess && !rc) e = cudaStreamWaitEvent(b->stream, b->done[i], 0);
    }
    cudaGraph_t gr = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b->stream, &gr);
    if (e == cudaSuccess) e = ee;
    if (!rc && e == cudaSuccess) e = cudaGraphInstantiate(&ng.exec, gr, 0);
    if (rc || e != cudaSuccess) {
      // nothing ran: put the states back
      if (gr) cudaGraphDestroy(gr);
      for (size_t k = 0; k < set.size(); ++k) {
        rotgp::ctx_set_buffer(b->ctx[set[k]], cur[k]);
        rotgp::ctx_add_steps(b->ctx[set[k]], steps0[k] - rotgp::ctx_steps(b->ctx[set[k]]));
      }
      cudaGetLastError();
      return rc ? rc : bfail(b, ROTGP_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    }
    ng.graph = gr;
    for (int i : set) ng.cur1.push_back(rotgp::ctx_buffer(b->ctx[i]));
    b->graphs.push_back(ng);
    g = &b->graphs.back();
  }
  if ((e = cudaGraphLaunch(g->exec, b->stream)) != cudaSuccess)
    return bfail(b, ROTGP_ECUDA, "graph launch: %s", cudaGetErrorString(e));
  ++b->graph_launches;
  return ROTGP_OK;
}

}  // namespace

extern "C" {

const char* rotgp_batch_last_error(const rotgp_batch* b) {
  return b ? b->err.c_str() : g_batch_error.c_str();
}

void rotgp_batch_destroy(rotgp_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graph(b);
  rotgp::batch_kernel_free(b->dev);
  for (auto* c : b->ctx) rotgp_destroy(c);
  for (auto s : b->streams) cudaStreamDestroy(s);
  for (auto ev : b->done) cudaEventDestroy(ev);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->user_ev) cudaEventDestroy(b->user_ev);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

int rotgp_batch_create(int count, const rotgp_grid* grids, const rotgp_phys* phys, int precision,
                       void* stream, rotgp_batch** out) {
  g_batch_error.clear();
  if (!out || !grids || !phys || count < 1)
    return bfail(nullptr, ROTGP_EINVAL, "count >= 1, grids, phys and out are required");
  *out = nullptr;
  rotgp_batch* b = new (std::nothrow) rotgp_batch();
  if (!b) return bfail(nullptr, ROTGP_ENOMEM, "host allocation failed");
  b->user = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->user_ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->streams.push_back(s);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->done.push_back(ev);
  }
  if (e != cudaSuccess) {
    const int rc = bfail(nullptr, ROTGP_ECUDA, "streams: %s", cudaGetErrorString(e));
    rotgp_batch_destroy(b);
    return rc;
  }
  for (int i = 0; i < count; ++i) {
    rotgp_ctx* c = nullptr;
    const int rc = rotgp_create(&grids[i], &phys[i], precision, b->streams[i], &c);
    if (rc) {
      bfail(nullptr, rc, "instance %d: %s", i, rotgp_last_error(nullptr));
      rotgp_batch_destroy(b);
      return rc;
    }
    b->ctx.push_back(c);
  }
  *out = b;
  return ROTGP_OK;
}

int rotgp_batch_count(const rotgp_batch* b) { return b ? (int)b->ctx.size() : 0; }

int rotgp_batch_context(rotgp_batch* b, int index, rotgp_ctx** ctx) {
  if (!b || !ctx) return ROTGP_EINVAL;
  if (index < 0 || index >= (int)b->ctx.size())
    return bfail(b, ROTGP_EINVAL, "index %d out of range", index);
  *ctx = b->ctx[index];
  return ROTGP_OK;
}

int rotgp_batch_autotune(rotgp_batch* b, int steps) {
  if (!b) return ROTGP_EINVAL;
  drop_graph(b);
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    const int rc = rotgp_autotune(b->ctx[i], steps, nullptr);
    if (rc) return bfail(b, rc, "instance %zu: %s", i, rotgp_last_error(b->ctx[i]));
  }
  return ROTGP_OK;
}

int rotgp_batch_step(rotgp_batch* b, long long n, int imag, int mode) {
  if (!b) return ROTGP_EINVAL;
  if (n < 0) return bfail(b, ROTGP_EINVAL, "negative step count");
  if (mode < ROTGP_BATCH_DIRECT || mode > ROTGP_BATCH_PERSISTENT)
    return bfail(b, ROTGP_EINVAL, "unknown batch mode %d", mode);
  std::vector<int> all(b->ctx.size());
  for (size_t i = 0; i < all.size(); ++i) all[i] = (int)i;
  return run_set(b, all, n, imag != 0, mode);
}

int rotgp_batch_sync(rotgp_batch* b) {
  if (!b) return ROTGP_EINVAL;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->user);
  if (e != cudaSuccess) return bfail(b, ROTGP_ECUDA, "synchronise: %s", cudaGetErrorString(e));
  int bf = 0;
  if ((e = rotgp::batch_kernel_flags(b->dev, b->stream, &bf)) != cudaSuccess)
    return bfail(b, ROTGP_ECUDA, "synchronise: %s", cudaGetErrorString(e));
  if (bf & 8)
    return bfail(b, ROTGP_ETIMEOUT, "a grid-barrier wait of the persistent batch step gave up");
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    const int rc = rotgp_sync(b->ctx[i]);
    if (rc) return bfail(b, rc, "instance %zu: %s", i, rotgp_last_error(b->ctx[i]));
  }
  return ROTGP_OK;
}

int rotgp_batch_observables(rotgp_batch* b, rotgp_obs* out) {
  if (!b || !out) return ROTGP_EINVAL;
  int rc = rotgp_batch_sync(b);
  for (size_t i = 0; i < b->ctx.size() && !rc; ++i) {
    rc = rotgp_observables(b->ctx[i], &out[i]);
    if (rc) bfail(b, rc, "instance %zu: %s", i, rotgp_last_error(b->ctx[i]));
  }
  return rc;
}

int rotgp_batch_converge(rotgp_batch* b, double rel_tol, long long check_every,
                         long long max_steps, int mode, long long* steps_out,
                         int* converged_out) {
  if (!b || !steps_out) return ROTGP_EINVAL;
  if (!(rel_tol > 0) || check_every < 1 || max_steps < 1)
    return bfail(b, ROTGP_EINVAL, "rel_tol > 0, check_every >= 1, max_steps >= 1 required");
  const int n = (int)b->ctx.size();
  std::vector<double> mu(n, NAN);
  std::vector<int> vort(n, -1);
  std::vector<char> conv(n, 0);
  for (int i = 0; i < n; ++i) steps_out[i] = 0;
  long long done_steps = 0;
  while (done_steps < max_steps) {
    std::vector<int> active;
    for (int i = 0; i < n; ++i)
      if (!conv[i]) active.push_back(i);
    if (active.empty()) break;
    const long long k = std::min(check_every, max_steps - done_steps);
    if (mode < ROTGP_BATCH_DIRECT || mode > ROTGP_BATCH_PERSISTENT)
      return bfail(b, ROTGP_EINVAL, "unknown batch mode %d", mode);
    int rc = run_set(b, active, k, true, mode);
    if (!rc) rc = rotgp_batch_sync(b);
    if (rc) return rc;
    done_steps += k;
    for (int i : active) {
      rotgp_obs o;
      rc = rotgp_observables(b->ctx[i], &o);
      if (rc) return bfail(b, rc, "instance %d: %s", i, rotgp_last_error(b->ctx[i]));
      steps_out[i] = done_steps;
      if (std::isfinite(mu[i]) && std::fabs(o.mu - mu[i]) <= rel_tol * std::fabs(o.mu) &&
          o.vortices == vort[i])
        conv[i] = 1;
      mu[i] = o.mu;
      vort[i] = o.vortices;
    }
  }
  if (converged_out)
    for (int i = 0; i < n; ++i) converged_out[i] = conv[i];
  return ROTGP_OK;
}

}  // extern "C"
