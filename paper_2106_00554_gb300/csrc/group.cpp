// Plan groups: many independent products issued as one unit (uw.h).  The
// instances are spread over internal streams forked from the caller's stream
// and joined back into it, so a stream capture records one multi-branch
// graph.  The tuner picks, per plan, the line-operator variant that times
// fastest on that plan's sizes.
#include <cuda_runtime.h>

#include <set>
#include <vector>

#include "uw_internal.h"

struct uw_plan : public uw::Plan {};

struct uw_group {
  std::vector<uw_plan*> plans;
  std::vector<int> saved_coarse;       // the plans' coarse-level choice before the group
  std::vector<cudaStream_t> streams;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
};

static int group_fail(int code, const char* msg) {
  uw::set_error(code, msg);
  return code;
}

static void group_free(uw_group* g) {
  for (cudaStream_t s : g->streams)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : g->join)
    if (e) cudaEventDestroy(e);
  if (g->fork) cudaEventDestroy(g->fork);
  delete g;
}

extern "C" {

uw_group* uw_group_create(uw_plan* const* plans, int n, int nstreams) {
  if (!plans || n < 1 || nstreams < 1 || nstreams > 64) {
    uw::set_error(UW_ERR_INVALID_ARG, "null plans, n < 1 or nstreams outside [1, 64]");
    return nullptr;
  }
  // one plan owns one workspace, so it may appear once in one live group:
  // two streams running the same plan would race on it
  std::set<const uw_plan*> seen;
  for (int i = 0; i < n; ++i) {
    if (!plans[i]) {
      uw::set_error(UW_ERR_INVALID_ARG, "null plan in the group");
      return nullptr;
    }
    if (!seen.insert(plans[i]).second) {
      uw::set_error(UW_ERR_INVALID_ARG, "a plan appears twice in the group");
      return nullptr;
    }
    if (plans[i]->group) {
      uw::set_error(UW_ERR_INVALID_ARG, "a plan already belongs to another live group");
      return nullptr;
    }
  }
  uw_group* g = new uw_group();
  g->plans.assign(plans, plans + n);
  const int ns = nstreams < n ? nstreams : n;
  g->streams.assign(ns, nullptr);
  g->join.assign(ns, nullptr);
  bool ok = cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; ok && k < ns; ++k)
    ok = cudaStreamCreateWithFlags(&g->streams[k], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&g->join[k], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    group_free(g);
    uw::set_error(UW_ERR_OOM, "stream or event creation failed");
    return nullptr;
  }
  for (uw_plan* P : g->plans) {
    g->saved_coarse.push_back(P->coarse_mode);
    P->coarse_mode = 1;
    P->group = g;
  }
  return g;
}

static int group_run(uw_group* g, int prec, bool fwd, const void* const* in, void* const* out, void* stream) {
  if (!g || !in || !out) return group_fail(UW_ERR_INVALID_ARG, "null group or buffer list");
  if (prec != UW_F64 && prec != UW_F32 && prec != UW_F32_SPLIT_BF16)
    return group_fail(UW_ERR_INVALID_ARG, "unknown precision");
  cudaStream_t s = (cudaStream_t)stream;
  const int ns = (int)g->streams.size();
  if (cudaEventRecord(g->fork, s) != cudaSuccess) return group_fail(UW_ERR_CUDA, "fork event failed");
  for (int k = 0; k < ns; ++k)
    if (cudaStreamWaitEvent(g->streams[k], g->fork, 0) != cudaSuccess) return group_fail(UW_ERR_CUDA, "fork wait failed");
  int st = UW_OK;
  for (size_t i = 0; i < g->plans.size() && st == UW_OK; ++i) {
    void* si = g->streams[i % ns];
    st = fwd ? uw_forward(g->plans[i], prec, in[i], out[i], 1, si)
             : uw_adjoint(g->plans[i], prec, in[i], out[i], 1, si);
  }
  // join every internal stream back into the caller's stream even after a
  // failing instance, so that a capture of `stream` can still end; the first
  // error is returned
  for (int k = 0; k < ns; ++k)
    if (cudaEventRecord(g->join[k], g->streams[k]) != cudaSuccess || cudaStreamWaitEvent(s, g->join[k], 0) != cudaSuccess)
      if (st == UW_OK) st = group_fail(UW_ERR_CUDA, "join failed");
  return st;
}

int uw_group_forward(uw_group* g, int prec, const void* const* x, void* const* y, void* stream) {
  return group_run(g, prec, true, x, y, stream);
}

int uw_group_adjoint(uw_group* g, int prec, const void* const* y, void* const* x, void* stream) {
  return group_run(g, prec, false, y, x, stream);
}

int uw_group_tune(uw_group* g, int prec, void* const* x, void* const* y, int reps, void* stream) {
  if (!g || !x || !y || reps < 1) return group_fail(UW_ERR_INVALID_ARG, "null group or buffers, or reps < 1");
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return group_fail(UW_ERR_OOM, "event creation failed");
  }
  int st = UW_OK;
  for (size_t i = 0; i < g->plans.size() && st == UW_OK; ++i) {
    uw_plan* P = g->plans[i];
    float best = 0.f;
    int best_v = 0;
    for (int v = 0; v < 2 && st == UW_OK; ++v) {
      P->line_variant = v;
      // one untimed pair (first-launch setup), then reps timed pairs
      for (int r = 0; r <= reps && st == UW_OK; ++r) {
        if (r == 1 && cudaEventRecord(e0, s) != cudaSuccess) st = group_fail(UW_ERR_CUDA, "event record failed");
        if (st == UW_OK) st = uw_forward(P, prec, x[i], y[i], 1, s);
        if (st == UW_OK) st = uw_adjoint(P, prec, y[i], x[i], 1, s);
      }
      if (st != UW_OK) break;
      float ms = 0.f;
      if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        st = group_fail(UW_ERR_CUDA, "timing failed");
        break;
      }
      if (v == 0 || ms < best) {
        best = ms;
        best_v = v;
      }
    }
    P->line_variant = best_v;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

void uw_group_destroy(uw_group* g) {
  if (!g) return;
  for (cudaStream_t s : g->streams) cudaStreamSynchronize(s);
  for (size_t i = 0; i < g->plans.size(); ++i) {
    g->plans[i]->coarse_mode = g->saved_coarse[i];
    g->plans[i]->group = nullptr;
  }
  group_free(g);
}

}  // extern "C"
