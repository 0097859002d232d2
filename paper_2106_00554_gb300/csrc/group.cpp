// Plan groups: many independent products issued as one unit (uw.h).  The
// instances are spread over internal streams forked from the caller's stream
// and joined back into it, so a stream capture records one multi-branch
// graph.  The tuner picks, per plan, the line-operator variant that times
// fastest on that plan's sizes.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <set>
#include <sstream>
#include <string>
#include <vector>

#include "uw_internal.h"

struct uw_plan : public uw::Plan {};

struct uw_group {
  std::vector<uw_plan*> plans;
  std::vector<int> saved_coarse;       // the plans' coarse-level choice before the group
  std::vector<cudaStream_t> streams;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  uw::PersistentGroup* pg = nullptr;   // one persistent launch for FP32 (null: not eligible)
  int use_pg = 1;                      // the tuner may prefer the forked streams
  unsigned* derr = nullptr;            // device word: a bounded wait of the persistent launch gave up
};

static int group_fail(int code, const char* msg) {
  uw::set_error(code, msg);
  return code;
}

static void group_free(uw_group* g) {
  uw::pgroup_destroy(g->pg);
  if (g->derr) cudaFree(g->derr);
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
  if (cudaMalloc(&g->derr, sizeof(unsigned)) != cudaSuccess || cudaMemset(g->derr, 0, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    for (size_t i = 0; i < g->plans.size(); ++i) {
      g->plans[i]->coarse_mode = g->saved_coarse[i];
      g->plans[i]->group = nullptr;
    }
    group_free(g);
    uw::set_error(UW_ERR_OOM, "group status word allocation failed");
    return nullptr;
  }
  {
    std::string why;
    std::vector<const uw::Plan*> pl(g->plans.begin(), g->plans.end());
    g->pg = uw::pgroup_create(pl.data(), n, why);
    cudaGetLastError();
  }
  uw::set_error(UW_OK, "");
  return g;
}

static int group_run(uw_group* g, int prec, bool fwd, const void* const* in, void* const* out, void* stream) {
  if (!g || !in || !out) return group_fail(UW_ERR_INVALID_ARG, "null group or buffer list");
  if (prec != UW_F64 && prec != UW_F32 && prec != UW_F32_SPLIT_BF16)
    return group_fail(UW_ERR_INVALID_ARG, "unknown precision");
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == UW_F32 && g->pg && (g->use_pg || getenv("UW_GROUP_PERSISTENT")) && !getenv("UW_GROUP_STREAMS")) {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != g->plans[0]->device)
      return group_fail(UW_ERR_INVALID_ARG, "the current CUDA device is not the group's device");
    for (size_t i = 0; i < g->plans.size(); ++i) {
      const bool need_in = fwd || g->plans[i]->m > 0, need_out = !fwd || g->plans[i]->m > 0;
      if ((need_in && !in[i]) || (need_out && !out[i])) return group_fail(UW_ERR_INVALID_ARG, "null buffer");
    }
    return uw::pgroup_run(g->pg, fwd, in, out, g->derr, stream);
  }
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

static int group_tune_variants(uw_group* g, int prec, void* const* x, void* const* y, int reps, void* stream) {
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


// ---------------------------------------------------------------------------
// tuner of the persistent launch, with a JSON cache
// ---------------------------------------------------------------------------
// ms per forward + adjoint pair of the whole group on the current settings
static int time_group_pairs(uw_group* g, int prec, void* const* x, void* const* y, int reps, void* stream, float* ms) {
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return group_fail(UW_ERR_OOM, "event creation failed");
  }
  int st = UW_OK;
  for (int r = 0; r <= reps && st == UW_OK; ++r) {
    if (r == 1 && cudaEventRecord(e0, s) != cudaSuccess) st = group_fail(UW_ERR_CUDA, "event record failed");
    if (st == UW_OK) st = group_run(g, prec, true, (const void* const*)x, y, stream);
    if (st == UW_OK) st = group_run(g, prec, false, (const void* const*)y, x, stream);
  }
  if (st == UW_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                      cudaEventElapsedTime(ms, e0, e1) != cudaSuccess))
    st = group_fail(UW_ERR_CUDA, "timing failed");
  if (st == UW_OK) *ms /= (float)reps;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

// cache key: GPU, dimension, the multiset of N over the instances, precision
static std::string tune_key(const uw_group* g, int prec) {
  cudaDeviceProp prop{};
  int dev = 0;
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&prop, dev);
  std::map<int, int> ns;
  for (const uw_plan* P : g->plans) ns[P->N]++;
  std::ostringstream k;
  k << prop.name << "|d2|n" << g->plans.size() << "|N";
  for (auto& kv : ns) k << kv.first << "x" << kv.second << ",";
  k << "|prec" << prec;
  std::string out = k.str();
  for (char& c : out)
    if (c == '"' || c == '\\') c = '_';
  return out;
}

// the cache file: one JSON object, "key": [lines, cols, tiles, rad, ctas, persistent]
static std::map<std::string, std::vector<int>> read_cache(const char* path) {
  std::map<std::string, std::vector<int>> m;
  std::ifstream f(path);
  if (!f) return m;
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string t = ss.str();
  size_t i = 0;
  while ((i = t.find('"', i)) != std::string::npos) {
    const size_t j = t.find('"', i + 1);
    if (j == std::string::npos) break;
    const std::string key = t.substr(i + 1, j - i - 1);
    const size_t a = t.find('[', j), b = t.find(']', j);
    if (a == std::string::npos || b == std::string::npos || b < a) break;
    std::vector<int> v;
    std::stringstream vs(t.substr(a + 1, b - a - 1));
    std::string tok;
    while (std::getline(vs, tok, ',')) v.push_back(atoi(tok.c_str()));
    m[key] = v;
    i = b + 1;
  }
  return m;
}
static void write_cache(const char* path, const std::map<std::string, std::vector<int>>& m) {
  std::ofstream f(path, std::ios::trunc);
  if (!f) return;
  f << "{\n";
  size_t n = 0;
  for (auto& kv : m) {
    f << "  \"" << kv.first << "\": [";
    for (size_t i = 0; i < kv.second.size(); ++i) f << (i ? ", " : "") << kv.second[i];
    f << "]" << (++n < m.size() ? "," : "") << "\n";
  }
  f << "}\n";
}

static int group_tune_persistent(uw_group* g, int prec, void* const* x, void* const* y, int reps, const char* cache,
                                 void* stream) {
  const std::string key = tune_key(g, prec);
  if (cache) {
    auto m = read_cache(cache);
    auto it = m.find(key);
    if (it != m.end() && it->second.size() == 6) {
      const auto& v = it->second;
      const int st = uw::pgroup_set_params(g->pg, v[0], v[1], v[2], v[3], v[4]);
      g->use_pg = v[5];
      return st;
    }
  }
  float t_streams = 0.f;
  g->use_pg = 0;
  int st = time_group_pairs(g, prec, x, y, reps, stream, &t_streams);
  g->use_pg = 1;
  if (st != UW_OK) return st;
  float best = 0.f;
  int bp[5] = {1, 4, 4, 16, 0};
  bool first = true;
  for (int lines : {1, 4, 16})
    for (int cols : {4, 16, 64})
      for (int tiles : {4, 16})
        for (int rad : {16, 8})
          for (int ctas : {0, 2}) {
            if ((st = uw::pgroup_set_params(g->pg, lines, cols, tiles, rad, ctas)) != UW_OK) return st;
            float t = 0.f;
            if ((st = time_group_pairs(g, prec, x, y, reps, stream, &t)) != UW_OK) return st;
            if (first || t < best) {
              best = t;
              const int v[5] = {lines, cols, tiles, rad, ctas};
              std::memcpy(bp, v, sizeof bp);
              first = false;
            }
          }
  if ((st = uw::pgroup_set_params(g->pg, bp[0], bp[1], bp[2], bp[3], bp[4])) != UW_OK) return st;
  g->use_pg = best <= t_streams ? 1 : 0;
  if (cache) {
    auto m = read_cache(cache);
    m[key] = {bp[0], bp[1], bp[2], bp[3], bp[4], g->use_pg};
    write_cache(cache, m);
  }
  return UW_OK;
}

int uw_group_tune_cached(uw_group* g, int prec, void* const* x, void* const* y, int reps, const char* cache,
                         void* stream) {
  int st = group_tune_variants(g, prec, x, y, reps, stream);
  if (st != UW_OK || prec != UW_F32 || !g->pg) return st;
  return group_tune_persistent(g, prec, x, y, reps, cache, stream);
}

int uw_group_tune(uw_group* g, int prec, void* const* x, void* const* y, int reps, void* stream) {
  return uw_group_tune_cached(g, prec, x, y, reps, nullptr, stream);
}

int uw_group_params(const uw_group* g, int* out7) {
  if (!g || !out7) return group_fail(UW_ERR_INVALID_ARG, "null group or output");
  out7[0] = g->pg ? 1 : 0;
  out7[1] = g->use_pg;
  if (g->pg) uw::pgroup_params(g->pg, out7 + 2);
  else
    for (int i = 2; i < 7; ++i) out7[i] = 0;
  return UW_OK;
}

int uw_group_device_status(uw_group* g) {
  if (!g) return group_fail(UW_ERR_INVALID_ARG, "null group");
  unsigned w = 0;
  if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpy(&w, g->derr, sizeof w, cudaMemcpyDeviceToHost) != cudaSuccess)
    return group_fail(UW_ERR_CUDA, "group status: device error");
  if (w) {
    cudaMemset(g->derr, 0, sizeof(unsigned));
    cudaDeviceSynchronize();
    return group_fail(UW_ERR_TIMEOUT, "a bounded wait of the persistent group launch gave up; results invalid");
  }
  return UW_OK;
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
