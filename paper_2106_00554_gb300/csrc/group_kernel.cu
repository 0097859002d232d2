// One persistent launch for a plan group: every instance's 2D product (any
// mix of R, q, p, boundary and masks) as tasks of one work queue.
//
// An instance's product is a sequence of phases; every item of a phase must
// be done before any item of the next phase of that instance starts:
//   forward (Algorithm 2 preceded by the Mallat IDWT, Sec. 5):
//     for each coarse level j = J0 .. R-2: rows, then columns (one line each)
//     transpose-in (32 x 32 tiles): the level R-1 array, rows <-> columns
//     dim-1 lines (last synthesis level, T, FWHT; one line each)
//     transpose (tiles)
//     dim-2 lines with the gather of the sampled sequency indices
//   adjoint: the same phases transposed and in reverse order.
// The host lays out the tasks (an instance, a phase, a run of items) phase
// by phase across all instances.  The CTAs of one persistent grid take tasks
// in that order from an atomic ticket; before a task runs, one thread waits
// until the instance's previous phase has counted all its items done
// (bounded: after the spin limit it records the failure in the error word and
// the CTA stops); after it, the count of its own phase grows.  A task only
// ever waits for tasks with smaller tickets, which CTAs already hold, so the
// queue always drains.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>

#include "line_common.cuh"

namespace uw {
namespace gk {

constexpr int MAXI = 1024;       // instances per launch (pointer arrays are kernel parameters)
constexpr int NTH = 256;

// one instance, as the kernel sees it (built on the host from its plan)
struct Inst {
  Geo G;
  Tables<float> tab;
  int J0;
  int nl;                        // coarse levels J0 .. R-2
  const uint32_t* mask;
  const int32_t* prefix;
  const uint16_t* pos;
  int wpr;
  int64_t m;
  float* XS;                     // (M/2)^2: coarse level outputs, alternating with XS2
  float* XS2;
  float* XT;                     // M x M
  float* VT;                     // M x N
  float* V;                      // N x M
  int done_off;                  // first of this instance's per-phase counters
};

struct Task {
  int inst, phase, item0, nitems;
};

struct Ptrs {
  const float* in[MAXI];
  float* out[MAXI];
};

// relaxed polling load and acquire / release of the per-phase counters
__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---------------------------------------------------------------------------
// coarse levels, one line per item, through shared memory (Sec. 3.2 two-scale
// relations with the boundary blocks, via syn_one / ana_one)
// ---------------------------------------------------------------------------
// synthesis, level j: row r of [[LL, HL], [LH, HH]] (LL = S_j) -> T[r][0, 2n0)
__device__ void syn_row(const Geo& G, const float* x, const float* S, int ldS, float* Tm, int j, int r,
                        const SmemTables<float>& st, float* sm, int tid) {
  const int n0 = 1 << j, n1 = 2 * n0, M = G.M;
  for (int c = tid; c < n1; c += NTH) sm[c] = (r < n0 && c < n0) ? S[(int64_t)r * ldS + c] : x[(int64_t)r * M + c];
  __syncthreads();
  Plain<float> lo{sm}, hi{sm + n0};
  for (int k = tid; k < n1; k += NTH) Tm[(int64_t)r * n1 + k] = syn_one<float>(k, n0, lo, hi, st, G);
}
// synthesis, level j: column c of T -> S_{j+1}[0, 2n0)[c]
__device__ void syn_col(const Geo& G, const float* Tm, float* Sout, int ldO, int j, int c, const SmemTables<float>& st,
                        float* sm, int tid) {
  const int n0 = 1 << j, n1 = 2 * n0;
  for (int k = tid; k < n1; k += NTH) sm[k] = Tm[(int64_t)k * n1 + c];
  __syncthreads();
  Plain<float> lo{sm}, hi{sm + n0};
  for (int k = tid; k < n1; k += NTH) Sout[(int64_t)k * ldO + c] = syn_one<float>(k, n0, lo, hi, st, G);
}
// analysis, level j: column c of S_{j+1} -> T[0, n0)[c] (lo), T[n0, 2n0)[c] (hi)
__device__ void ana_col(const Geo& G, const float* S, int ldS, float* Tm, int j, int c, const SmemTables<float>& st,
                        float* sm, int tid) {
  const int n0 = 1 << j, n1 = 2 * n0;
  for (int k = tid; k < n1; k += NTH) sm[k] = S[(int64_t)k * ldS + c];
  __syncthreads();
  Plain<float> s{sm};
  for (int m = tid; m < n0; m += NTH) {
    float lo, hi;
    ana_one<float>(m, n0, s, st, G, lo, hi);
    Tm[(int64_t)m * n1 + c] = lo;
    Tm[(int64_t)(n0 + m) * n1 + c] = hi;
  }
}
// analysis, level j: row r of T -> [lo | hi]; the LL quarter to S_j (or x at
// the coarsest level), the rest to x
__device__ void ana_row(const Geo& G, const float* Tm, float* x, float* Snext, int ldN, int j, int r,
                        const SmemTables<float>& st, float* sm, int tid) {
  const int n0 = 1 << j, n1 = 2 * n0, M = G.M;
  for (int k = tid; k < n1; k += NTH) sm[k] = Tm[(int64_t)r * n1 + k];
  __syncthreads();
  Plain<float> s{sm};
  for (int m = tid; m < n0; m += NTH) {
    float lo, hi;
    ana_one<float>(m, n0, s, st, G, lo, hi);
    if (r < n0) Snext[(int64_t)r * ldN + m] = lo;
    else x[(int64_t)r * M + m] = lo;
    x[(int64_t)r * M + n0 + m] = hi;
  }
}

// 32 x 32 tile of a transpose: out[c][r] = in(r, c) for the tile (tr, tc)
// of an R x C array; `in` gives element (r, c)
template <typename F, typename G2>
__device__ void tile_t(int tr, int tc, F&& in, G2&& out, float* sm, int tid) {
  const int r0 = 32 * tr, c0 = 32 * tc;
  for (int e = tid; e < 1024; e += NTH) {
    const int r = e >> 5, c = e & 31;
    sm[r * 33 + c] = in(r0 + r, c0 + c);
  }
  __syncthreads();
  for (int e = tid; e < 1024; e += NTH) {
    const int c = e >> 5, r = e & 31;
    out(c0 + c, r0 + r, sm[r * 33 + c]);
  }
}

// tunable launch parameters (the group's tuner picks them; see group.cpp)
struct Params {
  int lines_per_task;    // line phases
  int cols_per_task;     // coarse-level phases
  int tiles_per_task;    // transpose phases
  int rad;               // largest radix of the shared-memory FWHT passes (16, 8 or 4)
  int ctas_per_sm;
};

__host__ __device__ inline int nphases(const Inst& I) { return 2 * I.nl + 4; }

// items of phase ph of an instance (forward: fwd = 1)
__host__ __device__ inline int items_of(const Inst& I, int ph, int fwd) {
  const int M = I.G.M, N = I.G.N, L = I.nl;
  if (fwd) {
    if (ph < 2 * L) return 2 << (I.J0 + ph / 2);
    const int k = ph - 2 * L;
    if (k == 0) return (M / 32) * (M / 32);
    if (k == 1) return M;
    if (k == 2) return (M / 32) * (N / 32);
    return N;
  }
  if (ph == 0) return N;
  if (ph == 1) return (N / 32) * (M / 32);
  if (ph == 2) return M;
  if (ph == 3) return (M / 32) * (M / 32);
  const int k = (ph - 4) / 2;                         // analysis level j = R - 2 - k
  return 2 << (I.G.R - 2 - k);
}
// kind of a phase: 0 line, 1 coarse, 2 transpose
__host__ __device__ inline int kind_of(const Inst& I, int ph, int fwd) {
  if (fwd) {
    if (ph < 2 * I.nl) return 1;
    const int k = ph - 2 * I.nl;
    return (k == 0 || k == 2) ? 2 : 0;
  }
  if (ph == 1 || ph == 3) return 2;
  return ph < 4 ? 0 : 1;
}

__device__ void run_item(const Inst& I, const Geo& G, int ph, int it, int fwd, const float* in, float* out,
                         const SmemTables<float>& st, float* sm, int tid) {
  const int M = G.M, N = G.N, Mh = M / 2, L = I.nl;
  if (fwd) {
    if (ph < 2 * L) {
      const int k = ph / 2, j = I.J0 + k;
      const float* S = k == 0 ? in : (((k - 1) & 1) == 0 ? I.XS : I.XS2);
      const int ldS = k == 0 ? M : Mh;
      if ((ph & 1) == 0) syn_row(G, in, S, ldS, I.VT, j, it, st, sm, tid);
      else syn_col(G, I.VT, (k & 1) == 0 ? I.XS : I.XS2, Mh, j, it, st, sm, tid);
      return;
    }
    const int k = ph - 2 * L;
    if (k == 0) {   // the level R-1 array (LL quarter from the last coarse level) into XT, transposed
      const float* Sl = L == 0 ? nullptr : (((L - 1) & 1) == 0 ? I.XS : I.XS2);
      const int nt = M / 32;
      tile_t(
          it / nt, it % nt,
          [&](int r, int c) { return (Sl && r < Mh && c < Mh) ? Sl[(int64_t)r * Mh + c] : in[(int64_t)r * M + c]; },
          [&](int r, int c, float v) { I.XT[(int64_t)r * M + c] = v; }, sm, tid);
      return;
    }
    if (k == 2) {   // VT (M x N) -> V (N x M)
      const int nt = N / 32;
      tile_t(
          it / nt, it % nt, [&](int r, int c) { return I.VT[(int64_t)r * N + c]; },
          [&](int r, int c, float v) { I.V[(int64_t)r * M + c] = v; }, sm, tid);
      return;
    }
    LineIO io{};
    io.jlev = G.R - 1;
    if (k == 1) {
      io.in_stride = M; io.out_stride = N; io.lines = M; io.in_batch = (int64_t)M * M;
      io.out_batch = (int64_t)M * N; io.seq_rows = 0; io.mode = 0;
      line_fwd_one<float>(I.XT, I.VT, st, G, io, it, sm, tid, NTH);
    } else {
      io.in_stride = M; io.lines = N; io.in_batch = (int64_t)N * M; io.out_batch = I.m; io.seq_rows = 1;
      io.mode = 1; io.mask = I.mask; io.prefix = I.prefix; io.pos = I.pos; io.wpr = I.wpr; io.m = I.m;
      io.mask_rows = N;
      line_fwd_one<float>(I.V, out, st, G, io, it, sm, tid, NTH);
    }
    return;
  }
  if (ph == 0 || ph == 2) {
    LineIO io{};
    io.jlev = G.R - 1;
    if (ph == 0) {
      io.out_stride = M; io.lines = N; io.out_batch = (int64_t)N * M; io.seq_rows = 1; io.mode = 1;
      io.mask = I.mask; io.prefix = I.prefix; io.pos = I.pos; io.wpr = I.wpr; io.m = I.m; io.mask_rows = N;
      line_adj_one<float>(in, I.V, st, G, io, it, sm, tid, NTH);
    } else {
      io.in_stride = N; io.out_stride = M; io.lines = M; io.in_batch = (int64_t)M * N; io.out_batch = (int64_t)M * M;
      io.seq_rows = 0; io.mode = 0;
      line_adj_one<float>(I.VT, I.XT, st, G, io, it, sm, tid, NTH);
    }
    return;
  }
  if (ph == 1) {    // V (N x M) -> VT (M x N)
    const int nt = M / 32;
    tile_t(
        it / nt, it % nt, [&](int r, int c) { return I.V[(int64_t)r * M + c]; },
        [&](int r, int c, float v) { I.VT[(int64_t)r * N + c] = v; }, sm, tid);
    return;
  }
  if (ph == 3) {    // XT -> the level R-1 array: LL quarter to XS (or x), the rest to x
    const int nt = M / 32;
    tile_t(
        it / nt, it % nt, [&](int r, int c) { return I.XT[(int64_t)r * M + c]; },
        [&](int r, int c, float v) {
          if (L > 0 && r < Mh && c < Mh) I.XS[(int64_t)r * Mh + c] = v;
          else out[(int64_t)r * M + c] = v;
        },
        sm, tid);
    return;
  }
  const int k = (ph - 4) / 2, j = G.R - 2 - k;
  const float* S = k == 0 ? I.XS : (((k - 1) & 1) == 0 ? I.XS2 : I.XS);
  if (((ph - 4) & 1) == 0) {
    ana_col(G, S, Mh, I.V, j, it, st, sm, tid);
  } else {
    float* Sn = k == L - 1 ? out : ((k & 1) == 0 ? I.XS2 : I.XS);
    ana_row(G, I.V, out, Sn, k == L - 1 ? M : Mh, j, it, st, sm, tid);
  }
}

// smem floats of a task: the staged tables, then the largest item workspace
__host__ __device__ inline int item_floats(const Inst& I) {
  const int line = 2 * I.G.M + padlen(I.G.N);
  return line > 32 * 33 ? line : 32 * 33;
}

// MINB: CTAs per SM the register budget is sized for (2: no spills; 3: a
// few spilled values, more lines in flight); the tuner picks
template <int MINB>
__global__ void __launch_bounds__(NTH, MINB) k_group(const Inst* __restrict__ insts, const Task* __restrict__ tasks,
                                               int ntasks, int* done, int* ticket, unsigned* err, unsigned spin,
                                               int fwd, int rad, const __grid_constant__ Ptrs ptrs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);
  __shared__ int s_t, s_ok;
  const int tid = threadIdx.x;
  int staged = -1;                 // instance whose tables are in shared memory
  SmemTables<float> st{};
  int off = 0;
  for (;;) {
    if (tid == 0) s_t = atomicAdd(ticket, 1);
    __syncthreads();
    const int t = s_t;
    if (t >= ntasks) break;
    const Task tk = tasks[t];
    const Inst& I = insts[tk.inst];
    if (tid == 0) {
      int ok = 1;
      if (tk.phase > 0) {
        const int* c = done + I.done_off + tk.phase - 1;
        const int need = items_of(I, tk.phase - 1, fwd);
        unsigned n = 0;
        while (ld_relaxed(c) < need) {
          if (++n > spin) {
            ok = 0;
            break;
          }
          __nanosleep(64);
        }
        if (ok) (void)ld_acquire(c);
      }
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) {
      if (tid == 0) atomicExch(err, 1u);
      break;
    }
    Geo G = I.G;
    if (tk.inst != staged) {       // consecutive tasks of one instance keep its tables
      off = stage_tables(I.tab, G, sm, st, tid, NTH);
      staged = tk.inst;
      __syncthreads();
    }
    G.rad = rad;
    for (int k = 0; k < tk.nitems; ++k) {
      run_item(I, G, tk.phase, tk.item0 + k, fwd, ptrs.in[tk.inst], ptrs.out[tk.inst], st, sm + off, tid);
      __syncthreads();
    }
    if (tid == 0) {
      __threadfence();
      red_release_add(done + I.done_off + tk.phase, tk.nitems);
    }
  }
}

}  // namespace gk

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct PersistentGroup {
  int n = 0;
  std::vector<gk::Inst> hinst;
  gk::Inst* dinst = nullptr;
  gk::Task* dtasks[2] = {nullptr, nullptr};   // adjoint, forward
  int ntasks[2] = {0, 0};
  int* ddone = nullptr;                       // per-phase counters, then the ticket
  int ncount = 0;
  size_t smem = 0;
  gk::Params prm{1, 4, 4, 16, 0};
  int grid = 0;
};

static int phase_chunk(const gk::Params& prm, int kind) {
  return kind == 0 ? prm.lines_per_task : (kind == 1 ? prm.cols_per_task : prm.tiles_per_task);
}

// the task lists for the current parameters: phase by phase across all instances
static int pgroup_layout(PersistentGroup* g) {
  for (int fwd = 0; fwd < 2; ++fwd) {
    std::vector<gk::Task> t;
    int maxph = 0;
    for (const gk::Inst& I : g->hinst) maxph = std::max(maxph, gk::nphases(I));
    for (int ph = 0; ph < maxph; ++ph)
      for (int i = 0; i < g->n; ++i) {
        const gk::Inst& I = g->hinst[i];
        if (ph >= gk::nphases(I)) continue;
        const int items = gk::items_of(I, ph, fwd), ch = std::max(1, phase_chunk(g->prm, gk::kind_of(I, ph, fwd)));
        for (int a = 0; a < items; a += ch) t.push_back(gk::Task{i, ph, a, std::min(ch, items - a)});
      }
    cudaFree(g->dtasks[fwd]);
    g->dtasks[fwd] = nullptr;
    if (cudaMalloc(&g->dtasks[fwd], t.size() * sizeof(gk::Task)) != cudaSuccess ||
        cudaMemcpy(g->dtasks[fwd], t.data(), t.size() * sizeof(gk::Task), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      set_error(UW_ERR_OOM, "group task list allocation failed");
      return UW_ERR_OOM;
    }
    g->ntasks[fwd] = (int)t.size();
  }
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const void* fn = g->prm.ctas_per_sm == 2 ? (const void*)gk::k_group<2> : (const void*)gk::k_group<3>;
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g->smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, gk::NTH, g->smem);
  per = std::max(1, per);
  if (g->prm.ctas_per_sm > 0) per = std::min(per, g->prm.ctas_per_sm);
  g->grid = per * nsm;
  return UW_OK;
}

void pgroup_destroy(PersistentGroup* g) {
  if (!g) return;
  cudaFree(g->dinst);
  cudaFree(g->dtasks[0]);
  cudaFree(g->dtasks[1]);
  cudaFree(g->ddone);
  delete g;
}

// NULL (and why) if the group does not qualify: 2D plans with M >= 64 and a
// reserved workspace, at most gk::MAXI instances
PersistentGroup* pgroup_create(const Plan* const* plans, int n, std::string& why) {
  if (n > gk::MAXI) {
    why = "more instances than one persistent launch takes";
    return nullptr;
  }
  PersistentGroup* g = new PersistentGroup();
  g->n = n;
  size_t maxf = 0;
  int off = 0;
  for (int i = 0; i < n; ++i) {
    const Plan& P = *plans[i];
    if (P.d != 2 || P.M < 64 || !P.d_work || P.max_batch < 1) {
      why = "persistent launches serve 2D plans with M >= 64";
      pgroup_destroy(g);
      return nullptr;
    }
    gk::Inst I{};
    I.G.p = P.p; I.G.q = P.q; I.G.Q = P.Q; I.G.R = P.R; I.G.M = P.M; I.G.N = P.N; I.G.L = P.R + P.q;
    I.G.bd = P.bd; I.G.ntap = P.ntap; I.G.Lb = P.Lb;
    I.tab = P.t32;
    I.J0 = P.J0;
    I.nl = std::max(0, P.R - 1 - P.J0);
    I.mask = P.d_mask; I.prefix = P.d_prefix; I.pos = P.d_pos; I.wpr = P.wpr; I.m = P.m;
    const size_t M = P.M, N = P.N, Mh = M / 2;
    float* w = (float*)P.d_work;
    I.XS = w;
    I.XS2 = I.XS + Mh * Mh;
    I.XT = I.XS2 + Mh * Mh;
    I.VT = I.XT + M * M;
    I.V = I.VT + M * N;
    I.done_off = off;
    off += gk::nphases(I);
    maxf = std::max(maxf, (size_t)table_count(I.G) + 4 + (size_t)gk::item_floats(I));
    g->hinst.push_back(I);
  }
  g->ncount = off;
  g->smem = maxf * sizeof(float);
  if (cudaMalloc(&g->dinst, n * sizeof(gk::Inst)) != cudaSuccess ||
      cudaMemcpy(g->dinst, g->hinst.data(), n * sizeof(gk::Inst), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMalloc(&g->ddone, (off + 1) * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    why = "group descriptor allocation failed";
    pgroup_destroy(g);
    return nullptr;
  }
  if (pgroup_layout(g) != UW_OK) {
    why = "group task list allocation failed";
    pgroup_destroy(g);
    return nullptr;
  }
  return g;
}

static unsigned group_spin_limit() {
  const char* e = getenv("UW_GROUP_SPIN_LIMIT");
  if (e && *e) return (unsigned)strtoul(e, nullptr, 10);
  return 1u << 24;
}

// one launch over every instance; the counters start from zero on the stream
int pgroup_run(PersistentGroup* g, bool fwd, const void* const* in, void* const* out, unsigned* err, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  gk::Ptrs ptrs{};
  for (int i = 0; i < g->n; ++i) {
    ptrs.in[i] = (const float*)in[i];
    ptrs.out[i] = (float*)out[i];
  }
  if (cudaMemsetAsync(g->ddone, 0, (g->ncount + 1) * sizeof(int), s) != cudaSuccess) {
    set_error(UW_ERR_CUDA, "counter reset failed");
    return UW_ERR_CUDA;
  }
  const int f = fwd ? 1 : 0;
  if (g->prm.ctas_per_sm == 2)
    gk::k_group<2><<<g->grid, gk::NTH, g->smem, s>>>(g->dinst, g->dtasks[f], g->ntasks[f], g->ddone,
                                                     g->ddone + g->ncount, err, group_spin_limit(), f, g->prm.rad, ptrs);
  else
    gk::k_group<3><<<g->grid, gk::NTH, g->smem, s>>>(g->dinst, g->dtasks[f], g->ntasks[f], g->ddone,
                                                     g->ddone + g->ncount, err, group_spin_limit(), f, g->prm.rad, ptrs);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(UW_ERR_CUDA, std::string("persistent group launch failed: ") + cudaGetErrorString(e));
    return UW_ERR_CUDA;
  }
  return UW_OK;
}

int pgroup_set_params(PersistentGroup* g, int lines, int cols, int tiles, int rad, int ctas) {
  g->prm = gk::Params{std::max(1, lines), std::max(1, cols), std::max(1, tiles),
                      rad >= 16 ? 16 : (rad >= 8 ? 8 : 4), std::max(0, ctas)};
  return pgroup_layout(g);
}

void pgroup_params(const PersistentGroup* g, int* p5) {
  p5[0] = g->prm.lines_per_task;
  p5[1] = g->prm.cols_per_task;
  p5[2] = g->prm.tiles_per_task;
  p5[3] = g->prm.rad;
  p5[4] = g->prm.ctas_per_sm;
}

}  // namespace uw
