// Device helpers shared by the CUDA translation units of libuw: index
// helpers, table staging, and the per-output formulas of one synthesis /
// analysis level, of T and T^T, and the shared-memory Walsh-Hadamard passes.
// Paper: V. Antun, arXiv 2106.00554 (Sec. 3.1 FWHT, Sec. 3.2 DWT, Sec. 4.1 T).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "uw_internal.h"

namespace uw {

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int padi(int i) { return i + (i >> 4); }
__host__ __device__ __forceinline__ int padlen(int n) { return n + (n >> 4) + 1; }

__device__ __forceinline__ int seqrow(int n, int L) {
  return L == 0 ? 0 : (int)(__brev((unsigned)(n ^ (n >> 1))) >> (32 - L));
}

template <typename T>
struct SmemTables {  // tables staged in shared memory for one CTA
  T* h; T* g; T* taps; T* EL; T* ER; T* PL; T* QL; T* PR; T* QR;
};

struct Geo {  // geometry of one plan, passed by value
  int p, q, Q, R, M, N, L, bd, ntap, Lb;
  int rad = 16;  // largest radix of the shared-memory FWHT passes (16, 8 or 4)
};

__host__ __device__ inline int table_count(const Geo& G) {
  return 4 * G.p + G.ntap + 2 * G.p * G.ntap + 4 * G.p * G.Lb;
}

// Copy the tables into shared memory.  The host packs them contiguously in
// this order starting at t.h, so one batched loop moves them (every thread
// issues its loads before its stores).
template <typename T>
__device__ int stage_tables(const Tables<T>& t, const Geo& G, T* base, SmemTables<T>& s, int tid, int nthr) {
  const int n = table_count(G);
  constexpr int K = 8;
  for (int i0 = 0; i0 < n; i0 += K * nthr) {
    T a[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      int i = i0 + k * nthr + tid;
      a[k] = i < n ? t.h[i] : T(0);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      int i = i0 + k * nthr + tid;
      if (i < n) base[i] = a[k];
    }
  }
  s.h = base;
  s.g = s.h + 2 * G.p;
  s.taps = s.g + 2 * G.p;
  s.EL = s.taps + G.ntap;
  s.ER = s.EL + G.p * G.ntap;
  s.PL = s.ER + G.p * G.ntap;
  s.QL = s.PL + G.p * G.Lb;
  s.PR = s.QL + G.p * G.Lb;
  s.QR = s.PR + G.p * G.Lb;
  return n;
}


// Accessors: plain array, or padded shared-memory array.
template <typename T>
struct Plain {
  const T* a;
  __device__ __forceinline__ T operator[](int i) const { return a[i]; }
};
template <typename T>
struct Padded {
  const T* a;
  __device__ __forceinline__ T operator[](int i) const { return a[padi(i)]; }
};
template <typename T>
struct Strided {
  const T* a;
  int64_t s;
  __device__ __forceinline__ T operator[](int i) const { return a[(int64_t)i * s]; }
};

// ---------------------------------------------------------------------------
// one synthesis output (level j -> j+1): s_{j+1}[k] from lo = s_j, hi = d_j
// (Sec. 3.2: interior phi_{j,m} = sum_l h_l phi_{j+1,2m+l}, psi with g; the
// p edge functions at each side through the level-independent blocks).
// ---------------------------------------------------------------------------
template <typename T, typename AL, typename AH, typename TB>
__device__ __forceinline__ T syn_one(int k, int n0, const AL& lo, const AH& hi, const TB& t, const Geo& G) {
  const int p = G.p, n1 = 2 * n0;
  T acc = 0;
  if (G.bd == UW_BOUNDARY_PERIODIC) {
    for (int l = -p + 1; l <= p; ++l) {
      int km = k - l;
      km %= n1;
      if (km < 0) km += n1;
      if (km & 1) continue;
      int m = km >> 1;
      acc += t.h[l + p - 1] * lo[m] + t.g[l + p - 1] * hi[m];
    }
    return acc;
  }
  int mlo = max(p, (k - p + 1) >> 1);       // ceil((k - p) / 2): k - 2m <= p
  int mhi = min(n0 - p - 1, (k + p - 1) >> 1);
  for (int m = mlo; m <= mhi; ++m) {
    int l = k - 2 * m;
    acc += t.h[l + p - 1] * lo[m] + t.g[l + p - 1] * hi[m];
  }
  if (k < G.Lb)
    for (int m = 0; m < p; ++m) acc += t.PL[m * G.Lb + k] * lo[m] + t.QL[m * G.Lb + k] * hi[m];
  int c = n1 - 1 - k;
  if (c < G.Lb)
    for (int r = 0; r < p; ++r) acc += t.PR[r * G.Lb + c] * lo[n0 - 1 - r] + t.QR[r * G.Lb + c] * hi[n0 - 1 - r];
  return acc;
}

// one analysis output pair (level j+1 -> j): lo[m], hi[m] from s (length n1)
template <typename T, typename AS, typename TB>
__device__ __forceinline__ void ana_one(int m, int n0, const AS& s, const TB& t, const Geo& G, T& lo, T& hi) {
  const int p = G.p, n1 = 2 * n0;
  T a = 0, b = 0;
  if (G.bd == UW_BOUNDARY_PERIODIC) {
    for (int l = -p + 1; l <= p; ++l) {
      int k = (2 * m + l) % n1;
      if (k < 0) k += n1;
      T v = s[k];
      a += t.h[l + p - 1] * v;
      b += t.g[l + p - 1] * v;
    }
  } else if (m < p) {
    for (int c = 0; c < G.Lb; ++c) {
      T v = s[c];
      a += t.PL[m * G.Lb + c] * v;
      b += t.QL[m * G.Lb + c] * v;
    }
  } else if (m >= n0 - p) {
    int r = n0 - 1 - m;
    for (int c = 0; c < G.Lb; ++c) {
      T v = s[n1 - 1 - c];
      a += t.PR[r * G.Lb + c] * v;
      b += t.QR[r * G.Lb + c] * v;
    }
  } else {
    for (int l = -p + 1; l <= p; ++l) {
      T v = s[2 * m + l];
      a += t.h[l + p - 1] * v;
      b += t.g[l + p - 1] * v;
    }
  }
  lo = a;
  hi = b;
}

// one output of T (upsample by Q = 2^q, convolve with the cell integrals):
// v[k] = 2^{-R/2} (sum_{m interior} s[m] I_q[k - Q m] + edge rows)
template <typename T, typename AS, typename TB>
__device__ __forceinline__ T up_one(int k, const AS& s, const TB& t, const Geo& G) {
  const int p = G.p, Q = G.Q, M = G.M, N = G.N;
  T acc = 0;
  const int mbase = (k >> G.q) + (p - 1);
  const int t0 = k - mbase * Q + (p - 1) * Q;  // index into taps for j = 0
  for (int j = 0; j < 2 * p - 1; ++j) {
    int m = mbase - j;
    T tap = t.taps[t0 + j * Q];
    if (G.bd == UW_BOUNDARY_PERIODIC) {
      int mm = m % M;
      if (mm < 0) mm += M;
      acc += tap * s[mm];
    } else if (m >= p && m <= M - p - 1) {
      acc += tap * s[m];
    }
  }
  if (G.bd == UW_BOUNDARY_VMP) {
    if (k < G.ntap)
      for (int m = 0; m < p; ++m) acc += t.EL[m * G.ntap + k] * s[m];
    int kk = N - 1 - k;
    if (kk < G.ntap)
      for (int r = 0; r < p; ++r) acc += t.ER[r * G.ntap + kk] * s[M - 1 - r];
  }
  return acc;
}

// one output of T^T: s[m] = 2^{-R/2} sum_k T[k, m] v[k]
template <typename T, typename AV, typename TB>
__device__ __forceinline__ T upT_one(int m, const AV& v, const TB& t, const Geo& G) {
  const int p = G.p, Q = G.Q, M = G.M, N = G.N;
  T acc = 0;
  const int tmin = (-p + 1) * Q;
  if (G.bd == UW_BOUNDARY_PERIODIC) {
    for (int i = 0; i < G.ntap; ++i) {
      int k = (Q * m + tmin + i) % N;
      if (k < 0) k += N;
      acc += t.taps[i] * v[k];
    }
  } else if (m < p) {
    for (int k = 0; k < G.ntap; ++k) acc += t.EL[m * G.ntap + k] * v[k];
  } else if (m >= M - p) {
    int r = M - 1 - m;
    for (int kk = 0; kk < G.ntap; ++kk) acc += t.ER[r * G.ntap + kk] * v[N - 1 - kk];
  } else {
    const int k0 = Q * m + tmin;
    for (int i = 0; i < G.ntap; ++i) acc += t.taps[i] * v[k0 + i];
  }
  return acc;
}

// ---------------------------------------------------------------------------
// natural-order Walsh-Hadamard transform of a padded shared-memory line of
// length 2^L: radix-16 pencils in registers, one shared-memory round trip per
// 4 bits (pad of 1 word per 16 keeps the three access strides conflict-free).
// ---------------------------------------------------------------------------
template <typename T, int RAD>
__device__ __forceinline__ void fwht_pass(T* v, int L, int done, int tid, int nthr) {
  const int N = 1 << L;
  const int stride = 1 << done;
  const int npencil = N / RAD;
  for (int pc = tid; pc < npencil; pc += nthr) {
    int lowp = pc & (stride - 1);
    int highp = pc >> done;
    int base = lowp + highp * stride * RAD;
    T a[RAD];
#pragma unroll
    for (int i = 0; i < RAD; ++i) a[i] = v[padi(base + i * stride)];
#pragma unroll
    for (int hh = 1; hh < RAD; hh <<= 1)
#pragma unroll
      for (int i = 0; i < RAD; ++i)
        if (!(i & hh)) {
          T x = a[i], y = a[i + hh];
          a[i] = x + y;
          a[i + hh] = x - y;
        }
#pragma unroll
    for (int i = 0; i < RAD; ++i) v[padi(base + i * stride)] = a[i];
  }
}

template <typename T>
__device__ void fwht_smem(T* v, int L, int tid, int nthr, int rad = 16) {
  const int rb = rad >= 16 ? 4 : (rad >= 8 ? 3 : 2);
  int done = 0;
  while (done < L) {
    int r = min(rb, L - done);
    if (r == 4) fwht_pass<T, 16>(v, L, done, tid, nthr);
    else if (r == 3) fwht_pass<T, 8>(v, L, done, tid, nthr);
    else if (r == 2) fwht_pass<T, 4>(v, L, done, tid, nthr);
    else fwht_pass<T, 2>(v, L, done, tid, nthr);
    __syncthreads();
    done += r;
  }
}

// ---------------------------------------------------------------------------
// Fused line operators (one line per CTA, whole line in shared memory).
// ---------------------------------------------------------------------------
struct LineIO {
  // input / output addressing
  int64_t in_stride;     // elements between consecutive input lines
  int64_t out_stride;    // elements between consecutive output lines
  int lines;             // lines per batch instance
  int64_t in_batch;      // elements between batch instances (input)
  int64_t out_batch;     // elements between batch instances (output)
  int seq_rows;          // 1: line index is a sequency row n1; the data row is r(n1)
  int mode;              // forward: 0 store natural, 1 gather; adjoint: 0 load natural, 1 scatter
  int jlev;              // forward: first synthesis level; adjoint: last analysis level
  const uint32_t* mask;
  const int32_t* prefix;
  int wpr;               // mask words per row
  int64_t m;             // samples per instance
  int mask_rows;         // 1 for d = 1 (all lines use row 0), else = lines
  const uint16_t* pos;   // per sample: natural FWHT position in its row (or null)
};

// One line of the generic line operators, one CTA (any size), the whole
// line in shared memory at sm (2 M + padlen(N) values of T).  `item` is the
// line's index over all batch instances (line = item % io.lines).
// Forward: synthesis levels jlev .. R-1 of one line, T, natural-order FWHT,
// then the natural line is stored or the sampled sequency indices gathered.
template <typename T>
__device__ void line_fwd_one(const T* __restrict__ in, T* __restrict__ out, const SmemTables<T>& st, const Geo& G,
                             const LineIO& io, int item, T* sm, int tid, int nthr) {
  T* s0 = sm;
  T* s1 = s0 + G.M;
  T* v = s1 + G.M;
  const int line = item % io.lines;
  const int64_t b = item / io.lines;
  const int drow = io.seq_rows ? seqrow(line, G.L) : line;
  const T* src = in + b * io.in_batch + (int64_t)drow * io.in_stride;
  for (int i = tid; i < G.M; i += nthr) s0[i] = src[i];
  __syncthreads();
  // (a) synthesis levels jlev .. R-1; the last output must land in s1
  const int nlev = G.R - io.jlev;
  T* A = s0;
  T* Bf = (nlev & 1) ? s1 : v;
  for (int j = io.jlev; j < G.R; ++j) {
    const int n0 = 1 << j;
    Plain<T> lo{A}, hi{s0 + n0};
    for (int k = tid; k < 2 * n0; k += nthr) Bf[k] = syn_one<T>(k, n0, lo, hi, st, G);
    __syncthreads();
    T* nb = (A == s0) ? ((Bf == s1) ? v : s1) : A;
    A = Bf;
    Bf = nb;
  }
  if (nlev == 0) {
    for (int i = tid; i < G.M; i += nthr) s1[i] = s0[i];
    __syncthreads();
  }
  // (b) v = T s, scaled by 2^{-R/2}
  const T sc = (T)exp2(-0.5 * (double)G.R);
  {
    Plain<T> s{s1};
    for (int k = tid; k < G.N; k += nthr) v[padi(k)] = sc * up_one<T>(k, s, st, G);
  }
  __syncthreads();
  // (c) natural-order FWHT
  fwht_smem<T>(v, G.L, tid, nthr, G.rad);
  // (d) store natural order, or gather the sampled sequency indices
  if (io.mode == 0) {
    T* dst = out + b * io.out_batch + (int64_t)line * io.out_stride;
    for (int k = tid; k < G.N; k += nthr) dst[k] = v[padi(k)];
  } else {
    const int mrow = io.mask_rows == 1 ? 0 : line;
    const uint32_t* mk = io.mask + (int64_t)mrow * io.wpr;
    const int32_t* pf = io.prefix + (int64_t)mrow * io.wpr;
    T* y = out + b * io.m;
    for (int w = tid; w < io.wpr; w += nthr) {
      uint32_t bits = mk[w];
      int64_t pos = pf[w];
      while (bits) {
        int bb = __ffs(bits) - 1;
        bits &= bits - 1;
        int n = w * 32 + bb;
        y[pos++] = v[padi(seqrow(n, G.L))];
      }
    }
  }
}

// Adjoint of line_fwd_one: load the natural line or scatter the samples,
// FWHT (H is symmetric), T^T, analysis levels R-1 .. jlev.
template <typename T>
__device__ void line_adj_one(const T* __restrict__ in, T* __restrict__ out, const SmemTables<T>& st, const Geo& G,
                             const LineIO& io, int item, T* sm, int tid, int nthr) {
  T* s0 = sm;
  T* s1 = s0 + G.M;
  T* v = s1 + G.M;
  const int line = item % io.lines;
  const int64_t b = item / io.lines;
  if (io.mode == 0) {
    const T* src = in + b * io.in_batch + (int64_t)line * io.in_stride;
    for (int k = tid; k < G.N; k += nthr) v[padi(k)] = src[k];
  } else {
    for (int k = tid; k < padlen(G.N); k += nthr) v[k] = 0;
    __syncthreads();
    const int mrow = io.mask_rows == 1 ? 0 : line;
    const uint32_t* mk = io.mask + (int64_t)mrow * io.wpr;
    const int32_t* pf = io.prefix + (int64_t)mrow * io.wpr;
    const T* y = in + b * io.m;
    for (int w = tid; w < io.wpr; w += nthr) {
      uint32_t bits = mk[w];
      int64_t pos = pf[w];
      while (bits) {
        int bb = __ffs(bits) - 1;
        bits &= bits - 1;
        int n = w * 32 + bb;
        v[padi(seqrow(n, G.L))] = y[pos++];
      }
    }
  }
  __syncthreads();
  // (c^T) the Hadamard matrix is symmetric: same transform
  fwht_smem<T>(v, G.L, tid, nthr, G.rad);
  // (b^T) s = T^T v
  const T sc = (T)exp2(-0.5 * (double)G.R);
  {
    Padded<T> vv{v};
    for (int m = tid; m < G.M; m += nthr) s1[m] = sc * upT_one<T>(m, vv, st, G);
  }
  __syncthreads();
  // (a^T) analysis levels R-1 .. jlev; details go straight to s0
  T* A = s1;
  T* Bf = v;
  for (int j = G.R - 1; j >= io.jlev; --j) {
    const int n0 = 1 << j;
    Plain<T> s{A};
    for (int m = tid; m < n0; m += nthr) {
      T lo, hi;
      ana_one<T>(m, n0, s, st, G, lo, hi);
      Bf[m] = lo;
      s0[n0 + m] = hi;
    }
    __syncthreads();
    T* t = A;
    A = Bf;
    Bf = t;
  }
  const int nlo = 1 << io.jlev;
  for (int i = tid; i < nlo; i += nthr) s0[i] = A[i];
  __syncthreads();
  const int drow = io.seq_rows ? seqrow(line, G.L) : line;
  T* dst = out + b * io.out_batch + (int64_t)drow * io.out_stride;
  for (int i = tid; i < G.M; i += nthr) dst[i] = s0[i];
}

// position of the (r+1)-th set bit of x (0 <= r < popc(x)), branch-free
__device__ __forceinline__ int select_bit(unsigned x, int r) {
  int pos = 0, c;
  c = __popc(x & 0xFFFFu); if (r >= c) { r -= c; x >>= 16; pos += 16; }
  c = __popc(x & 0xFFu);   if (r >= c) { r -= c; x >>= 8;  pos += 8; }
  c = __popc(x & 0xFu);    if (r >= c) { r -= c; x >>= 4;  pos += 4; }
  c = __popc(x & 0x3u);    if (r >= c) { r -= c; x >>= 2;  pos += 2; }
  c = x & 1u;              if (r >= c) { pos += 1; }
  return pos;
}

// The sampled sequency indices of one mask row, one sample per thread: the
// row's words and word prefixes are staged in shared memory, a binary search
// finds the word of sample j and select_bit its bit.  Returns the row's first
// packed position r0 and its sample count; fills smask / spre.
__device__ __forceinline__ void stage_row(const LineIO& io, int mrow, int rows, uint32_t* smask, int* spre,
                                          int64_t& r0, int& cnt, int tid, int nthr) {
  const uint32_t* mk = io.mask + (int64_t)mrow * io.wpr;
  const int32_t* pf = io.prefix + (int64_t)mrow * io.wpr;
  r0 = pf[0];
  const int64_t r1 = (mrow + 1 < rows) ? (int64_t)io.prefix[(int64_t)(mrow + 1) * io.wpr] : io.m;
  cnt = (int)(r1 - r0);
  for (int w = tid; w < io.wpr; w += nthr) {
    smask[w] = mk[w];
    spre[w] = (int)(pf[w] - r0);
  }
}

__device__ __forceinline__ int sample_index(const uint32_t* smask, const int* spre, int wpr, int j) {
  int lo = 0, hi = wpr - 1;  // last word with spre[w] <= j
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (spre[mid] <= j) lo = mid;
    else hi = mid - 1;
  }
  return lo * 32 + select_bit(smask[lo], j - spre[lo]);
}

// Programmatic dependent launch: a kernel launched with launch_pdl may start
// while the previous kernel in the stream is still running; it stages its
// constant tables, lets the next kernel launch (pdl_trigger), and waits for
// the previous grid's completion and memory (pdl_wait) before it reads that
// grid's output or writes any global memory.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// [p, p + bytes) into L2 by bulk prefetches of up to 64 KB (one thread);
// skipped unless p and bytes are multiples of 16
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, int64_t bytes) {
  if ((reinterpret_cast<uintptr_t>(p) & 15) || (bytes & 15)) return;
  const char* a = reinterpret_cast<const char*>(p);
  for (int64_t o = 0; o < bytes; o += 65536) {
    const uint32_t n = (uint32_t)(bytes - o < 65536 ? bytes - o : 65536);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(a + o), "r"(n) : "memory");
  }
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// raise a kernel's dynamic shared-memory limit to the device maximum (once)
cudaError_t set_smem_limit(const void* fn);

// kernels_tc.cu: split-BF16 tensor-core line operators (last level only)
bool tc_eligible(const Plan& P, const LineIO& io, const void* in, const void* out, bool fwd);
cudaError_t tc_launch(bool fwd, const Plan& P, const float* in, float* out, const LineIO& io, int total,
                      cudaStream_t s);

// kernels_umma.cu: split-BF16 line operators on tcgen05 (last level, N = 4096, q = 1)
bool umma_eligible(const Plan& P, const LineIO& io, const void* in, const void* out, bool fwd, int total);
cudaError_t umma_launch(bool fwd, const Plan& P, const float* in, float* out, const LineIO& io, int total,
                        cudaStream_t s);

// kernels_f32.cu: persistent FP32 line operators (last level, N = 2048 / 4096)
bool f32_eligible(const Plan& P, const LineIO& io, const void* in, const void* out, bool fwd);
// long 1D lines on FP32 (kernels_f32.cu)
bool f32_seg_eligible(const Plan& P);
cudaError_t f32_seg_up(const Plan& P, const Geo& G, const float* s, float* v, int batch, cudaStream_t st);
cudaError_t f32_seg_fwht_upT(const Plan& P, const Geo& G, float* v, float* s, int batch, cudaStream_t st);
cudaError_t f32_syn1d_levels(const Plan& P, const Geo& G, const float* x, float* out, int jto, size_t smem, int batch,
                             cudaStream_t st);
cudaError_t f32_ana1d_levels(const Plan& P, const Geo& G, const float* in, float* x, int jfrom, size_t smem,
                             int batch, cudaStream_t st);
cudaError_t f32_syn1d_level(const Plan& P, const Geo& G, const float* lo, const float* hi, float* out, int n0, int batch,
                            cudaStream_t st);
cudaError_t f32_ana1d_level(const Plan& P, const Geo& G, const float* in, float* lo, float* hi, int n0, int batch,
                            cudaStream_t st);
cudaError_t f32_launch(bool fwd, const Plan& P, const float* in, float* out, const LineIO& io, int total,
                       cudaStream_t s);

// kernels_line.cu: register-blocked FP32 line operators
bool line2_eligible(const Plan& P);
cudaError_t line2_launch(bool fwd, const Plan& P, const Geo& G, const float* in, float* out, const LineIO& io,
                         int nblocks, cudaStream_t s);

}  // namespace uw
