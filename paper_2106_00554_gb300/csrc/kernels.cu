// CUDA kernels of libuw (sm_103a) and the forward / adjoint half of the C ABI.
//
// Paper: V. Antun, arXiv 2106.00554.  One product y = P_Omega U x is
//   (a) the IDWT from C_{psi,R} to B_{phi,R} (Remark 4.2; Sec. 3.2 bases),
//   (b) the upsample-by-2^q convolution with the cell integrals of phi and the
//       boundary rows, v = T s  (the D_l / Prop. 4.4 content of Sec. 4.1,
//       summed over l in the space domain so that one FWHT suffices),
//   (c) the sequency-ordered FWHT of size N (Sec. 3.1),
//   (d) the selection P_Omega (Sec. 1.1).
// The adjoint runs (d)..(a) transposed (Sec. 4.2).  In 2D (Sec. 5,
// Algorithm 2) the coarse levels of the Mallat IDWT run first; the last level
// is separable and is fused with (b)-(c) into a "line operator" applied along
// dimension 1 and then along dimension 2.
//
// Sequency order without a permutation pass: by Def. 3.1, with x = k / N,
// w_n(k/N) = (-1)^{sum_j (n^(j) xor n^(j+1)) k^(L+1-j)} = (-1)^{popcount(r(n) & k)},
// r(n) = bitreverse_L(n xor (n >> 1)).  So the natural-order (Hadamard) FWHT
// output at index r(n) is the sequency coefficient n, and (d) reads it there.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <type_traits>
#include <vector>

#include "uw_internal.h"

#include "line_common.cuh"

namespace uw {

template <typename T>
__global__ void __launch_bounds__(256) k_line_fwd(const T* __restrict__ in, T* __restrict__ out,
                                                  Tables<T> tab, Geo G, LineIO io) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  SmemTables<T> st;
  const int off = stage_tables(tab, G, sm, st, tid, nthr);
  pdl_trigger();
  pdl_wait();
  line_fwd_one<T>(in, out, st, G, io, blockIdx.x, sm + off, tid, nthr);
}

template <typename T>
__global__ void __launch_bounds__(256) k_line_adj(const T* __restrict__ in, T* __restrict__ out,
                                                  Tables<T> tab, Geo G, LineIO io) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  SmemTables<T> st;
  const int off = stage_tables(tab, G, sm, st, tid, nthr);
  pdl_trigger();
  pdl_wait();
  line_adj_one<T>(in, out, st, G, io, blockIdx.x, sm + off, tid, nthr);
}

// ---------------------------------------------------------------------------
// Global-memory kernels: one level of synthesis / analysis along lines with
// arbitrary strides (2D coarse levels, 1D fallback), T and T^T, FWHT split in
// two passes, gather / scatter, tiled transpose.
// ---------------------------------------------------------------------------
struct LineGeom {
  int64_t line_stride, elem_stride, batch_stride;
  int lines;          // lines per batch instance
  int lines_fastest;  // 1: consecutive threads walk lines (column access)
};

template <typename T>
__global__ void k_syn_level(const T* __restrict__ in, T* __restrict__ out, int n0, Tables<T> t, Geo G,
                            LineGeom gi, LineGeom go, int batch) {
  const int n1 = 2 * n0;
  const int64_t total = (int64_t)batch * gi.lines * n1;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int line, k;
    int64_t b;
    if (gi.lines_fastest) {
      line = (int)(idx % gi.lines);
      int64_t r = idx / gi.lines;
      k = (int)(r % n1);
      b = r / n1;
    } else {
      k = (int)(idx % n1);
      int64_t r = idx / n1;
      line = (int)(r % gi.lines);
      b = r / gi.lines;
    }
    const T* base = in + b * gi.batch_stride + line * gi.line_stride;
    Strided<T> lo{base, gi.elem_stride}, hi{base + n0 * gi.elem_stride, gi.elem_stride};
    out[b * go.batch_stride + line * go.line_stride + k * go.elem_stride] = syn_one<T>(k, n0, lo, hi, t, G);
  }
}

template <typename T>
__global__ void k_ana_level(const T* __restrict__ in, T* __restrict__ out, int n0, Tables<T> t, Geo G,
                            LineGeom gi, LineGeom go, int batch) {
  const int64_t total = (int64_t)batch * gi.lines * n0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int line, m;
    int64_t b;
    if (gi.lines_fastest) {
      line = (int)(idx % gi.lines);
      int64_t r = idx / gi.lines;
      m = (int)(r % n0);
      b = r / n0;
    } else {
      m = (int)(idx % n0);
      int64_t r = idx / n0;
      line = (int)(r % gi.lines);
      b = r / gi.lines;
    }
    const T* base = in + b * gi.batch_stride + line * gi.line_stride;
    Strided<T> s{base, gi.elem_stride};
    T lo, hi;
    ana_one<T>(m, n0, s, t, G, lo, hi);
    T* ob = out + b * go.batch_stride + line * go.line_stride;
    ob[m * go.elem_stride] = lo;
    ob[(n0 + m) * go.elem_stride] = hi;
  }
}

// 1D lines longer than one CTA's shared memory, batched along blockIdx.x
// (one line per CTA): the coarse synthesis levels J0 .. jto-1 of a line in
// shared memory (Sec. 3.2, the Mallat IDWT), ping-ponging between two
// buffers of 2^(jto-1).  Level j reads s_j from shared memory (the
// coarsest block from x) and the details d_j = x[2^j, 2^(j+1)) from global
// memory; the last of these levels writes s_jto to out[0, 2^jto) of the line.
template <typename T>
__global__ void __launch_bounds__(1024) k_syn1d_levels(const T* __restrict__ x, T* __restrict__ out, int64_t out_bs,
                                                       Tables<T> tab, Geo G, int J0, int jto, int64_t in_bs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  SmemTables<T> st;
  const int off = stage_tables(tab, G, sm, st, tid, nthr);
  pdl_trigger();
  pdl_wait();
  const T* xb = x + (int64_t)blockIdx.x * in_bs;
  T* ob = out + (int64_t)blockIdx.x * out_bs;
  // the whole line of coefficients into L2: each level here and the level
  // kernels after this one read their details from there instead of DRAM
  if (tid == 0) prefetch_l2_bulk(xb, (int64_t)sizeof(T) * in_bs);
  T* P0 = sm + ((off + 3) & ~3);
  T* P1 = P0 + (1 << (jto - 1));
  for (int k = tid; k < (1 << J0); k += nthr) P0[k] = xb[k];
  __syncthreads();
  T* src = P0;
  T* dst = P1;
  for (int j = J0; j < jto; ++j) {
    const int n0 = 1 << j;
    Plain<T> lo{src}, hi{xb + n0};
    T* o = j + 1 == jto ? ob : dst;
    for (int k = tid; k < 2 * n0; k += nthr) o[k] = syn_one<T>(k, n0, lo, hi, st, G);
    __syncthreads();
    T* t = src;
    src = dst;
    dst = t;
  }
}

// The transposed steps: the analysis levels jfrom-1 .. J0 of a line.  The
// first reads s_jfrom from in[0, 2^jfrom) of the line; every level writes
// its details d_j to x[2^j, 2^(j+1)) and its s_j to shared memory, the last
// one s_J0 to x[0, 2^J0).
template <typename T>
__global__ void __launch_bounds__(1024) k_ana1d_levels(const T* __restrict__ in, int64_t in_bs, T* __restrict__ x,
                                                       Tables<T> tab, Geo G, int J0, int jfrom, int64_t out_bs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  SmemTables<T> st;
  const int off = stage_tables(tab, G, sm, st, tid, nthr);
  pdl_trigger();
  pdl_wait();
  const T* ib = in + (int64_t)blockIdx.x * in_bs;
  T* xb = x + (int64_t)blockIdx.x * out_bs;
  T* P0 = sm + ((off + 3) & ~3);
  T* P1 = P0 + (1 << (jfrom - 1));
  const T* src = ib;
  T* dst = P0;
  for (int j = jfrom - 1; j >= J0; --j) {
    const int n0 = 1 << j;
    Plain<T> s{src};
    T* lo_out = j == J0 ? xb : dst;
    for (int m = tid; m < n0; m += nthr) {
      T lo, hi;
      ana_one<T>(m, n0, s, st, G, lo, hi);
      lo_out[m] = lo;
      xb[n0 + m] = hi;
    }
    __syncthreads();
    src = dst;
    dst = dst == P0 ? P1 : P0;
  }
}

// One synthesis level of a batch of 1D lines with the low-pass and detail
// inputs in separate arrays: out[k] = Syn(lo, hi)[k], k < 2 n0.
template <typename T>
__global__ void k_syn1d_level(const T* __restrict__ lo, int64_t lo_bs, const T* __restrict__ hi, int64_t hi_bs,
                              T* __restrict__ out, int64_t out_bs, int n0, Tables<T> t, Geo G, int batch) {
  const int64_t total = (int64_t)batch * 2 * n0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx % (2 * n0));
    const int64_t b = idx / (2 * n0);
    Plain<T> l{lo + b * lo_bs}, h{hi + b * hi_bs};
    out[b * out_bs + k] = syn_one<T>(k, n0, l, h, t, G);
  }
}

// One analysis level of a batch of 1D lines: lo to one array, the details
// hi to another.
template <typename T>
__global__ void k_ana1d_level(const T* __restrict__ in, int64_t in_bs, T* __restrict__ lo, int64_t lo_bs,
                              T* __restrict__ hi, int64_t hi_bs, int n0, Tables<T> t, Geo G, int batch) {
  const int64_t total = (int64_t)batch * n0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int m = (int)(idx % n0);
    const int64_t b = idx / n0;
    Plain<T> s{in + b * in_bs};
    T l, h;
    ana_one<T>(m, n0, s, t, G, l, h);
    lo[b * lo_bs + m] = l;
    hi[b * hi_bs + m] = h;
  }
}

template <typename T>
__global__ void k_up(const T* __restrict__ s, T* __restrict__ v, Tables<T> t, Geo G, int batch) {
  const T sc = (T)exp2(-0.5 * (double)G.R);
  const int64_t total = (int64_t)batch * G.N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int k = (int)(idx % G.N);
    int64_t b = idx / G.N;
    Plain<T> sa{s + b * G.M};
    v[idx] = sc * up_one<T>(k, sa, t, G);
  }
}

template <typename T>
__global__ void k_upT(const T* __restrict__ v, T* __restrict__ s, Tables<T> t, Geo G, int batch) {
  const T sc = (T)exp2(-0.5 * (double)G.R);
  const int64_t total = (int64_t)batch * G.M;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int m = (int)(idx % G.M);
    int64_t b = idx / G.M;
    Plain<T> va{v + b * G.N};
    s[idx] = sc * upT_one<T>(m, va, t, G);
  }
}

// FWHT on contiguous segments of length 2^L2 (one segment per CTA)
template <typename T>
__global__ void __launch_bounds__(256) k_fwht_seg(T* __restrict__ x, int L2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* v = reinterpret_cast<T*>(smem_raw);
  const int n = 1 << L2;
  T* seg = x + (int64_t)blockIdx.x * n;
  for (int k = threadIdx.x; k < n; k += blockDim.x) v[padi(k)] = seg[k];
  __syncthreads();
  fwht_smem<T>(v, L2, threadIdx.x, blockDim.x);
  for (int k = threadIdx.x; k < n; k += blockDim.x) seg[k] = v[padi(k)];
}

// FWHT across segments: length 2^L1 with stride 2^L2; a CTA takes COLS
// adjacent columns (coalesced rows of COLS elements).
template <typename T, int COLS>
__global__ void __launch_bounds__(256) k_fwht_cols(T* __restrict__ x, int L1, int L2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* v = reinterpret_cast<T*>(smem_raw);
  const int n1 = 1 << L1, n2 = 1 << L2;
  const int tiles = n2 / COLS;
  const int64_t b = blockIdx.x / tiles;
  const int c0 = (blockIdx.x % tiles) * COLS;
  T* base = x + b * ((int64_t)n1 * n2) + c0;
  // element (r, c) of the tile lives at v[c * padlen(n1) + padi(r)]
  const int pl = padlen(n1);
  for (int i = threadIdx.x; i < n1 * COLS; i += blockDim.x) {
    int r = i / COLS, c = i % COLS;
    v[c * pl + padi(r)] = base[(int64_t)r * n2 + c];
  }
  __syncthreads();
  // each column is an independent transform; split the threads over columns
  const int per = blockDim.x / COLS;
  const int c = threadIdx.x / per, tl = threadIdx.x % per;
  T* col = v + c * pl;
  int done = 0;
  while (done < L1) {
    int r = min(4, L1 - done);
    if (r == 4) fwht_pass<T, 16>(col, L1, done, tl, per);
    else if (r == 3) fwht_pass<T, 8>(col, L1, done, tl, per);
    else if (r == 2) fwht_pass<T, 4>(col, L1, done, tl, per);
    else fwht_pass<T, 2>(col, L1, done, tl, per);
    __syncthreads();
    done += r;
  }
  for (int i = threadIdx.x; i < n1 * COLS; i += blockDim.x) {
    int r = i / COLS, cc = i % COLS;
    base[(int64_t)r * n2 + cc] = v[cc * pl + padi(r)];
  }
}

// FWHT across segments for 3 <= L1 <= 6 (2^L1 rows of stride 2^L2): a CTA
// of 256 threads takes 32 adjacent columns, so every row is read and written
// as one 128-byte run (FP32).  Thread (g = tid / 32, c = tid % 32) first holds
// rows g + 8 i of column c and applies the stages of row bits 3 .. L1-1 in
// registers; one padded shared-memory exchange gives it rows 8 g + i, and the
// stages of bits 0-2 follow in registers.  Natural order throughout.  (The
// FP32 1D products use k_fwht_cols128 below, which also samples.)
template <typename T, int L1>
__global__ void __launch_bounds__(256) k_fwht_cols32(T* __restrict__ x, int L2) {
  constexpr int n1 = 1 << L1, NR = n1 / 8;
  __shared__ T S[n1][33];
  pdl_trigger();
  pdl_wait();
  const int tid = threadIdx.x, c = tid & 31, g = tid >> 5;
  const int64_t n2 = (int64_t)1 << L2;
  const int tiles = (int)(n2 / 32);
  const int64_t b = blockIdx.x / tiles;
  const int64_t col = (int64_t)(blockIdx.x % tiles) * 32 + c;
  T* base = x + b * ((int64_t)n1 << L2) + col;
  T v[8];
  if (g < 8) {
#pragma unroll
    for (int i = 0; i < NR; ++i) v[i] = base[(int64_t)(g + 8 * i) * n2];
#pragma unroll
    for (int h = 1; h < NR; h <<= 1)
#pragma unroll
      for (int i = 0; i < NR; ++i)
        if (!(i & h)) {
          const T a = v[i], d = v[i + h];
          v[i] = a + d;
          v[i + h] = a - d;
        }
#pragma unroll
    for (int i = 0; i < NR; ++i) S[g + 8 * i][c] = v[i];
  }
  __syncthreads();
  if (g < NR) {
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = S[8 * g + i][c];
#pragma unroll
    for (int h = 1; h < 8; h <<= 1)
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (!(i & h)) {
          const T a = v[i], d = v[i + h];
          v[i] = a + d;
          v[i + h] = a - d;
        }
#pragma unroll
    for (int i = 0; i < 8; ++i) base[(int64_t)(8 * g + i) * n2] = v[i];
  }
}



// FP32 butterfly of 4 adjacent columns: (a, d) <- (a + d, a - d), as two
// packed FP32x2 operations each (a - d = fma(d, -1, a), exact like the plain
// difference)
__device__ __forceinline__ void bfly_x4(float4& a, float4& d) {
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 a0 = make_float2(a.x, a.y), a1 = make_float2(a.z, a.w);
  const float2 d0 = make_float2(d.x, d.y), d1 = make_float2(d.z, d.w);
  const float2 s0 = __fadd2_rn(a0, d0), s1 = __fadd2_rn(a1, d1);
  const float2 t0 = __ffma2_rn(d0, m1, a0), t1 = __ffma2_rn(d1, m1, a1);
  a = make_float4(s0.x, s0.y, s1.x, s1.y);
  d = make_float4(t0.x, t0.y, t1.x, t1.y);
}

// k_fwht_cols32 for FP32 with 4 adjacent columns per thread (128 per CTA):
// the line is read and written as 16-byte vectors, the sample table 4
// entries at a time, and the butterflies run as packed FP32x2 operations;
// the same stages in the same order, so the results are those of
// k_fwht_cols32 bit for bit.  The kernel is bound by instruction issue, and
// this cuts its loads, stores and address arithmetic by 4 and its adds by 2.
template <int L1, int MODE>
__global__ void __launch_bounds__(256) k_fwht_cols128(float* __restrict__ x, int L2, const int32_t* __restrict__ n2y,
                                                      const float* __restrict__ yin, float* __restrict__ yout,
                                                      int64_t m) {
  constexpr int n1 = 1 << L1, NR = n1 / 8;
  __shared__ __align__(16) float4 S[n1][32];
  pdl_trigger();
  pdl_wait();
  const int tid = threadIdx.x, c4 = tid & 31, g = tid >> 5;
  const int64_t n2 = (int64_t)1 << L2;
  const int tiles = (int)(n2 / 128);
  const int64_t b = blockIdx.x / tiles;
  const int64_t col = (int64_t)(blockIdx.x % tiles) * 128 + 4 * c4;
  float* base = x + b * ((int64_t)n1 << L2) + col;
  const int32_t* tb = n2y + col;
  const float* yb = yin + b * m;
  float4 v[8];
#pragma unroll
  for (int i = 0; i < NR; ++i) {
    const int64_t r = g + 8 * i;
    if constexpr (MODE == 2) {
      const int4 t = __ldg(reinterpret_cast<const int4*>(tb + r * n2));
      v[i] = make_float4(t.x >= 0 ? __ldg(yb + t.x) : 0.f, t.y >= 0 ? __ldg(yb + t.y) : 0.f,
                         t.z >= 0 ? __ldg(yb + t.z) : 0.f, t.w >= 0 ? __ldg(yb + t.w) : 0.f);
    } else {
      v[i] = *reinterpret_cast<const float4*>(base + r * n2);
    }
  }
#pragma unroll
  for (int h = 1; h < NR; h <<= 1)
#pragma unroll
    for (int i = 0; i < NR; ++i)
      if (!(i & h)) bfly_x4(v[i], v[i + h]);
#pragma unroll
  for (int i = 0; i < NR; ++i) S[g + 8 * i][c4] = v[i];
  __syncthreads();
  if (g < NR) {
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = S[8 * g + i][c4];
#pragma unroll
    for (int h = 1; h < 8; h <<= 1)
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (!(i & h)) bfly_x4(v[i], v[i + h]);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t r = 8 * g + i;
      if constexpr (MODE == 1) {
        const int4 t = __ldg(reinterpret_cast<const int4*>(tb + r * n2));
        float* yo = yout + b * m;
        if (t.x >= 0) yo[t.x] = v[i].x;
        if (t.y >= 0) yo[t.y] = v[i].y;
        if (t.z >= 0) yo[t.z] = v[i].z;
        if (t.w >= 0) yo[t.w] = v[i].w;
      } else {
        *reinterpret_cast<float4*>(base + r * n2) = v[i];
      }
    }
  }
}

template <typename T>
__global__ void k_gather(const T* __restrict__ beta, T* __restrict__ y, const uint32_t* __restrict__ mask,
                         const int32_t* __restrict__ prefix, int64_t words, int L, int64_t N, int64_t m, int batch) {
  const int64_t total = (int64_t)batch * words;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t w = idx % words, b = idx / words;
    uint32_t bits = mask[w];
    int64_t pos = prefix[w];
    const T* be = beta + b * N;
    T* yb = y + b * m;
    while (bits) {
      int bb = __ffs(bits) - 1;
      bits &= bits - 1;
      int n = (int)(w * 32 + bb);
      yb[pos++] = be[seqrow(n, L)];
    }
  }
}

template <typename T>
__global__ void k_scatter(const T* __restrict__ y, T* __restrict__ beta, const uint32_t* __restrict__ mask,
                          const int32_t* __restrict__ prefix, int64_t words, int L, int64_t N, int64_t m, int batch) {
  const int64_t total = (int64_t)batch * words;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t w = idx % words, b = idx / words;
    uint32_t bits = mask[w];
    int64_t pos = prefix[w];
    T* be = beta + b * N;
    const T* yb = y + b * m;
    while (bits) {
      int bb = __ffs(bits) - 1;
      bits &= bits - 1;
      int n = (int)(w * 32 + bb);
      be[seqrow(n, L)] = yb[pos++];
    }
  }
}

// out[b][c][r] = in[b][r][c] for an R x C matrix, except that the
// sub-block r < br, c < bc is read from `alt` (leading dim ldalt) when
// alt != nullptr (forward: splice the coarse-level IDWT into x), or written
// to `altout` (adjoint: split the coarse block off for the DWT).
template <typename T>
__global__ void k_transpose(const T* __restrict__ in, T* __restrict__ out, int rows, int cols,
                            int64_t in_batch, int64_t out_batch, const T* __restrict__ alt, int64_t alt_batch,
                            T* __restrict__ altout, int br, int bc, int ldalt) {
  __shared__ T tile[32][33];
  pdl_trigger();
  pdl_wait();
  const int64_t b = blockIdx.z;
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    int r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) {
      T val;
      if (alt && r < br && c < bc) val = alt[b * alt_batch + (int64_t)r * ldalt + c];
      else val = in[b * in_batch + (int64_t)r * cols + c];
      tile[i][threadIdx.x] = val;
    }
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    int c = c0 + i, r = r0 + threadIdx.x;   // output row c, column r
    if (r < rows && c < cols) {
      T val = tile[threadIdx.x][i];
      if (altout && c < br && r < bc) altout[b * alt_batch + (int64_t)c * ldalt + r] = val;
      else out[b * out_batch + (int64_t)c * rows + r] = val;
    }
  }
}

// ---------------------------------------------------------------------------
// One coarse Mallat level, both directions of the separable step fused in one
// kernel: a CTA stages the input window it needs (with the halo of the
// filters, and the boundary rows of the VMP blocks) in shared memory, runs the
// row pass and the column pass there, and writes its output tile.
// ---------------------------------------------------------------------------
// window accessor: global index g -> window slot.  The window covers every
// index the per-output formulas read (the dependency ranges below), so no
// bounds check is needed; `wrap` (periodic windows that cross the end of the
// level) maps g modulo the power-of-two length with a mask.
template <typename T>
struct Win {
  const T* a;
  int start, stride, mask, wrap;
  __device__ __forceinline__ T operator[](int g) const {
    int w = g - start;
    if (wrap) w &= mask;
    return a[w * stride];
  }
};

// index range [lo, hi) of level-j coefficients that outputs [a, b) of level
// j+1 depend on (interior taps, and the VMP boundary blocks near the edges);
// periodic ranges may start below 0 and are read modulo n0
__host__ __device__ __forceinline__ void syn_dep(int a, int b, int n0, const Geo& G, int& lo, int& hi) {
  const int p = G.p, n1 = 2 * n0;
  lo = (a - p) >> 1;        // floor((a - p) / 2)
  hi = ((b - 1 + p - 1) >> 1) + 1;
  if (G.bd == UW_BOUNDARY_PERIODIC) {
    if (hi - lo > n0) { lo = 0; hi = n0; }
    return;
  }
  if (lo < 0) lo = 0;
  if (hi > n0) hi = n0;
  if (a < G.Lb) {  // left boundary block reads the p edge coefficients
    lo = 0;
    if (hi < p) hi = p;
  }
  if (b > n1 - G.Lb) {  // right boundary block
    hi = n0;
    if (lo > n0 - p) lo = n0 - p;
  }
}

// analysis: outputs m in [a, b) of level j need level-(j+1) samples [lo, hi)
__host__ __device__ __forceinline__ void ana_dep(int a, int b, int n0, const Geo& G, int& lo, int& hi) {
  const int p = G.p, n1 = 2 * n0;
  lo = 2 * a - p + 1;
  hi = 2 * (b - 1) + p + 1;
  if (G.bd == UW_BOUNDARY_PERIODIC) {
    if (hi - lo > n1) { lo = 0; hi = n1; }
    return;
  }
  if (lo < 0) lo = 0;
  if (hi > n1) hi = n1;
  if (a < p) {  // left boundary rows read the first Lb samples
    lo = 0;
    if (hi < G.Lb) hi = G.Lb;
  }
  if (b > n0 - p) {  // right boundary rows read the last Lb samples
    hi = n1;
    if (lo > n1 - G.Lb) lo = n1 - G.Lb;
  }
}

// Copy a rows x cols window into shared memory (row-major, leading dim
// cols): warps take 8 rows at a time, lanes take columns, and all 16 loads of
// a lane are issued before its stores so their latencies overlap.  addr(r, c)
// is the global address of window element (r, c).
template <typename T, typename Addr>
__device__ __forceinline__ void gather_window(T* dst, int rows, int cols, const Addr& addr) {
  constexpr int RB = 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r0 = warp * RB; r0 < rows; r0 += nw * RB)
    for (int c0 = 0; c0 < cols; c0 += 64) {
      T v[RB][2];
#pragma unroll
      for (int a = 0; a < RB; ++a)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r = r0 + a, c = c0 + lane + 32 * h;
          v[a][h] = (r < rows && c < cols) ? *addr(r, c) : T(0);
        }
#pragma unroll
      for (int a = 0; a < RB; ++a)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r = r0 + a, c = c0 + lane + 32 * h;
          if (r < rows && c < cols) dst[r * cols + c] = v[a][h];
        }
    }
}

// Interior formulas with the filter length P known at compile time (P = 0:
// the runtime p, loops not unrolled).  Synthesis: s[k] = sum over the p
// indices m with k - 2m in [-p+1, p] of h_{k-2m} lo[m] + g_{k-2m} hi[m];
// analysis: lo[m] = sum_l h_l s[2m+l], hi[m] = sum_l g_l s[2m+l]
// (Sec. 3.2, two-scale relations of the interior functions).
template <typename T, int P, typename AL, typename AH>
__device__ __forceinline__ T syn_interior(int k, int p_rt, const AL& lo, const AH& hi, const T* h, const T* g) {
  const int p = P ? P : p_rt;
  const int m0 = (k - p + 1) >> 1;
  const int l0 = k - 2 * m0 + p - 1;  // filter index of m0
  T acc = 0;
#pragma unroll
  for (int t = 0; t < (P ? P : 1); ++t) {
    if (!P) break;
    acc += h[l0 - 2 * t] * lo[m0 + t] + g[l0 - 2 * t] * hi[m0 + t];
  }
  if (!P)
    for (int t = 0; t < p; ++t) acc += h[l0 - 2 * t] * lo[m0 + t] + g[l0 - 2 * t] * hi[m0 + t];
  return acc;
}

template <typename T, int P, typename AS>
__device__ __forceinline__ void ana_interior(int m, int p_rt, const AS& s, const T* h, const T* g, T& lo, T& hi) {
  const int p = P ? P : p_rt;
  const int k0 = 2 * m - p + 1;
  T a = 0, b = 0;
#pragma unroll
  for (int l = 0; l < (P ? 2 * P : 1); ++l) {
    if (!P) break;
    const T v = s[k0 + l];
    a += h[l] * v;
    b += g[l] * v;
  }
  if (!P)
    for (int l = 0; l < 2 * p; ++l) {
      const T v = s[k0 + l];
      a += h[l] * v;
      b += g[l] * v;
    }
  lo = a;
  hi = b;
}

// The coarse kernels stage only the filters h and g (4p values) in shared
// memory; the boundary blocks PL, QL, PR, QR are read through L1 by the tiles
// that touch a VMP boundary.  Returns the number of staged values.
template <typename T>
__device__ __forceinline__ int stage_filters(const Tables<T>& t, const Geo& G, T* base, SmemTables<T>& s, int tid,
                                             int nthr) {
  const int n = 4 * G.p;
  for (int i = tid; i < n; i += nthr) base[i] = t.h[i];   // h and g are contiguous in the packed tables
  s.h = base;
  s.g = base + 2 * G.p;
  s.taps = nullptr;
  s.EL = s.ER = nullptr;
  s.PL = const_cast<T*>(t.PL);
  s.QL = const_cast<T*>(t.QL);
  s.PR = const_cast<T*>(t.PR);
  s.QR = const_cast<T*>(t.QR);
  return (n + 3) & ~3;
}

// tile edges: synthesis tiles of level-(j+1) samples, analysis tiles of
// level-j coefficients per quadrant; small levels take small tiles so every
// level launches at least 64 CTAs per instance (and the analysis column pass
// maps a window of at most 64 columns to lanes)
__host__ __device__ inline int syn_tile(int n1) { return n1 >= 512 ? 32 : (n1 >= 256 ? 16 : (n1 >= 8 ? 8 : n1)); }
__host__ __device__ inline int ana_tile(int n0) { return n0 >= 128 ? 16 : (n0 >= 8 ? 8 : n0); }

// synthesis level j -> j+1 on the n1 x n1 block [[LL, D1], [D2, D3]]:
// LL from llsrc (leading dim ldll), details from x; output S_{j+1} to dst.
// One TS x TS output tile `tile` of instance b; W is the CTA's shared window.
template <typename T, int P>
__device__ __forceinline__ void syn2d_tile(int tile, int64_t b, const T* llsrc, int64_t ldll,
                                           int64_t llb, const T* __restrict__ x, int M, T* __restrict__ dst,
                                           int64_t lddst, int64_t dstb, int j, int TS, const SmemTables<T>& st, T* W,
                                           const Geo& G, int tid, int nthr) {
  const int n0 = 1 << j, n1 = 2 * n0;
  const int tiles = n1 / TS;
  const int r0 = (tile / tiles) * TS, c0 = (tile % tiles) * TS;
  const bool per = G.bd == UW_BOUNDARY_PERIODIC;
  int dr0, dr1, dc0, dc1;
  syn_dep(r0, r0 + TS, n0, G, dr0, dr1);
  syn_dep(c0, c0 + TS, n0, G, dc0, dc1);
  const int nr = dr1 - dr0, nc = dc1 - dc0;
  const int wrapr = per, wrapc = per;  // periodic reads go through the power-of-two mask
  // window of the four subbands: W[q][i][m], q = 0 LL, 1 D1, 2 D2, 3 D3
  T* H = W + 4 * nr * nc;  // row-synthesised: H[half][i][c], half 0 = top rows, 1 = bottom rows
  const T* xb = x + b * (int64_t)M * M;
  const T* lb = llsrc + b * llb;
  {
    const int msk = per ? n0 - 1 : -1;
    auto addr = [&](int r, int m) -> const T* {  // window row r = q * nr + i
      const int q = r >= 2 * nr ? (r >= 3 * nr ? 3 : 2) : (r >= nr ? 1 : 0);
      const int gi = (dr0 + r - q * nr) & msk, gm = (dc0 + m) & msk;
      if (q == 0) return lb + (int64_t)gi * ldll + gm;
      return xb + (int64_t)((q >= 2 ? n0 : 0) + gi) * M + (q & 1 ? n0 : 0) + gm;
    };
    gather_window<T>(W, 4 * nr, nc, addr);
  }
  __syncthreads();
  // rows: for each window row i (top: LL|D1, bottom: D2|D3), outputs c in tile
  const int lg = __ffs(TS) - 1;
  for (int e = tid; e < 2 * nr * TS; e += nthr) {
    const int half = e >= nr * TS ? 1 : 0, rem = e - half * nr * TS, i = rem >> lg, cc = rem & (TS - 1);
    const T* lo = W + (half == 0 ? 0 : 2) * nr * nc + i * nc;
    const T* hi = W + (half == 0 ? 1 : 3) * nr * nc + i * nc;
    Win<T> wl{lo, dc0, 1, n0 - 1, wrapc}, wh{hi, dc0, 1, n0 - 1, wrapc};
    const int kk = c0 + cc;
    H[e] = (per || (kk >= G.Lb && kk < n1 - G.Lb)) ? syn_interior<T, P>(kk, G.p, wl, wh, st.h, st.g)
                                                   : syn_one<T>(kk, n0, wl, wh, st, G);
  }
  __syncthreads();
  // columns: outputs r in tile from the top (lo) and bottom (hi) H rows
  for (int e = tid; e < TS * TS; e += nthr) {
    const int rr = e >> lg, cc = e & (TS - 1);
    Win<T> wl{H + cc, dr0, TS, n0 - 1, wrapr}, wh{H + nr * TS + cc, dr0, TS, n0 - 1, wrapr};
    const int kr = r0 + rr;
    dst[b * dstb + (int64_t)kr * lddst + c0 + cc] = (per || (kr >= G.Lb && kr < n1 - G.Lb))
                                                        ? syn_interior<T, P>(kr, G.p, wl, wh, st.h, st.g)
                                                        : syn_one<T>(kr, n0, wl, wh, st, G);
  }
}

template <typename T, int P>
__global__ void __launch_bounds__(256) k_syn2d_level(const T* __restrict__ llsrc, int64_t ldll, int64_t llb,
                                                     const T* __restrict__ x, int M, T* __restrict__ dst, int64_t lddst,
                                                     int64_t dstb, int j, int TS, Tables<T> tab, Geo G) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  SmemTables<T> st;
  const int off = stage_filters(tab, G, sm, st, tid, nthr);
  pdl_trigger();
  pdl_wait();
  syn2d_tile<T, P>(blockIdx.x, blockIdx.y, llsrc, ldll, llb, x, M, dst, lddst, dstb, j, TS, st, sm + off, G, tid, nthr);
}

// analysis level j+1 -> j of the n1 x n1 block src (leading dim ldsrc): the
// low-pass block to lldst (or to x when lldst is null), details to x.  One
// tile of TS x TS coefficients per quadrant; S is the CTA's shared window.
template <typename T, int P>
__device__ __forceinline__ void ana2d_tile(int tile, int64_t b, const T* src, int64_t ldsrc,
                                           int64_t srcb, T* x, int M, T* lldst,
                                           int64_t ldll, int64_t llb, int j, int TS, const SmemTables<T>& st, T* S,
                                           const Geo& G, int tid, int nthr) {
  const int n0 = 1 << j, n1 = 2 * n0;
  const int tiles = n0 / TS;  // TS: output coefficients per dimension and quadrant
  const int m0 = (tile / tiles) * TS, k0 = (tile % tiles) * TS;
  const bool per = G.bd == UW_BOUNDARY_PERIODIC;
  int sr0, sr1, sc0, sc1;
  ana_dep(m0, m0 + TS, n0, G, sr0, sr1);
  ana_dep(k0, k0 + TS, n0, G, sc0, sc1);
  const int nr = sr1 - sr0, nc = sc1 - sc0;
  const int wrapr = per, wrapc = per;
  T* H = S + nr * nc;         // H[half][m][c]: column analysis, half 0 = low, 1 = high
  const T* sb = src + b * srcb;
  {
    const int msk = per ? n1 - 1 : -1;
    auto addr = [&](int i, int c) -> const T* {
      return sb + (int64_t)((sr0 + i) & msk) * ldsrc + ((sc0 + c) & msk);
    };
    gather_window<T>(S, nr, nc, addr);
  }
  __syncthreads();
  // columns: for each window column c (< 64 by the tile size), low/high
  // outputs m in [m0, m0 + TS)
  for (int e = tid; e < TS * 64; e += nthr) {
    const int mm = e >> 6, c = e & 63;
    if (c >= nc) continue;
    Win<T> s{S + c, sr0, nc, n1 - 1, wrapr};
    T lo, hi;
    const int m = m0 + mm;
    if (per || (m >= G.p && m < n0 - G.p)) ana_interior<T, P>(m, G.p, s, st.h, st.g, lo, hi);
    else ana_one<T>(m, n0, s, st, G, lo, hi);
    H[mm * nc + c] = lo;
    H[(TS + mm) * nc + c] = hi;
  }
  __syncthreads();
  // rows: each H row -> low/high outputs k in [k0, k0 + TS)
  T* xb = x + b * (int64_t)M * M;
  const int lg = __ffs(TS) - 1;
  for (int e = tid; e < 2 * TS * TS; e += nthr) {
    const int row = e >> lg, kk = e & (TS - 1);  // row < TS: low rows, else high rows
    Win<T> s{H + row * nc, sc0, 1, n1 - 1, wrapc};
    T lo, hi;
    const int m = k0 + kk;
    if (per || (m >= G.p && m < n0 - G.p)) ana_interior<T, P>(m, G.p, s, st.h, st.g, lo, hi);
    else ana_one<T>(m, n0, s, st, G, lo, hi);
    const int mm = row < TS ? m0 + row : m0 + row - TS;
    if (row < TS) {
      if (lldst) lldst[b * llb + (int64_t)mm * ldll + k0 + kk] = lo;
      else xb[(int64_t)mm * M + k0 + kk] = lo;
      xb[(int64_t)mm * M + n0 + k0 + kk] = hi;
    } else {
      xb[(int64_t)(n0 + mm) * M + k0 + kk] = lo;
      xb[(int64_t)(n0 + mm) * M + n0 + k0 + kk] = hi;
    }
  }
}

template <typename T, int P>
__global__ void __launch_bounds__(256) k_ana2d_level(const T* __restrict__ src, int64_t ldsrc, int64_t srcb,
                                                     T* __restrict__ x, int M, T* __restrict__ lldst, int64_t ldll,
                                                     int64_t llb, int j, int TS, Tables<T> tab, Geo G) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  SmemTables<T> st;
  const int off = stage_filters(tab, G, sm, st, tid, nthr);
  pdl_trigger();
  pdl_wait();
  ana2d_tile<T, P>(blockIdx.x, blockIdx.y, src, ldsrc, srcb, x, M, lldst, ldll, llb, j, TS, st, sm + off, G, tid, nthr);
}

// ---------------------------------------------------------------------------
// All coarse 2D levels in one cooperative launch: the CTAs of the grid (all
// resident at once) take the tiles of a level in turn and meet at a grid
// barrier before the next level, whose tiles read what every CTA wrote.
// The barrier spins a bounded number of times; a CTA that gives up records
// the failure in the barrier's error word and returns (uw_plan_device_status
// reports it as UW_ERR_TIMEOUT).
// ---------------------------------------------------------------------------
struct GridBarrier {
  unsigned int count;   // arrivals since the launch began (barrier k completes at (k + 1) x CTAs)
  unsigned int exits;   // CTAs that have finished the launch
  unsigned int err;     // set when a wait gave up
  unsigned int pad;
};

// relaxed polling load (no L1 invalidation per poll, which would evict the
// data of the CTAs still working on the same SM); one acquire load after the
// wait orders (and refreshes) what the CTA reads next
__device__ __forceinline__ unsigned int ld_relaxed_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_add_release_u32(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned int atom_add_acq_rel_u32(unsigned int* p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;\n" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Grid barrier number k of a launch: each CTA's thread 0 adds one arrival
// with a release (after the CTA barrier, so it releases the whole CTA's
// writes) and polls the count with relaxed loads until all (k + 1) x
// nblocks arrivals are in, then reads it once with acquire semantics.  The
// count only grows during a launch; grid_exit resets it.  Returns false (in
// every thread of the CTA) if the wait gave up.
__device__ __forceinline__ bool grid_barrier(GridBarrier* bar, unsigned int nblocks, int k, unsigned int limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int target = (unsigned int)(k + 1) * nblocks;
    red_add_release_u32(&bar->count, 1u);
    unsigned int it = 0;
    while (ld_relaxed_u32(&bar->count) < target) {
      if (++it > limit) {
        atomicExch(&bar->err, 1u);
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    (void)ld_acquire_u32(&bar->count);
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Every CTA calls this once at the end of the launch (also after a wait gave
// up); the last one resets the arrival count for the next launch on the stream.
__device__ __forceinline__ void grid_exit(GridBarrier* bar, unsigned int nblocks) {
  __syncthreads();
  if (threadIdx.x == 0) {
    if (atom_add_acq_rel_u32(&bar->exits, 1u) + 1u == nblocks) {
      atomicExch(&bar->count, 0u);
      atomicExch(&bar->exits, 0u);
    }
  }
}

// level buffers of the forward synthesis: level it (j = J0 + it) reads
// S_j (x itself for it = 0) and writes S_{j+1}; S_{R-1} ends in XS
constexpr int kMaxCoarse = 16;   // coarse levels of one fused launch (R - 1 - J0 <= 15)
template <typename T>
struct CoarseIO {
  const T* x;    // forward input (Mallat layout)
  T* xout;       // adjoint output (Mallat layout)
  T* XS;
  T* XS2;
  T* XT;         // transposed full-size buffer of the line passes, or null (see tx_share)
  int M, J0, nl, batch;
  // transpose items [tq0[it], tq0[it] + tnq[it]) ride with step it (host-computed, tx_share)
  int tq0[kMaxCoarse], tnq[kMaxCoarse];
};

// ---------------------------------------------------------------------------
// Register-window tiles of one coarse 2D level.  Both passes of a level use
// the interior formulas (two-scale relations of Sec. 3.2) on windows padded
// with zeros (VMP) or wrapped (periodic) at the ends; near a VMP boundary the
// exact level differs from that by a level-independent correction D that
// reads only the p lo and p hi coefficients at that end and reaches only the
// first / last Lb outputs (host-built: build_coarse).  The analysis applies
// the transposes.  Each thread computes several consecutive outputs from a
// register window.
// ---------------------------------------------------------------------------
template <typename T, int PM>
struct CTaps {
  T hp[2][PM + 1];   // synthesis, polyphase: hp[f][d + PM/2] = h_{2d+f}
  T gp[2][PM + 1];
  T ha[2 * PM];      // analysis: ha[l + PM - 1] = h_l, l in [-PM+1, PM]
  T ga[2 * PM];
};

__host__ __device__ constexpr int cup(int a, int b) { return (a + b - 1) / b * b; }
__host__ __device__ constexpr int ilog2c(int a) { return a <= 1 ? 0 : 1 + ilog2c(a / 2); }

// NW values from a 16-byte aligned shared address, 16-byte loads
template <typename T, int NW>
__device__ __forceinline__ void ld16(T (&w)[NW], const T* src) {
  if constexpr (sizeof(T) == 4) {
    static_assert(NW % 4 == 0, "float windows are loaded in fours");
#pragma unroll
    for (int i = 0; i < NW; i += 4) {
      const float4 u = *reinterpret_cast<const float4*>(src + i);
      w[i] = u.x; w[i + 1] = u.y; w[i + 2] = u.z; w[i + 3] = u.w;
    }
  } else {
    static_assert(NW % 2 == 0, "double windows are loaded in pairs");
#pragma unroll
    for (int i = 0; i < NW; i += 2) {
      const double2 u = *reinterpret_cast<const double2*>(src + i);
      w[i] = u.x; w[i + 1] = u.y;
    }
  }
}

// VMP edge corrections of the register-window tiles, staged in shared memory
// with zero padding to compile-time bounds (LBM = 3 PM - 1 >= Lb rows):
//   synthesis: D[LBM + 1][2 PM], row LBM zero (rows outside [0, LBM) read it);
//   analysis:  D^T[2 PM + 1][LBP], row 2 PM zero (columns outside [0, PM) read it).
// Rows are 16-byte aligned and loaded as vectors; the dot products of one
// thread's outputs are independent (no branch per output).  The lanes of a
// warp read rows 8 apart (synthesis rows) or 4 apart (analysis columns): one
// 16-byte unit of padding per 8 (4) rows puts those rows in different banks.
template <typename T, int PM>
struct EdgeT {
  static constexpr int VU = 16 / (int)sizeof(T);
  static constexpr int LBM = 3 * PM - 1;
  static constexpr int LBP = cup(LBM, VU);
  __host__ __device__ static constexpr int srow(int r) { return r * 2 * PM + VU * (r >> 3); }
  __host__ __device__ static constexpr int acol(int c) { return c * LBP + VU * (c >> 2); }
  static constexpr int syn_side = cup(srow(LBM) + 2 * PM, VU);
  static constexpr int ana_side = cup(acol(2 * PM) + LBP, VU);
  static constexpr int syn_words = 2 * syn_side;     // both sides
  static constexpr int ana_words = 2 * ana_side;
};

// output r of the synthesis edge band: D row r (zero outside [0, LBM)) . xe
template <typename T, int PM>
__device__ __forceinline__ T edge_dot(const T* D, int r, const T (&xe)[2 * PM]) {
  constexpr int LBM = 3 * PM - 1;
  T d[2 * PM];
  ld16(d, D + EdgeT<T, PM>::srow((unsigned)r < (unsigned)LBM ? r : LBM));
  T a0 = T(0), a1 = T(0);
#pragma unroll
  for (int c = 0; c < PM; ++c) {
    a0 = fma(d[c], xe[c], a0);
    a1 = fma(d[PM + c], xe[PM + c], a1);
  }
  return a0 + a1;
}

// column col of the analysis edge band: lo += D^T[col] . xe, hi += D^T[PM + col] . xe
template <typename T, int PM>
__device__ __forceinline__ void edge_dot_t(const T* DT, int col, const T (&xe)[EdgeT<T, PM>::LBP], T& lo, T& hi) {
  constexpr int LBP = EdgeT<T, PM>::LBP;
  const bool ok = (unsigned)col < (unsigned)PM;
  T dl[LBP], dh[LBP];
  ld16(dl, DT + EdgeT<T, PM>::acol(ok ? col : 2 * PM));
  ld16(dh, DT + EdgeT<T, PM>::acol(ok ? PM + col : 2 * PM));
  T x0 = T(0), x1 = T(0);
#pragma unroll
  for (int k = 0; k < LBP; ++k) {
    x0 = fma(dl[k], xe[k], x0);
    x1 = fma(dh[k], xe[k], x1);
  }
  lo += x0;
  hi += x1;
}

// synthesis tile geometry: TS x TS outputs of level j+1 from NR x NC windows
// of the four subbands (NR = NC = TS/2 + PM)
template <typename T, int PM, int TS>
struct SynGeom {
  static constexpr int VW = 16 / (int)sizeof(T);
  static constexpr int NR = TS / 2 + PM;
  static constexpr int NC = TS / 2 + PM;
  static constexpr int NCP = 48;                      // row stride (rows 16 banks apart)
  static constexpr int NWR = cup(4 + PM, VW);         // row-pass window
  static constexpr int TSP = TS + VW;                 // H row stride: an odd number of 16-byte units
  static constexpr int elems = 4 * NR * NCP + 2 * NR * TSP;
  static_assert((TSP / VW) % 2 == 1, "H rows must start in alternating bank groups");
  static_assert(4 * (TS / 8 - 1) + NWR <= NCP, "row window exceeds the padded row");
};

// analysis tile geometry: TSA x TSA coefficients per quadrant from an
// NR x NR window of level j+1 (NR = 2 TSA + 2 PM - 2)
template <typename T, int PM, int TSA>
struct AnaGeom {
  static constexpr int VW = 16 / (int)sizeof(T);
  static constexpr int NR = 2 * TSA + 2 * PM - 2;
  static constexpr int NRP = NR + 1;                  // row stride of the input window
  static constexpr int NWA = cup(2 * PM + 6, VW);     // row-pass window (2 PM + 6 used)
  static constexpr int NCH0 = cup(8 * (TSA / 4 - 1) + NWA, VW);
  // row stride of the column-pass result: an odd number of 16-byte units
  static constexpr int NCH = (NCH0 / VW) % 2 ? NCH0 : NCH0 + VW;
  static constexpr int HOFF = cup(NR * NRP, 4);       // the column-pass result starts 16-byte aligned
  static constexpr int elems = HOFF + 2 * TSA * NCH;
};

template <typename T, int PM, int TS>
__device__ __forceinline__ void syn_tile_rw(int tile, int64_t b, const T* llsrc, int64_t ldll,
                                            int64_t llb, const T* __restrict__ x, int M, T* __restrict__ dst,
                                            int64_t lddst, int64_t dstb, int j, const CTaps<T, PM>& ct, const T* Dl,
                                            const T* Dr, int p, int Lb, bool per, T* smem, int tid, int nthr,
                                            T* xt = nullptr) {
  using SG = SynGeom<T, PM, TS>;
  constexpr int NR = SG::NR, NC = SG::NC, NCP = SG::NCP, NWR = SG::NWR, TSP = SG::TSP;
  const int n0 = 1 << j, n1 = 2 * n0;
  const int lt = j + 1 - ilog2c(TS);          // tiles per row: n1 / TS = 2^lt
  const int r0 = (tile >> lt) * TS, c0 = (tile & ((1 << lt) - 1)) * TS;
  const int ir0 = (r0 >> 1) - PM / 2, ic0 = (c0 >> 1) - PM / 2;
  T* W = smem;                    // [4][NR][NCP]: LL, D1, D2, D3 windows
  T* H = W + 4 * NR * NCP;        // [2][NR][TSP]: row-synthesised top (LL|D1) and bottom (D2|D3) halves
  const T* xb = x + b * (int64_t)M * M;
  const T* lb = llsrc + b * llb;
  {
    // every load of the window is issued before the first store (one round
    // of memory latency); the kernels run 256 threads.  A thread takes the
    // same (row, column) of the four subbands.
    constexpr int TOT = NR * NC, CNT = (TOT + 255) / 256;
    // 32-bit offsets from per-subband bases (2D lines have M <= 2^13)
    const T* base[4] = {lb, xb + n0, xb + (int64_t)n0 * M, xb + (int64_t)n0 * M + n0};
    const int ld[4] = {(int)ldll, M, M, M};
    T v[CNT][4];
#pragma unroll
    for (int u = 0; u < CNT; ++u) {
      const int e = tid + u * 256;
      const int i = e / NC, m = e - i * NC;
      int gi = ir0 + i, gm = ic0 + m;
      bool ok = e < TOT;
      if (per) {
        gi &= n0 - 1;
        gm &= n0 - 1;
      } else {
        ok = ok && gi >= 0 && gi < n0 && gm >= 0 && gm < n0;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) v[u][q] = ok ? base[q][gi * ld[q] + gm] : T(0);
    }
#pragma unroll
    for (int u = 0; u < CNT; ++u) {
      const int e = tid + u * 256;
      if (e < TOT) {
        const int i = e / NC, m = e - i * NC;
#pragma unroll
        for (int q = 0; q < 4; ++q) W[(q * NR + i) * NCP + m] = v[u][q];
      }
    }
  }
  __syncthreads();
  // rows: H[h][i][8 g + e] from the lo (LL / D2) and hi (D1 / D3) windows
  {
    constexpr int GR = TS / 8;
    for (int t = tid; t < 2 * NR * GR; t += nthr) {
      const int h = t / (NR * GR), rem = t - h * (NR * GR), i = rem / GR, g = rem - i * GR;
      const T* rlo = W + ((2 * h) * NR + i) * NCP;
      const T* rhi = W + ((2 * h + 1) * NR + i) * NCP;
      T wl[NWR], wh[NWR];
      ld16(wl, rlo + 4 * g);
      ld16(wh, rhi + 4 * g);
      T o[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int f = e & 1, a2 = e >> 1;
        T acc = T(0);
#pragma unroll
        for (int d = -PM / 2; d <= PM / 2; ++d) {
          acc = fma(ct.hp[f][d + PM / 2], wl[a2 - d + PM / 2], acc);
          acc = fma(ct.gp[f][d + PM / 2], wh[a2 - d + PM / 2], acc);
        }
        o[e] = acc;
      }
      if (!per) {
        // edge corrections: the p lo and p hi inputs at the end into
        // registers, then unrolled dot products (loads issued up front)
        const bool left = c0 == 0 && 8 * g < Lb, right = c0 + TS == n1 && c0 + 8 * g + 8 > n1 - Lb;
        if (left || right) {
          const int m0e = left ? PM / 2 : n0 - p - ic0;
          const T* D = left ? Dl : Dr;
          T xe[2 * PM];
#pragma unroll
          for (int e = 0; e < PM; ++e) {
            xe[e] = rlo[m0e + e];
            xe[PM + e] = rhi[m0e + e];
          }
          const int rb = left ? 8 * g : c0 + 8 * g - (n1 - Lb);
#pragma unroll
          for (int e = 0; e < 8; ++e) o[e] += edge_dot<T, PM>(D, rb + e, xe);
        }
      }
      T* hrow = H + (h * NR + i) * TSP + 8 * g;    // 16-byte aligned
      if constexpr (sizeof(T) == 4) {
        reinterpret_cast<float4*>(hrow)[0] = make_float4(o[0], o[1], o[2], o[3]);
        reinterpret_cast<float4*>(hrow)[1] = make_float4(o[4], o[5], o[6], o[7]);
      } else {
#pragma unroll
        for (int e = 0; e < 8; e += 2) reinterpret_cast<double2*>(hrow)[e / 2] = make_double2(o[e], o[e + 1]);
      }
    }
  }
  __syncthreads();
  // columns: output rows 4 g4 + e of column cc from the top (lo) and bottom (hi) halves of H
  {
    constexpr int GC = TS / 4;
    for (int t = tid; t < TS * GC; t += nthr) {
      const int cc = t % TS, g4 = t / TS;
      T wl[2 + PM], wh[2 + PM];
#pragma unroll
      for (int w = 0; w < 2 + PM; ++w) {
        wl[w] = H[(2 * g4 + w) * TSP + cc];
        wh[w] = H[(NR + 2 * g4 + w) * TSP + cc];
      }
      T o[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int f = e & 1, b2 = e >> 1;
        T acc = T(0);
#pragma unroll
        for (int d = -PM / 2; d <= PM / 2; ++d) {
          acc = fma(ct.hp[f][d + PM / 2], wl[b2 - d + PM / 2], acc);
          acc = fma(ct.gp[f][d + PM / 2], wh[b2 - d + PM / 2], acc);
        }
        o[e] = acc;
      }
      if (!per) {
        const bool top = r0 == 0 && 4 * g4 < Lb, bottom = r0 + TS == n1 && r0 + 4 * g4 + 4 > n1 - Lb;
        if (top || bottom) {
          const int m0e = top ? PM / 2 : n0 - p - ir0;
          const T* D = top ? Dl : Dr;
          T xe[2 * PM];
#pragma unroll
          for (int e = 0; e < PM; ++e) {
            xe[e] = H[(m0e + e) * TSP + cc];
            xe[PM + e] = H[(NR + m0e + e) * TSP + cc];
          }
          const int rb = top ? 4 * g4 : r0 + 4 * g4 - (n1 - Lb);
#pragma unroll
          for (int e = 0; e < 4; ++e) o[e] += edge_dot<T, PM>(D, rb + e, xe);
        }
      }
      if (xt) {
        // transposed output: staged in the (no longer read) subband windows
#pragma unroll
        for (int e = 0; e < 4; ++e) W[cc * (TS + 1) + 4 * g4 + e] = o[e];
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) dst[b * dstb + (int64_t)r0 * lddst + c0 + ((4 * g4 + e) * (int)lddst + cc)] = o[e];
      }
    }
  }
  if (xt) {
    // row c0 + rr of the M x M transposed buffer, columns r0 .. r0 + TS - 1
    __syncthreads();
    T* xtt = xt + b * (int64_t)M * M + (int64_t)c0 * M + r0;
    for (int e = tid; e < TS * TS; e += nthr) {
      const int rr = e / TS, cl = e - rr * TS;
      xtt[rr * M + cl] = W[rr * (TS + 1) + cl];
    }
  }
}

template <typename T, int PM, int TSA>
__device__ __forceinline__ void ana_tile_rw(int tile, int64_t b, const T* src, int64_t ldsrc,
                                            int64_t srcb, T* x, int M, T* lldst,
                                            int64_t ldll, int64_t llb, int j, const CTaps<T, PM>& ct, const T* Dl,
                                            const T* Dr, int p, int Lb, bool per, T* smem, int tid, int nthr,
                                            const T* xt = nullptr) {
  using AG = AnaGeom<T, PM, TSA>;
  constexpr int NR = AG::NR, NRP = AG::NRP, NWA = AG::NWA, NCH = AG::NCH;
  const int n0 = 1 << j, n1 = 2 * n0;
  const int lt = j - ilog2c(TSA);             // tiles per row: n0 / TSA = 2^lt
  const int m0 = (tile >> lt) * TSA, k0 = (tile & ((1 << lt) - 1)) * TSA;
  const int ir0 = 2 * m0 - PM + 1, ic0 = 2 * k0 - PM + 1;
  T* S = smem;                    // [NR][NRP] window of level j+1
  T* Hc = S + AG::HOFF;           // [2][TSA][NCH]: column analysis, lo then hi
  const T* sb = src + b * srcb;
  {
    // xt: the level is read transposed from the M x M buffer (window rows
    // run fastest over the threads, so the loads stay coalesced)
    constexpr int TOT = NR * NR, CNT = (TOT + 255) / 256;
    const T* xtb = xt ? xt + b * (int64_t)M * M : nullptr;
    T v[CNT];
#pragma unroll
    for (int u = 0; u < CNT; ++u) {
      const int e = tid + u * 256;
      v[u] = T(0);
      if (e < TOT) {
        const int i = xt ? e % NR : e / NR, c = xt ? e / NR : e % NR;
        int gi = ir0 + i, gc = ic0 + c;
        bool ok = true;
        if (per) {
          gi &= n1 - 1;
          gc &= n1 - 1;
        } else {
          ok = gi >= 0 && gi < n1 && gc >= 0 && gc < n1;
        }
        if (ok) v[u] = xt ? xtb[gc * M + gi] : sb[gi * (int)ldsrc + gc];
      }
    }
#pragma unroll
    for (int u = 0; u < CNT; ++u) {
      const int e = tid + u * 256;
      if (e < TOT) {
        const int i = xt ? e % NR : e / NR, c = xt ? e / NR : e % NR;
        S[i * NRP + c] = v[u];
      }
    }
  }
  __syncthreads();
  // columns: lo / hi rows 4 g + e of window column c
  {
    constexpr int GC = TSA / 4;
    for (int t = tid; t < NR * GC; t += nthr) {
      const int c = t % NR, g = t / NR;
      T w[2 * PM + 6];
#pragma unroll
      for (int k = 0; k < 2 * PM + 6; ++k) w[k] = S[(8 * g + k) * NRP + c];
      T lo[4], hi[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        T x0 = T(0), x1 = T(0);
#pragma unroll
        for (int l = -PM + 1; l <= PM; ++l) {
          const T v = w[2 * e + l + PM - 1];
          x0 = fma(ct.ha[l + PM - 1], v, x0);
          x1 = fma(ct.ga[l + PM - 1], v, x1);
        }
        lo[e] = x0;
        hi[e] = x1;
      }
      if (!per) {
        // edge corrections (transposed): the Lb inputs at the end into
        // registers, then unrolled dot products
        const bool top = m0 == 0 && 4 * g < p, bottom = m0 + TSA == n0 && m0 + 4 * g + 4 > n0 - p;
        if (top || bottom) {
          constexpr int LBM = 3 * PM - 1, LBP = EdgeT<T, PM>::LBP;
          const int k0e = top ? -ir0 : n1 - Lb - ir0;
          const T* D = top ? Dl : Dr;
          T xe[LBP];
#pragma unroll
          for (int k = 0; k < LBP; ++k) xe[k] = k < LBM ? S[min(k0e + k, NR - 1) * NRP + c] : T(0);   // rows past Lb weigh zero
          const int cb = top ? 4 * g : m0 + 4 * g - (n0 - p);
#pragma unroll
          for (int e = 0; e < 4; ++e) edge_dot_t<T, PM>(D, cb + e, xe, lo[e], hi[e]);
        }
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        Hc[(4 * g + e) * NCH + c] = lo[e];
        Hc[(TSA + 4 * g + e) * NCH + c] = hi[e];
      }
    }
  }
  __syncthreads();
  // rows: lo / hi coefficients 4 g + e of each Hc row; quadrants
  // (col lo, row lo) = LL, (col lo, row hi) = D1, (col hi, row lo) = D2, (col hi, row hi) = D3
  {
    constexpr int GR = TSA / 4;
    T* xb = x + b * (int64_t)M * M;
    for (int t = tid; t < 2 * TSA * GR; t += nthr) {
      const int g = t % GR, row = t / GR;      // row < TSA: column-lo rows, else column-hi rows
      const T* hr = Hc + row * NCH;
      T w[NWA];
      ld16(w, hr + 8 * g);
      T lo[4], hi[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        T x0 = T(0), x1 = T(0);
#pragma unroll
        for (int l = -PM + 1; l <= PM; ++l) {
          const T v = w[2 * e + l + PM - 1];
          x0 = fma(ct.ha[l + PM - 1], v, x0);
          x1 = fma(ct.ga[l + PM - 1], v, x1);
        }
        lo[e] = x0;
        hi[e] = x1;
      }
      if (!per) {
        const bool left = k0 == 0 && 4 * g < p, right = k0 + TSA == n0 && k0 + 4 * g + 4 > n0 - p;
        if (left || right) {
          constexpr int LBM = 3 * PM - 1, LBP = EdgeT<T, PM>::LBP;
          const int k0e = left ? -ic0 : n1 - Lb - ic0;
          const T* D = left ? Dl : Dr;
          T xe[LBP];
#pragma unroll
          for (int k = 0; k < LBP; ++k) xe[k] = k < LBM ? hr[min(k0e + k, NR - 1)] : T(0);
          const int cb = left ? 4 * g : k0 + 4 * g - (n0 - p);
#pragma unroll
          for (int e = 0; e < 4; ++e) edge_dot_t<T, PM>(D, cb + e, xe, lo[e], hi[e]);
        }
      }
      const int mm = row < TSA ? m0 + row : m0 + row - TSA;
      const int kq = k0 + 4 * g;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (row < TSA) {
          if (lldst) lldst[b * llb + (mm * (int)ldll + kq + e)] = lo[e];
          else xb[mm * M + kq + e] = lo[e];
          xb[mm * M + n0 + kq + e] = hi[e];
        } else {
          xb[(n0 + mm) * M + kq + e] = lo[e];
          xb[(n0 + mm) * M + n0 + kq + e] = hi[e];
        }
      }
    }
  }
}

// which tile code a level takes: the register-window tiles need TS <= n1
// (synthesis) and TSA <= n0 (analysis); smaller levels take the generic tiles
__host__ __device__ inline int syn_rw_ts(int n1) { return n1 >= 32 ? 32 : (n1 >= 16 ? 16 : 0); }
__host__ __device__ inline int ana_rw_ts(int n0) { return n0 >= 16 ? 16 : (n0 >= 8 ? 8 : 0); }

// The line passes work on the transpose XT of the M x M coefficient array
// (S_{R-1} in the top-left Mh x Mh block, the level R-1 details in the other
// three quadrants).  The fused coarse-level launches make that layout change
// themselves: the forward writes its last level transposed into XT and the
// adjoint reads its first level transposed from XT, and the three detail
// quadrants move as 64 x 64 tile transposes given to the CTAs that a small
// level leaves idle.  Steps take at most one item per idle CTA, in order
// (forward: steps 0 .. nl-2, adjoint: steps 1 .. nl-1); the rest rides with
// step nl-1.  Step it runs items [q0, q0 + nq) of Q after its level tiles.
template <typename F>
static void tx_share(int it, int nl, bool fwd, int grid, int Q, F&& busy, int& q0, int& nq) {
  int used = 0;
  q0 = 0;
  nq = 0;
  for (int s = 0; s < nl - 1; ++s) {
    const int k = fwd ? s : s + 1;
    const int take = min(Q - used, max(0, grid - busy(k)));
    if (k == it) {
      q0 = used;
      nq = take;
    }
    used += take;
  }
  if (it == nl - 1) {
    if (fwd) q0 = used;   // forward: step nl-1 has no share of its own
    nq += Q - used;       // adjoint: the rest follows its own share
  }
}

// dst[(b0 + c) M + a0 + r] = src[(a0 + r) M + b0 + c], r, c < 64 (256 threads)
template <typename T>
__device__ __forceinline__ void tx_tile(const T* src, T* dst, int a0, int b0, int M, T* smem, int tid) {
  constexpr int CNT = 64 * 64 / 256;
  src += (int64_t)a0 * M + b0;
  dst += (int64_t)b0 * M + a0;
  T v[CNT];
#pragma unroll
  for (int u = 0; u < CNT; ++u) {
    const int e = tid + 256 * u, r = e >> 6, c = e & 63;
    v[u] = src[r * M + c];
  }
#pragma unroll
  for (int u = 0; u < CNT; ++u) {
    const int e = tid + 256 * u;
    smem[(e >> 6) * 65 + (e & 63)] = v[u];
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < CNT; ++u) {
    const int e = tid + 256 * u, rr = e >> 6, cl = e & 63;
    dst[rr * M + cl] = smem[cl * 65 + rr];
  }
}

// item q of the detail-quadrant transposes: instance, quadrant (0: rows
// [0, Mh) x columns [Mh, M), 1: [Mh, M) x [0, Mh), 2: [Mh, M) x [Mh, M)),
// 64 x 64 tile; forward x -> XT, adjoint XT -> x
template <typename T>
__device__ __forceinline__ void tx_item(int q, int M, const T* src, T* dst, bool fwd, T* smem, int tid) {
  const int Mh = M / 2, lnb = __ffs(Mh) - 7;   // nb = Mh / 64 = 2^lnb tiles per quadrant side
  const int bd = q >> (2 * lnb), r = q & ((1 << (2 * lnb)) - 1);
  const int b = bd / 3, d = bd - 3 * b;
  const int R0 = (d >= 1 ? Mh : 0) + (r >> lnb) * 64, C0 = (d != 1 ? Mh : 0) + (r & ((1 << lnb) - 1)) * 64;
  const int64_t off = (int64_t)b * M * M;
  if (fwd) tx_tile(src + off, dst + off, R0, C0, M, smem, tid);
  else tx_tile(src + off, dst + off, C0, R0, M, smem, tid);
}

template <typename T, int PM>
__global__ void __launch_bounds__(256, 2) k_syn2d_levels(CoarseIO<T> io, Tables<T> tab, Geo G, const __grid_constant__ CTaps<T, PM> ct,
                                                      const T* __restrict__ Dg, int rw, GridBarrier* bar,
                                                      unsigned int limit) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  SmemTables<T> st;
  int off = stage_filters(tab, G, sm, st, tid, nthr);
  const bool per = G.bd == UW_BOUNDARY_PERIODIC;
  // edge corrections [side][LBM + 1 rows][2PM cols], zero-padded (EdgeT)
  constexpr int LBM = 3 * PM - 1, DW = 2 * PM;
  const int nD = per ? 0 : 2 * (LBM + 1) * DW;      // entries (padding words are never read)
  T* Dl = sm + off;
  for (int i = tid; i < nD; i += nthr) {
    const int side = i / ((LBM + 1) * DW), rem = i - side * ((LBM + 1) * DW), r = rem / DW, c = rem - r * DW;
    const int e = c < PM ? c : c - PM;
    Dl[side * EdgeT<T, PM>::syn_side + EdgeT<T, PM>::srow(r) + c] =
        (r < G.Lb && e < G.p) ? Dg[(side * G.Lb + r) * 2 * G.p + (c < PM ? e : G.p + e)] : T(0);
  }
  const T* Dr = Dl + EdgeT<T, PM>::syn_side;
  off = cup(off + (per ? 0 : EdgeT<T, PM>::syn_words), 4);
  // constant tables staged: let the next kernel launch, then wait for the
  // previous grid (x may be its output)
  pdl_trigger();
  pdl_wait();
  const int M = io.M, Mh = M / 2;
  const int64_t HH = (int64_t)Mh * Mh, MM = (int64_t)M * M;
  const bool tx = io.XT != nullptr;
  {
    // the coarse levels read the top-left Mh x Mh block of x; bring it into
    // L2 now (one 128-byte line per prefetch, all threads of the grid)
    const int lpr = (int)((Mh * sizeof(T) + 127) / 128), total = Mh * lpr * io.batch;
    for (int i = blockIdx.x * nthr + tid; i < total; i += gridDim.x * nthr) {
      const int b = i / (Mh * lpr), r = (i / lpr) % Mh, l = i % lpr;
      const char* a = reinterpret_cast<const char*>(io.x + (int64_t)b * MM + (int64_t)r * M) + 128 * l;
      asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
    }
  }
  for (int it = 0; it < io.nl; ++it) {
    const int j = io.J0 + it, n1 = 2 << j;
    const int TR = rw ? syn_rw_ts(n1) : 0;
    const int TS = TR ? TR : syn_tile(n1), tiles = (n1 / TS) * (n1 / TS), ltiles = __ffs(tiles) - 1;
    const T* src = it == 0 ? io.x : ((io.nl - it) % 2 == 0 ? io.XS : io.XS2);
    const int64_t ld = it == 0 ? M : Mh, sb = it == 0 ? MM : HH;
    T* dst = (io.nl - 1 - it) % 2 == 0 ? io.XS : io.XS2;
    T* xt = tx && it == io.nl - 1 ? io.XT : nullptr;
    const int TB = tiles * io.batch, q0 = io.tq0[it], nq = tx ? io.tnq[it] : 0;
    for (int t = blockIdx.x; t < TB + nq; t += gridDim.x) {
      __syncthreads();   // the previous tile's windows are no longer read
      if (t >= TB)
        tx_item(q0 + t - TB, M, io.x, io.XT, true, sm + off, tid);
      else if (TR == 32)
        syn_tile_rw<T, PM, 32>(t & (tiles - 1), t >> ltiles, src, ld, sb, io.x, M, dst, (int64_t)Mh, HH, j, ct, Dl, Dr, G.p,
                               G.Lb, per, sm + off, tid, nthr, xt);
      else if (TR == 16)
        syn_tile_rw<T, PM, 16>(t & (tiles - 1), t >> ltiles, src, ld, sb, io.x, M, dst, (int64_t)Mh, HH, j, ct, Dl, Dr, G.p,
                               G.Lb, per, sm + off, tid, nthr, xt);
      else
        syn2d_tile<T, 0>(t & (tiles - 1), t >> ltiles, src, ld, sb, io.x, M, dst, (int64_t)Mh, HH, j, TS, st, sm + off, G,
                         tid, nthr);
    }
    if (it + 1 < io.nl && !grid_barrier(bar, gridDim.x, it, limit)) break;
  }
  grid_exit(bar, gridDim.x);
}

template <typename T, int PM>
__global__ void __launch_bounds__(256, 2) k_ana2d_levels(CoarseIO<T> io, Tables<T> tab, Geo G, const __grid_constant__ CTaps<T, PM> ct,
                                                      const T* __restrict__ Dg, int rw, GridBarrier* bar,
                                                      unsigned int limit) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  SmemTables<T> st;
  int off = stage_filters(tab, G, sm, st, tid, nthr);
  const bool per = G.bd == UW_BOUNDARY_PERIODIC;
  // edge corrections transposed, [side][2PM + 1 columns][LBP rows], zero-padded (EdgeT)
  constexpr int DW = 2 * PM, LBP = EdgeT<T, PM>::LBP;
  const int nD = per ? 0 : 2 * (DW + 1) * LBP;      // entries (padding words are never read)
  T* Dl = sm + off;
  for (int i = tid; i < nD; i += nthr) {
    const int side = i / ((DW + 1) * LBP), rem = i - side * ((DW + 1) * LBP), c = rem / LBP, r = rem - c * LBP;
    const int e = c < PM ? c : c - PM;
    Dl[side * EdgeT<T, PM>::ana_side + EdgeT<T, PM>::acol(c) + r] =
        (c < DW && r < G.Lb && e < G.p) ? Dg[(side * G.Lb + r) * 2 * G.p + (c < PM ? e : G.p + e)] : T(0);
  }
  const T* Dr = Dl + EdgeT<T, PM>::ana_side;
  off = cup(off + (per ? 0 : EdgeT<T, PM>::ana_words), 4);
  pdl_trigger();
  pdl_wait();
  const int M = io.M, Mh = M / 2;
  const int64_t HH = (int64_t)Mh * Mh;
  const int R = io.J0 + io.nl + 1;
  const bool tx = io.XT != nullptr;
  for (int it = 0; it < io.nl; ++it) {
    const int j = R - 2 - it, n0 = 1 << j;
    const int TR = rw ? ana_rw_ts(n0) : 0;
    const int TS = TR ? TR : ana_tile(n0), tiles = (n0 / TS) * (n0 / TS), ltiles = __ffs(tiles) - 1;
    const T* src = it % 2 == 0 ? io.XS : io.XS2;
    T* dst = it == io.nl - 1 ? nullptr : (it % 2 == 0 ? io.XS2 : io.XS);
    const T* xt = tx && it == 0 ? io.XT : nullptr;
    const int TB = tiles * io.batch, q0 = io.tq0[it], nq = tx ? io.tnq[it] : 0;
    for (int t = blockIdx.x; t < TB + nq; t += gridDim.x) {
      __syncthreads();
      if (t >= TB)
        tx_item(q0 + t - TB, M, (const T*)io.XT, io.xout, false, sm + off, tid);
      else if (TR == 16)
        ana_tile_rw<T, PM, 16>(t & (tiles - 1), t >> ltiles, src, (int64_t)Mh, HH, io.xout, M, dst, (int64_t)Mh, HH, j, ct,
                               Dl, Dr, G.p, G.Lb, per, sm + off, tid, nthr, xt);
      else if (TR == 8)
        ana_tile_rw<T, PM, 8>(t & (tiles - 1), t >> ltiles, src, (int64_t)Mh, HH, io.xout, M, dst, (int64_t)Mh, HH, j, ct,
                              Dl, Dr, G.p, G.Lb, per, sm + off, tid, nthr, xt);
      else
        ana2d_tile<T, 0>(t & (tiles - 1), t >> ltiles, src, (int64_t)Mh, HH, io.xout, M, dst, (int64_t)Mh, HH, j, TS, st,
                         sm + off, G, tid, nthr);
    }
    if (it + 1 < io.nl && !grid_barrier(bar, gridDim.x, it, limit)) break;
  }
  grid_exit(bar, gridDim.x);
}

// FP32 transpose with 64 x 64 tiles and 16-byte global accesses; rows,
// cols, br and bc are multiples of 64, so a tile is entirely inside or
// outside the spliced block (same semantics as k_transpose).
__global__ void __launch_bounds__(256) k_transpose64(const float* __restrict__ in, float* __restrict__ out, int rows,
                                                     int cols, int64_t in_batch, int64_t out_batch,
                                                     const float* __restrict__ alt, int64_t alt_batch,
                                                     float* __restrict__ altout, int br, int bc, int ldalt) {
  __shared__ float tile[64][65];
  pdl_trigger();
  pdl_wait();
  const int64_t b = blockIdx.z;
  const int r0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
  const int t = threadIdx.x, c4 = t & 15, rw = t >> 4;
  const bool from_alt = alt && r0 < br && c0 < bc;
  float4 v[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + rw + 16 * i;
    const float* src = from_alt ? alt + b * alt_batch + (int64_t)r * ldalt + c0
                                : in + b * in_batch + (int64_t)r * cols + c0;
    v[i] = __ldg(reinterpret_cast<const float4*>(src) + c4);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = rw + 16 * i;
    tile[r][4 * c4 + 0] = v[i].x;
    tile[r][4 * c4 + 1] = v[i].y;
    tile[r][4 * c4 + 2] = v[i].z;
    tile[r][4 * c4 + 3] = v[i].w;
  }
  __syncthreads();
  const bool to_alt = altout && c0 < br && r0 < bc;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int orow = rw + 16 * i;  // output row c0 + orow, columns r0 + 4 c4 ..
    float4 w;
    w.x = tile[4 * c4 + 0][orow];
    w.y = tile[4 * c4 + 1][orow];
    w.z = tile[4 * c4 + 2][orow];
    w.w = tile[4 * c4 + 3][orow];
    float* dst = to_alt ? altout + b * alt_batch + (int64_t)(c0 + orow) * ldalt + r0
                        : out + b * out_batch + (int64_t)(c0 + orow) * rows + r0;
    reinterpret_cast<float4*>(dst)[c4] = w;
  }
}

template <typename T>
__global__ void k_copy_block(const T* __restrict__ in, int64_t ldin, int64_t in_batch, T* __restrict__ out,
                             int64_t ldout, int64_t out_batch, int rows, int cols, int batch) {
  const int64_t total = (int64_t)batch * rows * cols;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int c = (int)(idx % cols);
    int64_t r2 = idx / cols;
    int r = (int)(r2 % rows);
    int64_t b = r2 / rows;
    out[b * out_batch + r * ldout + c] = in[b * in_batch + r * ldin + c];
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static Geo geo_of(const Plan& P) {
  Geo G;
  G.p = P.p; G.q = P.q; G.Q = P.Q; G.R = P.R; G.M = P.M; G.N = P.N; G.L = P.R + P.q;
  G.bd = P.bd; G.ntap = P.ntap; G.Lb = P.Lb;
  return G;
}

template <typename T>
static size_t line_smem(const Plan& P) {
  Geo G = geo_of(P);
  return sizeof(T) * ((size_t)table_count(G) + 2 * (size_t)P.M + (size_t)padlen(P.N));
}

static const size_t kSmemMax = 200 * 1024;

template <typename T>
static bool line_fits(const Plan& P) { return line_smem<T>(P) <= kSmemMax; }

// largest level whose 2^j x 2^j block (two copies) fits one CTA's shared memory
template <typename T>
static void set_table_ptrs(Tables<T>& t, const T* base, const std::vector<const std::vector<double>*>& parts) {
  const T** slots[9] = {&t.h, &t.g, &t.taps, &t.EL, &t.ER, &t.PL, &t.QL, &t.PR, &t.QR};
  size_t o = 0;
  for (int i = 0; i < 9; ++i) {
    *slots[i] = base + o;
    o += parts[i]->size();
  }
}

int upload_tables(Plan& P) {
  std::vector<const std::vector<double>*> parts = {&P.h, &P.g, &P.taps, &P.EL, &P.ER, &P.PL, &P.QL, &P.PR, &P.QR};
  size_t n = 0;
  for (auto v : parts) n += v->size();
  std::vector<double> d64;
  std::vector<float> d32;
  d64.reserve(n);
  for (auto v : parts) d64.insert(d64.end(), v->begin(), v->end());
  d32.assign(d64.begin(), d64.end());
  if (cudaMalloc(&P.d_tab64, n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&P.d_tab32, n * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    set_error(UW_ERR_OOM, "table allocation failed");
    return UW_ERR_OOM;
  }
  if (cudaMemcpy(P.d_tab64, d64.data(), n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(P.d_tab32, d32.data(), n * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
    set_error(UW_ERR_CUDA, "table upload failed");
    return UW_ERR_CUDA;
  }
  set_table_ptrs(P.t64, (const double*)P.d_tab64, parts);
  set_table_ptrs(P.t32, (const float*)P.d_tab32, parts);
  std::vector<uint32_t> tcw;
  build_tc(P, tcw);
  if (P.tc.ok) {
    if (cudaMalloc(&P.d_tc, tcw.size() * sizeof(uint32_t)) != cudaSuccess) {
      cudaGetLastError();
      set_error(UW_ERR_OOM, "tensor-core table allocation failed");
      return UW_ERR_OOM;
    }
    if (cudaMemcpy(P.d_tc, tcw.data(), tcw.size() * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess) {
      set_error(UW_ERR_CUDA, "tensor-core table upload failed");
      return UW_ERR_CUDA;
    }
  }
  std::vector<unsigned char> uw5;
  build_umma(P, uw5);
  if (P.umma.ok) {
    if (cudaMalloc(&P.d_umma, uw5.size()) != cudaSuccess) {
      cudaGetLastError();
      set_error(UW_ERR_OOM, "tensor-core operator allocation failed");
      return UW_ERR_OOM;
    }
    if (cudaMemcpy(P.d_umma, uw5.data(), uw5.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
      set_error(UW_ERR_CUDA, "tensor-core operator upload failed");
      return UW_ERR_CUDA;
    }
  }
  if (cudaMalloc(&P.d_sync, sizeof(GridBarrier)) != cudaSuccess) {
    cudaGetLastError();
    set_error(UW_ERR_OOM, "barrier allocation failed");
    return UW_ERR_OOM;
  }
  if (cudaMemset(P.d_sync, 0, sizeof(GridBarrier)) != cudaSuccess) {
    set_error(UW_ERR_CUDA, "barrier initialisation failed");
    return UW_ERR_CUDA;
  }
  {
    std::vector<double> D;
    P.coarse_ok = build_coarse(P, D) ? 1 : 0;
    if (P.coarse_ok && !D.empty()) {
      std::vector<float> Df(D.begin(), D.end());
      const size_t bytes = D.size() * (sizeof(double) + sizeof(float));
      if (cudaMalloc(&P.d_coarse, bytes) != cudaSuccess) {
        cudaGetLastError();
        set_error(UW_ERR_OOM, "coarse-level table allocation failed");
        return UW_ERR_OOM;
      }
      if (cudaMemcpy(P.d_coarse, D.data(), D.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy((double*)P.d_coarse + D.size(), Df.data(), Df.size() * sizeof(float),
                     cudaMemcpyHostToDevice) != cudaSuccess) {
        set_error(UW_ERR_CUDA, "coarse-level table upload failed");
        return UW_ERR_CUDA;
      }
    }
  }
  std::vector<float> f32w;
  build_f32(P, f32w);
  if (P.f32.ok && !f32w.empty()) {
    if (cudaMalloc(&P.d_f32, f32w.size() * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      set_error(UW_ERR_OOM, "edge-correction table allocation failed");
      return UW_ERR_OOM;
    }
    if (cudaMemcpy(P.d_f32, f32w.data(), f32w.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
      set_error(UW_ERR_CUDA, "edge-correction table upload failed");
      return UW_ERR_CUDA;
    }
  }
  return UW_OK;
}

size_t work2d_elems(const Plan& P, int batch);

size_t workspace_bytes(const Plan& P, int batch) {
  const size_t M = P.M, N = P.N, B = batch, e = sizeof(double);
  if (P.d == 1) {
    if (line_fits<double>(P) && line_fits<float>(P)) return 256;
    return e * B * (2 * M + N) + 256;
  }
  return e * work2d_elems(P, batch) + 1024;
}

// elements of scratch the 2D path (fwd2d / adj2d) uses for `batch` instances
size_t work2d_elems(const Plan& P, int batch) {
  const size_t M = P.M, N = P.N, B = batch, Mh = M / 2;
  size_t xs = 2 * B * Mh * Mh;   // XS, XS2: coarse level buffers
  size_t a = B * M * M;          // XT / X'T
  size_t vt = B * M * N;         // VT / QT
  size_t v = B * N * M;          // V / Q
  return xs + a + vt + v;
}

struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t next = 0;
  struct Rec { int id; cudaEvent_t a, b; };
  std::vector<Rec> pending;
  std::map<std::string, int> ids;
  std::vector<std::string> names;
  std::vector<double> ms, bytes;
  std::vector<int64_t> cnt;
  cudaEvent_t get() {
    if (next == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[next++];
  }
  void collect() {
    for (auto& r : pending) {
      float t = 0;
      cudaEventSynchronize(r.b);
      cudaEventElapsedTime(&t, r.a, r.b);
      ms[r.id] += t;
      cnt[r.id] += 1;
    }
    pending.clear();
    next = 0;
  }
};

void profiler_free(Plan& P) {
  if (!P.prof) return;
  for (auto e : P.prof->pool) cudaEventDestroy(e);
  delete P.prof;
  P.prof = nullptr;
}

struct Launcher {
  cudaStream_t s;
  bool split = false;      // UW_F32_SPLIT_BF16: line operators on the tensor cores where eligible
  int count = 0;
  cudaError_t err = cudaSuccess;
  Profiler* prof = nullptr;
  Profiler::Rec cur{};
  bool armed = false;
  // call before each kernel launch: name and algorithmic bytes of the launch
  void pre(const char* name, double bytes) {
    armed = false;
    if (!prof || !prof->on) return;
    auto it = prof->ids.find(name);
    int id;
    if (it == prof->ids.end()) {
      id = (int)prof->names.size();
      prof->ids[name] = id;
      prof->names.push_back(name);
      prof->ms.push_back(0);
      prof->bytes.push_back(0);
      prof->cnt.push_back(0);
    } else {
      id = it->second;
    }
    prof->bytes[id] = bytes;
    cur = {id, prof->get(), prof->get()};
    cudaEventRecord(cur.a, s);
    armed = true;
  }
  // record the status of a cudaLaunchKernelEx launch
  void note(cudaError_t e) {
    if (e != cudaSuccess && err == cudaSuccess) err = e;
  }
  // rename the armed launch (same bytes), e.g. when a line operator takes
  // the tensor-core kernel
  void retag(const std::string& name) {
    if (!armed) return;
    const double bytes = prof->bytes[cur.id];
    auto it = prof->ids.find(name);
    int id;
    if (it == prof->ids.end()) {
      id = (int)prof->names.size();
      prof->ids[name] = id;
      prof->names.push_back(name);
      prof->ms.push_back(0);
      prof->bytes.push_back(0);
      prof->cnt.push_back(0);
    } else {
      id = it->second;
    }
    prof->bytes[id] = bytes;
    cur.id = id;
  }
  void check() {
    ++count;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess && err == cudaSuccess) err = e;
    if (armed) {
      cudaEventRecord(cur.b, s);
      prof->pending.push_back(cur);
      if (prof->pending.size() > 4000) prof->collect();
      armed = false;
    }
  }
};

static int grid_for(int64_t total, int threads = 256) {
  int64_t g = (total + threads - 1) / threads;
  return (int)std::min<int64_t>(std::max<int64_t>(g, 1), 152 * 32);
}

template <typename T>
static const Tables<T>& tabs(const Plan& P);
template <>
const Tables<double>& tabs<double>(const Plan& P) { return P.t64; }
template <>
const Tables<float>& tabs<float>(const Plan& P) { return P.t32; }

// raise a kernel's dynamic shared-memory limit to the device maximum, once
// per kernel and device (the launch itself passes the bytes it uses)
cudaError_t set_smem_limit(const void* fn) {
  static std::mutex mu;
  static std::set<std::pair<int, const void*>> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({dev, fn})) return cudaSuccess;
  int mx = 0;
  cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, fn);
  if (e == cudaSuccess)   // the static shared memory of the kernel counts against the same limit
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, mx - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess) done.insert({dev, fn});
  else cudaGetLastError();   // leave no sticky status for the launch checks
  return e;
}

template <typename T>
static cudaError_t set_smem(const void* fn, size_t) {
  return set_smem_limit(fn);
}

static bool getenv_flag(const char* name) {
  const char* v = getenv(name);
  return v && v[0] && v[0] != '0';
}

static int line_threads(int N) { return N >= 4096 ? 256 : (N >= 1024 ? 128 : 64); }

// One launch of the line operator: the register-blocked FP32 kernels where
// they apply, the generic kernels otherwise.
template <typename T>
static void launch_line(bool fwd, const Plan& P, const Geo& G, const T* in, T* out, const LineIO& io, int nblocks,
                        Launcher& L) {
  size_t sm = line_smem<T>(P);
  if (fwd) {
    set_smem<T>((const void*)k_line_fwd<T>, sm);
    L.note(launch_pdl(k_line_fwd<T>, dim3(nblocks), dim3(line_threads(P.N)), sm, L.s, in, out, tabs<T>(P), G, io));
  } else {
    set_smem<T>((const void*)k_line_adj<T>, sm);
    L.note(launch_pdl(k_line_adj<T>, dim3(nblocks), dim3(line_threads(P.N)), sm, L.s, in, out, tabs<T>(P), G, io));
  }
}

template <>
void launch_line<float>(bool fwd, const Plan& P, const Geo& G, const float* in, float* out, const LineIO& io,
                        int nblocks, Launcher& L) {
  if (L.split && P.line_variant == 0 && !getenv_flag("UW_NO_UMMA") && umma_eligible(P, io, in, out, fwd, nblocks)) {
    if (L.armed) L.retag(P.prof->names[L.cur.id] + "_umma");
    L.note(umma_launch(fwd, P, in, out, io, nblocks, L.s));
    return;
  }
  if (L.split && P.line_variant == 0 && tc_eligible(P, io, in, out, fwd)) {
    if (L.armed) L.retag(P.prof->names[L.cur.id] + "_tc");
    L.note(tc_launch(fwd, P, in, out, io, nblocks, L.s));
    return;
  }
  const bool generic = P.line_variant == 1 || getenv_flag("UW_GENERIC_LINES");
  if (!L.split && !generic && f32_eligible(P, io, in, out, fwd)) {
    if (L.armed) L.retag(P.prof->names[L.cur.id] + "_f32");
    L.note(f32_launch(fwd, P, in, out, io, nblocks, L.s));
    return;
  }
  if (!generic && line2_eligible(P)) {
    L.note(line2_launch(fwd, P, G, in, out, io, nblocks, L.s));
    return;
  }
  size_t sm = line_smem<float>(P);
  if (fwd) {
    set_smem<float>((const void*)k_line_fwd<float>, sm);
    L.note(launch_pdl(k_line_fwd<float>, dim3(nblocks), dim3(line_threads(P.N)), sm, L.s, in, out, tabs<float>(P), G,
                      io));
  } else {
    set_smem<float>((const void*)k_line_adj<float>, sm);
    L.note(launch_pdl(k_line_adj<float>, dim3(nblocks), dim3(line_threads(P.N)), sm, L.s, in, out, tabs<float>(P), G,
                      io));
  }
}

// coarse levels J0 .. R-2 of the 2D Mallat transform, one fused kernel per
// level.  forward: S_{J0} and the details from x, S_{R-1} ends in XS;
// adjoint: S_{R-1} from XS, the low-pass block and details of every level
// end in x.  XS and XS2 (Mh x Mh per instance) alternate as level buffers.
// filter length as a compile-time constant for the FP32 coarse kernels
// (p = 1..10); FP64 runs the runtime-p variant (P = 0)
template <typename T, typename F>
static void coarse_dispatch(int p, F&& f) {
  if constexpr (sizeof(T) == 8) {
    f(std::integral_constant<int, 0>{});
  } else {
  switch (p) {
    case 1: f(std::integral_constant<int, 1>{}); break;
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 3: f(std::integral_constant<int, 3>{}); break;
    case 4: f(std::integral_constant<int, 4>{}); break;
    case 5: f(std::integral_constant<int, 5>{}); break;
    case 6: f(std::integral_constant<int, 6>{}); break;
    case 7: f(std::integral_constant<int, 7>{}); break;
    case 8: f(std::integral_constant<int, 8>{}); break;
    case 9: f(std::integral_constant<int, 9>{}); break;
    default: f(std::integral_constant<int, 10>{}); break;
  }
  }
}

static int coarse_tile_extent(const Geo& G, int j, bool syn) {
  const int n0 = 1 << j, n1 = 2 * n0;
  const int TS = syn ? syn_tile(n1) : ana_tile(n0);
  const int span = syn ? n1 : n0;
  int worst = 0;
  for (int a = 0; a < span; a += TS) {
    int lo, hi;
    if (syn) syn_dep(a, a + TS, n0, G, lo, hi);
    else ana_dep(a, a + TS, n0, G, lo, hi);
    worst = std::max(worst, hi - lo);
  }
  return worst;
}

// polls of a grid-barrier wait before it gives up (read at every launch)
static unsigned int barrier_spin_limit() {
  const char* e = getenv("UW_BARRIER_SPIN_LIMIT");
  return e && e[0] ? (unsigned int)strtoul(e, nullptr, 10) : (1u << 22);
}

template <typename T, int PM>
static CTaps<T, PM> make_ctaps(const Plan& P) {
  CTaps<T, PM> t;
  const int p = P.p;
  for (int f = 0; f < 2; ++f)
    for (int d = -PM / 2; d <= PM / 2; ++d) {
      const int l = 2 * d + f;
      const bool in = l >= -p + 1 && l <= p;
      t.hp[f][d + PM / 2] = in ? (T)P.h[l + p - 1] : T(0);
      t.gp[f][d + PM / 2] = in ? (T)P.g[l + p - 1] : T(0);
    }
  for (int l = -PM + 1; l <= PM; ++l) {
    const bool in = l >= -p + 1 && l <= p;
    t.ha[l + PM - 1] = in ? (T)P.h[l + p - 1] : T(0);
    t.ga[l + PM - 1] = in ? (T)P.g[l + p - 1] : T(0);
  }
  return t;
}

// filter length rounded up to an even compile-time PM >= p
template <typename F>
static void pm_dispatch(int p, F&& f) {
  if (p <= 2) f(std::integral_constant<int, 2>{});
  else if (p <= 4) f(std::integral_constant<int, 4>{});
  else if (p <= 6) f(std::integral_constant<int, 6>{});
  else if (p <= 8) f(std::integral_constant<int, 8>{});
  else f(std::integral_constant<int, 10>{});
}

// whether the fused coarse-level launch also makes the layout change of the
// line passes' transposed buffer (needs the register-window tiles at the
// finest coarse level and 64-aligned quadrants)
static bool coarse_tx_ok(const Plan& P) {
  const int nl = P.R - 1 - P.J0;
  return nl >= 2 && nl <= kMaxCoarse && P.d_sync && P.coarse_ok && P.M % 128 == 0 &&
         (P.bd == UW_BOUNDARY_PERIODIC || P.d_coarse) && P.coarse_mode == 0 && !getenv_flag("UW_COARSE_PER_LEVEL") &&
         !getenv_flag("UW_COARSE_GENERIC") && !getenv_flag("UW_COARSE_SEPARATE_TRANSPOSE");
}

// All coarse levels in one cooperative launch (grid barrier between levels);
// false if that launch is not possible here (then one launch per level).
// XT non-null (only when coarse_tx_ok): the launch also moves the M x M
// coefficient array between x and its transpose XT.
template <typename T>
static bool launch_coarse_fused(const Plan& P, const Geo& G, const T* x, T* xout, T* XS, T* XS2, T* XT, int batch,
                                bool fwd, Launcher& L) {
  const int nl = P.R - 1 - P.J0;
  if (nl < 2 || nl > kMaxCoarse || !P.d_sync || P.coarse_mode == 1 || getenv_flag("UW_COARSE_PER_LEVEL")) return false;
  const bool rw = P.coarse_ok && !getenv_flag("UW_COARSE_GENERIC");
  const T* Dg = nullptr;
  if (P.d_coarse && P.bd != UW_BOUNDARY_PERIODIC) {
    const size_t nD = (size_t)4 * P.Lb * P.p;
    Dg = sizeof(T) == 8 ? (const T*)P.d_coarse : (const T*)((const double*)P.d_coarse + nD);
  }
  if (rw && P.bd != UW_BOUNDARY_PERIODIC && !Dg) return false;
  bool ok = false;
  pm_dispatch(G.p, [&](auto pc) {
    constexpr int PM = decltype(pc)::value;
    const int nD = P.bd == UW_BOUNDARY_PERIODIC ? 0 : (fwd ? EdgeT<T, PM>::syn_words : EdgeT<T, PM>::ana_words);
    const size_t head = (size_t)cup(cup(4 * G.p, 4) + nD, 4);
    size_t sm = 0;
    int max_tiles = 0;
    double bytes = 0;
    for (int it = 0; it < nl; ++it) {
      const int j = fwd ? P.J0 + it : P.R - 2 - it;
      const int n0 = 1 << j, n1 = 2 * n0;
      size_t el = 0;
      int TS = 0;
      if (fwd) {
        const int TR = rw ? syn_rw_ts(n1) : 0;
        if (TR == 32) el = SynGeom<T, PM, 32>::elems;
        else if (TR == 16) el = SynGeom<T, PM, 16>::elems;
        else {
          const int w = coarse_tile_extent(G, j, true);
          el = 4 * (size_t)w * w + 2 * (size_t)w * syn_tile(n1);
        }
        TS = TR ? TR : syn_tile(n1);
        max_tiles = std::max(max_tiles, (n1 / TS) * (n1 / TS));
      } else {
        const int TR = rw ? ana_rw_ts(n0) : 0;
        if (TR == 16) el = AnaGeom<T, PM, 16>::elems;
        else if (TR == 8) el = AnaGeom<T, PM, 8>::elems;
        else {
          const int w = coarse_tile_extent(G, j, false);
          if (w > 64) return;
          el = (size_t)w * w + 2 * (size_t)ana_tile(n0) * w;
        }
        TS = TR ? TR : ana_tile(n0);
        max_tiles = std::max(max_tiles, (n0 / TS) * (n0 / TS));
      }
      sm = std::max(sm, sizeof(T) * (head + el));
      bytes += sizeof(T) * (double)batch * (4.0 * n0 * n0 + (double)n1 * n1);
    }
    int Q = 0;
    if (XT) {
      const int Mh = P.M / 2;
      Q = 3 * (Mh / 64) * (Mh / 64) * batch;
      sm = std::max(sm, sizeof(T) * (head + 64 * 65));
      bytes += sizeof(T) * (double)batch * 6.0 * Mh * Mh;
    }
    CoarseIO<T> io{x, xout, XS, XS2, XT, P.M, P.J0, nl, batch, {}, {}};
    const CTaps<T, PM> ct = make_ctaps<T, PM>(P);
    auto kern = fwd ? k_syn2d_levels<T, PM> : k_ana2d_levels<T, PM>;
    set_smem_limit((const void*)kern);
    int dev = 0, nsm = 0, per = 0, coop = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, sm) != cudaSuccess || per < 1) {
      cudaGetLastError();
      return;
    }
    // at most two CTAs per SM: fewer arrivals at each grid barrier
    const int grid = (int)std::min<int64_t>((int64_t)std::min(per, 2) * nsm, (int64_t)max_tiles * batch + Q);
    if (XT) {
      // the level tiles of step k, as the kernels count them
      auto busy = [&](int k) {
        int n, TS;
        if (fwd) {
          n = 2 << (P.J0 + k);
          const int TR = rw ? syn_rw_ts(n) : 0;
          TS = TR ? TR : syn_tile(n);
        } else {
          n = 1 << (P.R - 2 - k);
          const int TR = rw ? ana_rw_ts(n) : 0;
          TS = TR ? TR : ana_tile(n);
        }
        return (n / TS) * (n / TS) * batch;
      };
      for (int it = 0; it < nl; ++it) tx_share(it, nl, fwd, grid, Q, busy, io.tq0[it], io.tnq[it]);
    }
    L.pre(fwd ? "idwt2d_levels" : "dwt2d_levels", bytes);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = L.s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    // cooperative launch with programmatic serialization where the driver
    // takes it (first decided by a launch outside stream capture)
    static std::atomic<int> coop_pdl{-1};
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(L.s, &cap);
    const int known = coop_pdl.load();
    cfg.numAttrs = known == 1 || (known < 0 && cap == cudaStreamCaptureStatusNone) ? 2 : 1;
    auto go = [&] {
      return cudaLaunchKernelEx(&cfg, kern, io, tabs<T>(P), G, ct, Dg, rw ? 1 : 0, (GridBarrier*)P.d_sync,
                                barrier_spin_limit());
    };
    cudaError_t err = go();
    if (known < 0 && cfg.numAttrs == 2) {
      coop_pdl.store(err == cudaSuccess ? 1 : 0);
      if (err != cudaSuccess) {
        cudaGetLastError();
        cfg.numAttrs = 1;
        err = go();
      }
    }
    L.note(err);
    L.check();
    ok = true;
  });
  return ok;
}

template <typename T>
static void launch_transpose(const T* in, T* out, int rows, int cols, int64_t in_batch, int64_t out_batch,
                             const T* alt, int64_t alt_batch, T* altout, int br, int bc, int ldalt, int batch,
                             Launcher& L);

// the adjoint's layout change XT -> x (top-left Mh x Mh block into XS)
template <typename T>
static void transpose_out(const Plan& P, const T* XT, T* x, T* XS, int batch, Launcher& L) {
  const int M = P.M, Mh = M / 2;
  const int64_t MM = (int64_t)M * M;
  L.pre("transpose_out", sizeof(T) * 2.0 * batch * MM);
  launch_transpose<T>(XT, x, M, M, MM, MM, nullptr, (int64_t)Mh * Mh, XS, Mh, Mh, Mh, batch, L);
  L.check();
}

// All coarse levels.  XT non-null: the caller leaves the layout change of the
// transposed buffer to this call (forward: after the levels, adjoint: before);
// true when the fused launch made it, false when the forward caller still has
// to (the adjoint's fallback makes it here, ahead of the per-level launches).
template <typename T>
static bool launch_coarse_levels(const Plan& P, const Geo& G, const T* x, T* xout, T* XS, T* XS2, T* XT, int batch,
                                 bool fwd, Launcher& L) {
  if (launch_coarse_fused<T>(P, G, x, xout, XS, XS2, XT, batch, fwd, L)) return XT != nullptr;
  if (XT && !fwd) transpose_out<T>(P, XT, xout, XS, batch, L);
  const int M = P.M, Mh = M / 2;
  const int nl = P.R - 1 - P.J0;
  const int64_t HH = (int64_t)Mh * Mh, MM = (int64_t)M * M;
  for (int it = 0; it < nl; ++it) {
    const int j = fwd ? P.J0 + it : P.R - 2 - it;
    const int n0 = 1 << j, n1 = 2 * n0;
    const int w = coarse_tile_extent(G, j, fwd);
    if (!fwd && w > 64) {  // the analysis column pass maps window columns to 64 lanes
      L.err = cudaErrorInvalidConfiguration;
      return false;
    }
    if (fwd) {
      const int TS = syn_tile(n1), tiles = n1 / TS;
      const int thr = TS >= 32 ? 256 : 128;
      const size_t sm = sizeof(T) * (((size_t)4 * G.p + 3) / 4 * 4 + 4 * (size_t)w * w + 2 * (size_t)w * TS);
      const T* src = it == 0 ? x : ((nl - it) % 2 == 0 ? XS : XS2);
      const int64_t ld = it == 0 ? M : Mh, sb = it == 0 ? MM : HH;
      T* dst = (nl - 1 - it) % 2 == 0 ? XS : XS2;
      char name[32];
      snprintf(name, sizeof name, "idwt2d_level_j%d", j);
      L.pre(name, sizeof(T) * (double)batch * (4.0 * n0 * n0 + (double)n1 * n1));
      coarse_dispatch<T>(G.p, [&](auto pc) {
        constexpr int PP = decltype(pc)::value;
        set_smem_limit((const void*)k_syn2d_level<T, PP>);
        L.note(launch_pdl(k_syn2d_level<T, PP>, dim3(tiles * tiles, batch), dim3(thr), sm, L.s, src, ld, sb, x, M,
                          dst, (int64_t)Mh, HH, j, TS, tabs<T>(P), G));
      });
    } else {
      const int TS = ana_tile(n0), tiles = n0 / TS;
      const int thr = TS >= 16 ? 256 : 128;
      const size_t sm = sizeof(T) * (((size_t)4 * G.p + 3) / 4 * 4 + (size_t)w * w + 2 * (size_t)TS * w);
      const T* src = it % 2 == 0 ? XS : XS2;
      T* dst = it == nl - 1 ? nullptr : (it % 2 == 0 ? XS2 : XS);
      char name[32];
      snprintf(name, sizeof name, "dwt2d_level_j%d", j);
      L.pre(name, sizeof(T) * (double)batch * (4.0 * n0 * n0 + (double)n1 * n1));
      coarse_dispatch<T>(G.p, [&](auto pc) {
        constexpr int PP = decltype(pc)::value;
        set_smem_limit((const void*)k_ana2d_level<T, PP>);
        L.note(launch_pdl(k_ana2d_level<T, PP>, dim3(tiles * tiles, batch), dim3(thr), sm, L.s, src, (int64_t)Mh, HH,
                          xout, M, dst, (int64_t)Mh, HH, j, TS, tabs<T>(P), G));
      });
    }
    L.check();
  }
  return false;
}

// transpose dispatcher: the 64 x 64 FP32 kernel where shapes allow
template <typename T>
static void launch_transpose(const T* in, T* out, int rows, int cols, int64_t in_batch, int64_t out_batch,
                             const T* alt, int64_t alt_batch, T* altout, int br, int bc, int ldalt, int batch,
                             Launcher& L) {
  dim3 tb(32, 8);
  dim3 tg((cols + 31) / 32, (rows + 31) / 32, batch);
  L.note(launch_pdl(k_transpose<T>, tg, tb, 0, L.s, in, out, rows, cols, in_batch, out_batch, alt, alt_batch, altout,
                    br, bc, ldalt));
}

template <>
void launch_transpose<float>(const float* in, float* out, int rows, int cols, int64_t in_batch, int64_t out_batch,
                             const float* alt, int64_t alt_batch, float* altout, int br, int bc, int ldalt, int batch,
                             Launcher& L) {
  // 16-byte vector accesses: every base pointer and every stride must keep
  // 16-byte alignment, otherwise the scalar kernel runs
  auto al16 = [](const void* q) { return ((uintptr_t)q & 15u) == 0; };
  const bool ok = rows % 64 == 0 && cols % 64 == 0 && br % 64 == 0 && bc % 64 == 0 && ldalt % 4 == 0 &&
                  in_batch % 4 == 0 && out_batch % 4 == 0 && alt_batch % 4 == 0 && al16(in) && al16(out) &&
                  (!alt || al16(alt)) && (!altout || al16(altout));
  if (!ok) {
    dim3 tb(32, 8);
    dim3 tg((cols + 31) / 32, (rows + 31) / 32, batch);
    L.note(launch_pdl(k_transpose<float>, tg, tb, 0, L.s, in, out, rows, cols, in_batch, out_batch, alt, alt_batch,
                      altout, br, bc, ldalt));
    return;
  }
  dim3 tg(cols / 64, rows / 64, batch);
  L.note(launch_pdl(k_transpose64, tg, dim3(256), 0, L.s, in, out, rows, cols, in_batch, out_batch, alt, alt_batch,
                    altout, br, bc, ldalt));
}

// 1D, the whole line in shared memory.
template <typename T>
static void fwd1d_smem(const Plan& P, const T* x, T* y, int batch, Launcher& L) {
  const double e = sizeof(T);
  Geo G = geo_of(P);
  LineIO io{};
  io.in_stride = P.M; io.out_stride = P.N; io.lines = 1; io.in_batch = P.M; io.out_batch = P.m;
  io.seq_rows = 0; io.mode = 1; io.jlev = P.J0; io.mask = P.d_mask; io.prefix = P.d_prefix; io.pos = P.d_pos;
  io.wpr = P.wpr; io.m = P.m; io.mask_rows = 1;
  L.pre("line_fwd_1d", e * ((double)batch * (P.M + P.m)) + 8.0 * P.words);
  launch_line<T>(true, P, G, x, y, io, batch, L);
  L.check();
}

template <typename T>
static void adj1d_smem(const Plan& P, const T* y, T* x, int batch, Launcher& L) {
  const double e = sizeof(T);
  Geo G = geo_of(P);
  LineIO io{};
  io.in_stride = P.N; io.out_stride = P.M; io.lines = 1; io.in_batch = P.m; io.out_batch = P.M;
  io.seq_rows = 0; io.mode = 1; io.jlev = P.J0; io.mask = P.d_mask; io.prefix = P.d_prefix; io.pos = P.d_pos;
  io.wpr = P.wpr; io.m = P.m; io.mask_rows = 1;
  L.pre("line_adj_1d", e * ((double)batch * (P.M + P.m)) + 8.0 * P.words);
  launch_line<T>(false, P, G, y, x, io, batch, L);
  L.check();
}

// 1D, lines larger than shared memory: level kernels + T + two-pass FWHT.
// the stages across segments of 4096 (L1 = L - 12 in 3..6) with the gather
// (mode 1) or the scatter (mode 2) folded in; false if not applicable
// The stages of bits 12.. of FP32 1D lines across their segments of 4096,
// writing the sampled outputs straight into yout (mode 1) or reading the
// input from yin (mode 2) through the natural-position-to-sample table;
// false if the shape does not suit (the caller then runs the plain stages
// and a separate gather / scatter).
static bool cols_with_samples(const Plan& P, float* v, const float* yin, float* yout, int batch, int mode,
                              Launcher& Lc) {
  const int L = geo_of(P).L, L2 = 12, L1 = L - L2;
  if (!P.d_nat2y || L1 < 3 || L1 > 6) return false;
  Lc.pre(mode == 1 ? "fwht_cols_gather_1d" : "fwht_cols_scatter_1d",
         sizeof(float) * (double)batch * ((double)(1LL << L) + 2.0 * P.m) + 4.0 * (double)(1LL << L));
  auto go = [&](auto l1) {
    constexpr int LL = decltype(l1)::value;
    // 4 columns per thread: 16-byte accesses to the line (its base and the
    // table are 256-byte aligned; rows are 2^12 floats apart)
    const dim3 g4((unsigned)(batch * ((1 << L2) / 128)));
    if (mode == 1)
      Lc.note(launch_pdl(k_fwht_cols128<LL, 1>, g4, dim3(256), 0, Lc.s, v, L2, (const int32_t*)P.d_nat2y,
                         (const float*)nullptr, yout, (int64_t)P.m));
    else
      Lc.note(launch_pdl(k_fwht_cols128<LL, 2>, g4, dim3(256), 0, Lc.s, v, L2, (const int32_t*)P.d_nat2y, yin,
                         (float*)nullptr, (int64_t)P.m));
  };
  if (L1 == 3) go(std::integral_constant<int, 3>{});
  else if (L1 == 4) go(std::integral_constant<int, 4>{});
  else if (L1 == 5) go(std::integral_constant<int, 5>{});
  else go(std::integral_constant<int, 6>{});
  Lc.check();
  return true;
}

template <typename T>
static void fwht_big(T* v, int L, int batch, Launcher& Lc, bool segments = true) {
  int L2 = std::min(L, 12), L1 = L - L2;
  if (segments) {
    size_t sm2 = sizeof(T) * padlen(1 << L2);
    set_smem<T>((const void*)k_fwht_seg<T>, sm2);
    Lc.pre("fwht_seg", 2.0 * sizeof(T) * (double)batch * (double)(1LL << L));
    k_fwht_seg<T><<<(int64_t)batch << L1, 256, sm2, Lc.s>>>(v, L2);
    Lc.check();
  }
  if (L1 >= 3 && L1 <= 6 && L2 >= 5) {
    Lc.pre("fwht_cols", 2.0 * sizeof(T) * (double)batch * (double)(1LL << L));
    const dim3 grid((unsigned)(batch * ((1 << L2) / 32)));
    if (L1 == 3) k_fwht_cols32<T, 3><<<grid, 256, 0, Lc.s>>>(v, L2);
    else if (L1 == 4) k_fwht_cols32<T, 4><<<grid, 256, 0, Lc.s>>>(v, L2);
    else if (L1 == 5) k_fwht_cols32<T, 5><<<grid, 256, 0, Lc.s>>>(v, L2);
    else k_fwht_cols32<T, 6><<<grid, 256, 0, Lc.s>>>(v, L2);
    Lc.check();
  } else if (L1 > 0) {
    const int COLS = 8;
    size_t sm1 = sizeof(T) * COLS * padlen(1 << L1);
    set_smem<T>((const void*)k_fwht_cols<T, COLS>, sm1);
    Lc.pre("fwht_cols", 2.0 * sizeof(T) * (double)batch * (double)(1LL << L));
    k_fwht_cols<T, COLS><<<batch * ((1 << L2) / COLS), 256, sm1, Lc.s>>>(v, L1, L2);
    Lc.check();
  }
}

// Largest level jto <= R - 1 whose synthesis (analysis) levels below it fit
// one CTA's shared memory (the tables and two buffers of 2^(jto-1)); 0 if
// no level above J0 does.
template <typename T>
static int fused1d_top(const Plan& P) {
  const Geo G = geo_of(P);
  int jto = 0;
  for (int j = P.J0 + 1; j <= P.R - 1; ++j)
    if (sizeof(T) * ((size_t)table_count(G) + 4 + 2 * ((size_t)1 << (j - 1))) <= kSmemMax) jto = j;
  return jto;
}

template <typename T>
static size_t fused1d_smem(const Plan& P, int jto) {
  return sizeof(T) * ((size_t)table_count(geo_of(P)) + 4 + 2 * ((size_t)1 << (jto - 1)));
}

// 1D, lines larger than shared memory: the coarse levels of each line in one
// CTA, the levels above them one launch each, T, the two-pass FWHT, gather.
template <typename T>
static void fwd1d_big(const Plan& P, const T* x, T* y, int batch, T* work, Launcher& L) {
  const double e = sizeof(T);
  Geo G = geo_of(P);
  const int M = P.M, N = P.N;
  T* sA = work;
  T* sB = sA + (size_t)batch * M;
  T* v = sB + (size_t)batch * M;
  const int jto = fused1d_top<T>(P);
  const T* cur = x;          // s_j of every line at cur + b M (the coarsest block of x to start)
  int j = P.J0;
  constexpr bool f32 = std::is_same<T, float>::value;
  if (jto) {
    const size_t sm = fused1d_smem<T>(P, jto);
    L.pre("syn_levels_1d", e * 2.0 * batch * (double)(1 << jto));
    if constexpr (f32) {
      L.note(f32_syn1d_levels(P, G, x, sA, jto, sm, batch, L.s));
    } else {
      set_smem<T>((const void*)k_syn1d_levels<T>, sm);
      L.note(launch_pdl(k_syn1d_levels<T>, dim3(batch), dim3(1024), sm, L.s, x, sA, (int64_t)M, tabs<T>(P), G, P.J0,
                        jto, (int64_t)M));
    }
    L.check();
    cur = sA;
    j = jto;
  }
  for (; j < P.R; ++j) {
    const int n0 = 1 << j;
    T* o = cur == sB ? sA : sB;
    L.pre("syn_level_1d", e * 4.0 * batch * n0);
    if (f32 && n0 >= 4) {
      if constexpr (f32) L.note(f32_syn1d_level(P, G, cur, x + n0, o, n0, batch, L.s));
    } else {
      k_syn1d_level<T><<<grid_for((int64_t)batch * 2 * n0), 256, 0, L.s>>>(cur, M, x + n0, M, o, M, n0, tabs<T>(P), G,
                                                                            batch);
    }
    L.check();
    cur = o;
  }
  if constexpr (std::is_same<T, float>::value) {
    if (f32_seg_eligible(P)) {
      // T and the stages of bits 0-11 per segment of 4096, then bits 12..
      L.pre("upconv_fwht_seg_1d", e * (double)batch * (M + N));
      L.note(f32_seg_up(P, G, cur, v, batch, L.s));
      L.check();
      if (cols_with_samples(P, v, nullptr, y, batch, 1, L)) return;
      fwht_big<T>(v, G.L, batch, L, false);
      L.pre("gather_1d", e * 2.0 * batch * P.m + 8.0 * P.words);
      k_gather<T><<<grid_for((int64_t)batch * P.words), 256, 0, L.s>>>(v, y, P.d_mask, P.d_prefix, P.words, G.L, N, P.m,
                                                                        batch);
      L.check();
      return;
    }
  }
  L.pre("upconv_1d", e * (double)batch * (M + N));
  k_up<T><<<grid_for((int64_t)batch * N), 256, 0, L.s>>>(cur, v, tabs<T>(P), G, batch);
  L.check();
  fwht_big<T>(v, G.L, batch, L);
  L.pre("gather_1d", e * 2.0 * batch * P.m + 8.0 * P.words);
  k_gather<T><<<grid_for((int64_t)batch * P.words), 256, 0, L.s>>>(v, y, P.d_mask, P.d_prefix, P.words, G.L, N, P.m, batch);
  L.check();
}

template <typename T>
static void adj1d_big(const Plan& P, const T* y, T* x, int batch, T* work, Launcher& L) {
  const double e = sizeof(T);
  Geo G = geo_of(P);
  const int M = P.M, N = P.N;
  T* sA = work;
  T* sB = sA + (size_t)batch * M;
  T* v = sB + (size_t)batch * M;
  bool scattered = false;
  auto scatter = [&]() {
    cudaMemsetAsync(v, 0, sizeof(T) * (size_t)batch * N, L.s);
    L.pre("scatter_1d", e * 2.0 * batch * P.m + 8.0 * P.words);
    k_scatter<T><<<grid_for((int64_t)batch * P.words), 256, 0, L.s>>>(y, v, P.d_mask, P.d_prefix, P.words, G.L, N, P.m,
                                                                       batch);
    L.check();
  };
  bool done = false;
  if constexpr (std::is_same<T, float>::value) {
    if (f32_seg_eligible(P)) {
      // the stages of bits 12.. (reading the samples from y where the table
      // allows), then bits 0-11 per segment of 4096, then T^T
      scattered = cols_with_samples(P, v, y, nullptr, batch, 2, L);
      if (!scattered) {
        scatter();
        fwht_big<T>(v, G.L, batch, L, false);
      }
      L.pre("fwht_seg_upT_1d", e * (double)batch * (M + N));
      L.note(f32_seg_fwht_upT(P, G, v, sA, batch, L.s));
      L.check();
      done = true;
    }
  }
  if (!done) {
    scatter();
    fwht_big<T>(v, G.L, batch, L);
    L.pre("upconvT_1d", e * (double)batch * (M + N));
    k_upT<T><<<grid_for((int64_t)batch * M), 256, 0, L.s>>>(v, sA, tabs<T>(P), G, batch);
    L.check();
  }
  const int jfrom = fused1d_top<T>(P);
  const int jlow = jfrom ? jfrom : P.J0;
  T* cur = sA;               // s_(j+1) of every line at cur + b M
  // the FP32 level kernels store 16 bytes at a time into x
  const bool f32 = std::is_same<T, float>::value && ((uintptr_t)x & 15u) == 0;
  for (int j = P.R - 1; j >= jlow; --j) {
    const int n0 = 1 << j;
    T* lo = (!jfrom && j == P.J0) ? x : (cur == sA ? sB : sA);
    L.pre("ana_level_1d", e * 4.0 * batch * n0);
    if (f32 && n0 >= 4) {
      if constexpr (std::is_same<T, float>::value) L.note(f32_ana1d_level(P, G, cur, lo, x + n0, n0, batch, L.s));
    } else {
      k_ana1d_level<T><<<grid_for((int64_t)batch * n0), 256, 0, L.s>>>(cur, M, lo, M, x + n0, M, n0, tabs<T>(P), G,
                                                                         batch);
    }
    L.check();
    cur = lo;
  }
  if (jfrom) {
    const size_t sm = fused1d_smem<T>(P, jfrom);
    L.pre("ana_levels_1d", e * 2.0 * batch * (double)(1 << jfrom));
    // (the per-pair formula: windows of groups would read shared memory 8 words apart per lane)
    if (f32) {   // FP32, x 16-byte aligned (the groups store 16 bytes at a time into x)
      if constexpr (std::is_same<T, float>::value) L.note(f32_ana1d_levels(P, G, cur, x, jfrom, sm, batch, L.s));
    } else {
      set_smem<T>((const void*)k_ana1d_levels<T>, sm);
      L.note(launch_pdl(k_ana1d_levels<T>, dim3(batch), dim3(1024), sm, L.s, (const T*)cur, (int64_t)M, x, tabs<T>(P),
                        G, P.J0, jfrom, (int64_t)M));
    }
    L.check();
  }
}

// 2D (Algorithm 2 with the Mallat IDWT in front).
template <typename T>
static void fwd2d(const Plan& P, const T* x, T* y, int batch, T* work, Launcher& L) {
  const double e = sizeof(T);
  Geo G = geo_of(P);
  const int M = P.M, N = P.N, Mh = M / 2;
  const int64_t MM = (int64_t)M * M;
  T* XS = work;
  T* XS2 = XS + (size_t)batch * Mh * Mh;
  T* XT = XS2 + (size_t)batch * Mh * Mh;
  T* VT = XT + (size_t)batch * MM;
  T* V = VT + (size_t)batch * M * N;
  const bool coarse = (P.R - 1 > P.J0);
  bool moved = false;
  if (coarse) moved = launch_coarse_levels<T>(P, G, x, nullptr, XS, XS2, coarse_tx_ok(P) ? XT : nullptr, batch, true, L);
  if (!moved) {
    L.pre("transpose_in", e * 2.0 * batch * MM);
    launch_transpose<T>(x, XT, M, M, MM, MM, coarse ? XS : nullptr, (int64_t)Mh * Mh, nullptr, Mh, Mh, Mh, batch, L);
    L.check();
  }
  LineIO io{};
  io.in_stride = M; io.out_stride = N; io.lines = M; io.in_batch = MM; io.out_batch = (int64_t)M * N;
  io.seq_rows = 0; io.mode = 0; io.jlev = std::max(P.R - 1, P.J0);
  L.pre("line_fwd_dim1", e * (double)batch * (MM + (double)M * N));
  launch_line<T>(true, P, G, XT, VT, io, batch * M, L);
  L.check();
  L.pre("transpose_mid_fwd", e * 2.0 * batch * M * N);
  launch_transpose<T>(VT, V, M, N, (int64_t)M * N, (int64_t)M * N, nullptr, 0, nullptr, 0, 0, 4, batch, L);
  L.check();
  LineIO io2{};
  io2.in_stride = M; io2.lines = N; io2.in_batch = (int64_t)N * M; io2.out_batch = P.m;
  io2.seq_rows = 1; io2.mode = 1; io2.jlev = io.jlev; io2.mask = P.d_mask; io2.prefix = P.d_prefix; io2.pos = P.d_pos;
  io2.wpr = P.wpr; io2.m = P.m; io2.mask_rows = N;
  L.pre("line_fwd_dim2_gather", e * (double)batch * ((double)N * M + P.m) + 8.0 * P.words);
  launch_line<T>(true, P, G, V, y, io2, batch * N, L);
  L.check();
}

template <typename T>
static void adj2d(const Plan& P, const T* y, T* x, int batch, T* work, Launcher& L) {
  const double e = sizeof(T);
  Geo G = geo_of(P);
  const int M = P.M, N = P.N, Mh = M / 2;
  const int64_t MM = (int64_t)M * M;
  T* XS = work;
  T* XS2 = XS + (size_t)batch * Mh * Mh;
  T* XT = XS2 + (size_t)batch * Mh * Mh;
  T* QT = XT + (size_t)batch * MM;
  T* Qm = QT + (size_t)batch * M * N;
  const bool coarse = (P.R - 1 > P.J0);
  const int jl = std::max(P.R - 1, P.J0);
  LineIO io{};
  io.out_stride = M; io.lines = N; io.out_batch = (int64_t)N * M; io.seq_rows = 1; io.mode = 1; io.jlev = jl;
  io.mask = P.d_mask; io.prefix = P.d_prefix; io.pos = P.d_pos; io.wpr = P.wpr; io.m = P.m; io.mask_rows = N;
  L.pre("line_adj_dim2_scatter", e * (double)batch * ((double)N * M + P.m) + 8.0 * P.words);
  launch_line<T>(false, P, G, y, Qm, io, batch * N, L);
  L.check();
  L.pre("transpose_mid_adj", e * 2.0 * batch * M * N);
  launch_transpose<T>(Qm, QT, N, M, (int64_t)N * M, (int64_t)N * M, nullptr, 0, nullptr, 0, 0, 4, batch, L);
  L.check();
  LineIO io2{};
  io2.in_stride = N; io2.out_stride = M; io2.lines = M; io2.in_batch = (int64_t)M * N; io2.out_batch = MM;
  io2.seq_rows = 0; io2.mode = 0; io2.jlev = jl;
  L.pre("line_adj_dim1", e * (double)batch * (MM + (double)M * N));
  launch_line<T>(false, P, G, QT, XT, io2, batch * M, L);
  L.check();
  if (!coarse) {
    L.pre("transpose_out", e * 2.0 * batch * MM);
    launch_transpose<T>(XT, x, M, M, MM, MM, nullptr, (int64_t)Mh * Mh, nullptr, Mh, Mh, Mh, batch, L);
    L.check();
  } else {
    const bool tx = coarse_tx_ok(P);
    if (!tx) transpose_out<T>(P, XT, x, XS, batch, L);
    launch_coarse_levels<T>(P, G, nullptr, x, XS, XS2, tx ? XT : nullptr, batch, false, L);
  }
}

template <typename T>
static int run(const Plan& P, bool fwd, const void* in, void* out, int batch, cudaStream_t s, int* nl,
               bool split = false) {
  Launcher L;
  L.s = s;
  L.split = split;
  L.prof = P.prof;
  T* work = (T*)P.d_work;
  if (P.d == 1) {
    if (line_fits<T>(P)) {
      if (fwd) fwd1d_smem<T>(P, (const T*)in, (T*)out, batch, L);
      else adj1d_smem<T>(P, (const T*)in, (T*)out, batch, L);
    } else {
      if (fwd) fwd1d_big<T>(P, (const T*)in, (T*)out, batch, work, L);
      else adj1d_big<T>(P, (const T*)in, (T*)out, batch, work, L);
    }
  } else {
    if (!line_fits<T>(P)) {
      set_error(UW_ERR_UNSUPPORTED, "2D lines longer than one CTA's shared memory are not implemented");
      return UW_ERR_UNSUPPORTED;
    }
    if (fwd) fwd2d<T>(P, (const T*)in, (T*)out, batch, work, L);
    else adj2d<T>(P, (const T*)in, (T*)out, batch, work, L);
  }
  if (nl) *nl = L.count;
  if (L.err != cudaSuccess) {
    set_error(UW_ERR_CUDA, std::string("kernel launch failed: ") + cudaGetErrorString(L.err));
    return UW_ERR_CUDA;
  }
  return UW_OK;
}

int launch_forward(const Plan& P, int prec, const void* x, void* y, int batch, void* stream, int* nl) {
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == UW_F64) return run<double>(P, true, x, y, batch, s, nl);
  return run<float>(P, true, x, y, batch, s, nl, prec == UW_F32_SPLIT_BF16);
}

int launch_adjoint(const Plan& P, int prec, const void* y, void* x, int batch, void* stream, int* nl) {
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == UW_F64) return run<double>(P, false, y, x, batch, s, nl);
  return run<float>(P, false, y, x, batch, s, nl, prec == UW_F32_SPLIT_BF16);
}

}  // namespace uw

// ---------------------------------------------------------------------------
// Fixed scratch for uw_forward_noalloc: a file-scope device array that exists
// from the moment the library's module is loaded on a device, so the call
// needs no allocator.  Every element the 2D path reads from it is written
// earlier in the same call, so nothing in it has to start at zero.
// ---------------------------------------------------------------------------
static constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace uw {

// Unique id of the current CUDA context, 0 if it cannot be read.  The
// driver entry points come through the runtime, so the library needs no
// link against the driver library.
static unsigned long long current_context_id() {
  using GetCurrent = int (*)(void**);
  using GetId = int (*)(void*, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (GetCurrent)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (GetId)f;
    cudaGetLastError();
  });
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of g_noalloc_scratch on the current device.  It is looked up
// once per device and context: a reset of the device (cudaDeviceReset) makes
// a new context, which loads the module again at a new address, and the next
// call looks the address up again.  The first call on a device (or after a
// reset) should come before any stream capture: the lookup may load the
// library's module.
static int noalloc_scratch(void** out) {
  static std::mutex mu;
  static void* addr[128] = {};
  static unsigned long long ctx_of[128] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
    cudaGetLastError();
    set_error(UW_ERR_CUDA, "no usable current CUDA device");
    return UW_ERR_CUDA;
  }
  // make sure the primary context exists before its id is read
  cudaFree(nullptr);
  const unsigned long long ctx = current_context_id();
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev] || ctx == 0 || ctx != ctx_of[dev]) {
    void* a = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&a, g_noalloc_scratch);
    if (e != cudaSuccess || !a) {
      cudaGetLastError();
      addr[dev] = nullptr;
      set_error(UW_ERR_CUDA, std::string("cudaGetSymbolAddress of the fixed scratch failed: ") + cudaGetErrorString(e));
      return UW_ERR_CUDA;
    }
    addr[dev] = a;
    ctx_of[dev] = ctx;
  }
  *out = addr[dev];
  return UW_OK;
}

int launch_forward_noalloc(const Plan& P, int prec, const void* x, void* y, int batch, void* stream, int* nl) {
  if (P.d != 2) {
    set_error(UW_ERR_UNSUPPORTED, "uw_forward_noalloc serves 2D plans only");
    return UW_ERR_UNSUPPORTED;
  }
  if (prec != UW_F64 && prec != UW_F32) {
    set_error(UW_ERR_UNSUPPORTED, "uw_forward_noalloc supports UW_F64 and UW_F32");
    return UW_ERR_UNSUPPORTED;
  }
  const size_t e = prec == UW_F64 ? sizeof(double) : sizeof(float);
  const size_t need = e * work2d_elems(P, batch);
  if (need > kNoAllocScratchBytes) {
    set_error(UW_ERR_INVALID_ARG, "request needs " + std::to_string(need) + " bytes of scratch; the fixed scratch holds " +
                                      std::to_string(kNoAllocScratchBytes));
    return UW_ERR_INVALID_ARG;
  }
  if ((prec == UW_F64 && !line_fits<double>(P)) || (prec == UW_F32 && !line_fits<float>(P))) {
    set_error(UW_ERR_UNSUPPORTED, "2D lines longer than one CTA's shared memory are not implemented");
    return UW_ERR_UNSUPPORTED;
  }
  void* work = nullptr;
  int st = noalloc_scratch(&work);
  if (st != UW_OK) return st;
  Launcher L;
  L.s = (cudaStream_t)stream;
  L.prof = nullptr;  // the profiler's event pool may grow; keep this call free of it
  if (prec == UW_F64) fwd2d<double>(P, (const double*)x, (double*)y, batch, (double*)work, L);
  else fwd2d<float>(P, (const float*)x, (float*)y, batch, (float*)work, L);
  if (nl) *nl = L.count;
  if (L.err != cudaSuccess) {
    set_error(UW_ERR_CUDA, std::string("kernel launch failed: ") + cudaGetErrorString(L.err));
    return UW_ERR_CUDA;
  }
  return UW_OK;
}

}  // namespace uw

// ===========================================================================
// C ABI: forward / adjoint
// ===========================================================================
struct uw_plan : public uw::Plan {};

// The plan's tables, mask and workspace live on the device that was current
// when it was created; a call made with another device current would launch
// there and read them across devices.  Rejected before any lookup or launch.
static int check_device(const uw_plan* P) {
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    uw::set_error(UW_ERR_CUDA, "no usable current CUDA device");
    return UW_ERR_CUDA;
  }
  if (cur != P->device) {
    uw::set_error(UW_ERR_INVALID_ARG, "the current CUDA device (" + std::to_string(cur) +
                                          ") is not the plan's device (" + std::to_string(P->device) + ")");
    return UW_ERR_INVALID_ARG;
  }
  return UW_OK;
}

// x_ptr: the coefficient side, y_ptr: the sample side (may be NULL when the
// plan samples nothing, m == 0)
static int check_call(const uw_plan* P, int prec, const void* x_ptr, const void* y_ptr, int batch) {
  if (!P) { uw::set_error(UW_ERR_INVALID_ARG, "null plan"); return UW_ERR_INVALID_ARG; }
  if (prec != UW_F64 && prec != UW_F32 && prec != UW_F32_SPLIT_BF16) {
    uw::set_error(UW_ERR_INVALID_ARG, "unknown precision");
    return UW_ERR_INVALID_ARG;
  }
  if (batch < 1 || batch > P->max_batch) {
    uw::set_error(UW_ERR_INVALID_ARG, "batch must be in 1..reserved max_batch");
    return UW_ERR_INVALID_ARG;
  }
  if (!x_ptr || (!y_ptr && P->m > 0)) { uw::set_error(UW_ERR_INVALID_ARG, "null buffer"); return UW_ERR_INVALID_ARG; }
  return check_device(P);
}

extern "C" {

int uw_plan_device_status(uw_plan* P) {
  if (!P) {
    uw::set_error(UW_ERR_INVALID_ARG, "null plan");
    return UW_ERR_INVALID_ARG;
  }
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != P->device) cudaSetDevice(P->device);
  cudaError_t e = cudaDeviceSynchronize();
  unsigned int words[4] = {0, 0, 0, 0};
  if (e == cudaSuccess && P->d_sync) e = cudaMemcpy(words, P->d_sync, sizeof words, cudaMemcpyDeviceToHost);
  int st = UW_OK;
  if (e != cudaSuccess) {
    uw::set_error(UW_ERR_CUDA, std::string("device status: ") + cudaGetErrorString(e));
    st = UW_ERR_CUDA;
  } else if (words[2]) {
    cudaMemset(P->d_sync, 0, sizeof words);   // a fresh barrier for the next launch
    cudaDeviceSynchronize();
    uw::set_error(UW_ERR_TIMEOUT, "a grid barrier wait gave up; results of the affected calls are invalid");
    st = UW_ERR_TIMEOUT;
  }
  if (cur != P->device) cudaSetDevice(cur);
  return st;
}

int uw_forward(const uw_plan* P, int prec, const void* x, void* y, int batch, void* stream) {
  int st = check_call(P, prec, x, y, batch);
  if (st != UW_OK) return st;
  int nl = 0;
  st = uw::launch_forward(*P, prec, x, y, batch, stream, &nl);
  const_cast<uw_plan*>(P)->last_launches = nl;
  return st;
}

int uw_adjoint(const uw_plan* P, int prec, const void* y, void* x, int batch, void* stream) {
  int st = check_call(P, prec, x, y, batch);
  if (st != UW_OK) return st;
  int nl = 0;
  st = uw::launch_adjoint(*P, prec, y, x, batch, stream, &nl);
  const_cast<uw_plan*>(P)->last_launches = nl;
  return st;
}

int uw_forward_noalloc(const uw_plan* P, int prec, const void* x, void* y, int batch, void* stream) {
  if (!P) { uw::set_error(UW_ERR_INVALID_ARG, "null plan"); return UW_ERR_INVALID_ARG; }
  if (prec != UW_F64 && prec != UW_F32 && prec != UW_F32_SPLIT_BF16) {
    uw::set_error(UW_ERR_INVALID_ARG, "unknown precision");
    return UW_ERR_INVALID_ARG;
  }
  if (batch < 1) { uw::set_error(UW_ERR_INVALID_ARG, "batch must be >= 1"); return UW_ERR_INVALID_ARG; }
  if (!x || (!y && P->m > 0)) { uw::set_error(UW_ERR_INVALID_ARG, "null buffer"); return UW_ERR_INVALID_ARG; }
  const int dst = check_device(P);
  if (dst != UW_OK) return dst;
  int nl = 0;
  int st = uw::launch_forward_noalloc(*P, prec, x, y, batch, stream, &nl);
  const_cast<uw_plan*>(P)->last_launches = nl;
  return st;
}

static int host_call(const uw_plan* P, int prec, bool fwd, const void* in, void* out, int batch, void* stream) {
  int st = fwd ? check_call(P, prec, in, out, batch) : check_call(P, prec, out, in, batch);
  if (st != UW_OK) return st;
  // slot 0 may still be in use by an asynchronous host call
  if (uw_host_wait(P) != UW_OK) return UW_ERR_CUDA;
  const size_t e = prec == UW_F64 ? sizeof(double) : sizeof(float);
  const int64_t coeffs = P->d == 1 ? (int64_t)P->M : (int64_t)P->M * P->M;
  const size_t nin = (size_t)batch * (size_t)(fwd ? coeffs : P->m);
  const size_t nout = (size_t)batch * (size_t)(fwd ? P->m : coeffs);
  // input at the start of the staging area, output at the next 256-byte
  // boundary after the largest possible input
  auto up256 = [](size_t n) { return (n + 255) & ~(size_t)255; };
  char* din = (char*)P->d_stage;
  char* dout = din + up256((size_t)batch * (size_t)(fwd ? coeffs : P->m) * sizeof(double));
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(din, in, nin * e, cudaMemcpyHostToDevice, s) != cudaSuccess) {
    uw::set_error(UW_ERR_CUDA, "host-to-device copy failed");
    return UW_ERR_CUDA;
  }
  st = fwd ? uw_forward(P, prec, din, dout, batch, stream) : uw_adjoint(P, prec, din, dout, batch, stream);
  if (st != UW_OK) return st;
  if (cudaMemcpyAsync(out, dout, nout * e, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    uw::set_error(UW_ERR_CUDA, "device-to-host copy failed");
    return UW_ERR_CUDA;
  }
  return UW_OK;
}

int uw_forward_host(const uw_plan* P, int prec, const void* x, void* y, int batch, void* stream) {
  return host_call(P, prec, true, x, y, batch, stream);
}

int uw_adjoint_host(const uw_plan* P, int prec, const void* y, void* x, int batch, void* stream) {
  return host_call(P, prec, false, y, x, batch, stream);
}

// copy streams and per-slot events of the asynchronous host calls (created once)
static int host_async_init(uw_plan* P) {
  if (P->s_up) return UW_OK;
  cudaStream_t up = nullptr, down = nullptr, cap = nullptr;
  if (cudaStreamCreateWithFlags(&up, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&down, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    if (up) cudaStreamDestroy(up);
    if (down) cudaStreamDestroy(down);
    uw::set_error(UW_ERR_OOM, "copy stream creation failed");
    return UW_ERR_OOM;
  }
  for (auto& slot : P->ev)
    for (void*& e : slot) {
      cudaEvent_t ev = nullptr;
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        uw::set_error(UW_ERR_OOM, "event creation failed");
        cudaStreamDestroy(up);
        cudaStreamDestroy(down);
        cudaStreamDestroy(cap);
        return UW_ERR_OOM;
      }
      e = ev;
    }
  P->s_up = up;
  P->s_down = down;
  P->s_cap = cap;
  return UW_OK;
}

// the UW_* switches that change which kernels a product launches or their
// parameters
static std::string launch_env() {
  static const char* const names[] = {"UW_BARRIER_SPIN_LIMIT", "UW_COARSE_GENERIC", "UW_COARSE_PER_LEVEL",
                                      "UW_COARSE_SEPARATE_TRANSPOSE", "UW_GENERIC_LINES", "UW_NO_UMMA",
                                      "UW_TC_SPIN_LIMIT", "UW_TC_THREADS"};
  std::string sig;
  for (const char* n : names) {
    const char* v = getenv(n);
    sig += v ? v : "\x01";
    sig += '\x02';
  }
  return sig;
}

// The product of an asynchronous host call on stream s.  Replayed as a CUDA
// graph captured at the first call with the same signature (a graph's
// launches are fixed: new buffers, mask, coarsest level, group membership,
// line variant or launch switches capture anew); eager while the profiler
// is on or if the capture failed.
static int host_product(uw_plan* P, int prec, bool fwd, const void* din, void* dout, int batch, int slot,
                        cudaStream_t s) {
  auto eager = [&]() {
    return fwd ? uw_forward(P, prec, din, dout, batch, s) : uw_adjoint(P, prec, din, dout, batch, s);
  };
  if (P->prof && P->prof->on) return eager();
  uw::HostGraph key;
  key.fwd = fwd; key.prec = prec; key.slot = slot; key.batch = batch; key.J0 = P->J0;
  key.line_variant = P->line_variant; key.coarse_mode = P->coarse_mode; key.grouped = P->group != nullptr;
  key.m = P->m; key.work = P->d_work; key.stage = P->d_stage; key.mask = P->d_mask; key.pos = P->d_pos;
  key.env = launch_env();
  uw::HostGraph* g = nullptr;
  for (auto& h : P->hgraphs)
    if (h.fwd == key.fwd && h.prec == key.prec && h.slot == key.slot) g = &h;
  if (!g) {
    P->hgraphs.push_back(key);
    g = &P->hgraphs.back();
  } else if (!g->same(key)) {
    if (g->exec) cudaGraphExecDestroy((cudaGraphExec_t)g->exec);
    *g = key;
  }
  if (!g->tried) {
    // capture once, on the plan's own stream
    g->tried = true;
    cudaStream_t cs = (cudaStream_t)P->s_cap;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const int st = fwd ? uw_forward(P, prec, din, dout, batch, cs) : uw_adjoint(P, prec, din, dout, batch, cs);
      const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
      if (st == UW_OK && ce == cudaSuccess && graph && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess)
        g->exec = exec;
      if (graph) cudaGraphDestroy(graph);
    }
    cudaGetLastError();   // a refused capture leaves the eager path
  }
  if (!g->exec) return eager();
  if (cudaGraphLaunch((cudaGraphExec_t)g->exec, s) != cudaSuccess) {
    uw::set_error(UW_ERR_CUDA, "graph launch failed");
    return UW_ERR_CUDA;
  }
  return UW_OK;
}

static int host_call_async(const uw_plan* Pc, int prec, bool fwd, const void* in, void* out, int batch,
                           void* stream) {
  int st = fwd ? check_call(Pc, prec, in, out, batch) : check_call(Pc, prec, out, in, batch);
  if (st != UW_OK) return st;
  uw_plan* P = const_cast<uw_plan*>(Pc);
  if ((st = host_async_init(P)) != UW_OK) return st;
  const size_t e = prec == UW_F64 ? sizeof(double) : sizeof(float);
  const int64_t coeffs = P->d == 1 ? (int64_t)P->M : (int64_t)P->M * P->M;
  const size_t nin = (size_t)batch * (size_t)(fwd ? coeffs : P->m);
  const size_t nout = (size_t)batch * (size_t)(fwd ? P->m : coeffs);
  auto up256 = [](size_t n) { return (n + 255) & ~(size_t)255; };
  const int k = P->slot;
  P->slot ^= 1;
  char* din = (char*)P->d_stage + (size_t)k * P->stage_bytes;
  char* dout = din + up256((size_t)batch * (size_t)(fwd ? coeffs : P->m) * sizeof(double));
  cudaStream_t s = (cudaStream_t)stream, up = (cudaStream_t)P->s_up, down = (cudaStream_t)P->s_down;
  cudaEvent_t ev_up = (cudaEvent_t)P->ev[k][0], ev_prod = (cudaEvent_t)P->ev[k][1],
              ev_down = (cudaEvent_t)P->ev[k][2];
  // upload once the product that last read this slot is done
  if (cudaStreamWaitEvent(up, ev_prod, 0) != cudaSuccess ||
      cudaMemcpyAsync(din, in, nin * e, cudaMemcpyHostToDevice, up) != cudaSuccess ||
      cudaEventRecord(ev_up, up) != cudaSuccess) {
    uw::set_error(UW_ERR_CUDA, "host-to-device copy failed");
    return UW_ERR_CUDA;
  }
  // the product: after the upload and after the download that last read this slot's output
  if (cudaStreamWaitEvent(s, ev_up, 0) != cudaSuccess || cudaStreamWaitEvent(s, ev_down, 0) != cudaSuccess) {
    uw::set_error(UW_ERR_CUDA, "stream wait failed");
    return UW_ERR_CUDA;
  }
  st = host_product(P, prec, fwd, din, dout, batch, k, s);
  if (st != UW_OK) return st;
  if (cudaEventRecord(ev_prod, s) != cudaSuccess || cudaStreamWaitEvent(down, ev_prod, 0) != cudaSuccess ||
      cudaMemcpyAsync(out, dout, nout * e, cudaMemcpyDeviceToHost, down) != cudaSuccess ||
      cudaEventRecord(ev_down, down) != cudaSuccess) {
    uw::set_error(UW_ERR_CUDA, "device-to-host copy failed");
    return UW_ERR_CUDA;
  }
  return UW_OK;
}

int uw_forward_host_async(const uw_plan* P, int prec, const void* x, void* y, int batch, void* stream) {
  return host_call_async(P, prec, true, x, y, batch, stream);
}

int uw_adjoint_host_async(const uw_plan* P, int prec, const void* y, void* x, int batch, void* stream) {
  return host_call_async(P, prec, false, y, x, batch, stream);
}

int uw_host_wait(const uw_plan* P) {
  if (!P) {
    uw::set_error(UW_ERR_INVALID_ARG, "null plan");
    return UW_ERR_INVALID_ARG;
  }
  // downloads run in call order on one stream, each after its product
  if (P->s_down && cudaStreamSynchronize((cudaStream_t)P->s_down) != cudaSuccess) {
    uw::set_error(UW_ERR_CUDA, "asynchronous host call failed");
    return UW_ERR_CUDA;
  }
  return UW_OK;
}

}  // extern "C"

extern "C" {

int uw_plan_profile(uw_plan* P, int enable) {
  if (!P) { uw::set_error(UW_ERR_INVALID_ARG, "null plan"); return UW_ERR_INVALID_ARG; }
  if (!enable) {
    if (P->prof) P->prof->on = false;
    return UW_OK;
  }
  if (!P->prof) P->prof = new uw::Profiler();
  P->prof->collect();
  auto& f = *P->prof;
  std::fill(f.ms.begin(), f.ms.end(), 0.0);
  std::fill(f.cnt.begin(), f.cnt.end(), 0);
  f.on = true;
  return UW_OK;
}

int uw_plan_profile_read(uw_plan* P, int i, char* name, int cap, double* total_ms, int64_t* launches,
                         double* bytes_per_launch) {
  if (!P || !P->prof) return 0;
  auto& f = *P->prof;
  f.collect();
  int n = (int)f.names.size();
  if (i < 0 || i >= n) return n;
  if (name && cap > 0) {
    size_t k = std::min((size_t)cap - 1, f.names[i].size());
    std::memcpy(name, f.names[i].data(), k);
    name[k] = 0;
  }
  if (total_ms) *total_ms = f.ms[i];
  if (launches) *launches = f.cnt[i];
  if (bytes_per_launch) *bytes_per_launch = f.bytes[i];
  return n;
}

}  // extern "C"
