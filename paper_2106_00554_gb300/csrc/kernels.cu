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
#include <string>
#include <vector>

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
};

template <typename T>
__device__ int stage_tables(const Tables<T>& t, const Geo& G, T* base, SmemTables<T>& s, int tid, int nthr) {
  int off = 0;
  auto take = [&](T*& dst, const T* src, int n) {
    dst = base + off;
    for (int i = tid; i < n; i += nthr) dst[i] = src[i];
    off += n;
  };
  take(s.h, t.h, 2 * G.p);
  take(s.g, t.g, 2 * G.p);
  take(s.taps, t.taps, G.ntap);
  take(s.EL, t.EL, G.p * G.ntap);
  take(s.ER, t.ER, G.p * G.ntap);
  take(s.PL, t.PL, G.p * G.Lb);
  take(s.QL, t.QL, G.p * G.Lb);
  take(s.PR, t.PR, G.p * G.Lb);
  take(s.QR, t.QR, G.p * G.Lb);
  return off;
}

__host__ __device__ inline int table_count(const Geo& G) {
  return 4 * G.p + G.ntap + 2 * G.p * G.ntap + 4 * G.p * G.Lb;
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
__device__ void fwht_smem(T* v, int L, int tid, int nthr) {
  int done = 0;
  while (done < L) {
    int r = min(4, L - done);
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
};

template <typename T>
__global__ void __launch_bounds__(256) k_line_fwd(const T* __restrict__ in, T* __restrict__ out,
                                                  Tables<T> tab, Geo G, LineIO io) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  SmemTables<T> st;
  int off = stage_tables(tab, G, sm, st, tid, nthr);
  T* s0 = sm + off;
  T* s1 = s0 + G.M;
  T* v = s1 + G.M;
  const int line = blockIdx.x % io.lines;
  const int64_t b = blockIdx.x / io.lines;
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
  fwht_smem<T>(v, G.L, tid, nthr);
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

template <typename T>
__global__ void __launch_bounds__(256) k_line_adj(const T* __restrict__ in, T* __restrict__ out,
                                                  Tables<T> tab, Geo G, LineIO io) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  SmemTables<T> st;
  int off = stage_tables(tab, G, sm, st, tid, nthr);
  T* s0 = sm + off;
  T* s1 = s0 + G.M;
  T* v = s1 + G.M;
  const int line = blockIdx.x % io.lines;
  const int64_t b = blockIdx.x / io.lines;
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
  fwht_smem<T>(v, G.L, tid, nthr);
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
  return UW_OK;
}

size_t workspace_bytes(const Plan& P, int batch) {
  const size_t M = P.M, N = P.N, B = batch, e = sizeof(double);
  if (P.d == 1) {
    if (line_fits<double>(P) && line_fits<float>(P)) return 256;
    return e * B * (2 * M + N) + 256;
  }
  const size_t Mh = M / 2;
  size_t xs = 2 * B * Mh * Mh;
  size_t a = B * M * M;          // XT / X'T
  size_t vt = B * M * N;         // VT / QT
  size_t v = B * N * M;          // V / Q
  return e * (xs + a + vt + v) + 1024;
}

struct Launcher {
  cudaStream_t s;
  int count = 0;
  cudaError_t err = cudaSuccess;
  void check() {
    ++count;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess && err == cudaSuccess) err = e;
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

template <typename T>
static cudaError_t set_smem(const void* fn, size_t bytes) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

static int line_threads(int N) { return N >= 4096 ? 256 : (N >= 1024 ? 128 : 64); }

// 1D, the whole line in shared memory.
template <typename T>
static void fwd1d_smem(const Plan& P, const T* x, T* y, int batch, Launcher& L) {
  Geo G = geo_of(P);
  LineIO io{};
  io.in_stride = P.M; io.out_stride = P.N; io.lines = 1; io.in_batch = P.M; io.out_batch = P.m;
  io.seq_rows = 0; io.mode = 1; io.jlev = P.J0; io.mask = P.d_mask; io.prefix = P.d_prefix;
  io.wpr = P.wpr; io.m = P.m; io.mask_rows = 1;
  size_t sm = line_smem<T>(P);
  set_smem<T>((const void*)k_line_fwd<T>, sm);
  k_line_fwd<T><<<batch, line_threads(P.N), sm, L.s>>>(x, y, tabs<T>(P), G, io);
  L.check();
}

template <typename T>
static void adj1d_smem(const Plan& P, const T* y, T* x, int batch, Launcher& L) {
  Geo G = geo_of(P);
  LineIO io{};
  io.in_stride = P.N; io.out_stride = P.M; io.lines = 1; io.in_batch = P.m; io.out_batch = P.M;
  io.seq_rows = 0; io.mode = 1; io.jlev = P.J0; io.mask = P.d_mask; io.prefix = P.d_prefix;
  io.wpr = P.wpr; io.m = P.m; io.mask_rows = 1;
  size_t sm = line_smem<T>(P);
  set_smem<T>((const void*)k_line_adj<T>, sm);
  k_line_adj<T><<<batch, line_threads(P.N), sm, L.s>>>(y, x, tabs<T>(P), G, io);
  L.check();
}

// 1D, lines larger than shared memory: level kernels + T + two-pass FWHT.
template <typename T>
static void fwht_big(T* v, int L, int batch, Launcher& Lc) {
  int L2 = std::min(L, 12), L1 = L - L2;
  size_t sm2 = sizeof(T) * padlen(1 << L2);
  set_smem<T>((const void*)k_fwht_seg<T>, sm2);
  k_fwht_seg<T><<<(int64_t)batch << L1, 256, sm2, Lc.s>>>(v, L2);
  Lc.check();
  if (L1 > 0) {
    const int COLS = 8;
    size_t sm1 = sizeof(T) * COLS * padlen(1 << L1);
    set_smem<T>((const void*)k_fwht_cols<T, COLS>, sm1);
    k_fwht_cols<T, COLS><<<batch * ((1 << L2) / COLS), 256, sm1, Lc.s>>>(v, L1, L2);
    Lc.check();
  }
}

template <typename T>
static void fwd1d_big(const Plan& P, const T* x, T* y, int batch, T* work, Launcher& L) {
  Geo G = geo_of(P);
  const int M = P.M, N = P.N;
  T* sA = work;
  T* sB = sA + (size_t)batch * M;
  T* v = sB + (size_t)batch * M;
  cudaMemcpyAsync(sA, x, sizeof(T) * (size_t)batch * M, cudaMemcpyDeviceToDevice, L.s);
  for (int j = P.J0; j < P.R; ++j) {
    int n0 = 1 << j;
    LineGeom gi{M, 1, M, 1, 0}, go{M, 1, M, 1, 0};
    // lo from sA (synthesised so far), hi = details of x at [n0, 2n0): copied in sA
    k_syn_level<T><<<grid_for((int64_t)batch * 2 * n0), 256, 0, L.s>>>(sA, sB, n0, tabs<T>(P), G, gi, go, batch);
    L.check();
    // keep the untouched details of higher levels: copy the new prefix back
    k_copy_block<T><<<grid_for((int64_t)batch * 2 * n0), 256, 0, L.s>>>(sB, M, M, sA, M, M, 1, 2 * n0, batch);
    L.check();
  }
  k_up<T><<<grid_for((int64_t)batch * N), 256, 0, L.s>>>(sA, v, tabs<T>(P), G, batch);
  L.check();
  fwht_big<T>(v, G.L, batch, L);
  k_gather<T><<<grid_for((int64_t)batch * P.words), 256, 0, L.s>>>(v, y, P.d_mask, P.d_prefix, P.words, G.L, N, P.m, batch);
  L.check();
}

template <typename T>
static void adj1d_big(const Plan& P, const T* y, T* x, int batch, T* work, Launcher& L) {
  Geo G = geo_of(P);
  const int M = P.M, N = P.N;
  T* sA = work;
  T* sB = sA + (size_t)batch * M;
  T* v = sB + (size_t)batch * M;
  cudaMemsetAsync(v, 0, sizeof(T) * (size_t)batch * N, L.s);
  k_scatter<T><<<grid_for((int64_t)batch * P.words), 256, 0, L.s>>>(y, v, P.d_mask, P.d_prefix, P.words, G.L, N, P.m, batch);
  L.check();
  fwht_big<T>(v, G.L, batch, L);
  k_upT<T><<<grid_for((int64_t)batch * M), 256, 0, L.s>>>(v, sA, tabs<T>(P), G, batch);
  L.check();
  for (int j = P.R - 1; j >= P.J0; --j) {
    int n0 = 1 << j;
    LineGeom gi{M, 1, M, 1, 0}, go{M, 1, M, 1, 0};
    k_ana_level<T><<<grid_for((int64_t)batch * n0), 256, 0, L.s>>>(sA, sB, n0, tabs<T>(P), G, gi, go, batch);
    L.check();
    k_copy_block<T><<<grid_for((int64_t)batch * 2 * n0), 256, 0, L.s>>>(sB, M, M, sA, M, M, 1, 2 * n0, batch);
    L.check();
  }
  cudaMemcpyAsync(x, sA, sizeof(T) * (size_t)batch * M, cudaMemcpyDeviceToDevice, L.s);
}

// 2D (Algorithm 2 with the Mallat IDWT in front).
template <typename T>
static void fwd2d(const Plan& P, const T* x, T* y, int batch, T* work, Launcher& L) {
  Geo G = geo_of(P);
  const int M = P.M, N = P.N, Mh = M / 2;
  const int64_t MM = (int64_t)M * M;
  T* XS = work;
  T* XS2 = XS + (size_t)batch * Mh * Mh;
  T* XT = XS2 + (size_t)batch * Mh * Mh;
  T* VT = XT + (size_t)batch * MM;
  T* V = VT + (size_t)batch * M * N;
  const bool coarse = (P.R - 1 > P.J0);
  if (coarse) {
    k_copy_block<T><<<grid_for((int64_t)batch * Mh * Mh), 256, 0, L.s>>>(x, M, MM, XS, Mh, (int64_t)Mh * Mh, Mh, Mh, batch);
    L.check();
    for (int j = P.J0; j < P.R - 1; ++j) {
      int n0 = 1 << j, n1 = 2 * n0;
      LineGeom rows{Mh, 1, (int64_t)Mh * Mh, n1, 0};
      k_syn_level<T><<<grid_for((int64_t)batch * n1 * n1), 256, 0, L.s>>>(XS, XS2, n0, tabs<T>(P), G, rows, rows, batch);
      L.check();
      LineGeom cols{1, Mh, (int64_t)Mh * Mh, n1, 1};
      k_syn_level<T><<<grid_for((int64_t)batch * n1 * n1), 256, 0, L.s>>>(XS2, XS, n0, tabs<T>(P), G, cols, cols, batch);
      L.check();
    }
  }
  dim3 tb(32, 8);
  dim3 tg((M + 31) / 32, (M + 31) / 32, batch);
  k_transpose<T><<<tg, tb, 0, L.s>>>(x, XT, M, M, MM, MM, coarse ? XS : nullptr, (int64_t)Mh * Mh, nullptr,
                                     Mh, Mh, Mh);
  L.check();
  LineIO io{};
  io.in_stride = M; io.out_stride = N; io.lines = M; io.in_batch = MM; io.out_batch = (int64_t)M * N;
  io.seq_rows = 0; io.mode = 0; io.jlev = std::max(P.R - 1, P.J0);
  size_t sm = line_smem<T>(P);
  set_smem<T>((const void*)k_line_fwd<T>, sm);
  k_line_fwd<T><<<batch * M, line_threads(N), sm, L.s>>>(XT, VT, tabs<T>(P), G, io);
  L.check();
  dim3 tg2((N + 31) / 32, (M + 31) / 32, batch);
  k_transpose<T><<<tg2, tb, 0, L.s>>>(VT, V, M, N, (int64_t)M * N, (int64_t)M * N, nullptr, 0, nullptr, 0, 0, 1);
  L.check();
  LineIO io2{};
  io2.in_stride = M; io2.lines = N; io2.in_batch = (int64_t)N * M; io2.out_batch = P.m;
  io2.seq_rows = 1; io2.mode = 1; io2.jlev = io.jlev; io2.mask = P.d_mask; io2.prefix = P.d_prefix;
  io2.wpr = P.wpr; io2.m = P.m; io2.mask_rows = N;
  k_line_fwd<T><<<batch * N, line_threads(N), sm, L.s>>>(V, y, tabs<T>(P), G, io2);
  L.check();
}

template <typename T>
static void adj2d(const Plan& P, const T* y, T* x, int batch, T* work, Launcher& L) {
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
  size_t sm = line_smem<T>(P);
  set_smem<T>((const void*)k_line_adj<T>, sm);
  LineIO io{};
  io.out_stride = M; io.lines = N; io.out_batch = (int64_t)N * M; io.seq_rows = 1; io.mode = 1; io.jlev = jl;
  io.mask = P.d_mask; io.prefix = P.d_prefix; io.wpr = P.wpr; io.m = P.m; io.mask_rows = N;
  k_line_adj<T><<<batch * N, line_threads(N), sm, L.s>>>(y, Qm, tabs<T>(P), G, io);
  L.check();
  dim3 tb(32, 8);
  dim3 tg((M + 31) / 32, (N + 31) / 32, batch);
  k_transpose<T><<<tg, tb, 0, L.s>>>(Qm, QT, N, M, (int64_t)N * M, (int64_t)N * M, nullptr, 0, nullptr, 0, 0, 1);
  L.check();
  LineIO io2{};
  io2.in_stride = N; io2.out_stride = M; io2.lines = M; io2.in_batch = (int64_t)M * N; io2.out_batch = MM;
  io2.seq_rows = 0; io2.mode = 0; io2.jlev = jl;
  k_line_adj<T><<<batch * M, line_threads(N), sm, L.s>>>(QT, XT, tabs<T>(P), G, io2);
  L.check();
  dim3 tg2((M + 31) / 32, (M + 31) / 32, batch);
  k_transpose<T><<<tg2, tb, 0, L.s>>>(XT, x, M, M, MM, MM, nullptr, (int64_t)Mh * Mh, coarse ? XS : nullptr,
                                      Mh, Mh, Mh);
  L.check();
  if (coarse) {
    for (int j = P.R - 2; j >= P.J0; --j) {
      int n0 = 1 << j, n1 = 2 * n0;
      LineGeom cols{1, Mh, (int64_t)Mh * Mh, n1, 1};
      k_ana_level<T><<<grid_for((int64_t)batch * n1 * n0), 256, 0, L.s>>>(XS, XS2, n0, tabs<T>(P), G, cols, cols, batch);
      L.check();
      LineGeom rows{Mh, 1, (int64_t)Mh * Mh, n1, 0};
      k_ana_level<T><<<grid_for((int64_t)batch * n1 * n0), 256, 0, L.s>>>(XS2, XS, n0, tabs<T>(P), G, rows, rows, batch);
      L.check();
    }
    k_copy_block<T><<<grid_for((int64_t)batch * Mh * Mh), 256, 0, L.s>>>(XS, Mh, (int64_t)Mh * Mh, x, M, MM, Mh, Mh, batch);
    L.check();
  }
}

template <typename T>
static int run(const Plan& P, bool fwd, const void* in, void* out, int batch, cudaStream_t s, int* nl) {
  Launcher L;
  L.s = s;
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
  if (prec == UW_F32) return run<float>(P, true, x, y, batch, s, nl);
  set_error(UW_ERR_UNSUPPORTED, "split-bf16 tensor-core path is not built");
  return UW_ERR_UNSUPPORTED;
}

int launch_adjoint(const Plan& P, int prec, const void* y, void* x, int batch, void* stream, int* nl) {
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == UW_F64) return run<double>(P, false, y, x, batch, s, nl);
  if (prec == UW_F32) return run<float>(P, false, y, x, batch, s, nl);
  set_error(UW_ERR_UNSUPPORTED, "split-bf16 tensor-core path is not built");
  return UW_ERR_UNSUPPORTED;
}

}  // namespace uw

// ===========================================================================
// C ABI: forward / adjoint
// ===========================================================================
struct uw_plan : public uw::Plan {};

static int check_call(const uw_plan* P, int prec, const void* a, const void* b, int batch) {
  if (!P) { uw::set_error(UW_ERR_INVALID_ARG, "null plan"); return UW_ERR_INVALID_ARG; }
  if (prec != UW_F64 && prec != UW_F32 && prec != UW_F32_SPLIT_BF16) {
    uw::set_error(UW_ERR_INVALID_ARG, "unknown precision");
    return UW_ERR_INVALID_ARG;
  }
  if (batch < 1 || batch > P->max_batch) {
    uw::set_error(UW_ERR_INVALID_ARG, "batch must be in 1..reserved max_batch");
    return UW_ERR_INVALID_ARG;
  }
  if (!a || !b) { uw::set_error(UW_ERR_INVALID_ARG, "null buffer"); return UW_ERR_INVALID_ARG; }
  return UW_OK;
}

extern "C" {

int uw_forward(const uw_plan* P, int prec, const void* x, void* y, int batch, void* stream) {
  int st = check_call(P, prec, x, y, batch);
  if (st != UW_OK) return st;
  int nl = 0;
  st = uw::launch_forward(*P, prec, x, y, batch, stream, &nl);
  const_cast<uw_plan*>(P)->last_launches = nl;
  return st;
}

int uw_adjoint(const uw_plan* P, int prec, const void* y, void* x, int batch, void* stream) {
  int st = check_call(P, prec, y, x, batch);
  if (st != UW_OK) return st;
  int nl = 0;
  st = uw::launch_adjoint(*P, prec, y, x, batch, stream, &nl);
  const_cast<uw_plan*>(P)->last_launches = nl;
  return st;
}

static int host_call(const uw_plan* P, int prec, bool fwd, const void* in, void* out, int batch, void* stream) {
  int st = check_call(P, prec, in, out, batch);
  if (st != UW_OK) return st;
  const size_t e = prec == UW_F64 ? sizeof(double) : sizeof(float);
  const int64_t coeffs = P->d == 1 ? (int64_t)P->M : (int64_t)P->M * P->M;
  const size_t nin = (size_t)batch * (size_t)(fwd ? coeffs : P->m);
  const size_t nout = (size_t)batch * (size_t)(fwd ? P->m : coeffs);
  char* din = (char*)P->d_stage;
  char* dout = din + (size_t)batch * (size_t)coeffs * sizeof(double);
  if (!fwd) dout = din + (size_t)batch * (size_t)P->m * sizeof(double);
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

}  // extern "C"
