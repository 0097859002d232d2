// Register-blocked FP32 line operators (sm_103a) for the product with U and
// U^* -- the hot kernels of the 2D path (Sec. 5, Algorithm 2) and of short 1D
// lines.  One CTA transforms one line of length N = 2^L with N/16 threads:
//
//  forward:  last-level synthesis (Sec. 3.2)  ->  v = T s (Sec. 4.1 cell
//            integrals, upsampling by Q = 2^q)  ->  natural-order FWHT
//            (Sec. 3.1)  ->  store, or gather the sampled sequency indices;
//  adjoint:  load, or scatter  ->  FWHT  ->  s = T^T v  ->  analysis.
//
// Each thread computes a run of consecutive outputs from a window held in
// registers, so one shared-memory load feeds many FMAs, and the filter taps
// are kernel parameters (constant bank) zero-padded to a compile-time length
// PM >= p, so the FMAs read them directly.  The first four Walsh-Hadamard
// stages run in registers on the 16 consecutive outputs of T (or the last
// four before T^T); the remaining stages are radix-16 shared-memory passes.
// Threads whose window touches a boundary fall back to the exact per-output
// formulas of line_common.cuh (boundary rows and blocks, periodic wrap).
#include <cuda_runtime.h>

#include <algorithm>

#include "line_common.cuh"

namespace uw {

__host__ __device__ __forceinline__ int p32(int i) { return i + (i >> 5); }
__host__ __device__ __forceinline__ int p32len(int n) { return n + (n >> 5) + 1; }

template <typename T>
struct Pad32 {
  const T* a;
  int off;
  __device__ __forceinline__ T operator[](int i) const { return a[p32(i + off)]; }
};

// Zero-padded filters as kernel parameters.
//   hp[f][d + PM/2] = h_{2d+f},  gp likewise      (d in [-PM/2, PM/2])
//   tp[f][d + PM-1] = I_q[Q d + f]                (d in [-(PM-1), PM-1])
template <int PM, int Q>
struct FastTaps {
  float hp[2][PM + 1];
  float gp[2][PM + 1];
  float tp[Q][2 * PM - 1];
};

__device__ __forceinline__ void fwht16(float (&a)[16]) {
#pragma unroll
  for (int hh = 1; hh < 16; hh <<= 1)
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (!(i & hh)) {
        float x = a[i], y = a[i + hh];
        a[i] = x + y;
        a[i + hh] = x - y;
      }
}

// remaining Walsh-Hadamard passes on bits [from, L) of a padded line
__device__ __forceinline__ void fwht_from(float* v, int L, int from, int tid, int nthr) {
  int done = from;
  while (done < L) {
    int r = min(4, L - done);
    if (r == 4) fwht_pass<float, 16>(v, L, done, tid, nthr);
    else if (r == 3) fwht_pass<float, 8>(v, L, done, tid, nthr);
    else if (r == 2) fwht_pass<float, 4>(v, L, done, tid, nthr);
    else fwht_pass<float, 2>(v, L, done, tid, nthr);
    __syncthreads();
    done += r;
  }
}

// coalesced load of a line of K * nthr floats into a p32-padded buffer: all K
// loads are issued before the first shared-memory store, so their latencies
// overlap
template <int K>
__device__ __forceinline__ void load_line(const float* __restrict__ src, float* dst, int n, int tid, int nthr) {
  float a[K];
#pragma unroll
  for (int i = 0; i < K; ++i) a[i] = __ldg(src + tid + i * nthr);
#pragma unroll
  for (int i = 0; i < K; ++i) dst[p32(tid + i * nthr)] = a[i];
}

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------
template <int PM, int Q>
__global__ void __launch_bounds__(512) k_line2_fwd(const float* __restrict__ in, float* __restrict__ out,
                                                   Tables<float> tab, Geo G, LineIO io, FastTaps<PM, Q> ft) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  SmemTables<float> st;
  const int off = stage_tables(tab, G, sm, st, tid, nthr);
  pdl_trigger();
  pdl_wait();
  float* sIn = sm + off;
  float* sS = sIn + p32len(G.M);
  float* v = sS + p32len(G.M);
  uint32_t* smask = reinterpret_cast<uint32_t*>(v + padlen(G.N));
  int* spre = reinterpret_cast<int*>(smask + io.wpr);
  const int M = G.M, N = G.N, p = G.p;
  const bool per = G.bd == UW_BOUNDARY_PERIODIC;
  const int line = blockIdx.x % io.lines;
  const int64_t b = blockIdx.x / io.lines;
  const int drow = io.seq_rows ? seqrow(line, G.L) : line;
  const float* src = in + b * io.in_batch + (int64_t)drow * io.in_stride;
  load_line<16 / Q>(src, sIn, M, tid, nthr);
  __syncthreads();

  // (a) synthesis: levels jlev .. R-2 per output (1D only), level R-1 blocked
  const int nlev = G.R - io.jlev;
  if (nlev == 0) {
    for (int k = tid; k < M; k += nthr) sS[p32(k)] = sIn[p32(k)];
  } else {
    const int g = nlev - 1;
    float* lo_buf = sIn;
    float* outb = (g & 1) ? v : sS;
    for (int j = io.jlev; j < G.R - 1; ++j) {
      const int n0 = 1 << j;
      Pad32<float> lo{lo_buf, 0}, hi{sIn, n0};
      for (int k = tid; k < 2 * n0; k += nthr) outb[p32(k)] = syn_one<float>(k, n0, lo, hi, st, G);
      __syncthreads();
      lo_buf = outb;
      outb = (outb == v) ? sS : v;
    }
    const int n0 = M / 2;
    constexpr int B = 8 / Q;  // output pairs per thread
    const int i0 = tid * B;
    // interior formula on a masked (VMP) or wrapped (periodic) window
    float wl[B + PM], wh[B + PM];
#pragma unroll
    for (int w = 0; w < B + PM; ++w) {
      int m = i0 - PM / 2 + w;
      bool ok = per || (m >= p && m <= n0 - p - 1);
      int mi = per ? (m & (n0 - 1)) : m;
      wl[w] = ok ? lo_buf[p32(mi)] : 0.f;
      wh[w] = ok ? sIn[p32(n0 + mi)] : 0.f;
    }
    float acc[2 * B];
#pragma unroll
    for (int bb = 0; bb < B; ++bb)
#pragma unroll
      for (int f = 0; f < 2; ++f) {
        float a = 0.f;
#pragma unroll
        for (int d = -PM / 2; d <= PM / 2; ++d)
          a += ft.hp[f][d + PM / 2] * wl[bb - d + PM / 2] + ft.gp[f][d + PM / 2] * wh[bb - d + PM / 2];
        acc[2 * bb + f] = a;
      }
    // boundary blocks of the VMP synthesis (Sec. 3.2)
    if (!per && (2 * i0 < G.Lb || 2 * (i0 + B) > M - G.Lb)) {
#pragma unroll
      for (int u = 0; u < 2 * B; ++u) {
        const int k = 2 * i0 + u;
        if (k < G.Lb)
          for (int mm = 0; mm < p; ++mm)
            acc[u] += st.PL[mm * G.Lb + k] * lo_buf[p32(mm)] + st.QL[mm * G.Lb + k] * sIn[p32(n0 + mm)];
        const int c = M - 1 - k;
        if (c < G.Lb)
          for (int r = 0; r < p; ++r)
            acc[u] += st.PR[r * G.Lb + c] * lo_buf[p32(n0 - 1 - r)] + st.QR[r * G.Lb + c] * sIn[p32(2 * n0 - 1 - r)];
      }
    }
#pragma unroll
    for (int u = 0; u < 2 * B; ++u) sS[p32(2 * i0 + u)] = acc[u];
  }
  __syncthreads();

  // (b) v = 2^{-R/2} T s on 16 consecutive outputs, (c) first four FWHT stages
  const float sc = exp2f(-0.5f * (float)G.R);
  {
    constexpr int BI = 16 / Q;
    const int k0 = 16 * tid;
    const int i0 = k0 / Q;
    float ws[BI + 2 * PM - 2];
#pragma unroll
    for (int w = 0; w < BI + 2 * PM - 2; ++w) {
      int m = i0 - PM + 1 + w;
      bool ok = per || (m >= p && m <= M - p - 1);
      ws[w] = ok ? sS[p32(per ? (m & (M - 1)) : m)] : 0.f;
    }
    float a[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      float acc = 0.f;
#pragma unroll
      for (int d = -(PM - 1); d <= PM - 1; ++d) acc += ft.tp[u % Q][d + PM - 1] * ws[u / Q - d + PM - 1];
      a[u] = acc;
    }
    // boundary rows of T (cell integrals of the VMP edge functions)
    if (!per && (k0 < G.ntap || k0 + 16 > N - G.ntap)) {
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int k = k0 + u;
        if (k < G.ntap)
          for (int mm = 0; mm < p; ++mm) a[u] += st.EL[mm * G.ntap + k] * sS[p32(mm)];
        const int kk = N - 1 - k;
        if (kk < G.ntap)
          for (int r = 0; r < p; ++r) a[u] += st.ER[r * G.ntap + kk] * sS[p32(M - 1 - r)];
      }
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) a[u] *= sc;
    fwht16(a);
#pragma unroll
    for (int u = 0; u < 16; ++u) v[padi(k0 + u)] = a[u];
  }
  if (io.mode == 1) {
    int64_t r0;
    int cnt;
    stage_row(io, io.mask_rows == 1 ? 0 : line, io.mask_rows, smask, spre, r0, cnt, tid, nthr);
    __syncthreads();
    fwht_from(v, G.L, 4, tid, nthr);
    // (d) gather: one sample per thread, coalesced writes of y
    float* y = out + b * io.m + r0;
    for (int j = tid; j < cnt; j += nthr) y[j] = v[padi(seqrow(sample_index(smask, spre, io.wpr, j), G.L))];
  } else {
    __syncthreads();
    fwht_from(v, G.L, 4, tid, nthr);
    float* dst = out + b * io.out_batch + (int64_t)line * io.out_stride;
    for (int k = tid; k < N; k += nthr) dst[k] = v[padi(k)];
  }
}

// ---------------------------------------------------------------------------
// adjoint
// ---------------------------------------------------------------------------
template <int PM, int Q>
__global__ void __launch_bounds__(512) k_line2_adj(const float* __restrict__ in, float* __restrict__ out,
                                                   Tables<float> tab, Geo G, LineIO io, FastTaps<PM, Q> ft) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  SmemTables<float> st;
  const int off = stage_tables(tab, G, sm, st, tid, nthr);
  pdl_trigger();
  pdl_wait();
  float* sIn = sm + off;
  float* sS = sIn + p32len(G.M);
  float* v = sS + p32len(G.M);
  uint32_t* smask = reinterpret_cast<uint32_t*>(v + padlen(G.N));
  int* spre = reinterpret_cast<int*>(smask + io.wpr);
  const int M = G.M, N = G.N, p = G.p;
  const bool per = G.bd == UW_BOUNDARY_PERIODIC;
  const int line = blockIdx.x % io.lines;
  const int64_t b = blockIdx.x / io.lines;
  if (io.mode == 0) {
    const float* src = in + b * io.in_batch + (int64_t)line * io.in_stride;
    float a[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = __ldg(src + tid + i * nthr);
#pragma unroll
    for (int i = 0; i < 16; ++i) v[padi(tid + i * nthr)] = a[i];
  } else {
    // scatter: one sample per thread, coalesced reads of y
    int64_t r0;
    int cnt;
    stage_row(io, io.mask_rows == 1 ? 0 : line, io.mask_rows, smask, spre, r0, cnt, tid, nthr);
    for (int k = tid; k < padlen(N); k += nthr) v[k] = 0.f;
    __syncthreads();
    const float* y = in + b * io.m + r0;
    for (int j = tid; j < cnt; j += nthr) v[padi(seqrow(sample_index(smask, spre, io.wpr, j), G.L))] = __ldg(y + j);
  }
  __syncthreads();
  // the Hadamard stages commute: bits 4.. in shared memory, bits 0..3 in
  // registers right before T^T
  fwht_from(v, G.L, 4, tid, nthr);
  {
    float a[16];
    const int k0 = 16 * tid;
#pragma unroll
    for (int u = 0; u < 16; ++u) a[u] = v[padi(k0 + u)];
    fwht16(a);
#pragma unroll
    for (int u = 0; u < 16; ++u) v[padi(k0 + u)] = a[u];
  }
  __syncthreads();

  // (b^T) s = 2^{-R/2} T^T v, 16/Q consecutive outputs per thread
  const float sc = exp2f(-0.5f * (float)G.R);
  {
    constexpr int BM = 16 / Q;
    constexpr int W = Q * (BM + 2 * PM - 2);
    const int m0 = tid * BM;
    const int base = Q * (m0 - PM + 1);
    float wv[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
      int k = base + w;
      bool ok = per || (k >= 0 && k < N);
      wv[w] = ok ? v[padi(per ? (k & (N - 1)) : k)] : 0.f;
    }
    float acc[BM];
#pragma unroll
    for (int bb = 0; bb < BM; ++bb) {
      float a = 0.f;
#pragma unroll
      for (int d = -(PM - 1); d <= PM - 1; ++d)
#pragma unroll
        for (int f = 0; f < Q; ++f) a += ft.tp[f][d + PM - 1] * wv[Q * (bb + d + PM - 1) + f];
      acc[bb] = a;
    }
    // VMP edge columns: the transposed boundary rows replace the interior sum
    if (!per && (m0 < p || m0 + BM > M - p)) {
#pragma unroll
      for (int bb = 0; bb < BM; ++bb) {
        const int m = m0 + bb;
        if (m < p) {
          float a = 0.f;
          for (int k = 0; k < G.ntap; ++k) a += st.EL[m * G.ntap + k] * v[padi(k)];
          acc[bb] = a;
        } else if (m >= M - p) {
          const int r = M - 1 - m;
          float a = 0.f;
          for (int kk = 0; kk < G.ntap; ++kk) a += st.ER[r * G.ntap + kk] * v[padi(N - 1 - kk)];
          acc[bb] = a;
        }
      }
    }
#pragma unroll
    for (int bb = 0; bb < BM; ++bb) sS[p32(m0 + bb)] = sc * acc[bb];
  }
  __syncthreads();

  // (a^T) analysis: level R-1 register-blocked, then R-2 .. jlev per output
  const int nlev = G.R - io.jlev;
  if (nlev == 0) {
    for (int k = tid; k < M; k += nthr) sIn[p32(k)] = sS[p32(k)];
  } else {
    const int n0 = M / 2;
    float* lo_out = (nlev == 1) ? sIn : v;
    constexpr int BA = 8 / Q;
    const int m0 = tid * BA;
    float ws[2 * (BA + PM)];
#pragma unroll
    for (int w = 0; w < 2 * (BA + PM); ++w) {
      int k = 2 * (m0 - PM / 2) + w;
      bool ok = per || (k >= 0 && k < M);
      ws[w] = ok ? sS[p32(per ? (k & (M - 1)) : k)] : 0.f;
    }
    float alo[BA], ahi[BA];
#pragma unroll
    for (int bb = 0; bb < BA; ++bb) {
      float lo = 0.f, hi = 0.f;
#pragma unroll
      for (int d = -PM / 2; d <= PM / 2; ++d)
#pragma unroll
        for (int f = 0; f < 2; ++f) {
          float x = ws[2 * (bb + d + PM / 2) + f];
          lo += ft.hp[f][d + PM / 2] * x;
          hi += ft.gp[f][d + PM / 2] * x;
        }
      alo[bb] = lo;
      ahi[bb] = hi;
    }
    // VMP boundary blocks (transposed)
    if (!per && (m0 < p || m0 + BA > n0 - p)) {
#pragma unroll
      for (int bb = 0; bb < BA; ++bb) {
        const int mm = m0 + bb;
        if (mm < p) {
          float lo = 0.f, hi = 0.f;
          for (int c = 0; c < G.Lb; ++c) {
            float x = sS[p32(c)];
            lo += st.PL[mm * G.Lb + c] * x;
            hi += st.QL[mm * G.Lb + c] * x;
          }
          alo[bb] = lo;
          ahi[bb] = hi;
        } else if (mm >= n0 - p) {
          const int r = n0 - 1 - mm;
          float lo = 0.f, hi = 0.f;
          for (int c = 0; c < G.Lb; ++c) {
            float x = sS[p32(M - 1 - c)];
            lo += st.PR[r * G.Lb + c] * x;
            hi += st.QR[r * G.Lb + c] * x;
          }
          alo[bb] = lo;
          ahi[bb] = hi;
        }
      }
    }
#pragma unroll
    for (int bb = 0; bb < BA; ++bb) {
      lo_out[p32(m0 + bb)] = alo[bb];
      sIn[p32(n0 + m0 + bb)] = ahi[bb];
    }
    __syncthreads();
    // remaining levels (1D): scratch buffers alternate v, sS; the last writes sIn
    float* cur = v;
    for (int j = G.R - 2; j >= io.jlev; --j) {
      const int h0 = 1 << j;
      float* dst = (j == io.jlev) ? sIn : ((cur == v) ? sS : v);
      Pad32<float> sc_in{cur, 0};
      for (int m = tid; m < h0; m += nthr) {
        float lo, hi;
        ana_one<float>(m, h0, sc_in, st, G, lo, hi);
        dst[p32(m)] = lo;
        sIn[p32(h0 + m)] = hi;
      }
      __syncthreads();
      cur = dst;
    }
  }
  __syncthreads();
  const int drow = io.seq_rows ? seqrow(line, G.L) : line;
  float* dst = out + b * io.out_batch + (int64_t)drow * io.out_stride;
  for (int k = tid; k < M; k += nthr) dst[k] = sIn[p32(k)];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <int PM, int Q>
static FastTaps<PM, Q> make_taps(const Plan& P) {
  FastTaps<PM, Q> t;
  std::fill(&t.hp[0][0], &t.hp[0][0] + 2 * (PM + 1), 0.f);
  std::fill(&t.gp[0][0], &t.gp[0][0] + 2 * (PM + 1), 0.f);
  std::fill(&t.tp[0][0], &t.tp[0][0] + Q * (2 * PM - 1), 0.f);
  const int p = P.p;
  for (int f = 0; f < 2; ++f)
    for (int d = -PM / 2; d <= PM / 2; ++d) {
      int l = 2 * d + f;
      if (l >= -p + 1 && l <= p) {
        t.hp[f][d + PM / 2] = (float)P.h[l + p - 1];
        t.gp[f][d + PM / 2] = (float)P.g[l + p - 1];
      }
    }
  for (int f = 0; f < Q; ++f)
    for (int d = -(PM - 1); d <= PM - 1; ++d)
      if (d >= -(p - 1) && d <= p - 1) t.tp[f][d + PM - 1] = (float)P.taps[Q * d + f + (p - 1) * Q];
  return t;
}

static size_t line2_smem(const Plan& P) {
  Geo G;
  G.p = P.p; G.ntap = P.ntap; G.Lb = P.Lb;
  return sizeof(float) * ((size_t)table_count(G) + 2 * (size_t)p32len(P.M) + (size_t)padlen(P.N)) +
         2 * sizeof(int) * (size_t)P.wpr + 16;
}

bool line2_eligible(const Plan& P) {
  return (P.Q == 2 || P.Q == 4) && P.N >= 512 && P.N <= 8192 && P.p <= 10 && line2_smem(P) <= 200 * 1024;
}

template <int PM, int Q>
static cudaError_t go(bool fwd, const Plan& P, const Geo& G, const float* in, float* out, const LineIO& io,
                      int nblocks, cudaStream_t s) {
  FastTaps<PM, Q> ft = make_taps<PM, Q>(P);
  size_t sm = line2_smem(P);
  if (fwd) {
    set_smem_limit((const void*)k_line2_fwd<PM, Q>);
    return launch_pdl(k_line2_fwd<PM, Q>, dim3(nblocks), dim3(P.N / 16), sm, s, in, out, P.t32, G, io, ft);
  } else {
    set_smem_limit((const void*)k_line2_adj<PM, Q>);
    return launch_pdl(k_line2_adj<PM, Q>, dim3(nblocks), dim3(P.N / 16), sm, s, in, out, P.t32, G, io, ft);
  }
  return cudaGetLastError();
}

cudaError_t line2_launch(bool fwd, const Plan& P, const Geo& G, const float* in, float* out, const LineIO& io,
                         int nblocks, cudaStream_t s) {
  if (P.Q == 2) {
    if (P.p <= 4) return go<4, 2>(fwd, P, G, in, out, io, nblocks, s);
    if (P.p <= 8) return go<8, 2>(fwd, P, G, in, out, io, nblocks, s);
    return go<10, 2>(fwd, P, G, in, out, io, nblocks, s);
  }
  if (P.p <= 4) return go<4, 4>(fwd, P, G, in, out, io, nblocks, s);
  if (P.p <= 8) return go<8, 4>(fwd, P, G, in, out, io, nblocks, s);
  return go<10, 4>(fwd, P, G, in, out, io, nblocks, s);
}

}  // namespace uw
