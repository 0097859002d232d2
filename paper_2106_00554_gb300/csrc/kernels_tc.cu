// Split-BF16 tensor-core line operators (sm_103a) for the products with U and
// U^* (precision UW_F32_SPLIT_BF16): FP32 data in HBM; on the tensor cores
// each operand is a sum of three BF16 parts, x = x1 + x2 + x3 + O(2^-27 |x|)
// (x1 the BF16 rounding of x, x2 of x - x1, x3 of the rest), and a product
// keeps the six part products of order <= 2 (x1 y1, x1 y2, x2 y1, x1 y3,
// x2 y2, x3 y1), accumulated in FP32 by mma.sync m16n8k16: the result is as
// accurate as the FP32 CUDA-core path.
//
// Forward, one line of M coefficients -> N = 2^L natural-order Walsh values:
//   stage 1  the last synthesis level (Sec. 3.2), T (Sec. 4.1) and the
//            Walsh-Hadamard stages of bits 0-3 (Sec. 3.1) as one 16 x K block
//            matrix per 16 consecutive outputs, applied to im2col windows of
//            the coefficient line (6 MMAs per k-step);
//   stage 2  bits 4-7: the stage-1 accumulators of two adjacent n-tiles are
//            exactly the A operand of a 16 x 16 tile, multiplied by the exact
//            +-1 matrix H16 (3 MMAs, one per part);
//   stage 3  bits 8..L-1: one radix-2^(L-8) pass in shared memory (FP32);
//   then     store the line or gather the sampled sequency indices.
// Blocks next to a VMP boundary take dense FP32 matrices on CUDA cores.
// The adjoint runs the same stages transposed (Sec. 4.2).  The block matrices
// come from tc_plan.cpp.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>

#include "line_common.cuh"

namespace uw {

struct TcArgs {
  const uint32_t* Af;   // forward block matrix fragments (KS x 32 lanes x 8 words)
  const uint32_t* Aa;   // adjoint block matrix fragments (KSA x 32 x 8)
  const float* Ef;      // forward boundary matrix: 16 (EBl + EBr) rows of stride SF
  const float* Ea;      // adjoint boundary matrix: 16 (EAl + EAr) rows of stride SA
  int n0, M, N, L, per, nb, nbA;
  int W0, lw, bs, EBl, EBr, Xl;
  int W1, KSA, EAl, EAr, Wl, Q;
  int HL, HR, HLa, HRa;
  int SF, SA;
  int efs, eas;         // 1: the boundary matrix is staged in shared memory
};

// FP32 sample buffer: 8 words of padding per 32 keep the stage-2 fragment
// stores and loads free of bank conflicts and 16-byte alignment intact
__device__ __forceinline__ int pv(int k) { return k + 8 * (k >> 5); }
__host__ __device__ __forceinline__ int pvlen(int n) { return n + 8 * (n >> 5) + 8; }
// adjoint BF16 sample pairs: word w holds elements 2w, 2w+1; 4 words of
// padding per 16 spread the im2col fragment loads over the banks
__device__ __forceinline__ int pw(int w) { return w + 4 * (w >> 4); }

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// x0, x1 -> three BF16 pairs (p1, p2, p3), x0 in the lower halves: p1 the
// rounding of x, p2 of x - p1, p3 of x - p1 - p2 (both differences exact)
__device__ __forceinline__ void split3(float x0, float x1, uint32_t& p1, uint32_t& p2, uint32_t& p3) {
  uint32_t a, b, c;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;\n" : "=r"(a) : "f"(x1), "f"(x0));
  const float r0 = x0 - __uint_as_float(a << 16), r1 = x1 - __uint_as_float(a & 0xffff0000u);
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;\n" : "=r"(b) : "f"(r1), "f"(r0));
  const float s0 = r0 - __uint_as_float(b << 16), s1 = r1 - __uint_as_float(b & 0xffff0000u);
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;\n" : "=r"(c) : "f"(s1), "f"(s0));
  p1 = a;
  p2 = b;
  p3 = c;
}

// the six part products of order <= 2 of (A1 + A2 + A3)(B1 + B2 + B3): the
// three leading ones into d, the three small ones into e (two independent
// accumulation chains; the caller adds them)
__device__ __forceinline__ void mma_split(float (&d)[4], float (&e)[4], const uint32_t (&a1)[4],
                                          const uint32_t (&a2)[4], const uint32_t (&a3)[4],
                                          const uint32_t (&b)[3][2]) {
  mma_bf16(e, a3, b[0][0], b[0][1]);
  mma_bf16(d, a2, b[0][0], b[0][1]);
  mma_bf16(e, a2, b[1][0], b[1][1]);
  mma_bf16(d, a1, b[1][0], b[1][1]);
  mma_bf16(e, a1, b[2][0], b[2][1]);
  mma_bf16(d, a1, b[0][0], b[0][1]);
}

// asynchronous global -> shared copies (no register staging); completion is
// awaited with cp.async.wait_group
__device__ __forceinline__ void cp16(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc));
}
__device__ __forceinline__ void cp4(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_wait2() { asm volatile("cp.async.wait_group 2;\n" ::); }

// The mask row of line l (words and raw prefix counts, plus the next row's
// first prefix) copied asynchronously; r1 of the last row is the sample count.
__device__ __forceinline__ void issue_row(const LineIO& io, int mrow, uint32_t* smask, int* spraw, int tid, int nt) {
  const uint32_t* mk = io.mask + (int64_t)mrow * io.wpr;
  const int32_t* pf = io.prefix + (int64_t)mrow * io.wpr;
  for (int w4 = tid; w4 < io.wpr / 4; w4 += nt) {
    cp16(smask + 4 * w4, mk + 4 * w4);
    cp16(spraw + 4 * w4, pf + 4 * w4);
  }
  if (tid == 0 && mrow + 1 < io.mask_rows) cp4(spraw + io.wpr, pf + io.wpr);
}

// One dot product per boundary row: w row-major weights (stride ld, nin a
// multiple of 4), x the matching inputs; gsz threads per row, each taking
// float4 chunks part, part + gsz, ..., reduced with shuffles.  sink(o, v)
// receives row o from the first thread of its group.
template <typename XPTR, typename SINK>
__device__ __forceinline__ void row_dots(const float* w, int ld, int rows, int nin, int gsz, const XPTR& xrow,
                                         const SINK& sink, int tid, int nt) {
  const int nq = nin / 4;
  for (int ob = 0; ob < rows; ob += nt / gsz) {
    const int o = ob + tid / gsz, part = tid % gsz;
    float acc0 = 0.f, acc1 = 0.f;
    if (o < rows) {
      const float4* e = reinterpret_cast<const float4*>(w + (size_t)o * ld);
      const float4* x = reinterpret_cast<const float4*>(xrow(o));
      for (int c4 = part; c4 < nq; c4 += gsz) {
        const float4 ev = e[c4], xv = x[c4];
        acc0 = fmaf(ev.x, xv.x, acc0);
        acc1 = fmaf(ev.y, xv.y, acc1);
        acc0 = fmaf(ev.z, xv.z, acc0);
        acc1 = fmaf(ev.w, xv.w, acc1);
      }
    }
    float acc = acc0 + acc1;
    for (int off = gsz >> 1; off >= 1; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (o < rows && part == 0) sink(o, acc);
  }
}

// rows r0, r0 + 1 of H16 at column c as a BF16 pair (exact +-1)
__device__ __forceinline__ uint32_t hpair(int r0, int c) {
  const uint32_t a = (__popc(r0 & c) & 1) ? 0xBF80u : 0x3F80u;
  const uint32_t b = (__popc((r0 + 1) & c) & 1) ? 0xBF80u : 0x3F80u;
  return a | (b << 16);
}

// Walsh-Hadamard transform over bits 8..L-1 of the padded line: pencil
// `low` (< 256) holds low + 256 j, at pv(low) + 320 j
template <int R>
__device__ __forceinline__ void wht_pencil(float* sV, int low) {
  float* v = sV + pv(low);
  float a[R];
#pragma unroll
  for (int j = 0; j < R; ++j) a[j] = v[320 * j];
#pragma unroll
  for (int h = 1; h < R; h <<= 1)
#pragma unroll
    for (int j = 0; j < R; ++j)
      if (!(j & h)) {
        const float x = a[j], y = a[j + h];
        a[j] = x + y;
        a[j + h] = x - y;
      }
#pragma unroll
  for (int j = 0; j < R; ++j) v[320 * j] = a[j];
}

__device__ __forceinline__ void fwht_high(float* sV, int ng, int tid, int nt) {
  for (int low = tid; low < 256; low += nt) {
    switch (ng) {
      case 2: wht_pencil<2>(sV, low); break;
      case 4: wht_pencil<4>(sV, low); break;
      case 8: wht_pencil<8>(sV, low); break;
      case 16: wht_pencil<16>(sV, low); break;
      default: wht_pencil<32>(sV, low); break;
    }
  }
}

__device__ __forceinline__ uint32_t ld32(const uint16_t* p) { return *reinterpret_cast<const uint32_t*>(p); }

// Stages 1 and 2 of the forward operator for NG groups grp0, grp0 + gstep,
// ...: the block GEMM (6 part products per k-step, two accumulation chains
// per n-tile), the VMP boundary blocks replaced, bits 4-7 as an exact +-1
// MMA, results to the padded FP32 line.
template <int KS, int NG>
__device__ __forceinline__ void fwd_stage12(int grp0, int gstep, const uint4* sA, const uint16_t* cp0, int clen,
                                            int hoff, const TcArgs& a, int lane, int g, int t,
                                            const uint32_t (&Hb)[2][2], const float* sEdge, float* sV) {
  float c[NG][2][4], cs[NG][2][4];
#pragma unroll
  for (int gi = 0; gi < NG; ++gi)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) c[gi][j][r] = cs[gi][j][r] = 0.f;
#pragma unroll
  for (int ks = 0; ks < KS; ++ks) {
    uint32_t A1[4], A2[4], A3[4];
    {
      const uint4 u1 = sA[(ks * 32 + lane) * 3], u2 = sA[(ks * 32 + lane) * 3 + 1], u3 = sA[(ks * 32 + lane) * 3 + 2];
      A1[0] = u1.x; A1[1] = u1.y; A1[2] = u1.z; A1[3] = u1.w;
      A2[0] = u2.x; A2[1] = u2.y; A2[2] = u2.z; A2[3] = u2.w;
      A3[0] = u3.x; A3[1] = u3.y; A3[2] = u3.z; A3[3] = u3.w;
    }
#pragma unroll
    for (int gi = 0; gi < NG; ++gi)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        // window column kk = 16 ks + 2 t + 8 hh (< 2 lw = 16 KS): the lo
        // coefficients for kk < lw = 8 KS, the hi ones after
        const int grp = grp0 + gi * gstep;
        const uint16_t* Cb = cp0 + a.bs * (16 * grp + 8 * j + g) - a.W0 + a.HL + 2 * t;
        uint32_t bq[3][2];
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          constexpr int LW = 8 * KS;
          const int kk = 16 * ks + 8 * hh;
          const uint16_t* C = kk < LW ? Cb + kk : Cb + hoff + kk;
#pragma unroll
          for (int pt = 0; pt < 3; ++pt) bq[pt][hh] = ld32(C + pt * clen);
        }
        mma_split(c[gi][j], cs[gi][j], A1, A2, A3, bq);
      }
  }
#pragma unroll
  for (int gi = 0; gi < NG; ++gi) {
    const int grp = grp0 + gi * gstep;
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) c[gi][j][r] += cs[gi][j][r];
    if (!a.per) {
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int blk = 16 * grp + 8 * j + 2 * t + e;
          int o = -1;
          if (blk < a.EBl) o = 16 * blk;
          else if (blk >= a.nb - a.EBr) o = 16 * (a.EBl + blk - (a.nb - a.EBr));
          if (o >= 0) {
            c[gi][j][e] = sEdge[o + g];
            c[gi][j][2 + e] = sEdge[o + g + 8];
          }
        }
    }
    uint32_t q[3][4];
    split3(c[gi][0][0], c[gi][0][1], q[0][0], q[1][0], q[2][0]);
    split3(c[gi][0][2], c[gi][0][3], q[0][1], q[1][1], q[2][1]);
    split3(c[gi][1][0], c[gi][1][1], q[0][2], q[1][2], q[2][2]);
    split3(c[gi][1][2], c[gi][1][3], q[0][3], q[1][3], q[2][3]);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      float d[4] = {0.f, 0.f, 0.f, 0.f};
      mma_bf16(d, q[2], Hb[j][0], Hb[j][1]);
      mma_bf16(d, q[1], Hb[j][0], Hb[j][1]);
      mma_bf16(d, q[0], Hb[j][0], Hb[j][1]);
      // natural index 16 (16 grp + 8 j + 2 t + e) + g (+8) sits at
      // pv = 320 grp + 160 j + 40 t + 16 e + g (+8)
      float* v = sV + 320 * grp + 160 * j + 40 * t + g;
      v[0] = d[0];
      v[16] = d[1];
      v[8] = d[2];
      v[24] = d[3];
    }
  }
}

// ---------------------------------------------------------------------------
// forward: 256 threads, persistent over lines; the next line's coefficients
// (and mask row) are copied into shared memory while the current one runs
// ---------------------------------------------------------------------------
template <int KS, int NT>
__global__ void __launch_bounds__(NT, 512 / NT) k_tc_fwd(const float* __restrict__ in, float* __restrict__ out, TcArgs a,
                                                   LineIO io, int total) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int n0 = a.n0, N = a.N, M = a.M, ng = N >> 8;
  const int clen = a.HL + n0 + a.HR;
  const int wst = io.mode == 1 ? io.wpr + 4 : 0;     // staged mask words / prefixes per buffer
  float* sV = reinterpret_cast<float*>(smem_raw);
  uint4* sA = reinterpret_cast<uint4*>(sV + pvlen(N));            // KS x 32 lanes x 3 parts
  // three staging buffers: the lines two and one ahead are in flight while
  // the current one runs
  float* sIn = reinterpret_cast<float*>(sA + KS * 96);            // 3 x M staged coefficients
  float* sEdge = sIn + 3 * M;
  uint32_t* smask = reinterpret_cast<uint32_t*>(sEdge + 16 * (a.EBl + a.EBr) + 4);   // 3 x wst
  int* spraw = reinterpret_cast<int*>(smask + 3 * wst);                               // 3 x wst
  // coefficient parts: cp0[(3 * half + part) * clen + i], half 0 = lo, 1 = hi
  uint16_t* cp0 = reinterpret_cast<uint16_t*>(spraw + 3 * wst);
  // boundary matrix, staged when it fits (a.efs), else read from global memory
  const int Rf = 16 * (a.EBl + a.EBr);
  float* sEfs = reinterpret_cast<float*>(cp0 + ((6 * clen + 8 + 7) & ~7));
  const float* Ef = a.efs ? sEfs : a.Ef;
  if (a.efs)
    for (int i = tid; i < Rf * a.SF / 4; i += NT) reinterpret_cast<float4*>(sEfs)[i] = reinterpret_cast<const float4*>(a.Ef)[i];

  for (int i = tid; i < KS * 96; i += NT) sA[i] = reinterpret_cast<const uint4*>(a.Af)[i];
  uint32_t Hb[2][2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    Hb[j][0] = hpair(2 * t, g + 8 * j);
    Hb[j][1] = hpair(2 * t + 8, g + 8 * j);
  }
  // VMP halos stay zero (only boundary blocks, whose results are replaced,
  // read them)
  for (int i = tid; i < clen; i += NT)
    if (i < a.HL || i >= a.HL + n0)
      for (int c = 0; c < 6; ++c) cp0[c * clen + i] = 0;

  auto issue = [&](int ln, int bi) {
    const int l = ln % io.lines;
    const int64_t b = ln / io.lines;
    const int drow = io.seq_rows ? seqrow(l, a.L) : l;
    const float* src = in + b * io.in_batch + (int64_t)drow * io.in_stride;
    float* dst = sIn + bi * M;
    for (int e4 = tid; e4 < M / 4; e4 += NT) cp16(dst + 4 * e4, src + 4 * e4);
    if (io.mode == 1) issue_row(io, io.mask_rows == 1 ? 0 : l, smask + bi * wst, spraw + bi * wst, tid, NT);
  };
  pdl_trigger();
  pdl_wait();
  if ((int)blockIdx.x < total) issue(blockIdx.x, 0);
  cp_commit();
  if ((int)(blockIdx.x + gridDim.x) < total) issue(blockIdx.x + gridDim.x, 1);
  cp_commit();

  int buf = 0;
  for (int line = blockIdx.x; line < total; line += gridDim.x, buf = buf == 2 ? 0 : buf + 1) {
    if (line + 2 * (int)gridDim.x < total) issue(line + 2 * gridDim.x, buf == 0 ? 2 : buf - 1);
    cp_commit();
    cp_wait2();
    __syncthreads();
    const int l = line % io.lines;
    const int64_t b = line / io.lines;
    const float* xin = sIn + buf * M;
    // this line's sample positions, fetched now and used by the gather
    const uint16_t* posr = nullptr;
    uint16_t ppre[4] = {0, 0, 0, 0};
    int r0g = 0, r1g = 0;
    if (io.mode == 1) {
      const int* pr = spraw + buf * wst;
      const int mrow = io.mask_rows == 1 ? 0 : l;
      r0g = pr[0];
      r1g = mrow + 1 < io.mask_rows ? pr[io.wpr] : (int)io.m;
      if (io.pos) {
        posr = io.pos;   // positions are per plan (shared by the batch)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = r0g + tid + u * NT;
          if (j < r1g) ppre[u] = __ldg(posr + j);
        }
      }
    }
    // (1) split the staged line into BF16 parts (with periodic halos)
    for (int e4 = tid; e4 < M / 4; e4 += NT) {
      const float4 x = *reinterpret_cast<const float4*>(xin + 4 * e4);
      const int i = 4 * e4;
      const int half = i >= n0;
      const int ii = i - (half ? n0 : 0);
      uint32_t q01[3], q23[3];
      split3(x.x, x.y, q01[0], q01[1], q01[2]);
      split3(x.z, x.w, q23[0], q23[1], q23[2]);
#pragma unroll
      for (int pt = 0; pt < 3; ++pt) {
        uint16_t* C = cp0 + (3 * half + pt) * clen;
        const uint2 v = make_uint2(q01[pt], q23[pt]);
        *reinterpret_cast<uint2*>(C + a.HL + ii) = v;
        if (a.per) {
          if (ii < a.HR) *reinterpret_cast<uint2*>(C + a.HL + n0 + ii) = v;
          if (ii >= n0 - a.HL) *reinterpret_cast<uint2*>(C + ii - (n0 - a.HL)) = v;
        }
      }
    }
    // (2) VMP boundary blocks in FP32 from the staged line
    if (!a.per) {
      // row o: 16 (EBl + EBr) rows, two threads each (the lo and the hi
      // weights); the window starts at 0 (left rows) or n0 - Xl (right rows)
      const int nl = 16 * a.EBl, X4 = a.Xl;
      auto xrow = [&](int o2) {
        const int o = o2 >> 1, part = o2 & 1;
        return xin + (o < nl ? 0 : n0 - X4) + part * n0;
      };
      auto wrow = [&](int o2) { return Ef + (size_t)(o2 >> 1) * a.SF + (o2 & 1) * X4; };
      for (int ob = 0; ob < 2 * Rf; ob += NT) {
        const int o2 = ob + tid;
        float acc0 = 0.f, acc1 = 0.f;
        if (o2 < 2 * Rf) {
          const float4* e = reinterpret_cast<const float4*>(wrow(o2));
          const float4* x = reinterpret_cast<const float4*>(xrow(o2));
          for (int c4 = 0; c4 < X4 / 4; ++c4) {
            const float4 ev = e[c4], xv = x[c4];
            acc0 = fmaf(ev.x, xv.x, acc0);
            acc1 = fmaf(ev.y, xv.y, acc1);
            acc0 = fmaf(ev.z, xv.z, acc0);
            acc1 = fmaf(ev.w, xv.w, acc1);
          }
        }
        float acc = acc0 + acc1;
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        if (o2 < 2 * Rf && !(o2 & 1)) sEdge[o2 >> 1] = acc;
      }
    }
    __syncthreads();

    // (3) stages 1 and 2: groups of 16 blocks (256 outputs), NG of them per
    // warp step with their k-steps interleaved (independent MMA chains)
    const int hoff = 3 * clen - 8 * KS;   // from a lo column to the hi coefficient parts
    if (ng >= 2 * (NT / 32)) {
      for (int grp = warp; grp < ng; grp += 2 * (NT / 32))
        fwd_stage12<KS, 2>(grp, NT / 32, sA, cp0, clen, hoff, a, lane, g, t, Hb, sEdge, sV);
    } else {
      for (int grp = warp; grp < ng; grp += NT / 32)
        fwd_stage12<KS, 1>(grp, NT / 32, sA, cp0, clen, hoff, a, lane, g, t, Hb, sEdge, sV);
    }
    __syncthreads();
    // (4) bits 8..L-1
    fwht_high(sV, ng, tid, NT);
    __syncthreads();
    // (5) store the natural-order line or gather the samples
    if (io.mode == 1 && posr) {
      float* y = out + b * io.m;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = r0g + tid + u * NT;
        if (j < r1g) y[j] = sV[pv(ppre[u])];
      }
      for (int j = r0g + tid + 4 * NT; j < r1g; j += NT) y[j] = sV[pv(__ldg(posr + j))];
    } else if (io.mode == 1) {
      const uint32_t* mk = smask + buf * wst;
      const int* pr = spraw + buf * wst;
      const int mrow = io.mask_rows == 1 ? 0 : l;
      float* y = out + b * io.m;
      // half-word parallel: thread hw walks the set bits of 16 mask bits
      for (int hw = tid; hw < 2 * io.wpr; hw += NT) {
        const uint32_t wd = mk[hw >> 1];
        uint32_t bits = (hw & 1) ? wd >> 16 : wd & 0xffffu;
        int pos = pr[hw >> 1] + ((hw & 1) ? __popc(wd & 0xffffu) : 0);
        const int kb = 16 * hw;
        while (bits) {
          const int bit = __ffs(bits) - 1;
          bits &= bits - 1;
          y[pos++] = sV[pv(seqrow(kb + bit, a.L))];
        }
      }
      (void)mrow;
    } else {
      float4* dst = reinterpret_cast<float4*>(out + b * io.out_batch + (int64_t)l * io.out_stride);
      const float* v = sV + pv(4 * tid);
      for (int k4 = tid, o = 0; k4 < N / 4; k4 += NT, o += 5 * NT) dst[k4] = *reinterpret_cast<const float4*>(v + o);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// adjoint: 256 threads, persistent over lines; the next line's samples (a
// natural-order line, or the packed samples and the mask row) are copied into
// shared memory while the current one runs
// ---------------------------------------------------------------------------
template <int NT>
__global__ void __launch_bounds__(NT, 512 / NT) k_tc_adj(const float* __restrict__ in, float* __restrict__ out, TcArgs a,
                                                   LineIO io, int total) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int n0 = a.n0, N = a.N, ng = N >> 8;
  const int ulen = a.HLa + N + a.HRa;              // BF16 elements per part
  const int uwords = (pw(ulen / 2) + 4 + 3) & ~3;   // multiple of 4: later arrays stay 16-byte aligned
  const bool scat = io.mode == 1;
  const int wst = scat ? io.wpr + 4 : 0;
  const int vst = pvlen(N);
  // mode 0: two sample buffers sV[2][vst] (the staged line is transformed in
  // place); mode 1: one sV, staged packed samples sY[2][N] and mask rows
  float* sV0 = reinterpret_cast<float*>(smem_raw);
  uint4* sA = reinterpret_cast<uint4*>(sV0 + (scat ? 1 : 2) * vst);   // KSA x 32 lanes x 3 parts
  uint32_t* u0 = reinterpret_cast<uint32_t*>(sA + a.KSA * 96);        // 3 parts of uwords each
  uint32_t* smask = u0 + 3 * uwords;                                   // 2 x wst
  int* spraw = reinterpret_cast<int*>(smask + 2 * wst);                // 2 x wst
  // the packed samples of the next line and their natural positions (pairs
  // of 16-bit values per word): one buffer each, refilled after stage 2 of
  // the current line, whose scatter is then done
  float* sY = reinterpret_cast<float*>(spraw + 2 * wst);               // N (mode 1)
  const bool spos = scat && io.pos;
  const int pst = N / 2 + 4;
  uint32_t* sP = reinterpret_cast<uint32_t*>(sY + (scat ? N : 0));       // pst (when spos)
  // FP32 copies of the samples the boundary rows read (after bits 4..L-1):
  // [0, Wl) and [N - Wl, N); the boundary matrix, staged when it fits
  float* sUe = reinterpret_cast<float*>(sP + (spos ? pst : 0));
  const int Ra = 16 * (a.EAl + a.EAr);
  float* sEas = sUe + 2 * a.Wl;
  const float* Ea = a.eas ? sEas : a.Ea;
  if (a.eas)
    for (int i = tid; i < Ra * a.SA / 4; i += NT) reinterpret_cast<float4*>(sEas)[i] = reinterpret_cast<const float4*>(a.Ea)[i];

  for (int i = tid; i < a.KSA * 96; i += NT) sA[i] = reinterpret_cast<const uint4*>(a.Aa)[i];
  uint32_t Hb[2][2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    Hb[j][0] = hpair(2 * t, g + 8 * j);
    Hb[j][1] = hpair(2 * t + 8, g + 8 * j);
  }
  for (int w = tid; w < 3 * uwords; w += NT) u0[w] = 0u;   // halos (VMP) start and stay zero
  // staging: mode 0 copies the natural-order line into sV[bi]; mode 1 first
  // the mask row (issue_pre), later the packed samples (issue_y)
  auto issue_pre = [&](int ln, int bi) {
    const int l = ln % io.lines;
    const int64_t b = ln / io.lines;
    if (!scat) {
      const float* src = in + b * io.in_batch + (int64_t)l * io.in_stride;
      float* dst = sV0 + bi * vst;
      float* d0 = dst + pv(4 * tid);
      for (int k4 = tid, o = 0; k4 < N / 4; k4 += NT, o += 5 * NT) cp16(d0 + o, src + 4 * k4);
    } else {
      issue_row(io, io.mask_rows == 1 ? 0 : l, smask + bi * wst, spraw + bi * wst, tid, NT);
    }
  };
  auto row_range = [&](int ln, int& r0, int& r1) {
    const int mrow = io.mask_rows == 1 ? 0 : ln % io.lines;
    r0 = __ldg(io.prefix + (int64_t)mrow * io.wpr);
    r1 = mrow + 1 < io.mask_rows ? __ldg(io.prefix + (int64_t)(mrow + 1) * io.wpr) : (int)io.m;
  };
  auto issue_y = [&](int ln, int bi, int r0, int r1) {
    const float* y = in + (ln / io.lines) * io.m;
    (void)bi;
    for (int j = r0 + tid; j < r1; j += NT) cp4(sY + (j - r0), y + j);
    if (spos) {   // the words holding positions r0 .. r1 - 1
      const uint32_t* pw32 = reinterpret_cast<const uint32_t*>(io.pos);
      for (int w = (r0 >> 1) + tid; w < ((r1 + 1) >> 1); w += NT) cp4(sP + (w - (r0 >> 1)), pw32 + w);
    }
  };
  pdl_trigger();
  pdl_wait();
  if ((int)blockIdx.x < total) {
    issue_pre(blockIdx.x, 0);
    if (scat) {
      int r0, r1;
      row_range(blockIdx.x, r0, r1);
      issue_y(blockIdx.x, 0, r0, r1);
    }
  }
  cp_commit();
  __syncthreads();

  int buf = 0;
  for (int line = blockIdx.x; line < total; line += gridDim.x, buf ^= 1) {
    const int nxt = line + gridDim.x;
    int nr0 = 0, nr1 = 0;
    if (nxt < total) {
      issue_pre(nxt, buf ^ 1);
      if (scat) row_range(nxt, nr0, nr1);      // used after stage 2
    }
    cp_commit();
    cp_wait1();
    __syncthreads();
    const int l = line % io.lines;
    const int64_t b = line / io.lines;
    float* sV = sV0 + (scat ? 0 : buf * vst);
    // (1) mode 1: scatter the staged samples into zeros
    if (scat) {
      const uint32_t* mk = smask + buf * wst;
      const int* pr = spraw + buf * wst;
      const int mrow = io.mask_rows == 1 ? 0 : l;
      const int r0 = pr[0];
      const int r1 = mrow + 1 < io.mask_rows ? pr[io.wpr] : (int)io.m;
      for (int k4 = tid; k4 < vst / 4; k4 += NT) reinterpret_cast<float4*>(sV)[k4] = make_float4(0.f, 0.f, 0.f, 0.f);
      __syncthreads();
      const float* ys = sY;
      if (spos) {
        const uint16_t* ps = reinterpret_cast<const uint16_t*>(sP) + (r0 & 1);
        for (int j = tid; j < r1 - r0; j += NT) sV[pv(ps[j])] = ys[j];
      } else
      for (int hw = tid; hw < 2 * io.wpr; hw += NT) {
        const uint32_t wd = mk[hw >> 1];
        uint32_t bits = (hw & 1) ? wd >> 16 : wd & 0xffffu;
        int pos = pr[hw >> 1] - r0 + ((hw & 1) ? __popc(wd & 0xffffu) : 0);
        const int kb = 16 * hw;
        while (bits) {
          const int bit = __ffs(bits) - 1;
          bits &= bits - 1;
          sV[pv(seqrow(kb + bit, a.L))] = ys[pos++];
        }
      }
      (void)r1;
      __syncthreads();
    }
    // (2) bits 8..L-1 (the Hadamard stages commute)
    fwht_high(sV, ng, tid, NT);
    __syncthreads();
    // (3) bits 4-7 on the tensor cores; the result, split into BF16 parts,
    // is the im2col source of stage 1
    for (int grp = warp; grp < ng; grp += NT / 32) {
      const int k0 = 256 * grp;
      // element (row r, block n) of the group at pv(k0 + 16 n + r) =
      // 320 grp + 40 (n / 2) + 16 (n % 2) + r for n < 16, r < 16
      const float* v = sV + 320 * grp + 40 * t + g;
      uint32_t q[3][4];
      split3(v[0], v[16], q[0][0], q[1][0], q[2][0]);
      split3(v[8], v[24], q[0][1], q[1][1], q[2][1]);
      split3(v[160], v[176], q[0][2], q[1][2], q[2][2]);
      split3(v[168], v[184], q[0][3], q[1][3], q[2][3]);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        mma_bf16(d, q[2], Hb[j][0], Hb[j][1]);
        mma_bf16(d, q[1], Hb[j][0], Hb[j][1]);
        mma_bf16(d, q[0], Hb[j][0], Hb[j][1]);
        // pair rows (2i, 2i+1) across the lanes g, g^1 (lane ^ 4): the even
        // lane keeps rows (g, g+1), the odd one rows (g+7, g+8) of its partner's
        // numbering, so every store writes two adjacent elements
        const bool odd = g & 1;
        const float r0 = __shfl_xor_sync(0xffffffffu, odd ? d[0] : d[2], 4);
        const float r1 = __shfl_xor_sync(0xffffffffu, odd ? d[1] : d[3], 4);
        const int brow = odd ? g + 7 : g;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const float lo = odd ? (e ? r1 : r0) : d[e];
          const float hi = odd ? d[2 + e] : (e ? r1 : r0);
          const int kidx = k0 + 16 * (8 * j + 2 * t + e) + brow;   // even
          if (!a.per) {
            if (kidx < a.Wl) {
              sUe[kidx] = lo;
              sUe[kidx + 1] = hi;
            } else if (kidx >= N - a.Wl) {
              sUe[kidx - (N - 2 * a.Wl)] = lo;
              sUe[kidx + 1 - (N - 2 * a.Wl)] = hi;
            }
          }
          uint32_t w1, w2, w3;
          split3(lo, hi, w1, w2, w3);
          int s = pw((kidx + a.HLa) >> 1);
          u0[s] = w1;
          u0[uwords + s] = w2;
          u0[2 * uwords + s] = w3;
          if (a.per) {
            if (kidx < a.HRa) {
              s = pw((kidx + N + a.HLa) >> 1);
              u0[s] = w1;
              u0[uwords + s] = w2;
              u0[2 * uwords + s] = w3;
            }
            if (kidx >= N - a.HLa) {
              s = pw((kidx - N + a.HLa) >> 1);
              u0[s] = w1;
              u0[uwords + s] = w2;
              u0[2 * uwords + s] = w3;
            }
          }
        }
      }
    }
    __syncthreads();
    // the next line's packed samples (its row range was read above)
    if (scat && nxt < total) issue_y(nxt, buf ^ 1, nr0, nr1);
    cp_commit();
    const int drow = io.seq_rows ? seqrow(l, a.L) : l;
    float* dst = out + b * io.out_batch + (int64_t)drow * io.out_stride;
    // (4) VMP boundary blocks in FP32 (samples rebuilt from their parts)
    if (!a.per) {
      const int nl = 16 * a.EAl;
      const int q = NT / Ra, gsz = q >= 8 ? 8 : (q >= 4 ? 4 : (q >= 2 ? 2 : 1));
      auto xrow = [&](int o) { return sUe + (o < nl ? 0 : a.Wl); };
      auto sink = [&](int o, float v) {
        const bool left = o < nl;
        const int oo = left ? o : o - nl;
        const int c = (left ? 0 : a.nbA - a.EAr) + oo / 16, r = oo % 16;
        dst[r < 8 ? 8 * c + r : n0 + 8 * c + r - 8] = v;
      };
      row_dots(Ea, a.SA, Ra, a.Wl, gsz, xrow, sink, tid, NT);
    }
    // (5) stage 1: 8 lo and 8 hi outputs per block, 8 blocks per n-tile
    for (int tile = warp; tile < a.nbA / 8; tile += NT / 32) {
      float c[4] = {0.f, 0.f, 0.f, 0.f}, cs[4] = {0.f, 0.f, 0.f, 0.f};
      // window start 16 Q c - W1 + HLa = 16 Q c elements = 8 Q c words, a
      // multiple of 16 words: the padded word of 8 Q c + 8 ks + t is
      // 10 Q c + 8 ks + 4 (ks / 2) + t, and + 4 for the next 8 elements
      const uint32_t* ub = u0 + 10 * a.Q * (8 * tile + g) + t;
      for (int ks = 0; ks < a.KSA; ++ks) {
        const uint4 x1 = sA[(ks * 32 + lane) * 3], x2 = sA[(ks * 32 + lane) * 3 + 1], x3 = sA[(ks * 32 + lane) * 3 + 2];
        const uint32_t A1[4] = {x1.x, x1.y, x1.z, x1.w}, A2[4] = {x2.x, x2.y, x2.z, x2.w},
                       A3[4] = {x3.x, x3.y, x3.z, x3.w};
        const int s0 = 8 * ks + 4 * (ks >> 1), s1 = s0 + 4;
        uint32_t bq[3][2];
#pragma unroll
        for (int pt = 0; pt < 3; ++pt) {
          bq[pt][0] = ub[pt * uwords + s0];
          bq[pt][1] = ub[pt * uwords + s1];
        }
        mma_split(c, cs, A1, A2, A3, bq);
      }
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int cb = 8 * tile + 2 * t + e;
        if (a.per || (cb >= a.EAl && cb < a.nbA - a.EAr)) {
          dst[8 * cb + g] = c[e] + cs[e];
          dst[n0 + 8 * cb + g] = c[2 + e] + cs[2 + e];
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// boundary matrices up to this size are staged in shared memory
static const size_t kEdgeStage = 32 * 1024;
static size_t tc_efs_bytes(const Plan& P) { return sizeof(float) * 16 * (P.tc.EBl + P.tc.EBr) * (size_t)P.tc.SF; }
static size_t tc_eas_bytes(const Plan& P) { return sizeof(float) * 16 * (P.tc.EAl + P.tc.EAr) * (size_t)P.tc.SA; }

static TcArgs tc_args(const Plan& P) {
  const TcGeo& G = P.tc;
  const uint32_t* w = (const uint32_t*)P.d_tc;
  TcArgs a{};
  a.Af = w + G.oAf;
  a.Aa = w + G.oAa;
  a.Ef = (const float*)(w + G.oEf);
  a.Ea = (const float*)(w + G.oEa);
  a.SF = G.SF;
  a.SA = G.SA;
  a.efs = tc_efs_bytes(P) <= kEdgeStage;
  a.eas = tc_eas_bytes(P) <= kEdgeStage;
  a.n0 = P.M / 2; a.M = P.M; a.N = P.N;
  int L = 0;
  while ((1 << L) < P.N) ++L;
  a.L = L;
  a.per = P.bd == UW_BOUNDARY_PERIODIC;
  a.nb = P.N / 16; a.nbA = P.M / 16;
  a.W0 = G.W0; a.lw = G.lw; a.bs = G.bs; a.EBl = G.EBl; a.EBr = G.EBr; a.Xl = G.Xl;
  a.W1 = G.W1; a.KSA = G.KSA; a.EAl = G.EAl; a.EAr = G.EAr; a.Wl = G.Wl; a.Q = P.Q;
  a.HL = G.HL; a.HR = G.HR; a.HLa = G.HLa; a.HRa = G.HRa;
  return a;
}

static size_t tc_fwd_smem(const Plan& P, bool gather) {
  const TcGeo& G = P.tc;
  const size_t clen = (size_t)G.HL + P.M / 2 + G.HR;
  const size_t wst = gather ? (size_t)P.wpr + 4 : 0;
  const size_t ef = tc_efs_bytes(P) <= kEdgeStage ? tc_efs_bytes(P) : 0;
  return sizeof(float) * pvlen(P.N) + (size_t)G.KS * 96 * 16 + sizeof(float) * 3 * P.M +
         sizeof(float) * (16 * (G.EBl + G.EBr) + 4) + 3 * 2 * wst * 4 + ((6 * clen + 8 + 7) & ~(size_t)7) * 2 + ef +
         16;
}

static size_t tc_adj_smem(const Plan& P, bool scatter) {
  const TcGeo& G = P.tc;
  const int ulen = G.HLa + P.N + G.HRa;
  const size_t uwords = ((size_t)((ulen / 2) + 4 * ((ulen / 2) >> 4)) + 4 + 3) & ~(size_t)3;
  const size_t wst = scatter ? (size_t)P.wpr + 4 : 0;
  const size_t ea = tc_eas_bytes(P) <= kEdgeStage ? tc_eas_bytes(P) : 0;
  const size_t pstage = (scatter && P.d_pos) ? ((size_t)P.N / 2 + 4) * 4 : 0;
  return sizeof(float) * pvlen(P.N) * (scatter ? 1 : 2) + (size_t)G.KSA * 96 * 16 + 3 * uwords * 4 + 2 * 2 * wst * 4 +
         (scatter ? sizeof(float) * P.N : 0) + pstage + sizeof(float) * 2 * G.Wl + ea + 16;
}

bool tc_eligible(const Plan& P, const LineIO& io, const void* in, const void* out, bool fwd) {
  if (!P.tc.ok || !P.d_tc || io.jlev != P.R - 1) return false;
  auto al16 = [](const void* q) { return ((uintptr_t)q & 15u) == 0; };
  if (fwd) {
    if (!al16(in) || io.in_stride % 4 || io.in_batch % 4) return false;
    if (io.mode == 0 && (!al16(out) || io.out_stride % 4 || io.out_batch % 4)) return false;
    return tc_fwd_smem(P, io.mode == 1) <= 112 * 1024;
  }
  if (io.mode == 0 && (!al16(in) || io.in_stride % 4 || io.in_batch % 4)) return false;
  return tc_adj_smem(P, io.mode == 1) <= 112 * 1024;
}

template <typename K>
static int persistent_grid(K kernel, int nt, size_t smem, int total) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, nt, smem);
  return std::max(1, std::min(total, std::max(per, 1) * nsm));
}

template <int NT>
static cudaError_t tc_go(bool fwd, const Plan& P, const TcArgs& a, const float* in, float* out, const LineIO& io,
                         int total, cudaStream_t s) {
  if (fwd) {
    const size_t sm = tc_fwd_smem(P, io.mode == 1);
    auto go = [&](auto kern) {
      set_smem_limit((const void*)kern);
      return launch_pdl(kern, dim3(persistent_grid(kern, NT, sm, total)), dim3(NT), sm, s, in, out, a, io, total);
    };
    if (P.tc.KS == 1) return go(k_tc_fwd<1, NT>);
    if (P.tc.KS == 2) return go(k_tc_fwd<2, NT>);
    return go(k_tc_fwd<3, NT>);
  }
  const size_t sm = tc_adj_smem(P, io.mode == 1);
  set_smem_limit((const void*)k_tc_adj<NT>);
  return launch_pdl(k_tc_adj<NT>, dim3(persistent_grid(k_tc_adj<NT>, NT, sm, total)), dim3(NT), sm, s, in, out, a,
                    io, total);
}

cudaError_t tc_launch(bool fwd, const Plan& P, const float* in, float* out, const LineIO& io, int total,
                      cudaStream_t s) {
  const TcArgs a = tc_args(P);
  static const int nt = [] {
    const char* e = std::getenv("UW_TC_THREADS");
    return (e && std::atoi(e) == 128) ? 128 : 256;
  }();
  return nt == 256 ? tc_go<256>(fwd, P, a, in, out, io, total, s) : tc_go<128>(fwd, P, a, in, out, io, total, s);
}

}  // namespace uw
