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

#include "line_common.cuh"

namespace uw {

struct TcArgs {
  const uint32_t* Af;   // forward block matrix fragments (KS x 32 lanes x 8 words)
  const uint32_t* Aa;   // adjoint block matrix fragments (KSA x 32 x 8)
  const float* Efl;     // forward boundary matrices, input-major
  const float* Efr;
  const float* Eal;     // adjoint boundary matrices, input-major
  const float* Ear;
  int n0, M, N, L, per, nb, nbA;
  int W0, lw, bs, EBl, EBr, Xl;
  int W1, KSA, EAl, EAr, Wl, Q;
  int HL, HR, HLa, HRa;
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

// the six part products of order <= 2: d += (A1 + A2 + A3)(B1 + B2 + B3)
__device__ __forceinline__ void mma_split(float (&d)[4], const uint32_t (&a1)[4], const uint32_t (&a2)[4],
                                          const uint32_t (&a3)[4], const uint32_t (&b)[3][2]) {
  mma_bf16(d, a3, b[0][0], b[0][1]);
  mma_bf16(d, a2, b[1][0], b[1][1]);
  mma_bf16(d, a1, b[2][0], b[2][1]);
  mma_bf16(d, a2, b[0][0], b[0][1]);
  mma_bf16(d, a1, b[1][0], b[1][1]);
  mma_bf16(d, a1, b[0][0], b[0][1]);
}


// rows r0, r0 + 1 of H16 at column c as a BF16 pair (exact +-1)
__device__ __forceinline__ uint32_t hpair(int r0, int c) {
  const uint32_t a = (__popc(r0 & c) & 1) ? 0xBF80u : 0x3F80u;
  const uint32_t b = (__popc((r0 + 1) & c) & 1) ? 0xBF80u : 0x3F80u;
  return a | (b << 16);
}

// Walsh-Hadamard transform over bits 8..L-1 of the padded line: thread
// `low` (< 256) owns the pencil low + 256 j
template <int R>
__device__ __forceinline__ void wht_pencil(float* sV, int low) {
  float a[R];
#pragma unroll
  for (int j = 0; j < R; ++j) a[j] = sV[pv(low + 256 * j)];
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
  for (int j = 0; j < R; ++j) sV[pv(low + 256 * j)] = a[j];
}

__device__ __forceinline__ void fwht_high(float* sV, int ng, int tid) {
  switch (ng) {
    case 2: wht_pencil<2>(sV, tid); break;
    case 4: wht_pencil<4>(sV, tid); break;
    case 8: wht_pencil<8>(sV, tid); break;
    case 16: wht_pencil<16>(sV, tid); break;
    default: wht_pencil<32>(sV, tid); break;
  }
}

__device__ __forceinline__ uint32_t ld32(const uint16_t* p) { return *reinterpret_cast<const uint32_t*>(p); }

// ---------------------------------------------------------------------------
// forward: 256 threads, persistent over lines
// ---------------------------------------------------------------------------
template <int KS>
__global__ void __launch_bounds__(256, 2) k_tc_fwd(const float* __restrict__ in, float* __restrict__ out, TcArgs a,
                                                   LineIO io, int total) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int n0 = a.n0, N = a.N, ng = N >> 8;
  const int clen = a.HL + n0 + a.HR;
  float* sV = reinterpret_cast<float*>(smem_raw);
  uint4* sA = reinterpret_cast<uint4*>(sV + pvlen(N));            // KS x 32 lanes x 3 parts
  float* sEdge = reinterpret_cast<float*>(sA + KS * 96);
  // coefficient parts: cp[3 * half + part], half 0 = lo (scaling), 1 = hi (detail)
  uint16_t* cp0 = reinterpret_cast<uint16_t*>(sEdge + 16 * (a.EBl + a.EBr) + 4);
  uint32_t* smask = reinterpret_cast<uint32_t*>(cp0 + 6 * clen + 8);
  int* spre = reinterpret_cast<int*>(smask + io.wpr);

  for (int i = tid; i < KS * 96; i += 256) sA[i] = reinterpret_cast<const uint4*>(a.Af)[i];
  uint32_t Hb[2][2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    Hb[j][0] = hpair(2 * t, g + 8 * j);
    Hb[j][1] = hpair(2 * t + 8, g + 8 * j);
  }
  // VMP halos stay zero (only boundary blocks, whose results are replaced,
  // read them)
  for (int i = tid; i < clen; i += 256)
    if (i < a.HL || i >= a.HL + n0)
      for (int c = 0; c < 6; ++c) cp0[c * clen + i] = 0;

  for (int line = blockIdx.x; line < total; line += gridDim.x) {
    const int l = line % io.lines;
    const int64_t b = line / io.lines;
    const int drow = io.seq_rows ? seqrow(l, a.L) : l;
    const float* src = in + b * io.in_batch + (int64_t)drow * io.in_stride;
    // (1) load the coefficient line, split into BF16 parts (with periodic halos)
    for (int e4 = tid; e4 < a.M / 4; e4 += 256) {
      const float4 x = __ldg(reinterpret_cast<const float4*>(src) + e4);
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
    // (2) VMP boundary blocks in FP32 from the line itself
    if (!a.per) {
      for (int o = tid; o < 16 * (a.EBl + a.EBr); o += 256) {
        const bool left = o < 16 * a.EBl;
        const int oo = left ? o : o - 16 * a.EBl, rows = 16 * (left ? a.EBl : a.EBr);
        const float* E = left ? a.Efl : a.Efr;
        const int base = left ? 0 : n0 - a.Xl;
        float acc = 0.f;
        for (int c = 0; c < 2 * a.Xl; ++c) {
          const float x = __ldg(src + (c < a.Xl ? base + c : n0 + base + c - a.Xl));
          acc = fmaf(__ldg(E + c * rows + oo), x, acc);
        }
        sEdge[o] = acc;
      }
    }
    int64_t r0 = 0;
    int cnt = 0;
    if (io.mode == 1) stage_row(io, io.mask_rows == 1 ? 0 : l, io.mask_rows, smask, spre, r0, cnt, tid, 256);
    __syncthreads();

    // (3) stages 1 and 2, one group of 16 blocks (256 outputs) per warp step
    for (int grp = warp; grp < ng; grp += 8) {
      float c[2][4];
#pragma unroll
      for (int j = 0; j < 2; ++j) c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.f;
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
        uint32_t A1[4], A2[4], A3[4];
        {
          const uint4 u1 = sA[(ks * 32 + lane) * 3], u2 = sA[(ks * 32 + lane) * 3 + 1],
                      u3 = sA[(ks * 32 + lane) * 3 + 2];
          A1[0] = u1.x; A1[1] = u1.y; A1[2] = u1.z; A1[3] = u1.w;
          A2[0] = u2.x; A2[1] = u2.y; A2[2] = u2.z; A2[3] = u2.w;
          A3[0] = u3.x; A3[1] = u3.y; A3[2] = u3.z; A3[3] = u3.w;
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int base = a.bs * (16 * grp + 8 * j + g) - a.W0 + a.HL;
          uint32_t bq[3][2];
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            const int kk0 = 16 * ks + 2 * t + 8 * hh;
            const bool ok = kk0 < 2 * a.lw;   // zero columns of the block matrix past 2 lw
            const int kk = ok ? kk0 : 0;
            const int half = kk >= a.lw;
            const uint16_t* C = cp0 + 3 * half * clen + base + (half ? kk - a.lw : kk);
#pragma unroll
            for (int pt = 0; pt < 3; ++pt) {
              const uint32_t v = ld32(C + pt * clen);
              bq[pt][hh] = ok ? v : 0u;
            }
          }
          mma_split(c[j], A1, A2, A3, bq);
        }
      }
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
              c[j][e] = sEdge[o + g];
              c[j][2 + e] = sEdge[o + g + 8];
            }
          }
      }
      uint32_t q[3][4];
      split3(c[0][0], c[0][1], q[0][0], q[1][0], q[2][0]);
      split3(c[0][2], c[0][3], q[0][1], q[1][1], q[2][1]);
      split3(c[1][0], c[1][1], q[0][2], q[1][2], q[2][2]);
      split3(c[1][2], c[1][3], q[0][3], q[1][3], q[2][3]);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        mma_bf16(d, q[2], Hb[j][0], Hb[j][1]);
        mma_bf16(d, q[1], Hb[j][0], Hb[j][1]);
        mma_bf16(d, q[0], Hb[j][0], Hb[j][1]);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int kidx = 16 * (16 * grp + 8 * j + 2 * t + e) + g;
          sV[pv(kidx)] = d[e];
          sV[pv(kidx + 8)] = d[2 + e];
        }
      }
    }
    __syncthreads();
    // (4) bits 8..L-1
    fwht_high(sV, ng, tid);
    __syncthreads();
    // (5) store the natural-order line or gather the samples
    if (io.mode == 1) {
      float* y = out + b * io.m + r0;
      for (int j = tid; j < cnt; j += 256) y[j] = sV[pv(seqrow(sample_index(smask, spre, io.wpr, j), a.L))];
    } else {
      float4* dst = reinterpret_cast<float4*>(out + b * io.out_batch + (int64_t)l * io.out_stride);
      for (int k4 = tid; k4 < N / 4; k4 += 256) dst[k4] = *reinterpret_cast<const float4*>(sV + pv(4 * k4));
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// adjoint: 256 threads, persistent over lines
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 2) k_tc_adj(const float* __restrict__ in, float* __restrict__ out, TcArgs a,
                                                   LineIO io, int total) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int n0 = a.n0, N = a.N, ng = N >> 8;
  const int ulen = a.HLa + N + a.HRa;              // BF16 elements per part
  const int uwords = pw(ulen / 2) + 4;
  float* sV = reinterpret_cast<float*>(smem_raw);
  uint4* sA = reinterpret_cast<uint4*>(sV + pvlen(N));   // KSA x 32 lanes x 3 parts
  uint32_t* u0 = reinterpret_cast<uint32_t*>(sA + a.KSA * 96);   // 3 parts of uwords each
  uint32_t* smask = u0 + 3 * uwords;
  int* spre = reinterpret_cast<int*>(smask + io.wpr);

  for (int i = tid; i < a.KSA * 96; i += 256) sA[i] = reinterpret_cast<const uint4*>(a.Aa)[i];
  uint32_t Hb[2][2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    Hb[j][0] = hpair(2 * t, g + 8 * j);
    Hb[j][1] = hpair(2 * t + 8, g + 8 * j);
  }
  for (int w = tid; w < 3 * uwords; w += 256) u0[w] = 0u;   // halos (VMP) start and stay zero
  uint16_t* u16 = reinterpret_cast<uint16_t*>(u0);
  auto uidx = [&](int e) {  // element e in [-HLa, N + HRa) -> 16-bit slot of part 0
    const int x = e + a.HLa;
    return 2 * pw(x >> 1) + (x & 1);
  };
  __syncthreads();

  for (int line = blockIdx.x; line < total; line += gridDim.x) {
    const int l = line % io.lines;
    const int64_t b = line / io.lines;
    // (1) input: natural-order samples, or scatter of the sampled indices
    if (io.mode == 0) {
      const float4* src = reinterpret_cast<const float4*>(in + b * io.in_batch + (int64_t)l * io.in_stride);
      for (int k4 = tid; k4 < N / 4; k4 += 256) *reinterpret_cast<float4*>(sV + pv(4 * k4)) = __ldg(src + k4);
    } else {
      int64_t r0;
      int cnt;
      stage_row(io, io.mask_rows == 1 ? 0 : l, io.mask_rows, smask, spre, r0, cnt, tid, 256);
      for (int k = tid; k < pvlen(N); k += 256) sV[k] = 0.f;
      __syncthreads();
      const float* y = in + b * io.m + r0;
      for (int j = tid; j < cnt; j += 256) sV[pv(seqrow(sample_index(smask, spre, io.wpr, j), a.L))] = __ldg(y + j);
    }
    __syncthreads();
    // (2) bits 8..L-1 (the Hadamard stages commute)
    fwht_high(sV, ng, tid);
    __syncthreads();
    // (3) bits 4-7 on the tensor cores; the result, split into BF16 parts,
    // is the im2col source of stage 1
    for (int grp = warp; grp < ng; grp += 8) {
      const int k0 = 256 * grp;
      uint32_t q[3][4];
      split3(sV[pv(k0 + 16 * (2 * t) + g)], sV[pv(k0 + 16 * (2 * t + 1) + g)], q[0][0], q[1][0], q[2][0]);
      split3(sV[pv(k0 + 16 * (2 * t) + g + 8)], sV[pv(k0 + 16 * (2 * t + 1) + g + 8)], q[0][1], q[1][1], q[2][1]);
      split3(sV[pv(k0 + 16 * (2 * t + 8) + g)], sV[pv(k0 + 16 * (2 * t + 9) + g)], q[0][2], q[1][2], q[2][2]);
      split3(sV[pv(k0 + 16 * (2 * t + 8) + g + 8)], sV[pv(k0 + 16 * (2 * t + 9) + g + 8)], q[0][3], q[1][3],
             q[2][3]);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        mma_bf16(d, q[2], Hb[j][0], Hb[j][1]);
        mma_bf16(d, q[1], Hb[j][0], Hb[j][1]);
        mma_bf16(d, q[0], Hb[j][0], Hb[j][1]);
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
          const int kidx = k0 + 16 * (8 * j + 2 * t + (qq & 1)) + g + (qq >> 1) * 8;
          uint32_t w1, w2, w3;
          split3(d[qq], 0.f, w1, w2, w3);
          const uint16_t v1 = (uint16_t)(w1 & 0xffffu), v2 = (uint16_t)(w2 & 0xffffu), v3 = (uint16_t)(w3 & 0xffffu);
          int s = uidx(kidx);
          u16[s] = v1;
          u16[2 * uwords + s] = v2;
          u16[4 * uwords + s] = v3;
          if (a.per) {
            if (kidx < a.HRa) {
              s = uidx(kidx + N);
              u16[s] = v1;
              u16[2 * uwords + s] = v2;
              u16[4 * uwords + s] = v3;
            }
            if (kidx >= N - a.HLa) {
              s = uidx(kidx - N);
              u16[s] = v1;
              u16[2 * uwords + s] = v2;
              u16[4 * uwords + s] = v3;
            }
          }
        }
      }
    }
    __syncthreads();
    const int drow = io.seq_rows ? seqrow(l, a.L) : l;
    float* dst = out + b * io.out_batch + (int64_t)drow * io.out_stride;
    // (4) VMP boundary blocks in FP32 (samples rebuilt from their parts)
    if (!a.per) {
      for (int o = tid; o < 16 * (a.EAl + a.EAr); o += 256) {
        const bool left = o < 16 * a.EAl;
        const int oo = left ? o : o - 16 * a.EAl, rows = 16 * (left ? a.EAl : a.EAr);
        const float* E = left ? a.Eal : a.Ear;
        const int kb = left ? 0 : N - a.Wl;
        float acc = 0.f;
        for (int kk = 0; kk < a.Wl; ++kk) {
          const int s = uidx(kb + kk);
          const float u = __uint_as_float((uint32_t)u16[s] << 16) + __uint_as_float((uint32_t)u16[2 * uwords + s] << 16) +
                          __uint_as_float((uint32_t)u16[4 * uwords + s] << 16);
          acc = fmaf(__ldg(E + kk * rows + oo), u, acc);
        }
        const int c = (left ? 0 : a.nbA - a.EAr) + oo / 16, r = oo % 16;
        dst[r < 8 ? 8 * c + r : n0 + 8 * c + r - 8] = acc;
      }
    }
    // (5) stage 1: 8 lo and 8 hi outputs per block, 8 blocks per n-tile
    for (int tile = warp; tile < a.nbA / 8; tile += 8) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      const int base = 16 * a.Q * (8 * tile + g) - a.W1 + a.HLa;   // element offset, even
      for (int ks = 0; ks < a.KSA; ++ks) {
        const uint4 x1 = sA[(ks * 32 + lane) * 3], x2 = sA[(ks * 32 + lane) * 3 + 1], x3 = sA[(ks * 32 + lane) * 3 + 2];
        const uint32_t A1[4] = {x1.x, x1.y, x1.z, x1.w}, A2[4] = {x2.x, x2.y, x2.z, x2.w},
                       A3[4] = {x3.x, x3.y, x3.z, x3.w};
        const int w0 = (base + 16 * ks + 2 * t) >> 1;
        const int s0 = pw(w0), s1 = pw(w0 + 4);
        uint32_t bq[3][2];
#pragma unroll
        for (int pt = 0; pt < 3; ++pt) {
          bq[pt][0] = u0[pt * uwords + s0];
          bq[pt][1] = u0[pt * uwords + s1];
        }
        mma_split(c, A1, A2, A3, bq);
      }
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int cb = 8 * tile + 2 * t + e;
        if (a.per || (cb >= a.EAl && cb < a.nbA - a.EAr)) {
          dst[8 * cb + g] = c[e];
          dst[n0 + 8 * cb + g] = c[2 + e];
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static TcArgs tc_args(const Plan& P) {
  const TcGeo& G = P.tc;
  const uint32_t* w = (const uint32_t*)P.d_tc;
  TcArgs a{};
  a.Af = w + G.oAf;
  a.Aa = w + G.oAa;
  a.Efl = (const float*)(w + G.oEfl);
  a.Efr = (const float*)(w + G.oEfr);
  a.Eal = (const float*)(w + G.oEal);
  a.Ear = (const float*)(w + G.oEar);
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

static size_t tc_fwd_smem(const Plan& P) {
  const TcGeo& G = P.tc;
  const size_t clen = (size_t)G.HL + P.M / 2 + G.HR;
  return sizeof(float) * pvlen(P.N) + (size_t)G.KS * 96 * 16 + sizeof(float) * (16 * (G.EBl + G.EBr) + 4) +
         6 * clen * sizeof(uint16_t) + 16 + 2 * sizeof(uint32_t) * P.wpr + 16;
}

static size_t tc_adj_smem(const Plan& P) {
  const TcGeo& G = P.tc;
  const int ulen = G.HLa + P.N + G.HRa;
  const size_t uwords = (size_t)((ulen / 2) + 4 * ((ulen / 2) >> 4)) + 4;
  return sizeof(float) * pvlen(P.N) + (size_t)G.KSA * 96 * 16 + 3 * uwords * 4 + 2 * sizeof(uint32_t) * P.wpr + 16;
}

bool tc_eligible(const Plan& P, const LineIO& io, const void* in, const void* out, bool fwd) {
  if (!P.tc.ok || !P.d_tc || io.jlev != P.R - 1) return false;
  auto al16 = [](const void* q) { return ((uintptr_t)q & 15u) == 0; };
  if (fwd) {
    if (!al16(in) || io.in_stride % 4 || io.in_batch % 4) return false;
    if (io.mode == 0 && (!al16(out) || io.out_stride % 4 || io.out_batch % 4)) return false;
    return tc_fwd_smem(P) <= 110 * 1024;
  }
  if (io.mode == 0 && (!al16(in) || io.in_stride % 4 || io.in_batch % 4)) return false;
  return tc_adj_smem(P) <= 110 * 1024;
}

template <typename K>
static int persistent_grid(K kernel, size_t smem, int total) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, 256, smem);
  return std::max(1, std::min(total, std::max(per, 1) * nsm));
}

cudaError_t tc_launch(bool fwd, const Plan& P, const float* in, float* out, const LineIO& io, int total,
                      cudaStream_t s) {
  TcArgs a = tc_args(P);
  if (fwd) {
    const size_t sm = tc_fwd_smem(P);
    switch (P.tc.KS) {
      case 1: {
        set_smem_limit((const void*)k_tc_fwd<1>);
        k_tc_fwd<1><<<persistent_grid(k_tc_fwd<1>, sm, total), 256, sm, s>>>(in, out, a, io, total);
        break;
      }
      case 2: {
        set_smem_limit((const void*)k_tc_fwd<2>);
        k_tc_fwd<2><<<persistent_grid(k_tc_fwd<2>, sm, total), 256, sm, s>>>(in, out, a, io, total);
        break;
      }
      default: {
        set_smem_limit((const void*)k_tc_fwd<3>);
        k_tc_fwd<3><<<persistent_grid(k_tc_fwd<3>, sm, total), 256, sm, s>>>(in, out, a, io, total);
        break;
      }
    }
  } else {
    const size_t sm = tc_adj_smem(P);
    set_smem_limit((const void*)k_tc_adj);
    k_tc_adj<<<persistent_grid(k_tc_adj, sm, total), 256, sm, s>>>(in, out, a, io, total);
  }
  return cudaGetLastError();
}

}  // namespace uw
