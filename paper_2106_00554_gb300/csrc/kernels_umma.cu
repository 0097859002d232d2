// Split-BF16 line operators on the 5th-generation tensor cores (sm_103a):
// tcgen05.mma with FP32 accumulators in tensor memory, operands in shared
// memory described by matrix descriptors, lines staged by bulk copies (the
// TMA engine's 1D form).  They serve the 2D path (Sec. 5, Algorithm 2) for
// lines of N = 4096 samples with q = 1 (M = 2048 coefficients per line).
//
// A line's outputs are 128 blocks of 32, k = 32 b + r.  Forward:
//   GEMM1  D1[b][r] = sum_j W[b][j] B1[r][j]           (M = 128, N = 32, K = 48)
//          W[b][j] = lo[8 b - 8 + j] (j < 24), hi[8 b - 32 + j] (j >= 24): the
//          window of coefficients that block b reads, never materialised --
//          consecutive rows of a K-major operand without swizzling are 16
//          bytes (8 BF16 values) apart, exactly the shift of the window per
//          block, so a descriptor over the plain coefficient array is W
//          itself.  B1 = the last synthesis level (Sec. 3.2), T (Sec. 4.1)
//          and the Walsh-Hadamard stages of bits 0-4 (Sec. 3.1) of one block:
//          all of the line's multiply-adds.
//   bits 5-11 of the Walsh-Hadamard transform (the +-1 stages across blocks)
//          as two radix-16 / radix-8 passes in shared memory, then the line is
//          stored, or gathered at the sampled sequency indices (P_Omega,
//          Sec. 1.1).
// Adjoint (Sec. 4.2): stage or scatter the natural line, the same two passes
// (H is symmetric), then Z[b][j] = sum_r D[b][r] B1[r][j] (M = 128, N = 48,
// K = 32) on the tensor cores and lo[i], hi[i] = the sum of the three entries
// of Z whose window position is i.
//
// Why the +-1 stages are not a tensor-core contraction here: an MMA of
// M = 128, K = 16 costs about 50 cycles for any N <= 64 (measured on GB300),
// a line offers N = 32, and the contraction over 128 blocks would need the
// line's 4096 values in three BF16 parts (24 KB of shared memory per line in
// flight).  Folded into GEMM1 the stages of bits 0-4 cost nothing extra.
//
// Precision: every FP32 operand of an MMA is split into three BF16 parts
// (x = x1 + x2 + x3 + O(2^-24 |x|)); B1 likewise on the host, and the six part
// products of order <= 2 are kept.  The products are exact in FP32 and
// accumulate in FP32, and the +-1 passes run in FP32: as accurate as the FP32
// CUDA-core kernels.
//
// VMP boundaries: the windows read zero beyond the coefficient range; the
// exact operator differs from that by a host-built correction that reads the
// p lo and p hi coefficients at an end and reaches only the first / last KB
// blocks (added to D1; the adjoint adds its transpose).  Periodic plans wrap
// the windows instead (halo copies), which is exact.
//
// Organisation: one persistent CTA per SM with several warpgroups; each
// warpgroup runs its own sequence of lines (its own buffers, tensor-memory
// columns and mbarriers), so that the groups' CUDA-core work overlaps the
// tensor cores and each other's MMA latency.  One thread per group issues
// its MMAs.  Every wait is bounded: when one gives up, the group records it
// in the plan's error word, drains its copies and MMAs in flight (again
// bounded), and leaves; the tensor memory is freed before the CTA exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>

#include "line_common.cuh"
#include "umma.cuh"

namespace uw {
namespace ummak {

using namespace umma;

constexpr int NB = 128;            // blocks per line
constexpr int NL = 4096;           // samples per line
constexpr int ML = 2048;           // coefficients per line
constexpr int N0 = 1024;           // lo (and hi) coefficients per line
constexpr int GF = 4;              // warpgroups per CTA, forward
constexpr int GA = 3;              // warpgroups per CTA, adjoint

// shared memory (bytes)
constexpr int HANK_LEN = 1056;                       // bf16 per window array: e in [-8, 1048)
constexpr int HANK_BYTES = HANK_LEN * 2;             // 2112
constexpr int OFF_B1 = 0;                            // 3 x 3072 (forward: B1, adjoint: B1^T)
constexpr int OFF_C = 9216;                          // corrections C'[2][KB*32][2p], KB <= 4, p <= 8
constexpr int C_MAX = 2 * 4 * 32 * 16;               // floats
constexpr int OFF_G = OFF_C + C_MAX * 4;             // per-group regions
constexpr int LINE_FLOATS = 4608;                    // a padded FP32 line: element k at opad(k)
// forward group region
constexpr int F_STAGE = 0;                           // 8192: the FP32 input line
constexpr int F_HANK = 8192;                         // 6 x 2112 (L1 H1 L2 H2 L3 H3)
constexpr int F_LINE = F_HANK + 6 * HANK_BYTES;      // padded FP32 line
constexpr int F_CORR = F_LINE + LINE_FLOATS * 4;     // 2 x up to 256 floats (two lines in flight)
constexpr int F_BYTES = (F_CORR + 2048 + 1023) / 1024 * 1024;
constexpr int F_SMEM = OFF_G + GF * F_BYTES + 1024;  // + barriers
static_assert(F_LINE % 16 == 0 && F_CORR % 16 == 0, "alignment");
// adjoint group region
constexpr int A_STAGE = 0;                           // (4096 + 4) FP32: natural line or packed samples
constexpr int A_STAGE_LEN = 4100;
constexpr int A_LINE = A_STAGE_LEN * 4;              // padded FP32 line
constexpr int A_OPS = A_LINE + LINE_FLOATS * 4;      // 3 x 8192: the A operand parts of GEMM3
constexpr int A_EDGE = A_OPS + 3 * 8192;             // warp-boundary rows of Z: 4 warps x 2 x 16 floats
constexpr int A_YE = A_EDGE + 4 * 2 * 16 * 4;        // rows of the edge blocks: up to 2 x 4 x 32 floats
constexpr int A_CO = A_YE + 256 * 4;                 // corrections of the 4p edge outputs, two lines
constexpr int A_BYTES = (A_CO + 2 * 64 * 4 + 1023) / 1024 * 1024;
constexpr int A_SMEM = OFF_G + GA * A_BYTES + 1024;
static_assert(A_LINE % 16 == 0 && A_OPS % 16 == 0 && A_EDGE % 16 == 0, "alignment");

__host__ __device__ constexpr int opad(int k) { return k + 4 * (k >> 5); }

struct Args {
  const uint16_t* ops;    // d_umma: B1 parts (forward), B1^T parts (adjoint)
  const float* corr;      // C'[2][KB*32][2p] or null
  int KB, p, per;
  int L;                  // log2 N
  unsigned* err;          // plan error word (set when a wait gives up)
  unsigned spin;          // polls per wait
};

// Everything one group keeps across its line loop.
struct GroupBars {
  uint64_t load[2];
  uint64_t mma;
  uint32_t status;        // broadcast of the polling thread's result
  uint32_t pad;
};

// one thread of the group polls; the group learns the result at the barrier
__device__ __forceinline__ bool group_wait(GroupBars& gb, uint64_t* bar, uint32_t parity, unsigned spin, int wtid,
                                           int barid) {
  if (wtid == 0) gb.status = mbar_wait(bar, parity, spin) ? 1u : 0u;
  bar_sync(barid, 128);
  return gb.status != 0;
}

// Position of a group's lines: line index, instance, sequency / natural row.
struct LineAt {
  int l;
  int64_t b;
};
__device__ __forceinline__ LineAt line_at(int line, int lines) { return LineAt{line % lines, line / lines}; }

// packed-sample range [r0, r1) of mask row mrow
__device__ __forceinline__ void sample_range(const LineIO& io, int mrow, int& r0, int& r1) {
  r0 = __ldg(io.prefix + (int64_t)mrow * io.wpr);
  r1 = mrow + 1 < io.mask_rows ? __ldg(io.prefix + (int64_t)(mrow + 1) * io.wpr) : (int)io.m;
}



// Walsh-Hadamard transform of R values in registers, natural order: the first
// stage pairs neighbours, the later ones combine aligned pairs with the
// packed FP32x2 add.
template <int R>
__device__ __forceinline__ void wht_regs(float (&a)[R]) {
#pragma unroll
  for (int i = 0; i < R; i += 2) {
    const float x = a[i], y = a[i + 1];
    a[i] = x + y;
    a[i + 1] = x - y;
  }
  const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
  for (int h = 2; h < R; h <<= 1)
#pragma unroll
    for (int i = 0; i < R; i += 2)
      if (!(i & h)) {
        const float2 x = make_float2(a[i], a[i + 1]), y = make_float2(a[i + h], a[i + h + 1]);
        const float2 s = __fadd2_rn(x, y), d = __ffma2_rn(y, m1, x);
        a[i] = s.x;
        a[i + 1] = s.y;
        a[i + h] = d.x;
        a[i + h + 1] = d.y;
      }
}

// The Walsh-Hadamard stages of bits 5-8 of k = 32 b + r (b = 16 bh + bl):
// pencils of fixed (r, bh) over bl.  Thread t takes r = t % 32 and
// bh = t / 32, t / 32 + 4; for a fixed step the 32 lanes read 32 consecutive
// words (conflict-free in the padded layout and in the plain one).
// src: element k at src[k] (plain = true) or src[opad(k)]; dst padded.
template <bool PLAIN_SRC>
__device__ __forceinline__ void pass_bits5_8(const float* src, float* dst, int wtid) {
  const int r = wtid & 31;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int bh = (wtid >> 5) + 4 * h;
    float a[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int k = 32 * (16 * bh + i) + r;
      a[i] = src[PLAIN_SRC ? k : opad(k)];
    }
    wht_regs<16>(a);
#pragma unroll
    for (int i = 0; i < 16; ++i) dst[opad(32 * (16 * bh + i) + r)] = a[i];
  }
}
// bits 9-11: pencils of fixed (r, bl) over bh, in place on a padded line
__device__ __forceinline__ void pass_bits9_11(float* line, int wtid) {
  const int r = wtid & 31;
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const int bl = (wtid >> 5) + 4 * h;
    float a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = line[opad(32 * (bl + 16 * i) + r)];
    wht_regs<8>(a);
#pragma unroll
    for (int i = 0; i < 8; ++i) line[opad(32 * (bl + 16 * i) + r)] = a[i];
  }
}

// ---------------------------------------------------------------------------
// forward: lines of M = 2048 coefficients (lo | hi) -> N = 4096 outputs.
// Each group works on two lines at a time: it splits line i and issues its
// GEMM1, then, while those MMAs run, finishes line i - 1 from the other
// tensor-memory accumulator (Walsh stages of bits 5-11, store or gather).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void fwd_split(const float* stage, uint16_t* hank, int wtid, bool per) {
  const float4* s4 = reinterpret_cast<const float4*>(stage);
  const float4 l0 = s4[2 * wtid], l1 = s4[2 * wtid + 1];
  const float4 h0 = s4[N0 / 4 + 2 * wtid], h1 = s4[N0 / 4 + 2 * wtid + 1];
  uint32_t pl[3][4], ph[3][4];
  split3x2(l0.x, l0.y, pl[0][0], pl[1][0], pl[2][0]);
  split3x2(l0.z, l0.w, pl[0][1], pl[1][1], pl[2][1]);
  split3x2(l1.x, l1.y, pl[0][2], pl[1][2], pl[2][2]);
  split3x2(l1.z, l1.w, pl[0][3], pl[1][3], pl[2][3]);
  split3x2(h0.x, h0.y, ph[0][0], ph[1][0], ph[2][0]);
  split3x2(h0.z, h0.w, ph[0][1], ph[1][1], ph[2][1]);
  split3x2(h1.x, h1.y, ph[0][2], ph[1][2], ph[2][2]);
  split3x2(h1.z, h1.w, ph[0][3], ph[1][3], ph[2][3]);
#pragma unroll
  for (int P = 0; P < 3; ++P) {
    uint16_t* L = hank + (2 * P) * HANK_LEN;
    uint16_t* H = L + HANK_LEN;
    const uint4 vl = make_uint4(pl[P][0], pl[P][1], pl[P][2], pl[P][3]);
    const uint4 vh = make_uint4(ph[P][0], ph[P][1], ph[P][2], ph[P][3]);
    *reinterpret_cast<uint4*>(L + 8 + 8 * wtid) = vl;
    *reinterpret_cast<uint4*>(H + 8 + 8 * wtid) = vh;
    if (per) {   // window positions -8..-1 and 1024..1031 wrap around
      if (wtid == 0) {
        *reinterpret_cast<uint4*>(L + 8 + N0) = vl;
        *reinterpret_cast<uint4*>(H + 8 + N0) = vh;
      }
      if (wtid == 127) {
        *reinterpret_cast<uint4*>(L) = vl;
        *reinterpret_cast<uint4*>(H) = vh;
      }
    }
  }
}

__global__ void __launch_bounds__(128 * GF, 1) k_umma_fwd(const float* __restrict__ in, float* __restrict__ out, Args a,
                                                          LineIO io, int total) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, g = tid >> 7, wtid = tid & 127, wq = wtid >> 5;
  const int barid = 1 + g;
  uint16_t* sB1 = reinterpret_cast<uint16_t*>(sm + OFF_B1);
  unsigned char* G = sm + OFF_G + g * F_BYTES;
  float* stage = reinterpret_cast<float*>(G + F_STAGE);
  uint16_t* hank = reinterpret_cast<uint16_t*>(G + F_HANK);
  float* line_s = reinterpret_cast<float*>(G + F_LINE);
  float* scorr = reinterpret_cast<float*>(G + F_CORR);   // [2][256]
  GroupBars* bars = reinterpret_cast<GroupBars*>(sm + OFF_G + GF * F_BYTES);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + GF);
  GroupBars& gb = bars[g];
  const bool gather = io.mode == 1;

  if (tid < 32) tmem_alloc(tslot, 256);
  if (tid == 0) {
    for (int k = 0; k < GF; ++k) {
      mbar_init(&bars[k].load[0], 1);
      mbar_init(&bars[k].mma, 1);
    }
    mbar_fence_init();
  }
  for (int e = tid; e < 3 * 1536 / 8; e += 128 * GF)
    reinterpret_cast<uint4*>(sB1)[e] = __ldg(reinterpret_cast<const uint4*>(a.ops) + e);
  // corrections transposed, sC[e][row]: the 32 lanes that compute 32 rows
  // read consecutive words for each column e
  float* sC = reinterpret_cast<float*>(sm + OFF_C);
  {
    const int rows = 2 * a.KB * 32, cols = 2 * a.p;
    for (int e = tid; e < rows * cols; e += 128 * GF) sC[(e % cols) * rows + e / cols] = __ldg(a.corr + e);
  }
  // window halos start zero (VMP: zero padding); periodic halos are rewritten per line
  for (int e = tid; e < GF * 6 * HANK_BYTES / 16; e += 128 * GF) {
    const int k = e / (6 * HANK_BYTES / 16), r = e % (6 * HANK_BYTES / 16);
    reinterpret_cast<uint4*>(sm + OFF_G + k * F_BYTES + F_HANK)[r] = make_uint4(0, 0, 0, 0);
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t D1 = *tslot + 64u * g;          // two accumulators of 32 columns
  const uint32_t lane_off = (uint32_t)(32 * wq) << 16;

  pdl_trigger();
  pdl_wait();

  const int step = GF * gridDim.x;
  int line = GF * blockIdx.x + g;
  bool ok = true;
  uint32_t load_pend = 0, mma_pend = 0, ph_load = 0, ph_mma = 0;

  auto issue = [&](int ln) {   // one thread: the input line, once the previous one is consumed
    const LineAt at = line_at(ln, io.lines);
    const int drow = io.seq_rows ? seqrow(at.l, a.L) : at.l;
    fence_async_smem();
    mbar_expect_tx(&gb.load[0], ML * 4);
    bulk_g2s(stage, in + at.b * io.in_batch + (int64_t)drow * io.in_stride, ML * 4, &gb.load[0]);
  };
  auto wait_mma = [&]() -> bool {
    if (!group_wait(gb, &gb.mma, ph_mma, a.spin, wtid, barid)) return false;
    ph_mma ^= 1;
    mma_pend = 0;
    return true;
  };

  if (line < total) {
    if (wtid == 0) issue(line);
    load_pend = 1;
  }
  int prev = -1;                                   // the line whose GEMM1 is in flight
  // sample range and first positions of the line in flight, loaded while its
  // MMAs run (gather)
  int nr0 = 0, nr1 = 0;
  uint16_t npp[4] = {0, 0, 0, 0};
  for (int it = 0;; ++it) {
    const bool have = line < total;
    if (have) {
      if (!group_wait(gb, &gb.load[0], ph_load, a.spin, wtid, barid)) {
        ok = false;
        break;
      }
      ph_load ^= 1;
      load_pend = 0;
      // the previous GEMM1 has finished reading the windows
      if (mma_pend && !wait_mma()) {
        ok = false;
        break;
      }
      fwd_split(stage, hank, wtid, a.per);
      // VMP: the corrections of the first / last KB blocks, one value per thread
      if (a.KB) {
        float* sc = scorr + 256 * (it & 1);
        for (int c = wtid; c < 2 * a.KB * 32; c += 128) {
          const int side = c >= a.KB * 32;
          const int rows = 2 * a.KB * 32;
          const float* C = sC + c;                   // column e at C[e * rows]
          const float* xl = stage + (side ? N0 - a.p : 0);
          float acc0 = 0.f, acc1 = 0.f;
#pragma unroll 8
          for (int e = 0; e < a.p; ++e) {
            acc0 = fmaf(C[e * rows], xl[e], acc0);
            acc1 = fmaf(C[(a.p + e) * rows], xl[N0 + e], acc1);
          }
          sc[c] = acc0 + acc1;
        }
      }
      fence_async_smem();
      bar_sync(barid, 128);
      if (wtid == 0) {
        if (line + step < total) issue(line + step);
        tc_fence_after();
        const uint32_t d = D1 + 32u * (it & 1);
        const uint32_t id1 = idesc_bf16(128, 32, 0, 0);
        const uint32_t hk = smem_u32(hank), bb = smem_u32(sB1);
        uint32_t acc = 0;
#pragma unroll
        for (int dp = 0; dp < 3; ++dp)
#pragma unroll
          for (int op = 0; op + dp < 3; ++op) {
            const uint32_t L = hk + 2 * dp * HANK_BYTES, H = L + HANK_BYTES, Bp = bb + op * 3072;
            umma_bf16(d, sdesc(L, 16, 128), sdesc(Bp, 128, 768), id1, acc);
            umma_bf16(d, sdesc(L + 32, HANK_BYTES - 32, 128), sdesc(Bp + 256, 128, 768), id1, 1);
            umma_bf16(d, sdesc(H + 16, 16, 128), sdesc(Bp + 512, 128, 768), id1, 1);
            acc = 1;
          }
        umma_commit(&gb.mma);
      }
      if (line + step < total) load_pend = 1;
      mma_pend = 1;
    }
    // this line's sample range and first positions (consumed after the next
    // line's MMAs are issued)
    int tr0 = 0, tr1 = 0;
    uint16_t tpp[4] = {0, 0, 0, 0};
    if (have && gather) {
      sample_range(io, line_at(line, io.lines).l, tr0, tr1);
      if (io.m > 0) {   // clamped to the last sample: no wait on the row's count here
#pragma unroll
        for (int k = 0; k < 4; ++k) tpp[k] = __ldg(io.pos + min((int64_t)tr0 + wtid + 128 * k, io.m - 1));
      }
    }
    // the previous line: its accumulator is complete once the GEMM1 issued
    // after it started (the waits are in order), or once its own commit is seen
    if (prev >= 0) {
      if (!have && mma_pend && !wait_mma()) {
        ok = false;
        break;
      }
      const int ps_slot = (it - 1) & 1;
      const LineAt at = line_at(prev, io.lines);
      const int r0 = nr0, r1 = nr1;
      tc_fence_after();
      {
        float y[32];
        tmem_ld32(D1 + 32u * ps_slot + lane_off, y);
        const int b = wtid;
        if (a.KB) {
          int row = -1;
          if (b < a.KB) row = b;
          else if (b >= NB - a.KB) row = a.KB + b - (NB - a.KB);
          if (row >= 0) {
            const float* sc = scorr + 256 * ps_slot + 32 * row;
#pragma unroll
            for (int r = 0; r < 32; ++r) y[r] += sc[r];
          }
        }
        float* rowp = line_s + opad(32 * b);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          *reinterpret_cast<float4*>(rowp + 4 * q) = make_float4(y[4 * q], y[4 * q + 1], y[4 * q + 2], y[4 * q + 3]);
      }
      tc_fence_before();
      bar_sync(barid, 128);
      pass_bits5_8<false>(line_s, line_s, wtid);
      bar_sync(barid, 128);
      pass_bits9_11(line_s, wtid);
      bar_sync(barid, 128);
      if (gather) {
        float* y = out + at.b * io.m + r0;
        const int cnt = r1 - r0;
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (wtid + 128 * k < cnt) y[wtid + 128 * k] = line_s[opad(npp[k])];
        for (int j = wtid + 512; j < cnt; j += 128) y[j] = line_s[opad(__ldg(io.pos + r0 + j))];
      } else {
        float* dst = out + at.b * io.out_batch + (int64_t)at.l * io.out_stride;
#pragma unroll 4
        for (int c = wtid; c < NL / 4; c += 128)
          *reinterpret_cast<float4*>(dst + 4 * c) = *reinterpret_cast<const float4*>(line_s + opad(4 * c));
      }
    }
    if (!have) break;
    prev = line;
    line += step;
    nr0 = tr0;
    nr1 = tr1;
#pragma unroll
    for (int k = 0; k < 4; ++k) npp[k] = tpp[k];
  }
  if (!ok && wtid == 0) atomicExch(a.err, 1u);
  // drain what is still in flight (bounded), then free the tensor memory
  if (wtid == 0) {
    if (load_pend) mbar_wait(&gb.load[0], ph_load, 1u << 22);
    if (mma_pend) mbar_wait(&gb.mma, ph_mma, 1u << 22);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid < 32) tmem_dealloc(*tslot, 256);
}

// ---------------------------------------------------------------------------
// adjoint: natural lines of N = 4096 (mode 0) or the sampled entries of a
// sequency row (mode 1) -> M = 2048 coefficients (lo | hi).  Each group
// prepares line i (scatter, Walsh stages of bits 5-11, split) and issues its
// MMAs, then finishes line i - 1 from the other accumulator.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128 * GA, 1) k_umma_adj(const float* __restrict__ in, float* __restrict__ out, Args a,
                                                          LineIO io, int total) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, g = tid >> 7, wtid = tid & 127, wq = wtid >> 5, lane = tid & 31;
  const int barid = 1 + g;
  uint16_t* sBt = reinterpret_cast<uint16_t*>(sm + OFF_B1);
  unsigned char* G = sm + OFF_G + g * A_BYTES;
  float* stage = reinterpret_cast<float*>(G + A_STAGE);
  float* line_s = reinterpret_cast<float*>(G + A_LINE);
  unsigned char* ops = G + A_OPS;
  float* sedge = reinterpret_cast<float*>(G + A_EDGE);
  float* sye = reinterpret_cast<float*>(G + A_YE);
  float* sco = reinterpret_cast<float*>(G + A_CO);   // [2][64]
  GroupBars* bars = reinterpret_cast<GroupBars*>(sm + OFF_G + GA * A_BYTES);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + GA);
  GroupBars& gb = bars[g];
  const bool scat = io.mode == 1;

  if (tid < 32) tmem_alloc(tslot, 512);
  if (tid == 0) {
    for (int k = 0; k < GA; ++k) {
      mbar_init(&bars[k].load[0], 1);
      mbar_init(&bars[k].mma, 1);
    }
    mbar_fence_init();
  }
  for (int e = tid; e < 3 * 1536 / 8; e += 128 * GA)
    reinterpret_cast<uint4*>(sBt)[e] = __ldg(reinterpret_cast<const uint4*>(a.ops) + 3 * 1536 / 8 + e);
  float* sC = reinterpret_cast<float*>(sm + OFF_C);
  for (int e = tid; e < 2 * a.KB * 32 * 2 * a.p; e += 128 * GA) sC[e] = __ldg(a.corr + e);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t D3 = *tslot + 128u * g;         // two accumulators of 64 columns
  const uint32_t lane_off = (uint32_t)(32 * wq) << 16;

  pdl_trigger();
  pdl_wait();

  const int step = GA * gridDim.x;
  int line = GA * blockIdx.x + g;
  bool ok = true;
  uint32_t load_pend = 0, mma_pend = 0, ph_load = 0, ph_mma = 0;

  // one thread of the group: the natural line, or the aligned span of the
  // row's packed samples (whole 16-byte units inside [r0, r1)); sample k of
  // the row lands at stage[k - (r0 & ~3)], 16-byte aligned
  auto issue = [&](int ln) {
    const LineAt at = line_at(ln, io.lines);
    fence_async_smem();
    if (!scat) {
      mbar_expect_tx(&gb.load[0], NL * 4);
      bulk_g2s(stage, in + at.b * io.in_batch + (int64_t)at.l * io.in_stride, NL * 4, &gb.load[0]);
      return;
    }
    int r0, r1;
    sample_range(io, at.l, r0, r1);
    const int a0 = (r0 + 3) & ~3, a1 = r1 & ~3;
    const uint32_t ybytes = a1 > a0 ? (uint32_t)(4 * (a1 - a0)) : 0u;
    // an arrival with nothing to copy completes the phase at once
    mbar_expect_tx(&gb.load[0], ybytes);
    if (ybytes) bulk_g2s(stage + (a0 - (r0 & ~3)), in + at.b * io.m + a0, ybytes, &gb.load[0]);
  };
  auto wait_mma = [&]() -> bool {
    if (!group_wait(gb, &gb.mma, ph_mma, a.spin, wtid, barid)) return false;
    ph_mma ^= 1;
    mma_pend = 0;
    return true;
  };

  if (line < total) {
    if (wtid == 0) issue(line);
    load_pend = 1;
  }
  // sample range and first positions of a row (scatter), loaded one line ahead
  auto row_info = [&](int ln, int& r0, int& r1, uint16_t (&pp)[4]) {
    sample_range(io, line_at(ln, io.lines).l, r0, r1);
    if (io.m > 0) {   // clamped to the last sample: no wait on the row's count here
#pragma unroll
      for (int k = 0; k < 4; ++k) pp[k] = __ldg(io.pos + min((int64_t)r0 + wtid + 128 * k, io.m - 1));
    }
  };
  int nr0 = 0, nr1 = 0;
  uint16_t npp[4] = {0, 0, 0, 0};
  if (scat && line < total) row_info(line, nr0, nr1, npp);
  int prev = -1;
  for (int it = 0;; ++it) {
    const bool have = line < total;
    if (have) {
      const LineAt at = line_at(line, io.lines);
      const int r0 = nr0, r1 = nr1;
      uint16_t pp[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) pp[k] = npp[k];
      if (scat && line + step < total) row_info(line + step, nr0, nr1, npp);
      if (!group_wait(gb, &gb.load[0], ph_load, a.spin, wtid, barid)) {
        ok = false;
        break;
      }
      ph_load ^= 1;
      load_pend = 0;
      if (scat) {
        float* st = stage + (r0 & 3);   // relative sample j at st[j]
        const float* ysrc = in + at.b * io.m;
        // the unaligned head and tail of the samples with plain loads
        const int a0 = (r0 + 3) & ~3, a1 = r1 & ~3;
        if (a1 > a0) {
          if (wtid < a0 - r0) st[wtid] = __ldg(ysrc + r0 + wtid);
          if (wtid < r1 - a1) st[a1 - r0 + wtid] = __ldg(ysrc + a1 + wtid);
        } else {
          if (wtid < r1 - r0) st[wtid] = __ldg(ysrc + r0 + wtid);
        }
#pragma unroll
        for (int i = 0; i < LINE_FLOATS / 4 / 128; ++i)
          reinterpret_cast<float4*>(line_s)[wtid + 128 * i] = make_float4(0.f, 0.f, 0.f, 0.f);
        bar_sync(barid, 128);
        const int cnt = r1 - r0;
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (wtid + 128 * k < cnt) line_s[opad(pp[k])] = st[wtid + 128 * k];
        for (int j = wtid + 512; j < cnt; j += 128) line_s[opad(__ldg(io.pos + r0 + j))] = st[j];
        bar_sync(barid, 128);
        if (wtid == 0 && line + step < total) issue(line + step);
        pass_bits5_8<false>(line_s, line_s, wtid);
      } else {
        pass_bits5_8<true>(stage, line_s, wtid);
        bar_sync(barid, 128);
        if (wtid == 0 && line + step < total) issue(line + step);
      }
      if (line + step < total) load_pend = 1;
      bar_sync(barid, 128);
      pass_bits9_11(line_s, wtid);
      bar_sync(barid, 128);
      float y[32];
      {
        const float* rowp = line_s + opad(32 * wtid);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 u = *reinterpret_cast<const float4*>(rowp + 4 * q);
          y[4 * q] = u.x; y[4 * q + 1] = u.y; y[4 * q + 2] = u.z; y[4 * q + 3] = u.w;
        }
      }
      // the previous line's MMAs have finished reading the operand
      if (mma_pend && !wait_mma()) {
        ok = false;
        break;
      }
      {
        const int b = wtid;
        if (a.KB) {   // keep the edge blocks' rows for the corrections
          int row = -1;
          if (b < a.KB) row = b;
          else if (b >= NB - a.KB) row = a.KB + b - (NB - a.KB);
          if (row >= 0) {
#pragma unroll
            for (int r = 0; r < 32; r += 4)
              *reinterpret_cast<float4*>(sye + 32 * row + r) = make_float4(y[r], y[r + 1], y[r + 2], y[r + 3]);
          }
        }
        // K-major A operand of GEMM3: element (b, r) of part P at
        // P 8192 + (b % 8) 16 + (b / 8) 512 + (r % 8) 2 + (r / 8) 128
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          uint32_t w[3][4];
#pragma unroll
          for (int e = 0; e < 4; ++e) split3x2(y[8 * q + 2 * e], y[8 * q + 2 * e + 1], w[0][e], w[1][e], w[2][e]);
#pragma unroll
          for (int P = 0; P < 3; ++P)
            *reinterpret_cast<uint4*>(ops + P * 8192 + q * 128 + (b & 7) * 16 + (b >> 3) * 512) =
                make_uint4(w[P][0], w[P][1], w[P][2], w[P][3]);
        }
      }
      fence_async_smem();
      bar_sync(barid, 128);
      if (wtid == 0) {
        tc_fence_after();
        const uint32_t d = D3 + 64u * (it & 1);
        const uint32_t id3 = idesc_bf16(128, 48, 0, 0);
        const uint32_t aq = smem_u32(ops), bb = smem_u32(sBt);
        uint32_t acc = 0;
#pragma unroll
        for (int dp = 0; dp < 3; ++dp)
#pragma unroll
          for (int op = 0; op + dp < 3; ++op)
#pragma unroll
            for (int s = 0; s < 2; ++s) {
              umma_bf16(d, sdesc(aq + dp * 8192 + 256 * s, 128, 512), sdesc(bb + op * 3072 + 256 * s, 128, 512), id3,
                        acc);
              acc = 1;
            }
        umma_commit(&gb.mma);
      }
      mma_pend = 1;
      // VMP: corrections of this line's 4p edge outputs from its edge blocks' rows
      // (one lane per output: for each row the lanes read consecutive columns)
      if (a.KB && wtid < 4 * a.p) {
        const int side = wtid >= 2 * a.p, c = wtid - side * 2 * a.p;
        const float* C = sC + (size_t)side * a.KB * 32 * 2 * a.p + c;
        const float* ye = sye + side * a.KB * 32;
        float acc0 = 0.f, acc1 = 0.f;
        for (int k = 0; k < a.KB * 32; k += 2) {
          acc0 = fmaf(C[k * 2 * a.p], ye[k], acc0);
          acc1 = fmaf(C[(k + 1) * 2 * a.p], ye[k + 1], acc1);
        }
        sco[64 * (it & 1) + wtid] = acc0 + acc1;
      }
    }
    if (prev >= 0) {
      if (!have && mma_pend && !wait_mma()) {
        ok = false;
        break;
      }
      const int ps_slot = (it - 1) & 1;
      const LineAt at = line_at(prev, io.lines);
      tc_fence_after();
      // Z row b: 48 values; lo[8c + e] = Z[c+1][e] + Z[c][8+e] + Z[c-1][16+e],
      // hi[8c + e] = Z[c+1][24+e] + Z[c][32+e] + Z[c-1][40+e]
      float z[48];
      {
        float t32[32];
        float t16[16];
        tmem_ld32(D3 + 64u * ps_slot + lane_off, t32);
        tmem_ld16(D3 + 64u * ps_slot + lane_off + 32, t16);
#pragma unroll
        for (int i = 0; i < 32; ++i) z[i] = t32[i];
#pragma unroll
        for (int i = 0; i < 16; ++i) z[32 + i] = t16[i];
      }
      // rows that cross a warp boundary go through shared memory
      if (lane == 0) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          sedge[(wq * 2 + 0) * 16 + e] = z[e];
          sedge[(wq * 2 + 0) * 16 + 8 + e] = z[24 + e];
        }
      }
      if (lane == 31) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          sedge[(wq * 2 + 1) * 16 + e] = z[16 + e];
          sedge[(wq * 2 + 1) * 16 + 8 + e] = z[40 + e];
        }
      }
      tc_fence_before();
      bar_sync(barid, 128);
      const int c = wtid;
      const bool has_next = a.per || c + 1 < NB, has_prev = a.per || c > 0;
      float lo[8], hi[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        float nl = __shfl_down_sync(0xffffffffu, z[e], 1);
        float nh = __shfl_down_sync(0xffffffffu, z[24 + e], 1);
        float pl = __shfl_up_sync(0xffffffffu, z[16 + e], 1);
        float ph = __shfl_up_sync(0xffffffffu, z[40 + e], 1);
        if (lane == 31) {   // row c + 1 is lane 0 of the next warp (wrapping for periodic plans)
          const int w2 = (wq + 1) & 3;
          nl = sedge[(w2 * 2 + 0) * 16 + e];
          nh = sedge[(w2 * 2 + 0) * 16 + 8 + e];
        }
        if (lane == 0) {
          const int w0 = (wq + 3) & 3;
          pl = sedge[(w0 * 2 + 1) * 16 + e];
          ph = sedge[(w0 * 2 + 1) * 16 + 8 + e];
        }
        lo[e] = z[8 + e] + (has_next ? nl : 0.f) + (has_prev ? pl : 0.f);
        hi[e] = z[32 + e] + (has_next ? nh : 0.f) + (has_prev ? ph : 0.f);
      }
      if (a.KB) {
        const float* co = sco + 64 * ps_slot;
        if (c == 0) {
#pragma unroll
          for (int e = 0; e < 8; ++e)
            if (e < a.p) {
              lo[e] += co[e];
              hi[e] += co[a.p + e];
            }
        }
        if (c == NB - 1) {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int k = e - (8 - a.p);   // lo[n0 - p + k] sits at e = 8 - p + k
            if (k >= 0) {
              lo[e] += co[2 * a.p + k];
              hi[e] += co[3 * a.p + k];
            }
          }
        }
      }
      const int drow = io.seq_rows ? seqrow(at.l, a.L) : at.l;
      float* dst = out + at.b * io.out_batch + (int64_t)drow * io.out_stride;
      *reinterpret_cast<float4*>(dst + 8 * c) = make_float4(lo[0], lo[1], lo[2], lo[3]);
      *reinterpret_cast<float4*>(dst + 8 * c + 4) = make_float4(lo[4], lo[5], lo[6], lo[7]);
      *reinterpret_cast<float4*>(dst + N0 + 8 * c) = make_float4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<float4*>(dst + N0 + 8 * c + 4) = make_float4(hi[4], hi[5], hi[6], hi[7]);
    }
    if (!have) break;
    prev = line;
    line += step;
  }
  if (!ok && wtid == 0) atomicExch(a.err, 1u);
  if (wtid == 0) {
    if (load_pend) mbar_wait(&gb.load[0], ph_load, 1u << 22);
    if (mma_pend) mbar_wait(&gb.mma, ph_mma, 1u << 22);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid < 32) tmem_dealloc(*tslot, 512);
}

}  // namespace ummak

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static unsigned umma_spin_limit() {
  const char* e = getenv("UW_TC_SPIN_LIMIT");
  if (e && *e) return (unsigned)strtoul(e, nullptr, 10);
  return 1u << 22;
}

bool umma_eligible(const Plan& P, const LineIO& io, const void* in, const void* out, bool fwd, int total) {
  if (!P.umma.ok || !P.d_umma || io.jlev != P.R - 1) return false;
  if (P.N != ummak::NL || P.Q != 2 || P.M != ummak::ML || P.p > 8) return false;
  if (P.umma.KB > 4 || !P.d_sync) return false;
  if (io.mode == 1 && P.m > 0 && !io.pos) return false;
  auto al16 = [](const void* q) { return ((uintptr_t)q & 15u) == 0; };
  if (fwd) {
    if (!al16(in) || io.in_stride % 4 || io.in_batch % 4) return false;
    if (io.mode == 0 && (io.out_stride % 4 || io.out_batch % 4 || !al16(out))) return false;
  } else {
    if (io.mode == 0 && (!al16(in) || io.in_stride % 4 || io.in_batch % 4)) return false;
    // the aligned copies of a row's samples need every instance's samples to
    // start 16-byte aligned
    if (io.mode == 1 && (!al16(in) || (total > io.lines && io.m % 4))) return false;
    if (!al16(out) || io.out_stride % 4 || io.out_batch % 4) return false;
  }
  return true;
}

cudaError_t umma_launch(bool fwd, const Plan& P, const float* in, float* out, const LineIO& io, int total,
                        cudaStream_t s) {
  using namespace ummak;
  Args a{};
  a.ops = (const uint16_t*)P.d_umma;
  a.KB = P.umma.KB;
  a.corr = a.KB ? (const float*)P.d_umma + P.umma.oC : nullptr;
  a.p = P.p;
  a.per = P.bd == UW_BOUNDARY_PERIODIC;
  int L = 0;
  while ((1 << L) < P.N) ++L;
  a.L = L;
  a.err = (unsigned*)P.d_sync + 2;
  a.spin = umma_spin_limit();
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (fwd) {
    const int grid = std::max(1, std::min(nsm, (total + GF - 1) / GF));
    cudaFuncSetAttribute((const void*)k_umma_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, F_SMEM);
    return launch_pdl(k_umma_fwd, dim3(grid), dim3(128 * GF), (size_t)F_SMEM, s, in, out, a, io, total);
  }
  const int grid = std::max(1, std::min(nsm, (total + GA - 1) / GA));
  cudaFuncSetAttribute((const void*)k_umma_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, A_SMEM);
  return launch_pdl(k_umma_adj, dim3(grid), dim3(128 * GA), (size_t)A_SMEM, s, in, out, a, io, total);
}

}  // namespace uw
