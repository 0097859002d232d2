// FP32 line operators on the CUDA cores (sm_103a): the hot kernels of the 2D
// path (Sec. 5, Algorithm 2) for lines of N = 2048 or 4096 samples.
//
// forward, one line of M = N / Q coefficients (lo | hi of the last level):
//   (A) last synthesis level (Sec. 3.2): s = Syn(lo, hi), 16/Q values per
//       thread from a register window;
//   (B) v = T s (Sec. 4.1 cell integrals, upsampling by Q = 2^q), 16
//       consecutive outputs per thread, then the Walsh-Hadamard stages of
//       bits 0-3 in registers (Sec. 3.1, natural order);
//   (C) bits 4-7 and bits 8..L-1 as radix-16 (or 8) pencil passes in shared
//       memory;
//   then the natural-order line is stored, or the sampled sequency indices
//   are gathered (P_Omega, Sec. 1.1).
// adjoint (Sec. 4.2): stage or scatter -> the same Walsh stages -> s = T^T v
// -> analysis (lo, hi) -> store.
//
// Both (A) and (B) use the interior formulas on the whole line with zero
// padding beyond its ends (periodic plans: wrapped copies in halos).  Near a
// VMP boundary the exact operator differs from that by C x_edge, where
// x_edge holds the p lo and p hi coefficients at that end and C reaches only
// the first / last K outputs of T (built on the host, tc_plan.cpp); the rows
// of C are spread over the CTA during (A), and the owners of the affected
// outputs add them before the bits 0-3 stage.  The adjoint adds C^T applied
// to the first / last K transformed samples to the 2p edge outputs (8 lanes
// per output, combined with shuffles).
//
// CTAs are persistent (N / 16 threads, one 16-output block per thread) and
// copy the next line (and its sample positions) into shared memory with
// cp.async while the current line runs.  The shared-memory layouts (padded
// Walsh line, swizzled s line) and the lane orders keep every access but the
// data-dependent gather / scatter free of bank conflicts: the vector stores
// of (B), the pencils of (C), the vector window loads and the zeroing; the
// Walsh butterflies use the packed FP32x2 add of sm_100+.
#include <cuda_runtime.h>

#include <type_traits>

#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "line_common.cuh"

namespace uw {

namespace f32k {

// taps as kernel parameters (constant bank), zero-padded to PM >= p, with
// 2^{-R/2} folded into the cell integrals, in pairs for the packed FP32x2 FMA:
//   hp2[d + PM/2] = (h_{2d}, h_{2d+1}), gp2 likewise         (d in [-PM/2, PM/2])
//   tp2[k][d + PM-1] = 2^{-R/2} (I_q[Q d + 2k], I_q[Q d + 2k + 1])   (d in [-(PM-1), PM-1])
// The synthesis and T pair two outputs of adjacent phases (same window
// value, both taps); the analysis and T^T pair two adjacent window values
// of one output (their two taps) and add the halves at the end.
template <int PM, int Q>
struct Taps {
  float2 hp2[PM + 1];
  float2 gp2[PM + 1];
  float2 tp2[Q / 2][2 * PM - 1];
};

struct Args {
  const float* C;   // VMP edge corrections [2][K][CS], null for periodic plans
  int K, CS, p, per;
  int L;            // log2 N
};

// Walsh line: element k at vp(k), 4 words of padding per 16.  Consecutive
// 16-blocks are 20 words apart, so any 8 consecutive blocks start in 8
// different 4-bank groups (16-byte accesses of a quarter-warp never
// conflict); 256-blocks are VCH = 320 words apart, 0 mod 32 banks.
__host__ __device__ __forceinline__ constexpr int vp(int k) { return k + 4 * (k >> 4); }
constexpr int VCH = 320;
// s line.  Q = 2: every lane owns 8 consecutive s values, so a quarter-warp
// reads or writes 16 bytes at a stride of 8 words; swapping the 4-word
// groups of odd 32-word rows in pairs makes those 8 lanes cover all 32 banks
// wherever the first lane starts.  Q = 4: 4 values per lane, the plain line
// already spreads them over all banks.
template <int Q>
__host__ __device__ __forceinline__ constexpr int sp(int m) { return Q == 2 ? (m ^ (((m >> 5) & 1) << 2)) : m; }

__host__ __device__ constexpr int up4(int a) { return (a + 3) / 4 * 4; }

// geometry constants of one instantiation
template <int PM, int Q, int NT>
struct Geom {
  static constexpr int N = 16 * NT;          // samples per line
  static constexpr int M = N / Q;            // coefficients per line
  static constexpr int n0 = M / 2;
  static constexpr int BS = 16 / Q;          // s values per thread
  static constexpr int BL = BS / 2;          // lo (and hi) values per thread
  static constexpr int VW = BL >= 4 ? 4 : 2; // vector width of the coefficient window loads
  static constexpr int HX = 8;               // coefficient halo (per side, per half)
  static constexpr int XL = 2 * (n0 + 2 * HX);   // one staged coefficient line (lo region, hi region)
  static constexpr int HS = up4(PM + 3);     // s halo
  static constexpr int SL = up4(M + 2 * HS + 4);   // sp(m) <= m + 4
  // (A) synthesis window: lo[a0 - PM/2 + w'], loaded from an aligned start
  static constexpr int OFFX = ((HX - PM / 2) % VW + VW) % VW;
  static constexpr int NWX = (OFFX + BL + PM + VW - 1) / VW * VW;
  // (B) T window: s[i0 - PM + 1 + w']
  static constexpr int OFFB = ((HS - PM + 1) % 4 + 4) % 4;
  static constexpr int NWB = up4(OFFB + BS + 2 * PM - 2);
  // adjoint T^T window: v[Q (m0 - PM + 1) + w']
  static constexpr int OFFT = ((4 - (Q * (PM - 1)) % 4) % 4);
  static constexpr int NWT = up4(OFFT + Q * (BS + 2 * PM - 2));
  // adjoint analysis window: s[2 i0 - PM + w']
  static constexpr int OFFA = ((HS - PM) % 4 + 4) % 4;
  static constexpr int NWA = up4(OFFA + 2 * BL + 2 * PM);
  static constexpr int VH = 256;             // adjoint Walsh halo (whole 256-blocks)
  static constexpr int VLf = up4(vp(N - 1) + 1);
  // of the adjoint halo only the 16-blocks that T^T reads are allocated: HL
  // elements before the line, HR after it; the buffer starts at word VB of
  // the full padded layout
  static constexpr int HL = (Q * (PM - 1) + OFFT + 15) / 16 * 16;
  static constexpr int HR = (Q * (PM - 1) + 3 + 15) / 16 * 16;
  static constexpr int VB = vp(VH - HL);
  static constexpr int VLa = up4(vp(VH + N + HR - 1) + 1) - VB;
  static constexpr int PST = N / 2 + 4;      // sample-position words per buffer
  static_assert(M % NT == 0 && BS * NT == M, "one block of 16 outputs per thread");
  static_assert(HX >= PM / 2 + VW - 1, "coefficient halo too small");
  static_assert(HS >= PM + 3, "s halo too small");
  static_assert(Q * (PM - 1) + OFFT <= VH, "Walsh halo too small");
  static_assert(HL <= VH && HR <= VH && VB % 4 == 0, "trimmed halo outside the padded layout");
  // T^T window of the last thread: Q (M - BS - PM + 1) - OFFT + NWT - 1 < N + HR
  static_assert(Q * (M - BS - PM + 1) - OFFT + NWT <= N + HR, "T^T window past the right halo");
};

// In-register Walsh-Hadamard transform of R values (natural order): the
// first stage pairs neighbours; the later ones combine aligned pairs with the
// packed FP32x2 add.
template <int R>
__device__ __forceinline__ void wht(float (&a)[R]) {
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

// wht<16> with the stage of bit 2 written as (a[k], a[k + 4]) <-
// (sa a[k] + a[k + 4], a[k] - sa a[k + 4]) for k with bit 2 clear: sa = 1 is
// the plain butterfly.  With sa = -1 and a[i] loaded from element i ^ 4 of
// the pencil, register k ends holding output k ^ 4, bit for bit what the
// plain transform of the natural order leaves in register k ^ 4 (the stage
// only exchanges the two halves and negates one, both exact).
__device__ __forceinline__ void wht16_x4(float (&a)[16], float sa) {
#pragma unroll
  for (int i = 0; i < 16; i += 2) {
    const float x = a[i], y = a[i + 1];
    a[i] = x + y;
    a[i + 1] = x - y;
  }
  const float2 m1 = make_float2(-1.f, -1.f), s2 = make_float2(sa, sa), n2 = make_float2(-sa, -sa);
#pragma unroll
  for (int h = 2; h < 16; h <<= 1)
#pragma unroll
    for (int i = 0; i < 16; i += 2)
      if (!(i & h)) {
        const float2 x = make_float2(a[i], a[i + 1]), y = make_float2(a[i + h], a[i + h + 1]);
        const float2 lo = h == 4 ? __ffma2_rn(s2, x, y) : __fadd2_rn(x, y);
        const float2 hi = h == 4 ? __ffma2_rn(n2, y, x) : __ffma2_rn(y, m1, x);
        a[i] = lo.x;
        a[i + 1] = lo.y;
        a[i + h] = hi.x;
        a[i + h + 1] = hi.y;
      }
}

// One pencil of the bits-4..7 pass: elements low4 + 16 i + 256 h (i < 16) of
// the line whose element k sits at V[vp(k + off)], off a multiple of 256.
// With low4 < 16 their padded addresses are vp(low4 + 256 h + off) + 20 i.
// Lanes 0-15 of a warp take the 16 pencils of one 256-block and lanes 16-31
// those of the next, VCH = 0 mod 32 banks further: so the upper half-warp
// visits its elements in the order i ^ 4 (80 words = 16 banks away) and
// transforms them with wht16_x4, which hands back output i ^ 4 in register i
// for the same store order.
template <int NT>
__device__ __forceinline__ void pass_mid(float* V, int off, int tid) {
  const int up = (tid >> 4) & 1;
  float* b = V + vp((tid & 15) + 256 * (tid >> 4) + off);
  float* bp = b + 80 * up;   // i with bit 2 clear: element i + 4 for the upper half-warp
  float* bm = b - 80 * up;   // bit 2 set: element i - 4
  float a[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i] = ((i & 4) ? bm : bp)[20 * i];
  wht16_x4(a, up ? -1.f : 1.f);
#pragma unroll
  for (int i = 0; i < 16; ++i) ((i & 4) ? bm : bp)[20 * i] = a[i];
}

// the lowest element of pencil c (< 256) of the bits-8.. pass: the two
// half-warps of a warp take 16-blocks a and a + 4, whose padded addresses
// differ by 16 banks
__device__ __forceinline__ int high_pencil(int c) {
  const int hw = c >> 4, w = hw >> 1;
  const int a = (w & 3) + 8 * (w >> 2) + 4 * (hw & 1);
  return 16 * a + (c & 15);
}

// bits 8..L-1: 256 pencils e0 + 256 i (e0 < 256), at vp(e0 + off) + VCH i
template <int NT>
__device__ __forceinline__ void pass_high(float* V, int off, int tid) {
  constexpr int N = 16 * NT, RH = N / 256;
#pragma unroll
  for (int c = tid; c < 256; c += NT) {
    float* b = V + vp(high_pencil(c) + off);
    float a[RH];
#pragma unroll
    for (int i = 0; i < RH; ++i) a[i] = b[VCH * i];
    wht<RH>(a);
#pragma unroll
    for (int i = 0; i < RH; ++i) b[VCH * i] = a[i];
  }
}

__device__ __forceinline__ void cp16(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc));
}
__device__ __forceinline__ void cp4(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int NPEND>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(NPEND)); }

// Position (line l within its instance, instance b) of a CTA's lines, which
// advance by the grid size: the division happens once per kernel.
struct LinePos {
  int l;
  int64_t b;
  int lines, dl;
  int64_t db;
  __device__ __forceinline__ void init(int line, int step, int nlines) {
    lines = nlines;
    l = line % nlines;
    b = line / nlines;
    dl = step % nlines;
    db = step / nlines;
  }
  __device__ __forceinline__ LinePos next() const {
    LinePos q = *this;
    q.l += dl;
    q.b += db;
    if (q.l >= lines) {
      q.l -= lines;
      ++q.b;
    }
    return q;
  }
};

// packed-sample range [r0, r1) of mask row mrow
__device__ __forceinline__ void row_range(const LineIO& io, int mrow, int& r0, int& r1) {
  r0 = __ldg(io.prefix + (int64_t)mrow * io.wpr);
  r1 = mrow + 1 < io.mask_rows ? __ldg(io.prefix + (int64_t)(mrow + 1) * io.wpr) : (int)io.m;
}

// positions (uint16 pairs) of samples [r0, r1) into sP
__device__ __forceinline__ void issue_pos(const LineIO& io, int r0, int r1, uint32_t* sP, int tid, int nt) {
  const uint32_t* pw32 = reinterpret_cast<const uint32_t*>(io.pos);
  for (int w = (r0 >> 1) + tid; w < ((r1 + 1) >> 1); w += nt) cp4(sP + (w - (r0 >> 1)), pw32 + w);
}

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------
template <int PM, int Q, int NT>
__global__ void __launch_bounds__(NT, 3) k_f32_fwd(const float* __restrict__ in, float* __restrict__ out, Args a,
                                                   Taps<PM, Q> tp, LineIO io, int total) {
  using G = Geom<PM, Q, NT>;
  constexpr int N = G::N, M = G::M, n0 = G::n0, BS = G::BS, BL = G::BL, VW = G::VW, HX = G::HX, XL = G::XL;
  constexpr int HS = G::HS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x;
  const bool gather = io.mode == 1;
  float* sV = reinterpret_cast<float*>(smem_raw);
  float* sS = sV + G::VLf;
  float* sX = sS + G::SL;                                         // 2 x XL (this line, next line)
  float* sCorr = sX + 2 * XL;                                     // 2K (VMP)
  uint32_t* sP = reinterpret_cast<uint32_t*>(sCorr + up4(2 * a.K));  // PST (gather)

  // halos start zero (VMP) and periodic halos are rewritten per line
  for (int i = tid; i < G::SL; i += NT) sS[i] = 0.f;
  for (int i = tid; i < 2 * XL; i += NT) sX[i] = 0.f;
  __syncthreads();

  auto issue_in = [&](const LinePos& lp, int bi) {
    const int drow = io.seq_rows ? seqrow(lp.l, a.L) : lp.l;
    const float* src = in + lp.b * io.in_batch + (int64_t)drow * io.in_stride;
    float* dst = sX + bi * XL;
    for (int e4 = tid; e4 < M / 4; e4 += NT) {
      const int i = 4 * e4, half = i >= n0, ii = i - half * n0;
      float* reg = dst + half * (n0 + 2 * HX);
      cp16(reg + HX + ii, src + i);
      if (a.per) {
        if (ii < HX) cp16(reg + HX + n0 + ii, src + i);
        if (ii >= n0 - HX) cp16(reg + ii - (n0 - HX), src + i);
      }
    }
  };

  // VMP edge corrections of T with their weights in registers (they are the
  // same for every line; read per line from global memory they put an L2
  // round trip between two barriers of every line): thread t < 4K takes the
  // lo (t even) or hi (t odd) half of row t / 2 of C, p weights, and the two
  // halves of a row meet on adjacent lanes.  Other shapes read C per line.
  const bool creg = a.K && PM <= 8 && 4 * a.K <= NT;
  float cw[PM <= 8 ? PM : 1];
  int coff = 0, crow = 0;
  bool cact = false;
  if (creg) {
    cact = tid < 4 * a.K;
    crow = tid >> 1;
    const int half = tid & 1, side = crow >= a.K, r = crow - side * a.K;
    // offset of this half's first edge coefficient from lo[-HX] of a staged line
    coff = half * (n0 + 2 * HX) + HX + (side == 0 ? 0 : n0 - a.p);
#pragma unroll
    for (int k = 0; k < (PM <= 8 ? PM : 1); ++k)
      cw[k] = (cact && k < a.p) ? __ldg(a.C + (size_t)(side * a.K + r) * a.CS + half * a.p + k) : 0.f;
  }

  // cp.async groups, oldest first: in(line), pos(line), in(next), ... ; the
  // sample positions of a line are copied while the previous line's gather
  // is done, and awaited just before this line's gather
  pdl_trigger();
  pdl_wait();
  const int G0 = gridDim.x;
  int line = blockIdx.x;
  LinePos cur;
  cur.init(line, G0, io.lines);
  LinePos nx = cur.next();
  int cr0 = 0, cr1 = 0, xr0 = 0, xr1 = 0;
  if (line < total) issue_in(cur, 0);
  cp_commit();
  if (gather && line < total) {
    row_range(io, cur.l, cr0, cr1);
    issue_pos(io, cr0, cr1, sP, tid, NT);
  }
  cp_commit();
  if (gather && line + G0 < total) row_range(io, nx.l, xr0, xr1);

  for (int buf = 0; line < total; line += G0, buf ^= 1) {
    const int nxt = line + G0;
    const LinePos nn = nx.next();
    if (nxt < total) issue_in(nx, buf ^ 1);
    cp_commit();
    int yr0 = 0, yr1 = 0;
    if (gather && nxt + G0 < total) row_range(io, nn.l, yr0, yr1);
    cp_wait<2>();
    __syncthreads();
    const int l = cur.l;
    const int64_t b = cur.b;
    const float* xl = sX + buf * XL;           // lo[i] at xl[HX + i]
    const float* xh = xl + n0 + 2 * HX;        // hi[i] at xh[HX + i]

    // (A) s[BS u .. BS u + BS) = Syn(lo, hi), interior formula
    {
      const int a0 = BL * tid;
      const int i0 = HX + a0 - PM / 2 - G::OFFX;     // multiple of VW
      float wl[G::NWX], wh[G::NWX];
#pragma unroll
      for (int w = 0; w < G::NWX; w += VW) {
        if constexpr (VW == 4) {
          const float4 u = *reinterpret_cast<const float4*>(xl + i0 + w);
          const float4 v = *reinterpret_cast<const float4*>(xh + i0 + w);
          wl[w] = u.x; wl[w + 1] = u.y; wl[w + 2] = u.z; wl[w + 3] = u.w;
          wh[w] = v.x; wh[w + 1] = v.y; wh[w + 2] = v.z; wh[w + 3] = v.w;
        } else {
          const float2 u = *reinterpret_cast<const float2*>(xl + i0 + w);
          const float2 v = *reinterpret_cast<const float2*>(xh + i0 + w);
          wl[w] = u.x; wl[w + 1] = u.y;
          wh[w] = v.x; wh[w + 1] = v.y;
        }
      }
      float s[BS];
#pragma unroll
      for (int jj = 0; jj < BL; ++jj) {
        float2 acc = make_float2(0.f, 0.f);      // (s[2 a], s[2 a + 1]), a = a0 + jj
#pragma unroll
        for (int d = -PM / 2; d <= PM / 2; ++d) {
          const int w = jj - d + PM / 2 + G::OFFX;
          acc = __ffma2_rn(tp.hp2[d + PM / 2], make_float2(wl[w], wl[w]), acc);
          acc = __ffma2_rn(tp.gp2[d + PM / 2], make_float2(wh[w], wh[w]), acc);
        }
        s[2 * jj] = acc.x;
        s[2 * jj + 1] = acc.y;
      }
      const int m0 = BS * tid;
#pragma unroll
      for (int j = 0; j < BS; j += 4)
        *reinterpret_cast<float4*>(sS + sp<Q>(HS + m0 + j)) = make_float4(s[j], s[j + 1], s[j + 2], s[j + 3]);
      if (a.per) {
#pragma unroll
        for (int j = 0; j < BS; ++j) {
          const int m = m0 + j;
          if (m < HS) sS[sp<Q>(HS + M + m)] = s[j];
          if (m >= M - HS) sS[sp<Q>(HS + m - M)] = s[j];
        }
      }
    }
    // VMP edge corrections of T: one row of C (2p weights) per task, rows of
    // both ends spread over the CTA
    if (creg) {
      if (tid < ((4 * a.K + 31) & ~31)) {      // warp-uniform: the warps that hold weights
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < (PM <= 8 ? PM : 1); ++k) acc = fmaf(cw[k], xl[coff + k], acc);   // cw = 0 past p
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        if (cact && !(tid & 1)) sCorr[crow] = acc;
      }
    } else if (a.K) {
      for (int t = tid; t < 2 * a.K; t += NT) {
        const int side = t >= a.K, r = t - side * a.K;
        const float4* crow = reinterpret_cast<const float4*>(a.C + ((size_t)side * a.K + r) * a.CS);
        const int base = HX + (side == 0 ? 0 : n0 - a.p);
        float acc = 0.f;
        for (int c4 = 0; 4 * c4 < 2 * a.p; ++c4) {
          const float4 cw = __ldg(crow + c4);
          const float cv[4] = {cw.x, cw.y, cw.z, cw.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int c = 4 * c4 + e;
            if (c < 2 * a.p) acc = fmaf(cv[e], c < a.p ? xl[base + c] : xh[base + c - a.p], acc);
          }
        }
        sCorr[t] = acc;
      }
    }
    __syncthreads();

    // (B) v[16 u .. 16 u + 16) = T s, corrections, bits 0-3
    {
      constexpr int BI = BS;
      const int i0 = BI * tid;
      const int j0 = HS + i0 - PM + 1 - G::OFFB;        // multiple of 4
      float ws[G::NWB];
#pragma unroll
      for (int w = 0; w < G::NWB; w += 4) {
        const float4 u = *reinterpret_cast<const float4*>(sS + sp<Q>(j0 + w));
        ws[w] = u.x; ws[w + 1] = u.y; ws[w + 2] = u.z; ws[w + 3] = u.w;
      }
      float v[16];
#pragma unroll
      for (int r = 0; r < 16; r += 2) {          // outputs r, r + 1: phases f, f + 1 of one window position
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int d = -(PM - 1); d <= PM - 1; ++d) {
          const float x = ws[r / Q - d + PM - 1 + G::OFFB];
          acc = __ffma2_rn(tp.tp2[(r % Q) / 2][d + PM - 1], make_float2(x, x), acc);
        }
        v[r] = acc.x;
        v[r + 1] = acc.y;
      }
      if (a.K) {
        const int kb = a.K / 16;
        int o = -1;
        if (tid < kb) o = 16 * tid;
        else if (tid >= NT - kb) o = a.K + 16 * (tid - (NT - kb));
        if (o >= 0) {
#pragma unroll
          for (int r = 0; r < 16; ++r) v[r] += sCorr[o + r];
        }
      }
      wht<16>(v);
      float* dst = sV + vp(16 * tid);
#pragma unroll
      for (int r = 0; r < 16; r += 4) *reinterpret_cast<float4*>(dst + r) = make_float4(v[r], v[r + 1], v[r + 2], v[r + 3]);
    }
    __syncthreads();
    // (C) bits 4-7, then bits 8..L-1
    pass_mid<NT>(sV, 0, tid);
    __syncthreads();
    if (gather) {
      pass_high<NT>(sV, 0, tid);
      cp_wait<1>();              // this line's sample positions
      __syncthreads();
      const uint16_t* ps = reinterpret_cast<const uint16_t*>(sP) + (cr0 & 1);
      float* y = out + b * io.m + cr0;
      const int cnt = cr1 - cr0;
      for (int j = tid; j < cnt; j += NT) y[j] = sV[vp(ps[j])];
      __syncthreads();           // positions consumed: the next line's may land
      if (nxt < total) issue_pos(io, xr0, xr1, sP, tid, NT);
    } else {
      // the last pass writes the natural-order line straight to global memory
      float* dst = out + b * io.out_batch + (int64_t)l * io.out_stride;
      constexpr int RH = N / 256;
#pragma unroll
      for (int c = tid; c < 256; c += NT) {
        const int e0 = high_pencil(c);
        const float* src = sV + vp(e0);
        float v[RH];
#pragma unroll
        for (int i = 0; i < RH; ++i) v[i] = src[VCH * i];
        wht<RH>(v);
#pragma unroll
        for (int i = 0; i < RH; ++i) dst[e0 + 256 * i] = v[i];
      }
    }
    cp_commit();
    cr0 = xr0;
    cr1 = xr1;
    xr0 = yr0;
    xr1 = yr1;
    cur = nx;
    nx = nn;
  }
}

// ---------------------------------------------------------------------------
// adjoint
// ---------------------------------------------------------------------------
template <int PM, int Q, int NT>
__global__ void __launch_bounds__(NT, 4) k_f32_adj(const float* __restrict__ in, float* __restrict__ out, Args a,
                                                   Taps<PM, Q> tp, LineIO io, int total) {
  using G = Geom<PM, Q, NT>;
  constexpr int N = G::N, M = G::M, n0 = G::n0, BS = G::BS, BL = G::BL, HS = G::HS, VH = G::VH;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, lane = tid & 31;
  const bool scat = io.mode == 1;
  // mode 0: two staged Walsh lines (this one, the next), transformed in
  // place; mode 1: one Walsh line, the next line's packed samples and positions.
  // Element k of a Walsh line sits at sV[vp(VH + k)], sV = buffer start - VB.
  float* sV0 = reinterpret_cast<float*>(smem_raw);
  float* sS = sV0 + (scat ? 1 : 2) * G::VLa;
  float* sCorr = sS + G::SL;                                      // 4p (VMP)
  float* sY = sCorr + up4(4 * a.p);                               // N (mode 1)
  uint32_t* sP = reinterpret_cast<uint32_t*>(sY + (scat ? N : 0));   // PST (mode 1)

  for (int i = tid; i < (scat ? 1 : 2) * G::VLa; i += NT) sV0[i] = 0.f;
  for (int i = tid; i < G::SL; i += NT) sS[i] = 0.f;
  __syncthreads();

  auto issue_in = [&](const LinePos& lp, int bi, int r0, int r1) {
    const int l = lp.l;
    const int64_t b = lp.b;
    if (!scat) {
      const float* src = in + b * io.in_batch + (int64_t)l * io.in_stride;
      float* dst = sV0 + bi * G::VLa - G::VB;
      for (int e4 = tid; e4 < N / 4; e4 += NT) cp16(dst + vp(VH + 4 * e4), src + 4 * e4);
    } else {
      const float* y = in + b * io.m;
      for (int j = r0 + tid; j < r1; j += NT) cp4(sY + (j - r0), y + j);
      issue_pos(io, r0, r1, sP, tid, NT);
    }
  };

  // VMP: C^T on the first / last K transformed samples, with the weights in
  // registers (the same for every line; read per line from global memory
  // they put an L2 round trip between two barriers of every line).  Output
  // oc (side, column) is split into 8 parts of K/8 rows on 8 consecutive
  // lanes; thread t < 32p holds part t & 7 of output t >> 3.  Other shapes
  // read C per line.
  const bool creg = a.K && 32 * PM <= NT && a.K <= 64;
  float cw[8];
  int cv0 = 0, coc = 0;
  bool cact = false;
  if (creg) {
    const int kp = a.K / 8, part = tid & 7;
    cact = tid < 32 * a.p;
    coc = tid >> 3;
    const int side = coc >= 2 * a.p, c = coc - side * 2 * a.p;
    cv0 = (side == 0 ? 0 : N - a.K) + part * kp;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      cw[k] = (cact && k < kp) ? __ldg(a.C + ((size_t)side * a.K + (size_t)part * kp + k) * a.CS + c) : 0.f;
  }

  pdl_trigger();
  pdl_wait();
  const int G0 = gridDim.x;
  int line = blockIdx.x;
  LinePos cur;
  cur.init(line, G0, io.lines);
  LinePos nx = cur.next();
  int cr0 = 0, cr1 = 0, xr0 = 0, xr1 = 0;
  if (line < total) {
    if (scat) row_range(io, cur.l, cr0, cr1);
    issue_in(cur, 0, cr0, cr1);
  }
  cp_commit();
  if (scat && line + G0 < total) row_range(io, nx.l, xr0, xr1);

  for (int buf = 0; line < total; line += G0, buf ^= 1) {
    const int nxt = line + G0;
    const LinePos nn = nx.next();
    int yr0 = 0, yr1 = 0;
    if (!scat) {
      if (nxt < total) issue_in(nx, buf ^ 1, 0, 0);
      cp_commit();
      cp_wait<1>();
    } else {
      if (nxt + G0 < total) row_range(io, nn.l, yr0, yr1);
      cp_wait<0>();   // this line's samples, copied while the previous line ran
    }
    __syncthreads();
    const int l = cur.l;
    const int64_t b = cur.b;
    float* sV = sV0 + (scat ? 0 : buf * G::VLa) - G::VB;
    if (scat) {
      // zero the line, then scatter the staged samples to their natural positions
      // 4-word chunk c = r-th of 16-block (c & 7) + 8 (c >> 5), r = (c >> 3) & 3:
      // the 8 lanes of a quarter-warp write 8 consecutive blocks
#pragma unroll
      for (int i = 0; i < N / (4 * NT); ++i) {
        const int c = NT * i + tid, blk = (c & 7) + 8 * (c >> 5), r = (c >> 3) & 3;
        *reinterpret_cast<float4*>(sV + vp(VH + 16 * blk + 4 * r)) = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      __syncthreads();
      const uint16_t* ps = reinterpret_cast<const uint16_t*>(sP) + (cr0 & 1);
      const int cnt = cr1 - cr0;
      for (int j = tid; j < cnt; j += NT) sV[vp(VH + ps[j])] = sY[j];
      __syncthreads();
      // the staging buffers are free: copy the next line's samples now
      if (nxt < total) issue_in(nx, 0, xr0, xr1);
      cp_commit();
    }
    // Walsh stages (they commute): bits 8.., bits 4-7, then 0-3 in registers
    pass_high<NT>(sV, VH, tid);
    __syncthreads();
    pass_mid<NT>(sV, VH, tid);
    __syncthreads();
    {
      float v[16];
      float* src = sV + vp(VH + 16 * tid);
#pragma unroll
      for (int r = 0; r < 16; r += 4) {
        const float4 u = *reinterpret_cast<const float4*>(src + r);
        v[r] = u.x; v[r + 1] = u.y; v[r + 2] = u.z; v[r + 3] = u.w;
      }
      wht<16>(v);
#pragma unroll
      for (int r = 0; r < 16; r += 4) *reinterpret_cast<float4*>(src + r) = make_float4(v[r], v[r + 1], v[r + 2], v[r + 3]);
      if (a.per) {   // wrapped copies in the (trimmed) halos
        const int k0 = 16 * tid;
        if (k0 < G::HR) {
          float* h = sV + vp(VH + N + k0);
#pragma unroll
          for (int r = 0; r < 16; r += 4) *reinterpret_cast<float4*>(h + r) = make_float4(v[r], v[r + 1], v[r + 2], v[r + 3]);
        }
        if (k0 >= N - G::HL) {
          float* h = sV + vp(VH + k0 - N);
#pragma unroll
          for (int r = 0; r < 16; r += 4) *reinterpret_cast<float4*>(h + r) = make_float4(v[r], v[r + 1], v[r + 2], v[r + 3]);
        }
      }
    }
    __syncthreads();
    // VMP: C^T on the first / last K transformed samples.  Output oc (side,
    // column) is split into 8 parts of K/8 rows on 8 consecutive lanes,
    // combined with shuffles (every lane of a warp runs every round).
    if (creg) {
      if (tid < ((32 * a.p + 31) & ~31)) {      // warp-uniform: the warps that hold weights
        float acc = 0.f;
        if (a.K == 64 && (cv0 & 7) == 0) {        // 8 rows, an aligned run inside one 16-block
          const float* v = sV + vp(VH + cv0);
#pragma unroll
          for (int k = 0; k < 8; ++k) acc = fmaf(cw[k], v[k], acc);
        } else {
          // cw = 0 past K/8 rows; those reads stay in the line or its zero halo
#pragma unroll
          for (int k = 0; k < 8; ++k) acc = fmaf(cw[k], sV[vp(VH + cv0 + k)], acc);
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        acc += __shfl_xor_sync(0xffffffffu, acc, 4);
        if (cact && (lane & 7) == 0) sCorr[coc] = acc;
      }
    } else if (a.K) {
      const int ntask = 32 * a.p, kp = a.K / 8;
      for (int t0 = 0; t0 < ntask; t0 += NT) {
        if (t0 + (tid & ~31) >= ntask) break;        // warp-uniform: no lane of this warp has a task
        const int t = t0 + tid;
        const bool act = t < ntask;
        const int oc = t >> 3, part = t & 7;
        const int side = oc >= 2 * a.p, c = oc - side * 2 * a.p;
        float acc = 0.f;
        if (act) {
          const float* C = a.C + ((size_t)side * a.K + (size_t)part * kp) * a.CS + c;
          const int kbase = (side == 0 ? 0 : N - a.K) + part * kp;
          if (kp == 8 && (kbase & 7) == 0) {        // an aligned run of 8 inside one 16-block
            const float* v = sV + vp(VH + kbase);
#pragma unroll
            for (int k = 0; k < 8; ++k) acc = fmaf(__ldg(C + k * a.CS), v[k], acc);
          } else {
            for (int k = 0; k < kp; ++k) acc = fmaf(__ldg(C + (size_t)k * a.CS), sV[vp(VH + kbase + k)], acc);
          }
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        acc += __shfl_xor_sync(0xffffffffu, acc, 4);
        if (act && (lane & 7) == 0) sCorr[oc] = acc;
      }
    }
    // s[BS u .. BS u + BS) = T^T v
    {
      const int m0 = BS * tid;
      const int e0 = Q * m0 - Q * (PM - 1) - G::OFFT;     // multiple of 4
      float wv[G::NWT];
      {
        // the window starts at 16 tid + (16 - Q (PM - 1) - OFFT) mod 16 inside a
        // 16-block; the padded address of each 16-block is computed once
        constexpr int S0 = ((-(Q * (PM - 1) + G::OFFT)) % 16 + 16) % 16;     // offset of e0 in its block
        const int blk0 = VH + e0 - S0;                                        // multiple of 16
#pragma unroll
        for (int w = 0; w < G::NWT; w += 4) {
          const int rel = S0 + w;                                             // compile-time
          const float4 u = *reinterpret_cast<const float4*>(sV + vp(blk0 + 16 * (rel >> 4)) + (rel & 15));
          wv[w] = u.x; wv[w + 1] = u.y; wv[w + 2] = u.z; wv[w + 3] = u.w;
        }
      }
      float s[BS];
#pragma unroll
      for (int bb = 0; bb < BS; ++bb) {
        float2 acc = make_float2(0.f, 0.f);      // phases (2k, 2k + 1) of each tap position
#pragma unroll
        for (int d = -(PM - 1); d <= PM - 1; ++d)
#pragma unroll
          for (int k = 0; k < Q / 2; ++k) {
            const int w = Q * (bb + d + PM - 1) + 2 * k + G::OFFT;   // even: an aligned register pair
            acc = __ffma2_rn(tp.tp2[k][d + PM - 1], make_float2(wv[w], wv[w + 1]), acc);
          }
        s[bb] = acc.x + acc.y;
      }
#pragma unroll
      for (int j = 0; j < BS; j += 4)
        *reinterpret_cast<float4*>(sS + sp<Q>(HS + m0 + j)) = make_float4(s[j], s[j + 1], s[j + 2], s[j + 3]);
      if (a.per) {
#pragma unroll
        for (int j = 0; j < BS; ++j) {
          const int m = m0 + j;
          if (m < HS) sS[sp<Q>(HS + M + m)] = s[j];
          if (m >= M - HS) sS[sp<Q>(HS + m - M)] = s[j];
        }
      }
    }
    __syncthreads();
    // analysis: lo, hi [BL u .. BL u + BL), plus the VMP edge corrections
    {
      const int i0 = BL * tid;
      const int j0 = HS + 2 * i0 - PM - G::OFFA;        // multiple of 4
      float ws[G::NWA];
#pragma unroll
      for (int w = 0; w < G::NWA; w += 4) {
        const float4 u = *reinterpret_cast<const float4*>(sS + sp<Q>(j0 + w));
        ws[w] = u.x; ws[w + 1] = u.y; ws[w + 2] = u.z; ws[w + 3] = u.w;
      }
      float lo[BL], hi[BL];
#pragma unroll
      for (int bb = 0; bb < BL; ++bb) {
        float2 x = make_float2(0.f, 0.f), y = make_float2(0.f, 0.f);
#pragma unroll
        for (int d = -PM / 2; d <= PM / 2; ++d) {
          const int w = 2 * (bb + d) + PM + G::OFFA;                 // even: an aligned register pair
          const float2 sv = make_float2(ws[w], ws[w + 1]);
          x = __ffma2_rn(tp.hp2[d + PM / 2], sv, x);
          y = __ffma2_rn(tp.gp2[d + PM / 2], sv, y);
        }
        lo[bb] = x.x + x.y;
        hi[bb] = y.x + y.y;
      }
      if (a.K) {
#pragma unroll
        for (int bb = 0; bb < BL; ++bb) {
          const int i = i0 + bb;
          if (i < a.p) {
            lo[bb] += sCorr[i];
            hi[bb] += sCorr[a.p + i];
          } else if (i >= n0 - a.p) {
            const int e = i - (n0 - a.p);
            lo[bb] += sCorr[2 * a.p + e];
            hi[bb] += sCorr[3 * a.p + e];
          }
        }
      }
      const int drow = io.seq_rows ? seqrow(l, a.L) : l;
      float* dst = out + b * io.out_batch + (int64_t)drow * io.out_stride;
      if constexpr (BL == 4) {
        *reinterpret_cast<float4*>(dst + i0) = make_float4(lo[0], lo[1], lo[2], lo[3]);
        *reinterpret_cast<float4*>(dst + n0 + i0) = make_float4(hi[0], hi[1], hi[2], hi[3]);
      } else {
        *reinterpret_cast<float2*>(dst + i0) = make_float2(lo[0], lo[1]);
        *reinterpret_cast<float2*>(dst + n0 + i0) = make_float2(hi[0], hi[1]);
      }
    }
    cr0 = xr0;
    cr1 = xr1;
    xr0 = yr0;
    xr1 = yr1;
    cur = nx;
    nx = nn;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <int PM, int Q>
Taps<PM, Q> make_taps(const Plan& P) {
  Taps<PM, Q> t;
  const int p = P.p;
  const double sc = std::exp2(-0.5 * P.R);
  auto hf = [&](int l) { return (l >= -p + 1 && l <= p) ? (float)P.h[l + p - 1] : 0.f; };
  auto gf = [&](int l) { return (l >= -p + 1 && l <= p) ? (float)P.g[l + p - 1] : 0.f; };
  for (int d = -PM / 2; d <= PM / 2; ++d) {
    t.hp2[d + PM / 2] = make_float2(hf(2 * d), hf(2 * d + 1));
    t.gp2[d + PM / 2] = make_float2(gf(2 * d), gf(2 * d + 1));
  }
  auto tf = [&](int f, int d) {
    return (d >= -(p - 1) && d <= p - 1) ? (float)(sc * P.taps[Q * d + f + (p - 1) * Q]) : 0.f;
  };
  for (int k = 0; k < Q / 2; ++k)
    for (int d = -(PM - 1); d <= PM - 1; ++d) t.tp2[k][d + PM - 1] = make_float2(tf(2 * k, d), tf(2 * k + 1, d));
  return t;
}

template <int PM, int Q, int NT>
size_t smem_fwd(const Plan& P, bool gather) {
  using G = Geom<PM, Q, NT>;
  return sizeof(float) * ((size_t)G::VLf + G::SL + 2 * G::XL + up4(2 * P.f32.K)) +
         (gather ? sizeof(uint32_t) * (size_t)G::PST : 0);
}

template <int PM, int Q, int NT>
size_t smem_adj(const Plan& P, bool scat) {
  using G = Geom<PM, Q, NT>;
  return sizeof(float) * ((size_t)(scat ? 1 : 2) * G::VLa + G::SL + up4(4 * P.p)) +
         (scat ? sizeof(float) * (size_t)G::N + sizeof(uint32_t) * (size_t)G::PST : 0);
}

template <typename K>
int persistent_grid(K kernel, int nt, size_t smem, int total) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, nt, smem);
  return std::max(1, std::min(total, std::max(per, 1) * nsm));
}

template <int PM, int Q, int NT>
cudaError_t go(bool fwd, const Plan& P, const float* in, float* out, const LineIO& io, int total, cudaStream_t s) {
  Args a{};
  a.C = (const float*)P.d_f32;
  a.K = P.f32.K;
  a.CS = P.f32.CS;
  a.p = P.p;
  a.per = P.bd == UW_BOUNDARY_PERIODIC;
  int L = 0;
  while ((1 << L) < P.N) ++L;
  a.L = L;
  const Taps<PM, Q> t = make_taps<PM, Q>(P);
  if (fwd) {
    const size_t sm = smem_fwd<PM, Q, NT>(P, io.mode == 1);
    auto kern = k_f32_fwd<PM, Q, NT>;
    set_smem_limit((const void*)kern);
    cudaFuncSetAttribute((const void*)kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return launch_pdl(kern, dim3(persistent_grid(kern, NT, sm, total)), dim3(NT), sm, s, in, out, a, t, io, total);
  }
  const size_t sm = smem_adj<PM, Q, NT>(P, io.mode == 1);
  auto kern = k_f32_adj<PM, Q, NT>;
  set_smem_limit((const void*)kern);
  cudaFuncSetAttribute((const void*)kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  return launch_pdl(kern, dim3(persistent_grid(kern, NT, sm, total)), dim3(NT), sm, s, in, out, a, t, io, total);
}

template <int PM, int NT>
cudaError_t go_q(bool fwd, const Plan& P, const float* in, float* out, const LineIO& io, int total, cudaStream_t s) {
  if (P.Q == 2) return go<PM, 2, NT>(fwd, P, in, out, io, total, s);
  return go<PM, 4, NT>(fwd, P, in, out, io, total, s);
}

template <int NT>
cudaError_t go_nt(bool fwd, const Plan& P, const float* in, float* out, const LineIO& io, int total, cudaStream_t s) {
  if (P.p <= 4) return go_q<4, NT>(fwd, P, in, out, io, total, s);
  if (P.p <= 8) return go_q<8, NT>(fwd, P, in, out, io, total, s);
  return go_q<10, NT>(fwd, P, in, out, io, total, s);
}

// ---------------------------------------------------------------------------
// long 1D lines (N = 2^L, L > 12): segments of 4096 outputs
// ---------------------------------------------------------------------------
constexpr int SEGN = 4096, SEGNT = 256;
constexpr int SEGV = up4(vp(SEGN - 1) + 1);

// the rest of a segment after its 16-blocks are in V (natural order, bits
// 0-3 done): bits 4-7 in place, bits 8-11 on the way to out[0, 4096)
__device__ __forceinline__ void seg_finish(float* V, float* __restrict__ out, int tid) {
  __syncthreads();
  pass_mid<SEGNT>(V, 0, tid);
  __syncthreads();
  const int e0 = high_pencil(tid);
  const float* src = V + vp(e0);
  float v[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = src[VCH * i];
  wht<16>(v);
#pragma unroll
  for (int i = 0; i < 16; ++i) out[e0 + 256 * i] = v[i];
}

// v = T s on segment `seg` of line b, then the Walsh-Hadamard stages of bits
// 0-11 (Sec. 4.1, Sec. 3.1); the stages of bits 12.. across segments follow
// in another kernel.  Thread t computes outputs 16 t .. 16 t + 15 of the
// segment from a register window of s (interior formula, taps with
// 2^{-R/2} folded in; periodic plans wrap the window).  Outputs within ntap
// of a VMP end take the exact formula (boundary rows of T).
template <int PM, int Q>
__global__ void __launch_bounds__(SEGNT) k_up_seg(const float* __restrict__ s, float* __restrict__ v, Taps<PM, Q> tp,
                                                  Tables<float> tab, Geo G, int segs) {
  constexpr int BS = 16 / Q, NW = BS + 2 * PM - 2;
  __shared__ __align__(16) float sV[SEGV];
  pdl_trigger();
  pdl_wait();
  const int tid = threadIdx.x;
  const int64_t b = blockIdx.x / segs;
  const int seg = blockIdx.x - (int)(b * segs);
  const int M = G.M, N = G.N;
  const float* sb = s + b * M;
  const int K0 = seg * SEGN + 16 * tid;
  float o[16];
  if (G.bd == UW_BOUNDARY_VMP && (K0 < G.ntap || K0 + 16 > N - G.ntap)) {
    const float sc = exp2f(-0.5f * (float)G.R);
    Plain<float> sa{sb};
#pragma unroll 1
    for (int r = 0; r < 16; ++r) o[r] = sc * up_one<float>(K0 + r, sa, tab, G);
  } else {
    const int m0 = K0 / Q - PM + 1;
    float ws[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      int m = m0 + w;
      if (G.bd == UW_BOUNDARY_PERIODIC) m &= M - 1;
      ws[w] = (m >= 0 && m < M) ? __ldg(sb + m) : 0.f;
    }
#pragma unroll
    for (int r = 0; r < 16; r += 2) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int d = -(PM - 1); d <= PM - 1; ++d) {
        const float x = ws[r / Q - d + PM - 1];
        acc = __ffma2_rn(tp.tp2[(r % Q) / 2][d + PM - 1], make_float2(x, x), acc);
      }
      o[r] = acc.x;
      o[r + 1] = acc.y;
    }
  }
  wht<16>(o);
  float* dst = sV + vp(16 * tid);
#pragma unroll
  for (int r = 0; r < 16; r += 4) *reinterpret_cast<float4*>(dst + r) = make_float4(o[r], o[r + 1], o[r + 2], o[r + 3]);
  seg_finish(sV, v + b * N + (int64_t)seg * SEGN, tid);
}


// taps of T^T, 2^{-R/2} folded in, zero-padded to (2 PM - 1) Q entries:
// entry i multiplies v[Q m + (1 - PM) Q + i] for output s[m]
template <int PM, int Q>
struct TapsT {
  float2 t2[(2 * PM - 1) * Q / 2];
};

// outputs of T^T at each side of a segment that the fused kernel below
// leaves to seg_upT_fix (their window reaches the neighbouring segment, or a
// VMP end): NB, and the segment values those read, H at each end
template <int PM, int Q>
struct SegUT {
  static constexpr int CK = 4;                               // outputs per window step
  static constexpr int NB = (2 * PM + CK - 1) / CK * CK;     // >= max(PM - 1, p), whole steps
  static constexpr int H = ((NB + PM) * Q + 15) / 16 * 16;   // >= (NB + p) Q and >= (p - 1) Q
};

// The adjoint's segment kernel with 64 threads per segment of 4096: thread t
// loads the pencil t + 64 i (coalesced) and applies the stages of bits 6-11
// in registers; one exchange through shared memory (4 words of padding per
// 64, conflict-free both ways) gives it the 64 consecutive values 64 t + i,
// and the stages of bits 0-5 follow in registers (the stages commute).
// Shared-memory traffic per value: one store, one load and one store, and
// about 1.4 loads for the T^T windows, which slide through registers 4
// outputs at a time.  (With 256 threads, 16 values
// each and three passes of 4 stages, each value went through shared memory
// about 7.5 times, and the kernel was bound by it.)
constexpr int SEG64 = 64;
__host__ __device__ __forceinline__ constexpr int vq(int k) { return k + 4 * (k >> 6); }
constexpr int SEGV64 = up4(vq(SEGN - 1) + 1);

// the adjoint on segment `seg` of line b, after the stages across segments:
// the Walsh-Hadamard stages of bits 0-11, then s = T^T v for the segment's
// interior outputs (windows from shared memory), and the H values at each
// end of the transformed segment back to v for the boundary outputs
// (seg_upT_fix)
template <int PM, int Q>
__global__ void __launch_bounds__(SEG64) k_fwht_seg64_upT(float* __restrict__ v, float* __restrict__ s,
                                                          TapsT<PM, Q> tp, Geo G, int segs) {
  using U = SegUT<PM, Q>;
  pdl_trigger();
  pdl_wait();
  constexpr int BO = SEGN / Q / SEG64, NT2 = (2 * PM - 1) * Q / 2;   // outputs per thread: 16 or 32
  constexpr int OFF = (((1 - PM) * Q) % 4 + 4) % 4;          // window start below a 4-aligned index
  constexpr int CK = U::CK, ST = Q * CK;                     // outputs per window step, window advance
  constexpr int W = (OFF + Q * (CK + 2 * PM - 2) + 3) / 4 * 4;
  static_assert(BO % CK == 0 && W > ST && ST % 4 == 0, "window steps");
  __shared__ __align__(16) float sV[SEGV64];
  const int tid = threadIdx.x;
  const int64_t b = blockIdx.x / segs;
  const int seg = blockIdx.x - (int)(b * segs);
  float* vs = v + b * G.N + (int64_t)seg * SEGN;
  {
    float a[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) a[i] = vs[tid + 64 * i];
    wht<64>(a);
#pragma unroll
    for (int i = 0; i < 64; ++i) sV[vq(tid + 64 * i)] = a[i];
  }
  __syncthreads();
  {
    float a[64];
    float* row = sV + vq(64 * tid);
#pragma unroll
    for (int r = 0; r < 64; r += 4) {
      const float4 u = *reinterpret_cast<const float4*>(row + r);
      a[r] = u.x; a[r + 1] = u.y; a[r + 2] = u.z; a[r + 3] = u.w;
    }
    wht<64>(a);
#pragma unroll
    for (int r = 0; r < 64; r += 4) *reinterpret_cast<float4*>(row + r) = make_float4(a[r], a[r + 1], a[r + 2], a[r + 3]);
  }
  __syncthreads();
  // the ends of the transformed segment, for the boundary outputs
  for (int i = tid; i < 2 * U::H; i += SEG64) {
    const int k = i < U::H ? i : SEGN - 2 * U::H + i;
    vs[k] = sV[vq(k)];
  }
  // interior outputs: local m in [NB, SEGN / Q - NB), CK at a time
  const int ml = BO * tid;
  float* sb = s + b * G.M + (int64_t)seg * (SEGN / Q) + ml;
  auto step = [&](const float (&win)[W], int c) {
    float out[CK];
#pragma unroll
    for (int u = 0; u < CK; ++u) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < NT2; ++i)
        acc = __ffma2_rn(tp.t2[i], make_float2(win[OFF + Q * u + 2 * i], win[OFF + Q * u + 2 * i + 1]), acc);
      out[u] = acc.x + acc.y;
    }
    *reinterpret_cast<float4*>(sb + CK * c) = make_float4(out[0], out[1], out[2], out[3]);
  };
  // window of step c: v[Q (ml + CK c) + (1 - PM) Q - OFF ..) (a multiple of 4; inside the
  // segment whenever the step's outputs are interior)
  const int k0 = Q * ml + (1 - PM) * Q - OFF;
  float win[W];
  if (ml >= U::NB && ml + BO <= SEGN / Q - U::NB) {
    // every step interior: the window slides through registers
#pragma unroll
    for (int w = 0; w < W; w += 4) {
      const float4 u = *reinterpret_cast<const float4*>(sV + vq(k0 + w));   // 4 values inside one 64-block
      win[w] = u.x; win[w + 1] = u.y; win[w + 2] = u.z; win[w + 3] = u.w;
    }
#pragma unroll
    for (int c = 0; c < BO / CK; ++c) {
      step(win, c);
      if (c + 1 < BO / CK) {
#pragma unroll
        for (int w = 0; w < W - ST; ++w) win[w] = win[w + ST];
#pragma unroll
        for (int w = W - ST; w < W; w += 4) {
          const float4 u = *reinterpret_cast<const float4*>(sV + vq(k0 + ST * (c + 1) + w));
          win[w] = u.x; win[w + 1] = u.y; win[w + 2] = u.z; win[w + 3] = u.w;
        }
      }
    }
  } else {
    // the first and last thread: only the interior steps, each with its own window
#pragma unroll 1
    for (int c = 0; c < BO / CK; ++c) {
      const int m = ml + CK * c;
      if (m < U::NB || m + CK > SEGN / Q - U::NB) continue;
#pragma unroll
      for (int w = 0; w < W; w += 4) {
        const float4 u = *reinterpret_cast<const float4*>(sV + vq(k0 + ST * c + w));
        win[w] = u.x; win[w + 1] = u.y; win[w + 2] = u.z; win[w + 3] = u.w;
      }
      step(win, c);
    }
  }
}

// the boundary outputs of T^T that the fused segment kernel left: NB at
// each side of every segment, by the exact formula (reads v only inside the
// ends written)
template <int PM, int Q>
__global__ void __launch_bounds__(256) k_seg_upT_fix(const float* __restrict__ v, float* __restrict__ s,
                                                     Tables<float> tab, Geo G, int segs, int batch) {
  using U = SegUT<PM, Q>;
  pdl_trigger();
  pdl_wait();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per_line = (int64_t)segs * 2 * U::NB;
  if (idx >= (int64_t)batch * per_line) return;
  const int64_t b = idx / per_line;
  const int r = (int)(idx - b * per_line);
  const int seg = r / (2 * U::NB), j = r - seg * (2 * U::NB);
  const int m = seg * (SEGN / Q) + (j < U::NB ? j : SEGN / Q - 2 * U::NB + j);
  const float sc = exp2f(-0.5f * (float)G.R);
  Plain<float> va{v + b * G.N};
  s[b * G.M + m] = sc * upT_one<float>(m, va, tab, G);
}


// ---------------------------------------------------------------------------
// 1D wavelet levels (Sec. 3.2) with register windows: a thread makes 8
// synthesis outputs, or 4 analysis (lo, hi) pairs, by the interior formula;
// the outputs whose formula involves an edge function take the exact one
// (VMP); periodic plans wrap the windows, which is exact.
// ---------------------------------------------------------------------------
template <int PM>
struct HGTaps {
  float2 hp2[PM + 1];   // (h_{2d}, h_{2d+1}), d in [-PM/2, PM/2]
  float2 gp2[PM + 1];
};

// s_{j+1}[8 g .. 8 g + 8) from lo = s_j, hi = d_j (n0 values each)
template <int PM>
__device__ __forceinline__ void syn8(const float* lo, const float* hi, int n0, int g, bool per, const HGTaps<PM>& tp,
                                     float (&o)[8]) {
  constexpr int NW = 4 + PM;
  const int i0 = 4 * g - PM / 2;
  float wl[NW], wh[NW];
  // inside the line and 16-byte aligned: the window as aligned 16-byte
  // vectors from a0 = 4 g - S (lanes 16 bytes apart: no shared-memory bank
  // conflicts, a quarter of the load instructions)
  constexpr int S = (PM / 2 + 3) / 4 * 4, NV = (S + 4 + PM / 2 + 3) / 4;
  const int a0 = 4 * g - S;
  if (a0 >= 0 && a0 + 4 * NV <= n0 &&
      !((reinterpret_cast<uintptr_t>(lo + a0) | reinterpret_cast<uintptr_t>(hi + a0)) & 15)) {
    float vl[4 * NV], vh[4 * NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const float4 a = reinterpret_cast<const float4*>(lo + a0)[v];
      const float4 b = reinterpret_cast<const float4*>(hi + a0)[v];
      vl[4 * v] = a.x; vl[4 * v + 1] = a.y; vl[4 * v + 2] = a.z; vl[4 * v + 3] = a.w;
      vh[4 * v] = b.x; vh[4 * v + 1] = b.y; vh[4 * v + 2] = b.z; vh[4 * v + 3] = b.w;
    }
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      wl[w] = vl[w + S - PM / 2];
      wh[w] = vh[w + S - PM / 2];
    }
  } else {
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      int m = i0 + w;
      if (per) m &= n0 - 1;
      const bool ok = m >= 0 && m < n0;
      wl[w] = ok ? lo[m] : 0.f;
      wh[w] = ok ? hi[m] : 0.f;
    }
  }
#pragma unroll
  for (int jj = 0; jj < 4; ++jj) {
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int d = -PM / 2; d <= PM / 2; ++d) {
      const int w = jj - d + PM / 2;
      acc = __ffma2_rn(tp.hp2[d + PM / 2], make_float2(wl[w], wl[w]), acc);
      acc = __ffma2_rn(tp.gp2[d + PM / 2], make_float2(wh[w], wh[w]), acc);
    }
    o[2 * jj] = acc.x;
    o[2 * jj + 1] = acc.y;
  }
}

// (lo, hi)[4 g .. 4 g + 4) of level j from s = s_{j+1} (n1 = 2 n0 values)
template <int PM>
__device__ __forceinline__ void ana4(const float* s, int n1, int g, bool per, const HGTaps<PM>& tp, float (&lo)[4],
                                     float (&hi)[4]) {
  constexpr int NW = 8 + 2 * PM;
  const int i0 = 8 * g - PM;
  float ws[NW];
  // inside the line and 16-byte aligned: aligned 16-byte vectors from
  // a0 = 8 g - S (as in syn8)
  constexpr int S = (PM + 3) / 4 * 4, NV = (S + 8 + PM + 3) / 4;
  const int a0 = 8 * g - S;
  if (a0 >= 0 && a0 + 4 * NV <= n1 && !(reinterpret_cast<uintptr_t>(s + a0) & 15)) {
    float vs[4 * NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const float4 a = reinterpret_cast<const float4*>(s + a0)[v];
      vs[4 * v] = a.x; vs[4 * v + 1] = a.y; vs[4 * v + 2] = a.z; vs[4 * v + 3] = a.w;
    }
#pragma unroll
    for (int w = 0; w < NW; ++w) ws[w] = vs[w + S - PM];
  } else {
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      int k = i0 + w;
      if (per) k &= n1 - 1;
      ws[w] = (k >= 0 && k < n1) ? s[k] : 0.f;
    }
  }
#pragma unroll
  for (int bb = 0; bb < 4; ++bb) {
    float2 x = make_float2(0.f, 0.f), y = make_float2(0.f, 0.f);
#pragma unroll
    for (int d = -PM / 2; d <= PM / 2; ++d) {
      const int w = 2 * (bb + d) + PM;
      const float2 sv = make_float2(ws[w], ws[w + 1]);
      x = __ffma2_rn(tp.hp2[d + PM / 2], sv, x);
      y = __ffma2_rn(tp.gp2[d + PM / 2], sv, y);
    }
    lo[bb] = x.x + x.y;
    hi[bb] = y.x + y.y;
  }
}

// One output of a VMP synthesis level by the exact formula (Sec. 3.2
// boundary functions), the same sums in the same order as syn_one, with the
// loops unrolled to the compile-time filter bound so that all loads of the
// output are issued together.
template <int PM, typename TB>
__device__ __forceinline__ float syn_one_u(int k, int n0, const float* lo, const float* hi, const TB& t, const Geo& G) {
  const int p = G.p, n1 = 2 * n0, Lb = G.Lb;
  const int mlo = max(p, (k - p + 1) >> 1), mhi = min(n0 - p - 1, (k + p - 1) >> 1);   // at most p terms
  float acc = 0.f;
#pragma unroll
  for (int d = 0; d < PM; ++d) {
    const int m = mlo + d;
    if (m <= mhi) {
      const int l = k - 2 * m + p - 1;
      acc += t.h[l] * lo[m] + t.g[l] * hi[m];
    }
  }
  if (k < Lb) {
#pragma unroll
    for (int m = 0; m < PM; ++m)
      if (m < p) acc += t.PL[m * Lb + k] * lo[m] + t.QL[m * Lb + k] * hi[m];
  }
  const int c = n1 - 1 - k;
  if (c < Lb) {
#pragma unroll
    for (int r = 0; r < PM; ++r)
      if (r < p) acc += t.PR[r * Lb + c] * lo[n0 - 1 - r] + t.QR[r * Lb + c] * hi[n0 - 1 - r];
  }
  return acc;
}

// One output pair of a VMP analysis level by the exact formula, as ana_one
// (same sums, same order), unrolled to the compile-time filter bound.
template <int PM, typename TB>
__device__ __forceinline__ void ana_one_u(int m, int n0, const float* s, const TB& t, const Geo& G, float& lo,
                                          float& hi) {
  const int p = G.p, n1 = 2 * n0, Lb = G.Lb;   // Lb = 3p - 1 < 3 PM
  float a = 0.f, b = 0.f;
  if (m < p) {
#pragma unroll
    for (int c = 0; c < 3 * PM; ++c)
      if (c < Lb) {
        const float v = s[c];
        a += t.PL[m * Lb + c] * v;
        b += t.QL[m * Lb + c] * v;
      }
  } else if (m >= n0 - p) {
    const int r = n0 - 1 - m;
#pragma unroll
    for (int c = 0; c < 3 * PM; ++c)
      if (c < Lb) {
        const float v = s[n1 - 1 - c];
        a += t.PR[r * Lb + c] * v;
        b += t.QR[r * Lb + c] * v;
      }
  } else {
#pragma unroll
    for (int d = 0; d < 2 * PM; ++d)
      if (d < 2 * p) {
        const float v = s[2 * m + d - p + 1];
        a += t.h[d] * v;
        b += t.g[d] * v;
      }
  }
  lo = a;
  hi = b;
}

// the lane of warp-mask `em` that holds the j-th set bit (lane 0 if none)
__device__ __forceinline__ int nth_lane(unsigned em, int j) {
  for (int i = 0; i < j && em; ++i) em &= em - 1;
  return em ? __ffs(em) - 1 : 0;
}

// One synthesis level, groups of 8 outputs; every lane of the warp calls it
// (valid: the lane has a group).  Interior groups by the register-window
// formula.  The outputs of the groups near a VMP end are then shared out
// over the warp, one per lane, 4 groups per round: computed one after
// another by the group's own thread they put a chain of memory round trips
// on the critical path of the level.
template <int PM, typename TB>
__device__ __forceinline__ void syn_group(const float* lo, const float* hi, float* o, int n0, int g, bool valid,
                                          const HGTaps<PM>& tp, const TB& tab, const Geo& G) {
  const int n1 = 2 * n0, k0 = 8 * g;
  const bool per = G.bd == UW_BOUNDARY_PERIODIC;
  const bool edge = valid && !per && (k0 < G.Lb || k0 + 8 > n1 - G.Lb);
  if (valid && !edge) {
    float v[8];
    syn8<PM>(lo, hi, n0, g, per, tp, v);
    *reinterpret_cast<float4*>(o + k0) = make_float4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<float4*>(o + k0 + 4) = make_float4(v[4], v[5], v[6], v[7]);
  }
  const unsigned em = __ballot_sync(0xffffffffu, edge);
  if (!em) return;
  const int lane = threadIdx.x & 31, ne = __popc(em);
  for (int base = 0; base < ne; base += 4) {
    const int j = base + (lane >> 3), src = nth_lane(em, j);
    const int ks = __shfl_sync(0xffffffffu, k0, src) + (lane & 7);
    const float* ls = reinterpret_cast<const float*>(__shfl_sync(0xffffffffu, (unsigned long long)lo, src));
    const float* hs = reinterpret_cast<const float*>(__shfl_sync(0xffffffffu, (unsigned long long)hi, src));
    float* os = reinterpret_cast<float*>(__shfl_sync(0xffffffffu, (unsigned long long)o, src));
    if (j < ne) os[ks] = syn_one_u<PM>(ks, n0, ls, hs, tab, G);
  }
}

// One analysis level, groups of 4 pairs; every lane of the warp calls it.
// Interior groups by the register-window formula, the pairs of the groups
// near a VMP end shared out over the warp, one per lane, 8 groups per round.
template <int PM, typename TB>
__device__ __forceinline__ void ana_group(const float* s, float* lo, float* hi, int n0, int g, bool valid,
                                          const HGTaps<PM>& tp, const TB& tab, const Geo& G) {
  const int m0 = 4 * g;
  const bool per = G.bd == UW_BOUNDARY_PERIODIC;
  const bool edge = valid && !per && (m0 < G.p || m0 + 4 > n0 - G.p);
  if (valid && !edge) {
    float a[4], b[4];
    ana4<PM>(s, 2 * n0, g, per, tp, a, b);
    *reinterpret_cast<float4*>(lo + m0) = make_float4(a[0], a[1], a[2], a[3]);
    *reinterpret_cast<float4*>(hi + m0) = make_float4(b[0], b[1], b[2], b[3]);
  }
  const unsigned em = __ballot_sync(0xffffffffu, edge);
  if (!em) return;
  const int lane = threadIdx.x & 31, ne = __popc(em);
  for (int base = 0; base < ne; base += 8) {
    const int j = base + (lane >> 2), src = nth_lane(em, j);
    const int ms = __shfl_sync(0xffffffffu, m0, src) + (lane & 3);
    const float* ss = reinterpret_cast<const float*>(__shfl_sync(0xffffffffu, (unsigned long long)s, src));
    float* los = reinterpret_cast<float*>(__shfl_sync(0xffffffffu, (unsigned long long)lo, src));
    float* his = reinterpret_cast<float*>(__shfl_sync(0xffffffffu, (unsigned long long)hi, src));
    if (j < ne) {
      float a, b;
      ana_one_u<PM>(ms, n0, ss, tab, G, a, b);
      los[ms] = a;
      his[ms] = b;
    }
  }
}

// the coarse synthesis levels J0 .. jto-1 of one line per CTA in shared
// memory (two buffers of 2^(jto-1)); details from x, s_jto to out
template <int PM>
__global__ void __launch_bounds__(1024) k_syn1d_levels_f32(const float* __restrict__ x, float* __restrict__ out,
                                                           int64_t out_bs, HGTaps<PM> tp, Tables<float> tab, Geo G,
                                                           int J0, int jto, int64_t in_bs, int stage) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  SmemTables<float> st;
  const int off = stage_tables(tab, G, sm, st, tid, nthr);
  pdl_trigger();
  pdl_wait();
  const float* xb = x + (int64_t)blockIdx.x * in_bs;
  float* ob = out + (int64_t)blockIdx.x * out_bs;
  // the whole line of coefficients into L2: each level here and the level
  // kernels after this one read their details from there instead of DRAM
  if (tid == 0) prefetch_l2_bulk(xb, 4 * in_bs);
  float* P0 = sm + ((off + 3) & ~3);
  float* P1 = P0 + (1 << (jto - 1));
  // stage: the last level's details (2^(jto-1) values, the largest level)
  // are copied into shared memory while the lower levels run, so that level
  // does not wait on global memory once per group
  float* D = P1 + (1 << (jto - 1));
  if (stage)
    for (int i = 4 * tid; i < (1 << (jto - 1)); i += 4 * nthr) cp16(D + i, xb + (1 << (jto - 1)) + i);
  cp_commit();
  for (int k = tid; k < (1 << J0); k += nthr) P0[k] = xb[k];
  __syncthreads();
  float* src = P0;
  float* dst = P1;
  for (int j = J0; j < jto; ++j) {
    const int n0 = 1 << j, n1 = 2 * n0;
    float* o = j + 1 == jto ? ob : dst;
    const bool staged = stage && j + 1 == jto;
    if (staged) {
      cp_wait<0>();
      __syncthreads();
    }
    const float* hd = staged ? D : xb + n0;
    if (n1 / 8 >= nthr) {   // groups of 8 once they fill the CTA; small levels are latency-bound
      for (int g = tid; g < n1 / 8; g += nthr) syn_group<PM>(src, hd, o, n0, g, true, tp, st, G);
    } else if (G.bd == UW_BOUNDARY_PERIODIC) {
      Plain<float> lo{src}, hi{hd};
      for (int k = tid; k < n1; k += nthr) o[k] = syn_one<float>(k, n0, lo, hi, st, G);
    } else {
      for (int k = tid; k < n1; k += nthr) o[k] = syn_one_u<PM>(k, n0, src, hd, st, G);
    }
    __syncthreads();
    float* t = src;
    src = dst;
    dst = t;
  }
}

// The transposed steps: the analysis levels jfrom-1 .. J0 of one line per
// CTA.  Every level writes its details to x[2^j, 2^(j+1)) and its low-pass
// half to shared memory (the last one to x[0, 2^J0)); groups of 4 pairs
// once they fill the CTA, the per-pair formula below that.  stage: the
// input s_jfrom (2^jfrom values, the previous kernel's output) is first
// copied into the second buffer and the room after it, so the first level,
// the largest, reads shared memory rather than global memory pair by pair.
template <int PM>
__global__ void __launch_bounds__(1024) k_ana1d_levels_f32(const float* __restrict__ in, int64_t in_bs,
                                                           float* __restrict__ x, HGTaps<PM> tp, Tables<float> tab,
                                                           Geo G, int J0, int jfrom, int64_t out_bs, int stage) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);
  const int tid = threadIdx.x, nthr = blockDim.x;
  SmemTables<float> st;
  const int off = stage_tables(tab, G, sm, st, tid, nthr);
  pdl_trigger();
  pdl_wait();
  const float* ib = in + (int64_t)blockIdx.x * in_bs;
  float* xb = x + (int64_t)blockIdx.x * out_bs;
  float* P0 = sm + ((off + 3) & ~3);
  float* P1 = P0 + (1 << (jfrom - 1));
  const float* src = ib;
  if (stage) {
    for (int i = 4 * tid; i < (1 << jfrom); i += 4 * nthr) cp16(P1 + i, ib + i);
    cp_commit();
    cp_wait<0>();
    __syncthreads();
    src = P1;
  }
  float* dst = P0;
  for (int j = jfrom - 1; j >= J0; --j) {
    const int n0 = 1 << j;
    float* lo_out = j == J0 ? xb : dst;
    if (n0 / 4 >= nthr && j > J0) {   // groups of 4 pairs once they fill the CTA
      for (int g = tid; g < n0 / 4; g += nthr) ana_group<PM>(src, lo_out, xb + n0, n0, g, true, tp, st, G);
    } else {
      Plain<float> sa{src};
      for (int m = tid; m < n0; m += nthr) {
        float lo, hi;
        ana_one<float>(m, n0, sa, st, G, lo, hi);
        lo_out[m] = lo;
        xb[n0 + m] = hi;
      }
    }
    __syncthreads();
    src = dst;
    dst = dst == P0 ? P1 : P0;
  }
}

// one level over a batch of lines, a group of outputs per thread
template <int PM>
__global__ void __launch_bounds__(256) k_syn1d_level_f32(const float* __restrict__ lo, int64_t lo_bs,
                                                         const float* __restrict__ hi, int64_t hi_bs,
                                                         float* __restrict__ out, int64_t out_bs, int n0, HGTaps<PM> tp,
                                                         Tables<float> tab, Geo G, int batch) {
  pdl_trigger();
  pdl_wait();
  const int per = (2 * n0) / 8;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = idx < (int64_t)batch * per;     // whole warps take part in the edge rounds
  const int64_t b = valid ? idx / per : 0;
  syn_group<PM>(lo + b * lo_bs, hi + b * hi_bs, out + b * out_bs, n0, valid ? (int)(idx - b * per) : 0, valid, tp, tab,
                G);
}

template <int PM>
__global__ void __launch_bounds__(256) k_ana1d_level_f32(const float* __restrict__ in, int64_t in_bs,
                                                         float* __restrict__ lo, int64_t lo_bs, float* __restrict__ hi,
                                                         int64_t hi_bs, int n0, HGTaps<PM> tp, Tables<float> tab, Geo G,
                                                         int batch) {
  pdl_trigger();
  pdl_wait();
  const int per = n0 / 4;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = idx < (int64_t)batch * per;     // whole warps take part in the edge rounds
  const int64_t b = valid ? idx / per : 0;
  ana_group<PM>(in + b * in_bs, lo + b * lo_bs, hi + b * hi_bs, n0, valid ? (int)(idx - b * per) : 0, valid, tp, tab,
                G);
}

}  // namespace f32k

bool f32_eligible(const Plan& P, const LineIO& io, const void* in, const void* out, bool fwd) {
  if (!P.f32.ok || io.jlev != P.R - 1) return false;
  if (P.N != 2048 && P.N != 4096) return false;
  if (P.Q != 2 && P.Q != 4) return false;
  if (P.f32.K > 0 && !P.d_f32) return false;
  const int NT = P.N / 16;
  if (P.f32.K / 16 > NT / 2) return false;
  if (P.M / 2 < 16) return false;
  if (io.mode == 1 && !io.pos) return false;
  auto al16 = [](const void* q) { return ((uintptr_t)q & 15u) == 0; };
  if (fwd) {
    if (!al16(in) || io.in_stride % 4 || io.in_batch % 4) return false;
    if (io.mode == 0 && (!al16(out) || io.out_stride % 4 || io.out_batch % 4)) return false;
  } else {
    if (io.mode == 0 && (!al16(in) || io.in_stride % 4 || io.in_batch % 4)) return false;
    if (!al16(out) || io.out_stride % 4 || io.out_batch % 4) return false;
  }
  return true;
}

// long 1D lines on FP32: T with the Walsh-Hadamard stages of bits 0-11 per
// segment of 4096 (forward), those stages alone (adjoint), and T^T
bool f32_seg_eligible(const Plan& P) {
  return (P.Q == 2 || P.Q == 4) && P.N >= 2 * f32k::SEGN && P.M >= 16 && P.M % 4 == 0;
}

template <typename F>
static cudaError_t f32_pm_dispatch(const Plan& P, F&& f) {
  if (P.p <= 4) return P.Q == 2 ? f(std::integral_constant<int, 4>{}, std::integral_constant<int, 2>{})
                                 : f(std::integral_constant<int, 4>{}, std::integral_constant<int, 4>{});
  if (P.p <= 8) return P.Q == 2 ? f(std::integral_constant<int, 8>{}, std::integral_constant<int, 2>{})
                                 : f(std::integral_constant<int, 8>{}, std::integral_constant<int, 4>{});
  return P.Q == 2 ? f(std::integral_constant<int, 10>{}, std::integral_constant<int, 2>{})
                  : f(std::integral_constant<int, 10>{}, std::integral_constant<int, 4>{});
}

cudaError_t f32_seg_up(const Plan& P, const Geo& G, const float* s, float* v, int batch, cudaStream_t st) {
  const int segs = P.N / f32k::SEGN;
  return f32_pm_dispatch(P, [&](auto pm, auto q) {
    constexpr int PM = decltype(pm)::value, Q = decltype(q)::value;
    return launch_pdl(f32k::k_up_seg<PM, Q>, dim3((unsigned)(batch * segs)), dim3(f32k::SEGNT), 0, st, s, v,
                      f32k::make_taps<PM, Q>(P), P.t32, G, segs);
  });
}


template <int PM, int Q>
static f32k::TapsT<PM, Q> make_tapsT(const Plan& P) {
  f32k::TapsT<PM, Q> t;
  float* tv = reinterpret_cast<float*>(t.t2);
  const int p = P.p;
  const double sc = std::exp2(-0.5 * P.R);
  for (int i = 0; i < (2 * PM - 1) * Q; ++i) {
    const int tt = (1 - PM) * Q + i;                    // tap position
    const bool in = tt >= (1 - p) * Q && tt < p * Q;
    tv[i] = in ? (float)(sc * P.taps[tt + (p - 1) * Q]) : 0.f;
  }
  return t;
}

// the adjoint's segment stages (bits 0-11) fused with T^T for every
// segment's interior outputs, then the boundary outputs
cudaError_t f32_seg_fwht_upT(const Plan& P, const Geo& G, float* v, float* s, int batch, cudaStream_t st) {
  const int segs = P.N / f32k::SEGN;
  return f32_pm_dispatch(P, [&](auto pm, auto q) {
    constexpr int PM = decltype(pm)::value, Q = decltype(q)::value;
    constexpr int NTS = f32k::SEG64;
    cudaError_t e = launch_pdl(f32k::k_fwht_seg64_upT<PM, Q>, dim3((unsigned)(batch * segs)), dim3(NTS), 0, st, v,
                               s, make_tapsT<PM, Q>(P), G, segs);
    if (e != cudaSuccess) return e;
    const int64_t n = (int64_t)batch * segs * 2 * f32k::SegUT<PM, Q>::NB;
    return launch_pdl(f32k::k_seg_upT_fix<PM, Q>, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, st,
                      (const float*)v, s, P.t32, G, segs, batch);
  });
}


template <int PM>
static f32k::HGTaps<PM> make_hg(const Plan& P) {
  f32k::HGTaps<PM> t;
  const int p = P.p;
  auto hf = [&](int l) { return (l >= -p + 1 && l <= p) ? (float)P.h[l + p - 1] : 0.f; };
  auto gf = [&](int l) { return (l >= -p + 1 && l <= p) ? (float)P.g[l + p - 1] : 0.f; };
  for (int d = -PM / 2; d <= PM / 2; ++d) {
    t.hp2[d + PM / 2] = make_float2(hf(2 * d), hf(2 * d + 1));
    t.gp2[d + PM / 2] = make_float2(gf(2 * d), gf(2 * d + 1));
  }
  return t;
}

template <typename F>
static cudaError_t hg_dispatch(const Plan& P, F&& f) {
  if (P.p <= 4) return f(std::integral_constant<int, 4>{});
  if (P.p <= 8) return f(std::integral_constant<int, 8>{});
  return f(std::integral_constant<int, 10>{});
}

cudaError_t f32_syn1d_levels(const Plan& P, const Geo& G, const float* x, float* out, int jto, size_t smem, int batch,
                             cudaStream_t st) {
  return hg_dispatch(P, [&](auto pm) {
    constexpr int PM = decltype(pm)::value;
    auto kern = f32k::k_syn1d_levels_f32<PM>;
    // room for the last level's details as well: stage them in shared memory
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t add = sizeof(float) << (jto - 1);
    const int stage = smem + add <= (size_t)optin && ((uintptr_t)x & 15u) == 0 && P.M % 4 == 0 && jto >= 3;
    const size_t sm = stage ? smem + add : smem;
    cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    return launch_pdl(kern, dim3(batch), dim3(1024), sm, st, x, out, (int64_t)P.M, make_hg<PM>(P), P.t32, G, P.J0,
                      jto, (int64_t)P.M, stage);
  });
}

cudaError_t f32_ana1d_levels(const Plan& P, const Geo& G, const float* in, float* x, int jfrom, size_t smem,
                             int batch, cudaStream_t st) {
  return hg_dispatch(P, [&](auto pm) {
    constexpr int PM = decltype(pm)::value;
    auto kern = f32k::k_ana1d_levels_f32<PM>;
    // room for the whole input line: stage it in shared memory
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t add = sizeof(float) << (jfrom - 1);
    const int stage = smem + add <= (size_t)optin && ((uintptr_t)in & 15u) == 0 && P.M % 4 == 0 && jfrom >= 2;
    const size_t sm = stage ? smem + add : smem;
    cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    return launch_pdl(kern, dim3(batch), dim3(1024), sm, st, in, (int64_t)P.M, x, make_hg<PM>(P), P.t32, G, P.J0,
                      jfrom, (int64_t)P.M, stage);
  });
}

cudaError_t f32_syn1d_level(const Plan& P, const Geo& G, const float* lo, const float* hi, float* out, int n0, int batch,
                            cudaStream_t st) {
  const int64_t threads = (int64_t)batch * (2 * n0 / 8);
  return hg_dispatch(P, [&](auto pm) {
    constexpr int PM = decltype(pm)::value;
    return launch_pdl(f32k::k_syn1d_level_f32<PM>, dim3((unsigned)((threads + 255) / 256)), dim3(256), 0, st, lo,
                      (int64_t)P.M, hi, (int64_t)P.M, out, (int64_t)P.M, n0, make_hg<PM>(P), P.t32, G, batch);
  });
}

cudaError_t f32_ana1d_level(const Plan& P, const Geo& G, const float* in, float* lo, float* hi, int n0, int batch,
                            cudaStream_t st) {
  const int64_t threads = (int64_t)batch * (n0 / 4);
  return hg_dispatch(P, [&](auto pm) {
    constexpr int PM = decltype(pm)::value;
    return launch_pdl(f32k::k_ana1d_level_f32<PM>, dim3((unsigned)((threads + 255) / 256)), dim3(256), 0, st, in,
                      (int64_t)P.M, lo, (int64_t)P.M, hi, (int64_t)P.M, n0, make_hg<PM>(P), P.t32, G, batch);
  });
}

cudaError_t f32_launch(bool fwd, const Plan& P, const float* in, float* out, const LineIO& io, int total,
                       cudaStream_t s) {
  if (P.N == 4096) return f32k::go_nt<256>(fwd, P, in, out, io, total, s);
  return f32k::go_nt<128>(fwd, P, in, out, io, total, s);
}

}  // namespace uw
