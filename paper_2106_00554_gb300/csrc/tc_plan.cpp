// Host construction (FP64) of the block matrices of the split-BF16
// tensor-core line operators (kernels_tc.cu).
//
// The last synthesis level, the upsample-convolve T (Sec. 4.1 cell integrals)
// and the first four Walsh-Hadamard stages (Sec. 3.1, natural order, bits 0-3)
// are one linear map from a window of lo / hi coefficients to 16 consecutive
// outputs.  Away from the VMP boundaries it is the same matrix for every
// block (the interior two-scale and tap formulas are shift invariant), so the
// device applies it as a GEMM against im2col windows.  The adjoint applies the
// transposed map (Sec. 4.2) per block of 8 lo and 8 hi outputs.  Blocks that
// touch a VMP boundary function use dense matrices built here from the exact
// line operator (the formulas of Sec. 3.2 and 4.1 applied to unit vectors).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "uw_internal.h"

namespace uw {
namespace {

int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
int ceildiv(int a, int b) { return -floordiv(-a, b); }
int up16(int a) { return (a + 15) / 16 * 16; }
int up32(int a) { return (a + 31) / 32 * 32; }
int hsign(int a, int b) { return (__builtin_popcount((unsigned)(a & b)) & 1) ? -1 : 1; }

uint16_t bf16_rn(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;
  return (uint16_t)((u + 0x7fffu + ((u >> 16) & 1u)) >> 16);
}
float bf16_f(uint16_t b) {
  uint32_t u = (uint32_t)b << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
uint32_t fbits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
}

// The exact last-level line operator of one plan in FP64: the per-output
// formulas of the GPU FP64 path (synthesis with the boundary blocks, T with
// the boundary rows, their transposes), whole lines at a time.
struct Exact {
  const Plan& P;
  int p, Q, n0, M, N, Lb, ntap, tmin;
  double sc;
  bool per;
  explicit Exact(const Plan& pl)
      : P(pl), p(pl.p), Q(pl.Q), n0(pl.M / 2), M(pl.M), N(pl.N), Lb(pl.Lb), ntap(pl.ntap), tmin(-(pl.p - 1) * pl.Q),
        sc(std::exp2(-0.5 * pl.R)), per(pl.bd == UW_BOUNDARY_PERIODIC) {}
  static int wrap(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
  }
  void syn(const std::vector<double>& lo, const std::vector<double>& hi, std::vector<double>& s) const {
    s.assign(M, 0.0);
    for (int k = 0; k < M; ++k) {
      double acc = 0;
      if (per) {
        for (int l = -p + 1; l <= p; ++l) {
          int km = wrap(k - l, M);
          if (km & 1) continue;
          acc += P.h[l + p - 1] * lo[km >> 1] + P.g[l + p - 1] * hi[km >> 1];
        }
      } else {
        int mlo = std::max(p, ceildiv(k - p, 2)), mhi = std::min(n0 - p - 1, floordiv(k + p - 1, 2));
        for (int m = mlo; m <= mhi; ++m) acc += P.h[k - 2 * m + p - 1] * lo[m] + P.g[k - 2 * m + p - 1] * hi[m];
        if (k < Lb)
          for (int m = 0; m < p; ++m) acc += P.PL[m * Lb + k] * lo[m] + P.QL[m * Lb + k] * hi[m];
        int c = M - 1 - k;
        if (c < Lb)
          for (int r = 0; r < p; ++r) acc += P.PR[r * Lb + c] * lo[n0 - 1 - r] + P.QR[r * Lb + c] * hi[n0 - 1 - r];
      }
      s[k] = acc;
    }
  }
  void up(const std::vector<double>& s, std::vector<double>& v) const {
    v.assign(N, 0.0);
    for (int k = 0; k < N; ++k) {
      double acc = 0;
      for (int m = ceildiv(k - (p * Q - 1), Q); m <= floordiv(k - tmin, Q); ++m) {
        double tap = P.taps[k - Q * m - tmin];
        if (per) acc += tap * s[wrap(m, M)];
        else if (m >= p && m <= M - p - 1) acc += tap * s[m];
      }
      if (!per) {
        if (k < ntap)
          for (int m = 0; m < p; ++m) acc += P.EL[m * ntap + k] * s[m];
        int kk = N - 1 - k;
        if (kk < ntap)
          for (int r = 0; r < p; ++r) acc += P.ER[r * ntap + kk] * s[M - 1 - r];
      }
      v[k] = sc * acc;
    }
  }
  void upT(const std::vector<double>& v, std::vector<double>& s) const {
    s.assign(M, 0.0);
    for (int m = 0; m < M; ++m) {
      double acc = 0;
      if (per) {
        for (int i = 0; i < ntap; ++i) acc += P.taps[i] * v[wrap(Q * m + tmin + i, N)];
      } else if (m < p) {
        for (int k = 0; k < ntap; ++k) acc += P.EL[m * ntap + k] * v[k];
      } else if (m >= M - p) {
        int r = M - 1 - m;
        for (int kk = 0; kk < ntap; ++kk) acc += P.ER[r * ntap + kk] * v[N - 1 - kk];
      } else {
        for (int i = 0; i < ntap; ++i) acc += P.taps[i] * v[Q * m + tmin + i];
      }
      s[m] = sc * acc;
    }
  }
  void ana(const std::vector<double>& s, std::vector<double>& lo, std::vector<double>& hi) const {
    lo.assign(n0, 0.0);
    hi.assign(n0, 0.0);
    for (int m = 0; m < n0; ++m) {
      double a = 0, b = 0;
      if (per) {
        for (int l = -p + 1; l <= p; ++l) {
          double v = s[wrap(2 * m + l, M)];
          a += P.h[l + p - 1] * v;
          b += P.g[l + p - 1] * v;
        }
      } else if (m < p) {
        for (int c = 0; c < Lb; ++c) {
          a += P.PL[m * Lb + c] * s[c];
          b += P.QL[m * Lb + c] * s[c];
        }
      } else if (m >= n0 - p) {
        int r = n0 - 1 - m;
        for (int c = 0; c < Lb; ++c) {
          a += P.PR[r * Lb + c] * s[M - 1 - c];
          b += P.QR[r * Lb + c] * s[M - 1 - c];
        }
      } else {
        for (int l = -p + 1; l <= p; ++l) {
          a += P.h[l + p - 1] * s[2 * m + l];
          b += P.g[l + p - 1] * s[2 * m + l];
        }
      }
      lo[m] = a;
      hi[m] = b;
    }
  }
  // The interior formulas applied to the whole line with zero padding
  // beyond its ends (what the FP32 line kernels compute before their edge
  // corrections): synthesis with h, g for every coefficient index in
  // [0, n0), T with the taps for every s index in [0, M).
  void syn_int0(const std::vector<double>& lo, const std::vector<double>& hi, std::vector<double>& s) const {
    s.assign(M, 0.0);
    for (int k = 0; k < M; ++k) {
      double acc = 0;
      for (int l = -p + 1; l <= p; ++l) {
        const int km = k - l;
        if (km & 1) continue;
        const int i = km / 2;
        if (i < 0 || i >= n0) continue;
        acc += P.h[l + p - 1] * lo[i] + P.g[l + p - 1] * hi[i];
      }
      s[k] = acc;
    }
  }
  void up_int0(const std::vector<double>& s, std::vector<double>& v) const {
    v.assign(N, 0.0);
    for (int k = 0; k < N; ++k) {
      double acc = 0;
      for (int m = ceildiv(k - (p * Q - 1), Q); m <= floordiv(k - tmin, Q); ++m)
        if (m >= 0 && m < M) acc += P.taps[k - Q * m - tmin] * s[m];
      v[k] = sc * acc;
    }
  }
  // interior entry of the line matrix: d v[k] / d lo[i] (hi = false) or
  // d v[k] / d hi[i] (hi = true), any integers k, i (shift invariant)
  double interior(int k, int i, bool hi) const {
    double acc = 0;
    for (int m = ceildiv(k - (p * Q - 1), Q); m <= floordiv(k - tmin, Q); ++m) {
      int l = m - 2 * i;
      if (l < -p + 1 || l > p) continue;
      acc += P.taps[k - Q * m - tmin] * (hi ? P.g[l + p - 1] : P.h[l + p - 1]);
    }
    return sc * acc;
  }
};

// A (16 x 16 KS, row major, double) -> fragment-ordered BF16 parts of the
// m16n8k16 A operand, A = A1 + A2 + A3 + O(2^-27 |A|) (each part the BF16
// rounding of what the previous ones leave): per k-step and lane the words
// a0..a3 of A1, then of A2, then of A3; a register holds columns (2t, 2t+1)
// of row g (a0), g+8 (a1), and the same with columns + 8 (a2, a3); the lower
// 16 bits hold the lower column.
void pack_a(const std::vector<double>& A, int KS, std::vector<uint32_t>& w) {
  const int K = 16 * KS;
  for (int ks = 0; ks < KS; ++ks)
    for (int lane = 0; lane < 32; ++lane) {
      const int g = lane >> 2, t = lane & 3;
      const int rows[4] = {g, g + 8, g, g + 8};
      const int cols[4] = {2 * t, 2 * t, 2 * t + 8, 2 * t + 8};
      uint32_t part[3][4];
      for (int r = 0; r < 4; ++r) {
        uint16_t b[3][2];
        for (int e = 0; e < 2; ++e) {
          double rest = A[(size_t)rows[r] * K + 16 * ks + cols[r] + e];
          for (int s = 0; s < 3; ++s) {
            b[s][e] = bf16_rn((float)rest);
            rest -= (double)bf16_f(b[s][e]);
          }
        }
        for (int s = 0; s < 3; ++s) part[s][r] = (uint32_t)b[s][0] | ((uint32_t)b[s][1] << 16);
      }
      for (int s = 0; s < 3; ++s)
        for (int r = 0; r < 4; ++r) w.push_back(part[s][r]);
    }
}

}  // namespace

void build_tc(Plan& P, std::vector<uint32_t>& words) {
  words.clear();
  TcGeo& G = P.tc;
  G = TcGeo{};
  const int p = P.p, Q = P.Q, N = P.N, M = P.M, n0 = M / 2;
  int L = 0;
  while ((1 << L) < N) ++L;
  if ((Q != 2 && Q != 4) || L < 9 || L > 13 || p > 10) return;
  const bool per = P.bd == UW_BOUNDARY_PERIODIC;
  const int tmin = -(p - 1) * Q, tmax = p * Q - 1;
  Exact X(P);

  // forward window (block n = 0): coefficients [imin, imax] reach its outputs
  const int S0 = ceildiv(-tmax, Q), S1 = floordiv(15 - tmin, Q);
  const int imin = ceildiv(S0 - p, 2), imax = floordiv(S1 + p - 1, 2);
  G.bs = 8 / Q;
  G.W0 = -imin + ((-imin) & 1);                // even, so 32-bit pairs stay aligned
  G.lw = imax + G.W0 + 1;
  G.KS = (2 * G.lw + 15) / 16;
  G.lw = 8 * G.KS;                             // window padded with zero weights: 2 lw = 16 KS
  G.HL = 16;
  G.HR = 16;
  if (G.W0 > G.HL || G.lw - G.W0 - G.bs > G.HR || G.KS > 3) return;
  const int nb = N / 16;

  // adjoint window (block c = 0: outputs lo / hi [0, 8))
  const int kmin = Q * (-p + 1) + tmin, kmax = Q * (14 + p) + tmax;
  G.W1 = up16(-kmin);
  G.KSA = (kmax + G.W1 + 16) / 16;
  G.HLa = G.W1;                                // window starts are then multiples of 32 elements
  G.HRa = up32(std::max(0, 16 * G.KSA - 16 * Q - G.W1));
  if (G.KSA > 16) return;
  const int nbA = n0 / 8;

  // boundary blocks (VMP): a forward block is interior when every coefficient
  // and every s value it reads is an interior one; an adjoint block when its
  // outputs are interior coefficients
  if (!per) {
    auto fwd_interior = [&](int n) {
      const int a = G.bs * n + imin, b = G.bs * n + imax;
      const int s0 = 16 * n / Q + S0, s1 = 16 * n / Q + S1;
      return a >= p && b <= n0 - p - 1 && s0 >= P.Lb && s1 <= M - 1 - P.Lb && 16 * n >= P.ntap &&
             16 * n + 15 <= N - 1 - P.ntap;
    };
    int lo = 0;
    while (lo < nb && !fwd_interior(lo)) ++lo;
    int hi = nb - 1;
    while (hi >= 0 && !fwd_interior(hi)) --hi;
    if (lo > hi) return;
    for (int n = lo; n <= hi; ++n)
      if (!fwd_interior(n)) return;
    G.EBl = lo;
    G.EBr = nb - 1 - hi;
    const int reach_l = std::max(G.bs * (G.EBl - 1) + imax, p - 1) + 1;
    const int reach_r = n0 - std::min(G.bs * (nb - G.EBr) + imin, n0 - p);
    G.Xl = std::min(n0, std::max(reach_l, reach_r));
    if ((G.Xl + 3) / 4 * 4 > n0) return;
    G.EAl = (p + 7) / 8;
    G.EAr = (p + 7) / 8;
    if (G.EAl + G.EAr >= nbA) return;
    const int smax = std::max(2 * (8 * G.EAl - 1) + p, P.Lb - 1);
    G.Wl = up16(std::max(Q * smax + tmax, P.ntap - 1) + 1);
    if (2 * G.Wl > N) return;
  }

  // interior block matrices
  const int K = 16 * G.KS, KA = 16 * G.KSA;
  std::vector<double> Araw(16 * K, 0.0), A(16 * K, 0.0);
  for (int r = 0; r < 16; ++r)
    for (int c = 0; c < 2 * G.lw; ++c) {
      const bool hi = c >= G.lw;
      Araw[r * K + c] = X.interior(r, (c % G.lw) - G.W0, hi);
    }
  for (int r = 0; r < 16; ++r)
    for (int c = 0; c < K; ++c) {
      double a = 0;
      for (int rr = 0; rr < 16; ++rr) a += hsign(r, rr) * Araw[rr * K + c];
      A[r * K + c] = a;
    }
  std::vector<double> Braw(16 * KA, 0.0), B(16 * KA, 0.0);
  for (int o = 0; o < 16; ++o)
    for (int kk = 0; kk < KA; ++kk) Braw[o * KA + kk] = X.interior(kk - G.W1, o & 7, o >= 8);
  for (int o = 0; o < 16; ++o)
    for (int kk = 0; kk < KA; ++kk) {
      const int j = kk / 16, r = kk % 16;
      double a = 0;
      for (int rr = 0; rr < 16; ++rr) a += Braw[o * KA + 16 * j + rr] * hsign(rr, r);
      B[o * KA + kk] = a;
    }

  G.oAf = (int64_t)words.size();
  pack_a(A, G.KS, words);
  G.oAa = (int64_t)words.size();
  pack_a(B, G.KSA, words);

  // boundary matrices, stored input-major: E[c * rows + o]
  if (!per) {
    std::vector<double> lo(n0), hi(n0), s, v, u(N);
    // forward: rows (left blocks, then right blocks) of 16 outputs; a row
    // holds X4 lo then X4 hi coefficient weights (window [0, X4) on the left,
    // [n0 - X4, n0) on the right), padded to the stride SF
    const int X4 = (G.Xl + 3) / 4 * 4;
    G.Xl = X4;
    G.SF = 2 * X4 + 4;
    const int Rf = 16 * (G.EBl + G.EBr);
    std::vector<double> Ef((size_t)Rf * G.SF, 0.0);
    for (int side = 0; side < 2; ++side) {
      const bool left = side == 0;
      const int EB = left ? G.EBl : G.EBr, row0 = left ? 0 : 16 * G.EBl;
      for (int c = 0; c < 2 * X4; ++c) {
        std::fill(lo.begin(), lo.end(), 0.0);
        std::fill(hi.begin(), hi.end(), 0.0);
        const int i = (c % X4) + (left ? 0 : n0 - X4);
        (c < X4 ? lo : hi)[i] = 1.0;
        X.syn(lo, hi, s);
        X.up(s, v);
        for (int o = 0; o < 16 * EB; ++o) {
          const int blk = (left ? 0 : nb - EB) + o / 16, r = o % 16;
          double a = 0;
          for (int rr = 0; rr < 16; ++rr) a += hsign(r, rr) * v[16 * blk + rr];
          Ef[(size_t)(row0 + o) * G.SF + c] = a;
        }
      }
    }
    while (words.size() % 4) words.push_back(0);   // 16-byte aligned rows on the device
    G.oEf = (int64_t)words.size();
    for (double e : Ef) words.push_back(fbits((float)e));
    // adjoint: rows (left blocks, then right blocks) of 8 lo and 8 hi
    // outputs; a row holds the weights of the samples [0, Wl) on the left,
    // [N - Wl, N) on the right (before the bits 0-3 transform), stride SA
    G.SA = G.Wl + 4;
    const int Ra = 16 * (G.EAl + G.EAr);
    std::vector<double> Ea((size_t)Ra * G.SA, 0.0);
    for (int side = 0; side < 2; ++side) {
      const bool left = side == 0;
      const int EA = left ? G.EAl : G.EAr, row0 = left ? 0 : 16 * G.EAl;
      for (int kk = 0; kk < G.Wl; ++kk) {
        std::fill(u.begin(), u.end(), 0.0);
        const int kq = left ? kk : N - G.Wl + kk;
        std::vector<double> vv(N, 0.0);
        const int blk = kq / 16;
        for (int r = 0; r < 16; ++r) vv[16 * blk + r] = hsign(r, kq % 16);
        X.upT(vv, s);
        X.ana(s, lo, hi);
        for (int o = 0; o < 16 * EA; ++o) {
          const int c = (left ? 0 : nbA - EA) + o / 16, r = o % 16;
          Ea[(size_t)(row0 + o) * G.SA + kk] = r < 8 ? lo[8 * c + r] : hi[8 * c + r - 8];
        }
      }
    }
    while (words.size() % 4) words.push_back(0);
    G.oEa = (int64_t)words.size();
    for (double e : Ea) words.push_back(fbits((float)e));
  }
  G.words = (int64_t)words.size();
  G.ok = 1;
}

// Edge corrections of the FP32 line operators: C = E_exact - E_int0 on the
// columns of the p lo and p hi coefficients at each end, where E maps the
// coefficient line to v = T Syn x.  Every other column of the difference is
// zero (an interior coefficient reaches only interior s values through the
// interior filters, Sec. 3.2, and those meet only interior taps, Sec. 4.1);
// the construction checks that on the next columns and finds the rows K
// where the difference lives.
void build_f32(Plan& P, std::vector<float>& out) {
  out.clear();
  F32Geo& F = P.f32;
  F = F32Geo{};
  const int p = P.p, n0 = P.M / 2, N = P.N;
  if (P.bd == UW_BOUNDARY_PERIODIC) {
    F.ok = 1;
    return;
  }
  const int extra = 4;                 // columns past the edge that must show no difference
  const int Wc = p + extra;
  if (n0 < 2 * Wc + 8) return;
  Exact X(P);
  std::vector<double> lo(n0), hi(n0), s, ve, vi;
  // D[side][col][k]: col < Wc lo columns, then Wc hi columns
  std::vector<std::vector<std::vector<double>>> D(2, std::vector<std::vector<double>>(2 * Wc));
  double dmax = 0;
  for (int side = 0; side < 2; ++side)
    for (int c = 0; c < 2 * Wc; ++c) {
      std::fill(lo.begin(), lo.end(), 0.0);
      std::fill(hi.begin(), hi.end(), 0.0);
      const int i = side == 0 ? c % Wc : n0 - 1 - (c % Wc);
      (c < Wc ? lo : hi)[i] = 1.0;
      X.syn(lo, hi, s);
      X.up(s, ve);
      X.syn_int0(lo, hi, s);
      X.up_int0(s, vi);
      auto& d = D[side][c];
      d.resize(N);
      for (int k = 0; k < N; ++k) {
        d[k] = ve[k] - vi[k];
        dmax = std::max(dmax, std::fabs(d[k]));
      }
    }
  if (dmax == 0) {   // the boundary functions are interior ones cut at the ends (p = 1): no correction
    F.ok = 1;
    return;
  }
  const double tol = 1e-12 * dmax;
  int K = 0;
  for (int side = 0; side < 2; ++side)
    for (int c = 0; c < 2 * Wc; ++c) {
      const bool edge_col = (c % Wc) < p;
      for (int k = 0; k < N; ++k) {
        const double a = std::fabs(D[side][c][k]);
        if (a <= tol) continue;
        if (!edge_col) return;          // a difference outside the edge columns: not this structure
        const int r = side == 0 ? k : N - 1 - k;
        K = std::max(K, r + 1);
      }
    }
  K = (K + 15) / 16 * 16;
  if (K == 0 || 2 * K > N) return;
  F.K = K;
  F.CS = (2 * p + 3) / 4 * 4;
  out.assign((size_t)2 * K * F.CS, 0.f);
  for (int side = 0; side < 2; ++side)
    for (int r = 0; r < K; ++r)
      for (int c = 0; c < 2 * p; ++c) {
        // columns: lo[0..p), hi[0..p) on the left; lo[n0-p..n0), hi[n0-p..n0) on the right
        const int e = c % p, half = c / p;
        const int col = side == 0 ? half * Wc + e : half * Wc + (p - 1 - e);
        const int k = side == 0 ? r : N - K + r;
        out[((size_t)side * K + r) * F.CS + c] = (float)D[side][col][k];
      }
  F.words = (int64_t)out.size();
  F.ok = 1;
}

// Operators of the tcgen05 line kernels (UmmaGeo in uw_internal.h).  With
// q = 1 the interior map from the coefficients to the outputs of T is shift
// invariant under (k, i) -> (k + 32, i + 8), so one 32 x 48 matrix B1 serves
// every block of 32 outputs: B1[r][j] = sum_r' H32[r][r'] d v[r'] / d x[i_j],
// i_j = j - 8 (lo) or j - 32 (hi), folding the Walsh-Hadamard stages of bits
// 0-4 (natural order, Sec. 3.1) into the last synthesis level and T (Sec. 3.2,
// 4.1).  The window [-8, 16) must hold every i the interior map reaches
// (p <= 9); this is checked.
namespace {

// K-major canonical layout of a rows x K BF16 operand without swizzling:
// core matrix (row / 8, k / 8) at ((row / 8) (K / 8) + k / 8) 64 elements,
// inside it row % 8 then k % 8
void pack_kmajor3(const std::vector<double>& A, int rows, int K, uint16_t* out) {
  for (int part = 0; part < 3; ++part)
    for (int r = 0; r < rows; ++r)
      for (int k = 0; k < K; ++k) {
        double x = A[(size_t)r * K + k];
        uint16_t b1 = bf16_rn((float)x);
        double r1 = x - (double)bf16_f(b1);
        uint16_t b2 = bf16_rn((float)r1);
        double r2 = r1 - (double)bf16_f(b2);
        uint16_t b3 = bf16_rn((float)r2);
        const uint16_t b = part == 0 ? b1 : (part == 1 ? b2 : b3);
        out[(size_t)part * rows * K + ((size_t)(r / 8) * (K / 8) + k / 8) * 64 + (r % 8) * 8 + k % 8] = b;
      }
}

}  // namespace

void build_umma(Plan& P, std::vector<unsigned char>& bytes) {
  bytes.clear();
  UmmaGeo& U = P.umma;
  U = UmmaGeo{};
  if (P.Q != 2 || P.N != 4096 || P.p > 9) return;
  const int p = P.p, n0 = P.M / 2, N = P.N;
  Exact X(P);
  // window coverage: every interior entry of the first block lies in the window
  for (int r = 0; r < 32; ++r)
    for (int i = -3 * p - 8; i < 3 * p + 24; ++i) {
      if (i >= -8 && i < 16) continue;
      if (X.interior(r, i, false) != 0.0 || X.interior(r, i, true) != 0.0) return;
    }
  auto hs = [](int a, int b) { return (__builtin_popcount((unsigned)(a & b)) & 1) ? -1.0 : 1.0; };
  std::vector<double> B1(32 * 48), B1t(48 * 32);
  for (int r = 0; r < 32; ++r)
    for (int j = 0; j < 48; ++j) {
      const bool hi = j >= 24;
      const int i = hi ? j - 32 : j - 8;
      double acc = 0;
      for (int r2 = 0; r2 < 32; ++r2) acc += hs(r, r2) * X.interior(r2, i, hi);
      B1[(size_t)r * 48 + j] = acc;
      B1t[(size_t)j * 32 + r] = acc;
    }
  // VMP corrections: exact minus the windowed interior map (zero padding
  // beyond the coefficient range), for unit vectors at the edge columns; a
  // few columns past the edge must show no difference
  int KB = 0;
  std::vector<std::vector<std::vector<double>>> D;
  if (P.bd != UW_BOUNDARY_PERIODIC) {
    const int Wc = p + 4;
    if (n0 < 2 * Wc + 16) return;
    D.assign(2, std::vector<std::vector<double>>(2 * Wc, std::vector<double>(N, 0.0)));
    std::vector<double> lo(n0), hi(n0), s, ve;
    double dmax = 0;
    for (int side = 0; side < 2; ++side)
      for (int c = 0; c < 2 * Wc; ++c) {
        std::fill(lo.begin(), lo.end(), 0.0);
        std::fill(hi.begin(), hi.end(), 0.0);
        const int i = side == 0 ? c % Wc : n0 - 1 - (c % Wc);
        const bool h = c >= Wc;
        (h ? hi : lo)[i] = 1.0;
        X.syn(lo, hi, s);
        X.up(s, ve);
        for (int k = 0; k < N; ++k) {
          const double d = ve[k] - X.interior(k, i, h);
          D[side][c][k] = d;
          dmax = std::max(dmax, std::fabs(d));
        }
      }
    // differences below 1e-12 of the operator's own scale are rounding (the
    // exact and the windowed maps round differently), not structure
    double bmax = 0;
    for (double v : B1) bmax = std::max(bmax, std::fabs(v));
    const double tol = 1e-12 * bmax;
    (void)dmax;
    int K = 0;
    for (int side = 0; side < 2; ++side)
      for (int c = 0; c < 2 * Wc; ++c)
        for (int k = 0; k < N; ++k) {
          if (std::fabs(D[side][c][k]) <= tol) continue;
          if ((c % Wc) >= p) return;            // a difference outside the edge columns
          K = std::max(K, (side == 0 ? k : N - 1 - k) + 1);
        }
    KB = (K + 31) / 32;
    if (2 * KB > 128) return;
  }
  U.KB = KB;
  const size_t nb = 3 * 1536;                   // bf16 values per operator
  U.oF = 0;
  U.oA = (int64_t)nb;
  const size_t corr_floats = (size_t)2 * KB * 32 * 2 * p;
  U.oC = (int64_t)(2 * nb * sizeof(uint16_t) / sizeof(float));
  U.bytes = (int64_t)(2 * nb * sizeof(uint16_t) + corr_floats * sizeof(float));
  bytes.assign((size_t)U.bytes, 0);
  uint16_t* w = reinterpret_cast<uint16_t*>(bytes.data());
  pack_kmajor3(B1, 32, 48, w + U.oF);
  pack_kmajor3(B1t, 48, 32, w + U.oA);
  if (KB) {
    float* C = reinterpret_cast<float*>(bytes.data()) + U.oC;
    const int Wc = p + 4;
    for (int side = 0; side < 2; ++side)
      for (int row = 0; row < KB * 32; ++row) {
        const int bb = row / 32, r = row % 32;
        for (int c = 0; c < 2 * p; ++c) {
          // columns: lo[0..p), hi[0..p) on the left; lo[n0-p..n0), hi[n0-p..n0) on the right
          const int e = c % p, half = c / p;
          const int col = side == 0 ? half * Wc + e : half * Wc + (p - 1 - e);
          const int k0 = side == 0 ? 32 * bb : N - 32 * KB + 32 * bb;
          double acc = 0;
          for (int r2 = 0; r2 < 32; ++r2) acc += hs(r, r2) * D[side][col][k0 + r2];
          C[((size_t)side * KB * 32 + row) * 2 * p + c] = (float)acc;
        }
      }
  }
  U.ok = 1;
}

// Edge corrections of one 2D Mallat level (the coarse-level kernels): the
// exact VMP synthesis of a level (Sec. 3.2: interior two-scale relations plus
// the level-independent boundary blocks) differs from the interior formula
// with zero padding only in the first / last Lb outputs, and only through the
// p lo and p hi coefficients at that end.  D[side][r][c], r < Lb, c < 2p:
// left rows k = r, columns lo[c] (c < p) and hi[c - p]; right rows
// k = n1 - Lb + r, columns lo[n0 - p + c], hi[n0 - p + c - p].  The
// analysis of a level is the transpose.  Computed at a level with n0 = 4p + 4
// (the blocks do not depend on the level); returns false if a difference
// shows up outside that structure.
bool build_coarse(const Plan& P, std::vector<double>& D) {
  D.clear();
  if (P.bd == UW_BOUNDARY_PERIODIC) return true;
  const int p = P.p, Lb = P.Lb, n0 = 4 * p + 4, n1 = 2 * n0;
  auto syn_exact = [&](const std::vector<double>& lo, const std::vector<double>& hi, int k) {
    double acc = 0;
    const int mlo = std::max(p, ceildiv(k - p, 2)), mhi = std::min(n0 - p - 1, floordiv(k + p - 1, 2));
    for (int m = mlo; m <= mhi; ++m) acc += P.h[k - 2 * m + p - 1] * lo[m] + P.g[k - 2 * m + p - 1] * hi[m];
    if (k < Lb)
      for (int m = 0; m < p; ++m) acc += P.PL[m * Lb + k] * lo[m] + P.QL[m * Lb + k] * hi[m];
    const int c = n1 - 1 - k;
    if (c < Lb)
      for (int r = 0; r < p; ++r) acc += P.PR[r * Lb + c] * lo[n0 - 1 - r] + P.QR[r * Lb + c] * hi[n0 - 1 - r];
    return acc;
  };
  auto syn_int0 = [&](const std::vector<double>& lo, const std::vector<double>& hi, int k) {
    double acc = 0;
    for (int l = -p + 1; l <= p; ++l) {
      const int km = k - l;
      if (km & 1) continue;
      const int i = km / 2;
      if (i < 0 || i >= n0) continue;
      acc += P.h[l + p - 1] * lo[i] + P.g[l + p - 1] * hi[i];
    }
    return acc;
  };
  D.assign((size_t)2 * Lb * 2 * p, 0.0);
  std::vector<double> lo(n0), hi(n0);
  double dmax = 0, stray = 0;
  // columns: the p + 2 coefficients nearest each end (the last two must show no difference)
  for (int side = 0; side < 2; ++side)
    for (int half = 0; half < 2; ++half)
      for (int e = 0; e < p + 2; ++e) {
        std::fill(lo.begin(), lo.end(), 0.0);
        std::fill(hi.begin(), hi.end(), 0.0);
        const int i = side == 0 ? e : n0 - 1 - e;
        (half == 0 ? lo : hi)[i] = 1.0;
        for (int k = 0; k < n1; ++k) {
          const double d = syn_exact(lo, hi, k) - syn_int0(lo, hi, k);
          const int r = side == 0 ? k : k - (n1 - Lb);
          if (e < p && r >= 0 && r < Lb) {
            const int c = half * p + (side == 0 ? e : p - 1 - e);
            D[((size_t)side * Lb + r) * 2 * p + c] = d;
            dmax = std::max(dmax, std::fabs(d));
          } else {
            stray = std::max(stray, std::fabs(d));
          }
        }
      }
  if (stray > 1e-13 * std::max(dmax, 1.0)) {
    D.clear();
    return false;
  }
  return true;
}

}  // namespace uw
