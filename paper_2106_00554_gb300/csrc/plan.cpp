// Host planner of libuw: every input-independent table of the method, built in
// long double on the host, plus the plan half of the C ABI.
//
// Paper: V. Antun, arXiv 2106.00554.  The tables are the quantities that
// "can be computed a priori" (Sec. 4.1): the cell integrals of phi behind the
// taps W phi_{0,-l}(s), the boundary rows of Prop. 4.4, and the two-scale
// blocks of the boundary DWT (Sec. 3.2).
//
// Conventions (Sec. 3.2): supp phi = supp psi = [-p+1, p]; h_k, k = -p+1..p,
// phi(x) = sqrt2 sum_k h_k phi(2x-k); g_k = (-1)^k h_{1-k}.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "uw_internal.h"

namespace uw {

typedef long double LD;
typedef std::complex<LD> CLD;

// ---------------------------------------------------------------------------
// error state (per thread)
// ---------------------------------------------------------------------------
static thread_local int g_last_status = UW_OK;
static thread_local std::string g_last_msg;

void set_error(int status, const std::string& msg) {
  g_last_status = status;
  g_last_msg = msg;
}

// ---------------------------------------------------------------------------
// small dense linear algebra in long double
// ---------------------------------------------------------------------------
// Solve A x = b (n x n, row-major, copied) by Gaussian elimination with
// partial pivoting.  Returns false if a pivot vanishes.
static bool solve(std::vector<LD> A, std::vector<LD> b, int n, std::vector<LD>& x) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * n + c]) > std::fabs(A[(size_t)piv * n + c])) piv = r;
    if (std::fabs(A[(size_t)piv * n + c]) < 1e-300L) return false;
    if (piv != c) {
      for (int k = 0; k < n; ++k) std::swap(A[(size_t)c * n + k], A[(size_t)piv * n + k]);
      std::swap(b[c], b[piv]);
    }
    for (int r = c + 1; r < n; ++r) {
      LD f = A[(size_t)r * n + c] / A[(size_t)c * n + c];
      if (f == 0) continue;
      for (int k = c; k < n; ++k) A[(size_t)r * n + k] -= f * A[(size_t)c * n + k];
      b[r] -= f * b[c];
    }
  }
  x.assign(n, 0);
  for (int r = n - 1; r >= 0; --r) {
    LD s = b[r];
    for (int k = r + 1; k < n; ++k) s -= A[(size_t)r * n + k] * x[k];
    x[r] = s / A[(size_t)r * n + r];
  }
  return true;
}

// Compensated dot product (Ogita, Rump, Oishi, "Accurate sum and dot
// product", 2005, Algorithm Dot2): every product is split exactly with an FMA
// and every addition with TwoSum, so the result is as accurate as a plain sum
// in twice the working precision.  The edge-space sums pair large polynomial
// coefficients with tiny restricted overlaps and cancel heavily.
struct Dot2 {
  LD s = 0, c = 0;
  void add(LD a, LD b) {
    const LD p = a * b;
    const LD ep = std::fma(a, b, -p);
    const LD t = s + p;
    const LD z = t - s;
    const LD es = (s - (t - z)) + (p - z);
    s = t;
    c += ep + es;
  }
  LD get() const { return s + c; }
};

// ---------------------------------------------------------------------------
// Daubechies extremal-phase filter: roots of P(y) = sum_{k<p} C(p-1+k,k) y^k
// by Durand-Kerner iteration polished with Newton steps; each root y gives the
// reciprocal pair z, 1/z of z^2 - (2-4y) z + 1 and the root with |z| > 1 is a
// zero of m0(z) = sum_k h_k z^{k+p-1} (classical orientation, h_{-p+1} > 0).
// ---------------------------------------------------------------------------
static std::vector<CLD> poly_roots(const std::vector<LD>& c /* increasing */) {
  int n = (int)c.size() - 1;
  std::vector<CLD> z(n);
  if (n == 0) return z;
  CLD seed(0.4L, 0.9L), w(1, 0);
  for (int i = 0; i < n; ++i) { z[i] = w; w *= seed; }
  auto eval = [&](CLD x) {
    CLD s = 0;
    for (int k = n; k >= 0; --k) s = s * x + c[k];
    return s;
  };
  auto deriv = [&](CLD x) {
    CLD s = 0;
    for (int k = n; k >= 1; --k) s = s * x + (LD)k * c[k];
    return s;
  };
  for (int it = 0; it < 2000; ++it) {
    LD delta = 0;
    for (int i = 0; i < n; ++i) {
      CLD den = c[n];
      for (int j = 0; j < n; ++j)
        if (j != i) den *= (z[i] - z[j]);
      CLD step = eval(z[i]) / den;
      z[i] -= step;
      delta = std::max(delta, std::abs(step));
    }
    if (delta < 1e-30L) break;
  }
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < 5; ++k) {
      CLD dv = deriv(z[i]);
      if (std::abs(dv) == 0) break;
      z[i] -= eval(z[i]) / dv;
    }
  return z;
}

// Filter of m0(z) with a zero of order p at z = -1 and the given zeros,
// normalised to sum h = sqrt 2 (h_k, k = -p+1..p).
static std::vector<LD> filter_from_zeros(int p, const std::vector<CLD>& zeros) {
  std::vector<CLD> Q(1, CLD(1, 0));
  auto mul = [&](CLD a0, CLD a1) {  // Q *= (a0 + a1 z)
    std::vector<CLD> out(Q.size() + 1, CLD(0, 0));
    for (size_t i = 0; i < Q.size(); ++i) {
      out[i] += Q[i] * a0;
      out[i + 1] += Q[i] * a1;
    }
    Q.swap(out);
  };
  for (int i = 0; i < p; ++i) mul(1, 1);
  for (CLD z : zeros) mul(-z, 1);
  std::vector<LD> h(2 * p);
  LD s = 0;
  for (int i = 0; i < 2 * p; ++i) s += Q[i].real();
  for (int i = 0; i < 2 * p; ++i) h[i] = std::sqrt((LD)2) * Q[i].real() / s;
  return h;
}

// Least-asymmetric measure of the filter whose m0 has zeros of order p at -1
// and the given other zeros: m0(e^{-iw}) = c (1 + e^{-iw})^p R(e^{-iw}),
// R(z) = prod (z - z_k).  On (0, pi) the first factor has the linear phase
// -p w / 2, so the measure is the mean squared distance of
// psi(w) = arg R(e^{-iw}) - arg R(1) (unwrapped) from its least-squares line
// through the origin on w_k = pi (k + 1/2) / 256, k < 256.  (m0 itself is
// ill-conditioned near w = pi, where it has a zero of order p.)
static LD phase_asymmetry(const std::vector<CLD>& zeros) {
  const int K = 256;
  const LD pi = 3.141592653589793238462643383279502884L;
  CLD R1(1, 0);
  for (CLD z : zeros) R1 *= CLD(1, 0) - z;
  const LD a1 = std::atan2(R1.imag(), R1.real());
  std::vector<LD> ph(K), w(K);
  LD prev = 0, off = 0;
  for (int k = 0; k < K; ++k) {
    w[k] = pi * ((LD)k + 0.5L) / (LD)K;
    const CLD e = std::polar((LD)1, -w[k]);
    CLD Rw(1, 0);
    for (CLD z : zeros) Rw *= e - z;
    LD a = std::atan2(Rw.imag(), Rw.real()) - a1;
    if (k == 0) {
      a -= 2 * pi * std::nearbyint(a / (2 * pi));   // the branch nearest 0 at w -> 0
    } else {
      LD d = a + off - prev;                         // unwrap
      while (d > pi) { off -= 2 * pi; d -= 2 * pi; }
      while (d < -pi) { off += 2 * pi; d += 2 * pi; }
    }
    ph[k] = a + off;
    prev = ph[k];
  }
  LD sw = 0, sp = 0;
  for (int k = 0; k < K; ++k) {
    sw += w[k] * w[k];
    sp += ph[k] * w[k];
  }
  const LD b = sp / sw;
  LD e = 0;
  for (int k = 0; k < K; ++k) e += (ph[k] - b * w[k]) * (ph[k] - b * w[k]);
  return e / (LD)K;
}

// Daubechies filters with p vanishing moments.  Each root y of
// P(y) = sum_{k<p} C(p-1+k,k) y^k gives a reciprocal pair of zeros of m0.
// Extremal phase keeps every member outside the unit circle.  The symlet
// (least asymmetric) takes one member per pair -- a complex conjugate pair of
// roots of P chosen together so that h stays real -- minimising
// phase_asymmetry; a choice and its complement are mirror images, and the
// one whose energy centre lies in the first half of the taps is kept.
static std::vector<LD> daubechies(int p, bool symlet = false) {
  if (p == 1) return filter_from_zeros(1, {});
  std::vector<LD> P(p);
  LD binom = 1;  // C(p-1+k, k)
  for (int k = 0; k < p; ++k) {
    P[k] = binom;
    binom = binom * (LD)(p + k) / (LD)(k + 1);
  }
  const std::vector<CLD> ys = poly_roots(P);
  std::vector<CLD> zo, zi;   // member outside / inside the unit circle
  for (CLD y : ys) {
    CLD b = (LD)2 - (LD)4 * y;
    CLD d = std::sqrt(b * b - (LD)4);
    CLD z1 = (b + d) / (LD)2, z2 = (b - d) / (LD)2;
    zo.push_back(std::abs(z1) > 1 ? z1 : z2);
    zi.push_back(std::abs(z1) > 1 ? z2 : z1);
  }
  if (!symlet) return filter_from_zeros(p, zo);
  // groups of roots of P chosen together
  const int n = (int)ys.size();
  std::vector<std::vector<int>> groups;
  std::vector<bool> used(n, false);
  const LD tol = 1e-12L;
  for (int i = 0; i < n; ++i) {
    if (used[i]) continue;
    used[i] = true;
    if (std::abs(ys[i].imag()) < tol) {
      groups.push_back({i});
      continue;
    }
    int j = -1;
    LD best = 0;
    for (int k = 0; k < n; ++k)
      if (!used[k] && (j < 0 || std::abs(ys[k] - std::conj(ys[i])) < best)) {
        j = k;
        best = std::abs(ys[k] - std::conj(ys[i]));
      }
    used[j] = true;
    groups.push_back({i, j});
  }
  const int G = (int)groups.size();
  std::vector<LD> best_h;
  LD best_a = 0;
  for (int mask = 0; mask < (1 << (G - 1)); ++mask) {   // group 0 fixed: one of each mirror pair
    std::vector<CLD> zeros;
    for (int g = 0; g < G; ++g) {
      const bool inside = g > 0 && ((mask >> (g - 1)) & 1);
      for (int i : groups[g]) zeros.push_back(inside ? zi[i] : zo[i]);
    }
    const LD a = phase_asymmetry(zeros);
    if (best_h.empty() || a < best_a) {
      best_a = a;
      best_h = filter_from_zeros(p, zeros);
    }
  }
  LD c = 0, e = 0;
  for (int i = 0; i < 2 * p; ++i) {
    c += (LD)i * best_h[i] * best_h[i];
    e += best_h[i] * best_h[i];
  }
  if (!(c < (LD)(2 * p - 1) / 2 * e)) std::reverse(best_h.begin(), best_h.end());
  return best_h;
}

// ---------------------------------------------------------------------------
// Cell integrals I_q[t] through antiderivatives of phi: the lower one
// Phi(x) = int_{-inf}^x phi and the upper one Psi(x) = int_x^inf phi both satisfy
// X(x) = (1/sqrt2) sum_k h_k X(2x - k) (Phi = 0 left of the support and 1 right
// of it, Psi the other way round).  Solve at the integers, refine to the
// dyadics of level q, then take I_q[t] = Phi((t+1)/2^q) - Phi(t/2^q) on the
// left half of the support and Psi(t/2^q) - Psi((t+1)/2^q) on the right half:
// each difference is formed where its antiderivative is small, so the tiny
// cells at both ends keep their relative accuracy.
// ---------------------------------------------------------------------------
static std::map<long, LD> antiderivative(const std::vector<LD>& h, int p, int q, bool upper) {
  auto H = [&](int k) -> LD { int i = k + p - 1; return (i >= 0 && i < 2 * p) ? h[i] : 0; };
  const LD is2 = 1 / std::sqrt((LD)2);
  const LD left_val = upper ? 1 : 0, right_val = upper ? 0 : 1;
  int lo = -p + 2, hi = p - 1, n = std::max(0, hi - lo + 1);
  auto val = [&](const std::map<long, LD>& m, long i, long S) -> LD {
    if (i <= (-p + 1) * S) return left_val;
    if (i >= p * S) return right_val;
    auto it = m.find(i);
    return it == m.end() ? 0 : it->second;
  };
  std::map<long, LD> cur;
  if (n > 0) {
    std::vector<LD> A((size_t)n * n, 0), b(n, 0), x;
    for (int r = 0; r < n; ++r) {
      int nn = lo + r;
      A[(size_t)r * n + r] += 1;
      for (int k = -p + 1; k <= p; ++k) {
        long arg = 2L * nn - k;
        if (arg <= -p + 1 || arg >= p) b[r] += is2 * H(k) * (arg <= -p + 1 ? left_val : right_val);
        else A[(size_t)r * n + (arg - lo)] -= is2 * H(k);
      }
    }
    solve(A, b, n, x);
    for (int r = 0; r < n; ++r) cur[lo + r] = x[r];
  }
  long S = 1;
  for (int j = 1; j <= q; ++j) {
    std::map<long, LD> nxt;
    long S2 = S * 2;
    for (long i = (-p + 1) * S2; i <= p * S2; ++i) {
      // X(i/S2) = (1/sqrt2) sum_k h_k X(i/S - k)
      LD s = 0;
      for (int k = -p + 1; k <= p; ++k) s += H(k) * val(cur, i - k * S, S);
      nxt[i] = is2 * s;
    }
    cur.swap(nxt);
    S = S2;
  }
  // complete the table with the boundary values
  for (long i = (-p + 1) * S; i <= p * S; ++i) cur[i] = val(cur, i, S);
  return cur;
}

static std::vector<LD> cell_integrals(const std::vector<LD>& h, int p, int q) {
  std::map<long, LD> Phi = antiderivative(h, p, q, false), Psi = antiderivative(h, p, q, true);
  const long S = 1L << q;
  std::vector<LD> I;
  for (long t = (-p + 1) * S; t <= p * S - 1; ++t) {
    // the support [-p+1, p] has its centre at 1/2, i.e. at t + 1/2 = S/2
    if (2 * t + 1 < S) I.push_back(Phi[t + 1] - Phi[t]);
    else I.push_back(Psi[t] - Psi[t + 1]);
  }
  return I;
}

// ---------------------------------------------------------------------------
// Restricted Gram matrices through partial autocorrelations at integers:
//   Fb_d(y) = int_y^inf phi(u) phi(u-d) du
// satisfies Fb_d(y) = sum_{k,l} h_k h_l Fb_{2d+l-k}(2y-k) (substitute
// phi(u) = sqrt2 sum_k h_k phi(2u-k)), with Fb = delta_{d0} left of the common
// support [max(-p+1,d-p+1), min(p,d+p)] and 0 right of it.  Then
//   int_0^inf  phi(x-a) phi(x-b) dx = Fb_{b-a}(-a),
//   int_-inf^0 phi(x-a) phi(x-b) dx = delta_ab - Fb_{b-a}(-a).
// ---------------------------------------------------------------------------
struct Gram {
  int p;
  std::map<std::pair<int, int>, LD> F, Fb;
  static LD lookup(const std::map<std::pair<int, int>, LD>& X, int p, int d, long y, bool upper) {
    if (std::abs(d) > 2 * p - 2) return 0;
    long a = std::max(-p + 1, d - p + 1), b = std::min(p, d + p);
    LD full = d == 0 ? 1 : 0;
    if (y <= a) return upper ? full : 0;
    if (y >= b) return upper ? 0 : full;
    auto it = X.find({d, (int)y});
    return it == X.end() ? 0 : it->second;
  }
  // Only the upper integrals Fb are used: solved directly they keep relative
  // accuracy down to the smallest overlaps (F loses it in the upper part of
  // the support), and the lower integral is delta_{d0} - Fb.
  LD left(int a, int b) const { return lookup(Fb, p, b - a, -a, true); }
  LD right(int a, int b) const { return (a == b ? 1 : 0) - lookup(Fb, p, b - a, -a, true); }
};

static bool solve_autocorr(const std::vector<LD>& h, int p, bool upper, std::map<std::pair<int, int>, LD>& X) {
  auto H = [&](int k) -> LD { int i = k + p - 1; return (i >= 0 && i < 2 * p) ? h[i] : 0; };
  std::vector<std::pair<int, int>> unk;
  std::map<std::pair<int, int>, int> pos;
  for (int d = -(2 * p - 2); d <= 2 * p - 2; ++d) {
    long a = std::max(-p + 1, d - p + 1), b = std::min(p, d + p);
    for (long y = a + 1; y < b; ++y) {
      pos[{d, (int)y}] = (int)unk.size();
      unk.push_back({d, (int)y});
    }
  }
  int n = (int)unk.size();
  if (n == 0) return true;
  std::map<std::pair<int, int>, LD> empty;
  std::vector<LD> A((size_t)n * n, 0), rhs(n, 0), x;
  for (int r = 0; r < n; ++r) {
    int d = unk[r].first, y = unk[r].second;
    A[(size_t)r * n + r] += 1;
    for (int k = -p + 1; k <= p; ++k)
      for (int l = -p + 1; l <= p; ++l) {
        LD c = H(k) * H(l);
        if (c == 0) continue;
        int d2 = 2 * d + l - k;
        long y2 = 2L * y - k;
        auto it = pos.find({d2, (int)y2});
        if (it != pos.end()) A[(size_t)r * n + it->second] -= c;
        else rhs[r] += c * Gram::lookup(empty, p, d2, y2, upper);
      }
  }
  if (!solve(A, rhs, n, x)) return false;
  for (int r = 0; r < n; ++r) X[unk[r]] = x[r];
  return true;
}

static bool build_gram(const std::vector<LD>& h, int p, Gram& G) {
  G.p = p;
  return solve_autocorr(h, p, true, G.Fb);
}

// ---------------------------------------------------------------------------
// Boundary scaling functions (Cohen-Daubechies-Vial; Sec. 3.2).  Left: the
// polynomial-weighted restricted translates n = -p+1..p-1; the nested basis
// f_m(n) = prod_{k=m+1}^{p-1} (n - k) spans the functions supported in
// [0, p+m]; Gram-Schmidt in that order (G-metric) gives phi^left_m.  Right:
// translates n = -p..p-2, f_m(n) = prod_{k=-p}^{-m-2} (n - k).
// ---------------------------------------------------------------------------
static std::vector<std::vector<LD>> edge_fns(int p, const std::vector<int>& tr,
                                             const std::vector<std::vector<LD>>& Gm, bool left) {
  int n = (int)tr.size();
  std::vector<std::vector<LD>> out;
  for (int m = 0; m < p; ++m) {
    std::vector<LD> v(n);
    LD mx = 0;
    for (int j = 0; j < n; ++j) {
      // Lagrange polynomial of node m (left: nodes 0..p-1) or -m-1 (right:
      // nodes -1..-p): it vanishes on the nodes beyond m, so L_0..L_m span the
      // functions supported in [0, p+m] (resp. [-m-p, 0])
      const int node = left ? m : -m - 1;
      LD prod = 1;
      for (int i = 0; i < p; ++i) {
        const int nk = left ? i : -i - 1;
        if (nk != node) prod *= (LD)(tr[j] - nk) / (LD)(node - nk);
      }
      v[j] = prod;
      mx = std::max(mx, std::fabs(prod));
    }
    for (auto& e : v) e /= mx;
    auto dot = [&](const std::vector<LD>& a, const std::vector<LD>& b) {
      Dot2 outer;
      for (int i = 0; i < n; ++i) {
        Dot2 inner;
        for (int j = 0; j < n; ++j) inner.add(Gm[i][j], b[j]);
        outer.add(a[i], inner.s);  // keep the inner sum as the pair (s, c)
        outer.add(a[i], inner.c);
      }
      return outer.get();
    };
    for (int pass = 0; pass < 2; ++pass)
      for (auto& u : out) {
        LD c = dot(u, v);
        for (int i = 0; i < n; ++i) v[i] -= c * u[i];
      }
    LD nr = std::sqrt(dot(v, v));
    for (auto& e : v) e /= nr;
    int anchor = left ? m : -m - 1;
    for (int j = 0; j < n; ++j)
      if (tr[j] == anchor && v[j] < 0)
        for (auto& e : v) e = -e;
    out.push_back(v);
  }
  return out;
}

// ---------------------------------------------------------------------------
// Level-independent two-scale blocks at one edge.  Side coordinates at level
// 1: c < p is the edge scaling function c of level 1, c >= p the interior
// translate (left: index c; right: index -1-c).  Boundary wavelets span the
// complement of the level-0 space and of the interior wavelets; they are the
// projections P_C e_i (P_C = I - sum over the orthonormal constraint rows),
// turned into the basis whose m-th vector ends at coordinate p + 2m by Givens
// rotations taken from the last coordinate down.
// ---------------------------------------------------------------------------
static void side_blocks(int p, bool left, const std::vector<LD>& h, const Gram& G,
                        const std::vector<std::vector<LD>>& E, const std::vector<int>& tr,
                        std::vector<LD>& Pout, std::vector<LD>& Qout, int Lb) {
  auto H = [&](int k) -> LD { int i = k + p - 1; return (i >= 0 && i < 2 * p) ? h[i] : 0; };
  auto Gf = [&](int a, int b) { return left ? G.left(a, b) : G.right(a, b); };
  auto keep = [&](int i) { return left ? i >= -p + 1 : i <= p - 2; };
  auto coord = [&](int i) { return left ? i : -1 - i; };
  const int W = 8 * p + 16;
  std::vector<std::vector<LD>> rows;
  // level-0 edge scaling functions
  for (int m = 0; m < p; ++m) {
    std::map<int, Dot2> cacc;
    for (size_t j = 0; j < tr.size(); ++j)
      for (int k = -p + 1; k <= p; ++k) {
        int i = 2 * tr[j] + k;
        if (keep(i)) cacc[i].add(E[m][j], H(k));
      }
    std::map<int, LD> c;
    for (auto& kv : cacc) c[kv.first] = kv.second.get();
    std::vector<LD> v(W, 0);
    for (int mp = 0; mp < p; ++mp) {
      Dot2 outer;
      for (auto& kv : c) {
        Dot2 inner;
        for (size_t j2 = 0; j2 < tr.size(); ++j2) inner.add(Gf(kv.first, tr[j2]), E[mp][j2]);
        outer.add(kv.second, inner.s);
        outer.add(kv.second, inner.c);
      }
      v[mp] = outer.get();
    }
    for (auto& kv : c)
      if (coord(kv.first) >= p) v[coord(kv.first)] += kv.second;
    rows.push_back(v);
  }
  // interior phi(.-n), psi(.-n) touching the window
  for (int t = 0; t < W; ++t) {
    int n = left ? p + t : -p - 1 - t;
    bool any = false;
    std::vector<LD> vh(W, 0), vg(W, 0);
    for (int k = -p + 1; k <= p; ++k) {
      int c = coord(2 * n + k);
      if (c < W) {
        any = true;
        vh[c] = H(k);
        vg[c] = ((k % 2 == 0) ? 1 : -1) * H(1 - k);
      }
    }
    if (!any) break;
    rows.push_back(vh);
    rows.push_back(vg);
  }
  // projections of e_i, i < Lb, onto the complement
  std::vector<std::vector<LD>> V;
  for (int i = 0; i < Lb; ++i) {
    std::vector<LD> v(W, 0);
    v[i] = 1;
    for (auto& r : rows) {
      LD c = r[i];
      if (c == 0) continue;
      for (int k = 0; k < W; ++k) v[k] -= c * r[k];
    }
    V.push_back(v);
  }
  // orthonormal basis of their span: the complement has dimension exactly p,
  // so take p directions by Gram-Schmidt with pivoting (largest residual
  // first) -- no tolerance decides the rank
  std::vector<std::vector<LD>> B;
  std::vector<std::vector<LD>> Rv = V;
  for (int it = 0; it < p; ++it) {
    int best = -1;
    LD bn = -1;
    for (size_t i = 0; i < Rv.size(); ++i) {
      LD nr = 0;
      for (int k = 0; k < W; ++k) nr += Rv[i][k] * Rv[i][k];
      if (nr > bn) { bn = nr; best = (int)i; }
    }
    std::vector<LD> u = Rv[best];
    for (int pass = 0; pass < 2; ++pass)
      for (auto& w : B) {
        LD c = 0;
        for (int k = 0; k < W; ++k) c += w[k] * u[k];
        for (int k = 0; k < W; ++k) u[k] -= c * w[k];
      }
    LD nr = 0;
    for (int k = 0; k < W; ++k) nr += u[k] * u[k];
    nr = std::sqrt(nr);
    for (auto& e : u) e /= nr;
    B.push_back(u);
    for (auto& r : Rv) {
      LD c = 0;
      for (int k = 0; k < W; ++k) c += u[k] * r[k];
      for (int k = 0; k < W; ++k) r[k] -= c * u[k];
    }
  }
  // staggered basis: the m-th wavelet ends at coordinate p + 2m; from the
  // last such coordinate down, rotate the remaining vectors so that one of
  // them carries the coordinate, and keep it
  std::vector<int> active;
  for (int i = 0; i < p; ++i) active.push_back(i);
  std::vector<std::vector<LD>> U(p);
  LD sgn = left ? (((p % 2) == 0 ? 1 : -1) * h[0]) : ((((p + 1) % 2) == 0 ? 1 : -1) * h[2 * p - 1]);
  for (int m = p - 1; m >= 0; --m) {
    int c = p + 2 * m;
    int piv = active[0];
    for (int a : active)
      if (std::fabs(B[a][c]) > std::fabs(B[piv][c])) piv = a;
    for (int a : active) {
      if (a == piv || B[a][c] == 0) continue;
      LD x = B[piv][c], y = B[a][c], r = std::hypot(x, y);
      LD cs = x / r, sn = y / r;
      for (int k = 0; k < W; ++k) {
        LD u = B[piv][k], w = B[a][k];
        B[piv][k] = cs * u + sn * w;
        B[a][k] = -sn * u + cs * w;
      }
    }
    std::vector<LD> u = B[piv];
    if ((u[c] < 0) != (sgn < 0))
      for (auto& e : u) e = -e;
    U[m] = u;
    active.erase(std::find(active.begin(), active.end(), piv));
  }
  Pout.assign((size_t)p * Lb, 0);
  Qout.assign((size_t)p * Lb, 0);
  for (int m = 0; m < p; ++m)
    for (int c = 0; c < Lb; ++c) {
      Pout[(size_t)m * Lb + c] = rows[m][c];
      Qout[(size_t)m * Lb + c] = U[m].empty() ? 0 : U[m][c];
    }
}

static bool build_tables_uncached(Plan& P, std::string& err) {
  const int p = P.p, q = P.q, Q = 1 << q;
  P.Q = Q;
  P.Lb = 3 * p - 1;
  P.ntap = (2 * p - 1) * Q;
  std::vector<LD> h = daubechies(p, P.family == 1);
  std::vector<LD> I = cell_integrals(h, p, q);
  if ((int)I.size() != P.ntap) { err = "cell integral table size"; return false; }
  P.h.resize(2 * p);
  P.g.resize(2 * p);
  for (int k = -p + 1; k <= p; ++k) {
    P.h[k + p - 1] = (double)h[k + p - 1];
    int i = 1 - k + p - 1;
    P.g[k + p - 1] = (double)(((k % 2) == 0 ? 1 : -1) * h[i]);
  }
  P.taps.assign(I.begin(), I.end());
  Gram G;
  if (!build_gram(h, p, G)) { err = "restricted Gram system is singular"; return false; }
  std::vector<int> trL, trR;
  for (int n = -p + 1; n <= p - 1; ++n) trL.push_back(n);
  for (int n = -p; n <= p - 2; ++n) trR.push_back(n);
  std::vector<std::vector<LD>> GL(trL.size(), std::vector<LD>(trL.size())), GR = GL;
  for (size_t a = 0; a < trL.size(); ++a)
    for (size_t b = 0; b < trL.size(); ++b) {
      GL[a][b] = G.left(trL[a], trL[b]);
      GR[a][b] = G.right(trR[a], trR[b]);
    }
  auto A = edge_fns(p, trL, GL, true);
  auto B = edge_fns(p, trR, GR, false);
  auto Iq = [&](long t) -> LD {
    long i = t + (long)(-(-p + 1)) * Q;
    return (i >= 0 && i < P.ntap) ? I[i] : 0;
  };
  P.EL.assign((size_t)p * P.ntap, 0);
  P.ER.assign((size_t)p * P.ntap, 0);
  for (int m = 0; m < p; ++m)
    for (int k = 0; k < P.ntap; ++k) {
      Dot2 sl, sr;
      for (size_t j = 0; j < trL.size(); ++j) sl.add(A[m][j], Iq((long)k - (long)Q * trL[j]));
      for (size_t j = 0; j < trR.size(); ++j) sr.add(B[m][j], Iq(-(long)(k + 1) - (long)Q * trR[j]));
      P.EL[(size_t)m * P.ntap + k] = (double)sl.get();
      P.ER[(size_t)m * P.ntap + k] = (double)sr.get();
    }
  std::vector<LD> pl, ql, pr, qr;
  side_blocks(p, true, h, G, A, trL, pl, ql, P.Lb);
  side_blocks(p, false, h, G, B, trR, pr, qr, P.Lb);
  P.PL.assign(pl.begin(), pl.end());
  P.QL.assign(ql.begin(), ql.end());
  P.PR.assign(pr.begin(), pr.end());
  P.QR.assign(qr.begin(), qr.end());
  return true;
}

// The tables depend on (p, q, filter family) only and take up to ~0.1 s to
// build at p = 10: they are built once per process and copied into every
// later plan with the same three.
bool build_tables(Plan& P, std::string& err) {
  struct Set {
    std::vector<double> h, g, taps, EL, ER, PL, QL, PR, QR;
  };
  static std::mutex mu;
  static std::map<std::tuple<int, int, int>, Set> cache;
  const auto key = std::make_tuple(P.p, P.q, P.family);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      const Set& c = it->second;
      P.Q = 1 << P.q;
      P.Lb = 3 * P.p - 1;
      P.ntap = (2 * P.p - 1) * P.Q;
      P.h = c.h; P.g = c.g; P.taps = c.taps; P.EL = c.EL; P.ER = c.ER;
      P.PL = c.PL; P.QL = c.QL; P.PR = c.PR; P.QR = c.QR;
      return true;
    }
  }
  if (!build_tables_uncached(P, err)) return false;
  std::lock_guard<std::mutex> lock(mu);
  cache.emplace(key, Set{P.h, P.g, P.taps, P.EL, P.ER, P.PL, P.QL, P.PR, P.QR});
  return true;
}

}  // namespace uw

// ===========================================================================
// C ABI: plan half
// ===========================================================================
using uw::Plan;

struct uw_plan : public Plan {};

static int fail(int st, const std::string& m) {
  uw::set_error(st, m);
  return st;
}

static int J0_min(int p) {
  int J = 0;
  while ((1 << J) < 2 * (2 * p - 1)) ++J;
  return J;
}

static int upload_mask(uw_plan* P, const int64_t* omega, int64_t m) {
  const int64_t N = P->N;
  const int wpr = (int)((N + 31) / 32);
  const int64_t rows = P->d == 1 ? 1 : N;
  const int64_t words = rows * wpr;
  const int64_t total = P->d == 1 ? N : N * N;
  std::vector<uint32_t> mask(words, 0);
  if (omega == nullptr || m < 0) {
    for (int64_t r = 0; r < rows; ++r)
      for (int64_t n = 0; n < N; ++n) mask[r * wpr + n / 32] |= 1u << (n % 32);
    m = total;
  } else {
    int64_t prev = -1;
    for (int64_t i = 0; i < m; ++i) {
      int64_t v = omega[i];
      if (v <= prev || v >= total) return fail(UW_ERR_INVALID_ARG, "Omega must be strictly increasing in [0, N^d)");
      prev = v;
      int64_t r = P->d == 1 ? 0 : v / N, n = P->d == 1 ? v : v % N;
      mask[r * wpr + n / 32] |= 1u << (n % 32);
    }
  }
  std::vector<int32_t> pre(words);
  int64_t acc = 0;
  for (int64_t w = 0; w < words; ++w) {
    pre[w] = (int32_t)acc;
    acc += __builtin_popcount(mask[w]);
  }
  if (acc != m) return fail(UW_ERR_INTERNAL, "mask count mismatch");
  // natural-order position of every sample, in packed order: the sequency
  // index n of a row reads the FWHT output at bitrev_L(n xor (n >> 1))
  std::vector<uint16_t> pos;
  if (N <= 65536) {
    int L = 0;
    while ((int64_t(1) << L) < N) ++L;
    std::vector<uint16_t> seqpos((size_t)N);
    for (int64_t n = 0; n < N; ++n) {
      uint32_t gry = (uint32_t)(n ^ (n >> 1)), rev = 0;
      for (int b = 0; b < L; ++b) rev |= ((gry >> b) & 1u) << (L - 1 - b);
      seqpos[(size_t)n] = (uint16_t)rev;
    }
    pos.reserve((size_t)m);
    for (int64_t w = 0; w < words; ++w)
      for (uint32_t bits = mask[w]; bits; bits &= bits - 1)
        pos.push_back(seqpos[(size_t)((w % wpr) * 32 + __builtin_ctz(bits))]);
  }
  uint16_t* dpos = nullptr;
  if (!pos.empty()) {
    // padding: positions are also read in 32-bit pairs and copied in whole
    // 16-byte units (up to 7 entries past a row's last sample)
    pos.resize((pos.size() + 7) / 8 * 8 + 8, 0);
    if (cudaMalloc(&dpos, pos.size() * sizeof(uint16_t)) != cudaSuccess) {
      cudaGetLastError();
      return fail(UW_ERR_OOM, "sample position allocation failed");
    }
    if (cudaMemcpy(dpos, pos.data(), pos.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(dpos);
      return fail(UW_ERR_CUDA, "sample position upload failed");
    }
  }
  // 1D long lines: the sample of every natural FWHT position (the products
  // gather and scatter in the kernel that applies the last Walsh stages)
  int32_t* dn2y = nullptr;
  if (P->d == 1 && N >= 8192 && N <= (int64_t(1) << 22)) {
    int L = 0;
    while ((int64_t(1) << L) < N) ++L;
    std::vector<int32_t> n2y((size_t)N, -1);
    int32_t rank = 0;
    for (int64_t w = 0; w < wpr; ++w)
      for (uint32_t bits = mask[w]; bits; bits &= bits - 1) {
        const uint32_t n = (uint32_t)(w * 32 + __builtin_ctz(bits));
        const uint32_t gry = n ^ (n >> 1);
        uint32_t rev = 0;
        for (int b = 0; b < L; ++b) rev |= ((gry >> b) & 1u) << (L - 1 - b);
        n2y[rev] = rank++;
      }
    if (cudaMalloc(&dn2y, n2y.size() * sizeof(int32_t)) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(dpos);
      return fail(UW_ERR_OOM, "sample table allocation failed");
    }
    if (cudaMemcpy(dn2y, n2y.data(), n2y.size() * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(dn2y);
      cudaFree(dpos);
      return fail(UW_ERR_CUDA, "sample table upload failed");
    }
  }
  uint32_t* dm = nullptr;
  int32_t* dp = nullptr;
  if (cudaMalloc(&dm, words * sizeof(uint32_t)) != cudaSuccess ||
      cudaMalloc(&dp, words * sizeof(int32_t)) != cudaSuccess) {
    cudaFree(dm);
    cudaFree(dpos);
    cudaFree(dn2y);
    cudaGetLastError();
    return fail(UW_ERR_OOM, "mask allocation failed");
  }
  if (cudaMemcpy(dm, mask.data(), words * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(dp, pre.data(), words * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(dm);
    cudaFree(dp);
    cudaFree(dpos);
    cudaFree(dn2y);
    return fail(UW_ERR_CUDA, "mask upload failed");
  }
  cudaFree(P->d_mask);
  cudaFree(P->d_prefix);
  cudaFree(P->d_pos);
  cudaFree(P->d_nat2y);
  P->d_mask = dm;
  P->d_prefix = dp;
  P->d_pos = dpos;
  P->d_nat2y = dn2y;
  P->m = m;
  P->words = words;
  P->wpr = wpr;
  return UW_OK;
}

extern "C" {

uw_plan* uw_plan_create(int d, int R, int q, int p, int boundary) {
  const int family = (p & UW_FILTER_SYMLET) ? 1 : 0;
  p &= ~UW_FILTER_SYMLET;
  if (d != 1 && d != 2) { fail(UW_ERR_INVALID_ARG, "d must be 1 or 2"); return nullptr; }
  if (p < 1 || p > 10) { fail(UW_ERR_INVALID_ARG, "p must be in 1..10"); return nullptr; }
  if (q < 0 || q > 6) { fail(UW_ERR_INVALID_ARG, "q must be in 0..6"); return nullptr; }
  if (boundary != UW_BOUNDARY_PERIODIC && boundary != UW_BOUNDARY_VMP) {
    fail(UW_ERR_INVALID_ARG, "boundary must be 0 (periodic) or 1 (VMP)");
    return nullptr;
  }
  int J0 = J0_min(p);
  if (R < J0 || d * (R + q) > 26) { fail(UW_ERR_INVALID_ARG, "need J0(p) <= R and d (R + q) <= 26"); return nullptr; }
  uw_plan* P = new (std::nothrow) uw_plan();
  if (!P) { fail(UW_ERR_OOM, "host allocation failed"); return nullptr; }
  P->d = d; P->R = R; P->q = q; P->p = p; P->bd = boundary; P->J0 = J0; P->family = family;
  P->M = 1 << R;
  P->N = 1 << (R + q);
  cudaGetDevice(&P->device);
  std::string err;
  try {
    if (!uw::build_tables(*P, err)) { fail(UW_ERR_INTERNAL, err); delete P; return nullptr; }
  } catch (const std::bad_alloc&) {
    fail(UW_ERR_OOM, "host allocation failed");
    delete P;
    return nullptr;
  } catch (...) {
    fail(UW_ERR_INTERNAL, "table construction failed");
    delete P;
    return nullptr;
  }
  int st = uw::upload_tables(*P);
  if (st != UW_OK) { uw_plan_destroy(P); return nullptr; }
  if (upload_mask(P, nullptr, -1) != UW_OK) { uw_plan_destroy(P); return nullptr; }
  if (uw_plan_reserve(P, 1) != UW_OK) { uw_plan_destroy(P); return nullptr; }
  uw::set_error(UW_OK, "");
  return P;
}

int uw_plan_set_coarsest(uw_plan* P, int J0) {
  if (!P) return fail(UW_ERR_INVALID_ARG, "null plan");
  if (J0 < J0_min(P->p) || J0 > P->R) return fail(UW_ERR_INVALID_ARG, "J0 out of range");
  P->J0 = J0;
  return UW_OK;
}

int uw_plan_set_mask(uw_plan* P, const int64_t* omega, int64_t m) {
  if (!P) return fail(UW_ERR_INVALID_ARG, "null plan");
  int st = upload_mask(P, omega, m);
  if (st != UW_OK) return st;
  // staging for the host API depends on m
  return uw_plan_reserve(P, P->max_batch > 0 ? P->max_batch : 1);
}

int uw_plan_reserve(uw_plan* P, int max_batch) {
  if (!P || max_batch < 1) return fail(UW_ERR_INVALID_ARG, "null plan or max_batch < 1");
  size_t wb = uw::workspace_bytes(*P, max_batch);
  int64_t coeffs = P->d == 1 ? (int64_t)P->M : (int64_t)P->M * P->M;
  // bytes per staging slot, a multiple of 256 so that the second slot keeps
  // the alignment of the first (the line kernels copy 16-byte chunks)
  size_t sb = ((size_t)max_batch * (size_t)(coeffs + P->m) * sizeof(double) + 512 + 255) & ~(size_t)255;
  if (P->d_stage && wb <= P->work_bytes && sb <= P->stage_bytes) {
    // the buffers already hold this batch (a smaller mask after the default
    // one, or a smaller batch): keep them, and their slot stride
    P->max_batch = max_batch;
    return UW_OK;
  }
  void* w = nullptr;
  void* s = nullptr;
  if (wb && cudaMalloc(&w, wb) != cudaSuccess) { cudaGetLastError(); return fail(UW_ERR_OOM, "workspace allocation failed"); }
  if (sb && cudaMalloc(&s, 2 * sb) != cudaSuccess) { cudaFree(w); cudaGetLastError(); return fail(UW_ERR_OOM, "staging allocation failed"); }
  uw_host_wait(P);   // no asynchronous host call may still use the old buffers
  cudaFree(P->d_work);
  cudaFree(P->d_stage);
  P->d_work = w;
  P->work_bytes = wb;
  P->d_stage = s;
  P->stage_bytes = sb;
  P->max_batch = max_batch;
  return UW_OK;
}

int64_t uw_plan_num_samples(const uw_plan* P) { return P ? P->m : -1; }
int64_t uw_plan_num_coeffs(const uw_plan* P) { return P ? (P->d == 1 ? (int64_t)P->M : (int64_t)P->M * P->M) : -1; }
int uw_plan_coarsest(const uw_plan* P) { return P ? P->J0 : -1; }
int64_t uw_plan_n(const uw_plan* P) { return P ? P->N : -1; }
int uw_plan_last_launches(const uw_plan* P) { return P ? P->last_launches : -1; }

int64_t uw_plan_table(const uw_plan* P, int which, double* out, int64_t cap) {
  if (!P) return -1;
  const std::vector<double>* v = nullptr;
  switch (which) {
    case 0: v = &P->h; break;
    case 1: v = &P->taps; break;
    case 2: v = &P->EL; break;
    case 3: v = &P->ER; break;
    case 4: v = &P->PL; break;
    case 5: v = &P->QL; break;
    case 6: v = &P->PR; break;
    case 7: v = &P->QR; break;
    default: return -1;
  }
  int64_t n = (int64_t)v->size();
  if (out && cap > 0) std::memcpy(out, v->data(), sizeof(double) * (size_t)std::min(n, cap));
  return n;
}

int64_t uw_host_table(int p, int q, int which, double* out, int64_t cap) {
  const int family = (p & UW_FILTER_SYMLET) ? 1 : 0;
  p &= ~UW_FILTER_SYMLET;
  if (p < 1 || p > 10 || q < 0 || q > 6) return -1;
  uw_plan T;
  T.p = p;
  T.family = family;
  T.q = q;
  std::string err;
  try {
    if (!uw::build_tables(T, err)) return -1;
  } catch (...) {
    return -1;
  }
  return uw_plan_table(&T, which, out, cap);
}

void uw_plan_destroy(uw_plan* P) {
  if (!P) return;
  uw_host_wait(P);
  for (auto& slot : P->ev)
    for (void*& e : slot)
      if (e) cudaEventDestroy((cudaEvent_t)e);
  if (P->s_up) cudaStreamDestroy((cudaStream_t)P->s_up);
  if (P->s_down) cudaStreamDestroy((cudaStream_t)P->s_down);
  for (auto& g : P->hgraphs)
    if (g.exec) cudaGraphExecDestroy((cudaGraphExec_t)g.exec);
  if (P->s_cap) cudaStreamDestroy((cudaStream_t)P->s_cap);
  uw::profiler_free(*P);
  cudaFree(P->d_tab64);
  cudaFree(P->d_tab32);
  cudaFree(P->d_mask);
  cudaFree(P->d_prefix);
  cudaFree(P->d_work);
  cudaFree(P->d_stage);
  cudaFree(P->d_tc);
  cudaFree(P->d_umma);
  cudaFree(P->d_f32);
  cudaFree(P->d_sync);
  cudaFree(P->d_coarse);
  cudaFree(P->d_pos);
  cudaFree(P->d_nat2y);
  delete P;
}

int uw_last_error(void) { return uw::g_last_status; }
const char* uw_last_message(void) { return uw::g_last_msg.c_str(); }

const char* uw_status_string(int s) {
  switch (s) {
    case UW_OK: return "ok";
    case UW_ERR_INVALID_ARG: return "invalid argument";
    case UW_ERR_UNSUPPORTED: return "unsupported";
    case UW_ERR_OOM: return "out of memory";
    case UW_ERR_CUDA: return "CUDA error";
    case UW_ERR_TIMEOUT: return "timeout";
    case UW_ERR_INTERNAL: return "internal error";
    default: return "unknown status";
  }
}

}  // extern "C"
