// One polynomial and its gradient at one point in the integer format of
// ht_mpi.cuh (host+device: the evaluation kernel runs it per lane, the host
// tests run it as is).  The reverse-mode sweep is the one of ht_eval.cuh.
#pragma once
#include <cmath>

#include "ht_mpi.cuh"

namespace ht {
namespace mpi {

template <int L>
struct IntW;
template <>
struct IntW<1> {
  static constexpr int W = 3, WA = 2;
};
template <>
struct IntW<2> {
  static constexpr int W = 5, WA = 4;  // product limbs, accumulator limbs (2L)
};
template <>
struct IntW<4> {
  static constexpr int W = 8, WA = 8;
};

// log2 |z| from the leading limbs (-1000 for zero)
HT_HD float log2_mod(double re, double im) {
  if (re == 0.0 && im == 0.0) return -1000.0f;
  const int er = re == 0.0 ? -1100 : ilog2(re), ei = im == 0.0 ? -1100 : ilog2(im);
  const int e = er > ei ? er : ei;
  const double a = std::ldexp(re, -e), b = std::ldexp(im, -e);
  return (float)e + 0.5f * std::log2((float)(a * a + b * b));
}

// Accumulator frames for polynomial m0..m1 at a point, one per output: the
// returned frame for the value, Fv[i] for the derivative by x_i.  Each frame
// lies above the largest bound on that output's terms -- log2 |c| + sum a
// log2 |x| for a value term; that minus log2 |x_v| plus log2 a_v for the
// derivative by x_v -- with one bit of margin for the float bounds and
// log2(terms + 1) + 1 bits of headroom for the sums, so every output is exact
// to its own last limb relative to its own largest term.
template <int WA>
HT_HD int frame_of(float E, int cnt) {
  int head = 1;
  while ((1 << head) < cnt + 1) ++head;
  const int Eint = (int)std::ceil((E > -3.0e4f ? E : -3.0e4f) + 1.0f) + head + 1;
  return Eint - (RB * (WA - 1) + 28);
}
template <int WA, class LG>
HT_HD int frames_for_poly(const int32_t* mon_off, const uint16_t* pairs, const float* clg, int m0, int m1,
                          const LG& lg, int nv, int* Fv) {
  float Ev[64];
  for (int i = 0; i < nv; ++i) Ev[i] = -3.0e4f;
  float E = -3.0e4f;
  for (int m = m0; m < m1; ++m) {
    const int beg = mon_off[m], k = mon_off[m + 1] - beg;
    float lt = clg[m];
    for (int r = 0; r < k; ++r) {
      const uint16_t q = pairs[beg + r];
      lt += (float)(q >> 8) * lg[q & 0xff];
    }
    E = E > lt ? E : lt;
    for (int r = 0; r < k; ++r) {
      const uint16_t q = pairs[beg + r];
      const int v = q & 0xff;
      const float d = lt - lg[v] + std::log2((float)(q >> 8));
      Ev[v] = Ev[v] > d ? Ev[v] : d;
    }
  }
  const int cnt = m1 - m0;
  for (int i = 0; i < nv; ++i) Fv[i] = frame_of<WA>(Ev[i], cnt);
  return frame_of<WA>(E, cnt);
}

// Value (through val_add(term)) and gradient (through acc.add(var, d, e,
// Fv[var])) of monomial m at the point X (converted variables); P is scratch
// for k forward products.
//
// The reverse-mode sweep of one monomial c x_{v_0}^{a_0} ... x_{v_{k-1}}^{a_{k-1}}
// is a sequence of steps, each at most one product followed by one action:
//   common factor  cf <- cf x_{v_r}              (a_r - 1 times for each r)
//   forward        P_r <- (r ? P_{r-1} : cf) x_{v_r};  value += P_{k-1}
//   backward       d_{k-1} = P_{k-2}; S = x_{v_{k-1}};
//                  for r = k-2 .. 1: d_r = P_{r-1} S, S <- S x_{v_r};
//                  d_0 = cf S                     (k = 1: d_0 = cf)
// with every d_r added into the row as a_r d_r (acc.add) and the value through
// val_add.  The loop runs the steps of a monomial through a single product
// and a single accumulation site, so the multi-limb product is emitted once
// (the 8-limb product is several hundred instructions) and its operands stay
// in registers.
template <int L, class XA, class Acc, class ValAdd, class PS>
HT_HD void sweep_monomial(const int32_t* mon_off, const uint16_t* pairs, const fz<IntW<L>::W>* cfz, int m,
                          const XA& X, const int* Fv, Acc& acc, ValAdd& val_add, PS* P) {
  constexpr int W = IntW<L>::W;
  using Z = fz<W>;
  enum : int { CHAIN, FWD, BWD0, BWD_D, BWD_S, LAST, DONE };
  const int beg = mon_off[m], k = mon_off[m + 1] - beg;
  const uint16_t* pr = pairs + beg;
  Z cf = cfz[m], S = cf;
  if (k == 0) {
    val_add(cf);
    return;
  }
  int phase = CHAIN, r = 0, e = 1;
  while (phase != DONE) {
    // the step: operands, whether to multiply, and the action
    Z lhs, rhs;
    bool prod = true;
    int act = 0;  // 0 cf, 1 P[r] (+ value at r = k - 1), 2 S, 3 row entry of var
    int var = 0, ex = 1;
    if (phase == CHAIN) {
      while (r < k && e >= (pr[r] >> 8)) {  // next variable with exponent left
        ++r;
        e = 1;
      }
      if (r == k) {
        phase = FWD;
        r = 0;
        continue;
      }
      lhs = cf;
      rhs = X[pr[r] & 0xff];
      act = 0;
      ++e;
    } else if (phase == FWD) {
      lhs = r == 0 ? cf : static_cast<Z>(P[r - 1]);
      rhs = X[pr[r] & 0xff];
      act = 1;
    } else if (phase == BWD0) {  // d_{k-1} = P_{k-2} (k >= 2) or d_0 = cf (k = 1)
      lhs = k == 1 ? cf : static_cast<Z>(P[k - 2]);
      prod = false;
      act = 3;
      var = pr[k - 1] & 0xff;
      ex = pr[k - 1] >> 8;
    } else if (phase == BWD_D) {
      lhs = static_cast<Z>(P[r - 1]);
      rhs = S;
      act = 3;
      var = pr[r] & 0xff;
      ex = pr[r] >> 8;
    } else if (phase == BWD_S) {
      lhs = S;
      rhs = X[pr[r] & 0xff];
      act = 2;
    } else {  // LAST: d_0 = cf S
      lhs = cf;
      rhs = S;
      act = 3;
      var = pr[0] & 0xff;
      ex = pr[0] >> 8;
    }
    const Z t = prod ? mul<W>(lhs, rhs) : lhs;
    if (act == 0) {
      cf = t;
    } else if (act == 1) {
      if (r == k - 1)
        val_add(t);  // the last forward product is the value; the backward sweep never reads it
      else
        P[r] = t;
    } else if (act == 2) {
      S = t;
    } else {
      acc.add(var, t, ex, Fv[var]);
    }
    // next step
    if (phase == FWD) {
      if (++r == k) phase = BWD0;
    } else if (phase == BWD0) {
      if (k == 1) {
        phase = DONE;
      } else {
        S = X[pr[k - 1] & 0xff];
        r = k - 2;
        phase = r >= 1 ? BWD_D : LAST;
      }
    } else if (phase == BWD_D) {
      phase = BWD_S;
    } else if (phase == BWD_S) {
      --r;
      phase = r >= 1 ? BWD_D : LAST;
    } else if (phase == LAST) {
      phase = DONE;
    }
  }
}

// Multiplications of one monomial's sweep (for balancing work over lanes).
HT_HD int sweep_products(const uint16_t* pr, int k) {
  int c = 0;
  for (int r = 0; r < k; ++r) c += (pr[r] >> 8) - 1;
  return k == 0 ? 0 : c + (k == 1 ? 1 : 3 * k - 3);
}

// Value (fixed-point vr, vi in frame F) and gradient of the monomials m0..m1.
// X is anything indexable by variable that yields the converted limb string
// (a local array, or a view of shared memory).
template <int L, class XA, class Acc, class PS>
HT_HD void eval_poly_int(const int32_t* mon_off, const uint16_t* pairs, const fz<IntW<L>::W>* cfz, int m0, int m1,
                         const XA& X, int F, const int* Fv, Acc& acc, int32_t* vr, int32_t* vi, PS* P) {
  constexpr int W = IntW<L>::W, WA = IntW<L>::WA;
  auto val_add = [&](const fz<W>& t) { acc_add_fast<W, WA>(vr, vi, t, 1, F); };
  for (int m = m0; m < m1; ++m) sweep_monomial<L>(mon_off, pairs, cfz, m, X, Fv, acc, val_add, P);
}

}  // namespace mpi
}  // namespace ht
