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
template <int WA>
HT_HD int frames_for_poly(const int32_t* mon_off, const uint16_t* pairs, const float* clg, int m0, int m1,
                          const float* lg, int nv, int* Fv) {
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

// The complex product as called from the sweep.  On the device the 5- and
// 8-limb products (a few hundred instructions each when unrolled) run out of
// line, one copy for all call sites, so the sweep's code stays within the
// instruction cache.
#if defined(__CUDA_ARCH__)
template <int W>
__device__ __noinline__ fz<W> mul_ool(const fz<W>& a, const fz<W>& b) {
  return mul<W>(a, b);
}
#endif
template <int W>
HT_HD fz<W> mul_sw(const fz<W>& a, const fz<W>& b) {
#if defined(__CUDA_ARCH__)
  if constexpr (W >= 5) return mul_ool<W>(a, b);
#endif
  return mul<W>(a, b);
}

// Value (fixed-point vr, vi in frame F) and gradient (through acc.add(var, d,
// e, Fv[var])) of the monomials m0..m1 at the point X (converted variables);
// P is scratch for k forward products.
template <int L, class Acc>
HT_HD void eval_poly_int(const int32_t* mon_off, const uint16_t* pairs, const fz<IntW<L>::W>* cfz, int m0, int m1,
                         const fz<IntW<L>::W>* X, int F, const int* Fv, Acc& acc, int32_t* vr, int32_t* vi,
                         fz<IntW<L>::W>* P) {
  constexpr int W = IntW<L>::W, WA = IntW<L>::WA;
  using Z = fz<W>;
  for (int m = m0; m < m1; ++m) {
    const int beg = mon_off[m], k = mon_off[m + 1] - beg;
    const uint16_t* pr = pairs + beg;
    Z cf = cfz[m];
    for (int r = 0; r < k; ++r) {
      const uint16_t q = pr[r];
      for (int e = 1; e < (q >> 8); ++e) cf = mul_sw<W>(cf, X[q & 0xff]);
    }
    if (k == 0) {
      acc_add_fast<W, WA>(vr, vi, cf, 1, F);
      continue;
    }
    for (int r = 0; r < k; ++r) P[r] = mul_sw<W>(r == 0 ? cf : P[r - 1], X[pr[r] & 0xff]);
    acc_add_fast<W, WA>(vr, vi, P[k - 1], 1, F);
    if (k == 1) {
      acc.add(pr[0] & 0xff, cf, pr[0] >> 8, Fv[pr[0] & 0xff]);
      continue;
    }
    uint16_t q = pr[k - 1];
    acc.add(q & 0xff, P[k - 2], q >> 8, Fv[q & 0xff]);
    Z S = X[q & 0xff];
    for (int r = k - 2; r >= 1; --r) {
      q = pr[r];
      acc.add(q & 0xff, mul_sw<W>(P[r - 1], S), q >> 8, Fv[q & 0xff]);
      S = mul_sw<W>(S, X[q & 0xff]);
    }
    q = pr[0];
    acc.add(q & 0xff, mul_sw<W>(cf, S), q >> 8, Fv[q & 0xff]);
  }
}

}  // namespace mpi
}  // namespace ht
