// General arithmetic on the floating limb strings of ht_mpi.cuh for the
// tracker's linear algebra: signed sums of a few terms through one fixed-point
// frame, renormalisation, conjugation, conversion of reals, and 1/sqrt by
// Newton's iteration.  Host+device, like ht_mpi.cuh.
#pragma once
#include <cmath>

#include "ht_mpi.cuh"

namespace ht {
namespace mpi {

// ------------------------------------------------------------ general sums
// Smallest E with |re|, |im| < 2^E (from the top limb; lower limbs add less
// than one unit of it).  Zero gives a very small E.
template <int W>
HT_HD int bound_exp(const fz<W>& z) {
  for (int k = W - 1; k >= 0; --k) {
    const int32_t ar = z.r[k] < 0 ? -z.r[k] : z.r[k], ai = z.i[k] < 0 ? -z.i[k] : z.i[k];
    const int32_t mx = ar > ai ? ar : ai;
    if (mx != 0) {
      return z.f + RB * k + bitlen32((uint32_t)mx) + 1;  // (mx + 1) 2^(29 k + f) bounds the lower limbs too
    }
  }
  return -30000;
}

// Fixed-point complex (WA limbs each, frame F) to a floating fz<W>: the W
// limbs from the highest significant one down (the sign folded into the top).
template <int WA, int W>
HT_HD fz<W> fixed_to_fz(const int32_t* ar_in, const int32_t* ai_in, int F) {
  int64_t r[WA], im[WA], mr[WA], mi[WA];
  for (int k = 0; k < WA; ++k) {
    r[k] = ar_in[k];
    im[k] = ai_in[k];
  }
  carry<WA>(r);
  carry<WA>(im);
  const bool nr = r[WA - 1] < 0, ni = im[WA - 1] < 0;
  for (int k = 0; k < WA; ++k) {
    mr[k] = nr ? -r[k] : r[k];
    mi[k] = ni ? -im[k] : im[k];
  }
  carry<WA>(mr);
  carry<WA>(mi);
  int t = 0;
  for (int k = 0; k < WA; ++k)
    if (mr[k] != 0 || mi[k] != 0) t = k;
  fz<W> z;
  const int lo = t - (W - 1);  // window [lo, t]
  z.f = F + RB * lo;
  for (int k = 0; k < W; ++k) {
    const int src = lo + k;
    z.r[k] = src >= 0 ? (int32_t)r[src] : 0;
    z.i[k] = src >= 0 ? (int32_t)im[src] : 0;
  }
  if (t < WA - 1) {  // fold the sign extension above t into the window's top
    if (nr) z.r[W - 1] -= (1 << RB);
    if (ni) z.i[W - 1] -= (1 << RB);
  } else {
    z.r[W - 1] = (int32_t)r[WA - 1];
    z.i[W - 1] = (int32_t)im[WA - 1];
  }
  normalize_top<W>(z);
  return z;
}

// s times a fixed-point complex (WA limbs each, frame F), s a double, to
// fz<W>: the product is formed exactly in WA + 2 limbs per component (s's
// significand in a 24-bit and a 29-bit part) and cut to W limbs as
// fixed_to_fz does.
template <int WA, int W>
HT_HD fz<W> fixed_scaled_to_fz(const int32_t* ar, const int32_t* ai, int F, double s) {
  int64_t ms;
  int es;
  decompose(s, ms, es);  // s = ms 2^es, |ms| < 2^53
  const bool neg = ms < 0;
  const uint64_t u = (uint64_t)(neg ? -ms : ms);
  const int64_t lo = (int64_t)(u & (uint64_t)MASK), hi = (int64_t)(u >> RB);
  int64_t cr[WA + 2], ci[WA + 2];
  for (int k = 0; k < WA + 2; ++k) cr[k] = ci[k] = 0;
  for (int k = 0; k < WA; ++k) {  // |a_k lo| < 2^58, |a_k hi| < 2^53
    cr[k] += (int64_t)ar[k] * lo;
    cr[k + 1] += (int64_t)ar[k] * hi;
    ci[k] += (int64_t)ai[k] * lo;
    ci[k + 1] += (int64_t)ai[k] * hi;
  }
  if (neg)
    for (int k = 0; k < WA + 2; ++k) {
      cr[k] = -cr[k];
      ci[k] = -ci[k];
    }
  carry<WA + 2>(cr);
  carry<WA + 2>(ci);
  int32_t br[WA + 2], bi[WA + 2];  // top limbs below 2^24 in magnitude
  for (int k = 0; k < WA + 2; ++k) {
    br[k] = (int32_t)cr[k];
    bi[k] = (int32_t)ci[k];
  }
  return fixed_to_fz<WA + 2, W>(br, bi, F + es);
}

template <int W>
HT_HD bool is_zero(const fz<W>& z) {
  int32_t o = 0;
  for (int k = 0; k < W; ++k) o |= z.r[k] | z.i[k];
  return o == 0;
}

// sum_k e_k z_k (e_k small signed integers, n <= N terms), rounded to fz<W>.
// One fixed frame F of WA = W + 1 limbs: its top holds the largest bound plus
// headroom for the n terms, and F lies at most 28 bits below every nonzero
// term's limb 0 (the shift rule of acc_add_fast).  A nonzero term's top limb
// is nonzero, so F is at least 29 (W - 1) + 28 bits below the largest term's
// magnitude: each term's truncation is below 2^(1 - 29 W) times the largest.
template <int W, int N>
HT_HD fz<W> sum(const fz<W>* z, const int* e, int n) {
  constexpr int WA = W + 1;
  int E = -30000, fmax = -30000;
  for (int k = 0; k < n; ++k) {
    if (e[k] == 0 || is_zero<W>(z[k])) continue;
    const int ek = e[k] < 0 ? -e[k] : e[k];
    const int b = bound_exp<W>(z[k]) + bitlen32((uint32_t)(ek - 1));  // + ceil(log2 |e_k|)
    E = b > E ? b : E;
    fmax = z[k].f > fmax ? z[k].f : fmax;
  }
  int32_t ar[WA], ai[WA];
  for (int k = 0; k < WA; ++k) ar[k] = ai[k] = 0;
  if (fmax == -30000) {
    fz<W> zero;
    zero.f = 0;
    for (int k = 0; k < W; ++k) zero.r[k] = zero.i[k] = 0;
    return zero;
  }
  const int head = bitlen32((uint32_t)n) > 1 ? bitlen32((uint32_t)n) : 1;  // 2^head >= n + 1
  int F = E + head - (RB * (WA - 1) + 28);
  F = F > fmax - (RB - 1) ? F : fmax - (RB - 1);
  for (int k = 0; k < n; ++k)
    if (e[k] != 0 && !is_zero<W>(z[k])) acc_add_fast<W, WA>(ar, ai, z[k], e[k], F);
  return fixed_to_fz<WA, W>(ar, ai, F);
}
template <int W>
HT_HD fz<W> add(const fz<W>& a, const fz<W>& b) {
  fz<W> t[2] = {a, b};
  const int e[2] = {1, 1};
  return sum<W, 2>(t, e, 2);
}
template <int W>
HT_HD fz<W> sub(const fz<W>& a, const fz<W>& b) {
  fz<W> t[2] = {a, b};
  const int e[2] = {1, -1};
  return sum<W, 2>(t, e, 2);
}
template <int W>
HT_HD fz<W> conj(fz<W> a) {
  for (int k = 0; k < W; ++k) a.i[k] = -a.i[k];
  return a;
}
template <int W>
HT_HD fz<W> from_real(double d) {
  const double zero = 0.0;
  return from_doubles<W, 1>(&d, &zero);
}
// Value of the real part rounded to double (for norms, seeds and decisions).
template <int W>
HT_HD double real_to_double(const fz<W>& z) {
  double acc = 0.0;
  for (int k = W - 1; k >= 0; --k) {
    double lim = (double)z.r[k];
    int ex = z.f + RB * k;
    while (ex > 600) {
      lim *= bitsd((int64_t)(1023 + 600) << 52);
      ex -= 600;
    }
    while (ex < -600) {
      lim *= bitsd((int64_t)(1023 - 600) << 52);
      ex += 600;
    }
    acc += lim * bitsd((int64_t)(1023 + ex) << 52);
  }
  return acc;
}
// 1 / sqrt(v) for a positive real v (im = 0): Newton's iteration
// y <- y (3 - v y^2) / 2 from the double seed; each step doubles the bits.
template <int W>
HT_HD fz<W> inv_sqrt(const fz<W>& v, int steps) {
  const double vd = real_to_double<W>(v);
  fz<W> y = from_real<W>(1.0 / std::sqrt(vd));
  const fz<W> three = from_real<W>(3.0);
  for (int it = 0; it < steps; ++it) {
    fz<W> vy2 = mul<W>(v, mul<W>(y, y));
    fz<W> c = sub<W>(three, vy2);
    y = mul<W>(y, c);
    y.f -= 1;  // halve
  }
  return y;
}

// ------------------------------------------------------------ least squares
// Building blocks of modified Gram-Schmidt on columns of limb strings (the
// tracker's corrector, Section 2): every dot product and norm is one exact
// fixed-point sum of its products, rounded once.
template <int W>
HT_HD int inv_sqrt_steps() {
  return W >= 8 ? 3 : 2;  // from a 53-bit seed: 2 steps give 212 bits, 3 give 424
}
// sum_i conj(q_i) a_i over i < rows (rows <= N; scratch holds rows entries)
template <int W, int N>
HT_HD fz<W> dot_conj(const fz<W>* q, const fz<W>* a, int rows, fz<W>* scratch) {
  int e[N];
  for (int i = 0; i < rows; ++i) {
    scratch[i] = mul<W>(conj<W>(q[i]), a[i]);
    e[i] = 1;
  }
  return sum<W, N>(scratch, e, rows);
}
// sum_i |a_i|^2 (imaginary part exactly zero: the cross columns cancel)
template <int W, int N>
HT_HD fz<W> norm2(const fz<W>* a, int rows, fz<W>* scratch) {
  int e[N];
  for (int i = 0; i < rows; ++i) {
    scratch[i] = mul<W>(a[i], conj<W>(a[i]));
    e[i] = 1;
  }
  return sum<W, N>(scratch, e, rows);
}
// a_i -= r q_i
template <int W>
HT_HD void sub_scaled(fz<W>* a, const fz<W>& r, const fz<W>* q, int rows) {
  for (int i = 0; i < rows; ++i) a[i] = sub<W>(a[i], mul<W>(r, q[i]));
}
// sum_k e_k z_k with e = (1, -1, -1, ...): b - sum_j r_j x_j for the back
// substitution (terms[0] = b, terms[1..n] = the products)
template <int W, int N>
HT_HD fz<W> first_minus_rest(const fz<W>* terms, int n) {
  int e[N];
  for (int k = 0; k < n; ++k) e[k] = k == 0 ? 1 : -1;
  return sum<W, N>(terms, e, n);
}
// Limb string to L doubles per component (the fixed-point reading of the
// limbs: limbs 0..W-2 in [0, 2^29), top signed, frame f).
template <int W, int L>
HT_HD void to_doubles(const fz<W>& z, double* re, double* im) {
  fixed_to_doubles<W, L>(z.r, z.f, re);
  fixed_to_doubles<W, L>(z.i, z.f, im);
}

}  // namespace mpi
}  // namespace ht
