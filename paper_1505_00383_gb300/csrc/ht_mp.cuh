// Complex double, double double and quad double arithmetic on the device.
//
// Section 1 of Verschelde & Yu (2015) computes in complex double double and
// quad double arithmetic built from error-free transformations.  This header
// is this library's own version of that arithmetic, written for the fused
// multiply-add of sm_103a:
//   * two_prod(a, b) is one multiply and one fma (no Veltkamp splitting);
//   * a double double product sums the cross terms with fma into the error of
//     the leading product;
//   * a quad double product and sum group the partial terms by their order of
//     magnitude (u^0 .. u^3, u = 2^-53): terms of orders 0..2 are summed with
//     two_sum so that their rounding errors move to the next order, order-3
//     terms are summed plainly, and the four resulting components are
//     renormalised by one bottom-up and one top-down sweep of two_sum;
//   * the complex product computes each component as one fused two-term dot
//     product (a.re b.re - a.im b.im) instead of two products and a sum;
//   * the complex quad double operations are out-of-line functions: inlined,
//     each is a thousand instructions, and the kernels would spend their time
//     waiting for instruction fetch.
// The error of every operation is a small multiple of u^L times the sum of the
// moduli of its operands' terms, which is the scale the library's accuracy
// contract is stated in.  All primitives use explicitly rounded intrinsics so
// that no compiler contraction can change an error-free transformation.
#pragma once
#include <cstdint>

namespace ht {

// ------------------------------------------------------------ primitives
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = __dadd_rn(a, b);
  double bv = __dsub_rn(s, a);
  e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bv)), __dsub_rn(b, bv));
}
// Requires exponent(a) >= exponent(b) or a == 0.
__device__ __forceinline__ void fast_two_sum(double a, double b, double& s, double& e) {
  s = __dadd_rn(a, b);
  e = __dsub_rn(b, __dsub_rn(s, a));
}
__device__ __forceinline__ void two_prod(double a, double b, double& p, double& e) {
  p = __dmul_rn(a, b);
  e = __fma_rn(a, b, -p);
}

// ------------------------------------------------------------ double double
struct dd {
  double hi, lo;
};
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  double s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __dadd_rn(e, __dadd_rn(a.lo, b.lo));
  dd r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ dd dd_neg(dd a) { return dd{-a.hi, -a.lo}; }
__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  double p, e;
  two_prod(a.hi, b.hi, p, e);
  e = __fma_rn(a.hi, b.lo, e);
  e = __fma_rn(a.lo, b.hi, e);
  dd r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ dd dd_mul_d(dd a, double b) {
  double p, e;
  two_prod(a.hi, b, p, e);
  e = __fma_rn(a.lo, b, e);
  dd r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}
// a * b + c * d as one rounding to double double.
__device__ __forceinline__ dd dd_dot2(dd a, dd b, dd c, dd d) {
  double p1, e1, p2, e2, s, t;
  two_prod(a.hi, b.hi, p1, e1);
  two_prod(c.hi, d.hi, p2, e2);
  two_sum(p1, p2, s, t);
  t = __dadd_rn(t, __dadd_rn(e1, e2));
  t = __fma_rn(a.hi, b.lo, t);
  t = __fma_rn(a.lo, b.hi, t);
  t = __fma_rn(c.hi, d.lo, t);
  t = __fma_rn(c.lo, d.hi, t);
  dd r;
  fast_two_sum(s, t, r.hi, r.lo);
  return r;
}
// Reciprocal and square root by one Newton step from the double value.
__device__ __forceinline__ dd dd_div(dd a, dd b) {
  double q1 = __ddiv_rn(a.hi, b.hi);
  dd r = dd_sub(a, dd_mul_d(b, q1));  // remainder
  double q2 = __ddiv_rn(r.hi, b.hi);
  dd q;
  fast_two_sum(q1, q2, q.hi, q.lo);
  r = dd_sub(r, dd_mul_d(b, q2));
  double q3 = __ddiv_rn(r.hi, b.hi);
  return dd_add(q, dd{q3, 0.0});
}
__device__ __forceinline__ dd dd_sqrt(dd a) {
  if (a.hi <= 0.0) return dd{__dsqrt_rn(a.hi), 0.0};
  double y = __dsqrt_rn(a.hi);
  // y + (a - y^2) / (2 y)
  double p, e;
  two_prod(y, y, p, e);
  dd r = dd_sub(a, dd{p, e});
  double c = __ddiv_rn(r.hi, 2.0 * y);
  dd out;
  fast_two_sum(y, c, out.hi, out.lo);
  return out;
}

// ------------------------------------------------------------ quad double
struct qd {
  double x[4];
};
// One bottom-up and one top-down sweep of two_sum: preserves the exact sum,
// leaves the leading component the rounded total and spreads the rest.
__device__ __forceinline__ qd qd_renorm(double c0, double c1, double c2, double c3) {
  two_sum(c2, c3, c2, c3);
  two_sum(c1, c2, c1, c2);
  two_sum(c0, c1, c0, c1);
  two_sum(c1, c2, c1, c2);
  two_sum(c2, c3, c2, c3);
  return qd{{c0, c1, c2, c3}};
}
__device__ __forceinline__ qd qd_neg(qd a) { return qd{{-a.x[0], -a.x[1], -a.x[2], -a.x[3]}}; }
__device__ __forceinline__ qd qd_add(qd a, qd b) {
  double s0, e0, s1, e1, s2, e2, t, t2, t3;
  two_sum(a.x[0], b.x[0], s0, e0);  // order 0, error of order 1
  two_sum(a.x[1], b.x[1], s1, e1);  // order 1, error of order 2
  two_sum(a.x[2], b.x[2], s2, e2);  // order 2, error of order 3
  double s3 = __dadd_rn(a.x[3], b.x[3]);
  two_sum(s1, e0, s1, t);   // order 1
  two_sum(s2, e1, s2, t2);  // order 2
  two_sum(s2, t, s2, t3);
  s3 = __dadd_rn(s3, __dadd_rn(e2, __dadd_rn(t2, t3)));
  return qd_renorm(s0, s1, s2, s3);
}
__device__ __forceinline__ qd qd_sub(qd a, qd b) { return qd_add(a, qd_neg(b)); }

// Accumulate the terms of one order: s absorbs v, the rounding error of the
// sum goes to the next order's plain accumulator.
__device__ __forceinline__ void acc2(double& s, double v, double& next) {
  double e;
  two_sum(s, v, s, e);
  next = __dadd_rn(next, e);
}
// sum over i of sign_i a_i * b_i for up to two products (np = 1 or 2), rounded
// once to quad double.
template <int NP>
__device__ __forceinline__ qd qd_dot(const qd* a, const qd* b, const double* sign) {
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  double o2 = 0;  // order-2 accumulator fed by order-1 rounding errors (summed with two_sum below)
  // order 0 and 1 products with errors
  double p00[NP], q00[NP], p01[NP], q01[NP], p10[NP], q10[NP];
  double p02[NP], q02[NP], p11[NP], q11[NP], p20[NP], q20[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    double sa = sign[k];
    two_prod(sa * a[k].x[0], b[k].x[0], p00[k], q00[k]);
    two_prod(sa * a[k].x[0], b[k].x[1], p01[k], q01[k]);
    two_prod(sa * a[k].x[1], b[k].x[0], p10[k], q10[k]);
    two_prod(sa * a[k].x[0], b[k].x[2], p02[k], q02[k]);
    two_prod(sa * a[k].x[1], b[k].x[1], p11[k], q11[k]);
    two_prod(sa * a[k].x[2], b[k].x[0], p20[k], q20[k]);
  }
  // order 0
  s0 = p00[0];
  double o1e = 0;  // order-1 terms produced by order-0 sums
  if (NP == 2) two_sum(s0, p00[1], s0, o1e);
  // order 1: p01, p10, q00 (+ o1e); errors go to order 2 (kept exactly in a list)
  double o2e[2 * NP + 2];
  int n2 = 0;
  s1 = o1e;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    double e;
    two_sum(s1, p01[k], s1, e);
    o2e[n2++] = e;
    two_sum(s1, p10[k], s1, e);
    o2e[n2++] = e;
    two_sum(s1, q00[k], s1, e);
    o2e[n2++] = e;
  }
  // order 2: p02, p11, p20, q01, q10 and the order-1 errors; errors to order 3
  s2 = 0;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    acc2(s2, p02[k], s3);
    acc2(s2, p11[k], s3);
    acc2(s2, p20[k], s3);
    acc2(s2, q01[k], s3);
    acc2(s2, q10[k], s3);
  }
#pragma unroll
  for (int i = 0; i < 3 * NP; ++i) acc2(s2, o2e[i], s3);
  (void)o2;
  // order 3: plain
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    double sa = sign[k];
    double t = __dmul_rn(sa * a[k].x[0], b[k].x[3]);
    t = __fma_rn(sa * a[k].x[1], b[k].x[2], t);
    t = __fma_rn(sa * a[k].x[2], b[k].x[1], t);
    t = __fma_rn(sa * a[k].x[3], b[k].x[0], t);
    t = __dadd_rn(t, __dadd_rn(q02[k], __dadd_rn(q11[k], q20[k])));
    s3 = __dadd_rn(s3, t);
  }
  return qd_renorm(s0, s1, s2, s3);
}
__device__ __forceinline__ qd qd_mul(qd a, qd b) {
  const double one[1] = {1.0};
  return qd_dot<1>(&a, &b, one);
}
__device__ __forceinline__ qd qd_mul_d(qd a, double b) {
  double p0, q0, p1, q1, p2, q2;
  two_prod(a.x[0], b, p0, q0);
  two_prod(a.x[1], b, p1, q1);
  two_prod(a.x[2], b, p2, q2);
  double s1, e1, s2 = 0, s3 = 0;
  two_sum(p1, q0, s1, e1);
  acc2(s2, p2, s3);
  acc2(s2, q1, s3);
  acc2(s2, e1, s3);
  s3 = __dadd_rn(s3, __fma_rn(a.x[3], b, q2));
  return qd_renorm(p0, s1, s2, s3);
}
__device__ __forceinline__ qd qd_from(double d) { return qd{{d, 0.0, 0.0, 0.0}}; }
// Long division: three quotient digits from the double quotient, each followed
// by an exact-enough remainder update, then a fourth digit.
__device__ __forceinline__ qd qd_div(qd a, qd b) {
  double q0 = __ddiv_rn(a.x[0], b.x[0]);
  qd r = qd_sub(a, qd_mul_d(b, q0));
  double q1 = __ddiv_rn(r.x[0], b.x[0]);
  r = qd_sub(r, qd_mul_d(b, q1));
  double q2 = __ddiv_rn(r.x[0], b.x[0]);
  r = qd_sub(r, qd_mul_d(b, q2));
  double q3 = __ddiv_rn(r.x[0], b.x[0]);
  r = qd_sub(r, qd_mul_d(b, q3));
  double q4 = __ddiv_rn(r.x[0], b.x[0]);
  qd q = qd_renorm(q0, q1, q2, q3);
  return qd_add(q, qd_from(q4));
}
// Square root: Newton y <- y + (a - y^2) / (2 y) twice from the double root.
__device__ __forceinline__ qd qd_sqrt(qd a) {
  if (a.x[0] <= 0.0) return qd_from(__dsqrt_rn(a.x[0]));
  qd y = qd_from(__dsqrt_rn(a.x[0]));
  for (int it = 0; it < 3; ++it) {
    qd r = qd_sub(a, qd_mul(y, y));
    qd c = qd_div(r, qd_mul_d(y, 2.0));
    y = qd_add(y, c);
  }
  return y;
}

// ------------------------------------------------------------ complex types
template <int L>
struct cx;
template <>
struct cx<1> {
  double re, im;
};
template <>
struct cx<2> {
  dd re, im;
};
template <>
struct cx<4> {
  qd re, im;
};

// Leading limb of a real part (for norms and tests in double).
__device__ __forceinline__ double lead(double a) { return a; }
__device__ __forceinline__ double lead(dd a) { return a.hi; }
__device__ __forceinline__ double lead(qd a) { return a.x[0]; }

template <int L>
__device__ __forceinline__ cx<L> czero();
template <>
__device__ __forceinline__ cx<1> czero<1>() { return cx<1>{0.0, 0.0}; }
template <>
__device__ __forceinline__ cx<2> czero<2>() { return cx<2>{dd{0, 0}, dd{0, 0}}; }
template <>
__device__ __forceinline__ cx<4> czero<4>() { return cx<4>{qd{{0, 0, 0, 0}}, qd{{0, 0, 0, 0}}}; }

template <int L>
__device__ __forceinline__ cx<L> creal(double d);
template <>
__device__ __forceinline__ cx<1> creal<1>(double d) { return cx<1>{d, 0.0}; }
template <>
__device__ __forceinline__ cx<2> creal<2>(double d) { return cx<2>{dd{d, 0}, dd{0, 0}}; }
template <>
__device__ __forceinline__ cx<4> creal<4>(double d) { return cx<4>{qd_from(d), qd_from(0.0)}; }

// complex double
__device__ __forceinline__ cx<1> cadd(cx<1> a, cx<1> b) { return cx<1>{__dadd_rn(a.re, b.re), __dadd_rn(a.im, b.im)}; }
__device__ __forceinline__ cx<1> csub(cx<1> a, cx<1> b) { return cx<1>{__dsub_rn(a.re, b.re), __dsub_rn(a.im, b.im)}; }
__device__ __forceinline__ cx<1> cmul(cx<1> a, cx<1> b) {
  return cx<1>{__fma_rn(a.re, b.re, -__dmul_rn(a.im, b.im)), __fma_rn(a.re, b.im, __dmul_rn(a.im, b.re))};
}
// acc + e * d with e a small real (an exponent)
__device__ __forceinline__ cx<1> caxpy(cx<1> acc, double e, cx<1> d) {
  return cx<1>{__fma_rn(e, d.re, acc.re), __fma_rn(e, d.im, acc.im)};
}
__device__ __forceinline__ cx<1> cscale(cx<1> a, double s) { return cx<1>{__dmul_rn(a.re, s), __dmul_rn(a.im, s)}; }

// complex double double
__device__ __forceinline__ cx<2> cadd(cx<2> a, cx<2> b) { return cx<2>{dd_add(a.re, b.re), dd_add(a.im, b.im)}; }
__device__ __forceinline__ cx<2> csub(cx<2> a, cx<2> b) { return cx<2>{dd_sub(a.re, b.re), dd_sub(a.im, b.im)}; }
__device__ __forceinline__ cx<2> cmul(cx<2> a, cx<2> b) {
  return cx<2>{dd_dot2(a.re, b.re, dd_neg(a.im), b.im), dd_dot2(a.re, b.im, a.im, b.re)};
}
__device__ __forceinline__ cx<2> cscale(cx<2> a, double s) { return cx<2>{dd_mul_d(a.re, s), dd_mul_d(a.im, s)}; }
__device__ __forceinline__ cx<2> caxpy(cx<2> acc, double e, cx<2> d) { return cadd(acc, cscale(d, e)); }

// complex quad double
static __device__ __noinline__ cx<4> cadd(cx<4> a, cx<4> b) { return cx<4>{qd_add(a.re, b.re), qd_add(a.im, b.im)}; }
static __device__ __noinline__ cx<4> csub(cx<4> a, cx<4> b) { return cx<4>{qd_sub(a.re, b.re), qd_sub(a.im, b.im)}; }
static __device__ __noinline__ cx<4> cmul(cx<4> a, cx<4> b) {
  qd x1[2] = {a.re, a.im}, y1[2] = {b.re, b.im};
  const double s1[2] = {1.0, -1.0};
  qd x2[2] = {a.re, a.im}, y2[2] = {b.im, b.re};
  const double s2[2] = {1.0, 1.0};
  return cx<4>{qd_dot<2>(x1, y1, s1), qd_dot<2>(x2, y2, s2)};
}
static __device__ __noinline__ cx<4> cscale(cx<4> a, double s) { return cx<4>{qd_mul_d(a.re, s), qd_mul_d(a.im, s)}; }
static __device__ __noinline__ cx<4> caxpy(cx<4> acc, double e, cx<4> d) { return cadd(acc, cscale(d, e)); }

// ------------------------------------------------------------ L-limb reals
template <int L>
struct rtype;
template <>
struct rtype<1> {
  using t = double;
};
template <>
struct rtype<2> {
  using t = dd;
};
template <>
struct rtype<4> {
  using t = qd;
};
template <int L>
using rl = typename rtype<L>::t;

__device__ __forceinline__ double r_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double r_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double r_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double r_div(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double r_sqrt(double a) { return __dsqrt_rn(a); }
__device__ __forceinline__ dd r_add(dd a, dd b) { return dd_add(a, b); }
__device__ __forceinline__ dd r_sub(dd a, dd b) { return dd_sub(a, b); }
__device__ __forceinline__ dd r_mul(dd a, dd b) { return dd_mul(a, b); }
__device__ __forceinline__ dd r_div(dd a, dd b) { return dd_div(a, b); }
__device__ __forceinline__ dd r_sqrt(dd a) { return dd_sqrt(a); }
__device__ __forceinline__ qd r_add(qd a, qd b) { return qd_add(a, b); }
__device__ __forceinline__ qd r_sub(qd a, qd b) { return qd_sub(a, b); }
__device__ __forceinline__ qd r_mul(qd a, qd b) { return qd_mul(a, b); }
static __device__ __noinline__ qd r_div(qd a, qd b) { return qd_div(a, b); }
static __device__ __noinline__ qd r_sqrt(qd a) { return qd_sqrt(a); }
template <int L>
__device__ __forceinline__ rl<L> r_from(double d);
template <>
__device__ __forceinline__ double r_from<1>(double d) { return d; }
template <>
__device__ __forceinline__ dd r_from<2>(double d) { return dd{d, 0.0}; }
template <>
__device__ __forceinline__ qd r_from<4>(double d) { return qd_from(d); }
// a - b for two doubles, in L-limb precision (exact for L >= 2)
template <int L>
__device__ __forceinline__ rl<L> r_diff(double a, double b) {
  if constexpr (L == 1) {
    return __dsub_rn(a, b);
  } else {
    double s, e;
    two_sum(a, -b, s, e);
    if constexpr (L == 2) {
      return dd{s, e};
    } else {
      return qd{{s, e, 0.0, 0.0}};
    }
  }
}
// Limb l of an L-limb real, and an L-limb real from its limbs (for staging
// values in shared memory).
__device__ __forceinline__ double r_limb(double a, int) { return a; }
__device__ __forceinline__ double r_limb(dd a, int l) { return l == 0 ? a.hi : a.lo; }
__device__ __forceinline__ double r_limb(qd a, int l) { return a.x[l]; }
template <int L>
__device__ __forceinline__ rl<L> r_of(const double* v) {
  if constexpr (L == 1) {
    return v[0];
  } else if constexpr (L == 2) {
    return dd{v[0], v[1]};
  } else {
    return qd{{v[0], v[1], v[2], v[3]}};
  }
}
__device__ __forceinline__ bool r_finite(double a) { return isfinite(a); }
__device__ __forceinline__ bool r_finite(dd a) { return isfinite(a.hi) && isfinite(a.lo); }
__device__ __forceinline__ bool r_finite(qd a) {
  return isfinite(a.x[0]) && isfinite(a.x[1]) && isfinite(a.x[2]) && isfinite(a.x[3]);
}

// ------------------------------------------------------------ complex helpers
// |a|^2, conj(a) * b and a * s (s an L-limb real), one rounding per component.
__device__ __forceinline__ double cabs2(cx<1> a) { return __fma_rn(a.re, a.re, __dmul_rn(a.im, a.im)); }
__device__ __forceinline__ dd cabs2(cx<2> a) { return dd_dot2(a.re, a.re, a.im, a.im); }
static __device__ __noinline__ qd cabs2(cx<4> a) {
  qd x[2] = {a.re, a.im};
  const double s[2] = {1.0, 1.0};
  return qd_dot<2>(x, x, s);
}
__device__ __forceinline__ cx<1> cconjmul(cx<1> a, cx<1> b) {
  return cx<1>{__fma_rn(a.re, b.re, __dmul_rn(a.im, b.im)), __fma_rn(a.re, b.im, -__dmul_rn(a.im, b.re))};
}
__device__ __forceinline__ cx<2> cconjmul(cx<2> a, cx<2> b) {
  return cx<2>{dd_dot2(a.re, b.re, a.im, b.im), dd_dot2(a.re, b.im, dd_neg(a.im), b.re)};
}
static __device__ __noinline__ cx<4> cconjmul(cx<4> a, cx<4> b) {
  qd x1[2] = {a.re, a.im}, y1[2] = {b.re, b.im};
  const double s1[2] = {1.0, 1.0};
  qd x2[2] = {a.re, a.im}, y2[2] = {b.im, b.re};
  const double s2[2] = {1.0, -1.0};
  return cx<4>{qd_dot<2>(x1, y1, s1), qd_dot<2>(x2, y2, s2)};
}
__device__ __forceinline__ cx<1> cscale_r(cx<1> a, double s) { return cscale(a, s); }
__device__ __forceinline__ cx<2> cscale_r(cx<2> a, dd s) { return cx<2>{dd_mul(a.re, s), dd_mul(a.im, s)}; }
static __device__ __noinline__ cx<4> cscale_r(cx<4> a, qd s) { return cx<4>{qd_mul(a.re, s), qd_mul(a.im, s)}; }
// Modulus from the leading limbs in double (used for norms and tests only).
template <int L>
__device__ __forceinline__ double cabs_lead(cx<L> a) {
  double r = lead(a.re), i = lead(a.im);
  return __dsqrt_rn(__dadd_rn(__dmul_rn(r, r), __dmul_rn(i, i)));
}
template <int L>
__device__ __forceinline__ bool cfinite(cx<L> a) {
  return r_finite(a.re) && r_finite(a.im);
}

// ------------------------------------------------------------ SoA access
// A point batch is [count][2][L][n] doubles: plane (i, c, l) holds component
// c (0 re, 1 im), limb l of entry i for all n points, point index fastest.
template <int L>
__device__ __forceinline__ cx<L> ld(const double* base, int64_t i, int64_t n, int64_t p);
template <>
__device__ __forceinline__ cx<1> ld<1>(const double* b, int64_t i, int64_t n, int64_t p) {
  const double* q = b + (i * 2) * n + p;
  return cx<1>{q[0], q[n]};
}
template <>
__device__ __forceinline__ cx<2> ld<2>(const double* b, int64_t i, int64_t n, int64_t p) {
  const double* q = b + (i * 4) * n + p;
  return cx<2>{dd{q[0], q[n]}, dd{q[2 * n], q[3 * n]}};
}
template <>
__device__ __forceinline__ cx<4> ld<4>(const double* b, int64_t i, int64_t n, int64_t p) {
  const double* q = b + (i * 8) * n + p;
  return cx<4>{qd{{q[0], q[n], q[2 * n], q[3 * n]}}, qd{{q[4 * n], q[5 * n], q[6 * n], q[7 * n]}}};
}
template <int L>
__device__ __forceinline__ void st(double* base, int64_t i, int64_t n, int64_t p, cx<L> z);
template <>
__device__ __forceinline__ void st<1>(double* b, int64_t i, int64_t n, int64_t p, cx<1> z) {
  double* q = b + (i * 2) * n + p;
  q[0] = z.re;
  q[n] = z.im;
}
template <>
__device__ __forceinline__ void st<2>(double* b, int64_t i, int64_t n, int64_t p, cx<2> z) {
  double* q = b + (i * 4) * n + p;
  q[0] = z.re.hi;
  q[n] = z.re.lo;
  q[2 * n] = z.im.hi;
  q[3 * n] = z.im.lo;
}
template <>
__device__ __forceinline__ void st<4>(double* b, int64_t i, int64_t n, int64_t p, cx<4> z) {
  double* q = b + (i * 8) * n + p;
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    q[l * n] = z.re.x[l];
    q[(4 + l) * n] = z.im.x[l];
  }
}
// Coefficients are stored per monomial as [2][L] doubles (AoS: all lanes read
// the same monomial at the same time, so one broadcast line serves the warp).
template <int L>
__device__ __forceinline__ cx<L> ld_coef(const double* c) {
  if constexpr (L == 1) {
    return cx<1>{__ldg(c), __ldg(c + 1)};
  } else if constexpr (L == 2) {
    return cx<2>{dd{__ldg(c), __ldg(c + 1)}, dd{__ldg(c + 2), __ldg(c + 3)}};
  } else {
    return cx<4>{qd{{__ldg(c), __ldg(c + 1), __ldg(c + 2), __ldg(c + 3)}},
                 qd{{__ldg(c + 4), __ldg(c + 5), __ldg(c + 6), __ldg(c + 7)}}};
  }
}

}  // namespace ht
