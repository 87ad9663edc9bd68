// Plain CPU oracle for many-path polynomial homotopy tracking
// (Verschelde & Yu, "Tracking Many Solution Paths of a Polynomial Homotopy on
// a Graphics Processing Unit", 2015).
//
// TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
// baseline leg of the benchmark call this library; the product path (the CUDA
// library) never does, and the two share no code, headers or tables.
//
// It is deliberately slow and plain:
//   * arithmetic in L-limb precision (L = 1 double, 2 double double, 4 quad
//     double; Section 1 and Section 4.1) is done exactly with floating-point
//     expansions and then rounded limb by limb: every real operation returns the
//     exact result rounded to the nearest L-limb number whose limbs are each the
//     correctly rounded remainder.  The exact sums use Shewchuk's expansion
//     accumulation ("Adaptive precision floating-point arithmetic", 1997) and
//     Dekker's two-product with Veltkamp splitting (no fused multiply-add);
//   * evaluation follows the host pseudo code of Table tabcpugpu (each monomial
//     evaluated and differentiated, then added to the polynomial and to the
//     Jacobian), once by the textbook product rule and once by the reverse mode
//     of Table tabmoneval;
//   * the corrector solves J dx = -h in the least squares sense by modified
//     Gram-Schmidt (Section 1, Section 2);
//   * the tracker follows Section 2: predict by extrapolation through the current
//     and up to four previous points, then evaluate-correct rounds, then step
//     control and a status of 0 (continue), -1 (failure) or 1 (success).
// Compile with -ffp-contract=off: the error-free transformations need every
// product and sum rounded on its own.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

namespace {

// ---------------------------------------------------------------- exact sums
// Veltkamp's split of a double into two 26-bit halves.
inline void split(double a, double& hi, double& lo) {
  double c = 134217729.0 * a;  // 2^27 + 1
  hi = c - (c - a);
  lo = a - hi;
}

// Dekker's two-product without fma: p + e == a * b exactly.
inline void two_prod(double a, double b, double& p, double& e) {
  p = a * b;
  double ah, al, bh, bl;
  split(a, ah, al);
  split(b, bh, bl);
  e = ((ah * bh - p) + ah * bl + al * bh) + al * bl;
}

// Exact accumulator: a nonoverlapping expansion kept in increasing magnitude
// (Shewchuk's grow-expansion with zero elimination).  round() returns the
// correctly rounded (to nearest, ties to even) value of the exact sum.
struct Acc {
  static const int CAP = 96;
  double p[CAP];
  int n = 0;

  void add(double x) {
    int i = 0;
    for (int j = 0; j < n; ++j) {
      double y = p[j];
      if (std::fabs(x) < std::fabs(y)) std::swap(x, y);
      double hi = x + y;
      double lo = y - (hi - x);
      if (lo != 0.0) p[i++] = lo;
      x = hi;
    }
    n = i;
    if (n >= CAP) std::abort();
    p[n++] = x;
  }
  void add_prod(double a, double b) {
    double q, e;
    two_prod(a, b, q, e);
    add(q);
    add(e);
  }
  double round() const {
    int k = n;
    if (k == 0) return 0.0;
    double hi = p[--k], lo = 0.0;
    while (k > 0) {
      double x = hi, y = p[--k];
      hi = x + y;
      double yr = hi - x;
      lo = y - yr;
      if (lo != 0.0) break;
    }
    // Half-way case: the discarded tail decides the direction of the tie.
    if (k > 0 && ((lo < 0.0 && p[k - 1] < 0.0) || (lo > 0.0 && p[k - 1] > 0.0))) {
      double y = lo * 2.0, x = hi + y, yr = x - hi;
      if (y == yr) hi = x;
    }
    return hi;
  }
};

// ---------------------------------------------------------- L-limb numbers
template <int L>
struct R {
  double v[L];
};

template <int L>
inline R<L> rzero() {
  R<L> r;
  for (int i = 0; i < L; ++i) r.v[i] = 0.0;
  return r;
}
template <int L>
inline R<L> rfrom(double d) {
  R<L> r = rzero<L>();
  r.v[0] = d;
  return r;
}

// Round the exact sum held in acc to L limbs, limb by limb.
template <int L>
inline R<L> extract(Acc acc) {
  R<L> r;
  for (int i = 0; i < L; ++i) {
    double x = acc.round();
    r.v[i] = x;
    acc.add(-x);
  }
  return r;
}

template <int L>
inline R<L> radd(const R<L>& a, const R<L>& b) {
  if constexpr (L == 1) {
    R<1> r{{a.v[0] + b.v[0]}};
    return r;
  } else {
    Acc s;
    for (int i = 0; i < L; ++i) s.add(a.v[i]);
    for (int i = 0; i < L; ++i) s.add(b.v[i]);
    return extract<L>(s);
  }
}
template <int L>
inline R<L> rneg(const R<L>& a) {
  R<L> r;
  for (int i = 0; i < L; ++i) r.v[i] = -a.v[i];
  return r;
}
template <int L>
inline R<L> rsub(const R<L>& a, const R<L>& b) {
  return radd<L>(a, rneg<L>(b));
}
template <int L>
inline R<L> rmul(const R<L>& a, const R<L>& b) {
  if constexpr (L == 1) {
    R<1> r{{a.v[0] * b.v[0]}};
    return r;
  } else {
    Acc s;
    for (int i = 0; i < L; ++i)
      for (int j = 0; j < L; ++j) s.add_prod(a.v[i], b.v[j]);
    return extract<L>(s);
  }
}
// Long division with an exact remainder: each quotient digit removes about 52
// bits of the remainder; L + 2 digits are more than the L limbs need.
template <int L>
inline R<L> rdiv(const R<L>& a, const R<L>& b) {
  if constexpr (L == 1) {
    R<1> r{{a.v[0] / b.v[0]}};
    return r;
  } else {
    Acc rem, q;
    for (int i = 0; i < L; ++i) rem.add(a.v[i]);
    double b0 = b.v[0];
    for (int it = 0; it < L + 2; ++it) {
      double qi = rem.round() / b0;
      if (qi == 0.0 || !std::isfinite(qi)) {
        if (!std::isfinite(qi)) q.add(qi);
        break;
      }
      q.add(qi);
      for (int j = 0; j < L; ++j) {
        double p, e;
        two_prod(qi, b.v[j], p, e);
        rem.add(-p);
        rem.add(-e);
      }
    }
    return extract<L>(q);
  }
}
// Square root by Newton's iteration y <- (y + a / y) / 2 from the double root;
// each step doubles the number of correct bits.
template <int L>
inline R<L> rsqrt(const R<L>& a) {
  if constexpr (L == 1) {
    R<1> r{{std::sqrt(a.v[0])}};
    return r;
  } else {
    double s = std::sqrt(a.v[0]);
    if (s == 0.0 || !std::isfinite(s)) return rfrom<L>(s);
    R<L> y = rfrom<L>(s);
    R<L> half = rfrom<L>(0.5);
    for (int it = 0; it < L; ++it) y = rmul<L>(radd<L>(y, rdiv<L>(a, y)), half);
    return y;
  }
}
template <int L>
inline double rd(const R<L>& a) {  // value rounded to double
  if constexpr (L == 1) {
    return a.v[0];
  } else {
    Acc s;
    for (int i = 0; i < L; ++i) s.add(a.v[i]);
    return s.round();
  }
}

// ---------------------------------------------------------- complex numbers
template <int L>
struct C {
  R<L> re, im;
};
template <int L>
inline C<L> czero() {
  return C<L>{rzero<L>(), rzero<L>()};
}
template <int L>
inline C<L> cadd(const C<L>& a, const C<L>& b) {
  return C<L>{radd<L>(a.re, b.re), radd<L>(a.im, b.im)};
}
template <int L>
inline C<L> csub(const C<L>& a, const C<L>& b) {
  return C<L>{rsub<L>(a.re, b.re), rsub<L>(a.im, b.im)};
}
template <int L>
inline C<L> cmul(const C<L>& a, const C<L>& b) {
  return C<L>{rsub<L>(rmul<L>(a.re, b.re), rmul<L>(a.im, b.im)),
              radd<L>(rmul<L>(a.re, b.im), rmul<L>(a.im, b.re))};
}
template <int L>
inline C<L> cscale(const C<L>& a, const R<L>& s) {
  return C<L>{rmul<L>(a.re, s), rmul<L>(a.im, s)};
}
// conj(a) * b
template <int L>
inline C<L> cconjmul(const C<L>& a, const C<L>& b) {
  return C<L>{radd<L>(rmul<L>(a.re, b.re), rmul<L>(a.im, b.im)),
              rsub<L>(rmul<L>(a.re, b.im), rmul<L>(a.im, b.re))};
}
template <int L>
inline R<L> cabs2(const C<L>& a) {
  return radd<L>(rmul<L>(a.re, a.re), rmul<L>(a.im, a.im));
}
template <int L>
inline double cabs_d(const C<L>& a) {  // modulus from the leading limbs, in double
  return std::sqrt(a.re.v[0] * a.re.v[0] + a.im.v[0] * a.im.v[0]);
}
template <int L>
inline bool cfinite(const C<L>& a) {
  for (int i = 0; i < L; ++i)
    if (!std::isfinite(a.re.v[i]) || !std::isfinite(a.im.v[i])) return false;
  return true;
}

// Layout helpers: point batches are [n_vars][2][L][n_pts] (Section 3: all
// paths' values of one quantity are stored next to each other).
template <int L>
inline C<L> load_soa(const double* base, int64_t i, int64_t p, int64_t npts) {
  C<L> z;
  for (int l = 0; l < L; ++l) {
    z.re.v[l] = base[((i * 2 + 0) * L + l) * npts + p];
    z.im.v[l] = base[((i * 2 + 1) * L + l) * npts + p];
  }
  return z;
}
template <int L>
inline void store_soa(double* base, int64_t i, int64_t p, int64_t npts, const C<L>& z) {
  for (int l = 0; l < L; ++l) {
    base[((i * 2 + 0) * L + l) * npts + p] = z.re.v[l];
    base[((i * 2 + 1) * L + l) * npts + p] = z.im.v[l];
  }
}

// ---------------------------------------------------------- the system
// Instructions of Table tabmemory: per monomial its exponents (idx) and its
// coefficient (cff), shared by all paths.
template <int L>
struct Sys {
  int nv = 0, np = 0;
  std::vector<int> off;          // [np + 1] monomial range of each polynomial
  std::vector<int8_t> exps;      // [M][nv]
  std::vector<C<L>> coef;        // [M]
  int max_deg = 0;
};

template <int L>
Sys<L> make_sys(int nv, int np, const int32_t* n_terms, const int8_t* exps, const double* coef) {
  Sys<L> s;
  s.nv = nv;
  s.np = np;
  s.off.resize(np + 1);
  s.off[0] = 0;
  for (int j = 0; j < np; ++j) s.off[j + 1] = s.off[j] + n_terms[j];
  int M = s.off[np];
  s.exps.assign(exps, exps + (size_t)M * nv);
  s.coef.resize(M);
  for (int m = 0; m < M; ++m) {
    for (int l = 0; l < L; ++l) {
      s.coef[m].re.v[l] = coef[((size_t)m * 2 + 0) * L + l];
      s.coef[m].im.v[l] = coef[((size_t)m * 2 + 1) * L + l];
    }
    int d = 0;
    for (int i = 0; i < nv; ++i) d += s.exps[(size_t)m * nv + i];
    s.max_deg = std::max(s.max_deg, d);
  }
  return s;
}

// Textbook evaluation (Table tabcpugpu, host side): every monomial c * prod x_i^a_i
// by repeated multiplication, every derivative a_i c x_i^(a_i - 1) prod_{l != i} x_l^a_l
// by the product rule, summed into h and J.
template <int L>
void eval_naive(const Sys<L>& s, const C<L>* x, C<L>* val, C<L>* jac) {
  for (int j = 0; j < s.np; ++j) {
    val[j] = czero<L>();
    for (int i = 0; i < s.nv; ++i) jac[(size_t)j * s.nv + i] = czero<L>();
    for (int m = s.off[j]; m < s.off[j + 1]; ++m) {
      const int8_t* a = &s.exps[(size_t)m * s.nv];
      C<L> term = s.coef[m];
      for (int i = 0; i < s.nv; ++i)
        for (int e = 0; e < a[i]; ++e) term = cmul<L>(term, x[i]);
      val[j] = cadd<L>(val[j], term);
      for (int i = 0; i < s.nv; ++i) {
        if (a[i] == 0) continue;
        C<L> d = cscale<L>(s.coef[m], rfrom<L>((double)a[i]));
        for (int l = 0; l < s.nv; ++l) {
          int e = a[l] - (l == i ? 1 : 0);
          for (int r = 0; r < e; ++r) d = cmul<L>(d, x[l]);
        }
        jac[(size_t)j * s.nv + i] = cadd<L>(jac[(size_t)j * s.nv + i], d);
      }
    }
  }
}

// Reverse mode on a product x_1 x_2 ... x_k of k variables, in the slot order of
// Table tabmoneval (written there for k = 4, generalised here):
//   slots 0..k-2     forward products x_1, x_1x_2, ..., x_1...x_{k-1}
//                    (slot k-2 is the derivative with respect to x_k),
//   slot 2k-1        the value x_1...x_k,
//   slot 2k-2        the derivative with respect to x_{k-1},
//   slot k-1         the running backward product x_j...x_k,
//   slots k..2k-3    the derivatives with respect to x_{k-2}, ..., x_1 in the
//                    order they are computed.
// For k >= 2 it takes 3k - 5 multiplications.  d[i] receives the derivative with
// respect to x_{i+1}; the return value is the number of multiplications.
template <int L>
int speelpenning(int k, const C<L>* xs, C<L>* slots, C<L>* value, C<L>* d) {
  if (k == 1) {
    slots[0] = xs[0];
    slots[1] = C<L>{rfrom<L>(1.0), rzero<L>()};
    *value = xs[0];
    d[0] = slots[1];
    return 0;
  }
  int nmul = 0;
  slots[0] = xs[0];
  for (int j = 1; j <= k - 2; ++j) {  // forward products
    slots[j] = cmul<L>(slots[j - 1], xs[j]);
    ++nmul;
  }
  slots[2 * k - 1] = cmul<L>(slots[k - 2], xs[k - 1]);  // value
  ++nmul;
  *value = slots[2 * k - 1];
  d[k - 1] = slots[k - 2];
  if (k == 2) {
    slots[1] = xs[1];  // backward product x_2: no multiplication
    slots[2] = xs[1];  // derivative with respect to x_1
    d[0] = xs[1];
    return nmul;
  }
  slots[2 * k - 2] = cmul<L>(slots[k - 3], xs[k - 1]);  // d / d x_{k-1}
  ++nmul;
  d[k - 2] = slots[2 * k - 2];
  slots[k - 1] = xs[k - 1];  // backward product x_k
  int out = k;
  for (int j = k - 2; j >= 1; --j) {  // derivative with respect to x_j (1-based)
    if (j >= 2) {
      slots[k - 1] = cmul<L>(xs[j], slots[k - 1]);  // x_{j+1} ... x_k
      slots[out] = cmul<L>(slots[j - 2], slots[k - 1]);
      nmul += 2;
    } else {
      slots[out] = cmul<L>(xs[1], slots[k - 1]);  // x_2 ... x_k
      nmul += 1;
    }
    d[j - 1] = slots[out];
    ++out;
  }
  return nmul;
}

// Reverse-mode evaluation: per monomial the common factor
// c * prod_{a_i > 1} x_i^(a_i - 1) (Section 1: the factor shared by all
// derivatives), times the Speelpenning products of the variables with
// positive exponent.
template <int L>
void eval_speel(const Sys<L>& s, const C<L>* x, C<L>* val, C<L>* jac) {
  std::vector<C<L>> xs(s.nv), slots(2 * s.nv + 2), d(s.nv);
  std::vector<int> var(s.nv), ex(s.nv);
  for (int j = 0; j < s.np; ++j) {
    val[j] = czero<L>();
    for (int i = 0; i < s.nv; ++i) jac[(size_t)j * s.nv + i] = czero<L>();
    for (int m = s.off[j]; m < s.off[j + 1]; ++m) {
      const int8_t* a = &s.exps[(size_t)m * s.nv];
      int k = 0;
      C<L> cf = s.coef[m];
      for (int i = 0; i < s.nv; ++i) {
        if (a[i] <= 0) continue;
        var[k] = i;
        ex[k] = a[i];
        xs[k] = x[i];
        ++k;
        for (int e = 1; e < a[i]; ++e) cf = cmul<L>(cf, x[i]);
      }
      if (k == 0) {
        val[j] = cadd<L>(val[j], cf);
        continue;
      }
      C<L> value;
      speelpenning<L>(k, xs.data(), slots.data(), &value, d.data());
      val[j] = cadd<L>(val[j], cmul<L>(cf, value));
      for (int r = 0; r < k; ++r) {
        C<L> scaled = cscale<L>(cf, rfrom<L>((double)ex[r]));
        size_t idx = (size_t)j * s.nv + var[r];
        jac[idx] = cadd<L>(jac[idx], cmul<L>(scaled, d[r]));
      }
    }
  }
}

// Sum of the moduli of the terms of each output, in double: the scale that
// makes a relative error meaningful under cancellation.
template <int L>
void eval_magnitude(const Sys<L>& s, const C<L>* x, double* val, double* jac) {
  std::vector<double> ax(s.nv);
  for (int i = 0; i < s.nv; ++i) ax[i] = cabs_d<L>(x[i]);
  for (int j = 0; j < s.np; ++j) {
    val[j] = 0;
    for (int i = 0; i < s.nv; ++i) jac[(size_t)j * s.nv + i] = 0;
    for (int m = s.off[j]; m < s.off[j + 1]; ++m) {
      const int8_t* a = &s.exps[(size_t)m * s.nv];
      double c = cabs_d<L>(s.coef[m]);
      double t = c;
      for (int i = 0; i < s.nv; ++i) t *= std::pow(ax[i], (double)a[i]);
      val[j] += t;
      for (int i = 0; i < s.nv; ++i) {
        if (a[i] == 0) continue;
        double dd = c * a[i];
        for (int l = 0; l < s.nv; ++l) dd *= std::pow(ax[l], (double)(a[l] - (l == i ? 1 : 0)));
        jac[(size_t)j * s.nv + i] += dd;
      }
    }
  }
}

// ---------------------------------------------------------- least squares
// Modified Gram-Schmidt on the augmented matrix [A | b_0 .. b_{nrhs-1}]
// (rows >= cols), then back substitution R x_k = Q^H b_k for every right-hand
// side.  A is row major [rows][cols], b is [nrhs][rows], x is [nrhs][cols].
template <int L>
void mgs_solve_multi(int rows, int cols, int nrhs, const std::vector<C<L>>& A, const C<L>* b, C<L>* x) {
  const int W = cols + nrhs;
  std::vector<C<L>> M((size_t)rows * W);
  for (int i = 0; i < rows; ++i) {
    for (int j = 0; j < cols; ++j) M[(size_t)i * W + j] = A[(size_t)i * cols + j];
    for (int k = 0; k < nrhs; ++k) M[(size_t)i * W + cols + k] = b[(size_t)k * rows + i];
  }
  std::vector<C<L>> Rm((size_t)cols * W, czero<L>());
  for (int q = 0; q < cols; ++q) {
    R<L> nrm2 = rzero<L>();
    for (int i = 0; i < rows; ++i) nrm2 = radd<L>(nrm2, cabs2<L>(M[(size_t)i * W + q]));
    R<L> rqq = rsqrt<L>(nrm2);
    Rm[(size_t)q * W + q] = C<L>{rqq, rzero<L>()};
    for (int i = 0; i < rows; ++i) {
      C<L>& e = M[(size_t)i * W + q];
      e = C<L>{rdiv<L>(e.re, rqq), rdiv<L>(e.im, rqq)};
    }
    for (int j = q + 1; j < W; ++j) {
      C<L> r = czero<L>();
      for (int i = 0; i < rows; ++i) r = cadd<L>(r, cconjmul<L>(M[(size_t)i * W + q], M[(size_t)i * W + j]));
      Rm[(size_t)q * W + j] = r;
      for (int i = 0; i < rows; ++i)
        M[(size_t)i * W + j] = csub<L>(M[(size_t)i * W + j], cmul<L>(r, M[(size_t)i * W + q]));
    }
  }
  for (int k = 0; k < nrhs; ++k) {
    C<L>* xk = x + (size_t)k * cols;
    for (int q = cols - 1; q >= 0; --q) {
      C<L> acc = Rm[(size_t)q * W + cols + k];
      for (int j = q + 1; j < cols; ++j) acc = csub<L>(acc, cmul<L>(Rm[(size_t)q * W + j], xk[j]));
      R<L> rqq = Rm[(size_t)q * W + q].re;
      xk[q] = C<L>{rdiv<L>(acc.re, rqq), rdiv<L>(acc.im, rqq)};
    }
  }
}
template <int L>
void mgs_solve(int rows, int cols, std::vector<C<L>>& A, std::vector<C<L>>& b, C<L>* x) {
  mgs_solve_multi<L>(rows, cols, 1, A, b.data(), x);
}

// ---------------------------------------------------------- start solutions
// Path p <-> mixed-radix digits k_i (digit of variable 0 varies fastest);
// x_i = exp(2 pi i k_i / d_i), a root of x_i^d_i - 1.  d = 1, 2, 4 give exact
// values; otherwise the double cos/sin value is refined by Newton's method on
// z^d - 1 in L-limb precision.
template <int L>
C<L> cpow_int(const C<L>& z, int e) {
  C<L> r{rfrom<L>(1.0), rzero<L>()};
  for (int i = 0; i < e; ++i) r = cmul<L>(r, z);
  return r;
}
template <int L>
C<L> cdiv(const C<L>& a, const C<L>& b) {
  R<L> den = cabs2<L>(b);
  C<L> num = cconjmul<L>(b, a);  // conj(b) a
  return C<L>{rdiv<L>(num.re, den), rdiv<L>(num.im, den)};
}
template <int L>
C<L> root_of_unity(int d, int k) {
  if (d == 1) return C<L>{rfrom<L>(1.0), rzero<L>()};
  if (2 * k == d) return C<L>{rfrom<L>(-1.0), rzero<L>()};
  if (k == 0) return C<L>{rfrom<L>(1.0), rzero<L>()};
  if (4 * k == d) return C<L>{rzero<L>(), rfrom<L>(1.0)};
  if (4 * k == 3 * d) return C<L>{rzero<L>(), rfrom<L>(-1.0)};
  const double pi = 3.14159265358979323846;
  double th = 2.0 * pi * (double)k / (double)d;
  C<L> z{rfrom<L>(std::cos(th)), rfrom<L>(std::sin(th))};
  if (L > 1) {
    for (int it = 0; it < 3; ++it) {
      C<L> zd1 = cpow_int<L>(z, d - 1);
      C<L> f = csub<L>(cmul<L>(zd1, z), C<L>{rfrom<L>(1.0), rzero<L>()});
      C<L> fp = cscale<L>(zd1, rfrom<L>((double)d));
      z = csub<L>(z, cdiv<L>(f, fp));
    }
  }
  return z;
}
template <int L>
void start_solution(int n, const int32_t* deg, int64_t path, C<L>* x) {
  int64_t r = path;
  for (int i = 0; i < n; ++i) {
    int k = (int)(r % deg[i]);
    r /= deg[i];
    x[i] = root_of_unity<L>(deg[i], k);
  }
}

// ---------------------------------------------------------- tracker
// Parameters, in this order, as doubles (Section 2 leaves all of them open):
enum {
  P_H0, P_HMIN, P_HMAX, P_FUP, P_FDOWN, P_NEWTON_MAX, P_TOL_DX, P_TOL_RES,
  P_POLISH_MAX, P_TOL_POLISH, P_RDIV, P_MAX_STEPS, P_MAX_ORDER, P_PREDICTOR, P_COUNT
};

template <int L>
struct Homotopy {
  Sys<L> f;
  std::vector<int32_t> d;  // start system g_i = x_i^d_i - 1
  C<L> gamma;
  int deg_max;
};

// h(x, t) = gamma (1 - t) g(x) + t f(x)  (Eq. eqlinhom), its Jacobian in x,
// and (ht != nullptr) its derivative in t, f(x) - gamma g(x).
template <int L>
void eval_homotopy(const Homotopy<L>& H, const C<L>* x, double t, C<L>* h, C<L>* J, C<L>* ht = nullptr) {
  const int n = H.f.nv;
  std::vector<C<L>> fv(n), fj((size_t)n * n);
  eval_speel<L>(H.f, x, fv.data(), fj.data());
  R<L> tt = rfrom<L>(t);
  R<L> omt = rsub<L>(rfrom<L>(1.0), tt);
  C<L> gs = cscale<L>(H.gamma, omt);  // gamma (1 - t)
  for (int i = 0; i < n; ++i) {
    C<L> xd1 = cpow_int<L>(x[i], H.d[i] - 1);
    C<L> g = csub<L>(cmul<L>(xd1, x[i]), C<L>{rfrom<L>(1.0), rzero<L>()});
    C<L> dg = cscale<L>(xd1, rfrom<L>((double)H.d[i]));
    h[i] = cadd<L>(cmul<L>(gs, g), cscale<L>(fv[i], tt));
    if (ht) ht[i] = csub<L>(fv[i], cmul<L>(H.gamma, g));
    for (int j = 0; j < n; ++j) {
      C<L> v = cscale<L>(fj[(size_t)i * n + j], tt);
      if (j == i) v = cadd<L>(v, cmul<L>(gs, dg));
      J[(size_t)i * n + j] = v;
    }
  }
}

template <int L>
double norm_inf(const C<L>* v, int n) {
  double m = 0;
  for (int i = 0; i < n; ++i) m = std::max(m, cabs_d<L>(v[i]));
  return m;
}
template <int L>
bool all_finite(const C<L>* v, int n) {
  for (int i = 0; i < n; ++i)
    if (!cfinite<L>(v[i])) return false;
  return true;
}

// One Newton step at (x, t): x <- x + dx with J dx = -h by least squares.
// Returns |dx|_inf and |h|_inf (at x before the update).  With tan !=
// nullptr the same factorisation also solves J v = -dh/dt, the tangent of the
// path (Section 2's predictor stage): v is written to tan.
template <int L>
void newton_step(const Homotopy<L>& H, std::vector<C<L>>& x, double t, double* ndx, double* nres,
                 std::vector<C<L>>* tan = nullptr) {
  const int n = H.f.nv;
  const int nrhs = tan ? 2 : 1;
  std::vector<C<L>> h(n), J((size_t)n * n), rhs((size_t)nrhs * n), sol((size_t)nrhs * n), dht(n);
  eval_homotopy<L>(H, x.data(), t, h.data(), J.data(), tan ? dht.data() : nullptr);
  for (int i = 0; i < n; ++i) rhs[i] = C<L>{rneg<L>(h[i].re), rneg<L>(h[i].im)};
  if (tan)
    for (int i = 0; i < n; ++i) rhs[n + i] = C<L>{rneg<L>(dht[i].re), rneg<L>(dht[i].im)};
  mgs_solve_multi<L>(n, n, nrhs, J, rhs.data(), sol.data());
  std::vector<C<L>> dx(sol.begin(), sol.begin() + n);
  if (tan) tan->assign(sol.begin() + n, sol.end());
  for (int i = 0; i < n; ++i) x[i] = cadd<L>(x[i], dx[i]);
  *ndx = norm_inf<L>(dx.data(), n);
  *nres = norm_inf<L>(h.data(), n);
  if (!all_finite<L>(dx.data(), n)) *ndx = NAN;
}

// Extrapolation through the accepted points (t_j, x_j), j = 0..m-1, to t1, in
// Lagrange form: x(t1) = sum_j x_j prod_{i != j} (t1 - t_i) / (t_j - t_i).
template <int L>
void predict(const std::vector<double>& ht, const std::vector<std::vector<C<L>>>& hx, int m, double t1,
             std::vector<C<L>>& out) {
  const int n = (int)out.size();
  const int base = (int)ht.size() - m;
  std::vector<R<L>> w(m);
  for (int j = 0; j < m; ++j) {
    R<L> num = rfrom<L>(1.0), den = rfrom<L>(1.0);
    for (int i = 0; i < m; ++i) {
      if (i == j) continue;
      num = rmul<L>(num, rsub<L>(rfrom<L>(t1), rfrom<L>(ht[base + i])));
      den = rmul<L>(den, rsub<L>(rfrom<L>(ht[base + j]), rfrom<L>(ht[base + i])));
    }
    w[j] = rdiv<L>(num, den);
  }
  for (int c = 0; c < n; ++c) {
    C<L> acc = czero<L>();
    for (int j = 0; j < m; ++j) acc = cadd<L>(acc, cscale<L>(hx[base + j][c], w[j]));
    out[c] = acc;
  }
}

// Predictors from tangents (Section 2's predictor stage, with the tangent
// v = dx/dt of the path from J v = -dh/dt):
//   Euler    x(t1) = x1 + (t1 - s1) v1 through the current point (s1, x1, v1);
//   Hermite  the cubic that matches (s0, x0, v0) and (s1, x1, v1), evaluated
//            at t1: with d = s1 - s0 and u = (t1 - s0) / d,
//            x(t1) = (2u^3 - 3u^2 + 1) x0 + (u^3 - 2u^2 + u) d v0
//                  + (-2u^3 + 3u^2) x1 + (u^3 - u^2) d v1.
template <int L>
void predict_euler(double s1, const std::vector<C<L>>& x1, const std::vector<C<L>>& v1, double t1,
                   std::vector<C<L>>& out) {
  R<L> dt = rsub<L>(rfrom<L>(t1), rfrom<L>(s1));
  for (size_t c = 0; c < out.size(); ++c) out[c] = cadd<L>(x1[c], cscale<L>(v1[c], dt));
}
template <int L>
void predict_hermite(double s0, const std::vector<C<L>>& x0, const std::vector<C<L>>& v0, double s1,
                     const std::vector<C<L>>& x1, const std::vector<C<L>>& v1, double t1, std::vector<C<L>>& out) {
  const R<L> d = rsub<L>(rfrom<L>(s1), rfrom<L>(s0));
  const R<L> u = rdiv<L>(rsub<L>(rfrom<L>(t1), rfrom<L>(s0)), d);
  const R<L> u2 = rmul<L>(u, u), u3 = rmul<L>(u2, u);
  const R<L> one = rfrom<L>(1.0), two = rfrom<L>(2.0), three = rfrom<L>(3.0);
  const R<L> a0 = radd<L>(rsub<L>(rmul<L>(two, u3), rmul<L>(three, u2)), one);
  const R<L> b0 = rmul<L>(radd<L>(rsub<L>(u3, rmul<L>(two, u2)), u), d);
  const R<L> a1 = rsub<L>(rmul<L>(three, u2), rmul<L>(two, u3));
  const R<L> b1 = rmul<L>(rsub<L>(u3, u2), d);
  for (size_t c = 0; c < out.size(); ++c) {
    C<L> acc = cscale<L>(x0[c], a0);
    acc = cadd<L>(acc, cscale<L>(v0[c], b0));
    acc = cadd<L>(acc, cscale<L>(x1[c], a1));
    acc = cadd<L>(acc, cscale<L>(v1[c], b1));
    out[c] = acc;
  }
}

struct PathResult {
  int8_t status;
  double t;
  int32_t steps, rejects, newton;
};

// Status codes: 0 continue, 1 success, -1 failure (Section 2), -2 diverged
// (a failure whose cause is |x| > r_div).
template <int L>
PathResult track_one(const Homotopy<L>& H, const double* P, std::vector<C<L>>& x) {
  const int n = H.f.nv;
  const double h0 = P[P_H0], hmin = P[P_HMIN], hmax = P[P_HMAX], fup = P[P_FUP], fdown = P[P_FDOWN];
  const int newton_max = (int)P[P_NEWTON_MAX], polish_max = (int)P[P_POLISH_MAX];
  const int max_steps = (int)P[P_MAX_STEPS], max_order = (int)P[P_MAX_ORDER];
  const double tol_dx = P[P_TOL_DX], tol_res = P[P_TOL_RES], tol_polish = P[P_TOL_POLISH];
  const double rdiv_ = P[P_RDIV];
  // predictor: 0 extrapolation through up to max_order + 1 accepted points;
  // 1 Euler on the tangent of the current point; 2 cubic Hermite on the
  // current and the previous point and their tangents.  The start point has
  // no tangent: until one exists the extrapolation predictor of order 0
  // (Euler: also until then; Hermite: Euler with one tangent).
  const int pmode = (int)P[P_PREDICTOR];

  std::vector<double> ht{0.0};
  std::vector<std::vector<C<L>>> hx{x};
  std::vector<std::vector<C<L>>> hv{std::vector<C<L>>()};  // tangents (empty: none)
  double t = 0.0, h = h0;
  PathResult res{0, 0.0, 0, 0, 0};
  std::vector<C<L>> xp(n), tan_last;
  while (res.status == 0) {
    double step = std::min(h, 1.0 - t);
    double t1 = (step >= 1.0 - t) ? 1.0 : t + step;
    const size_t nh = ht.size();
    const bool v1 = !hv[nh - 1].empty(), v0 = nh >= 2 && !hv[nh - 2].empty();
    if (pmode == 2 && v1 && v0) {
      predict_hermite<L>(ht[nh - 2], hx[nh - 2], hv[nh - 2], ht[nh - 1], hx[nh - 1], hv[nh - 1], t1, xp);
    } else if (pmode >= 1 && v1) {
      predict_euler<L>(ht[nh - 1], hx[nh - 1], hv[nh - 1], t1, xp);
    } else {
      int m = std::min<int>((int)ht.size(), pmode >= 1 ? 1 : max_order + 1);
      predict<L>(ht, hx, m, t1, xp);
    }
    bool ok = false;
    for (int it = 0; it < newton_max; ++it) {
      double ndx, nres;
      newton_step<L>(H, xp, t1, &ndx, &nres, pmode >= 1 ? &tan_last : nullptr);
      ++res.newton;
      if (!(ndx == ndx)) break;  // NaN: reject
      double sx = std::max(1.0, norm_inf<L>(xp.data(), n));
      double lim = tol_res;  // tol_res * sx^deg_max
      for (int e = 0; e < H.deg_max; ++e) lim *= sx;
      if (ndx <= tol_dx * sx && nres <= lim) {
        ok = true;
        break;
      }
    }
    ++res.steps;
    if (ok) {
      t = t1;
      x = xp;
      ht.push_back(t);
      hx.push_back(x);
      hv.push_back(pmode >= 1 ? tan_last : std::vector<C<L>>());
      if ((int)ht.size() > max_order + 1) {
        ht.erase(ht.begin());
        hx.erase(hx.begin());
        hv.erase(hv.begin());
      }
      h = std::min(hmax, fup * h);
      if (norm_inf<L>(x.data(), n) > rdiv_) {
        res.status = -2;
      } else if (t == 1.0) {
        for (int it = 0; it < polish_max; ++it) {
          double ndx, nres;
          std::vector<C<L>> xs = x;
          newton_step<L>(H, xs, 1.0, &ndx, &nres);
          ++res.newton;
          if (!(ndx == ndx)) break;
          x = xs;
          if (ndx <= tol_polish * std::max(1.0, norm_inf<L>(x.data(), n))) break;
        }
        res.status = all_finite<L>(x.data(), n) ? 1 : -1;
      }
    } else {
      ++res.rejects;
      h = fdown * h;
      if (h < hmin) res.status = -1;
    }
    if (res.status == 0 && res.steps >= max_steps) res.status = -1;
  }
  res.t = t;
  return res;
}


// ---------------------------------------------------------- learned step MLP
// Three dense layers 16 -> 64 -> 64 -> 2 with ReLU between them, fp64.
// Parameters flat: W1[64][16] b1[64] W2[64][64] b2[64] W3[2][64] b3[2].
constexpr int MI = 16, MH = 64, MO = 2;
constexpr int MLP_NPARAM = MH * MI + MH + MH * MH + MH + MO * MH + MO;

struct MlpView {
  const double *W1, *b1, *W2, *b2, *W3, *b3;
  explicit MlpView(const double* p)
      : W1(p), b1(p + MH * MI), W2(b1 + MH), b2(W2 + MH * MH), W3(b2 + MH), b3(W3 + MO * MH) {}
};

void mlp_forward_one(const MlpView& w, const double* x, double* z1, double* h1, double* z2, double* h2, double* y) {
  for (int o = 0; o < MH; ++o) {
    double a = w.b1[o];
    for (int i = 0; i < MI; ++i) a += w.W1[o * MI + i] * x[i];
    z1[o] = a;
    h1[o] = a > 0 ? a : 0;
  }
  for (int o = 0; o < MH; ++o) {
    double a = w.b2[o];
    for (int i = 0; i < MH; ++i) a += w.W2[o * MH + i] * h1[i];
    z2[o] = a;
    h2[o] = a > 0 ? a : 0;
  }
  for (int o = 0; o < MO; ++o) {
    double a = w.b3[o];
    for (int i = 0; i < MH; ++i) a += w.W3[o * MH + i] * h2[i];
    y[o] = a;
  }
}

template <typename F>
void parallel_for(int64_t n, int n_threads, F f) {
  if (n_threads <= 0) n_threads = (int)std::max(1u, std::thread::hardware_concurrency());
  if (n_threads == 1 || n <= 1) {
    for (int64_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<int64_t> next(0);
  std::vector<std::thread> th;
  for (int w = 0; w < n_threads; ++w)
    th.emplace_back([&]() {
      for (;;) {
        int64_t i = next.fetch_add(1);
        if (i >= n) break;
        f(i);
      }
    });
  for (auto& x : th) x.join();
}

// ----------------------------------------------------------- typed drivers
template <int L>
int eval_points(int method, int nv, int np, const int32_t* n_terms, const int8_t* exps, const double* coef,
                int64_t n_pts, const int64_t* pts, int64_t n_sel, const double* x, double* val, double* jac,
                int n_threads) {
  Sys<L> s = make_sys<L>(nv, np, n_terms, exps, coef);
  parallel_for(n_sel, n_threads, [&](int64_t q) {
    int64_t p = pts ? pts[q] : q;
    std::vector<C<L>> xv(nv), v(np), J((size_t)np * nv);
    for (int i = 0; i < nv; ++i) xv[i] = load_soa<L>(x, i, p, n_pts);
    if (method == 0)
      eval_naive<L>(s, xv.data(), v.data(), J.data());
    else
      eval_speel<L>(s, xv.data(), v.data(), J.data());
    for (int j = 0; j < np; ++j) store_soa<L>(val, j, q, n_sel, v[j]);
    for (int j = 0; j < np; ++j)
      for (int i = 0; i < nv; ++i) store_soa<L>(jac, (int64_t)j * nv + i, q, n_sel, J[(size_t)j * nv + i]);
  });
  return 0;
}

template <int L>
int magnitude_points(int nv, int np, const int32_t* n_terms, const int8_t* exps, const double* coef,
                     int64_t n_pts, const int64_t* pts, int64_t n_sel, const double* x, double* val,
                     double* jac) {
  Sys<L> s = make_sys<L>(nv, np, n_terms, exps, coef);
  std::vector<C<L>> xv(nv);
  std::vector<double> v(np), J((size_t)np * nv);
  for (int64_t q = 0; q < n_sel; ++q) {
    int64_t p = pts ? pts[q] : q;
    for (int i = 0; i < nv; ++i) xv[i] = load_soa<L>(x, i, p, n_pts);
    eval_magnitude<L>(s, xv.data(), v.data(), J.data());
    for (int j = 0; j < np; ++j) val[(size_t)j * n_sel + q] = v[j];
    for (size_t e = 0; e < J.size(); ++e) jac[e * n_sel + q] = J[e];
  }
  return 0;
}

template <int L>
int mgs_batch(int rows, int cols, int64_t n_sys, const double* A, const double* b, double* x) {
  for (int64_t s = 0; s < n_sys; ++s) {
    std::vector<C<L>> Am((size_t)rows * cols), bm(rows), xm(cols);
    // A: [n_sys][rows][cols][2][L], b: [n_sys][rows][2][L], x: [n_sys][cols][2][L]
    for (int i = 0; i < rows * cols; ++i)
      for (int l = 0; l < L; ++l) {
        Am[i].re.v[l] = A[(((size_t)s * rows * cols + i) * 2 + 0) * L + l];
        Am[i].im.v[l] = A[(((size_t)s * rows * cols + i) * 2 + 1) * L + l];
      }
    for (int i = 0; i < rows; ++i)
      for (int l = 0; l < L; ++l) {
        bm[i].re.v[l] = b[(((size_t)s * rows + i) * 2 + 0) * L + l];
        bm[i].im.v[l] = b[(((size_t)s * rows + i) * 2 + 1) * L + l];
      }
    mgs_solve<L>(rows, cols, Am, bm, xm.data());
    for (int i = 0; i < cols; ++i)
      for (int l = 0; l < L; ++l) {
        x[(((size_t)s * cols + i) * 2 + 0) * L + l] = xm[i].re.v[l];
        x[(((size_t)s * cols + i) * 2 + 1) * L + l] = xm[i].im.v[l];
      }
  }
  return 0;
}

template <int L>
int start_batch(int n, const int32_t* deg, int64_t first, int64_t count, double* x) {
  std::vector<C<L>> xv(n);
  for (int64_t p = 0; p < count; ++p) {
    start_solution<L>(n, deg, first + p, xv.data());
    for (int i = 0; i < n; ++i) store_soa<L>(x, i, p, count, xv[i]);
  }
  return 0;
}

template <int L>
int track_batch(int n, const int32_t* n_terms, const int8_t* exps, const double* coef, const int32_t* start_deg,
                const double* gamma, int64_t n_paths, const int64_t* path_ids, const double* params,
                int n_threads, double* x_end, int8_t* status, double* t_end, int32_t* steps, int32_t* rejects,
                int32_t* newton) {
  Homotopy<L> H;
  H.f = make_sys<L>(n, n, n_terms, exps, coef);
  H.d.assign(start_deg, start_deg + n);
  H.gamma = C<L>{rfrom<L>(gamma[0]), rfrom<L>(gamma[1])};
  H.deg_max = H.f.max_deg;
  for (int i = 0; i < n; ++i) H.deg_max = std::max<int>(H.deg_max, start_deg[i]);
  parallel_for(n_paths, n_threads, [&](int64_t q) {
    std::vector<C<L>> x(n);
    start_solution<L>(n, start_deg, path_ids[q], x.data());
    PathResult r = track_one<L>(H, params, x);
    for (int i = 0; i < n; ++i) store_soa<L>(x_end, i, q, n_paths, x[i]);
    status[q] = r.status;
    t_end[q] = r.t;
    steps[q] = r.steps;
    rejects[q] = r.rejects;
    newton[q] = r.newton;
  });
  return 0;
}

// The predictor alone: m points (ts [m], xs [m][n][2][L]) extrapolated to t1
// (out [n][2][L]).
template <int L>
int predict_one(int n, int m, const double* ts, const double* xs, double t1, double* out) {
  std::vector<double> ht(ts, ts + m);
  std::vector<std::vector<C<L>>> hx(m, std::vector<C<L>>(n));
  for (int j = 0; j < m; ++j)
    for (int i = 0; i < n; ++i)
      for (int l = 0; l < L; ++l) {
        hx[j][i].re.v[l] = xs[(((size_t)j * n + i) * 2 + 0) * L + l];
        hx[j][i].im.v[l] = xs[(((size_t)j * n + i) * 2 + 1) * L + l];
      }
  std::vector<C<L>> o(n);
  predict<L>(ht, hx, m, t1, o);
  for (int i = 0; i < n; ++i)
    for (int l = 0; l < L; ++l) {
      out[(i * 2 + 0) * L + l] = o[i].re.v[l];
      out[(i * 2 + 1) * L + l] = o[i].im.v[l];
    }
  return 0;
}

// The homotopy alone: h(x, t) [n][2][L][n_pts] and its Jacobian in x
// [n][n][2][L][n_pts] at the points x [n][2][L][n_pts].
template <int L>
int homotopy_points(int n, const int32_t* n_terms, const int8_t* exps, const double* coef, const int32_t* start_deg,
                    const double* gamma, double t, int64_t n_pts, const double* x, double* h, double* J) {
  Homotopy<L> H;
  H.f = make_sys<L>(n, n, n_terms, exps, coef);
  H.d.assign(start_deg, start_deg + n);
  H.gamma = C<L>{rfrom<L>(gamma[0]), rfrom<L>(gamma[1])};
  H.deg_max = H.f.max_deg;
  std::vector<C<L>> xv(n), hv(n), Jv((size_t)n * n);
  for (int64_t p = 0; p < n_pts; ++p) {
    for (int i = 0; i < n; ++i) xv[i] = load_soa<L>(x, i, p, n_pts);
    eval_homotopy<L>(H, xv.data(), t, hv.data(), Jv.data());
    for (int i = 0; i < n; ++i) store_soa<L>(h, i, p, n_pts, hv[i]);
    for (size_t e = 0; e < Jv.size(); ++e) store_soa<L>(J, (int64_t)e, p, n_pts, Jv[e]);
  }
  return 0;
}

// The path tangent at points x [n][2][L][n_pts] and time t: v solves
// J_x v = -dh/dt by the least squares of the Newton step (out [n][2][L][n_pts]).
template <int L>
int tangent_points(int n, const int32_t* n_terms, const int8_t* exps, const double* coef, const int32_t* start_deg,
                   const double* gamma, double t, int64_t n_pts, const double* x, double* v) {
  Homotopy<L> H;
  H.f = make_sys<L>(n, n, n_terms, exps, coef);
  H.d.assign(start_deg, start_deg + n);
  H.gamma = C<L>{rfrom<L>(gamma[0]), rfrom<L>(gamma[1])};
  H.deg_max = H.f.max_deg;
  std::vector<C<L>> xv(n), tv;
  for (int64_t p = 0; p < n_pts; ++p) {
    for (int i = 0; i < n; ++i) xv[i] = load_soa<L>(x, i, p, n_pts);
    double ndx, nres;
    newton_step<L>(H, xv, t, &ndx, &nres, &tv);
    for (int i = 0; i < n; ++i) store_soa<L>(v, i, p, n_pts, tv[i]);
  }
  return 0;
}

// The tangent predictors alone: mode 1 Euler from (s1, x1, v1), mode 2 cubic
// Hermite from (s0, x0, v0) and (s1, x1, v1); points [n][2][L].
template <int L>
int predict_tangent_one(int n, int mode, double s0, const double* x0, const double* v0, double s1, const double* x1,
                        const double* v1, double t1, double* out) {
  auto load = [&](const double* a) {
    std::vector<C<L>> z(n);
    for (int i = 0; i < n; ++i)
      for (int l = 0; l < L; ++l) {
        z[i].re.v[l] = a[(i * 2 + 0) * L + l];
        z[i].im.v[l] = a[(i * 2 + 1) * L + l];
      }
    return z;
  };
  std::vector<C<L>> o(n);
  if (mode == 1)
    predict_euler<L>(s1, load(x1), load(v1), t1, o);
  else
    predict_hermite<L>(s0, load(x0), load(v0), s1, load(x1), load(v1), t1, o);
  for (int i = 0; i < n; ++i)
    for (int l = 0; l < L; ++l) {
      out[(i * 2 + 0) * L + l] = o[i].re.v[l];
      out[(i * 2 + 1) * L + l] = o[i].im.v[l];
    }
  return 0;
}

}  // namespace

template <template <int> class F, typename... A>
int dispatch_l(int L, A... args) {
  switch (L) {
    case 1: return F<1>::run(args...);
    case 2: return F<2>::run(args...);
    case 4: return F<4>::run(args...);
    default: return -1;
  }
}
template <int L> struct EvalF { template <typename... A> static int run(A... a) { return eval_points<L>(a...); } };
template <int L> struct MagF { template <typename... A> static int run(A... a) { return magnitude_points<L>(a...); } };
template <int L> struct MgsF { template <typename... A> static int run(A... a) { return mgs_batch<L>(a...); } };
template <int L> struct StartF { template <typename... A> static int run(A... a) { return start_batch<L>(a...); } };
template <int L> struct TrackF { template <typename... A> static int run(A... a) { return track_batch<L>(a...); } };
template <int L> struct PredF { template <typename... A> static int run(A... a) { return predict_one<L>(a...); } };
template <int L> struct HomF { template <typename... A> static int run(A... a) { return homotopy_points<L>(a...); } };
template <int L> struct TanF { template <typename... A> static int run(A... a) { return tangent_points<L>(a...); } };
template <int L> struct PTanF { template <typename... A> static int run(A... a) { return predict_tangent_one<L>(a...); } };
template <int L>
struct SlotsF {
  static int run(int k, const double* x, double* slots) {
    std::vector<C<L>> xs(k), sl(2 * k), d(k);
    C<L> v;
    for (int i = 0; i < k; ++i)
      for (int l = 0; l < L; ++l) {
        xs[i].re.v[l] = x[(i * 2 + 0) * L + l];
        xs[i].im.v[l] = x[(i * 2 + 1) * L + l];
      }
    for (auto& e : sl) e = czero<L>();
    int nmul = speelpenning<L>(k, xs.data(), sl.data(), &v, d.data());
    for (int i = 0; i < 2 * k; ++i)
      for (int l = 0; l < L; ++l) {
        slots[(i * 2 + 0) * L + l] = sl[i].re.v[l];
        slots[(i * 2 + 1) * L + l] = sl[i].im.v[l];
      }
    return nmul;
  }
};

extern "C" {

int hto_version(void) { return 1; }
int hto_param_count(void) { return P_COUNT; }

// Element-wise real arithmetic on L-limb numbers, for pinning the arithmetic:
// op 0 add, 1 sub, 2 mul, 3 div, 4 sqrt (b unused).  Arrays are [n][L].
int hto_real_op(int op, int L, int64_t n, const double* a, const double* b, double* out) {
  auto run = [&](auto tag) -> int {
    constexpr int LL = decltype(tag)::value;
    for (int64_t i = 0; i < n; ++i) {
      R<LL> x, y, z;
      for (int l = 0; l < LL; ++l) {
        x.v[l] = a[i * LL + l];
        y.v[l] = b ? b[i * LL + l] : 0.0;
      }
      switch (op) {
        case 0: z = radd<LL>(x, y); break;
        case 1: z = rsub<LL>(x, y); break;
        case 2: z = rmul<LL>(x, y); break;
        case 3: z = rdiv<LL>(x, y); break;
        case 4: z = rsqrt<LL>(x); break;
        default: return -1;
      }
      for (int l = 0; l < LL; ++l) out[i * LL + l] = z.v[l];
    }
    return 0;
  };
  switch (L) {
    case 1: return run(std::integral_constant<int, 1>());
    case 2: return run(std::integral_constant<int, 2>());
    case 4: return run(std::integral_constant<int, 4>());
    default: return -1;
  }
}

// out[i] = (sum of a's limbs - sum of b's limbs), the exact difference of two
// L-limb values rounded once to double.  Arrays are [n][L].
int hto_value_diff(int L, int64_t n, const double* a, const double* b, double* out) {
  for (int64_t i = 0; i < n; ++i) {
    Acc s;
    for (int l = 0; l < L; ++l) {
      s.add(a[i * L + l]);
      s.add(-b[i * L + l]);
    }
    out[i] = s.round();
  }
  return 0;
}

// Evaluate and differentiate a system at selected points.
// method 0: textbook product rule; 1: reverse mode (Table tabmoneval).
// coef: [M][2][L]; x: [nv][2][L][n_pts]; pts: the n_sel point indices to
// evaluate (NULL: 0..n_sel-1); val: [np][2][L][n_sel]; jac: [np][nv][2][L][n_sel].
int hto_eval(int method, int L, int nv, int np, const int32_t* n_terms, const int8_t* exps, const double* coef,
             int64_t n_pts, const int64_t* pts, int64_t n_sel, const double* x, double* val, double* jac,
             int n_threads) {
  return dispatch_l<EvalF>(L, method, nv, np, n_terms, exps, coef, n_pts, pts, n_sel, x, val, jac, n_threads);
}

// Sum over the terms of each output of the modulus of the term, in double:
// val: [np][n_sel]; jac: [np][nv][n_sel].
int hto_eval_magnitude(int L, int nv, int np, const int32_t* n_terms, const int8_t* exps, const double* coef,
                       int64_t n_pts, const int64_t* pts, int64_t n_sel, const double* x, double* val,
                       double* jac) {
  return dispatch_l<MagF>(L, nv, np, n_terms, exps, coef, n_pts, pts, n_sel, x, val, jac);
}

// The slots of Table tabmoneval for one product of k variables; x: [k][2][L],
// slots: [2k][2][L].  Returns the number of multiplications.
int hto_speelpenning_slots(int L, int k, const double* x, double* slots) {
  return dispatch_l<SlotsF>(L, k, x, slots);
}

// Least squares by modified Gram-Schmidt for n_sys independent systems:
// A: [n_sys][rows][cols][2][L], b: [n_sys][rows][2][L], x: [n_sys][cols][2][L].
int hto_mgs_solve(int L, int rows, int cols, int64_t n_sys, const double* A, const double* b, double* x) {
  return dispatch_l<MgsF>(L, rows, cols, n_sys, A, b, x);
}

// The tracker's extrapolation predictor (Section 2) through m points:
// ts [m], xs [m][n][2][L] -> out [n][2][L], the extrapolated point at t1.
int hto_predict(int L, int n, int m, const double* ts, const double* xs, double t1, double* out) {
  if (n < 1 || m < 1) return -1;
  return dispatch_l<PredF>(L, n, m, ts, xs, t1, out);
}

// The homotopy gamma (1 - t) g(x) + t f(x) of Eq. eqlinhom, g_i = x_i^d_i - 1,
// and its Jacobian in x at the points x [n][2][L][n_pts]:
// h [n][2][L][n_pts], J [n][n][2][L][n_pts].
int hto_homotopy(int L, int n, const int32_t* n_terms, const int8_t* exps, const double* coef,
                 const int32_t* start_deg, const double* gamma, double t, int64_t n_pts, const double* x, double* h,
                 double* J) {
  return dispatch_l<HomF>(L, n, n_terms, exps, coef, start_deg, gamma, t, n_pts, x, h, J);
}

// The path tangent v = dx/dt of Eq. eqlinhom at points x [n][2][L][n_pts] and
// time t, from J_x v = -dh/dt (v [n][2][L][n_pts]).
int hto_tangent(int L, int n, const int32_t* n_terms, const int8_t* exps, const double* coef,
                const int32_t* start_deg, const double* gamma, double t, int64_t n_pts, const double* x, double* v) {
  return dispatch_l<TanF>(L, n, n_terms, exps, coef, start_deg, gamma, t, n_pts, x, v);
}

// The tracker's tangent predictors: mode 1 Euler, 2 cubic Hermite (points
// [n][2][L]; mode 1 reads only s1, x1, v1).
int hto_predict_tangent(int L, int n, int mode, double s0, const double* x0, const double* v0, double s1,
                        const double* x1, const double* v1, double t1, double* out) {
  if (n < 1 || (mode != 1 && mode != 2)) return -1;
  return dispatch_l<PTanF>(L, n, mode, s0, x0, v0, s1, x1, v1, t1, out);
}

// Start solutions of x_i^d_i - 1 = 0 for paths first..first+count-1:
// x: [n][2][L][count].
int hto_start_solutions(int L, int n, const int32_t* deg, int64_t first, int64_t count, double* x) {
  return dispatch_l<StartF>(L, n, deg, first, count, x);
}

// Table tabjobidx: inclusive scan of (status == 0); path_idx receives the
// indices of the paths that continue, in increasing order; returns their count.
int64_t hto_compact(const int8_t* status, int64_t m, int64_t* scan, int32_t* path_idx) {
  int64_t c = 0;
  for (int64_t i = 0; i < m; ++i) {
    if (status[i] == 0) path_idx[c++] = (int32_t)i;
    if (scan) scan[i] = c;
  }
  return c;
}

// Track the paths path_ids[0..n_paths-1] of gamma (1 - t) g(x) + t f(x) = 0,
// g_i = x_i^d_i - 1, from t = 0 to t = 1.  gamma: [2] (double re, im);
// params: hto_param_count() doubles; outputs x_end: [n][2][L][n_paths],
// status, t_end, steps, rejects, newton: [n_paths].
int hto_track(int L, int n, const int32_t* n_terms, const int8_t* exps, const double* coef,
              const int32_t* start_deg, const double* gamma, int64_t n_paths, const int64_t* path_ids,
              const double* params, int n_threads, double* x_end, int8_t* status, double* t_end, int32_t* steps,
              int32_t* rejects, int32_t* newton) {
  return dispatch_l<TrackF>(L, n, n_terms, exps, coef, start_deg, gamma, n_paths, path_ids, params, n_threads,
                            x_end, status, t_end, steps, rejects, newton);
}


int hto_mlp_nparam(void) { return MLP_NPARAM; }

// y[b][2] = MLP(x[b][16]) for b < B.
int hto_mlp_forward(int64_t B, const double* x, const double* params, double* y) {
  MlpView w(params);
  double z1[MH], h1[MH], z2[MH], h2[MH];
  for (int64_t b = 0; b < B; ++b) mlp_forward_one(w, x + b * MI, z1, h1, z2, h2, y + b * MO);
  return 0;
}

// Mean squared error L = (1/B) sum_b sum_o (y_bo - t_bo)^2 and its gradient
// with respect to every parameter (reverse mode through the three layers).
double hto_mlp_loss_grad(int64_t B, const double* x, const double* target, const double* params, double* grad) {
  MlpView w(params);
  std::memset(grad, 0, sizeof(double) * MLP_NPARAM);
  double *gW1 = grad, *gb1 = gW1 + MH * MI, *gW2 = gb1 + MH, *gb2 = gW2 + MH * MH, *gW3 = gb2 + MH,
         *gb3 = gW3 + MO * MH;
  double loss = 0;
  double z1[MH], h1[MH], z2[MH], h2[MH], y[MO], dy[MO], dh2[MH], dz2[MH], dh1[MH], dz1[MH];
  for (int64_t b = 0; b < B; ++b) {
    const double* xb = x + b * MI;
    mlp_forward_one(w, xb, z1, h1, z2, h2, y);
    for (int o = 0; o < MO; ++o) {
      double e = y[o] - target[b * MO + o];
      loss += e * e;
      dy[o] = 2.0 * e / (double)B;
    }
    for (int i = 0; i < MH; ++i) dh2[i] = 0;
    for (int o = 0; o < MO; ++o) {
      gb3[o] += dy[o];
      for (int i = 0; i < MH; ++i) {
        gW3[o * MH + i] += dy[o] * h2[i];
        dh2[i] += dy[o] * w.W3[o * MH + i];
      }
    }
    for (int i = 0; i < MH; ++i) dz2[i] = z2[i] > 0 ? dh2[i] : 0;
    for (int i = 0; i < MH; ++i) dh1[i] = 0;
    for (int o = 0; o < MH; ++o) {
      gb2[o] += dz2[o];
      for (int i = 0; i < MH; ++i) {
        gW2[o * MH + i] += dz2[o] * h1[i];
        dh1[i] += dz2[o] * w.W2[o * MH + i];
      }
    }
    for (int i = 0; i < MH; ++i) dz1[i] = z1[i] > 0 ? dh1[i] : 0;
    for (int o = 0; o < MH; ++o) {
      gb1[o] += dz1[o];
      for (int i = 0; i < MI; ++i) gW1[o * MI + i] += dz1[o] * xb[i];
    }
  }
  return loss / (double)B;
}

// Rigorous bounds on how far a reduced-precision evaluation of the network,
// its loss and its gradient can lie from the exact values computed above.
// The model of the reduced-precision side, stated per operation:
//   * weights and inputs are the same numbers on both sides;
//   * a dot product of K terms plus a bias is accumulated with error at most
//     acc (K + 1) |b| + sum |terms|, acc = 2^-23 (FP32 accumulation, products
//     of the rounded operands exact);
//   * the hidden activations relu(z) that feed the next layer, and the
//     weight-gradient operands, are rounded with relative error at most
//     u_act and u_grad (2^-8 for BF16 with round to nearest);
//   * the loss derivative 2 (y - t) / B, and the loss, are formed in FP32.
// Each quantity v of the exact computation gets a bound e_v on the distance
// of the reduced-precision value, propagated forward in the evaluation order:
//   |a' b' - a b| <= e_a (|b| + e_b) + |a| e_b,   |relu(a') - relu(a)| <= e_a.
// Where |z| <= e_z the ReLU mask of the two sides may differ, and the bound
// of the masked gradient is the whole |gradient| + its own bound.
// Outputs: ybound [B][2], gbound [MLP_NPARAM], *lbound (loss).
int hto_mlp_error_bound(int64_t B, const double* x, const double* target, const double* params, double u_act,
                        double u_grad, double* ybound, double* gbound, double* lbound) {
  MlpView w(params);
  const double acc = std::ldexp(1.0, -23), u32 = std::ldexp(1.0, -24);
  std::memset(gbound, 0, sizeof(double) * MLP_NPARAM);
  // magnitudes of the gradient sums (for their accumulation error)
  std::vector<double> gmag(MLP_NPARAM, 0.0);
  double *eW1 = gbound, *eb1 = eW1 + MH * MI, *eW2 = eb1 + MH, *eb2 = eW2 + MH * MH, *eW3 = eb2 + MH,
         *eb3 = eW3 + MO * MH;
  double *mW1 = gmag.data(), *mb1 = mW1 + MH * MI, *mW2 = mb1 + MH, *mb2 = mW2 + MH * MH, *mW3 = mb2 + MH,
         *mb3 = mW3 + MO * MH;
  double z1[MH], h1[MH], z2[MH], h2[MH], y[MO];
  double ez1[MH], eh1[MH], ez2[MH], eh2[MH], ey[MO];
  double dy[MO], edy[MO], g2[MH], eg2[MH], dz2[MH], edz2[MH], g1[MH], eg1[MH], dz1[MH], edz1[MH];
  double lmag = 0.0, lerr = 0.0;
  // rounding of an operand that carries error e: the rounded value differs
  // from the exact one by at most e + u (|v| + e)
  auto rnd = [](double v, double e, double u) { return e + u * (std::fabs(v) + e); };
  for (int64_t b = 0; b < B; ++b) {
    const double* xb = x + b * MI;
    mlp_forward_one(w, xb, z1, h1, z2, h2, y);
    for (int o = 0; o < MH; ++o) {  // layer 1: exact operands, FP32 sum
      double m = std::fabs(w.b1[o]);
      for (int i = 0; i < MI; ++i) m += std::fabs(w.W1[o * MI + i] * xb[i]);
      ez1[o] = acc * (MI + 1) * m;
      eh1[o] = rnd(h1[o], ez1[o], u_act);
    }
    for (int o = 0; o < MH; ++o) {  // layer 2: rounded h1
      double m = std::fabs(w.b2[o]), e = 0.0;
      for (int i = 0; i < MH; ++i) {
        const double a = std::fabs(w.W2[o * MH + i]);
        e += a * eh1[i];
        m += a * (h1[i] + eh1[i]);
      }
      ez2[o] = e + acc * (MH + 1) * m;
      eh2[o] = rnd(h2[o], ez2[o], u_act);
    }
    for (int o = 0; o < MO; ++o) {  // layer 3: rounded h2
      double m = std::fabs(w.b3[o]), e = 0.0;
      for (int i = 0; i < MH; ++i) {
        const double a = std::fabs(w.W3[o * MH + i]);
        e += a * eh2[i];
        m += a * (h2[i] + eh2[i]);
      }
      ey[o] = e + acc * (MH + 1) * m;
      ybound[b * MO + o] = ey[o];
    }
    for (int o = 0; o < MO; ++o) {  // loss terms and dL/dy = 2 (y - t) / B (two FP32 roundings)
      const double r = std::fabs(y[o] - target[b * MO + o]);
      lerr += 2.0 * r * ey[o] + ey[o] * ey[o];
      lmag += (r + ey[o]) * (r + ey[o]);
      dy[o] = 2.0 * (y[o] - target[b * MO + o]) / (double)B;
      const double ed = 2.0 * ey[o] / (double)B;
      edy[o] = ed + 2.0 * u32 * (std::fabs(dy[o]) + ed);
    }
    for (int i = 0; i < MH; ++i) {  // dh2 = W3^T dy, then the layer-2 mask
      double v = 0.0, e = 0.0, m = 0.0;
      for (int o = 0; o < MO; ++o) {
        const double a = w.W3[o * MH + i];
        v += a * dy[o];
        e += std::fabs(a) * edy[o];
        m += std::fabs(a) * (std::fabs(dy[o]) + edy[o]);
      }
      g2[i] = v;
      eg2[i] = e + acc * (MO + 1) * m;
      if (z2[i] > ez2[i]) {
        dz2[i] = g2[i];
        edz2[i] = eg2[i];
      } else if (z2[i] < -ez2[i]) {
        dz2[i] = 0.0;
        edz2[i] = 0.0;
      } else {  // the masks may differ
        dz2[i] = z2[i] > 0 ? g2[i] : 0.0;
        edz2[i] = std::fabs(g2[i]) + eg2[i];
      }
    }
    for (int i = 0; i < MH; ++i) {  // dh1 = W2^T dz2 with rounded dz2, then the layer-1 mask
      double v = 0.0, e = 0.0, m = 0.0;
      for (int o = 0; o < MH; ++o) {
        const double a = w.W2[o * MH + i];
        v += a * dz2[o];
        const double eo = rnd(dz2[o], edz2[o], u_grad);
        e += std::fabs(a) * eo;
        m += std::fabs(a) * (std::fabs(dz2[o]) + eo);
      }
      g1[i] = v;
      eg1[i] = e + acc * (MH + 1) * m;
      if (z1[i] > ez1[i]) {
        dz1[i] = g1[i];
        edz1[i] = eg1[i];
      } else if (z1[i] < -ez1[i]) {
        dz1[i] = 0.0;
        edz1[i] = 0.0;
      } else {
        dz1[i] = z1[i] > 0 ? g1[i] : 0.0;
        edz1[i] = std::fabs(g1[i]) + eg1[i];
      }
    }
    // weight gradients: sum over samples of (rounded gradient) x (rounded activation)
    auto term = [&](double a, double ea, double c, double ec, double* e, double* m) {
      const double ear = rnd(a, ea, u_grad);
      *e += ear * (std::fabs(c) + ec) + std::fabs(a) * ec;
      *m += (std::fabs(a) + ear) * (std::fabs(c) + ec);
    };
    for (int o = 0; o < MO; ++o) {
      eb3[o] += edy[o];
      mb3[o] += std::fabs(dy[o]) + edy[o];
      for (int i = 0; i < MH; ++i) term(dy[o], edy[o], h2[i], eh2[i], &eW3[o * MH + i], &mW3[o * MH + i]);
    }
    for (int o = 0; o < MH; ++o) {
      eb2[o] += edz2[o];
      mb2[o] += std::fabs(dz2[o]) + edz2[o];
      for (int i = 0; i < MH; ++i) term(dz2[o], edz2[o], h1[i], eh1[i], &eW2[o * MH + i], &mW2[o * MH + i]);
    }
    for (int o = 0; o < MH; ++o) {
      eb1[o] += edz1[o];
      mb1[o] += std::fabs(dz1[o]) + edz1[o];
      for (int i = 0; i < MI; ++i) term(dz1[o], edz1[o], xb[i], 0.0, &eW1[o * MI + i], &mW1[o * MI + i]);
    }
  }
  for (int p = 0; p < MLP_NPARAM; ++p) gbound[p] += acc * (double)(B + 1) * gmag[p];
  *lbound = (lerr + acc * (double)(2 * B + 2) * lmag) / (double)B;
  return 0;
}

// One Adam step (Kingma & Ba 2015) on fp64 parameters; step is 1-based.
int hto_adam_step(int64_t n, double* p, const double* g, double* m, double* v, double lr, double b1, double b2,
                  double eps, int step) {
  double c1 = 1.0 - std::pow(b1, step), c2 = 1.0 - std::pow(b2, step);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    p[i] -= lr * (m[i] / c1) / (std::sqrt(v[i] / c2) + eps);
  }
  return 0;
}

}  // extern "C"
