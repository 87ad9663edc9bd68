// Host build of the library's multi-limb integer arithmetic (csrc/ht_mpi.cuh)
// for CPU tests of that arithmetic against the oracle.
#include <cstdint>
#include <cstdio>
#include <vector>

#include "../paper_1505_00383_gb300/csrc/ht_mpi.cuh"
#include "../paper_1505_00383_gb300/csrc/ht_mpi_ops.cuh"

using namespace ht::mpi;

// Fixed frame F so that |value| < 2^(29 (WA - 1) + 28 + F), with `head` bits
// of headroom above the value's exponent e.
template <int WA>
static int frame_for(int e, int head) { return e + 1 + head - (RB * (WA - 1) + 28); }

template <int W, int WA, int L>
static void roundtrip(int64_t n, const double* in, double* out) {
  for (int64_t q = 0; q < n; ++q) {
    const double* re = in + q * 2 * L;
    const double* im = re + L;
    fz<W> z = from_doubles<W, L>(re, im);
    int32_t ar[WA] = {0}, ai[WA] = {0};
    // the value's exponent: top limb bit 28 at most
    const int F = frame_for<WA>(z.f + RB * (W - 1) + 28, 2);
    acc_add<W, WA>(ar, ai, z, 1, F);
    fixed_to_doubles<WA, L>(ar, F, out + q * 2 * L);
    fixed_to_doubles<WA, L>(ai, F, out + q * 2 * L + L);
  }
}

template <int W, int WA, int L>
static void product(int64_t n, const double* a, const double* b, int e_mul, double* out) {
  for (int64_t q = 0; q < n; ++q) {
    fz<W> x = from_doubles<W, L>(a + q * 2 * L, a + q * 2 * L + L);
    fz<W> y = from_doubles<W, L>(b + q * 2 * L, b + q * 2 * L + L);
    fz<W> z = mul<W>(x, y);
    int32_t ar[WA] = {0}, ai[WA] = {0};
    const int F = frame_for<WA>(z.f + RB * (W - 1) + 28, 4);
    acc_add<W, WA>(ar, ai, z, e_mul, F);
    fixed_to_doubles<WA, L>(ar, F, out + q * 2 * L);
    fixed_to_doubles<WA, L>(ai, F, out + q * 2 * L + L);
  }
}

// sum_j e_j * (a_j * b_j) accumulated in one fixed frame (the Jacobian-entry
// pattern of the evaluation kernel); terms [n][k][2][L].
template <int W, int WA, int L, bool FAST>
static void dot(int64_t n, int k, const double* a, const double* b, const int* e, int head, double* out) {
  for (int64_t q = 0; q < n; ++q) {
    int32_t ar[WA] = {0}, ai[WA] = {0};
    int emax = -100000;
    fz<W> zs[64];
    for (int j = 0; j < k; ++j) {
      const double* pa = a + (q * k + j) * 2 * L;
      const double* pb = b + (q * k + j) * 2 * L;
      zs[j] = mul<W>(from_doubles<W, L>(pa, pa + L), from_doubles<W, L>(pb, pb + L));
      const int ez = zs[j].f + RB * (W - 1) + 28 + 2;  // |e z| < 2^(ez) with e <= 3
      if (ez > emax) emax = ez;
    }
    const int F = frame_for<WA>(emax, head);
    for (int j = 0; j < k; ++j) {
      if (FAST)
        acc_add_fast<W, WA>(ar, ai, zs[j], e[j], F);
      else
        acc_add<W, WA>(ar, ai, zs[j], e[j], F);
    }
    fixed_to_doubles<WA, L>(ar, F, out + q * 2 * L);
    fixed_to_doubles<WA, L>(ai, F, out + q * 2 * L + L);
  }
}

extern "C" {
int mpi_roundtrip(int L, int64_t n, const double* in, double* out) {
  if (L == 2) roundtrip<5, 4, 2>(n, in, out);
  else if (L == 4) roundtrip<8, 8, 4>(n, in, out);
  else return -1;
  return 0;
}
int mpi_product(int L, int64_t n, const double* a, const double* b, int e, double* out) {
  if (L == 2) product<5, 4, 2>(n, a, b, e, out);
  else if (L == 4) product<8, 8, 4>(n, a, b, e, out);
  else return -1;
  return 0;
}
int mpi_dot(int L, int64_t n, int k, const double* a, const double* b, const int* e, int head, double* out) {
  if (k > 64) return -1;
  if (L == 2) dot<5, 4, 2, false>(n, k, a, b, e, head, out);
  else if (L == 4) dot<8, 8, 4, false>(n, k, a, b, e, head, out);
  else return -1;
  return 0;
}
int mpi_dot_fast(int L, int64_t n, int k, const double* a, const double* b, const int* e, int head, double* out) {
  if (k > 64) return -1;
  if (L == 2) dot<5, 4, 2, true>(n, k, a, b, e, head, out);
  else if (L == 4) dot<8, 8, 4, true>(n, k, a, b, e, head, out);
  else return -1;
  return 0;
}
}

// acc_add_fast against the generic acc_add for shifts s = F - f in [smin, smax]
// (negative s: the term's frame lies above the accumulator's).  For the left
// shifts the term is first moved one limb up (top limb empty) so that it fits.
// Returns the largest difference of the two accumulated values in units of
// the accumulator's last limb (they may differ by the truncation of the
// dropped bits: the generic version truncates each limb toward zero).
template <int W, int WA, int L>
static int64_t compare_acc(int64_t n, const double* in, int smin, int smax, int e) {
  int64_t worst = 0;
  for (int64_t q = 0; q < n; ++q) {
    fz<W> z0 = from_doubles<W, L>(in + q * 2 * L, in + q * 2 * L + L);
    fz<W> z1 = z0;  // same value up to the dropped low limb, one limb down
    for (int k = 0; k + 1 < W; ++k) {
      z1.r[k] = z0.r[k + 1];
      z1.i[k] = z0.i[k + 1];
    }
    // the old top limb is signed; below the top a limb lies in [0, 2^29), so
    // a negative top moves down as its two's complement digit and the new top
    // carries the sign (-1)
    z1.r[W - 2] = z0.r[W - 1] & MASK;
    z1.i[W - 2] = z0.i[W - 1] & MASK;
    z1.r[W - 1] = z0.r[W - 1] < 0 ? -1 : 0;
    z1.i[W - 1] = z0.i[W - 1] < 0 ? -1 : 0;
    z1.f = z0.f + RB;
    for (int s = smin; s <= smax; ++s) {
      const fz<W>& z = s < 0 ? z1 : z0;
      const int F = z.f + s;
      // the fast routine's precondition: 3 |z| < 2^(29 (WA - 1) + 28 + F);
      // skip the frames it excludes (for DD, WA = W - 1, every s < 0)
      int top = -1;
      for (int k = W - 1; k >= 0 && top < 0; --k)
        if (z.r[k] != 0 || z.i[k] != 0) top = k;
      if (top >= 0) {
        const int64_t mr = z.r[top] < 0 ? -(int64_t)z.r[top] : z.r[top];
        const int64_t mi = z.i[top] < 0 ? -(int64_t)z.i[top] : z.i[top];
        int b = 0;
        while (((mr > mi ? mr : mi) >> b) != 0) ++b;
        const int ae = e < 0 ? -e : e;
        int eb = 0;
        while ((ae >> eb) != 0) ++eb;
        const int bits = z.f + RB * top + b + eb + 1;  // bit length of |e z|, bound from above
        if (bits > RB * (WA - 1) + 28 + F) continue;
      }
      int32_t a1[WA] = {0}, b1[WA] = {0}, a2[WA] = {0}, b2[WA] = {0};
      a1[0] = a2[0] = 12345;
      b1[WA - 1] = b2[WA - 1] = -7;
      acc_add<W, WA>(a1, b1, z, e, F);
      acc_add_fast<W, WA>(a2, b2, z, e, F);
      // exact difference of the values, limb by limb from the top (it is small)
      long double dr = 0, di = 0;
      for (int k = WA - 1; k >= 0; --k) {
        dr = dr * (long double)(1 << RB) + (long double)(a1[k] - a2[k]);
        di = di * (long double)(1 << RB) + (long double)(b1[k] - b2[k]);
      }
      // a difference beyond int64 is reported as such (no overflowing cast)
      const long double big = 9.0e18L;
      const long double adr = dr < 0 ? -dr : dr, adi = di < 0 ? -di : di;
      const int64_t m = adr >= big ? INT64_MAX : (int64_t)adr, mi = adi >= big ? INT64_MAX : (int64_t)adi;
      if (m > worst) worst = m;
      if (mi > worst) worst = mi;
    }
  }
  return worst;
}
extern "C" int64_t mpi_compare_acc(int L, int64_t n, const double* in, int smin, int smax, int e) {
  if (L == 2) return compare_acc<5, 4, 2>(n, in, smin, smax, e);
  if (L == 4) return compare_acc<8, 8, 4>(n, in, smin, smax, e);
  return -1;
}

// ---- the integer evaluation of whole systems (the kernel's per-lane code)
#include <cmath>
#include <vector>

#include "../paper_1505_00383_gb300/csrc/ht_mpi_eval.cuh"

template <int L>
struct HostRowAcc {
  static constexpr int WA = IntW<L>::WA;
  std::vector<int32_t> r, i;  // [nv][WA]
  void add(int v, const fz<IntW<L>::W>& d, int e, int F) { acc_add_fast<IntW<L>::W, WA>(&r[v * WA], &i[v * WA], d, e, F); }
};

template <int L>
static void eval_int(int nv, int np, const int32_t* n_terms, const int8_t* exps, const double* coef, int64_t n_pts,
                     const double* x, double* val, double* jac) {
  constexpr int W = IntW<L>::W, WA = IntW<L>::WA;
  std::vector<int32_t> poly_off(np + 1, 0), mon_off(1, 0);
  std::vector<uint16_t> pairs;
  for (int j = 0; j < np; ++j) poly_off[j + 1] = poly_off[j] + n_terms[j];
  const int M = poly_off[np];
  std::vector<fz<W>> cfz(M);
  std::vector<float> clg(M);
  for (int m = 0; m < M; ++m) {
    for (int i = 0; i < nv; ++i)
      if (exps[m * nv + i] > 0) pairs.push_back((uint16_t)(i | (exps[m * nv + i] << 8)));
    mon_off.push_back((int32_t)pairs.size());
    const double* re = coef + (size_t)m * 2 * L;
    cfz[m] = from_doubles<W, L>(re, re + L);
    const double mod = std::hypot(re[0], re[L]);
    clg[m] = mod == 0.0 ? -1000.0f : (float)std::log2(mod);
  }
  std::vector<fz<W>> X(nv), P(64);
  std::vector<float> lg(nv);
  for (int64_t p = 0; p < n_pts; ++p) {
    for (int i = 0; i < nv; ++i) {
      double re[L], im[L];
      for (int l = 0; l < L; ++l) {
        re[l] = x[((int64_t)(i * 2) * L + l) * n_pts + p];
        im[l] = x[((int64_t)(i * 2 + 1) * L + l) * n_pts + p];
      }
      X[i] = from_doubles<W, L>(re, im);
      lg[i] = log2_mod(re[0], im[0]);
    }
    for (int j = 0; j < np; ++j) {
      int Fv[64];
      const int F = frames_for_poly<WA>(mon_off.data(), pairs.data(), clg.data(), poly_off[j], poly_off[j + 1], lg.data(),
                                        nv, Fv);
      HostRowAcc<L> acc;
      acc.r.assign(nv * WA, 0);
      acc.i.assign(nv * WA, 0);
      int32_t vr[WA] = {0}, vi[WA] = {0};
      eval_poly_int<L>(mon_off.data(), pairs.data(), cfz.data(), poly_off[j], poly_off[j + 1], X.data(), F, Fv, acc, vr,
                       vi, P.data());
      double o[L];
      fixed_to_doubles<WA, L>(vr, F, o);
      for (int l = 0; l < L; ++l) val[((int64_t)(j * 2) * L + l) * n_pts + p] = o[l];
      fixed_to_doubles<WA, L>(vi, F, o);
      for (int l = 0; l < L; ++l) val[((int64_t)(j * 2 + 1) * L + l) * n_pts + p] = o[l];
      for (int i = 0; i < nv; ++i) {
        fixed_to_doubles<WA, L>(&acc.r[i * WA], Fv[i], o);
        for (int l = 0; l < L; ++l) jac[((((int64_t)j * nv + i) * 2) * L + l) * n_pts + p] = o[l];
        fixed_to_doubles<WA, L>(&acc.i[i * WA], Fv[i], o);
        for (int l = 0; l < L; ++l) jac[((((int64_t)j * nv + i) * 2 + 1) * L + l) * n_pts + p] = o[l];
      }
    }
  }
}

extern "C" int mpi_eval(int L, int nv, int np, const int32_t* n_terms, const int8_t* exps, const double* coef,
                        int64_t n_pts, const double* x, double* val, double* jac) {
  if (L == 1) eval_int<1>(nv, np, n_terms, exps, coef, n_pts, x, val, jac);
  else if (L == 2) eval_int<2>(nv, np, n_terms, exps, coef, n_pts, x, val, jac);
  else if (L == 4) eval_int<4>(nv, np, n_terms, exps, coef, n_pts, x, val, jac);
  else return -1;
  return 0;
}

// ---- general sums, normalisation, inverse square root
template <int W, int L>
static void sums(int64_t n, int k, const double* z, const int* e, double* out) {
  for (int64_t q = 0; q < n; ++q) {
    fz<W> t[16];
    for (int j = 0; j < k; ++j) t[j] = from_doubles<W, L>(z + (q * k + j) * 2 * L, z + (q * k + j) * 2 * L + L);
    fz<W> r = sum<W, 16>(t, e, k);
    // to doubles through a fixed frame
    int32_t ar[W + 1] = {0}, ai[W + 1] = {0};
    const int F = r.f;  // the value fits the frame: s = 0
    acc_add_fast<W, W + 1>(ar, ai, r, 1, F);
    fixed_to_doubles<W + 1, L>(ar, F, out + q * 2 * L);
    fixed_to_doubles<W + 1, L>(ai, F, out + q * 2 * L + L);
  }
}
template <int W, int L>
static void invsqrt(int64_t n, const double* v, double* out, int steps) {
  for (int64_t q = 0; q < n; ++q) {
    const double zero[L] = {0};
    fz<W> x = from_doubles<W, L>(v + q * L, zero);
    fz<W> y = inv_sqrt<W>(x, steps);
    int32_t ar[W + 1] = {0}, ai[W + 1] = {0};
    const int F = y.f;
    acc_add_fast<W, W + 1>(ar, ai, y, 1, F);
    fixed_to_doubles<W + 1, L>(ar, F, out + q * L);
  }
}
extern "C" int mpi_sum(int L, int64_t n, int k, const double* z, const int* e, double* out) {
  if (k > 16) return -1;
  if (L == 1) sums<3, 1>(n, k, z, e, out);
  else if (L == 2) sums<5, 2>(n, k, z, e, out);
  else if (L == 4) sums<8, 4>(n, k, z, e, out);
  else return -1;
  return 0;
}
extern "C" int mpi_invsqrt(int L, int64_t n, const double* v, double* out) {
  if (L == 1) invsqrt<3, 1>(n, v, out, 1);
  else if (L == 2) invsqrt<5, 2>(n, v, out, 2);
  else if (L == 4) invsqrt<8, 4>(n, v, out, 3);
  else return -1;
  return 0;
}

// ---- least squares by modified Gram-Schmidt on limb strings (one system)
template <int W, int L>
static void mgs_seq(int rows, int cols, const double* Ab, double* x) {
  constexpr int N = 64;
  using Z = fz<W>;
  const int C = cols + 1;
  std::vector<Z> A((size_t)rows * C), col(rows), Q(rows), scratch(rows), R((size_t)cols * C);
  for (int i = 0; i < rows; ++i)
    for (int j = 0; j < C; ++j) {
      const double* e = Ab + ((size_t)i * C + j) * 2 * L;
      A[(size_t)i * C + j] = from_doubles<W, L>(e, e + L);
    }
  auto column = [&](int j, std::vector<Z>& out) {
    for (int i = 0; i < rows; ++i) out[i] = A[(size_t)i * C + j];
  };
  auto put = [&](int j, const std::vector<Z>& in) {
    for (int i = 0; i < rows; ++i) A[(size_t)i * C + j] = in[i];
  };
  for (int q = 0; q < cols; ++q) {
    column(q, Q);
    Z nrm = norm2<W, N>(Q.data(), rows, scratch.data());
    Z inv = inv_sqrt<W>(nrm, inv_sqrt_steps<W>());
    for (int i = 0; i < rows; ++i) Q[i] = mul<W>(Q[i], inv);
    put(q, Q);
    R[(size_t)q * C + q] = inv;
    for (int j = q + 1; j < C; ++j) {
      column(j, col);
      Z r = dot_conj<W, N>(Q.data(), col.data(), rows, scratch.data());
      R[(size_t)q * C + j] = r;
      sub_scaled<W>(col.data(), r, Q.data(), rows);
      put(j, col);
    }
  }
  std::vector<Z> X(cols), terms(cols + 1);
  for (int q = cols - 1; q >= 0; --q) {
    int k = 0;
    terms[k++] = R[(size_t)q * C + cols];
    for (int j = q + 1; j < cols; ++j) terms[k++] = mul<W>(R[(size_t)q * C + j], X[j]);
    X[q] = mul<W>(first_minus_rest<W, N + 1>(terms.data(), k), R[(size_t)q * C + q]);
  }
  for (int q = 0; q < cols; ++q) to_doubles<W, L>(X[q], x + (size_t)q * 2 * L, x + (size_t)q * 2 * L + L);
}
extern "C" int mpi_mgs(int L, int rows, int cols, int64_t n_sys, const double* Ab, double* x) {
  if (rows < cols || cols < 1 || rows > 64) return -1;
  const size_t sa = (size_t)rows * (cols + 1) * 2 * L, sx = (size_t)cols * 2 * L;
  for (int64_t s = 0; s < n_sys; ++s) {
    if (L == 2) mgs_seq<5, 2>(rows, cols, Ab + s * sa, x + s * sx);
    else if (L == 4) mgs_seq<8, 4>(rows, cols, Ab + s * sa, x + s * sx);
    else if (L == 1) mgs_seq<3, 1>(rows, cols, Ab + s * sa, x + s * sx);
    else return -1;
  }
  return 0;
}

// s * a for fixed-point limb strings a (n rows of WA int32 limbs, frame F)
// and doubles s[n], to L doubles per row (out), and the unscaled conversion
// of the same strings (plain) for comparison.
template <int WA, int L>
static void scaled(int64_t n, const int32_t* a, int F, const double* s, double* out, double* plain) {
  for (int64_t q = 0; q < n; ++q) {
    fixed_scaled_to_doubles<WA, L>(a + q * WA, F, s[q], out + q * L);
    fixed_to_doubles<WA, L>(a + q * WA, F, plain + q * L);
  }
}
extern "C" int mpi_scaled_convert(int L, int64_t n, const int32_t* a, int F, const double* s, double* out,
                                  double* plain) {
  if (L == 1) scaled<2, 1>(n, a, F, s, out, plain);
  else if (L == 2) scaled<4, 2>(n, a, F, s, out, plain);
  else if (L == 4) scaled<8, 4>(n, a, F, s, out, plain);
  else return -1;
  return 0;
}

// s * (ar + i ai) for fixed-point limb strings (n rows of WA int32 limbs per
// component, frame F) and doubles s[n], as limb strings: out gets, per row,
// the exponent and the W re and W im limbs (2 W + 1 int32).
template <int WA, int W>
static void scaled_fz(int64_t n, const int32_t* ar, const int32_t* ai, int F, const double* s, int32_t* out) {
  for (int64_t q = 0; q < n; ++q) {
    const fz<W> z = fixed_scaled_to_fz<WA, W>(ar + q * WA, ai + q * WA, F, s[q]);
    int32_t* o = out + q * (2 * W + 1);
    o[0] = z.f;
    for (int k = 0; k < W; ++k) {
      o[1 + k] = z.r[k];
      o[1 + W + k] = z.i[k];
    }
  }
}
extern "C" int mpi_scaled_fz(int L, int64_t n, const int32_t* ar, const int32_t* ai, int F, const double* s,
                             int32_t* out) {
  if (L == 2) scaled_fz<4, 5>(n, ar, ai, F, s, out);
  else if (L == 4) scaled_fz<8, 8>(n, ar, ai, F, s, out);
  else return -1;
  return 0;
}
