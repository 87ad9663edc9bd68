// Reverse-mode evaluation of one polynomial and its gradient at one point per
// lane (Section 3 and Table tabmoneval of Verschelde & Yu 2015), shared by the
// evaluation kernel and the tracker's Newton step.
//
// Per monomial c * prod_r x_{v_r}^{a_r} with k variables of positive exponent:
//   cf    = c * prod_{a_r > 1} x_{v_r}^(a_r - 1)        (common factor, Section 1)
//   P_r   = cf * x_{v_0} ... x_{v_r}                    forward products, k mults
//   value = P_{k-1}
//   dv_r  = a_r * P_{r-1} * (x_{v_{r+1}} ... x_{v_{k-1}}) backward sweep
// i.e. the reverse mode of Table tabmoneval with the common factor folded into
// the first forward product: 3k - 3 complex multiplications for the value and
// all k derivatives (the table's 3k - 5 products plus k + 1 multiplications by
// the common factor would take 4k - 4).
#pragma once
#include "ht_mp.cuh"

namespace ht {

// The "instructions" of Table tabmemory as the kernels read them, plus where
// the points live: x is [nv][2][L][stride] and lane p reads column p.
struct PolyView {
  const int32_t* mon_off;   // [M + 1] range of each monomial in pairs
  const uint16_t* pairs;    // variable | exponent << 8
  const double* coef;       // [M][2][L]
  const double* x;
  int64_t npts;             // column stride of x and of the Jacobian row
};

// J += e * d for a derivative d and its exponent e.  In complex double the fma
// with e = 1 rounds exactly like the add, so no branch is taken there.
template <int L>
__device__ __forceinline__ cx<L> jacc(cx<L> J, double e, cx<L> d) {
  if constexpr (L == 1) {
    return caxpy(J, e, d);
  } else {
    return e == 1.0 ? cadd(J, d) : caxpy(J, e, d);
  }
}

template <int L, int K>
__device__ __forceinline__ void mono_fixed(const PolyView& a, int m, int64_t p, double* jrow, cx<L>& accv) {
  const uint16_t* pr = a.pairs + __ldg(a.mon_off + m);
  int var[K];
  double ex[K];
  cx<L> xs[K], J[K];
#pragma unroll
  for (int r = 0; r < K; ++r) {
    uint16_t q = __ldg(pr + r);
    var[r] = q & 0xff;
    ex[r] = (double)(q >> 8);
  }
#pragma unroll
  for (int r = 0; r < K; ++r) xs[r] = ld<L>(a.x, var[r], a.npts, p);
#pragma unroll
  for (int r = 0; r < K; ++r) J[r] = ld<L>(jrow, var[r], a.npts, p);
  cx<L> cf = ld_coef<L>(a.coef + (int64_t)m * 2 * L);
#pragma unroll
  for (int r = 0; r < K; ++r)
    for (int e = 1; e < (int)ex[r]; ++e) cf = cmul(cf, xs[r]);
  cx<L> P[K];
  P[0] = cmul(cf, xs[0]);
#pragma unroll
  for (int r = 1; r < K; ++r) P[r] = cmul(P[r - 1], xs[r]);
  accv = cadd(accv, P[K - 1]);
  if constexpr (K == 1) {
    J[0] = jacc<L>(J[0], ex[0], cf);
  } else {
    J[K - 1] = jacc<L>(J[K - 1], ex[K - 1], P[K - 2]);
    cx<L> S = xs[K - 1];
#pragma unroll
    for (int r = K - 2; r >= 1; --r) {
      cx<L> d = cmul(P[r - 1], S);
      J[r] = jacc<L>(J[r], ex[r], d);
      S = cmul(S, xs[r]);
    }
    cx<L> d0 = cmul(cf, S);
    J[0] = jacc<L>(J[0], ex[0], d0);
  }
#pragma unroll
  for (int r = 0; r < K; ++r) st<L>(jrow, var[r], a.npts, p, J[r]);
}

// The same sweep with runtime bounds: one compact body for every support size
// (forward products in local memory).  It performs the operations of
// mono_fixed in the same order, so both give bitwise identical results; the
// compact body keeps the instruction cache warm when supports vary.
template <int L>
__device__ __noinline__ void mono_loop(const PolyView& a, int m, int64_t p, double* jrow, cx<L>& accv) {
  const int beg = __ldg(a.mon_off + m), k = __ldg(a.mon_off + m + 1) - beg;
  const uint16_t* pr = a.pairs + beg;
  cx<L> P[64];
  cx<L> cf = ld_coef<L>(a.coef + (int64_t)m * 2 * L);
  for (int r = 0; r < k; ++r) {
    uint16_t q = __ldg(pr + r);
    cx<L> xr = ld<L>(a.x, q & 0xff, a.npts, p);
    for (int e = 1; e < (q >> 8); ++e) cf = cmul(cf, xr);
  }
  for (int r = 0; r < k; ++r) {
    cx<L> xr = ld<L>(a.x, __ldg(pr + r) & 0xff, a.npts, p);
    P[r] = cmul(r == 0 ? cf : P[r - 1], xr);
  }
  accv = cadd(accv, P[k - 1]);
  if (k == 1) {
    uint16_t q = __ldg(pr);
    st<L>(jrow, q & 0xff, a.npts, p, jacc<L>(ld<L>(jrow, q & 0xff, a.npts, p), (double)(q >> 8), cf));
    return;
  }
  uint16_t q = __ldg(pr + k - 1);
  int v = q & 0xff;
  st<L>(jrow, v, a.npts, p, jacc<L>(ld<L>(jrow, v, a.npts, p), (double)(q >> 8), P[k - 2]));
  cx<L> S = ld<L>(a.x, v, a.npts, p);
  for (int r = k - 2; r >= 1; --r) {
    q = __ldg(pr + r);
    v = q & 0xff;
    cx<L> d = cmul(P[r - 1], S);
    st<L>(jrow, v, a.npts, p, jacc<L>(ld<L>(jrow, v, a.npts, p), (double)(q >> 8), d));
    S = cmul(S, ld<L>(a.x, v, a.npts, p));
  }
  q = __ldg(pr);
  v = q & 0xff;
  cx<L> d0 = cmul(cf, S);
  st<L>(jrow, v, a.npts, p, jacc<L>(ld<L>(jrow, v, a.npts, p), (double)(q >> 8), d0));
}

// Value of polynomial j (monomials m0..m1-1) at column p; its gradient is
// accumulated into jrow ([nv][2][L][npts], zeroed here first).
// LOOP selects the compact body for every monomial; otherwise supports of up
// to 8 variables use the unrolled bodies.
template <int L, bool LOOP = true>
__device__ __forceinline__ cx<L> eval_poly(const PolyView& a, int m0, int m1, int nv, int64_t p, double* jrow) {
  for (int i = 0; i < nv; ++i) st<L>(jrow, i, a.npts, p, czero<L>());
  cx<L> accv = czero<L>();
  for (int m = m0; m < m1; ++m) {
    const int k = __ldg(a.mon_off + m + 1) - __ldg(a.mon_off + m);
    if (LOOP && k > 0) {
      mono_loop<L>(a, m, p, jrow, accv);
      continue;
    }
    switch (k) {
      case 0: accv = cadd(accv, ld_coef<L>(a.coef + (int64_t)m * 2 * L)); break;
      case 1: mono_fixed<L, 1>(a, m, p, jrow, accv); break;
      case 2: mono_fixed<L, 2>(a, m, p, jrow, accv); break;
      case 3: mono_fixed<L, 3>(a, m, p, jrow, accv); break;
      case 4: mono_fixed<L, 4>(a, m, p, jrow, accv); break;
      case 5: mono_fixed<L, 5>(a, m, p, jrow, accv); break;
      case 6: mono_fixed<L, 6>(a, m, p, jrow, accv); break;
      case 7: mono_fixed<L, 7>(a, m, p, jrow, accv); break;
      case 8: mono_fixed<L, 8>(a, m, p, jrow, accv); break;
      default: mono_loop<L>(a, m, p, jrow, accv); break;
    }
  }
  return accv;
}

}  // namespace ht
