// Fused evaluation and differentiation of a polynomial system at many points
// (Section 3 of Verschelde & Yu 2015: the coeff, mon and sum kernels of
// Table tabcpugpu, here one kernel).
//
// Work decomposition.  A unit is (32 consecutive points, one polynomial).  One
// warp evaluates a unit: each lane owns one point, all lanes walk the same
// monomials in the same order, so every branch and every load of the system
// ("instructions" of Table tabmemory) is warp-uniform and served by one
// broadcast.  Units are dealt round-robin to the warps of a grid sized to the
// SMs, which balances the per-SMSP arithmetic pipe the kernel is bound by.
//
// Per monomial c * prod_{r} x_{v_r}^{a_r} with k variables of positive exponent:
//   cf    = c * prod_{a_r > 1} x_{v_r}^(a_r - 1)        (common factor, Section 1)
//   P_r   = cf * x_{v_0} ... x_{v_r}                    forward products, k mults
//   value = P_{k-1}
//   dv_r  = a_r * P_{r-1} * (x_{v_{r+1}} ... x_{v_{k-1}}) backward sweep
// which is the reverse mode of Table tabmoneval with the common factor folded
// into the first forward product: 3k - 3 complex multiplications for value and
// all k derivatives (the table's 3k - 5 products plus k + 1 multiplications by
// the common factor would take 4k - 4).
//
// Outputs are written in the vertical layout of Table tabtranspose; the
// Jacobian row of the unit's polynomial accumulates in place in the output
// array (it stays in L2 while the unit runs), so no scratch memory is used.
#include "ht_internal.h"
#include "ht_mp.cuh"

namespace ht {

struct EvalArgs {
  const int32_t* poly_off;
  const int32_t* mon_off;
  const uint16_t* pairs;
  const double* coef;
  int nv, np;
  int64_t npts;
  const double* x;
  double* val;
  double* jac;
  int64_t n_units;
};

template <int L, int K>
__device__ __forceinline__ void mono_fixed(const EvalArgs& a, int m, int64_t p, double* jrow, cx<L>& accv) {
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
    J[0] = (ex[0] == 1.0) ? cadd(J[0], cf) : caxpy(J[0], ex[0], cf);
  } else {
    J[K - 1] = (ex[K - 1] == 1.0) ? cadd(J[K - 1], P[K - 2]) : caxpy(J[K - 1], ex[K - 1], P[K - 2]);
    cx<L> S = xs[K - 1];
#pragma unroll
    for (int r = K - 2; r >= 1; --r) {
      cx<L> d = cmul(P[r - 1], S);
      J[r] = (ex[r] == 1.0) ? cadd(J[r], d) : caxpy(J[r], ex[r], d);
      S = cmul(S, xs[r]);
    }
    cx<L> d0 = cmul(cf, S);
    J[0] = (ex[0] == 1.0) ? cadd(J[0], d0) : caxpy(J[0], ex[0], d0);
  }
#pragma unroll
  for (int r = 0; r < K; ++r) st<L>(jrow, var[r], a.npts, p, J[r]);
}

// Supports wider than 8 variables: the same sweep with runtime bounds (local
// memory arrays); rare in practice.
template <int L>
__device__ __noinline__ void mono_wide(const EvalArgs& a, int m, int64_t p, double* jrow, cx<L>& accv) {
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
  cx<L> S = creal<L>(1.0);
  for (int r = k - 1; r >= 0; --r) {
    uint16_t q = __ldg(pr + r);
    int v = q & 0xff;
    double e = (double)(q >> 8);
    cx<L> d = (r == 0) ? cmul(cf, S) : cmul(P[r - 1], S);
    cx<L> Jv = ld<L>(jrow, v, a.npts, p);
    st<L>(jrow, v, a.npts, p, e == 1.0 ? cadd(Jv, d) : caxpy(Jv, e, d));
    if (r > 0) S = cmul(S, ld<L>(a.x, v, a.npts, p));
  }
}

template <int L>
__global__ void __launch_bounds__(128) evaldiff_kernel(EvalArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t plane = (int64_t)a.nv * 2 * L * a.npts;  // doubles per Jacobian row
  for (int64_t u = warp; u < a.n_units; u += n_warps) {
    const int j = (int)(u % a.np);
    const int64_t p = (u / a.np) * 32 + lane;
    if (p >= a.npts) continue;  // lanes past the ragged tail sit the unit out
    double* jrow = a.jac + (int64_t)j * plane;
    for (int i = 0; i < a.nv; ++i) st<L>(jrow, i, a.npts, p, czero<L>());
    cx<L> accv = czero<L>();
    const int m0 = __ldg(a.poly_off + j), m1 = __ldg(a.poly_off + j + 1);
    for (int m = m0; m < m1; ++m) {
      const int k = __ldg(a.mon_off + m + 1) - __ldg(a.mon_off + m);
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
        default: mono_wide<L>(a, m, p, jrow, accv); break;
      }
    }
    st<L>(a.val, j, a.npts, p, accv);
  }
}

template <int L>
int launch_evaldiff_l(const ht_system* s, int64_t n_pts, const double* x, double* val, double* jac, cudaStream_t st) {
  EvalArgs a;
  a.poly_off = s->d_poly_off;
  a.mon_off = s->d_mon_off;
  a.pairs = s->d_pairs;
  a.coef = s->d_coef;
  a.nv = s->nv;
  a.np = s->np;
  a.npts = n_pts;
  a.x = x;
  a.val = val;
  a.jac = jac;
  a.n_units = ((n_pts + 31) / 32) * s->np;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, evaldiff_kernel<L>, 128, 0);
  if (per_sm < 1) per_sm = 1;
  int64_t want = (a.n_units + 3) / 4;  // 4 warps per block
  int64_t grid = (int64_t)sm_count() * per_sm;
  if (grid > want) grid = want;
  evaldiff_kernel<L><<<(unsigned)grid, 128, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "ht_eval_diff: launch");
  return HT_OK;
}

#ifndef HT_LIMBS
#error "compile once per precision with -DHT_LIMBS=1, 2 or 4"
#endif
template int launch_evaldiff_l<HT_LIMBS>(const ht_system*, int64_t, const double*, double*, double*, cudaStream_t);

}  // namespace ht
