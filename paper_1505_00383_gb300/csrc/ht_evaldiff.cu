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
#include "ht_eval.cuh"
#include "ht_internal.h"
#include "ht_int_row.cuh"

namespace ht {

struct EvalArgs {
  PolyView v;
  const int32_t* poly_off;  // advanced to the first polynomial of the range
  int nv, np;               // np: polynomials in the range; val and jac hold them from index 0
  double* val;
  double* jac;
  int64_t n_units;
};

template <int L, bool LOOP>
__global__ void __launch_bounds__(256) evaldiff_kernel(EvalArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t n = a.v.npts;
  const int64_t plane = (int64_t)a.nv * 2 * L * n;  // doubles per Jacobian row
  for (int64_t u = warp; u < a.n_units; u += n_warps) {
    const int j = (int)(u % a.np);
    const int64_t p = (u / a.np) * 32 + lane;
    if (p >= n) continue;  // lanes past the ragged tail sit the unit out
    cx<L> v = eval_poly<L, LOOP>(a.v, __ldg(a.poly_off + j), __ldg(a.poly_off + j + 1), a.nv, p, a.jac + (int64_t)j * plane);
    st<L>(a.val, j, n, p, v);
  }
}

template <int L, bool LOOP>
static int launch_v(const EvalArgs& a, int threads, cudaStream_t st) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, evaldiff_kernel<L, LOOP>, threads, 0);
  if (per_sm < 1) per_sm = 1;
  const int wpb = threads / 32;
  int64_t want = (a.n_units + wpb - 1) / wpb;
  int64_t grid = (int64_t)sm_count() * per_sm;
  if (grid > want) grid = want;
  evaldiff_kernel<L, LOOP><<<(unsigned)grid, threads, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "ht_eval_diff: launch");
  return HT_OK;
}


// ------------------------------------------------------------------------
// Integer-pipe variant for double double and quad double (see ht_mpi.cuh):
// the same reverse-mode sweep on multi-limb integer complex numbers.  Per unit
// (polynomial j, 32 points) each lane
//   1. converts its point's variables once (local memory) and their log2 moduli;
//   2. bounds every term of polynomial j -- log2|c| + sum a log2|x| for the
//      value, minus log2|x_v| plus log2 a_v for a derivative -- and fixes one
//      accumulator frame above the largest bound plus log2 of the term count;
//   3. accumulates value and Jacobian row as fixed-point limbs: the row lives
//      in place in the output (2L doubles hold exactly 2 x 2L int32 limbs);
//   4. converts the accumulators to L doubles.
template <int L>
__global__ void __launch_bounds__(128, 4) evaldiff_int_kernel(EvalArgs a, const mpi::fz<IntW<L>::W>* __restrict__ cfz,
                                                           const float* __restrict__ clg) {
  using Z = mpi::fz<IntW<L>::W>;
  Z X[kIntMaxVars];
  float lg[kIntMaxVars];
  mpi::fzs<IntW<L>::W> P[64];
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t n = a.v.npts;
  const int64_t plane = (int64_t)a.nv * 2 * L * n;
  for (int64_t u = warp; u < a.n_units; u += n_warps) {
    const int j = (int)(u % a.np);
    const int64_t p = (u / a.np) * 32 + lane;
    if (p >= n) continue;
    int_point<L>(a.v.x, a.nv, n, p, X, lg);
    double vre[L], vim[L];
    int_row<L>(a.v.mon_off, a.v.pairs, cfz, clg, a.poly_off[j], a.poly_off[j + 1], X, lg, a.nv,
               a.jac + (int64_t)j * plane, n, p, vre, vim, P);
#pragma unroll
    for (int l = 0; l < L; ++l) {
      a.val[((int64_t)(j * 2) * L + l) * n + p] = vre[l];
      a.val[((int64_t)(j * 2 + 1) * L + l) * n + p] = vim[l];
    }
  }
}

// Block organisation of the same unit: a CTA takes a block of 32 points and
// a group of polynomials (as many as it has warps: one each; 16 warps when
// the system has at least 16 polynomials, else 8).  The block's
// converted points live once in shared memory (lane-interleaved, so every
// access is a conflict-free 32-word row) instead of once per lane and unit
// in local memory; the warp still walks one monomial with all lanes in step.
// Work items (polynomial group, point block) are ordered group-major, so a
// CTA keeps one group's monomials and coefficients (a QD coefficient is 68
// bytes) in its L1 across point blocks; the points are converted once per
// item.  The sums are the same exact integers, so the results are those of
// the per-unit kernel bit for bit.
template <int L>
__global__ void __launch_bounds__(512, 1) evaldiff_intblk_kernel(EvalArgs a, const mpi::fz<IntW<L>::W>* __restrict__ cfz,
                                                              const float* __restrict__ clg) {
  constexpr int W = IntW<L>::W;
  using Z = mpi::fz<W>;
  extern __shared__ __align__(16) int32_t xs[];  // [nv][2W+1][32] limb strings, then [nv][32] log2 moduli
  float* lgs = reinterpret_cast<float*>(xs + (int64_t)a.nv * (2 * W + 1) * 32);
  mpi::fzs<IntW<L>::W> P[64];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, T = blockDim.x >> 5;
  const int64_t n = a.v.npts, plane = (int64_t)a.nv * 2 * L * n, n_blocks = (n + 31) / 32;
  const int n_groups = (a.np + T - 1) / T;
  const SmemPoints<L> X{xs, lane};
  const SmemLog lg{lgs, lane};
  for (int64_t item = blockIdx.x; item < n_blocks * n_groups; item += gridDim.x) {
    const int64_t b = item % n_blocks;
    const int g = (int)(item / n_blocks);
    const int64_t p = b * 32 + lane;
    const bool live = p < n;
    __syncthreads();  // the previous block's points are no longer read
    for (int v = warp; v < a.nv; v += T) {
      double re[L], im[L];
#pragma unroll
      for (int l = 0; l < L; ++l) {
        re[l] = live ? a.v.x[((int64_t)(v * 2) * L + l) * n + p] : 0.0;
        im[l] = live ? a.v.x[((int64_t)(v * 2 + 1) * L + l) * n + p] : 0.0;
      }
      store_point<L>(xs, v, lane, mpi::from_doubles<W, L>(re, im));
      lgs[v * 32 + lane] = mpi::log2_mod(re[0], im[0]);
    }
    __syncthreads();
    if (!live) continue;  // lanes past the ragged tail sit the block out
    for (int j = g * T + warp; j < a.np && j < (g + 1) * T; j += T) {
      double vre[L], vim[L];
      int_row<L>(a.v.mon_off, a.v.pairs, cfz, clg, a.poly_off[j], a.poly_off[j + 1], X, lg, a.nv,
                 a.jac + (int64_t)j * plane, n, p, vre, vim, P);
#pragma unroll
      for (int l = 0; l < L; ++l) {
        a.val[((int64_t)(j * 2) * L + l) * n + p] = vre[l];
        a.val[((int64_t)(j * 2 + 1) * L + l) * n + p] = vim[l];
      }
    }
  }
}

template <int L>
static int launch_int(const EvalArgs& a, const ht_system* s, int threads, cudaStream_t st) {
  const auto* cf = reinterpret_cast<const mpi::fz<IntW<L>::W>*>(s->d_coef_fz);
  if (threads == 256) {  // block organisation (points in shared memory)
    // 16 warps share one copy of the points where there are polynomials for
    // them: half the shared memory of two 8-warp CTAs per SM, so more of the
    // SM's L1 holds the lanes' forward products (8 % faster for QD at
    // n = 32); the register cap (128) is the same for both sizes
    const int cta = a.np >= 16 ? 512 : 256;
    const size_t smem = (size_t)a.nv * 32 * ((2 * IntW<L>::W + 1) * sizeof(int32_t) + sizeof(float));
    // raise the kernel's dynamic shared-memory limit (per device) only when a
    // larger system needs more, not on every launch
    static size_t smem_set[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || smem > smem_set[dev]) {
      cudaFuncSetAttribute(evaldiff_intblk_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (dev >= 0 && dev < 64) smem_set[dev] = smem;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, evaldiff_intblk_kernel<L>, cta, smem);
    if (per_sm < 1) per_sm = 1;
    const int wpc = cta / 32;
    int64_t want = (a.v.npts + 31) / 32 * ((a.np + wpc - 1) / wpc);  // (point block, polynomial group) items
    int64_t grid = (int64_t)sm_count() * per_sm;
    if (grid > want) grid = want;
    evaldiff_intblk_kernel<L><<<(unsigned)grid, cta, smem, st>>>(a, cf, s->d_coef_lg);
  } else {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, evaldiff_int_kernel<L>, 128, 0);
    if (per_sm < 1) per_sm = 1;
    int64_t want = (a.n_units + 3) / 4;
    int64_t grid = (int64_t)sm_count() * per_sm;
    if (grid > want) grid = want;
    evaldiff_int_kernel<L><<<(unsigned)grid, 128, 0, st>>>(a, cf, s->d_coef_lg);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "ht_eval_diff: launch");
  return HT_OK;
}

template <int L>
int launch_evaldiff_l(const ht_system* s, int64_t n_pts, int j0, int j1, const double* x, double* val, double* jac,
                      cudaStream_t st) {
  EvalArgs a;
  a.v.mon_off = s->d_mon_off;
  a.v.pairs = s->d_pairs;
  a.v.coef = s->d_coef;
  a.v.x = x;
  a.v.npts = n_pts;
  a.poly_off = s->d_poly_off + j0;  // polynomials j0 .. j1 - 1, written from output row 0
  a.nv = s->nv;
  a.np = j1 - j0;
  a.val = val;
  a.jac = jac;
  a.n_units = ((n_pts + 31) / 32) * a.np;
  const int threads = s->eval_threads > 0 ? s->eval_threads : 128;
  if (s->eval_variant == 2 && s->d_coef_fz && s->nv <= kIntMaxVars && s->max_k <= 64)
    return launch_int<L>(a, s, threads, st);
  const bool loop = s->eval_variant != 0;  // default: compact bodies
  return loop ? launch_v<L, true>(a, threads, st) : launch_v<L, false>(a, threads, st);
}

#ifndef HT_LIMBS
#error "compile once per precision with -DHT_LIMBS=1, 2 or 4"
#endif
template int launch_evaldiff_l<HT_LIMBS>(const ht_system*, int64_t, int, int, const double*, double*, double*,
                                         cudaStream_t);

}  // namespace ht
