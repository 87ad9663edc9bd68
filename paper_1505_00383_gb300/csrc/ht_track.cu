// Many-path predictor-corrector tracking of gamma (1 - t) g(x) + t f(x) = 0
// (Section 2 of Verschelde & Yu 2015), with g_i = x_i^d_i - 1.
//
// Execution model.  A CTA serves a group of 32 paths (one per lane) with T
// warps; warp r is "team member" r for all 32 paths.  Every warp executes the
// same instruction stream for its 32 paths (the SIMT picture of Table
// tabsimtprecor), and the work of one Newton step is split over the T warps:
//   * evaluation: warp r evaluates the polynomials j = r, r + T, ...;
//   * modified Gram-Schmidt: warp r owns the columns j = r, r + T, ... of the
//     augmented matrix [J | -h]; the owner of column q normalises it, then
//     every warp projects its later columns (no cross-warp reductions: each
//     dot product runs down a whole column in one warp);
//   * prediction and the Newton update: warp r owns coordinates r, r + T, ...
// One kernel launch runs `iters` Newton steps of every path of its groups; a
// path's step (predict, 1..newton_max evaluate-correct rounds, accept or
// reject, step-size control) is a small state machine advanced once per Newton
// step, so lanes never wait for a predictor they do not need.  Between
// launches the active paths are compacted by the scan of Table tabjobidx;
// only the active count reaches the host.
//
// Per-path state lives in device memory in the vertical layout of Section 3
// ([entry][2][L][m], path index fastest) -- the "work space for multiple
// paths" of Table tabmemory.
#include "ht_eval.cuh"
#include "ht_int_row.cuh"
#include "ht_internal.h"
#include "ht_mpi_ops.cuh"
#include "ht_mlp.cuh"
#include "ht_track.h"

namespace ht {

enum : int8_t { PH_TRACK = 0, PH_POLISH = 1 };

// max over values that lets a NaN through (a NaN norm rejects the step)
__device__ __forceinline__ double nanmax(double m, double v) { return (v > m || v != v) ? v : m; }

template <int L>
__device__ __forceinline__ cx<L> root_of_unity(int d, int k) {
  if (d == 1 || k == 0) return creal<L>(1.0);
  if (2 * k == d) return creal<L>(-1.0);
  cx<L> z = czero<L>();
  if (4 * k == d) {
    z.im = r_from<L>(1.0);
    return z;
  }
  if (4 * k == 3 * d) {
    z.im = r_from<L>(-1.0);
    return z;
  }
  double th = 2.0 * 3.14159265358979323846 * (double)k / (double)d;
  double c, s;
  sincos(th, &s, &c);
  z.re = r_from<L>(c);
  z.im = r_from<L>(s);
  if constexpr (L > 1) {
    // Newton on z^d - 1: z <- z - (z^d - 1) / (d z^(d-1))
    for (int it = 0; it < 3; ++it) {
      cx<L> zd1 = creal<L>(1.0);
      for (int e = 0; e < d - 1; ++e) zd1 = cmul(zd1, z);
      cx<L> f = csub(cmul(zd1, z), creal<L>(1.0));
      cx<L> fp = cscale(zd1, (double)d);
      rl<L> den = cabs2(fp);
      cx<L> num = cconjmul(fp, f);
      rl<L> inv = r_div(r_from<L>(1.0), den);
      z = csub(z, cscale_r(num, inv));
    }
  }
  return z;
}

// Path q's start point: mixed-radix digits of first + q, variable 0 fastest.
template <int L>
__global__ void start_kernel(int n, const int32_t* __restrict__ deg, int64_t first, int64_t count,
                             double* __restrict__ x) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = first + q;
    for (int i = 0; i < n; ++i) {
      int d = __ldg(deg + i);
      int k = (int)(r % d);
      r /= d;
      st<L>(x, i, count, q, root_of_unity<L>(d, k));
    }
  }
}

// Features of a path at the start of a step, for the learned step-size
// proposer.  History values are read as hv(q) = hx[q * stride] with plane q
// of the history array ([cap][n][2][L]); t values as tv[j * tstride].
//   f0 t, f1 log10 h, f2 log10 |dx/dt|_inf / 4 (from the last two accepted
//   points, 0 with fewer), f3 log10 |dx| of the last round / 16, f4 log10 |h|
//   of the last round / 16, f5 rounds of the last step / newton_max, f6 last
//   step rejected, f7 history length / cap, f8 log10(1 - t) / 16,
//   f9 log10 |d2x/dt2|_inf / 8 (twice the second divided difference of the
//   last three accepted points, 0 with fewer), f10 log10(h / the last
//   accepted step) / 2 (0 with fewer than two points); each clamped to
//   [-4, 4]; f11..f15 zero.
template <int L>
__device__ __forceinline__ void step_features(float* f, double t, double h, int nh, int cap, int n,
                                              const double* tv, int64_t tstride, const double* hx, int64_t stride,
                                              double last_dx, double last_res, int last_its, int last_rej,
                                              int newton_max) {
  double dxdt = 0.0, d2 = 0.0, hr = 0.0;
  auto pt = [&](int s, int i, int c) { return hx[((((int64_t)s * n + i) * 2) * L + (int64_t)c * L) * stride]; };
  auto tt = [&](int s) { return tv[(int64_t)s * tstride]; };
  if (nh >= 2) {
    const double dt = tt(nh - 1) - tt(nh - 2);
    double mx = 0.0;
    for (int i = 0; i < n; ++i) {
      const double dr = pt(nh - 1, i, 0) - pt(nh - 2, i, 0);
      const double di = pt(nh - 1, i, 1) - pt(nh - 2, i, 1);
      mx = fmax(mx, sqrt(dr * dr + di * di));
    }
    dxdt = dt > 0.0 ? mx / dt : 0.0;
    hr = dt > 0.0 ? log10(h / dt) / 2.0 : 0.0;
  }
  if (nh >= 3) {
    const double t2 = tt(nh - 1), t1 = tt(nh - 2), t0 = tt(nh - 3);
    if (t2 > t1 && t1 > t0) {
      double mx = 0.0;
      for (int i = 0; i < n; ++i) {
        const double ar = (pt(nh - 1, i, 0) - pt(nh - 2, i, 0)) / (t2 - t1) - (pt(nh - 2, i, 0) - pt(nh - 3, i, 0)) / (t1 - t0);
        const double ai = (pt(nh - 1, i, 1) - pt(nh - 2, i, 1)) / (t2 - t1) - (pt(nh - 2, i, 1) - pt(nh - 3, i, 1)) / (t1 - t0);
        mx = fmax(mx, sqrt(ar * ar + ai * ai));
      }
      d2 = 2.0 * mx / (t2 - t0);
    }
  }
  double v[11] = {t,
                  log10(h),
                  log10(dxdt + 1e-30) / 4.0,
                  log10(last_dx + 1e-300) / 16.0,
                  log10(last_res + 1e-300) / 16.0,
                  (double)last_its / (double)newton_max,
                  (double)last_rej,
                  (double)nh / (double)cap,
                  log10(1.0 - t + 1e-16) / 16.0,
                  nh >= 3 ? log10(d2 + 1e-30) / 8.0 : 0.0,
                  hr};
  for (int i = 0; i < 11; ++i) f[i] = (float)fmin(4.0, fmax(-4.0, v[i]));
  for (int i = 11; i < FEAT; ++i) f[i] = 0.0f;
}

// Start points of selected paths: entry q is path first + ids[q].
template <int L>
__global__ void start_at_kernel(int n, const int32_t* __restrict__ deg, int64_t first, const int32_t* __restrict__ ids,
                                const int32_t* __restrict__ count, double* __restrict__ x, int64_t ld) {
  const int64_t cnt = *count;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < cnt; q += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = first + ids[q];
    for (int i = 0; i < n; ++i) {
      int d = __ldg(deg + i);
      int k = (int)(r % d);
      r /= d;
      st<L>(x, i, ld, q, root_of_unity<L>(d, k));
    }
  }
}

// Results of selected paths into the full arrays: path ids[q] of dst takes
// entry q of src (points [n][2][L][ld_src] and [n][2][L][m]).
template <int L>
__global__ void scatter_kernel(int n, const int32_t* __restrict__ ids, const int32_t* __restrict__ count,
                               const double* __restrict__ xs, const int8_t* __restrict__ ss,
                               const double* __restrict__ ts, int64_t ld_src, double* __restrict__ xd,
                               int8_t* __restrict__ sd, double* __restrict__ td, int64_t m) {
  const int64_t cnt = *count;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < cnt; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = ids[q];
    for (int i = 0; i < n; ++i) st<L>(xd, i, m, p, ld<L>(xs, i, ld_src, q));
    sd[p] = ss[q];
    td[p] = ts[q];
  }
}

template <int L>
__global__ void features_kernel(const double* __restrict__ rec, int64_t n_rec, int n, int cap, int newton_max,
                                float* __restrict__ feat) {
  const int64_t R = rec_size(n, L, cap);
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_rec; r += (int64_t)gridDim.x * blockDim.x) {
    const double* h = rec + r * R;
    step_features<L>(feat + r * FEAT, h[1], h[2], (int)h[3], cap, n, h + REC_HDR, 1, h + REC_HDR + cap, 1, h[4], h[5],
                     (int)h[6], (int)h[7], newton_max);
  }
}

template <int L>
__global__ void init_kernel(TrackArgs a) {
  const int cap = a.prm.max_order + 1;
  const int64_t R = rec_size(a.n, L, cap);
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.m; p += (int64_t)gridDim.x * blockDim.x) {
    if (a.init_rec) {  // resume from a recorded step start
      const double* r = a.init_rec + p * R;
      int nh = (int)r[3];
      nh = nh < 1 ? 1 : (nh > cap ? cap : nh);
      for (int s = 0; s < nh; ++s) {
        a.ht[(int64_t)s * a.m + p] = r[REC_HDR + s];
        for (int i = 0; i < a.n; ++i)
          for (int c = 0; c < 2 * L; ++c)
            a.hx[(((int64_t)s * a.n + i) * 2 * L + c) * a.m + p] = r[REC_HDR + cap + ((int64_t)s * a.n + i) * 2 * L + c];
      }
      for (int i = 0; i < a.n; ++i)
        for (int c = 0; c < 2 * L; ++c)
          a.x[((int64_t)i * 2 * L + c) * a.m + p] = r[REC_HDR + cap + ((int64_t)(nh - 1) * a.n + i) * 2 * L + c];
      a.t[p] = r[1];
      a.h[p] = r[2];
      a.nh[p] = (int8_t)nh;
      a.last_dx[p] = r[4];
      a.last_res[p] = r[5];
      a.last_its[p] = (int8_t)r[6];
      a.last_rej[p] = (int8_t)r[7];
    } else {
      if (a.x0) {  // the caller's start points, x0_limbs limbs each (missing limbs zero)
        for (int i = 0; i < a.n; ++i)
          for (int c = 0; c < 2; ++c)
            for (int l = 0; l < L; ++l)
              a.x[(((int64_t)i * 2 + c) * L + l) * a.m + p] =
                  l < a.x0_limbs ? a.x0[(((int64_t)i * 2 + c) * a.x0_limbs + l) * a.m + p] : 0.0;
      }
      for (int i = 0; i < a.n; ++i) st<L>(a.hx, i, a.m, p, ld<L>(a.x, i, a.m, p));
      a.ht[p] = a.polish_only ? 1.0 : 0.0;
      a.t[p] = a.polish_only ? 1.0 : 0.0;
      a.h[p] = a.prm.h0;
      a.nh[p] = 1;
      a.last_dx[p] = 0.0;
      a.last_res[p] = 0.0;
      a.last_its[p] = 0;
      a.last_rej[p] = 0;
    }
    a.t1[p] = 0.0;
    a.status[p] = 0;
    a.it[p] = 0;
    a.phase[p] = (a.polish_only && !a.init_rec) ? PH_POLISH : PH_TRACK;
    a.fallback[p] = 0;
    a.ntan[p] = 0;
    a.steps[p] = 0;
    a.rejects[p] = 0;
    a.newton[p] = 0;
    if (a.newton_out) a.newton_out[p] = 0;
    a.idx0[p] = (int32_t)p;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.count0 = (int32_t)a.m;
}

// Modified Gram-Schmidt least squares on the augmented matrix [A | b] of one
// path per lane (rows >= cols), columns dealt to the T warps of the CTA:
// for q: r_qq = |a_q|, q_q = a_q / r_qq; for j > q: r_qj = q_q^H a_j,
// a_j -= r_qj q_q; then back substitution R x = Q^H b.  A is
// [rows][cols + 1][2][L][m], R is [cols][cols + 1][2][L][m] (R[q][q] holds
// 1 / r_qq), x is [cols][2][L][m].  Every thread of the CTA must call this
// (it contains barriers); lanes with act == false only take the barriers.
// The three accumulations of MGS.  In double each is a chain of fused
// multiply-adds (4 FMAs for r + conj(a) b and for a - r q, 2 for s + |v|^2
// against 6, 6 and 3 instructions through the complex helpers); in DD and QD
// the helpers' fused two-term products.
template <int L>
__device__ __forceinline__ cx<L> acc_conj_mul(cx<L> r, const cx<L>& a, const cx<L>& b) {
  if constexpr (L == 1) {
    r.re = fma(a.re, b.re, r.re);
    r.re = fma(a.im, b.im, r.re);
    r.im = fma(a.re, b.im, r.im);
    r.im = fma(-a.im, b.re, r.im);
    return r;
  } else {
    return cadd(r, cconjmul(a, b));
  }
}
template <int L>
__device__ __forceinline__ cx<L> sub_mul(cx<L> a, const cx<L>& r, const cx<L>& q) {
  if constexpr (L == 1) {
    a.re = fma(-r.re, q.re, a.re);
    a.re = fma(r.im, q.im, a.re);
    a.im = fma(-r.re, q.im, a.im);
    a.im = fma(-r.im, q.re, a.im);
    return a;
  } else {
    return csub(a, cmul(r, q));
  }
}
template <int L>
__device__ __forceinline__ rl<L> acc_abs2(rl<L> s, const cx<L>& v) {
  if constexpr (L == 1) {
    return fma(v.im, v.im, fma(v.re, v.re, s));
  } else {
    return r_add(s, cabs2(v));
  }
}

// The warp that handles column j in the phase that projects on q_q: the
// pivot column q + 1 (which its warp also normalises) goes to warp
// wp = (q + 1) % T; with 4 or more warps the other columns go round-robin to
// the other T - 1 warps, so the pivot's normalisation is not stacked on a
// second projection; with fewer warps they go round-robin to all, starting
// after wp.
__device__ __forceinline__ int mgs_col_warp(int j, int q, int T) {
  const int wp = (q + 1) % T;
  if (j == q + 1) return wp;
  const int k = j - q - 2;  // index among the other columns
  return T >= 4 ? (wp + 1 + k % (T - 1)) % T : (wp + 1 + k) % T;
}

template <int L>
__device__ void mgs_team(double* A, double* R, double* x, int rows, int cols, int64_t m, int64_t p, bool act,
                         int warp, int T, int nrhs = 1, double* x2 = nullptr) {
  const int W = cols + nrhs;
  // normalise column q (its squared norm given): a_q <- a_q / r_qq, R[q][q] = 1 / r_qq
  auto normalise = [&](int q, rl<L> nrm) {
    rl<L> rqq = r_sqrt(nrm);
    rl<L> inv = r_div(r_from<L>(1.0), rqq);
    for (int i = 0; i < rows; ++i) {
      int64_t e = (int64_t)i * W + q;
      st<L>(A, e, m, p, cscale_r(ld<L>(A, e, m, p), inv));
    }
    cx<L> rv = czero<L>();
    rv.re = inv;
    st<L>(R, (int64_t)q * W + q, m, p, rv);
  };
  if (warp == 0 && act) {  // column 0 by its owner
    rl<L> s = r_from<L>(0.0);
    for (int i = 0; i < rows; ++i) s = acc_abs2<L>(s, ld<L>(A, (int64_t)i * W, m, p));
    normalise(0, s);
  }
  __syncthreads();
  // Look-ahead: in the phase that projects the later columns on q_q, the
  // warp of column q + 1 projects it and normalises it at once, while the
  // other warps project the other columns (mgs_col_warp); one barrier per
  // column.  Every column sees the same operations in the same order as
  // without look-ahead.
  for (int q = 0; q < cols; ++q) {
    for (int j = q + 1; j < W; ++j) {
      if (!act || mgs_col_warp(j, q, T) != warp) continue;
      cx<L> r = czero<L>();
      for (int i = 0; i < rows; ++i)
        r = acc_conj_mul<L>(r, ld<L>(A, (int64_t)i * W + q, m, p), ld<L>(A, (int64_t)i * W + j, m, p));
      st<L>(R, (int64_t)q * W + j, m, p, r);
      rl<L> s = r_from<L>(0.0);
      for (int i = 0; i < rows; ++i) {
        int64_t e = (int64_t)i * W + j;
        cx<L> v = sub_mul<L>(ld<L>(A, e, m, p), r, ld<L>(A, (int64_t)i * W + q, m, p));
        st<L>(A, e, m, p, v);
        if (j == q + 1) s = acc_abs2<L>(s, v);
      }
      if (j == q + 1 && j < cols) normalise(j, s);  // the next pivot column, ready for the next phase
    }
    __syncthreads();
  }
  // back substitution, the right-hand sides dealt to the warps (the second
  // solves into x2)
  for (int k = warp; act && k < nrhs; k += T) {
    double* xs = k == 0 ? x : x2;
    for (int q = cols - 1; q >= 0; --q) {
      cx<L> acc = ld<L>(R, (int64_t)q * W + cols + k, m, p);
      for (int j = q + 1; j < cols; ++j) acc = sub_mul<L>(acc, ld<L>(R, (int64_t)q * W + j, m, p), ld<L>(xs, j, m, p));
      st<L>(xs, q, m, p, cscale_r(acc, ld<L>(R, (int64_t)q * W + q, m, p).re));
    }
  }
  __syncthreads();
}

// The same least squares on the integer pipe (DD, QD): entries are read as
// limb strings (from stored limb strings, or by exact conversion of stored
// doubles), every dot product and norm is one exact fixed-point sum of its
// products rounded once, 1/r_qq comes from Newton's iteration for 1/sqrt, and
// results are stored back in the same form; the solution is stored as
// doubles.  The column owner loads and normalises column q; the other warps
// reload it after the barrier.  Layouts and R's diagonal (1/r_qq) as above.
template <int L>
__device__ __forceinline__ mpi::fz<IntW<L>::W> ldz(const double* base, int64_t e, int64_t m, int64_t p) {
  const double* q = base + (e * 2) * L * m + p;
  double re[L], im[L];
#pragma unroll
  for (int l = 0; l < L; ++l) {
    re[l] = q[l * m];
    im[l] = q[(L + l) * m];
  }
  return mpi::from_doubles<IntW<L>::W, L>(re, im);
}
template <int L>
__device__ __forceinline__ void stz(double* base, int64_t e, int64_t m, int64_t p, const mpi::fz<IntW<L>::W>& z) {
  double* q = base + (e * 2) * L * m + p;
  double re[L], im[L];
  mpi::to_doubles<IntW<L>::W, L>(z, re, im);
#pragma unroll
  for (int l = 0; l < L; ++l) {
    q[l * m] = re[l];
    q[(L + l) * m] = im[l];
  }
}

// Storage of A and R for the integer least squares: the vertical doubles
// (converted on every load and store) or limb strings in [entry][2W+1][m]
// int32 words (exponent, re limbs, im limbs; loaded and stored as they are).
template <int L>
struct DblStore {
  double* base;
  int64_t m, p;
  __device__ __forceinline__ mpi::fz<IntW<L>::W> ld(int64_t e) const { return ldz<L>(base, e, m, p); }
  __device__ __forceinline__ void st(int64_t e, const mpi::fz<IntW<L>::W>& z) const { stz<L>(base, e, m, p, z); }
};
template <int L>
struct FzStore {
  static constexpr int W = IntW<L>::W;
  int32_t* base;
  int64_t m, p;
  __device__ __forceinline__ mpi::fz<W> ld(int64_t e) const {
    const int32_t* q = base + e * (2 * W + 1) * m + p;
    mpi::fz<W> z;
    z.f = q[0];
#pragma unroll
    for (int k = 0; k < W; ++k) {
      z.r[k] = q[(1 + k) * m];
      z.i[k] = q[(1 + W + k) * m];
    }
    return z;
  }
  __device__ __forceinline__ void st(int64_t e, const mpi::fz<W>& z) const {
    int32_t* q = base + e * (2 * W + 1) * m + p;
    q[0] = z.f;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      q[(1 + k) * m] = z.r[k];
      q[(1 + W + k) * m] = z.i[k];
    }
  }
};

template <int L, int N, class ST>
__device__ void mgs_team_int(const ST& A, const ST& R, double* x, int rows, int cols, int64_t m, int64_t p, bool act,
                             int warp, int T, int nrhs = 1, double* x2 = nullptr) {
  constexpr int W = IntW<L>::W;  // rows <= N
  using Z = mpi::fz<W>;
  const int Wc = cols + nrhs;
  Z Q[N], col[N], S[N + 1];
  // normalise the column held in v[] as column q: stored scaled by 1/r_qq, R[q][q] = 1/r_qq
  auto normalise = [&](int q, Z* v) {
    const Z nrm = mpi::norm2<W, N>(v, rows, S);
    const Z inv = mpi::inv_sqrt<W>(nrm, mpi::inv_sqrt_steps<W>());
    for (int i = 0; i < rows; ++i) A.st((int64_t)i * Wc + q, mpi::mul<W>(v[i], inv));
    R.st((int64_t)q * Wc + q, inv);
  };
  if (warp == 0 && act) {  // column 0 by its owner
    for (int i = 0; i < rows; ++i) Q[i] = A.ld((int64_t)i * Wc);
    normalise(0, Q);
  }
  __syncthreads();
  // Look-ahead as in mgs_team: the warp of column q + 1 projects it and
  // normalises it at once, the other columns go to the other warps; one
  // barrier per column.
  for (int q = 0; q < cols; ++q) {
    bool any = false;  // this warp has a column in this phase
    for (int j = q + 1; j < Wc; ++j) any = any || mgs_col_warp(j, q, T) == warp;
    if (act && any) {
      for (int i = 0; i < rows; ++i) Q[i] = A.ld((int64_t)i * Wc + q);
      for (int j = q + 1; j < Wc; ++j) {
        if (mgs_col_warp(j, q, T) != warp) continue;
        for (int i = 0; i < rows; ++i) col[i] = A.ld((int64_t)i * Wc + j);
        const Z r = mpi::dot_conj<W, N>(Q, col, rows, S);
        R.st((int64_t)q * Wc + j, r);
        mpi::sub_scaled<W>(col, r, Q, rows);
        for (int i = 0; i < rows; ++i) A.st((int64_t)i * Wc + j, col[i]);
        if (j == q + 1 && j < cols) {
          // the pivot column from its stored values, as the owner's reload
          // would give (for stored doubles the limb strings of the doubles
          // just written; stored limb strings come back as they were)
          for (int i = 0; i < rows; ++i) col[i] = A.ld((int64_t)i * Wc + j);
          normalise(j, col);
        }
      }
    }
    __syncthreads();
  }
  // back substitution, the right-hand sides dealt to the warps, solution in col[]
  for (int r = warp; act && r < nrhs; r += T) {
    for (int q = cols - 1; q >= 0; --q) {
      int k = 0;
      S[k++] = R.ld((int64_t)q * Wc + cols + r);
      for (int j = q + 1; j < cols; ++j) S[k++] = mpi::mul<W>(R.ld((int64_t)q * Wc + j), col[j]);
      col[q] = mpi::mul<W>(mpi::first_minus_rest<W, N + 1>(S, k), R.ld((int64_t)q * Wc + q));
    }
    double* xs = r == 0 ? x : x2;
    for (int q = 0; q < cols; ++q) stz<L>(xs, q, m, p, col[q]);
  }
  __syncthreads();
}

// Standalone batched least squares (one system per lane, one warp per CTA).
template <int L, bool INT>
__global__ void __launch_bounds__(32) mgs_kernel(double* A, double* R, double* x, int rows, int cols, int64_t n_sys) {
  int64_t p = (int64_t)blockIdx.x * 32 + threadIdx.x;
  if constexpr (INT)
    mgs_team_int<L, kIntMaxVars>(DblStore<L>{A, n_sys, p}, DblStore<L>{R, n_sys, p}, x, rows, cols, n_sys, p,
                                 p < n_sys, 0, 1);
  else
    mgs_team<L>(A, R, x, rows, cols, n_sys, p, p < n_sys, 0, 1);
}

// The learned proposal for the paths of one warp (all 32 lanes call it; want
// marks the lanes whose path starts a learned step): features, the network
// on the tensor cores, and h e^rho clamped.  Out of line so that the
// network's registers do not weigh on the Newton rounds' allocation.
template <int L>
__device__ __noinline__ double learned_step(const TrackArgs& a, MlpWarpSmem& stage, bool want, int64_t p, double t,
                                            double h, int nh, int cap, double* alpha) {
  float f[FEAT];
  if (want)
    step_features<L>(f, t, h, nh, cap, a.n, a.ht + p, a.m, a.hx + p, a.m, a.last_dx[p], a.last_res[p],
                     (int)a.last_its[p], (int)a.last_rej[p], a.prm.newton_max);
  else
    for (int i = 0; i < FEAT; ++i) f[i] = 0.0f;
  float y[2];
  mlp_forward_warp(*static_cast<const MlpSmem*>(a.mlp_img), stage, f, y);
  double hs = h;
  *alpha = 0.0;
  if (want) {
    const double rho = fmin(a.rho_max, fmax(a.rho_min, (double)y[0]));
    hs = fmin(a.prm.h_max, fmax(a.prm.h_min, h * exp(rho)));
    if (a.alpha_max > 0.0) *alpha = fmin(a.alpha_max, fmax(-a.alpha_max, (double)y[1]));
  }
  return hs;
}

// One Newton step (plus the bookkeeping around it) for `iters` rounds.
// LEARN: at every step start warp 0 evaluates the step-size network for its 32
// paths on the tensor cores and scales the step (see ht_track_paths_ex).
// Largest n for which DD/QD tracking runs on the integer pipe (local arrays
// of the evaluation and of MGS are sized by it).
constexpr int kIntMaxTrack = 32;

// An L-limb complex as a limb string (exact).
template <int L>
__device__ __forceinline__ mpi::fz<IntW<L>::W> fz_of(const cx<L>& z) {
  double re[L], im[L];
#pragma unroll
  for (int l = 0; l < L; ++l) {
    re[l] = r_limb(z.re, l);
    im[l] = r_limb(z.im, l);
  }
  return mpi::from_doubles<IntW<L>::W, L>(re, im);
}
template <int L>
__device__ __forceinline__ cx<L> cx_from(const double* re, const double* im) {
  if constexpr (L == 1) {
    return cx<1>{re[0], im[0]};
  } else if constexpr (L == 2) {
    return cx<2>{dd{re[0], re[1]}, dd{im[0], im[1]}};
  } else {
    return cx<4>{qd{{re[0], re[1], re[2], re[3]}}, qd{{im[0], im[1], im[2], im[3]}}};
  }
}

// INT: f and its Jacobian rows on the integer pipe (int_row: exact sums in
// per-output fixed-point frames), the rest of the round in FP64 arithmetic.
// MAXT: the largest team (8, or 16 for the wide instantiation that serves
// few groups of double and double-double paths with more warps each, and
// any group when the autotuner picks 16).
template <int L, bool LEARN, bool INT, int MAXT = 8>
__global__ void __launch_bounds__(32 * MAXT, MAXT > 8 ? 1 : (L == 1 ? 3 : (L == 2 ? 2 : 1))) track_kernel(TrackArgs a) {
  __shared__ double red[4][MAXT][32];  // per-warp partials: residual, update, point norms; finiteness
  __shared__ double sh_h[32];       // learned step of each lane's path
  __shared__ double sh_alpha[32];   // learned tangent correction of each lane's path
  __shared__ long long sh_slot[32]; // trace record slot of each lane's path (-1: none)
  __shared__ double sh_w[L > 1 ? 8 : 1][L][32];  // extrapolation weights (DD, QD), [point][limb][lane]
  // The network's weights are read from the device image (L1/L2): staging
  // them in shared memory would enlarge the shared-memory carveout and take
  // L1 capacity from the Newton workspace.  Only warp 0's sample staging
  // lives in shared memory.
  __shared__ MlpWarpSmem mlp_stage;
  // INT: the group's converted working points ([n][2W+1][32] words, then
  // [n][32] log2 moduli), dynamic shared memory sized by the launcher
  extern __shared__ __align__(16) int32_t xs_int[];
  float* lgs_int = reinterpret_cast<float*>(xs_int + (int64_t)a.n * (2 * IntW<L>::W + 1) * 32);
  const int cap = a.prm.max_order + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, T = blockDim.x >> 5;
  // the tangent predictors solve J v = -dh/dt as a second right-hand side
  const int pmode = a.prm.predictor, nrhs = pmode > 0 ? 2 : 1;
  const int n = a.n, W = n + nrhs;
  const int64_t m = a.m;
  const int count = *a.count_in;
  const int64_t rowA = (int64_t)W * 2 * L * m;  // doubles per row of A
  // DD and QD with integer evaluation keep A and R as limb strings
  // ([entry][2W+1][m] words) from the evaluation through the least squares:
  // no conversions
  constexpr bool FZ = INT && L >= 2;
  const int64_t rowZ = (int64_t)W * (2 * IntW<L>::W + 1) * m;  // words per row of A
  PolyView v;
  v.mon_off = a.mon_off;
  v.pairs = a.pairs;
  v.coef = a.coef;
  v.x = a.xp;
  v.npts = m;
  const cx<L> gamma = [&] {
    cx<L> g = czero<L>();
    g.re = r_from<L>(a.gamma_re);
    g.im = r_from<L>(a.gamma_im);
    return g;
  }();
  // Groups of 32 active paths are taken from a queue (one counter per
  // launch, zeroed by the compaction before it): a CTA whose groups finish
  // early takes more, instead of a fixed share of them.
  __shared__ int sh_group;
  for (;;) {
    if (threadIdx.x == 0) sh_group = atomicAdd(a.queue, 1);
    __syncthreads();
    const int64_t g = sh_group;
    __syncthreads();  // every thread has read the group before the next take
    if (g * 32 >= count) break;
    const int64_t slot = g * 32 + lane;
    const int64_t p = slot < count ? a.idx_in[slot] : -1;
    for (int iter = 0; iter < a.iters; ++iter) {
      int8_t stt = p >= 0 ? a.status[p] : (int8_t)1;
      const bool act = stt == 0;
      const int8_t ph = act ? a.phase[p] : (int8_t)0;
      int it = act ? a.it[p] : 0;
      double t = act ? a.t[p] : 0.0, h = act ? a.h[p] : 0.0, t1 = act ? a.t1[p] : 0.0;
      int nh = act ? a.nh[p] : 1;
      int ntan = act && pmode > 0 ? a.ntan[p] : 0;
      int fb = act ? a.fallback[p] : 0;
      double alpha = 0.0;  // tangent correction of a learned step (0: the plain predictor)
      const bool start = act && ph == PH_TRACK && it == 0;
      // ---- A0: record the step start, propose a learned step
      if (a.trace) {
        if (warp == 0) {
          long long slot = -1;
          if (start && a.steps[p] % a.trace_stride == 0) {
            slot = (long long)atomicAdd(a.trace_count, 1ULL);
            if (slot >= a.trace_cap) slot = -1;
          }
          sh_slot[lane] = slot;
          if (slot >= 0) {
            double* r = a.trace + slot * rec_size(n, L, cap);
            r[0] = (double)p;
            r[1] = t;
            r[2] = h;
            r[3] = (double)nh;
            r[4] = a.last_dx[p];
            r[5] = a.last_res[p];
            r[6] = (double)a.last_its[p];
            r[7] = (double)a.last_rej[p];
            for (int k = 8; k < REC_HDR; ++k) r[k] = 0.0;
            for (int s2 = 0; s2 < cap; ++s2) r[REC_HDR + s2] = s2 < nh ? a.ht[(int64_t)s2 * m + p] : 0.0;
          }
        }
        __syncthreads();
        const long long slot = sh_slot[lane];
        if (slot >= 0) {
          double* r = a.trace + slot * rec_size(n, L, cap) + REC_HDR + cap;
          for (int s2 = 0; s2 < cap; ++s2)
            for (int i = warp; i < n; i += T)
              for (int c = 0; c < 2 * L; ++c)
                r[((int64_t)s2 * n + i) * 2 * L + c] =
                    s2 < nh ? a.hx[(((int64_t)s2 * n + i) * 2 * L + c) * m + p] : 0.0;
        }
      }
      if constexpr (LEARN) {
        // warp 0 runs the network only in rounds where one of its paths
        // starts a learned step (about one round in three)
        if (warp == 0 && __any_sync(0xffffffffu, start && fb == 0))
          sh_h[lane] = learned_step<L>(a, mlp_stage, start && fb == 0, p, t, h, nh, cap, &sh_alpha[lane]);
        __syncthreads();
        if (start && fb == 0) {
          h = sh_h[lane];
          alpha = sh_alpha[lane];
          fb = -1;  // this step is a learned one
        }
      }
      // ---- A: predictor (first Newton round of a step) or polish copy
      // The extrapolation weights (a product and a QD division per history
      // point) are dealt to the warps, one point each, and shared through
      // shared memory: every warp used to compute all of them, contending
      // for the FP64 pipe.  Each weight is the same sequence of operations
      // as before, so the predicted points are bitwise unchanged.
      const bool herm = start && pmode == 2 && ntan >= 2 && nh >= 2;
      const bool euler = start && !herm && pmode >= 1 && ntan >= 1;
      const int mm = !start ? 0 : ((herm || euler) ? 0 : (pmode >= 1 ? 1 : min(nh, a.prm.max_order + 1)));
      const int base = nh - mm;
      // weight of history point j (Lagrange, at t1)
      auto weight = [&](int j) {
        rl<L> num = r_from<L>(1.0), den = r_from<L>(1.0);
        double tj = a.ht[(int64_t)(base + j) * m + p];
        for (int i = 0; i < mm; ++i) {
          if (i == j) continue;
          double ti = a.ht[(int64_t)(base + i) * m + p];
          num = r_mul(num, r_diff<L>(t1, ti));
          den = r_mul(den, r_diff<L>(tj, ti));
        }
        return r_div(num, den);
      };
      if (start) {
        double step = fmin(h, 1.0 - t);
        t1 = (step >= 1.0 - t) ? 1.0 : t + step;
        if constexpr (L > 1) {
          for (int j = warp; j < mm; j += T) {
            const rl<L> wj = weight(j);
#pragma unroll
            for (int l = 0; l < L; ++l) sh_w[j][l][lane] = r_limb(wj, l);
          }
        }
      }
      // (in double a weight is a few instructions: every warp computes them,
      // without the barrier)
      if constexpr (L > 1) __syncthreads();
      if (start) {
        // tangent predictors: cubic Hermite on the last two points and their
        // tangents, Euler on the last one; until a tangent exists, x itself
        rl<L> ca = r_from<L>(0.0), cb = r_from<L>(0.0), cc = r_from<L>(0.0), cd = r_from<L>(0.0);
        if (herm) {  // x0, v0 at s0 = ht[nh-2]; x1, v1 at s1 = ht[nh-1]
          const double s0 = a.ht[(int64_t)(nh - 2) * m + p], s1 = a.ht[(int64_t)(nh - 1) * m + p];
          const rl<L> d = r_diff<L>(s1, s0), u = r_div(r_diff<L>(t1, s0), d);
          const rl<L> u2 = r_mul(u, u), u3 = r_mul(u2, u);
          const rl<L> two = r_from<L>(2.0), three = r_from<L>(3.0);
          ca = r_add(r_sub(r_mul(two, u3), r_mul(three, u2)), r_from<L>(1.0));  // weight of x0
          cb = r_mul(r_add(r_sub(u3, r_mul(two, u2)), u), d);                  // of v0
          cc = r_sub(r_mul(three, u2), r_mul(two, u3));                        // of x1
          cd = r_mul(r_sub(u3, u2), d);                                        // of v1
        } else if (euler) {
          cd = r_diff<L>(t1, a.ht[(int64_t)(nh - 1) * m + p]);
        }
        rl<L> w[8];
        for (int j = 0; j < mm; ++j) {
          if constexpr (L > 1) {
            double wl[L];
#pragma unroll
            for (int l = 0; l < L; ++l) wl[l] = sh_w[j][l][lane];
            w[j] = r_of<L>(wl);
          } else {
            w[j] = weight(j);
          }
        }
        for (int i = warp; i < n; i += T) {
          cx<L> acc = czero<L>();
          bool fz_done = false;
          if constexpr (FZ && L == 4) {
            // QD extrapolation on the integer pipe: the history points times
            // their weights as limb-string products, summed exactly and
            // rounded once (a QD complex-by-real product on the FP64 pipe is
            // about 200 FP64 instructions)
            if (!herm && !euler && mm > 0) {
              constexpr int WZ = IntW<L>::W;
              const double zero4[4] = {0.0, 0.0, 0.0, 0.0};
              mpi::fz<WZ> terms[8];
              int ones[8];
              for (int j = 0; j < mm; ++j) {
                const mpi::fz<WZ> wz = mpi::from_doubles<WZ, 4>(w[j].x, zero4);
                terms[j] = mpi::mul<WZ>(fz_of<L>(ld<L>(a.hx, (int64_t)(base + j) * n + i, m, p)), wz);
                ones[j] = 1;
              }
              double re[4], im[4];
              mpi::to_doubles<WZ, 4>(mpi::sum<WZ, 8>(terms, ones, mm), re, im);
              acc = cx_from<L>(re, im);
              fz_done = true;
            }
          }
          if (!fz_done)
            for (int j = 0; j < mm; ++j)
              acc = cadd(acc, cscale_r(ld<L>(a.hx, (int64_t)(base + j) * n + i, m, p), w[j]));
          if (herm) {
            acc = cscale_r(ld<L>(a.hx, (int64_t)(nh - 2) * n + i, m, p), ca);
            acc = cadd(acc, cscale_r(ld<L>(a.tx, (int64_t)(nh - 2) * n + i, m, p), cb));
            acc = cadd(acc, cscale_r(ld<L>(a.hx, (int64_t)(nh - 1) * n + i, m, p), cc));
            acc = cadd(acc, cscale_r(ld<L>(a.tx, (int64_t)(nh - 1) * n + i, m, p), cd));
          } else if (euler) {
            acc = cadd(ld<L>(a.hx, (int64_t)(nh - 1) * n + i, m, p),
                       cscale_r(ld<L>(a.tx, (int64_t)(nh - 1) * n + i, m, p), cd));
          }
          if (alpha != 0.0) {  // learned tangent correction: x + (1 + alpha)(pred - x)
            const cx<L> xc = ld<L>(a.hx, (int64_t)(nh - 1) * n + i, m, p);
            acc = cadd(xc, cscale_r(csub(acc, xc), r_from<L>(1.0 + alpha)));
          }
          st<L>(a.xp, i, m, p, acc);
        }
      } else if (act && ph == PH_POLISH) {
        for (int i = warp; i < n; i += T) st<L>(a.xp, i, m, p, ld<L>(a.x, i, m, p));
      }
      const double tt = (ph == PH_POLISH) ? 1.0 : t1;
      __syncthreads();
      // ---- B: h(x, tt) = gamma (1 - tt) (x_j^d_j - 1) + tt f_j(x), Jacobian rows
      double pres = 0.0;
      using Z = mpi::fz<IntW<L>::W>;
      if constexpr (INT) {
        // the group's working points, converted once into shared memory
        // (warps take the coordinates round-robin; lanes without an active
        // path store zeros), read by every warp's polynomials
        for (int i = warp; i < n; i += T) {
          double re[L], im[L];
#pragma unroll
          for (int l = 0; l < L; ++l) {
            re[l] = act ? a.xp[((int64_t)(i * 2) * L + l) * m + p] : 0.0;
            im[l] = act ? a.xp[((int64_t)(i * 2 + 1) * L + l) * m + p] : 0.0;
          }
          store_point<L>(xs_int, i, lane, mpi::from_doubles<IntW<L>::W, L>(re, im));
          lgs_int[i * 32 + lane] = mpi::log2_mod(re[0], im[0]);
        }
        __syncthreads();
      }
      if constexpr (FZ) {
       if (act) {
        // DD and QD on the integer pipe throughout: the row, the start
        // system's terms and the homotopy in limb-string arithmetic (a QD
        // complex product on the FP64 pipe costs about 30 times a limb-string
        // one)
        using ZW = mpi::fz<IntW<L>::W>;
        constexpr int WZ = IntW<L>::W;
        mpi::fzs<IntW<L>::W> P[INT ? kIntMaxTrack : 1];
        const SmemPoints<L> X{xs_int, lane};
        const SmemLog lg{lgs_int, lane};
        const ZW gz = fz_of<L>(gamma);
        const ZW gsz = fz_of<L>(cscale_r(gamma, r_diff<L>(1.0, tt)));  // gamma (1 - tt)
        const ZW ttz = mpi::from_real<WZ>(tt), one = mpi::from_real<WZ>(1.0);
        for (int j = warp; j < n; j += T) {
          const FzStore<L> Zrow{reinterpret_cast<int32_t*>(a.A) + (int64_t)j * rowZ, m, p};
          double vre[L], vim[L];
          // the row comes out as tt times the gradient, scaled in the exact
          // fixed-point sums, as the limb strings the least squares reads
          int_row_fz<L>(a.mon_off, a.pairs, static_cast<const Z*>(a.cfz), a.clg, __ldg(a.poly_off + j),
                        __ldg(a.poly_off + j + 1), X, lg, n, Zrow.base, m, p, vre, vim, P, tt);
          const ZW fj = mpi::from_doubles<WZ, L>(vre, vim);
          const int d = __ldg(a.deg + j);
          const ZW xj = X[j];
          ZW xd1 = one;  // x_j^(d-1)
          for (int e = 0; e < d - 1; ++e) xd1 = e == 0 ? xj : mpi::mul<WZ>(xd1, xj);
          const ZW gval = mpi::sub<WZ>(mpi::mul<WZ>(xd1, xj), one);  // x_j^d - 1
          ZW t2[2] = {mpi::mul<WZ>(gsz, gval), mpi::mul<WZ>(ttz, fj)};
          const int e_add[2] = {1, 1}, e_neg[2] = {-1, -1};
          const ZW hj = mpi::sum<WZ, 2>(t2, e_add, 2);
          const ZW mh = mpi::sum<WZ, 2>(t2, e_neg, 2);
          const int e_d[1] = {d};
          const ZW dg = mpi::mul<WZ>(gsz, mpi::sum<WZ, 1>(&xd1, e_d, 1));  // gamma (1 - tt) d x_j^(d-1)
          Zrow.st(j, mpi::add<WZ>(Zrow.ld(j), dg));
          Zrow.st(n, mh);
          if (nrhs == 2) Zrow.st(n + 1, mpi::sub<WZ>(mpi::mul<WZ>(gz, gval), fj));  // -dh/dt = gamma g - f
          // the residual's modulus from its leading limb; a non-finite
          // coordinate (which limb strings cannot carry) makes it NaN
          double hr, hi;
          mpi::to_doubles<WZ, 1>(hj, &hr, &hi);
          const bool fin = cfinite(ld<L>(a.xp, j, m, p)) && isfinite(hr) && isfinite(hi);
          pres = nanmax(pres, fin ? __dsqrt_rn(__dadd_rn(__dmul_rn(hr, hr), __dmul_rn(hi, hi)))
                                  : __longlong_as_double(0x7ff8000000000000LL));
        }
       }
      } else if (act) {
        cx<L> gs = cscale_r(gamma, r_diff<L>(1.0, tt));
        mpi::fzs<IntW<L>::W> P[INT ? kIntMaxTrack : 1];
        const SmemPoints<L> X{xs_int, lane};
        const SmemLog lg{lgs_int, lane};
        for (int j = warp; j < n; j += T) {
          double* Arow = a.A + (int64_t)j * rowA;
          cx<L> fj;
          if constexpr (INT) {
            double vre[L], vim[L];
            // the row comes out as tt times the gradient, scaled in the
            // exact fixed-point sums (one rounding, no FP64 multiplies)
            int_row<L>(a.mon_off, a.pairs, static_cast<const Z*>(a.cfz), a.clg, __ldg(a.poly_off + j),
                       __ldg(a.poly_off + j + 1), X, lg, n, Arow, m, p, vre, vim, P, tt);
            fj = cx_from<L>(vre, vim);
          } else {
            fj = eval_poly<L>(v, __ldg(a.poly_off + j), __ldg(a.poly_off + j + 1), n, p, Arow);
            for (int i = 0; i < n; ++i) st<L>(Arow, i, m, p, cscale(ld<L>(Arow, i, m, p), tt));
          }
          const int d = __ldg(a.deg + j);
          cx<L> xj = ld<L>(a.xp, j, m, p);
          cx<L> xd1 = creal<L>(1.0);
          for (int e = 0; e < d - 1; ++e) xd1 = cmul(xd1, xj);
          cx<L> gval = csub(cmul(xd1, xj), creal<L>(1.0));
          cx<L> hj = cadd(cmul(gs, gval), cscale(fj, tt));
          cx<L> dg = cmul(gs, cscale(xd1, (double)d));
          st<L>(Arow, j, m, p, cadd(ld<L>(Arow, j, m, p), dg));
          cx<L> mh = czero<L>();
          mh = csub(mh, hj);
          st<L>(Arow, n, m, p, mh);
          if (nrhs == 2) st<L>(Arow, n + 1, m, p, csub(cmul(gamma, gval), fj));  // -dh/dt = gamma g - f
          pres = nanmax(pres, cfinite(hj) ? cabs_lead(hj) : __longlong_as_double(0x7ff8000000000000LL));
        }
      }
      __syncthreads();
      // ---- C: least squares J dx = -h by modified Gram-Schmidt
      // DD and QD with integer evaluation solve on the integer pipe, on the
      // limb strings in A and R (for DD the FP64 MGS had been faster while
      // every load and store converted: 1.6 s against 3.1 s for the n = 12,
      // 4,096-path run; without conversions the integer path takes 1.08 s
      // against 1.43 s)
      if constexpr (FZ)
        mgs_team_int<L, kIntMaxTrack>(FzStore<L>{reinterpret_cast<int32_t*>(a.A), m, p},
                                      FzStore<L>{reinterpret_cast<int32_t*>(a.R), m, p}, a.dx, n, n, m, p, act, warp,
                                      T, nrhs, a.tdx);
      else
        mgs_team<L>(a.A, a.R, a.dx, n, n, m, p, act, warp, T, nrhs, a.tdx);
      // ---- D: x <- x + dx on this warp's coordinates; partial norms
      double pdx = 0.0, pxp = 0.0;
      if (act) {
        for (int i = warp; i < n; i += T) {
          cx<L> d = ld<L>(a.dx, i, m, p);
          cx<L> xn = cadd(ld<L>(a.xp, i, m, p), d);
          st<L>(a.xp, i, m, p, xn);
          pdx = nanmax(pdx, cfinite(d) ? cabs_lead(d) : __longlong_as_double(0x7ff8000000000000LL));
          pxp = nanmax(pxp, cabs_lead(xn));
        }
      }
      red[0][warp][lane] = pres;
      red[1][warp][lane] = pdx;
      red[2][warp][lane] = pxp;
      __syncthreads();
      double nres = 0.0, ndx = 0.0, nxp = 0.0;
      for (int w = 0; w < T; ++w) {
        nres = nanmax(nres, red[0][w][lane]);
        ndx = nanmax(ndx, red[1][w][lane]);
        nxp = nanmax(nxp, red[2][w][lane]);
      }
      // ---- E: the state machine of a step (identical in every warp)
      bool accept_point = false;  // copy xp into x (and maybe history)
      bool push_hist = false;
      bool step_end = false;
      int last_its_v = 0, last_rej_v = 0;
      int newton = 0, steps = 0, rejects = 0;
      if (act) {
        newton = a.newton[p] + 1;
        steps = a.steps[p];
        rejects = a.rejects[p];
        const bool nan = !(ndx == ndx);
        if (ph == PH_TRACK) {
          ++it;
          bool ok = false;
          if (!nan) {
            double sx = fmax(1.0, nxp);
            double lim = a.prm.tol_res;
            for (int e = 0; e < a.prm.deg_max; ++e) lim = __dmul_rn(lim, sx);
            ok = ndx <= a.prm.tol_dx * sx && nres <= lim;
          }
          if (ok || nan || it >= a.prm.newton_max) {  // the step ends here
            ++steps;
            last_its_v = it;
            last_rej_v = ok ? 0 : 1;
            step_end = true;
            if (fb == -1)
              fb = ok ? 0 : a.fallback_steps;
            else if (fb > 0)
              --fb;
            it = 0;
            if (ok) {
              t = t1;
              accept_point = true;
              push_hist = true;
              h = fmin(a.prm.h_max, a.prm.f_up * h);
              if (nxp > a.prm.r_div) {
                stt = -2;
              } else if (t == 1.0) {
                if (a.prm.polish_max > 0) {
                  // polish at t = 1 in the following rounds
                } else {
                  stt = 1;
                }
              }
            } else {
              ++rejects;
              h = a.prm.f_down * h;
              if (h < a.prm.h_min) stt = -1;
            }
            if (stt == 0 && steps >= a.prm.max_steps && !(ok && t == 1.0)) stt = -1;
          }
        } else {  // polish round at t = 1
          if (nan) {
            stt = 2;  // finished: status decided below from x
          } else {
            accept_point = true;
            ++it;
            if (ndx <= a.prm.tol_polish * fmax(1.0, nxp) || it >= a.prm.polish_max) stt = 2;
          }
        }
      }
      // copy the point and push the history on this warp's coordinates
      bool xfinite = true;
      if (act && accept_point) {
        const int cap = a.prm.max_order + 1;
        for (int i = warp; i < n; i += T) {
          cx<L> xv = ld<L>(a.xp, i, m, p);
          st<L>(a.x, i, m, p, xv);
          if (push_hist) {
            if (nh < cap) {
              st<L>(a.hx, (int64_t)nh * n + i, m, p, xv);
            } else {
              for (int s = 0; s + 1 < cap; ++s) st<L>(a.hx, (int64_t)s * n + i, m, p, ld<L>(a.hx, (int64_t)(s + 1) * n + i, m, p));
              st<L>(a.hx, (int64_t)(cap - 1) * n + i, m, p, xv);
            }
            if (pmode > 0) {  // the tangent of the accepted point: its last round's second solution
              const cx<L> tv = ld<L>(a.tdx, i, m, p);
              if (nh < cap) {
                st<L>(a.tx, (int64_t)nh * n + i, m, p, tv);
              } else {
                for (int s = 0; s + 1 < cap; ++s)
                  st<L>(a.tx, (int64_t)s * n + i, m, p, ld<L>(a.tx, (int64_t)(s + 1) * n + i, m, p));
                st<L>(a.tx, (int64_t)(cap - 1) * n + i, m, p, tv);
              }
            }
          }
        }
      }
      if (act && stt == 2) {
        for (int i = warp; i < n; i += T) xfinite = xfinite && cfinite(ld<L>(a.x, i, m, p));
      }
      red[3][warp][lane] = xfinite ? 1.0 : 0.0;
      __syncthreads();
      if (act && stt == 2) {
        bool allf = true;
        for (int w = 0; w < T; ++w) allf = allf && red[3][w][lane] != 0.0;
        stt = allf ? 1 : -1;
      }
      if (warp == 0 && act) {
        int8_t phn = ph;
        if (ph == PH_TRACK && push_hist && stt == 0 && t == 1.0) {
          phn = PH_POLISH;
          it = 0;
        }
        if (push_hist) {
          const int cap = a.prm.max_order + 1;
          if (pmode > 0) a.ntan[p] = (int8_t)min(ntan + 1, cap);
          if (nh < cap) {
            a.ht[(int64_t)nh * m + p] = t;
            ++nh;
          } else {
            for (int s = 0; s + 1 < cap; ++s) a.ht[(int64_t)s * m + p] = a.ht[(int64_t)(s + 1) * m + p];
            a.ht[(int64_t)(cap - 1) * m + p] = t;
          }
        }
        a.status[p] = stt;
        a.phase[p] = phn;
        a.it[p] = (int8_t)it;
        a.t[p] = t;
        a.h[p] = h;
        a.t1[p] = t1;
        a.nh[p] = (int8_t)nh;
        a.steps[p] = steps;
        a.rejects[p] = rejects;
        a.newton[p] = newton;
        if (a.newton_out) a.newton_out[p] = newton;
        a.fallback[p] = (int8_t)fb;
        if (step_end) {
          a.last_dx[p] = ndx;
          a.last_res[p] = nres;
          a.last_its[p] = (int8_t)last_its_v;
          a.last_rej[p] = (int8_t)last_rej_v;
        } else if (ph == PH_POLISH) {  // norms of the latest polish round
          a.last_dx[p] = ndx;
          a.last_res[p] = nres;
        }
      }
      __syncthreads();
    }
  }
}

#if HT_LIMBS == 1
// Table tabjobidx: the paths whose status is 0 keep their relative order;
// one CTA, 1024 threads, warp ballots for the scan.
__global__ void __launch_bounds__(1024) compact_kernel(const int32_t* __restrict__ idx_in,
                                                       const int32_t* __restrict__ count_in,
                                                       const int8_t* __restrict__ status, int32_t* __restrict__ idx_out,
                                                       int32_t* __restrict__ count_out, int32_t* __restrict__ reset) {
  __shared__ int wsum[32];
  __shared__ int base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n = *count_in;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int start = 0; start < n; start += 1024) {
    const int i = start + threadIdx.x;
    int32_t id = i < n ? idx_in[i] : -1;
    const bool keep = i < n && status[id] == 0;
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    if (warp == 0) {
      int v = wsum[lane];
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
      }
      wsum[lane] = v;  // inclusive prefix over warps
    }
    __syncthreads();
    const int before = (warp ? wsum[warp - 1] : 0) + __popc(bal & ((1u << lane) - 1u));
    if (keep) idx_out[base + before] = id;
    __syncthreads();
    if (threadIdx.x == 0) base += wsum[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *count_out = base;
    if (reset) *reset = 0;
  }
}

#endif

// --------------------------------------------------------------- host side
template <int L>
int launch_start_l(int n, const int32_t* d_deg, int64_t first, int64_t count, double* x, cudaStream_t st) {
  if (count == 0) return HT_OK;
  int64_t blocks = (count + 127) / 128;
  if (blocks > 4096) blocks = 4096;
  start_kernel<L><<<(unsigned)blocks, 128, 0, st>>>(n, d_deg, first, count, x);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HT_OK : cuda_fail(e, "start solutions launch");
}

template <int L>
int launch_mgs_l(double* A, double* R, double* x, int rows, int cols, int64_t n_sys, int variant, cudaStream_t st) {
  if (n_sys == 0) return HT_OK;
  if (variant == 2 && L > 1)
    mgs_kernel<L, L != 1><<<(unsigned)((n_sys + 31) / 32), 32, 0, st>>>(A, R, x, rows, cols, n_sys);
  else
    mgs_kernel<L, false><<<(unsigned)((n_sys + 31) / 32), 32, 0, st>>>(A, R, x, rows, cols, n_sys);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HT_OK : cuda_fail(e, "mgs launch");
}

#if HT_LIMBS == 1
__global__ void __launch_bounds__(256) mlp_image_kernel(MlpSmem* img, const __nv_bfloat16* __restrict__ wbf,
                                                        const float* __restrict__ master) {
  mlp_load(*img, wbf, master);
}
size_t mlp_image_bytes() { return sizeof(MlpSmem); }
int launch_mlp_image(void* img, const __nv_bfloat16* wbf, const float* master, cudaStream_t st) {
  mlp_image_kernel<<<1, 256, 0, st>>>(static_cast<MlpSmem*>(img), wbf, master);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HT_OK : cuda_fail(e, "mlp image launch");
}

int launch_compact(const int32_t* idx_in, const int32_t* count_in, const int8_t* status, int32_t* idx_out,
                   int32_t* count_out, cudaStream_t st, int32_t* reset) {
  compact_kernel<<<1, 1024, 0, st>>>(idx_in, count_in, status, idx_out, count_out, reset);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HT_OK : cuda_fail(e, "compact launch");
}
#endif

template <int L>
int launch_init_l(const TrackArgs& a, cudaStream_t st) {
  int64_t blocks = (a.m + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  init_kernel<L><<<(unsigned)blocks, 256, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HT_OK : cuda_fail(e, "init launch");
}

template <int L>
int launch_track_l(const TrackArgs& a, int team, int64_t max_groups, cudaStream_t st) {
  const bool learn = a.mlp_img != nullptr;
  const bool in = L > 1 && a.int_eval;  // the double tracker keeps FP64 evaluation
  // dynamic shared memory of the integer instantiations: the converted points
  const size_t dsm = in ? (size_t)a.n * 32 * ((2 * IntW<L>::W + 1) * sizeof(int32_t) + sizeof(float)) : 0;
  auto go = [&](auto kern) {
    // the kernel's static shared memory counts against the same 48 KB default,
    // so the limit is raised for any dynamic size (n = 32 DD asks for 48 KB)
    if (dsm > 0) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * team, dsm);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)sm_count() * per_sm;
    if (grid > max_groups) grid = max_groups;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, 32 * team, dsm, st>>>(a);
  };
  if (team > 8) {  // wide teams: double and double double (the host only asks for these)
    if (L == 4) return set_error(HT_EUNSUPPORTED, "track launch: teams above 8 warps need D or DD");
    if (learn)
      in ? go(track_kernel<L, true, L == 2, 16>) : go(track_kernel<L, true, false, 16>);
    else
      in ? go(track_kernel<L, false, L == 2, 16>) : go(track_kernel<L, false, false, 16>);
  } else if (learn) {
    in ? go(track_kernel<L, true, L != 1>) : go(track_kernel<L, true, false>);
  } else {
    in ? go(track_kernel<L, false, L != 1>) : go(track_kernel<L, false, false>);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HT_OK : cuda_fail(e, "track launch");
}

template <int L>
int launch_start_at_l(int n, const int32_t* d_deg, int64_t first, const int32_t* ids, const int32_t* count,
                      int64_t cap, double* x, cudaStream_t st) {
  if (cap == 0) return HT_OK;
  int64_t blocks = (cap + 127) / 128;
  if (blocks > 4096) blocks = 4096;
  start_at_kernel<L><<<(unsigned)blocks, 128, 0, st>>>(n, d_deg, first, ids, count, x, cap);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HT_OK : cuda_fail(e, "start points launch");
}

template <int L>
int launch_scatter_l(int n, const int32_t* ids, const int32_t* count, int64_t cap, const double* xs, const int8_t* ss,
                     const double* ts, double* xd, int8_t* sd, double* td, int64_t m, cudaStream_t st) {
  if (cap == 0) return HT_OK;
  int64_t blocks = (cap + 127) / 128;
  if (blocks > 4096) blocks = 4096;
  scatter_kernel<L><<<(unsigned)blocks, 128, 0, st>>>(n, ids, count, xs, ss, ts, cap, xd, sd, td, m);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HT_OK : cuda_fail(e, "scatter launch");
}

template <int L>
int launch_features_l(const double* rec, int64_t n_rec, int n, int cap, int newton_max, float* feat, cudaStream_t st) {
  if (n_rec == 0) return HT_OK;
  int64_t blocks = (n_rec + 127) / 128;
  if (blocks > 4096) blocks = 4096;
  features_kernel<L><<<(unsigned)blocks, 128, 0, st>>>(rec, n_rec, n, cap, newton_max, feat);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HT_OK : cuda_fail(e, "features launch");
}

template <int L>
int track_occupancy_l(int team) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, track_kernel<L, false, false>, 32 * team, 0);
  return per_sm;
}

#ifndef HT_LIMBS
#error "compile once per precision with -DHT_LIMBS=1, 2 or 4"
#endif
template int launch_start_l<HT_LIMBS>(int, const int32_t*, int64_t, int64_t, double*, cudaStream_t);
template int launch_mgs_l<HT_LIMBS>(double*, double*, double*, int, int, int64_t, int, cudaStream_t);
template int launch_init_l<HT_LIMBS>(const TrackArgs&, cudaStream_t);
template int launch_track_l<HT_LIMBS>(const TrackArgs&, int, int64_t, cudaStream_t);
template int track_occupancy_l<HT_LIMBS>(int);
template int launch_features_l<HT_LIMBS>(const double*, int64_t, int, int, int, float*, cudaStream_t);
template int launch_start_at_l<HT_LIMBS>(int, const int32_t*, int64_t, const int32_t*, const int32_t*, int64_t, double*,
                                         cudaStream_t);
template int launch_scatter_l<HT_LIMBS>(int, const int32_t*, const int32_t*, int64_t, const double*, const int8_t*,
                                        const double*, double*, int8_t*, double*, int64_t, cudaStream_t);

}  // namespace ht
