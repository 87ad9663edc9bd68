// One polynomial's value and gradient row on the integer pipe, for one point
// per lane (device only): the per-output frames, the reverse-mode sweep of
// ht_mpi_eval.cuh with the row's fixed-point accumulators in place in the
// caller's output row, and the conversion of every output to L doubles.  The
// evaluation kernel and the tracker both call it.
#pragma once
#include "ht_mpi_eval.cuh"
#include "ht_mpi_ops.cuh"

namespace ht {

using mpi::IntW;
constexpr int kIntMaxVars = 64;

// The fixed-point accumulators of entry i of a row in the vertical layout
// [i][2][L][n] (path/point index p fastest): 2L doubles hold 2 x 2L int32.
template <int L>
__device__ __forceinline__ void ld_fix(const double* jrow, int64_t i, int64_t n, int64_t p, int32_t* r, int32_t* im) {
  const unsigned long long* q = reinterpret_cast<const unsigned long long*>(jrow) + (i * 2) * L * n + p;
#pragma unroll
  for (int t = 0; t < L; ++t) {
    const unsigned long long a = q[t * n], b = q[(L + t) * n];
    r[2 * t] = (int32_t)(uint32_t)a;
    r[2 * t + 1] = (int32_t)(uint32_t)(a >> 32);
    im[2 * t] = (int32_t)(uint32_t)b;
    im[2 * t + 1] = (int32_t)(uint32_t)(b >> 32);
  }
}
template <int L>
__device__ __forceinline__ void st_fix(double* jrow, int64_t i, int64_t n, int64_t p, const int32_t* r,
                                       const int32_t* im) {
  unsigned long long* q = reinterpret_cast<unsigned long long*>(jrow) + (i * 2) * L * n + p;
#pragma unroll
  for (int t = 0; t < L; ++t) {
    q[t * n] = (unsigned long long)(uint32_t)r[2 * t] | ((unsigned long long)(uint32_t)r[2 * t + 1] << 32);
    q[(L + t) * n] = (unsigned long long)(uint32_t)im[2 * t] | ((unsigned long long)(uint32_t)im[2 * t + 1] << 32);
  }
}

// The Jacobian row accumulates in place in the output slots: in the doubles
// of the vertical layout (2L doubles hold the 2 x 2L int32 limbs) ...
template <int L>
struct RowAcc {
  double* jrow;
  int64_t n, p;
  static constexpr int WA = IntW<L>::WA;
  __device__ __forceinline__ void zero(int v) {
    int32_t z[WA];
#pragma unroll
    for (int k = 0; k < WA; ++k) z[k] = 0;
    st_fix<L>(jrow, v, n, p, z, z);
  }
  __device__ __forceinline__ void add(int v, const mpi::fz<IntW<L>::W>& d, int e, int F) {
    int32_t ar[WA], ai[WA];
    ld_fix<L>(jrow, v, n, p, ar, ai);
    mpi::acc_add_fast<IntW<L>::W, WA>(ar, ai, d, e, F);
    st_fix<L>(jrow, v, n, p, ar, ai);
  }
  // entry v as L doubles per component, times scale (rounded once)
  __device__ __forceinline__ void finish(int v, int F, double scale) {
    int32_t ar[WA], ai[WA];
    ld_fix<L>(jrow, v, n, p, ar, ai);
    double o[L];
    if (scale == 1.0)
      mpi::fixed_to_doubles<WA, L>(ar, F, o);
    else
      mpi::fixed_scaled_to_doubles<WA, L>(ar, F, scale, o);
#pragma unroll
    for (int l = 0; l < L; ++l) jrow[((int64_t)(v * 2) * L + l) * n + p] = o[l];
    if (scale == 1.0)
      mpi::fixed_to_doubles<WA, L>(ai, F, o);
    else
      mpi::fixed_scaled_to_doubles<WA, L>(ai, F, scale, o);
#pragma unroll
    for (int l = 0; l < L; ++l) jrow[((int64_t)(v * 2 + 1) * L + l) * n + p] = o[l];
  }
};

// ... or in limb-string slots ([entry][2W+1][n] int32 words: exponent, re
// limbs, im limbs; the accumulators use the limb words), finished as limb
// strings for the integer least squares.
template <int L>
struct RowAccFz {
  int32_t* zrow;
  int64_t n, p;
  static constexpr int W = IntW<L>::W, WA = IntW<L>::WA;
  static_assert(WA <= W, "the accumulator limbs must fit the limb words");
  __device__ __forceinline__ int32_t* at(int v) const { return zrow + (int64_t)v * (2 * W + 1) * n + p; }
  __device__ __forceinline__ void zero(int v) {
    int32_t* q = at(v);
#pragma unroll
    for (int k = 0; k < WA; ++k) q[(1 + k) * n] = q[(1 + W + k) * n] = 0;
  }
  __device__ __forceinline__ void add(int v, const mpi::fz<W>& d, int e, int F) {
    int32_t* q = at(v);
    int32_t ar[WA], ai[WA];
#pragma unroll
    for (int k = 0; k < WA; ++k) {
      ar[k] = q[(1 + k) * n];
      ai[k] = q[(1 + W + k) * n];
    }
    mpi::acc_add_fast<W, WA>(ar, ai, d, e, F);
#pragma unroll
    for (int k = 0; k < WA; ++k) {
      q[(1 + k) * n] = ar[k];
      q[(1 + W + k) * n] = ai[k];
    }
  }
  __device__ __forceinline__ void finish(int v, int F, double scale) {
    int32_t* q = at(v);
    int32_t ar[WA], ai[WA];
#pragma unroll
    for (int k = 0; k < WA; ++k) {
      ar[k] = q[(1 + k) * n];
      ai[k] = q[(1 + W + k) * n];
    }
    const mpi::fz<W> z = mpi::fixed_scaled_to_fz<WA, W>(ar, ai, F, scale);
    q[0] = z.f;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      q[(1 + k) * n] = z.r[k];
      q[(1 + W + k) * n] = z.i[k];
    }
  }
};

// The lane's point converted once: X[i] (limb string) and lg[i] = log2 |x_i|,
// from x in the layout [nv][2][L][n].
template <int L>
__device__ __forceinline__ void int_point(const double* __restrict__ x, int nv, int64_t n, int64_t p,
                                          mpi::fz<IntW<L>::W>* X, float* lg) {
  for (int i = 0; i < nv; ++i) {
    double re[L], im[L];
#pragma unroll
    for (int l = 0; l < L; ++l) {
      re[l] = x[((int64_t)(i * 2) * L + l) * n + p];
      im[l] = x[((int64_t)(i * 2 + 1) * L + l) * n + p];
    }
    X[i] = mpi::from_doubles<IntW<L>::W, L>(re, im);
    lg[i] = mpi::log2_mod(re[0], im[0]);
  }
}

// Monomials m0..m1 of one polynomial at the lane's point: the value as L
// doubles per component (vre, vim) and the gradient times scale in the row
// storage (RowAcc: doubles in jrow's layout [nv][2][L][n]; RowAccFz: limb
// strings), each entry rounded once from its exact fixed-point product.  X
// and lg are indexable by variable (local arrays or shared-memory views); P
// is scratch for the forward products (max monomial size entries).
template <int L, class XA, class LG, class PS, class Row>
__device__ void int_row_in(const int32_t* __restrict__ mon_off, const uint16_t* __restrict__ pairs,
                           const mpi::fz<IntW<L>::W>* __restrict__ cfz, const float* __restrict__ clg, int m0,
                           int m1, const XA& X, const LG& lg, int nv, Row& row, double* vre, double* vim, PS* P,
                           double scale) {
  constexpr int WA = IntW<L>::WA;
  int Fv[kIntMaxVars];
  const int F = mpi::frames_for_poly<WA>(mon_off, pairs, clg, m0, m1, lg, nv, Fv);
  int32_t vr[WA], vi[WA];
#pragma unroll
  for (int k = 0; k < WA; ++k) vr[k] = vi[k] = 0;
  for (int i = 0; i < nv; ++i) row.zero(i);
  mpi::eval_poly_int<L>(mon_off, pairs, cfz, m0, m1, X, F, Fv, row, vr, vi, P);
  mpi::fixed_to_doubles<WA, L>(vr, F, vre);
  mpi::fixed_to_doubles<WA, L>(vi, F, vim);
  for (int i = 0; i < nv; ++i) row.finish(i, Fv[i], scale);
}
template <int L, class XA, class LG, class PS>
__device__ void int_row(const int32_t* __restrict__ mon_off, const uint16_t* __restrict__ pairs,
                        const mpi::fz<IntW<L>::W>* __restrict__ cfz, const float* __restrict__ clg, int m0, int m1,
                        const XA& X, const LG& lg, int nv, double* jrow, int64_t n, int64_t p, double* vre,
                        double* vim, PS* P, double scale = 1.0) {
  RowAcc<L> row{jrow, n, p};
  int_row_in<L>(mon_off, pairs, cfz, clg, m0, m1, X, lg, nv, row, vre, vim, P, scale);
}
template <int L, class XA, class LG, class PS>
__device__ void int_row_fz(const int32_t* __restrict__ mon_off, const uint16_t* __restrict__ pairs,
                           const mpi::fz<IntW<L>::W>* __restrict__ cfz, const float* __restrict__ clg, int m0,
                           int m1, const XA& X, const LG& lg, int nv, int32_t* zrow, int64_t n, int64_t p,
                           double* vre, double* vim, PS* P, double scale) {
  RowAccFz<L> row{zrow, n, p};
  int_row_in<L>(mon_off, pairs, cfz, clg, m0, m1, X, lg, nv, row, vre, vim, P, scale);
}

// Views of a CTA's converted points in shared memory, lane-interleaved so a
// warp's load of one word is 32 consecutive words: limb string words
// [var][2W+1][32] (word 0 the exponent, then re limbs, then im limbs) and
// log2 moduli [var][32].
template <int L>
struct SmemPoints {
  static constexpr int W = IntW<L>::W, WORDS = 2 * W + 1;
  const int32_t* x;
  int lane;
  __device__ __forceinline__ mpi::fz<W> operator[](int v) const {
    const int32_t* q = x + (int64_t)v * WORDS * 32 + lane;
    mpi::fz<W> z;
    z.f = q[0];
#pragma unroll
    for (int k = 0; k < W; ++k) {
      z.r[k] = q[(1 + k) * 32];
      z.i[k] = q[(1 + W + k) * 32];
    }
    return z;
  }
};
struct SmemLog {
  const float* g;
  int lane;
  __device__ __forceinline__ float operator[](int v) const { return g[v * 32 + lane]; }
};
template <int L>
__device__ __forceinline__ void store_point(int32_t* x, int v, int lane, const mpi::fz<IntW<L>::W>& z) {
  constexpr int W = IntW<L>::W, WORDS = 2 * W + 1;
  int32_t* q = x + (int64_t)v * WORDS * 32 + lane;
  q[0] = z.f;
#pragma unroll
  for (int k = 0; k < W; ++k) {
    q[(1 + k) * 32] = z.r[k];
    q[(1 + W + k) * 32] = z.i[k];
  }
}

}  // namespace ht
