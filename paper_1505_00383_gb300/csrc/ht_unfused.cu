// The paper's organisation of evaluation and differentiation as three
// kernels over a workspace in device memory (Section 3, Tables tabcpugpu and
// tabmemory), kept as an ablation of the fused kernel (ht_evaldiff.cu):
//   coeff  the coefficient c of every monomial at every point (c(t) in the
//          homotopy; here the system's coefficient), written to the
//          workspace's cff rows;
//   mon    every monomial and its derivatives at every point, by the reverse
//          mode of Table tabmoneval (the fused kernel's sweep, operation for
//          operation), written to the workspace's mon rows: the value, then
//          the k derivatives (before their exponent factor);
//   sum    every output (polynomial value, Jacobian entry) at every point:
//          the sum of its terms from the mon rows in monomial order.
// All rows are vertical ([row][2][L][points], point fastest: Table
// tabtranspose), so every kernel's loads and stores are coalesced.  The sums
// take the fused kernel's operations in its order, so results are bitwise
// identical to ht_eval_diff's FP64 bodies.
#include <chrono>
#include <cstring>
#include <vector>

#include "ht_eval.cuh"
#include "ht_internal.h"

namespace ht {

// coeff: cff row m = c_m at every point of the chunk.
template <int L>
__global__ void uf_coeff_kernel(const double* __restrict__ coef, int64_t M, int64_t cc, double* __restrict__ cff) {
  const int64_t total = M * cc;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = e / cc, p = e % cc;
    st<L>(cff, m, cc, p, ld_coef<L>(coef + m * 2 * L));
  }
}

// mon: block (points, monomial m = blockIdx.y).  Row slot_off[m] of the
// workspace (rows counted from its start, past the M coefficient rows) gets
// the value, rows slot_off[m] + 1 + r the derivative by the r-th variable of
// the support (without the exponent factor).
template <int L>
__global__ void __launch_bounds__(128) uf_mon_kernel(const int32_t* __restrict__ mon_off,
                                                     const uint16_t* __restrict__ pairs,
                                                     const int32_t* __restrict__ slot_off, const double* __restrict__ x,
                                                     int64_t ldx, int64_t p0, int64_t cc, const double* __restrict__ cff,
                                                     double* __restrict__ mon) {
  const int m = blockIdx.y;
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= cc) return;
  const int beg = __ldg(mon_off + m), k = __ldg(mon_off + m + 1) - beg;
  const uint16_t* pr = pairs + beg;
  const int64_t s0 = __ldg(slot_off + m);
  cx<L> cf = ld<L>(cff, m, cc, p);
  if (k == 0) {
    st<L>(mon, s0, cc, p, cf);
    return;
  }
  cx<L> P[64];
  for (int r = 0; r < k; ++r) {
    const uint16_t q = __ldg(pr + r);
    const cx<L> xr = ld<L>(x, q & 0xff, ldx, p0 + p);
    for (int e = 1; e < (q >> 8); ++e) cf = cmul(cf, xr);
  }
  for (int r = 0; r < k; ++r) {
    const cx<L> xr = ld<L>(x, __ldg(pr + r) & 0xff, ldx, p0 + p);
    P[r] = cmul(r == 0 ? cf : P[r - 1], xr);
  }
  st<L>(mon, s0, cc, p, P[k - 1]);
  if (k == 1) {
    st<L>(mon, s0 + 1, cc, p, cf);
    return;
  }
  st<L>(mon, s0 + k, cc, p, P[k - 2]);
  cx<L> S = ld<L>(x, __ldg(pr + k - 1) & 0xff, ldx, p0 + p);
  for (int r = k - 2; r >= 1; --r) {
    st<L>(mon, s0 + 1 + r, cc, p, cmul(P[r - 1], S));
    S = cmul(S, ld<L>(x, __ldg(pr + r) & 0xff, ldx, p0 + p));
  }
  st<L>(mon, s0 + 1, cc, p, cmul(cf, S));
}

// sum: block (points, output o = blockIdx.y): outputs are polynomial j's
// value (o = j (nv + 1)) and its derivatives (o = j (nv + 1) + 1 + i).
// Terms out_slot[out_off[o] ..] in monomial order, scaled by out_exp (the
// exponent; 0 marks a value term, added as is).
template <int L>
__global__ void __launch_bounds__(128) uf_sum_kernel(const int32_t* __restrict__ out_off,
                                                     const int32_t* __restrict__ out_slot,
                                                     const int32_t* __restrict__ out_exp, int nv, int64_t ldo,
                                                     int64_t p0, int64_t cc, const double* __restrict__ mon,
                                                     double* __restrict__ val, double* __restrict__ jac) {
  const int o = blockIdx.y;
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= cc) return;
  cx<L> acc = czero<L>();
  const int b = __ldg(out_off + o), e = __ldg(out_off + o + 1);
  for (int t = b; t < e; ++t) {
    const cx<L> v = ld<L>(mon, __ldg(out_slot + t), cc, p);
    const int ex = __ldg(out_exp + t);
    acc = ex == 0 ? cadd(acc, v) : jacc<L>(acc, (double)ex, v);
  }
  const int j = o / (nv + 1), r = o % (nv + 1);
  if (r == 0)
    st<L>(val, j, ldo, p0 + p, acc);
  else
    st<L>(jac, (int64_t)j * nv + (r - 1), ldo, p0 + p, acc);
}

template <int L>
int launch_unfused_l(const ht_system* s, int64_t n, int64_t p0, int64_t cc, const double* x, double* val, double* jac,
                     double* ws, cudaEvent_t* ev, cudaStream_t st) {
  const int32_t* out_off = (const int32_t*)s->d_uf;
  const int64_t n_out = (int64_t)s->np * (s->nv + 1);
  const int32_t* out_slot = out_off + n_out + 1;
  const int32_t* out_exp = out_slot + s->uf_terms;
  const int32_t* slot_off = out_exp + s->uf_terms;
  // one array of rows: the coefficients in rows 0 .. M-1, the monomials'
  // values and derivatives in the rows slot_off[m] .. (slot_off[0] = M)
  double* cff = ws;
  double* mon = ws;
  const unsigned gx = (unsigned)((cc + 127) / 128);
  if (ev) cudaEventRecord(ev[0], st);
  int64_t blocks = (s->M * cc + 255) / 256;
  if (blocks > (int64_t)sm_count() * 16) blocks = (int64_t)sm_count() * 16;
  uf_coeff_kernel<L><<<(unsigned)blocks, 256, 0, st>>>(s->d_coef, s->M, cc, cff);
  if (ev) cudaEventRecord(ev[1], st);
  if (ev) cudaEventRecord(ev[2], st);
  uf_mon_kernel<L><<<dim3(gx, (unsigned)s->M), 128, 0, st>>>(s->d_mon_off, s->d_pairs, slot_off, x, n, p0, cc, cff,
                                                             mon);
  if (ev) cudaEventRecord(ev[3], st);
  if (ev) cudaEventRecord(ev[4], st);
  uf_sum_kernel<L><<<dim3(gx, (unsigned)n_out), 128, 0, st>>>(out_off, out_slot, out_exp, s->nv, n, p0, cc, mon, val,
                                                              jac);
  if (ev) cudaEventRecord(ev[5], st);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HT_OK : cuda_fail(e, "ht_eval_diff_unfused: launch");
}

#ifndef HT_LIMBS
#error "compile once per precision with -DHT_LIMBS=1, 2 or 4"
#endif
template int launch_unfused_l<HT_LIMBS>(const ht_system*, int64_t, int64_t, int64_t, const double*, double*, double*,
                                        double*, cudaEvent_t*, cudaStream_t);

#if HT_LIMBS == 1
// Output lists of the sum kernel and workspace slots of the mon kernel, built
// from the host copy of the system.
static int uf_prepare(ht_system* s) {
  if (s->d_uf) return HT_OK;
  const int nv = s->nv, np = s->np;
  const int64_t n_out = (int64_t)np * (nv + 1);
  std::vector<int32_t> slot_off(s->M + 1);
  int64_t slot = s->M;  // rows 0 .. M-1 hold the coefficients
  for (int64_t m = 0; m < s->M; ++m) {
    slot_off[m] = (int32_t)slot;
    const int k = s->h_mon_off[m + 1] - s->h_mon_off[m];
    slot += k + 1;
  }
  slot_off[s->M] = (int32_t)slot;
  std::vector<std::vector<int32_t>> sl(n_out), ex(n_out);
  for (int j = 0; j < np; ++j)
    for (int m = s->h_poly_off[j]; m < s->h_poly_off[j + 1]; ++m) {
      const int o = j * (nv + 1);
      sl[o].push_back(slot_off[m]);
      ex[o].push_back(0);
      const int b = s->h_mon_off[m], k = s->h_mon_off[m + 1] - b;
      for (int r = 0; r < k; ++r) {
        const uint16_t q = s->h_pairs[b + r];
        sl[o + 1 + (q & 0xff)].push_back(slot_off[m] + 1 + r);
        ex[o + 1 + (q & 0xff)].push_back(q >> 8);
      }
    }
  std::vector<int32_t> off(n_out + 1, 0), slots, exps;
  for (int64_t o = 0; o < n_out; ++o) {
    slots.insert(slots.end(), sl[o].begin(), sl[o].end());
    exps.insert(exps.end(), ex[o].begin(), ex[o].end());
    off[o + 1] = (int32_t)slots.size();
  }
  const int64_t T = (int64_t)slots.size();
  std::vector<int32_t> blob;
  blob.reserve(n_out + 1 + 2 * T + s->M + 1);
  blob.insert(blob.end(), off.begin(), off.end());
  blob.insert(blob.end(), slots.begin(), slots.end());
  blob.insert(blob.end(), exps.begin(), exps.end());
  blob.insert(blob.end(), slot_off.begin(), slot_off.end());
  cudaError_t e = cudaMalloc(&s->d_uf, blob.size() * 4);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(HT_ENOMEM, "ht_eval_diff_unfused: output lists");
  }
  e = cudaMemcpy(s->d_uf, blob.data(), blob.size() * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "ht_eval_diff_unfused: upload");
  s->uf_slots = slot;
  s->uf_terms = T;
  return HT_OK;
}

int run_unfused(ht_system* s, int64_t n_pts, const double* x, double* val, double* jac, ht_unfused_stats* stats,
                cudaStream_t st) {
  if (s->M > 65535 || (int64_t)s->np * (s->nv + 1) > 65535)
    return set_error(HT_EUNSUPPORTED, "ht_eval_diff_unfused: at most 65,535 monomials and outputs");
  int rc = uf_prepare(s);
  if (rc != HT_OK) return rc;
  const int L = s->limbs;
  // chunk of points whose workspace ([slots][2][L][chunk]) fits in 2 GiB
  const size_t per_pt = (size_t)s->uf_slots * 2 * L * sizeof(double);
  int64_t chunk = (int64_t)(((size_t)2 << 30) / per_pt) / 128 * 128;
  if (chunk < 128) chunk = 128;
  if (chunk > n_pts) chunk = n_pts;
  const size_t need = per_pt * (size_t)chunk;
  if (s->uf_ws_bytes < need) {
    if (s->d_uf_ws) {
      cudaStreamSynchronize(st);
      cudaFree(s->d_uf_ws);
      s->d_uf_ws = nullptr;
      s->uf_ws_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&s->d_uf_ws, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_error(HT_ENOMEM, "ht_eval_diff_unfused: workspace of %zu bytes", need);
    }
    s->uf_ws_bytes = need;
  }
  cudaEvent_t ev[6] = {};
  if (stats)
    for (auto& e : ev)
      if (cudaEventCreate(&e) != cudaSuccess) return cuda_fail(cudaGetLastError(), "ht_eval_diff_unfused: events");
  int64_t kvars = 0;  // variable occurrences over all monomials
  for (int64_t m = 0; m < s->M; ++m) kvars += s->h_mon_off[m + 1] - s->h_mon_off[m];
  const double cxb = 16.0 * L;
  for (int64_t p0 = 0; p0 < n_pts && rc == HT_OK; p0 += chunk) {
    const int64_t cc = n_pts - p0 < chunk ? n_pts - p0 : chunk;
    rc = [&]() {
      switch (L) {
        case 1: return launch_unfused_l<1>(s, n_pts, p0, cc, x, val, jac, (double*)s->d_uf_ws, stats ? ev : nullptr, st);
        case 2: return launch_unfused_l<2>(s, n_pts, p0, cc, x, val, jac, (double*)s->d_uf_ws, stats ? ev : nullptr, st);
        default: return launch_unfused_l<4>(s, n_pts, p0, cc, x, val, jac, (double*)s->d_uf_ws, stats ? ev : nullptr, st);
      }
    }();
    if (rc == HT_OK && stats) {
      cudaError_t e = cudaEventSynchronize(ev[5]);
      if (e != cudaSuccess) {
        rc = cuda_fail(e, "ht_eval_diff_unfused");
        break;
      }
      float a = 0, b = 0, c = 0;
      cudaEventElapsedTime(&a, ev[0], ev[1]);
      cudaEventElapsedTime(&b, ev[2], ev[3]);
      cudaEventElapsedTime(&c, ev[4], ev[5]);
      stats->ms_coeff += a;
      stats->ms_mon += b;
      stats->ms_sum += c;
      // algorithmic bytes: coeff writes M rows; mon reads its coefficient row
      // and k variables and writes k + 1 rows; sum reads every term and
      // writes every output
      const double rows_mon = (double)(s->uf_slots - s->M);
      stats->bytes_coeff += cxb * cc * (double)s->M;
      stats->bytes_mon += cxb * cc * ((double)s->M + (double)kvars + rows_mon);
      stats->bytes_sum += cxb * cc * ((double)s->uf_terms + (double)s->np * (s->nv + 1));
    }
  }
  if (stats)
    for (auto& e : ev) cudaEventDestroy(e);
  if (rc == HT_OK && stats) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "ht_eval_diff_unfused");
  }
  return rc;
}

}  // namespace ht

using namespace ht;

extern "C" int ht_eval_diff_unfused(ht_system* s, int64_t n_pts, const double* x, double* val, double* jac,
                                    ht_unfused_stats* stats, void* stream) {
  clear_error();
  if (stats) std::memset(stats, 0, sizeof *stats);
  if (!s) return set_error(HT_EINVAL, "ht_eval_diff_unfused: NULL system");
  if (n_pts < 0) return set_error(HT_EINVAL, "ht_eval_diff_unfused: n_pts < 0");
  if (n_pts == 0) return HT_OK;
  if (!x || !val || !jac || !is_device_ptr(x) || !is_device_ptr(val) || !is_device_ptr(jac) ||
      (((uintptr_t)x | (uintptr_t)val | (uintptr_t)jac) & 7))
    return set_error(HT_EINVAL, "ht_eval_diff_unfused: x, val and jac must be device memory");
  return run_unfused(s, n_pts, x, val, jac, stats, (cudaStream_t)stream);
}
#else
}  // namespace ht
#endif
