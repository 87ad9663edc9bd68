// Host driver of the many-path tracker and the standalone entry points for its
// stages (start solutions, least squares, compaction).
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "ht_internal.h"
#include "ht_track.h"

namespace ht {
const float* mlp_master(const ht_mlp* net);
const __nv_bfloat16* mlp_bf16(const ht_mlp* net);
}

namespace ht {

template <typename F>
static int by_limbs(int L, F f) {
  switch (L) {
    case 1: return f(std::integral_constant<int, 1>());
    case 2: return f(std::integral_constant<int, 2>());
    case 4: return f(std::integral_constant<int, 4>());
  }
  return set_error(HT_EINVAL, "limbs=%d must be 1, 2 or 4", L);
}

static size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

// Grow the system's tracker workspace to `bytes` (device) and make sure the
// pinned host word for the active count exists.
static int ensure_track_ws(ht_system* s, size_t bytes, cudaStream_t st) {
  if (s->track_ws_bytes < bytes) {
    if (s->d_track_ws) {
      cudaStreamSynchronize(st);
      cudaFree(s->d_track_ws);
      s->d_track_ws = nullptr;
      s->track_ws_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&s->d_track_ws, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_error(HT_ENOMEM, "ht_track_paths: workspace of %zu bytes", bytes);
    }
    s->track_ws_bytes = bytes;
  }
  if (!s->h_count) {
    cudaError_t e = cudaHostAlloc((void**)&s->h_count, 2 * sizeof(int32_t), cudaHostAllocDefault);
    if (e != cudaSuccess) return cuda_fail(e, "ht_track_paths: pinned count");
  }
  return HT_OK;
}

// Probe records: record r repeated for every multiplier, its step scaled.
__global__ void probe_records_kernel(const double* __restrict__ rec, int64_t n_rec, int64_t R, int n_mult,
                                     const double* __restrict__ mults, double* __restrict__ out) {
  const int64_t total = n_rec * n_mult * R;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = e / R, k = e % R, r = q / n_mult;
    const int j = (int)(q % n_mult);
    double v = rec[r * R + k];
    if (k == 2) v *= mults[j];
    out[e] = v;
  }
}

// Label of record r:
//   rho   among the multipliers whose single probe step was accepted (t
//         moved past the record's t), the one with the most progress per
//         Newton round, mu_j / rounds_j (ties to the larger mu_j); rho = its
//         log, or the log of the smallest multiplier if no probe was accepted;
//   alpha for that accepted probe, the scale of the predictor's displacement
//         that best reaches the corrected point: with x the record's current
//         point, p the extrapolation predictor's point at the probe's t1 and
//         x* the probe's corrected point, alpha = Re <p - x, x* - p> / |p - x|^2
//         over all coordinates (leading limbs), clamped to [-1, 1]; 0 if no
//         probe was accepted or p = x.
// px is the probes' end points [n][2][L][n_rec n_mult].
__global__ void labels_kernel(const double* __restrict__ rec, int64_t n_rec, int64_t R, int n, int L, int cap,
                              int n_mult, const double* __restrict__ mults, const double* __restrict__ t_end,
                              const int32_t* __restrict__ rounds, const double* __restrict__ px,
                              float* __restrict__ labels) {
  const int64_t P = n_rec * n_mult;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_rec; r += (int64_t)gridDim.x * blockDim.x) {
    const double* h = rec + r * R;
    const double t0 = h[1];
    double best = -1.0, best_eff = -1.0, lo = mults[0];
    int jb = -1;
    for (int j = 0; j < n_mult; ++j) {
      lo = fmin(lo, mults[j]);
      if (t_end[r * n_mult + j] > t0) {
        const int k = rounds[r * n_mult + j];
        const double eff = mults[j] / (double)(k > 0 ? k : 1);
        if (eff > best_eff || (eff == best_eff && mults[j] > best)) {
          best_eff = eff;
          best = mults[j];
          jb = j;
        }
      }
    }
    double alpha = 0.0;
    if (jb >= 0) {
      // the predictor of the tracker at t1 (Lagrange form over the history)
      int nh = (int)h[3];
      nh = nh < 1 ? 1 : (nh > cap ? cap : nh);
      const double step = fmin(h[2] * mults[jb], 1.0 - t0);
      const double t1 = (step >= 1.0 - t0) ? 1.0 : t0 + step;
      const int mm = nh < cap ? nh : cap, base = nh - mm;
      double w[8];
      for (int j = 0; j < mm; ++j) {
        double num = 1.0, den = 1.0;
        for (int i = 0; i < mm; ++i) {
          if (i == j) continue;
          num *= t1 - h[REC_HDR + base + i];
          den *= h[REC_HDR + base + j] - h[REC_HDR + base + i];
        }
        w[j] = num / den;
      }
      const double* hx = h + REC_HDR + cap;  // [cap][n][2][L]
      const int64_t q = r * n_mult + jb;
      double dot = 0.0, nrm = 0.0;
      for (int i = 0; i < n; ++i) {
        double pre = 0.0, pim = 0.0;
        for (int j = 0; j < mm; ++j) {
          pre += w[j] * hx[(((int64_t)(base + j) * n + i) * 2 + 0) * L];
          pim += w[j] * hx[(((int64_t)(base + j) * n + i) * 2 + 1) * L];
        }
        const double xre = hx[(((int64_t)(nh - 1) * n + i) * 2 + 0) * L];
        const double xim = hx[(((int64_t)(nh - 1) * n + i) * 2 + 1) * L];
        const double sre = px[((int64_t)(i * 2 + 0) * L) * P + q], sim = px[((int64_t)(i * 2 + 1) * L) * P + q];
        const double dre = pre - xre, dim = pim - xim;
        dot += dre * (sre - pre) + dim * (sim - pim);
        nrm += dre * dre + dim * dim;
      }
      alpha = nrm > 0.0 ? fmin(1.0, fmax(-1.0, dot / nrm)) : 0.0;
    }
    labels[r * 2 + 0] = (float)log(best > 0.0 ? best : lo);
    labels[r * 2 + 1] = (float)alpha;
  }
}

static void drop_graphs(ht_system* s) {
  for (auto& g : s->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  s->graphs.clear();
}

}  // namespace ht

using namespace ht;

extern "C" {

int ht_default_params(int limbs, ht_params* p) {
  clear_error();
  if (!p) return set_error(HT_EINVAL, "ht_default_params: NULL");
  if (limbs != 1 && limbs != 2 && limbs != 4) return set_error(HT_EINVAL, "ht_default_params: limbs=%d", limbs);
  std::memset(p, 0, sizeof *p);
  p->h0 = 0.05;
  p->h_min = 1e-5;
  p->h_max = 0.1;
  p->f_up = 1.5;
  p->f_down = 0.5;
  p->tol_dx = 1e-6;
  p->tol_res = 1e-4;
  p->tol_polish = limbs == 1 ? 1e-12 : (limbs == 2 ? 1e-24 : 1e-48);
  p->r_div = 1e8;
  p->newton_max = 3;
  p->polish_max = 4;
  p->max_steps = 2000;
  p->max_order = 4;
  return HT_OK;
}

int ht_start_solutions(int n, const int32_t* degrees, int limbs, int64_t first, int64_t count, double* x0,
                       void* stream) {
  clear_error();
  if (n < 1 || !degrees || first < 0 || count < 0) return set_error(HT_EINVAL, "ht_start_solutions: bad arguments");
  for (int i = 0; i < n; ++i)
    if (degrees[i] < 1) return set_error(HT_EINVAL, "ht_start_solutions: degree %d of variable %d", degrees[i], i);
  if (count == 0) return HT_OK;
  if (!x0 || ((uintptr_t)x0 & 7) || !is_device_ptr(x0))
    return set_error(HT_EINVAL, "ht_start_solutions: x0 must be device memory");
  cudaStream_t st = (cudaStream_t)stream;
  int32_t* d_deg = nullptr;
  cudaError_t e = cudaMallocAsync(&d_deg, n * sizeof(int32_t), st);
  if (e != cudaSuccess) return cuda_fail(e, "ht_start_solutions: alloc");
  e = cudaMemcpyAsync(d_deg, degrees, n * sizeof(int32_t), cudaMemcpyHostToDevice, st);
  int rc = e == cudaSuccess ? by_limbs(limbs, [&](auto c) { return launch_start_l<decltype(c)::value>(n, d_deg, first, count, x0, st); })
                            : cuda_fail(e, "ht_start_solutions: copy");
  cudaFreeAsync(d_deg, st);
  if (rc == HT_OK) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "ht_start_solutions");
  }
  return rc;
}

int ht_mgs_solve(int limbs, int rows, int cols, int64_t n_sys, double* Ab, double* R, double* x, void* stream) {
  return ht_mgs_solve_ex(limbs, 0, rows, cols, n_sys, Ab, R, x, stream);
}

int ht_mgs_solve_ex(int limbs, int variant, int rows, int cols, int64_t n_sys, double* Ab, double* R, double* x,
                    void* stream) {
  clear_error();
  if (rows < 1 || cols < 1 || rows < cols || n_sys < 0)
    return set_error(HT_EINVAL, "ht_mgs_solve: need rows >= cols >= 1, n_sys >= 0");
  if (variant != 0 && variant != 2) return set_error(HT_EINVAL, "ht_mgs_solve_ex: variant %d (0 or 2)", variant);
  if (variant == 2 && (limbs == 1 || rows > 64))
    return set_error(HT_EUNSUPPORTED, "ht_mgs_solve_ex: integer limbs need DD or QD and at most 64 rows");
  if (n_sys == 0) return HT_OK;
  if (!Ab || !R || !x || (((uintptr_t)Ab | (uintptr_t)R | (uintptr_t)x) & 7) || !is_device_ptr(Ab) ||
      !is_device_ptr(R) || !is_device_ptr(x))
    return set_error(HT_EINVAL, "ht_mgs_solve: buffers must be device memory");
  cudaStream_t st = (cudaStream_t)stream;
  return by_limbs(limbs,
                  [&](auto c) { return launch_mgs_l<decltype(c)::value>(Ab, R, x, rows, cols, n_sys, variant, st); });
}

int ht_compact(const int8_t* status, int64_t m, int32_t* path_idx, int32_t* count, void* stream) {
  clear_error();
  if (m < 0 || m > 0x7fffffff) return set_error(HT_EINVAL, "ht_compact: m=%lld", (long long)m);
  if (!count || !is_device_ptr(count) || (m > 0 && (!status || !path_idx || !is_device_ptr(status) ||
                                                     !is_device_ptr(path_idx))))
    return set_error(HT_EINVAL, "ht_compact: buffers must be device memory");
  cudaStream_t st = (cudaStream_t)stream;
  // identity index list in a temporary buffer, then the stable compaction
  int32_t* tmp = nullptr;
  cudaError_t e = cudaMallocAsync(&tmp, (m + 1) * sizeof(int32_t), st);
  if (e != cudaSuccess) return cuda_fail(e, "ht_compact: alloc");
  std::vector<int32_t> h(m + 1);
  for (int64_t i = 0; i < m; ++i) h[i] = (int32_t)i;
  h[m] = (int32_t)m;
  e = cudaMemcpyAsync(tmp, h.data(), (m + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, st);
  int rc = e == cudaSuccess ? launch_compact(tmp, tmp + m, status, path_idx, count, st) : cuda_fail(e, "ht_compact");
  if (rc == HT_OK) e = cudaStreamSynchronize(st);
  cudaFreeAsync(tmp, st);
  if (rc == HT_OK && e != cudaSuccess) rc = cuda_fail(e, "ht_compact");
  return rc;
}

int ht_track_paths_ex(ht_system* s, const int32_t* start_deg, const double* gamma, int64_t n_paths,
                      int64_t first_path, const double* x0, const ht_params* prm_in, double* x_end, int8_t* status,
                      double* t_end, int32_t* steps, ht_stats* stats, const ht_track_io* io, void* stream) {
  clear_error();
  auto t_start = std::chrono::steady_clock::now();
  if (!s) return set_error(HT_EINVAL, "ht_track_paths: NULL system");
  if (s->np != s->nv) return set_error(HT_EINVAL, "ht_track_paths: system must be square (%d x %d)", s->np, s->nv);
  const int n = s->nv, L = s->limbs;
  if (!start_deg || !gamma) return set_error(HT_EINVAL, "ht_track_paths: NULL start_deg or gamma");
  if (n_paths < 0 || n_paths > 0x7fffffff || first_path < 0)
    return set_error(HT_EINVAL, "ht_track_paths: n_paths=%lld first_path=%lld", (long long)n_paths, (long long)first_path);
  int deg_max = s->max_deg;
  for (int i = 0; i < n; ++i) {
    if (start_deg[i] < 1 || start_deg[i] > 64) return set_error(HT_EINVAL, "ht_track_paths: start degree %d", start_deg[i]);
    if (start_deg[i] > deg_max) deg_max = start_deg[i];
  }
  if (!std::isfinite(gamma[0]) || !std::isfinite(gamma[1]) || (gamma[0] == 0.0 && gamma[1] == 0.0))
    return set_error(HT_EINVAL, "ht_track_paths: gamma must be finite and nonzero");
  ht_params P;
  if (prm_in)
    P = *prm_in;
  else
    ht_default_params(L, &P);
  if (!(P.h0 > 0) || !(P.h_min > 0) || !(P.h_max >= P.h_min) || !(P.f_up >= 1) || !(P.f_down > 0 && P.f_down < 1) ||
      P.newton_max < 1 || P.newton_max > 100 || P.polish_max < 0 || P.polish_max > 100 || P.max_steps < 1 ||
      P.max_order < 0 || P.max_order > 7 || P.team_warps < 0 || P.team_warps > 16 || (P.team_warps > 8 && L == 4) || P.iters_per_launch < 0 ||
      P.rounds_per_sync < 0 || (P.rounds_per_sync & 1) || !(P.tol_dx > 0) || !(P.tol_res > 0) || !(P.tol_polish > 0) || !(P.r_div > 0) ||
      P.predictor < 0 || P.predictor > 2)
    return set_error(HT_EINVAL, "ht_track_paths: invalid parameters");
  ht_track_io IO;
  std::memset(&IO, 0, sizeof IO);
  if (io) IO = *io;
  if (IO.trace && (IO.trace_stride < 1 || IO.trace_capacity < 0 || !IO.trace_count || !is_device_ptr(IO.trace) ||
                   !is_device_ptr(IO.trace_count)))
    return set_error(HT_EINVAL, "ht_track_paths_ex: trace needs a device buffer, a device counter and stride >= 1");
  if (IO.init_records && !is_device_ptr(IO.init_records))
    return set_error(HT_EINVAL, "ht_track_paths_ex: init_records must be device memory");
  if (IO.mlp && (IO.fallback_steps < 0 || IO.fallback_steps > 100 || !(IO.rho_max >= IO.rho_min) ||
                 !(IO.alpha_max >= 0.0 && IO.alpha_max <= 1.0)))
    return set_error(HT_EINVAL, "ht_track_paths_ex: invalid learned-step settings");
  const int x0_limbs = IO.x0_limbs > 0 ? IO.x0_limbs : L;
  if (IO.x0_limbs < 0 || x0_limbs > L || (x0_limbs == 3))
    return set_error(HT_EINVAL, "ht_track_paths_ex: x0_limbs=%d (1, 2 or 4, at most the system's %d)", IO.x0_limbs, L);
  if (IO.polish_only && (!x0 || IO.init_records || P.polish_max < 1))
    return set_error(HT_EINVAL, "ht_track_paths_ex: polish_only needs x0, no init_records and polish_max >= 1");
  if ((IO.last_dx_out && !is_device_ptr(IO.last_dx_out)) || (IO.last_res_out && !is_device_ptr(IO.last_res_out)) ||
      (IO.newton_out && !is_device_ptr(IO.newton_out)))
    return set_error(HT_EINVAL, "ht_track_paths_ex: last_dx_out, last_res_out and newton_out must be device memory");
  if (stats) std::memset(stats, 0, sizeof *stats);
  if (n_paths == 0) return HT_OK;
  if (!x_end || !status || !t_end || !is_device_ptr(x_end) || !is_device_ptr(status) || !is_device_ptr(t_end) ||
      (x0 && !is_device_ptr(x0)) || (steps && !is_device_ptr(steps)) || (((uintptr_t)x_end | (uintptr_t)t_end) & 7))
    return set_error(HT_EINVAL, "ht_track_paths: outputs (and x0) must be device memory");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t m = n_paths;
  const int cap = P.max_order + 1;
  const size_t cxb = (size_t)2 * L * m * sizeof(double);  // one complex entry for all paths
  // workspace layout
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t o = off;
    off += up256(b);
    return o;
  };
  const int nrhs = P.predictor > 0 ? 2 : 1;  // the tangent predictors add J v = -dh/dt
  // DD and QD (n <= 32) evaluate f and solve the Newton systems on the
  // integer pipe unless an FP64 variant was chosen for this system
  // (ht_set_eval_config 0 or 1), and keep A and R as limb strings of 2 W + 1
  // int32 words an entry (QD 68 bytes against 64 for the doubles, DD 44
  // against 32)
  const bool int_eval = L > 1 && s->d_coef_fz && n <= 32 && (s->eval_variant == -1 || s->eval_variant == 2);
  const size_t ab = int_eval ? (size_t)(L == 4 ? 17 : 11) * 4 * m : cxb;  // bytes of one entry of A and R
  size_t o_xp = take(n * cxb), o_hx = take((size_t)cap * n * cxb), o_ht = take((size_t)cap * m * 8),
         o_A = take((size_t)n * (n + nrhs) * ab), o_R = take((size_t)n * (n + nrhs) * ab), o_dx = take(n * cxb),
         o_tx = P.predictor > 0 ? take((size_t)cap * n * cxb) : 0, o_tdx = P.predictor > 0 ? take(n * cxb) : 0,
         o_ntan = take(m),
         o_h = take(m * 8), o_t1 = take(m * 8), o_it = take(m), o_ph = take(m), o_nh = take(m),
         o_steps = take(m * 4), o_rej = take(m * 4), o_newt = take(m * 4), o_idx0 = take((m + 1) * 4),
         o_idx1 = take((m + 1) * 4), o_cnt = take(4 * 4), o_deg = take(n * 4), o_ldx = take(m * 8),
         o_lres = take(m * 8), o_lits = take(m), o_lrej = take(m), o_fb = take(m),
         o_img = IO.mlp ? take(mlp_image_bytes()) : 0;
  int rc = ensure_track_ws(s, off, st);
  if (rc != HT_OK) return rc;
  char* w = (char*)s->d_track_ws;
  TrackArgs a;
  a.poly_off = s->d_poly_off;
  a.mon_off = s->d_mon_off;
  a.pairs = s->d_pairs;
  a.coef = s->d_coef;
  a.cfz = s->d_coef_fz;
  a.clg = s->d_coef_lg;
  a.int_eval = int_eval;
  a.deg = (const int32_t*)(w + o_deg);
  a.gamma_re = gamma[0];
  a.gamma_im = gamma[1];
  a.n = n;
  a.m = m;
  a.prm = TrackPrm{P.h0, P.h_min, P.h_max, P.f_up, P.f_down, P.tol_dx, P.tol_res, P.tol_polish, P.r_div,
                   P.newton_max, P.polish_max, P.max_steps, P.max_order, deg_max, P.predictor};
  a.x = x_end;
  a.xp = (double*)(w + o_xp);
  a.hx = (double*)(w + o_hx);
  a.ht = (double*)(w + o_ht);
  a.A = (double*)(w + o_A);
  a.R = (double*)(w + o_R);
  a.dx = (double*)(w + o_dx);
  a.tx = P.predictor > 0 ? (double*)(w + o_tx) : nullptr;
  a.tdx = P.predictor > 0 ? (double*)(w + o_tdx) : nullptr;
  a.ntan = (int8_t*)(w + o_ntan);
  a.t = t_end;
  a.h = (double*)(w + o_h);
  a.t1 = (double*)(w + o_t1);
  a.status = status;
  a.it = (int8_t*)(w + o_it);
  a.phase = (int8_t*)(w + o_ph);
  a.nh = (int8_t*)(w + o_nh);
  a.steps = steps ? steps : (int32_t*)(w + o_steps);
  a.rejects = (int32_t*)(w + o_rej);
  a.newton = (int32_t*)(w + o_newt);
  int32_t* idx[2] = {(int32_t*)(w + o_idx0), (int32_t*)(w + o_idx1)};
  int32_t* cnt[2] = {(int32_t*)(w + o_cnt), (int32_t*)(w + o_cnt) + 1};
  // group queues of the track launches (alternating; each compaction zeroes
  // the next launch's), zero before the first
  int32_t* queue[2] = {(int32_t*)(w + o_cnt) + 2, (int32_t*)(w + o_cnt) + 3};
  {
    cudaError_t eq = cudaMemsetAsync(queue[0], 0, 2 * sizeof(int32_t), st);
    if (eq != cudaSuccess) return cuda_fail(eq, "ht_track_paths: queue");
  }
  a.idx0 = idx[0];
  a.count0 = cnt[0];
  a.last_dx = (double*)(w + o_ldx);
  a.last_res = (double*)(w + o_lres);
  a.last_its = (int8_t*)(w + o_lits);
  a.last_rej = (int8_t*)(w + o_lrej);
  a.fallback = (int8_t*)(w + o_fb);
  a.init_rec = IO.init_records;
  a.trace = IO.trace;
  a.trace_count = (unsigned long long*)IO.trace_count;
  a.trace_cap = IO.trace_capacity;
  a.trace_stride = IO.trace_stride > 0 ? IO.trace_stride : 1;
  a.mlp_img = IO.mlp ? (const void*)(w + o_img) : nullptr;
  a.newton_out = IO.newton_out;
  a.fallback_steps = IO.fallback_steps;
  a.rho_min = IO.rho_min;
  a.rho_max = IO.rho_max;
  a.alpha_max = IO.mlp ? IO.alpha_max : 0.0;
  a.x0 = IO.init_records ? nullptr : x0;
  a.x0_limbs = x0_limbs;
  a.polish_only = IO.polish_only ? 1 : 0;
  if (a.x0 && x0_limbs != L) {  // the widening copy in init_kernel must not read what it writes
    const char *b0 = (const char*)x0, *e0 = b0 + (size_t)n * 2 * x0_limbs * m * sizeof(double);
    const char *b1 = (const char*)x_end, *e1 = b1 + n * cxb;
    if (b0 < e1 && b1 < e0) return set_error(HT_EINVAL, "ht_track_paths_ex: x0 with fewer limbs overlaps x_end");
  }
  cudaError_t e = cudaMemcpyAsync((void*)a.deg, start_deg, n * sizeof(int32_t), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "ht_track_paths: upload degrees");
  if (IO.init_records) {
    // the init kernel takes every path's state from its record
  } else if (x0) {
    // the init kernel copies (and widens) x0 into x_end
  } else {
    rc = by_limbs(L, [&](auto c) { return launch_start_l<decltype(c)::value>(n, a.deg, first_path, m, x_end, st); });
    if (rc != HT_OK) return rc;
  }
  rc = by_limbs(L, [&](auto c) { return launch_init_l<decltype(c)::value>(a, st); });
  if (rc != HT_OK) return rc;
  if (IO.mlp) {
    rc = launch_mlp_image(w + o_img, mlp_bf16(IO.mlp), mlp_master(IO.mlp), st);
    if (rc != HT_OK) return rc;
  }

  // Rounds: [track (iters Newton steps) ; compact] x rounds_per_sync per host
  // read of the active count, captured once per team size as a CUDA graph.
  const int iters = P.iters_per_launch > 0 ? P.iters_per_launch : (s->track_iters > 0 ? s->track_iters : 4);
  const int rounds = P.rounds_per_sync > 0 ? P.rounds_per_sync : 8;
  // Team size: the largest power of two up to 8 warps and n.  More warps per
  // group means fewer groups in flight for the same FP64 issue rate, so the
  // per-path workspace (A and R, 2 n (n + 1) complex entries per path) of the
  // resident groups stays in L2; on the n = 16 double workload 8 warps beat 1
  // warp by 1.7x and 4 warps by 4 %.
  // While fewer groups are active than there are SMs (a small batch, or the
  // tail of any run), a double or double-double group with more than 8 MGS
  // columns gets 16 warps: every SM then runs at most one group, and the
  // wider team shortens that group's round (fewer columns and polynomials per
  // warp).  QD (200+ registers a thread) keeps 8.
  const bool wide_ok = L <= 2 && n + 1 > 8;
  auto pick_team = [&](int64_t active) {
    if (P.team_warps > 0) return P.team_warps;
    int t = 1;
    if (s->track_team > 0 && s->track_team <= 16) {
      t = s->track_team;
    } else {
      while (t < 8 && 2 * t <= n) t *= 2;
    }
    if (t == 8 && wide_ok && (active + 31) / 32 < sm_count()) t = 16;
    return t;
  };
  int64_t active = m;
  int64_t max_loops = (int64_t)P.max_steps * (P.newton_max + 1) + P.polish_max + 8;
  int64_t loops = 0;
  int launches = 0, syncs = 0;
  drop_graphs(s);
  while (active > 0) {
    int team = pick_team(active);
    int64_t groups = (active + 31) / 32;
    // graph for this (team, iters, rounds, workspace, outputs) configuration
    ht_system::GraphEntry* ge = nullptr;
    for (auto& g : s->graphs)
      if (g.team == team && g.key_a == (const void*)x_end && g.key_b == (const void*)status && g.groups >= groups) ge = &g;
    if (!ge) {
      cudaGraph_t graph;
      cudaStream_t cs;
      e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(e, "ht_track_paths: capture stream");
      e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        return cuda_fail(e, "ht_track_paths: begin capture");
      }
      int crc = HT_OK;
      for (int r = 0; r < rounds && crc == HT_OK; ++r) {
        TrackArgs ar = a;
        ar.idx_in = idx[r & 1];
        ar.count_in = cnt[r & 1];
        ar.queue = queue[r & 1];
        ar.iters = iters;
        crc = by_limbs(L, [&](auto c) { return launch_track_l<decltype(c)::value>(ar, team, groups, cs); });
        if (crc == HT_OK)
          crc = launch_compact(idx[r & 1], cnt[r & 1], status, idx[(r + 1) & 1], cnt[(r + 1) & 1], cs,
                               queue[(r + 1) & 1]);
      }
      graph = nullptr;
      cudaError_t ee = cudaStreamEndCapture(cs, &graph);
      cudaStreamDestroy(cs);
      if (crc != HT_OK || ee != cudaSuccess) {
        // a launch that failed inside the capture invalidates it; ending the
        // capture then records that as the thread's last error, which would
        // otherwise surface in the next call's launch checks
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return crc != HT_OK ? crc : cuda_fail(ee, "ht_track_paths: end capture");
      }
      ht_system::GraphEntry g;
      g.team = team;
      g.groups = groups;
      g.key_a = x_end;
      g.key_b = status;
      ee = cudaGraphInstantiate(&g.exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ee != cudaSuccess) return cuda_fail(ee, "ht_track_paths: instantiate");
      s->graphs.push_back(g);
      ge = &s->graphs.back();
    }
    e = cudaGraphLaunch(ge->exec, st);
    if (e != cudaSuccess) return cuda_fail(e, "ht_track_paths: graph launch");
    launches += 2 * rounds;
    e = cudaMemcpyAsync(s->h_count, cnt[0], sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "ht_track_paths: read active count");
    ++syncs;
    active = s->h_count[0];
    loops += (int64_t)rounds * iters;
    if (loops > max_loops && active > 0) return set_error(HT_ETIMEOUT, "ht_track_paths: paths still active after %lld Newton rounds", (long long)loops);
  }
  if (IO.last_dx_out) e = cudaMemcpyAsync(IO.last_dx_out, a.last_dx, m * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && IO.last_res_out)
    e = cudaMemcpyAsync(IO.last_res_out, a.last_res, m * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "ht_track_paths: last norms");
  if (stats) {
    std::vector<int8_t> hs(m);
    std::vector<int32_t> hst(m), hrj(m), hnw(m);
    e = cudaMemcpyAsync(hs.data(), status, m, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hst.data(), a.steps, m * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hrj.data(), a.rejects, m * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hnw.data(), a.newton, m * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "ht_track_paths: stats");
    for (int64_t q = 0; q < m; ++q) {
      stats->converged += hs[q] == 1;
      stats->failed += hs[q] == -1;
      stats->diverged += hs[q] == -2;
      stats->steps += hst[q];
      stats->rejects += hrj[q];
      stats->newton += hnw[q];
    }
    stats->launches = launches;
    stats->syncs = syncs;
    stats->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  }
  return HT_OK;
}

}  // extern "C"

extern "C" {

int ht_tune_track(ht_system* s, const int32_t* start_deg, const double* gamma, int64_t n_paths, const ht_params* p,
                  int* team_warps, int* iters_per_launch, double* best_ms, void* stream) {
  clear_error();
  if (!s || n_paths < 1 || n_paths > 0x7fffffff) return set_error(HT_EINVAL, "ht_tune_track: bad arguments");
  const int n = s->nv, L = s->limbs;
  ht_params P;
  if (p)
    P = *p;
  else
    ht_default_params(L, &P);
  const size_t bx = (size_t)n * 2 * L * n_paths * sizeof(double), bt = (size_t)n_paths * sizeof(double);
  char* buf = nullptr;
  cudaError_t e = cudaMalloc((void**)&buf, bx + bt + (size_t)n_paths + 512);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(HT_ENOMEM, "ht_tune_track: output buffers");
  }
  double* x = (double*)buf;
  double* t = (double*)(buf + bx);
  int8_t* st = (int8_t*)(buf + bx + bt);
  const int saved_team = s->track_team, saved_iters = s->track_iters;
  double best = 1e300;
  int bt_team = 0, bt_iters = 0, rc = HT_OK;
  const int teams[5] = {1, 2, 4, 8, 16}, its[3] = {2, 4, 8};
  for (int a = 0; a < 5 && rc == HT_OK; ++a) {
    if (teams[a] > 1 && teams[a] > n) continue;
    if (teams[a] > 8 && (L == 4 || n + 1 <= 8)) continue;  // wide teams: D and DD with more than 8 columns
    for (int b = 0; b < 3 && rc == HT_OK; ++b) {
      ht_params Q = P;
      Q.team_warps = teams[a];
      Q.iters_per_launch = its[b];
      ht_stats stats;
      rc = ht_track_paths_ex(s, start_deg, gamma, n_paths, 0, nullptr, &Q, x, st, t, nullptr, &stats, nullptr, stream);
      if (rc == HT_OK && stats.ms < best) {
        best = stats.ms;
        bt_team = teams[a];
        bt_iters = its[b];
      }
    }
  }
  cudaFree(buf);
  if (rc != HT_OK) {
    s->track_team = saved_team;
    s->track_iters = saved_iters;
    return rc;
  }
  s->track_team = bt_team;
  s->track_iters = bt_iters;
  if (team_warps) *team_warps = bt_team;
  if (iters_per_launch) *iters_per_launch = bt_iters;
  if (best_ms) *best_ms = best;
  return HT_OK;
}

int ht_track_paths(ht_system* s, const int32_t* start_deg, const double* gamma, int64_t n_paths, int64_t first_path,
                   const double* x0, const ht_params* p, double* x_end, int8_t* status, double* t_end, int32_t* steps,
                   ht_stats* stats, void* stream) {
  return ht_track_paths_ex(s, start_deg, gamma, n_paths, first_path, x0, p, x_end, status, t_end, steps, stats,
                           nullptr, stream);
}

int ht_step_labels(ht_system* s, const int32_t* start_deg, const double* gamma, const ht_params* prm, int64_t n_rec,
                   const double* records, int n_mult, const double* mults, int newton_max, float* labels,
                   void* stream) {
  clear_error();
  if (!s || !prm || n_rec < 0 || n_mult < 1 || n_mult > 64 || !mults || newton_max < 1)
    return set_error(HT_EINVAL, "ht_step_labels: bad arguments");
  for (int j = 0; j < n_mult; ++j)
    if (!(mults[j] > 0)) return set_error(HT_EINVAL, "ht_step_labels: multipliers must be positive");
  if (n_rec == 0) return HT_OK;
  if (!records || !labels || !is_device_ptr(records) || !is_device_ptr(labels))
    return set_error(HT_EINVAL, "ht_step_labels: buffers must be device memory");
  const int n = s->nv, L = s->limbs;
  const int64_t R = rec_size(n, L, prm->max_order + 1), P = n_rec * n_mult;
  if (P > 0x7fffffff) return set_error(HT_EINVAL, "ht_step_labels: too many probes");
  cudaStream_t st = (cudaStream_t)stream;
  size_t b_rec = (size_t)P * R * 8, b_x = (size_t)n * 2 * L * P * 8, b_t = (size_t)P * 8, b_m = 64 * 8,
         b_k = ((size_t)P * 4 + 255) / 256 * 256;
  char* buf = nullptr;
  cudaError_t e = cudaMalloc((void**)&buf, b_rec + b_x + b_t + b_k + (size_t)P + b_m + 1024);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(HT_ENOMEM, "ht_step_labels: probe workspace");
  }
  double* prec = (double*)buf;
  double* px = (double*)(buf + b_rec);
  double* pt = (double*)(buf + b_rec + b_x);
  double* pm = (double*)(buf + b_rec + b_x + b_t);
  int32_t* pk = (int32_t*)(buf + b_rec + b_x + b_t + b_m);
  int8_t* pst = (int8_t*)(buf + b_rec + b_x + b_t + b_m + b_k);
  int rc = HT_OK;
  e = cudaMemcpyAsync(pm, mults, n_mult * 8, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) rc = cuda_fail(e, "ht_step_labels");
  if (rc == HT_OK) {
    probe_records_kernel<<<1024, 256, 0, st>>>(records, n_rec, R, n_mult, pm, prec);
    ht_params pp = *prm;
    pp.max_steps = 1;
    pp.newton_max = newton_max;
    pp.polish_max = 0;
    pp.h_min = 1e-300;
    ht_track_io io;
    std::memset(&io, 0, sizeof io);
    io.init_records = prec;
    io.newton_out = pk;
    rc = ht_track_paths_ex(s, start_deg, gamma, P, 0, nullptr, &pp, px, pst, pt, nullptr, nullptr, &io, stream);
  }
  if (rc == HT_OK) {
    labels_kernel<<<256, 256, 0, st>>>(records, n_rec, R, n, L, prm->max_order + 1, n_mult, pm, pt, pk, px, labels);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "ht_step_labels");
  }
  cudaFree(buf);
  return rc;
}

int64_t ht_record_size(int n, int limbs, int max_order) {
  if (n < 1 || (limbs != 1 && limbs != 2 && limbs != 4) || max_order < 0 || max_order > 7) return -1;
  return rec_size(n, limbs, max_order + 1);
}

int ht_step_features(int n, int limbs, int max_order, int newton_max, int64_t n_rec, const double* records,
                     float* features, void* stream) {
  clear_error();
  if (ht_record_size(n, limbs, max_order) < 0 || newton_max < 1 || n_rec < 0)
    return set_error(HT_EINVAL, "ht_step_features: bad arguments");
  if (n_rec == 0) return HT_OK;
  if (!records || !features || !is_device_ptr(records) || !is_device_ptr(features))
    return set_error(HT_EINVAL, "ht_step_features: buffers must be device memory");
  cudaStream_t st = (cudaStream_t)stream;
  return by_limbs(limbs, [&](auto c) {
    return launch_features_l<decltype(c)::value>(records, n_rec, n, max_order + 1, newton_max, features, st);
  });
}

}  // extern "C"
