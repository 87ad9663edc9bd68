// Mixed-precision tracking ("quality up", Sections 1 and 4.4 of Verschelde &
// Yu 2015: the speed of the device spent on accuracy).  Every path is
// tracked in a low precision; converged endpoints are refined by Newton's
// method in a high precision; the paths that failed, diverged or whose
// refinement did not converge are tracked again from their start points in
// the high precision.  The result is the high-precision run's up to the
// refinement of paths that both precisions track to the same root.
#include <chrono>
#include <cstring>
#include <vector>

#include "ht_internal.h"
#include "ht_track.h"

namespace ht {

template <typename F>
static int refine_by_limbs(int L, F f) {
  switch (L) {
    case 1: return f(std::integral_constant<int, 1>());
    case 2: return f(std::integral_constant<int, 2>());
    case 4: return f(std::integral_constant<int, 4>());
  }
  return set_error(HT_EINVAL, "limbs=%d must be 1, 2 or 4", L);
}

// keep[q] = 0 for the paths to track again (failed or diverged in the low
// precision, refinement not finite, or its last Newton update above
// tol max(1, |x|_inf)), 1 otherwise; ids[q] = q and ids[m] = m for the
// compaction that lists them.
__global__ void refine_select_kernel(int n, int L, int64_t m, const int8_t* __restrict__ st_lo,
                                     const int8_t* __restrict__ st_hi, const double* __restrict__ last_dx,
                                     const double* __restrict__ x, double tol, int8_t* __restrict__ keep,
                                     int32_t* __restrict__ ids) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += (int64_t)gridDim.x * blockDim.x) {
    double nx = 0.0;
    for (int i = 0; i < n; ++i) {
      const double re = x[((int64_t)(i * 2) * L) * m + q], im = x[((int64_t)(i * 2 + 1) * L) * m + q];
      nx = fmax(nx, sqrt(re * re + im * im));
    }
    const bool ok = st_lo[q] == 1 && st_hi[q] == 1 && last_dx[q] <= tol * fmax(1.0, nx);
    keep[q] = ok ? 1 : 0;
    ids[q] = (int32_t)q;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) ids[m] = (int32_t)m;
}

static double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace ht

using namespace ht;

extern "C" int ht_track_refined(ht_system* lo, ht_system* hi, const int32_t* start_deg, const double* gamma,
                                int64_t n_paths, int64_t first_path, const ht_params* p_lo, const ht_params* p_hi,
                                double* x_end, int8_t* status, double* t_end, ht_refine_stats* rs, void* stream) {
  clear_error();
  if (!lo || !hi) return set_error(HT_EINVAL, "ht_track_refined: NULL system");
  if (lo->nv != hi->nv || lo->np != hi->np || lo->M != hi->M || lo->limbs >= hi->limbs)
    return set_error(HT_EINVAL, "ht_track_refined: the two systems must have the same shape, lo in fewer limbs");
  if (lo->exps != hi->exps || lo->n_terms != hi->n_terms)
    return set_error(HT_EINVAL, "ht_track_refined: the two systems must have the same monomials");
  if (rs) std::memset(rs, 0, sizeof *rs);
  if (n_paths < 0 || n_paths > 0x7fffffff) return set_error(HT_EINVAL, "ht_track_refined: n_paths=%lld", (long long)n_paths);
  if (n_paths == 0) return HT_OK;
  if (!x_end || !status || !t_end || !is_device_ptr(x_end) || !is_device_ptr(status) || !is_device_ptr(t_end))
    return set_error(HT_EINVAL, "ht_track_refined: outputs must be device memory");
  const int n = lo->nv, Ll = lo->limbs, Lh = hi->limbs;
  const int64_t m = n_paths;
  ht_params Ph;
  if (p_hi)
    Ph = *p_hi;
  else
    ht_default_params(Lh, &Ph);
  if (Ph.polish_max < 1) return set_error(HT_EINVAL, "ht_track_refined: p_hi->polish_max must be >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  // workspace: low-precision points, statuses, t, last updates, selection
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t b_xl = up((size_t)n * 2 * Ll * m * 8), b_m8 = up((size_t)m * 8), b_m1 = up((size_t)m),
               b_ids = up((size_t)(m + 1) * 4), b_cnt = up(32 + (size_t)n * 4);
  char* w = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&w, b_xl + 2 * b_m8 + 2 * b_m1 + 2 * b_ids + b_cnt, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(HT_ENOMEM, "ht_track_refined: workspace");
  }
  double* x_lo = (double*)w;
  double* t_lo = (double*)(w + b_xl);
  double* ldx = (double*)(w + b_xl + b_m8);
  int8_t* s_lo = (int8_t*)(w + b_xl + 2 * b_m8);
  int8_t* keep = s_lo + b_m1;
  int32_t* ids_all = (int32_t*)(keep + b_m1);
  int32_t* ids = ids_all + b_ids / 4;
  int32_t* d_cnt = (int32_t*)((char*)ids + b_ids);
  int32_t* d_deg = d_cnt + 8;
  char* big = nullptr;  // re-track buffers, sized by the count
  int rc = HT_OK;
  int32_t count = 0;
  ht_stats sl;
  auto t0 = std::chrono::steady_clock::now();
  // 1. every path in the low precision
  rc = ht_track_paths_ex(lo, start_deg, gamma, m, first_path, nullptr, p_lo, x_lo, s_lo, t_lo, nullptr, &sl, nullptr,
                         stream);
  double ms_lo = ms_since(t0);
  // 2. refinement in the high precision, from the low-precision endpoints
  auto t1 = std::chrono::steady_clock::now();
  if (rc == HT_OK) {
    ht_track_io io;
    std::memset(&io, 0, sizeof io);
    io.x0_limbs = Ll;
    io.polish_only = 1;
    io.last_dx_out = ldx;
    rc = ht_track_paths_ex(hi, start_deg, gamma, m, 0, x_lo, &Ph, x_end, status, t_end, nullptr, nullptr, &io, stream);
  }
  if (rc == HT_OK) {
    int64_t blocks = (m + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    refine_select_kernel<<<(unsigned)blocks, 256, 0, st>>>(n, Lh, m, s_lo, status, ldx, x_end, Ph.tol_polish, keep,
                                                           ids_all);
    e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(e, "ht_track_refined: select");
  }
  if (rc == HT_OK) rc = launch_compact(ids_all, ids_all + m, keep, ids, d_cnt, st);
  if (rc == HT_OK) {
    e = cudaMemcpyAsync(&count, d_cnt, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "ht_track_refined: count");
  }
  double ms_ref = ms_since(t1);
  // 3. the selected paths again, from their start points, in the high precision
  auto t2 = std::chrono::steady_clock::now();
  if (rc == HT_OK && count > 0) {
    const size_t b_xh = up((size_t)n * 2 * Lh * count * 8);
    e = cudaMallocAsync((void**)&big, 2 * b_xh + up((size_t)count * 8) + up((size_t)count) + 256, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      rc = set_error(HT_ENOMEM, "ht_track_refined: re-track buffers");
    }
    double* x0 = (double*)big;
    double* xr = (double*)(big + b_xh);
    double* tr = (double*)(big + 2 * b_xh);
    int8_t* sr = (int8_t*)(big + 2 * b_xh + up((size_t)count * 8));
    if (rc == HT_OK) {
      e = cudaMemcpyAsync(d_deg, start_deg, n * sizeof(int32_t), cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) rc = cuda_fail(e, "ht_track_refined: degrees");
    }
    if (rc == HT_OK)
      rc = refine_by_limbs(Lh, [&](auto c) {
        return launch_start_at_l<decltype(c)::value>(n, d_deg, first_path, ids, d_cnt, count, x0, st);
      });
    if (rc == HT_OK)
      rc = ht_track_paths_ex(hi, start_deg, gamma, count, 0, x0, p_hi, xr, sr, tr, nullptr, nullptr, nullptr, stream);
    if (rc == HT_OK)
      rc = refine_by_limbs(Lh, [&](auto c) {
        return launch_scatter_l<decltype(c)::value>(n, ids, d_cnt, count, xr, sr, tr, x_end, status, t_end, m, st);
      });
  }
  if (rc == HT_OK) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "ht_track_refined");
  }
  double ms_re = ms_since(t2);
  if (rc == HT_OK && rs) {
    std::vector<int8_t> h(m);
    e = cudaMemcpy(h.data(), status, m, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "ht_track_refined: statuses");
    } else {
      for (int64_t q = 0; q < m; ++q) {
        rs->converged += h[q] == 1;
        rs->failed += h[q] == -1;
        rs->diverged += h[q] == -2;
      }
      rs->lo_converged = sl.converged;
      rs->retracked = count;
      rs->ms_lo = ms_lo;
      rs->ms_refine = ms_ref;
      rs->ms_retrack = ms_re;
    }
  }
  if (big) cudaFreeAsync(big, st);
  cudaFreeAsync(w, st);
  if (rc == HT_OK) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "ht_track_refined: free");
  }
  return rc;
}
