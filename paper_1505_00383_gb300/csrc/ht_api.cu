// C ABI entry points: argument checks, system upload, dispatch.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include <cmath>

#include "ht_internal.h"
#include "ht_mpi.cuh"

namespace ht {

static thread_local std::string g_err;

int set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}
void clear_error() { g_err.clear(); }
int cuda_fail(cudaError_t e, const char* what) {
  return set_error(HT_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}
bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}
int launch_evaldiff_range(const ht_system* s, int64_t n_pts, int j0, int j1, const double* x, double* val,
                          double* jac, cudaStream_t st) {
  switch (s->limbs) {
    case 1: return launch_evaldiff_l<1>(s, n_pts, j0, j1, x, val, jac, st);
    case 2: return launch_evaldiff_l<2>(s, n_pts, j0, j1, x, val, jac, st);
    case 4: return launch_evaldiff_l<4>(s, n_pts, j0, j1, x, val, jac, st);
  }
  return set_error(HT_EINVAL, "ht_eval_diff: limbs=%d", s->limbs);
}
int launch_evaldiff(const ht_system* s, int64_t n_pts, const double* x, double* val, double* jac, cudaStream_t st) {
  // the three-kernel organisation keeps its workspace in the system, a cache
  // that does not change what the system is
  if (s->eval_variant == 3) return run_unfused(const_cast<ht_system*>(s), n_pts, x, val, jac, nullptr, st);
  return launch_evaldiff_range(s, n_pts, 0, s->np, x, val, jac, st);
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

}  // namespace ht

using namespace ht;

extern "C" {

const char* ht_last_error(void) { return g_err.c_str(); }

int ht_create_system(int n_vars, int n_polys, const int32_t* n_terms, const int8_t* exps, const double* coef,
                     int limbs, ht_system** out) {
  clear_error();
  if (!out) return set_error(HT_EINVAL, "ht_create_system: out is NULL");
  *out = nullptr;
  if (n_vars < 1 || n_vars > 255) return set_error(HT_EINVAL, "ht_create_system: n_vars=%d not in 1..255", n_vars);
  if (n_polys < 1) return set_error(HT_EINVAL, "ht_create_system: n_polys=%d < 1", n_polys);
  if (limbs != 1 && limbs != 2 && limbs != 4) return set_error(HT_EINVAL, "ht_create_system: limbs=%d", limbs);
  if (!n_terms || !exps || !coef) return set_error(HT_EINVAL, "ht_create_system: NULL array");
  ht_system* s = new (std::nothrow) ht_system();
  if (!s) return set_error(HT_ENOMEM, "ht_create_system: host allocation");
  s->nv = n_vars;
  s->np = n_polys;
  s->limbs = limbs;
  cudaGetDevice(&s->device);
  s->h_poly_off.assign(n_polys + 1, 0);
  for (int j = 0; j < n_polys; ++j) {
    if (n_terms[j] < 1) {
      delete s;
      return set_error(HT_EINVAL, "ht_create_system: n_terms[%d]=%d < 1", j, n_terms[j]);
    }
    s->h_poly_off[j + 1] = s->h_poly_off[j] + n_terms[j];
  }
  s->M = s->h_poly_off[n_polys];
  s->n_terms.assign(n_terms, n_terms + n_polys);
  s->exps.assign(exps, exps + s->M * n_vars);
  s->coef.assign(coef, coef + s->M * 2 * limbs);
  s->h_mon_off.assign(s->M + 1, 0);
  for (int64_t m = 0; m < s->M; ++m) {
    int k = 0, deg = 0;
    for (int i = 0; i < n_vars; ++i) {
      int a = exps[m * n_vars + i];
      if (a < 0) {
        delete s;
        return set_error(HT_EINVAL, "ht_create_system: negative exponent at monomial %lld", (long long)m);
      }
      if (a > 0) {
        s->h_pairs.push_back((uint16_t)(i | (a << 8)));
        ++k;
        deg += a;
        if (a > s->max_exp) s->max_exp = a;
      }
    }
    for (int c = 0; c < 2 * limbs; ++c) {
      double v = coef[m * 2 * limbs + c];
      if (!(v == v) || v - v != 0.0) {
        delete s;
        return set_error(HT_EINVAL, "ht_create_system: coefficient of monomial %lld is not finite", (long long)m);
      }
    }
    if (k > 64) {
      delete s;
      return set_error(HT_EUNSUPPORTED, "ht_create_system: monomial %lld has %d variables (max 64)", (long long)m, k);
    }
    if (k > s->max_k) s->max_k = k;
    if (deg > s->max_deg) s->max_deg = deg;
    s->h_mon_off[m + 1] = (int32_t)s->h_pairs.size();
  }
  s->n_pairs = (int64_t)s->h_pairs.size();
  // one allocation: coef | poly_off | mon_off | pairs
  size_t b_coef = (size_t)s->M * 2 * limbs * sizeof(double);
  size_t b_poly = (size_t)(n_polys + 1) * sizeof(int32_t);
  size_t b_mon = (size_t)(s->M + 1) * sizeof(int32_t);
  size_t b_pairs = (size_t)(s->n_pairs + 1) * sizeof(uint16_t);
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  size_t total = up(b_coef) + up(b_poly) + up(b_mon) + up(b_pairs);
  cudaError_t e = cudaMalloc(&s->d_block, total);
  if (e != cudaSuccess) {
    delete s;
    cudaGetLastError();
    return set_error(HT_ENOMEM, "ht_create_system: cudaMalloc(%zu): %s", total, cudaGetErrorString(e));
  }
  char* base = (char*)s->d_block;
  s->d_coef = (double*)base;
  s->d_poly_off = (int32_t*)(base + up(b_coef));
  s->d_mon_off = (int32_t*)(base + up(b_coef) + up(b_poly));
  s->d_pairs = (uint16_t*)(base + up(b_coef) + up(b_poly) + up(b_mon));
  e = cudaMemcpy(s->d_coef, coef, b_coef, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->d_poly_off, s->h_poly_off.data(), b_poly, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->d_mon_off, s->h_mon_off.data(), b_mon, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && s->n_pairs)
    e = cudaMemcpy(s->d_pairs, s->h_pairs.data(), s->n_pairs * sizeof(uint16_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(s->d_block);
    delete s;
    return cuda_fail(e, "ht_create_system: upload");
  }
  // integer-format coefficients for the integer evaluation variant
  {
    const size_t zsz = limbs == 1 ? sizeof(mpi::fz<3>) : (limbs == 2 ? sizeof(mpi::fz<5>) : sizeof(mpi::fz<8>));
    std::vector<unsigned char> hz((size_t)s->M * zsz);
    std::vector<float> hl(s->M);
    for (int64_t m = 0; m < s->M; ++m) {
      const double* re = coef + m * 2 * limbs;
      const double* im = re + limbs;
      if (limbs == 1) {
        mpi::fz<3> z = mpi::from_doubles<3, 1>(re, im);
        std::memcpy(&hz[m * zsz], &z, zsz);
      } else if (limbs == 2) {
        mpi::fz<5> z = mpi::from_doubles<5, 2>(re, im);
        std::memcpy(&hz[m * zsz], &z, zsz);
      } else {
        mpi::fz<8> z = mpi::from_doubles<8, 4>(re, im);
        std::memcpy(&hz[m * zsz], &z, zsz);
      }
      const double mod = std::hypot(re[0], im[0]);
      hl[m] = mod == 0.0 ? -1000.0f : (float)std::log2(mod);
    }
    void* blk = nullptr;
    e = cudaMalloc(&blk, hz.size() + hl.size() * sizeof(float) + 256);
    if (e == cudaSuccess) {
      s->d_coef_fz = blk;
      s->d_coef_lg = (float*)((char*)blk + ((hz.size() + 255) & ~(size_t)255));
      e = cudaMemcpy(s->d_coef_fz, hz.data(), hz.size(), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(s->d_coef_lg, hl.data(), hl.size() * sizeof(float), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (s->d_coef_fz) cudaFree(s->d_coef_fz);
      cudaFree(s->d_block);
      delete s;
      return set_error(HT_ENOMEM, "ht_create_system: integer coefficients");
    }
  }
  *out = s;
  return HT_OK;
}

int ht_destroy_system(ht_system* s) {
  clear_error();
  if (!s) return HT_OK;
  cudaDeviceSynchronize();
  if (s->d_block) cudaFree(s->d_block);
  if (s->d_ws) cudaFree(s->d_ws);
  if (s->d_track_ws) cudaFree(s->d_track_ws);
  if (s->d_coef_fz) cudaFree(s->d_coef_fz);
  if (s->d_uf) cudaFree(s->d_uf);
  if (s->d_uf_ws) cudaFree(s->d_uf_ws);
  if (s->h_count) cudaFreeHost(s->h_count);
  for (auto& hs : s->host_streams)
    if (hs) cudaStreamDestroy(hs);
  for (auto& g : s->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  delete s;
  return HT_OK;
}

int ht_system_info(const ht_system* s, int* n_vars, int* n_polys, int* limbs, int64_t* n_monomials) {
  clear_error();
  if (!s) return set_error(HT_EINVAL, "ht_system_info: NULL system");
  if (n_vars) *n_vars = s->nv;
  if (n_polys) *n_polys = s->np;
  if (limbs) *limbs = s->limbs;
  if (n_monomials) *n_monomials = s->M;
  return HT_OK;
}

static int check_eval_args(const ht_system* s, int64_t n_pts, const void* x, const void* val, const void* jac,
                           bool device) {
  if (!s) return set_error(HT_EINVAL, "eval: NULL system");
  if (n_pts < 0) return set_error(HT_EINVAL, "eval: n_pts=%lld < 0", (long long)n_pts);
  if (n_pts == 0) return HT_OK;
  if (!x || !val || !jac) return set_error(HT_EINVAL, "eval: NULL buffer");
  if (((uintptr_t)x | (uintptr_t)val | (uintptr_t)jac) & 7)
    return set_error(HT_EINVAL, "eval: buffers must be 8-byte aligned");
  if (device && (!is_device_ptr(x) || !is_device_ptr(val) || !is_device_ptr(jac)))
    return set_error(HT_EINVAL, "eval: x, val and jac must be device memory of the current device");
  const size_t L = s->limbs;
  const char* xb = (const char*)x;
  size_t xbytes = (size_t)s->nv * 2 * L * n_pts * 8;
  const char* ob[2] = {(const char*)val, (const char*)jac};
  size_t obytes[2] = {(size_t)s->np * 2 * L * n_pts * 8, (size_t)s->np * s->nv * 2 * L * n_pts * 8};
  for (int i = 0; i < 2; ++i)
    if (xb < ob[i] + obytes[i] && ob[i] < xb + xbytes) return set_error(HT_EINVAL, "eval: x overlaps an output");
  return HT_OK;
}

int ht_eval_diff(const ht_system* s, int64_t n_pts, const double* x, double* val, double* jac, void* stream) {
  clear_error();
  int rc = check_eval_args(s, n_pts, x, val, jac, true);
  if (rc != HT_OK || n_pts == 0) return rc;
  return launch_evaldiff(s, n_pts, x, val, jac, (cudaStream_t)stream);
}

int ht_eval_diff_host(ht_system* s, int64_t n_pts, const double* x_host, double* val_host, double* jac_host,
                      void* stream) {
  clear_error();
  int rc = check_eval_args(s, n_pts, x_host, val_host, jac_host, false);
  if (rc != HT_OK || n_pts == 0) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  // Pipelined over blocks of polynomials: the points go to the device in one
  // copy; then one stream evaluates the blocks, each into one of up to three
  // slabs, while a second stream copies every finished slab back.  In the
  // point-fastest layouts a block of polynomials is a contiguous range of
  // val and of jac on both sides, so every copy back is one contiguous
  // transfer.  Events order the two streams: a slab's copy waits for its
  // evaluation, and the evaluation that reuses a slab waits for that slab's
  // previous copy, so the evaluations never wait for a copy still in flight
  // unless three are.  Blocks hold at least 8 polynomials (the
  // block-organised integer kernel deals polynomials to 8 warps); the
  // three-kernel variant takes one block.
  const size_t L = s->limbs;
  const int64_t rx = (int64_t)s->nv * 2 * L, rv = 2 * L, rj = (int64_t)s->nv * 2 * L;  // doubles per point per row
  int nb = s->np;
  if (s->eval_variant != 3) {
    nb = (s->np + 7) / 8;
    if (nb < 8) nb = 8;
    if (nb > s->np) nb = s->np;
  }
  const int n_blocks = (s->np + nb - 1) / nb;
  const int slots = n_blocks < 3 ? n_blocks : 3;
  const size_t b_x = (size_t)rx * n_pts * 8, b_slot = (size_t)nb * (rv + rj) * n_pts * 8;
  const size_t need = b_x + b_slot * slots;
  if (s->ws_bytes < need) {
    if (s->d_ws) {
      cudaDeviceSynchronize();
      cudaFree(s->d_ws);
      s->d_ws = nullptr;
      s->ws_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&s->d_ws, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_error(HT_ENOMEM, "ht_eval_diff_host: workspace of %zu bytes", need);
    }
    s->ws_bytes = need;
  }
  for (int k = 0; k < 2; ++k)
    if (!s->host_streams[k]) {
      cudaError_t e = cudaStreamCreateWithFlags(&s->host_streams[k], cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(e, "ht_eval_diff_host: stream");
    }
  cudaStream_t comp = s->host_streams[0], copy = s->host_streams[1];
  cudaEvent_t ev[7] = {};  // [0] ordering after the caller's stream, [1..3] evaluated, [4..6] copied
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 7 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);  // after the work already queued by the caller
  if (e == cudaSuccess) e = cudaStreamWaitEvent(comp, ev[0], 0);
  double* dx = (double*)s->d_ws;
  if (e == cudaSuccess) e = cudaMemcpyAsync(dx, x_host, b_x, cudaMemcpyHostToDevice, comp);
  for (int b = 0; b < n_blocks && rc == HT_OK && e == cudaSuccess; ++b) {
    const int j0 = b * nb, j1 = j0 + nb < s->np ? j0 + nb : s->np, k = b % slots;
    double* dv = (double*)((char*)s->d_ws + b_x + b_slot * k);
    double* dj = dv + (int64_t)nb * rv * n_pts;
    if (b >= slots) e = cudaStreamWaitEvent(comp, ev[4 + k], 0);  // the slab's previous copy is done
    if (e != cudaSuccess) break;
    rc = s->eval_variant == 3 ? launch_evaldiff(s, n_pts, dx, dv, dj, comp)
                              : launch_evaldiff_range(s, n_pts, j0, j1, dx, dv, dj, comp);
    if (rc != HT_OK) break;
    e = cudaEventRecord(ev[1 + k], comp);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(copy, ev[1 + k], 0);
    const size_t cv = (size_t)(j1 - j0) * rv * n_pts * 8, cj = (size_t)(j1 - j0) * rj * n_pts * 8;
    if (e == cudaSuccess) e = cudaMemcpyAsync(val_host + (int64_t)j0 * rv * n_pts, dv, cv, cudaMemcpyDeviceToHost, copy);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(jac_host + (int64_t)j0 * rj * n_pts, dj, cj, cudaMemcpyDeviceToHost, copy);
    if (e == cudaSuccess) e = cudaEventRecord(ev[4 + k], copy);
  }
  cudaError_t e2 = cudaStreamSynchronize(comp);
  cudaError_t e3 = cudaStreamSynchronize(copy);
  for (auto& x : ev)
    if (x) cudaEventDestroy(x);
  if (rc != HT_OK) return rc;
  if (e == cudaSuccess) e = e2 != cudaSuccess ? e2 : e3;
  if (e != cudaSuccess) return cuda_fail(e, "ht_eval_diff_host: copies");
  return HT_OK;
}

int ht_set_eval_config(ht_system* s, int variant, int threads) {
  clear_error();
  if (!s) return set_error(HT_EINVAL, "ht_set_eval_config: NULL system");
  if (variant < -1 || variant > 3) return set_error(HT_EINVAL, "ht_set_eval_config: variant=%d", variant);
  if (variant == 3 && (s->M > 65535 || (int64_t)s->np * (s->nv + 1) > 65535))
    return set_error(HT_EUNSUPPORTED, "ht_set_eval_config: the three-kernel variant takes at most 65,535 monomials and outputs");
  if (variant == 2 && s->nv > 64)
    return set_error(HT_EUNSUPPORTED, "ht_set_eval_config: the integer variant supports at most 64 variables");
  if (threads != 0 && threads != 64 && threads != 128 && threads != 256)
    return set_error(HT_EINVAL, "ht_set_eval_config: threads=%d (0, 64, 128 or 256)", threads);
  s->eval_variant = variant;
  s->eval_threads = threads;
  return HT_OK;
}

int ht_tune_eval(ht_system* s, int64_t n_pts, const double* x, double* val, double* jac, int reps, int* variant,
                 int* threads, float* best_ms, void* stream) {
  clear_error();
  int rc = check_eval_args(s, n_pts, x, val, jac, true);
  if (rc != HT_OK) return rc;
  if (n_pts == 0 || reps < 1) return set_error(HT_EINVAL, "ht_tune_eval: need n_pts > 0 and reps >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int variants[4] = {1, 0, 3, 2}, sizes[3] = {128, 64, 256};
  const bool int_ok = s->nv <= 64, uf_ok = s->M <= 65535 && (int64_t)s->np * (s->nv + 1) <= 65535;
  float best = 1e30f;
  int bv = 1, bt = 128;
  for (int vi = 0; vi < 4 && rc == HT_OK; ++vi)
    for (int ti = 0; ti < 3 && rc == HT_OK; ++ti) {
      if (variants[vi] == 2 && (!int_ok || ti == 1)) continue;  // integer limbs: 128 (per unit) or 256 (per block)
      if (variants[vi] == 3 && (!uf_ok || ti > 0)) continue;     // three kernels: one shape
      s->eval_variant = variants[vi];
      s->eval_threads = sizes[ti];
      rc = launch_evaldiff(s, n_pts, x, val, jac, st);  // warm-up
      cudaEventRecord(e0, st);
      for (int r = 0; r < reps && rc == HT_OK; ++r) rc = launch_evaldiff(s, n_pts, x, val, jac, st);
      cudaEventRecord(e1, st);
      cudaError_t e = cudaEventSynchronize(e1);
      float ms = 0;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess && rc == HT_OK) rc = cuda_fail(e, "ht_tune_eval");
      if (rc == HT_OK && ms / reps < best) {
        best = ms / reps;
        bv = variants[vi];
        bt = sizes[ti];
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  s->eval_variant = bv;
  s->eval_threads = bt;
  // leave the chosen configuration's results in val and jac
  if (rc == HT_OK) rc = launch_evaldiff(s, n_pts, x, val, jac, st);
  if (rc == HT_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "ht_tune_eval");
  }
  if (variant) *variant = bv;
  if (threads) *threads = bt;
  if (best_ms) *best_ms = best;
  return rc;
}

}  // extern "C"
