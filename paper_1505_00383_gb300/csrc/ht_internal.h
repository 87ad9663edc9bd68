// Host-side internals shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "ht.h"

// The "instructions" of Table tabmemory: monomial supports and coefficients,
// stored once on the device and read by all paths.
struct ht_system {
  int nv = 0, np = 0, limbs = 0, device = 0;
  int64_t M = 0, n_pairs = 0;
  int max_k = 0, max_exp = 0, max_deg = 0;
  int eval_variant = -1;         // 0 unrolled, 1 compact FP64 bodies, 2 integer limbs, -1 default
  int eval_threads = 0;          // CTA size of the evaluation kernel, 0 = default (128)
  int track_team = 0;            // tuned tracker team size and rounds per launch (0: defaults)
  int track_iters = 0;
  std::vector<int32_t> n_terms;  // host copies
  std::vector<int8_t> exps;
  std::vector<double> coef;
  std::vector<int32_t> h_poly_off, h_mon_off;
  std::vector<uint16_t> h_pairs;
  void* d_block = nullptr;       // one device allocation holding the arrays below
  int32_t* d_poly_off = nullptr; // [np + 1] monomial range of each polynomial
  int32_t* d_mon_off = nullptr;  // [M + 1] range of each monomial in d_pairs
  uint16_t* d_pairs = nullptr;   // variable | exponent << 8, variables increasing
  double* d_coef = nullptr;      // [M][2][L]
  void* d_coef_fz = nullptr;     // [M] coefficients in the integer format (L = 2, 4)
  float* d_coef_lg = nullptr;    // [M] log2 |c| (-1000 for zero)
  void* d_ws = nullptr;          // workspace for the host-buffer entry points
  size_t ws_bytes = 0;
  cudaStream_t host_streams[2] = {nullptr, nullptr};  // pipelined host-buffer evaluation
  void* d_track_ws = nullptr;    // per-path tracker state (grown on demand)
  size_t track_ws_bytes = 0;
  int32_t* h_count = nullptr;    // pinned host word: active paths after a round
  struct GraphEntry {            // captured rounds of the tracker for one team size
    int team = 0;
    int64_t groups = 0;
    const void* key_a = nullptr;
    const void* key_b = nullptr;
    cudaGraphExec_t exec = nullptr;
  };
  std::vector<GraphEntry> graphs;
  // three-kernel evaluation (ht_eval_diff_unfused): the output lists of the
  // sum kernel and the workspace, built on first use
  void* d_uf = nullptr;          // out_off [np (nv + 1) + 1] | out_slot [T] | out_exp [T] | slot_off [M + 1] (int32)
  int64_t uf_slots = 0;          // workspace entries per point: M (coefficients) + sum over monomials of k + 1
  int64_t uf_terms = 0;          // T: summands over all outputs
  void* d_uf_ws = nullptr;
  size_t uf_ws_bytes = 0;
};

namespace ht {

int set_error(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
void clear_error();
// True when p is device (or managed) memory of the current device.
bool is_device_ptr(const void* p);
int sm_count();

// Polynomials j0 .. j1 - 1 at n_pts points: val and jac receive them from
// their row 0 (val [j1 - j0][2][L][n_pts], jac [j1 - j0][nv][2][L][n_pts]).
template <int L>
int launch_evaldiff_l(const ht_system* s, int64_t n_pts, int j0, int j1, const double* x, double* val, double* jac,
                      cudaStream_t st);
int launch_evaldiff_range(const ht_system* s, int64_t n_pts, int j0, int j1, const double* x, double* val,
                          double* jac, cudaStream_t st);
int launch_evaldiff(const ht_system* s, int64_t n_pts, const double* x, double* val, double* jac,
                    cudaStream_t st);

// ht_eval_diff_unfused after argument checks (also ht_eval_diff with
// variant 3); stats may be NULL (then nothing blocks).
int run_unfused(ht_system* s, int64_t n_pts, const double* x, double* val, double* jac, ht_unfused_stats* stats,
                cudaStream_t st);

// The three kernels of ht_eval_diff_unfused on points p0 .. p0 + cc - 1 of
// x/val/jac (column stride n) through the workspace ws ([slots][2][L][cc]);
// with ev (6 events) the kernels are bracketed for timing.
template <int L>
int launch_unfused_l(const ht_system* s, int64_t n, int64_t p0, int64_t cc, const double* x, double* val,
                     double* jac, double* ws, cudaEvent_t* ev, cudaStream_t st);

}  // namespace ht
