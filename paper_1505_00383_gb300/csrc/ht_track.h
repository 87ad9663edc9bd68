// Internal interface of the tracker kernels (ht_track.cu, one object per
// precision) to the host driver (ht_track_host.cu).
#pragma once
#include <cuda_runtime.h>

#include <cuda_bf16.h>

#include <cstdint>

namespace ht {

// Step-start record (doubles): a 16-double header
//   [0] path id  [1] t  [2] h  [3] nh  [4] |dx| of the last round  [5] |h| of
//   the last round  [6] rounds of the last step  [7] last step rejected
//   [8..15] zero
// then t of the cap history points, then the history points [cap][n][2][L]
// (cap = max_order + 1, oldest first; entries past nh are zero).
constexpr int REC_HDR = 16;
inline __host__ __device__ int64_t rec_size(int n, int L, int cap) { return REC_HDR + cap + (int64_t)cap * n * 2 * L; }
constexpr int FEAT = 16;

struct TrackPrm {
  double h0, h_min, h_max, f_up, f_down, tol_dx, tol_res, tol_polish, r_div;
  int newton_max, polish_max, max_steps, max_order, deg_max;
  int predictor;  // 0 extrapolation, 1 Euler, 2 cubic Hermite on tangents
};

// Device pointers of the homotopy and of the per-path state, all paths' values
// of one entry contiguous ([entry][2][L][m] for complex data, [m] for scalars).
struct TrackArgs {
  const int32_t* poly_off;
  const int32_t* mon_off;
  const uint16_t* pairs;
  const double* coef;
  const void* cfz;     // coefficients in the integer format (mpi::fz<W>), for int_eval
  const float* clg;    // log2 |c|
  int int_eval;        // DD/QD: evaluate f on the integer pipe
  const int32_t* deg;  // start system degrees [n]
  double gamma_re, gamma_im;
  int n;
  int64_t m;
  int iters;
  TrackPrm prm;
  double* x;   // [n]     accepted point (the caller's x_end)
  double* xp;  // [n]     working point
  double* hx;  // [cap][n] accepted history, oldest first (cap = max_order + 1)
  double* ht;  // [cap]   their t values
  double* A;   // [n][n+nrhs] [J | -h (| -dh/dt)], then Q
  double* R;   // [n][n+nrhs] triangular factor, 1/r_qq on the diagonal
  double* dx;  // [n]
  double* tx;  // [cap][n] tangents of the history points (predictor > 0)
  double* tdx; // [n]     tangent solved in the latest Newton round
  int8_t* ntan;  // history points, most recent first, that carry a tangent
  double* t;   // the caller's t_end
  double* h;
  double* t1;
  int8_t* status;  // the caller's status
  int8_t* it;
  int8_t* phase;
  int8_t* nh;
  int32_t* steps;
  int32_t* rejects;
  int32_t* newton;
  int32_t* newton_out;     // per-path Newton rounds ([m]) or nullptr
  const double* x0;        // caller's start points ([n][2][x0_limbs][m]) or nullptr
  int x0_limbs;
  int polish_only;         // start every path at t = 1 in the polish phase
  const int32_t* idx_in;   // active path indices of this launch
  const int32_t* count_in; // their number (device)
  int32_t* queue;          // next 32-path group to take (device; zero at launch)
  int32_t* idx0;           // init: identity index list
  int32_t* count0;
  // last step summary (features of the learned step) and learned-step state
  double* last_dx;
  double* last_res;
  int8_t* last_its;
  int8_t* last_rej;
  int8_t* fallback;        // plain steps left after a rejected learned step
  // optional: start from records, record step starts, learned proposals
  const double* init_rec;  // [m][rec] or nullptr
  double* trace;           // [trace_cap][rec] or nullptr
  unsigned long long* trace_count;
  int64_t trace_cap;
  int trace_stride;
  const void* mlp_img;     // network image (MlpSmem layout, device memory); nullptr: plain rule
  int fallback_steps;
  double rho_min, rho_max;
  double alpha_max;        // learned tangent correction clamp (0: off)
};

template <int L>
int launch_start_l(int n, const int32_t* d_deg, int64_t first, int64_t count, double* x, cudaStream_t st);
template <int L>
int launch_mgs_l(double* A, double* R, double* x, int rows, int cols, int64_t n_sys, int variant, cudaStream_t st);
template <int L>
int launch_init_l(const TrackArgs& a, cudaStream_t st);
template <int L>
int launch_track_l(const TrackArgs& a, int team, int64_t max_groups, cudaStream_t st);
template <int L>
int track_occupancy_l(int team);
template <int L>
int launch_features_l(const double* rec, int64_t n_rec, int n, int cap, int newton_max, float* feat, cudaStream_t st);
// Start points of paths first + ids[q] for q < *count (x: [n][2][L][cap]).
template <int L>
int launch_start_at_l(int n, const int32_t* d_deg, int64_t first, const int32_t* ids, const int32_t* count,
                      int64_t cap, double* x, cudaStream_t st);
// Entry q of (xs [n][2][L][cap], ss, ts) into path ids[q] of (xd [n][2][L][m], sd, td), q < *count.
template <int L>
int launch_scatter_l(int n, const int32_t* ids, const int32_t* count, int64_t cap, const double* xs, const int8_t* ss,
                     const double* ts, double* xd, int8_t* sd, double* td, int64_t m, cudaStream_t st);
int launch_mlp_image(void* img, const __nv_bfloat16* wbf, const float* master, cudaStream_t st);
size_t mlp_image_bytes();
// Stable compaction of idx_in[0..*count_in) to the paths with status 0;
// reset (if given) is set to zero as well (the next launch's group queue).
int launch_compact(const int32_t* idx_in, const int32_t* count_in, const int8_t* status, int32_t* idx_out,
                   int32_t* count_out, cudaStream_t st, int32_t* reset = nullptr);

}  // namespace ht
