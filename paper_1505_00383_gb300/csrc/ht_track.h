// Internal interface of the tracker kernels (ht_track.cu, one object per
// precision) to the host driver (ht_track_host.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace ht {

struct TrackPrm {
  double h0, h_min, h_max, f_up, f_down, tol_dx, tol_res, tol_polish, r_div;
  int newton_max, polish_max, max_steps, max_order, deg_max;
};

// Device pointers of the homotopy and of the per-path state, all paths' values
// of one entry contiguous ([entry][2][L][m] for complex data, [m] for scalars).
struct TrackArgs {
  const int32_t* poly_off;
  const int32_t* mon_off;
  const uint16_t* pairs;
  const double* coef;
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
  double* A;   // [n][n+1] [J | -h], then Q
  double* R;   // [n][n+1] triangular factor, 1/r_qq on the diagonal
  double* dx;  // [n]
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
  const int32_t* idx_in;   // active path indices of this launch
  const int32_t* count_in; // their number (device)
  int32_t* idx0;           // init: identity index list
  int32_t* count0;
};

template <int L>
int launch_start_l(int n, const int32_t* d_deg, int64_t first, int64_t count, double* x, cudaStream_t st);
template <int L>
int launch_mgs_l(double* A, double* R, double* x, int rows, int cols, int64_t n_sys, cudaStream_t st);
template <int L>
int launch_init_l(const TrackArgs& a, cudaStream_t st);
template <int L>
int launch_track_l(const TrackArgs& a, int team, int64_t max_groups, cudaStream_t st);
template <int L>
int track_occupancy_l(int team);
int launch_compact(const int32_t* idx_in, const int32_t* count_in, const int8_t* status, int32_t* idx_out,
                   int32_t* count_out, cudaStream_t st);

}  // namespace ht
