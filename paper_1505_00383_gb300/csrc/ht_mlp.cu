// Learned step-size network: inference and training kernels and the ht_mlp_*
// entry points.  The products of the forward pass (ht_mlp.cuh) and of the
// backward pass run on the tensor cores with BF16 operands and FP32
// accumulation: per chunk of 64 samples one CTA forms the activation
// gradients (dh1 = W2^T dz2 on the tensor cores) and the chunk's weight
// gradients (dz^T h), and a second kernel sums the chunks' partial gradients
// in chunk order, so gradients are deterministic.  Adam runs on the FP32
// masters.  The network's role in tracking is described in ht_track.cu.
#include <cmath>
#include <cstring>
#include <vector>

#include "ht_internal.h"
#include "ht_mlp.cuh"

struct ht_mlp {
  float* master = nullptr;       // [MLP_NPARAM] FP32 parameters
  __nv_bfloat16* wbf = nullptr;  // [MLP_NPARAM] BF16 copy the products use
  float* m = nullptr;            // Adam first moments
  float* v = nullptr;            // Adam second moments
  float* grad = nullptr;         // gradient of the last batch
  float* loss = nullptr;         // [1] loss of the last batch
  void* ws = nullptr;            // training workspace (grown on demand)
  size_t ws_bytes = 0;
  int step = 0;                  // Adam steps taken since the parameters were set
};

namespace ht {

constexpr int kMlpThreads = 128;  // 4 warps, 32 samples each

struct MlpFwdSmem {
  MlpSmem net;
  MlpWarpSmem w[kMlpThreads / 32];
};

// y = MLP(x) for B samples; if z1 is given, also the pre-activations of both
// hidden layers (z1, z2 sized for B rounded up to a multiple of 32 rows).
__global__ void __launch_bounds__(kMlpThreads) mlp_forward_kernel(const __nv_bfloat16* __restrict__ wbf,
                                                                  const float* __restrict__ master, int64_t B,
                                                                  const float* __restrict__ x, float* __restrict__ y,
                                                                  float* __restrict__ z1, float* __restrict__ z2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpFwdSmem& sm = *reinterpret_cast<MlpFwdSmem*>(smem_raw);
  mlp_load(sm.net, wbf, master);
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t n_warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t w0 = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid; w0 * 32 < B; w0 += n_warps) {
    const int64_t s = w0 * 32 + lane;
    float xs[MLP_IN], ys[MLP_OUT];
    for (int i = 0; i < MLP_IN; ++i) xs[i] = s < B ? x[s * MLP_IN + i] : 0.0f;
    if (z1)
      mlp_forward_warp(sm.net, sm.w[wid], xs, ys, z1 + w0 * 32 * MLP_HID, z2 + w0 * 32 * MLP_HID);
    else
      mlp_forward_warp(sm.net, sm.w[wid], xs, ys);
    if (s < B) {
      y[s * MLP_OUT + 0] = ys[0];
      y[s * MLP_OUT + 1] = ys[1];
    }
  }
}

// ------------------------------------------------------------- backward
// One CTA per chunk of kBwdChunk samples.  Shared memory holds the chunk's
// operands in BF16, each laid out for the fragment it feeds: row-major [m][k]
// for A and [n][k] for B (mma.m16n8k16 .row.col), rows padded to 72 elements
// so the 8 row groups of a fragment load fall in distinct banks.
constexpr int kBwdChunk = 64, kBwdThreads = 128, LDC = kBwdChunk + 8, LDH = MLP_HID + 8;
struct MlpBwdSmem {
  __nv_bfloat16 W2T[MLP_HID * LDH];   // [i][o] = W2[o][i]: B operand of dh1 = dz2 W2
  __nv_bfloat16 dz2r[kBwdChunk * LDH];  // [s][o]: A operand of dh1
  __nv_bfloat16 dz2T[MLP_HID * LDC];  // [o][s]: A operand of dW2
  __nv_bfloat16 dz1T[MLP_HID * LDC];  // [o][s]: A operand of dW1
  __nv_bfloat16 dyT[16 * LDC];        // [o][s] (rows 2..15 zero): A operand of dW3
  __nv_bfloat16 h1T[MLP_HID * LDC];   // [i][s] = bf16(relu(z1)): B operand of dW2
  __nv_bfloat16 h2T[MLP_HID * LDC];   // [i][s] = bf16(relu(z2)): B operand of dW3
  __nv_bfloat16 xT[MLP_IN * LDC];     // [i][s] = bf16(x): B operand of dW1
  float W3[MLP_OUT * MLP_HID];
  float dz1f[kBwdChunk * MLP_HID];    // FP32 activation gradients for the bias sums
  float dz2f[kBwdChunk * MLP_HID];
  float dyf[kBwdChunk * MLP_OUT];
  float z2[kBwdChunk * MLP_HID];
  unsigned long long mask1[kBwdChunk];  // bit i: z1[s][i] > 0
  float err2[kBwdChunk];
};

// A 16x8 output tile over K = 16 k16 steps: C += A[m0.., k] B[k, n0..]; A is
// [m][k] with row stride lda, B is [n][k] with row stride ldb (bf16).
__device__ __forceinline__ void mma_tile(float* c, const __nv_bfloat16* A, int lda, const __nv_bfloat16* Bm, int ldb,
                                         int m0, int n0, int ksteps) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  for (int kk = 0; kk < ksteps; ++kk) {
    const int k = 16 * kk + 2 * t;
    uint32_t a[4];
    a[0] = ld_b32(&A[(m0 + g) * lda + k]);
    a[1] = ld_b32(&A[(m0 + g + 8) * lda + k]);
    a[2] = ld_b32(&A[(m0 + g) * lda + k + 8]);
    a[3] = ld_b32(&A[(m0 + g + 8) * lda + k + 8]);
    mma_bf16(c, a, ld_b32(&Bm[(n0 + g) * ldb + k]), ld_b32(&Bm[(n0 + g) * ldb + k + 8]));
  }
}

// Chunk c of the batch: dL/dy = 2 (y - target) / B, the activation gradients
// through both ReLU layers, and the chunk's partial gradient of every
// parameter (part[c][MLP_NPARAM]) and partial loss (loss_part[c]).  The
// activations are recomputed from the stored pre-activations exactly as the
// forward pass rounded them.
__global__ void __launch_bounds__(kBwdThreads) mlp_backward_kernel(
    const __nv_bfloat16* __restrict__ wbf, int64_t B, const float* __restrict__ x, const float* __restrict__ y,
    const float* __restrict__ target, const float* __restrict__ z1, const float* __restrict__ z2,
    float* __restrict__ part, float* __restrict__ loss_part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpBwdSmem& sm = *reinterpret_cast<MlpBwdSmem*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, g = lane >> 2, t = lane & 3;
  const int64_t s0 = (int64_t)blockIdx.x * kBwdChunk;
  const int ns = (int)min((int64_t)kBwdChunk, B - s0);
  const __nv_bfloat16 zero = __float2bfloat16(0.0f);
  // ---- stage weights and the chunk's activations
  for (int e = tid; e < MLP_HID * MLP_HID; e += kBwdThreads) {
    const int o = e / MLP_HID, i = e % MLP_HID;
    sm.W2T[i * LDH + o] = wbf[OFF_W2 + e];
  }
  for (int e = tid; e < MLP_OUT * MLP_HID; e += kBwdThreads) sm.W3[e] = __bfloat162float(wbf[OFF_W3 + e]);
  for (int e = tid; e < kBwdChunk * MLP_HID; e += kBwdThreads) {
    const int sl = e / MLP_HID, i = e % MLP_HID;
    const bool live = sl < ns;
    const float a = live ? z1[(s0 + sl) * MLP_HID + i] : 0.0f;
    const float b = live ? z2[(s0 + sl) * MLP_HID + i] : 0.0f;
    sm.h1T[i * LDC + sl] = __float2bfloat16(fmaxf(a, 0.0f));
    sm.h2T[i * LDC + sl] = __float2bfloat16(fmaxf(b, 0.0f));
    sm.z2[sl * MLP_HID + i] = b;
  }
  for (int e = tid; e < kBwdChunk * MLP_IN; e += kBwdThreads) {
    const int sl = e / MLP_IN, i = e % MLP_IN;
    sm.xT[i * LDC + sl] = sl < ns ? __float2bfloat16(x[(s0 + sl) * MLP_IN + i]) : zero;
  }
  for (int e = tid; e < 16 * LDC; e += kBwdThreads) sm.dyT[e] = zero;
  if (tid < kBwdChunk) {  // layer-1 ReLU mask of sample tid
    unsigned long long mk = 0;
    if (tid < ns)
      for (int i = 0; i < MLP_HID; ++i) mk |= (unsigned long long)(z1[(s0 + tid) * MLP_HID + i] > 0.0f) << i;
    sm.mask1[tid] = mk;
  }
  __syncthreads();
  // ---- per sample: dy, dh2 = W3^T dy (K = 2, FP32) and the layer-2 mask
  if (tid < kBwdChunk) {
    const int sl = tid;
    const bool live = sl < ns;
    float d[MLP_OUT], err = 0.0f;
    for (int o = 0; o < MLP_OUT; ++o) {
      const float e = live ? y[(s0 + sl) * MLP_OUT + o] - target[(s0 + sl) * MLP_OUT + o] : 0.0f;
      err += e * e;
      d[o] = 2.0f * e / (float)B;
      sm.dyf[sl * MLP_OUT + o] = d[o];
      sm.dyT[o * LDC + sl] = __float2bfloat16(d[o]);
    }
    sm.err2[sl] = err;
    for (int i = 0; i < MLP_HID; ++i) {
      float a = 0.0f;
      for (int o = 0; o < MLP_OUT; ++o) a += d[o] * sm.W3[o * MLP_HID + i];
      const float dz = sm.z2[sl * MLP_HID + i] > 0.0f ? a : 0.0f;
      sm.dz2f[sl * MLP_HID + i] = dz;
      const __nv_bfloat16 q = __float2bfloat16(dz);
      sm.dz2r[sl * LDH + i] = q;
      sm.dz2T[i * LDC + sl] = q;
    }
  }
  __syncthreads();
  // ---- dh1 = dz2 W2 on the tensor cores (warp w: samples 16w..16w+15), layer-1 mask
  for (int nt = 0; nt < MLP_HID / 8; ++nt) {
    float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    mma_tile(c, sm.dz2r, LDH, sm.W2T, LDH, 16 * warp, 8 * nt, MLP_HID / 16);
    const int r0 = 16 * warp + g, r1 = r0 + 8, col = 8 * nt + 2 * t;
    const float v[4] = {c[0], c[1], c[2], c[3]};
    const int rows[4] = {r0, r0, r1, r1}, cols[4] = {col, col + 1, col, col + 1};
    for (int q = 0; q < 4; ++q) {
      const float dz = (sm.mask1[rows[q]] >> cols[q]) & 1ull ? v[q] : 0.0f;
      sm.dz1f[rows[q] * MLP_HID + cols[q]] = dz;
      sm.dz1T[cols[q] * LDC + rows[q]] = __float2bfloat16(dz);
    }
  }
  __syncthreads();
  // ---- the chunk's weight gradients dW = dz^T h (K = the chunk's samples)
  float* out = part + (int64_t)blockIdx.x * MLP_NPARAM;
  constexpr int T2 = (MLP_HID / 16) * (MLP_HID / 8), T1 = (MLP_HID / 16) * (MLP_IN / 8), T3 = MLP_HID / 8;
  for (int tile = warp; tile < T2 + T1 + T3; tile += kBwdThreads / 32) {
    float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    int m0, n0, ldo, off, rows;
    if (tile < T2) {  // dW2[o][i] = sum_s dz2[s][o] h1[s][i]
      m0 = 16 * (tile / (MLP_HID / 8));
      n0 = 8 * (tile % (MLP_HID / 8));
      mma_tile(c, sm.dz2T, LDC, sm.h1T, LDC, m0, n0, kBwdChunk / 16);
      ldo = MLP_HID, off = OFF_W2, rows = MLP_HID;
    } else if (tile < T2 + T1) {  // dW1[o][i] = sum_s dz1[s][o] x[s][i]
      const int u = tile - T2;
      m0 = 16 * (u / (MLP_IN / 8));
      n0 = 8 * (u % (MLP_IN / 8));
      mma_tile(c, sm.dz1T, LDC, sm.xT, LDC, m0, n0, kBwdChunk / 16);
      ldo = MLP_IN, off = OFF_W1, rows = MLP_HID;
    } else {  // dW3[o][i] = sum_s dy[s][o] h2[s][i]
      m0 = 0;
      n0 = 8 * (tile - T2 - T1);
      mma_tile(c, sm.dyT, LDC, sm.h2T, LDC, m0, n0, kBwdChunk / 16);
      ldo = MLP_HID, off = OFF_W3, rows = MLP_OUT;
    }
    const int r0 = m0 + g, r1 = r0 + 8, col = n0 + 2 * t;
    if (r0 < rows) {
      out[off + r0 * ldo + col] = c[0];
      out[off + r0 * ldo + col + 1] = c[1];
    }
    if (r1 < rows) {
      out[off + r1 * ldo + col] = c[2];
      out[off + r1 * ldo + col + 1] = c[3];
    }
  }
  // ---- bias gradients and the loss: FP32 sums over the chunk's samples in order
  if (tid < MLP_HID) {
    float a = 0.0f, b = 0.0f;
    for (int sl = 0; sl < kBwdChunk; ++sl) {
      a += sm.dz1f[sl * MLP_HID + tid];
      b += sm.dz2f[sl * MLP_HID + tid];
    }
    out[OFF_B1 + tid] = a;
    out[OFF_B2 + tid] = b;
  } else if (tid < MLP_HID + MLP_OUT) {
    const int o = tid - MLP_HID;
    float a = 0.0f;
    for (int sl = 0; sl < kBwdChunk; ++sl) a += sm.dyf[sl * MLP_OUT + o];
    out[OFF_B3 + o] = a;
  } else if (tid == MLP_HID + MLP_OUT) {
    float a = 0.0f;
    for (int sl = 0; sl < kBwdChunk; ++sl) a += sm.err2[sl];
    loss_part[blockIdx.x] = a;
  }
}

// grad[p] = sum over chunks (in chunk order) of part[c][p]; loss = sum / B.
__global__ void mlp_grad_reduce_kernel(int n_chunks, int64_t B, const float* __restrict__ part,
                                       const float* __restrict__ loss_part, float* __restrict__ grad,
                                       float* __restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0) {
    float l = 0.0f;
    for (int c = 0; c < n_chunks; ++c) l += loss_part[c];
    *loss = l / (float)B;
  }
  if (p >= MLP_NPARAM) return;
  float a = 0.0f;
  for (int c = 0; c < n_chunks; ++c) a += part[(int64_t)c * MLP_NPARAM + p];
  grad[p] = a;
}

// Adam (Kingma & Ba 2015) on the FP32 masters, then the BF16 copy.
__global__ void mlp_adam_kernel(float* __restrict__ w, __nv_bfloat16* __restrict__ wbf, float* __restrict__ m,
                                float* __restrict__ v, const float* __restrict__ g, float lr, float b1, float b2,
                                float eps, float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= MLP_NPARAM) return;
  const float gp = g[p];
  const float mp = b1 * m[p] + (1.0f - b1) * gp;
  const float vp = b2 * v[p] + (1.0f - b2) * gp * gp;
  m[p] = mp;
  v[p] = vp;
  const float wp = w[p] - lr * (mp / c1) / (sqrtf(vp / c2) + eps);
  w[p] = wp;
  wbf[p] = __float2bfloat16(wp);
}

__global__ void mlp_to_bf16_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ wbf) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < MLP_NPARAM) wbf[p] = __float2bfloat16(w[p]);
}

static int mlp_fwd_launch(const ht_mlp* net, int64_t B, const float* x, float* y, float* z1, float* z2,
                          cudaStream_t st) {
  const size_t smem = sizeof(MlpFwdSmem);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set = true;
  }
  int64_t warps = (B + 31) / 32;
  int64_t grid = (warps + 3) / 4;
  int64_t cap = (int64_t)sm_count() * 8;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  mlp_forward_kernel<<<(unsigned)grid, kMlpThreads, smem, st>>>(net->wbf, net->master, B, x, y, z1, z2);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HT_OK : cuda_fail(e, "mlp forward launch");
}

// Workspace for a batch of B samples (Bp = B rounded up to 32 rows, C chunks
// of kBwdChunk samples): y [Bp][2]; z1, z2 [Bp][64]; partial gradients
// [C][MLP_NPARAM]; partial losses [C].
static int mlp_ws(ht_mlp* net, int64_t B, float** y, float** z1, float** z2, float** part, float** lpart,
                  cudaStream_t st) {
  const int64_t Bp = (B + 31) / 32 * 32, C = (B + kBwdChunk - 1) / kBwdChunk;
  size_t need = ((size_t)Bp * (MLP_OUT + 2 * MLP_HID) + (size_t)C * (MLP_NPARAM + 1)) * sizeof(float);
  if (net->ws_bytes < need) {
    if (net->ws) {
      cudaStreamSynchronize(st);
      cudaFree(net->ws);
      net->ws = nullptr;
      net->ws_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&net->ws, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_error(HT_ENOMEM, "mlp workspace of %zu bytes", need);
    }
    net->ws_bytes = need;
  }
  float* f = (float*)net->ws;
  *y = f;
  f += Bp * MLP_OUT;
  *z1 = f;
  f += Bp * MLP_HID;
  *z2 = f;
  f += Bp * MLP_HID;
  *part = f;
  f += C * MLP_NPARAM;
  *lpart = f;
  return HT_OK;
}

static int mlp_grad_batch(ht_mlp* net, int64_t B, const float* x, const float* target, cudaStream_t st) {
  float *y, *z1, *z2, *part, *lpart;
  int rc = mlp_ws(net, B, &y, &z1, &z2, &part, &lpart, st);
  if (rc != HT_OK) return rc;
  rc = mlp_fwd_launch(net, B, x, y, z1, z2, st);
  if (rc != HT_OK) return rc;
  const int64_t C = (B + kBwdChunk - 1) / kBwdChunk;
  const size_t smem = sizeof(MlpBwdSmem);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(mlp_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set = true;
  }
  mlp_backward_kernel<<<(unsigned)C, kBwdThreads, smem, st>>>(net->wbf, B, x, y, target, z1, z2, part, lpart);
  mlp_grad_reduce_kernel<<<(MLP_NPARAM + 127) / 128, 128, 0, st>>>((int)C, B, part, lpart, net->grad, net->loss);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HT_OK : cuda_fail(e, "mlp backward launch");
}

static int mlp_adam_launch(ht_mlp* net, const float* grad, float lr, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  ++net->step;
  // bias corrections 1 - beta^k in double, rounded once: in FP32, 1 - powf
  // would amplify powf's rounding by beta^k / (1 - beta^k) (about 1000 at k = 1)
  const float c1 = (float)(1.0 - std::pow((double)b1, (double)net->step));
  const float c2 = (float)(1.0 - std::pow((double)b2, (double)net->step));
  mlp_adam_kernel<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(net->master, net->wbf, net->m, net->v, grad, lr, b1, b2,
                                                            eps, c1, c2);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HT_OK : cuda_fail(e, "mlp adam launch");
}

const float* mlp_master(const ht_mlp* net) { return net->master; }
const __nv_bfloat16* mlp_bf16(const ht_mlp* net) { return net->wbf; }

}  // namespace ht

using namespace ht;

extern "C" {

int ht_mlp_create(ht_mlp** out) {
  clear_error();
  if (!out) return set_error(HT_EINVAL, "ht_mlp_create: NULL");
  *out = nullptr;
  ht_mlp* net = new (std::nothrow) ht_mlp();
  if (!net) return set_error(HT_ENOMEM, "ht_mlp_create");
  const size_t nf = MLP_NPARAM;
  char* blk = nullptr;
  size_t bytes = nf * 4 * 4 + nf * 2 + 256;
  cudaError_t e = cudaMalloc((void**)&blk, bytes);
  if (e != cudaSuccess) {
    delete net;
    cudaGetLastError();
    return set_error(HT_ENOMEM, "ht_mlp_create: cudaMalloc");
  }
  cudaMemset(blk, 0, bytes);
  net->master = (float*)blk;
  net->m = net->master + nf;
  net->v = net->m + nf;
  net->grad = net->v + nf;
  net->loss = (float*)(blk + nf * 4 * 4);
  net->wbf = (__nv_bfloat16*)(blk + nf * 4 * 4 + 64);
  *out = net;
  return HT_OK;
}

int ht_mlp_destroy(ht_mlp* net) {
  clear_error();
  if (!net) return HT_OK;
  cudaDeviceSynchronize();
  cudaFree(net->master);
  if (net->ws) cudaFree(net->ws);
  delete net;
  return HT_OK;
}

int ht_mlp_set_params(ht_mlp* net, const float* params) {
  clear_error();
  if (!net || !params) return set_error(HT_EINVAL, "ht_mlp_set_params: NULL");
  cudaError_t e = cudaMemcpy(net->master, params, MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(net->m, 0, 2 * MLP_NPARAM * sizeof(float));
  if (e != cudaSuccess) return cuda_fail(e, "ht_mlp_set_params");
  net->step = 0;
  mlp_to_bf16_kernel<<<(MLP_NPARAM + 255) / 256, 256>>>(net->master, net->wbf);
  e = cudaDeviceSynchronize();
  return e == cudaSuccess ? HT_OK : cuda_fail(e, "ht_mlp_set_params");
}

int ht_mlp_get_params(const ht_mlp* net, float* params) {
  clear_error();
  if (!net || !params) return set_error(HT_EINVAL, "ht_mlp_get_params: NULL");
  cudaError_t e = cudaMemcpy(params, net->master, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? HT_OK : cuda_fail(e, "ht_mlp_get_params");
}

int ht_mlp_forward(const ht_mlp* net, int64_t B, const float* x, float* y, void* stream) {
  clear_error();
  if (!net || B < 0) return set_error(HT_EINVAL, "ht_mlp_forward: bad arguments");
  if (B == 0) return HT_OK;
  if (!x || !y || !is_device_ptr(x) || !is_device_ptr(y) || (((uintptr_t)x | (uintptr_t)y) & 3))
    return set_error(HT_EINVAL, "ht_mlp_forward: x and y must be device memory");
  return mlp_fwd_launch(net, B, x, y, nullptr, nullptr, (cudaStream_t)stream);
}

int ht_mlp_loss_grad(ht_mlp* net, int64_t B, const float* x, const float* target, float* grad, float* loss,
                     void* stream) {
  clear_error();
  if (!net || B < 1 || !x || !target || !is_device_ptr(x) || !is_device_ptr(target) ||
      (grad && !is_device_ptr(grad)) || (loss && !is_device_ptr(loss)))
    return set_error(HT_EINVAL, "ht_mlp_loss_grad: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  int rc = mlp_grad_batch(net, B, x, target, st);
  if (rc != HT_OK) return rc;
  cudaError_t e = cudaSuccess;
  if (grad) e = cudaMemcpyAsync(grad, net->grad, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, net->loss, sizeof(float), cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? HT_OK : cuda_fail(e, "ht_mlp_loss_grad");
}

int ht_mlp_train(ht_mlp* net, int64_t n, const float* x, const float* target, int epochs, int64_t batch, float lr,
                 float* epoch_loss, void* stream) {
  clear_error();
  if (!net || n < 1 || epochs < 1 || batch < 1 || !(lr > 0) || !x || !target || !is_device_ptr(x) ||
      !is_device_ptr(target))
    return set_error(HT_EINVAL, "ht_mlp_train: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  for (int ep = 0; ep < epochs; ++ep) {
    double sum = 0.0;
    int nb = 0;
    for (int64_t off = 0; off < n; off += batch) {
      const int64_t B = (off + batch <= n) ? batch : n - off;
      int rc = mlp_grad_batch(net, B, x + off * MLP_IN, target + off * MLP_OUT, st);
      if (rc != HT_OK) return rc;
      rc = mlp_adam_launch(net, net->grad, lr, st);
      if (rc != HT_OK) return rc;
      if (epoch_loss) {
        float l = 0;
        cudaError_t e = cudaMemcpyAsync(&l, net->loss, sizeof(float), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "ht_mlp_train");
        sum += l;
        ++nb;
      }
    }
    if (epoch_loss) epoch_loss[ep] = (float)(sum / (nb ? nb : 1));
  }
  cudaError_t e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? HT_OK : cuda_fail(e, "ht_mlp_train");
}

int ht_mlp_adam_step(ht_mlp* net, const float* grad, float lr, void* stream) {
  clear_error();
  if (!net || !grad || !is_device_ptr(grad) || !(lr > 0) || ((uintptr_t)grad & 3))
    return set_error(HT_EINVAL, "ht_mlp_adam_step: bad arguments");
  return mlp_adam_launch(net, grad, lr, (cudaStream_t)stream);
}

int ht_mlp_get_moments(const ht_mlp* net, float* m, float* v, int32_t* step) {
  clear_error();
  if (!net) return set_error(HT_EINVAL, "ht_mlp_get_moments: NULL");
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess && m) e = cudaMemcpy(m, net->m, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && v) e = cudaMemcpy(v, net->v, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "ht_mlp_get_moments");
  if (step) *step = net->step;
  return HT_OK;
}

}  // extern "C"
