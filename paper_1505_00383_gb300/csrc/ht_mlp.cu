// Learned step-size network: inference and training kernels and the ht_mlp_*
// entry points.  Forward products run on the tensor cores (ht_mlp.cuh);
// the backward pass (activation gradients per sample, then one thread per
// parameter summing over the batch in a fixed order, so gradients are
// deterministic) and Adam run on the FP32 pipe.  The network's role in
// tracking is described in ht_track.cu.
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
};

namespace ht {

constexpr int kMlpThreads = 128;  // 4 warps, 32 samples each
constexpr int kLossBlocks = 256;

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

__device__ __forceinline__ float bfr(float v) { return __bfloat162float(__float2bfloat16(v)); }

// Per sample: the squared error, dL/dy = 2 (y - target) / B, and the
// activation gradients dz2, dz1 through both ReLU layers (the BF16 rounding of
// the forward pass is passed through unchanged).  Block partial losses go to
// loss_part[blockIdx.x].
__global__ void __launch_bounds__(256) mlp_backward_act_kernel(const __nv_bfloat16* __restrict__ wbf, int64_t B,
                                                               const float* __restrict__ y,
                                                               const float* __restrict__ target, float* __restrict__ dy,
                                                               const float* __restrict__ z1, const float* __restrict__ z2,
                                                               float* __restrict__ dz1, float* __restrict__ dz2,
                                                               float* __restrict__ loss_part) {
  __shared__ float W2s[MLP_HID * MLP_HID];
  __shared__ float W3s[MLP_OUT * MLP_HID];
  __shared__ float red[256];
  for (int i = threadIdx.x; i < MLP_HID * MLP_HID; i += blockDim.x) W2s[i] = __bfloat162float(wbf[OFF_W2 + i]);
  for (int i = threadIdx.x; i < MLP_OUT * MLP_HID; i += blockDim.x) W3s[i] = __bfloat162float(wbf[OFF_W3 + i]);
  __syncthreads();
  float part = 0.0f;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < B; s += (int64_t)gridDim.x * blockDim.x) {
    float d[MLP_OUT];
    for (int o = 0; o < MLP_OUT; ++o) {
      float e = y[s * MLP_OUT + o] - target[s * MLP_OUT + o];
      part += e * e;
      d[o] = 2.0f * e / (float)B;
      dy[s * MLP_OUT + o] = d[o];
    }
    float g2[MLP_HID];
    for (int i = 0; i < MLP_HID; ++i) {
      float a = 0.0f;
      for (int o = 0; o < MLP_OUT; ++o) a += d[o] * W3s[o * MLP_HID + i];
      g2[i] = z2[s * MLP_HID + i] > 0.0f ? a : 0.0f;
      dz2[s * MLP_HID + i] = g2[i];
    }
    for (int i = 0; i < MLP_HID; ++i) {
      float a = 0.0f;
      for (int o = 0; o < MLP_HID; ++o) a += g2[o] * W2s[o * MLP_HID + i];
      dz1[s * MLP_HID + i] = z1[s * MLP_HID + i] > 0.0f ? a : 0.0f;
    }
  }
  red[threadIdx.x] = part;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss_part[blockIdx.x] = red[0];
}

// One thread per parameter: sum over the batch, samples in order.  The inputs
// of each layer are the BF16-rounded values the forward products used.
__global__ void mlp_weight_grad_kernel(int64_t B, const float* __restrict__ x, const float* __restrict__ z1,
                                       const float* __restrict__ z2, const float* __restrict__ dy,
                                       const float* __restrict__ dz1, const float* __restrict__ dz2,
                                       const float* __restrict__ loss_part, int n_part, float* __restrict__ grad,
                                       float* __restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0) {
    float l = 0.0f;
    for (int i = 0; i < n_part; ++i) l += loss_part[i];
    *loss = l / (float)B;
  }
  if (p >= MLP_NPARAM) return;
  float acc = 0.0f;
  if (p < OFF_B1) {
    const int o = p / MLP_IN, i = p % MLP_IN;
    for (int64_t s = 0; s < B; ++s) acc += dz1[s * MLP_HID + o] * bfr(x[s * MLP_IN + i]);
  } else if (p < OFF_W2) {
    const int o = p - OFF_B1;
    for (int64_t s = 0; s < B; ++s) acc += dz1[s * MLP_HID + o];
  } else if (p < OFF_B2) {
    const int o = (p - OFF_W2) / MLP_HID, i = (p - OFF_W2) % MLP_HID;
    for (int64_t s = 0; s < B; ++s) acc += dz2[s * MLP_HID + o] * bfr(fmaxf(z1[s * MLP_HID + i], 0.0f));
  } else if (p < OFF_W3) {
    const int o = p - OFF_B2;
    for (int64_t s = 0; s < B; ++s) acc += dz2[s * MLP_HID + o];
  } else if (p < OFF_B3) {
    const int o = (p - OFF_W3) / MLP_HID, i = (p - OFF_W3) % MLP_HID;
    for (int64_t s = 0; s < B; ++s) acc += dy[s * MLP_OUT + o] * bfr(fmaxf(z2[s * MLP_HID + i], 0.0f));
  } else {
    const int o = p - OFF_B3;
    for (int64_t s = 0; s < B; ++s) acc += dy[s * MLP_OUT + o];
  }
  grad[p] = acc;
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

// Workspace for a batch of B samples: y, dy [Bp][2]; z1, z2, dz1, dz2 [Bp][64];
// loss partials (Bp = B rounded up to 32).
static int mlp_ws(ht_mlp* net, int64_t B, float** y, float** dy, float** z1, float** z2, float** dz1, float** dz2,
                  float** part, cudaStream_t st) {
  const int64_t Bp = (B + 31) / 32 * 32;
  size_t need = ((size_t)Bp * (2 * MLP_OUT + 4 * MLP_HID) + kLossBlocks) * sizeof(float);
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
  *dy = f;
  f += Bp * MLP_OUT;
  *z1 = f;
  f += Bp * MLP_HID;
  *z2 = f;
  f += Bp * MLP_HID;
  *dz1 = f;
  f += Bp * MLP_HID;
  *dz2 = f;
  f += Bp * MLP_HID;
  *part = f;
  return HT_OK;
}

static int mlp_grad_batch(ht_mlp* net, int64_t B, const float* x, const float* target, cudaStream_t st) {
  float *y, *dy, *z1, *z2, *dz1, *dz2, *part;
  int rc = mlp_ws(net, B, &y, &dy, &z1, &z2, &dz1, &dz2, &part, st);
  if (rc != HT_OK) return rc;
  rc = mlp_fwd_launch(net, B, x, y, z1, z2, st);
  if (rc != HT_OK) return rc;
  mlp_backward_act_kernel<<<kLossBlocks, 256, 0, st>>>(net->wbf, B, y, target, dy, z1, z2, dz1, dz2, part);
  mlp_weight_grad_kernel<<<(MLP_NPARAM + 127) / 128, 128, 0, st>>>(B, x, z1, z2, dy, dz1, dz2, part, kLossBlocks,
                                                                  net->grad, net->loss);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HT_OK : cuda_fail(e, "mlp backward launch");
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
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  int step = 0;
  for (int ep = 0; ep < epochs; ++ep) {
    double sum = 0.0;
    int nb = 0;
    for (int64_t off = 0; off < n; off += batch) {
      const int64_t B = (off + batch <= n) ? batch : n - off;
      int rc = mlp_grad_batch(net, B, x + off * MLP_IN, target + off * MLP_OUT, st);
      if (rc != HT_OK) return rc;
      ++step;
      const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
      mlp_adam_kernel<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(net->master, net->wbf, net->m, net->v, net->grad, lr,
                                                                b1, b2, eps, c1, c2);
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

}  // extern "C"
