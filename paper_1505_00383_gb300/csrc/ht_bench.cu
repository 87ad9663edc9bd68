// FP64 pipe throughput probe (measurement helper, see include/ht_bench.h).
#include "ht_bench.h"
#include "ht_internal.h"

namespace ht {

constexpr int kChains = 8;

// Each thread runs kChains independent DFMA chains; the single store keeps the
// work alive.  out has one slot per thread of the grid.
__global__ void fp64_rate_kernel(double* out, int iters, double a, double b) {
  double acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = threadIdx.x * 1e-3 + c;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = __fma_rn(acc[c], a, b);
  double s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Independent chains of 64-bit multiply-adds per thread; each product's
// 32-bit operand is the previous result's low word, so no chain folds.
__global__ void imad_rate_kernel(unsigned long long* out, int iters, unsigned a) {
  unsigned long long acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = threadIdx.x * 2654435761u + c;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = (unsigned long long)(unsigned)acc[c] * a + acc[c];
  unsigned long long s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s ^= acc[c];
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace ht

using namespace ht;

extern "C" int ht_bench_fp64_rate(int iters, double* ops_per_s, void* stream) {
  clear_error();
  if (!ops_per_s || iters < 1) return set_error(HT_EINVAL, "ht_bench_fp64_rate: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  const int threads = 256, blocks = sm_count() * 8;
  const int inner = 256;  // DFMA per chain per iteration unit
  double* out = nullptr;
  cudaError_t e = cudaMalloc(&out, (size_t)blocks * threads * sizeof(double));
  if (e != cudaSuccess) return cuda_fail(e, "ht_bench_fp64_rate: cudaMalloc");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fp64_rate_kernel<<<blocks, threads, 0, st>>>(out, inner, 0.999999, 1e-7);  // warm-up
  cudaEventRecord(e0, st);
  for (int i = 0; i < iters; ++i) fp64_rate_kernel<<<blocks, threads, 0, st>>>(out, inner, 0.999999, 1e-7);
  cudaEventRecord(e1, st);
  e = cudaEventSynchronize(e1);
  float ms = 0;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return cuda_fail(e, "ht_bench_fp64_rate");
  double ops = (double)iters * blocks * threads * inner * kChains;
  *ops_per_s = ops / (ms * 1e-3);
  return HT_OK;
}

extern "C" int ht_bench_imad_rate(int iters, double* ops_per_s, void* stream) {
  clear_error();
  if (!ops_per_s || iters < 1) return set_error(HT_EINVAL, "ht_bench_imad_rate: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  const int threads = 256, blocks = sm_count() * 8;
  const int inner = 4096;
  unsigned long long* out = nullptr;
  cudaError_t e = cudaMalloc(&out, (size_t)blocks * threads * sizeof(unsigned long long));
  if (e != cudaSuccess) return cuda_fail(e, "ht_bench_imad_rate: cudaMalloc");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  imad_rate_kernel<<<blocks, threads, 0, st>>>(out, inner, 2654435761u);
  cudaEventRecord(e0, st);
  for (int i = 0; i < iters; ++i) imad_rate_kernel<<<blocks, threads, 0, st>>>(out, inner, 2654435761u + i);
  cudaEventRecord(e1, st);
  e = cudaEventSynchronize(e1);
  float ms = 0;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return cuda_fail(e, "ht_bench_imad_rate");
  *ops_per_s = (double)iters * blocks * threads * inner * kChains / (ms * 1e-3);
  return HT_OK;
}
