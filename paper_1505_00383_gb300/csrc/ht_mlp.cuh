// Learned step-size proposer: a 16 -> 64 -> 64 -> 2 ReLU network evaluated by
// a warp for 32 samples at once on the tensor cores (BF16 operands, FP32
// accumulation, mma.sync m16n8k16), shared by the standalone inference and
// training kernels and by the tracker kernel.
//
// Parameters (FP32 masters, flat): W1[64][16] b1[64] W2[64][64] b2[64]
// W3[2][64] b3[2].  The device copy used for the products is BF16, laid out in
// shared memory with padded rows so that the B-fragment loads of the eight
// row groups of a warp fall in distinct banks.
#pragma once
#include <cuda_bf16.h>

#include <cstdint>

namespace ht {

constexpr int MLP_IN = 16, MLP_HID = 64, MLP_OUT = 2;
constexpr int MLP_NPARAM = MLP_HID * MLP_IN + MLP_HID + MLP_HID * MLP_HID + MLP_HID + MLP_OUT * MLP_HID + MLP_OUT;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + MLP_HID * MLP_IN, OFF_W2 = OFF_B1 + MLP_HID,
              OFF_B2 = OFF_W2 + MLP_HID * MLP_HID, OFF_W3 = OFF_B2 + MLP_HID, OFF_B3 = OFF_W3 + MLP_OUT * MLP_HID;
// padded row strides (bf16 elements) of the weights in shared memory
constexpr int LD1 = MLP_IN + 8, LD2 = MLP_HID + 8, LD3 = MLP_HID + 8, LDX = MLP_IN + 8;

// Shared-memory image of the network for one CTA.
struct MlpSmem {
  __nv_bfloat16 W1[MLP_HID * LD1];
  __nv_bfloat16 W2[MLP_HID * LD2];
  __nv_bfloat16 W3[8 * LD3];  // rows 2..7 zero: one 8-wide n-tile
  float b1[MLP_HID], b2[MLP_HID], b3[8];
};
// Per-warp staging of inputs and outputs (rows = the warp's 32 samples).
struct MlpWarpSmem {
  __nv_bfloat16 X[32 * LDX];
  float Y[32][2];
};

// Copy the BF16 weights (flat, unpadded, same order as the FP32 masters) and
// FP32 biases into shared memory; all threads of the CTA take part.
__device__ __forceinline__ void mlp_load(MlpSmem& s, const __nv_bfloat16* __restrict__ wbf,
                                         const float* __restrict__ master) {
  for (int i = threadIdx.x; i < MLP_HID * MLP_IN; i += blockDim.x) s.W1[(i / MLP_IN) * LD1 + i % MLP_IN] = wbf[OFF_W1 + i];
  for (int i = threadIdx.x; i < MLP_HID * MLP_HID; i += blockDim.x)
    s.W2[(i / MLP_HID) * LD2 + i % MLP_HID] = wbf[OFF_W2 + i];
  for (int i = threadIdx.x; i < 8 * MLP_HID; i += blockDim.x)
    s.W3[(i / MLP_HID) * LD3 + i % MLP_HID] = i < MLP_OUT * MLP_HID ? wbf[OFF_W3 + i] : __float2bfloat16(0.0f);
  for (int i = threadIdx.x; i < MLP_HID; i += blockDim.x) {
    s.b1[i] = master[OFF_B1 + i];
    s.b2[i] = master[OFF_B2 + i];
  }
  for (int i = threadIdx.x; i < 8; i += blockDim.x) s.b3[i] = i < MLP_OUT ? master[OFF_B3 + i] : 0.0f;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x = lo (low 16 bits)
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ uint32_t ld_b32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// D = A (16x16, row) * B (16x8, col) + C, BF16 x BF16 -> FP32.
__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Forward pass for the warp's 32 samples.  Each lane passes the features of
// its own sample (x[16]) and receives its outputs y[2].  If z1_rows is given,
// the pre-activations of both hidden layers are also written to z1_rows and
// z2_rows ([32][64] each, row = sample of the warp) for the backward pass.
// All 32 lanes must call it.
__device__ __forceinline__ void mlp_forward_warp(const MlpSmem& s, MlpWarpSmem& w, const float* x, float* y,
                                                 float* z1_rows = nullptr, float* z2_rows = nullptr) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  for (int i = 0; i < MLP_IN; i += 2) *reinterpret_cast<uint32_t*>(&w.X[lane * LDX + i]) = pack_bf16(x[i], x[i + 1]);
  __syncwarp();
  for (int mt = 0; mt < 2; ++mt) {  // two m-tiles of 16 samples
    const int r0 = 16 * mt + g, r1 = r0 + 8;
    uint32_t a[4];
    a[0] = ld_b32(&w.X[r0 * LDX + 2 * t]);
    a[1] = ld_b32(&w.X[r1 * LDX + 2 * t]);
    a[2] = ld_b32(&w.X[r0 * LDX + 2 * t + 8]);
    a[3] = ld_b32(&w.X[r1 * LDX + 2 * t + 8]);
    // layer 1: 8 n-tiles of the 64 hidden units, one k-step
    float h1[8][4];
    for (int j = 0; j < 8; ++j) {
      const int n = 8 * j + g;
      float c0 = s.b1[8 * j + 2 * t], c1 = s.b1[8 * j + 2 * t + 1];
      h1[j][0] = c0;
      h1[j][1] = c1;
      h1[j][2] = c0;
      h1[j][3] = c1;
      mma_bf16(h1[j], a, ld_b32(&s.W1[n * LD1 + 2 * t]), ld_b32(&s.W1[n * LD1 + 2 * t + 8]));
    }
    // ReLU; C fragments of layer 1 become A fragments of layer 2 (k = hidden unit)
    uint32_t a2[4][4];
    for (int kk = 0; kk < 4; ++kk) {
      float* u = h1[2 * kk];
      float* v = h1[2 * kk + 1];
      a2[kk][0] = pack_bf16(fmaxf(u[0], 0.f), fmaxf(u[1], 0.f));
      a2[kk][1] = pack_bf16(fmaxf(u[2], 0.f), fmaxf(u[3], 0.f));
      a2[kk][2] = pack_bf16(fmaxf(v[0], 0.f), fmaxf(v[1], 0.f));
      a2[kk][3] = pack_bf16(fmaxf(v[2], 0.f), fmaxf(v[3], 0.f));
    }
    // layer 2: 8 n-tiles x 4 k-steps
    float h2[8][4];
    for (int j = 0; j < 8; ++j) {
      const int n = 8 * j + g;
      float c0 = s.b2[8 * j + 2 * t], c1 = s.b2[8 * j + 2 * t + 1];
      h2[j][0] = c0;
      h2[j][1] = c1;
      h2[j][2] = c0;
      h2[j][3] = c1;
      for (int kk = 0; kk < 4; ++kk)
        mma_bf16(h2[j], a2[kk], ld_b32(&s.W2[n * LD2 + 16 * kk + 2 * t]), ld_b32(&s.W2[n * LD2 + 16 * kk + 2 * t + 8]));
    }
    uint32_t a3[4][4];
    for (int kk = 0; kk < 4; ++kk) {
      float* u = h2[2 * kk];
      float* v = h2[2 * kk + 1];
      a3[kk][0] = pack_bf16(fmaxf(u[0], 0.f), fmaxf(u[1], 0.f));
      a3[kk][1] = pack_bf16(fmaxf(u[2], 0.f), fmaxf(u[3], 0.f));
      a3[kk][2] = pack_bf16(fmaxf(v[0], 0.f), fmaxf(v[1], 0.f));
      a3[kk][3] = pack_bf16(fmaxf(v[2], 0.f), fmaxf(v[3], 0.f));
    }
    // layer 3: one n-tile (outputs 0, 1 real), 4 k-steps
    float o[4] = {s.b3[2 * t], s.b3[2 * t + 1], s.b3[2 * t], s.b3[2 * t + 1]};
    for (int kk = 0; kk < 4; ++kk)
      mma_bf16(o, a3[kk], ld_b32(&s.W3[g * LD3 + 16 * kk + 2 * t]), ld_b32(&s.W3[g * LD3 + 16 * kk + 2 * t + 8]));
    if (t == 0) {
      w.Y[r0][0] = o[0];
      w.Y[r0][1] = o[1];
      w.Y[r1][0] = o[2];
      w.Y[r1][1] = o[3];
    }
    // pre-activations for training: scatter this lane's fragment entries
    if (z1_rows) {
      for (int j = 0; j < 8; ++j) {
        const int c = 8 * j + 2 * t;
        z1_rows[(size_t)r0 * MLP_HID + c] = h1[j][0];
        z1_rows[(size_t)r0 * MLP_HID + c + 1] = h1[j][1];
        z1_rows[(size_t)r1 * MLP_HID + c] = h1[j][2];
        z1_rows[(size_t)r1 * MLP_HID + c + 1] = h1[j][3];
        z2_rows[(size_t)r0 * MLP_HID + c] = h2[j][0];
        z2_rows[(size_t)r0 * MLP_HID + c + 1] = h2[j][1];
        z2_rows[(size_t)r1 * MLP_HID + c] = h2[j][2];
        z2_rows[(size_t)r1 * MLP_HID + c + 1] = h2[j][3];
      }
    }
  }
  __syncwarp();
  y[0] = w.Y[lane][0];
  y[1] = w.Y[lane][1];
  __syncwarp();
}

}  // namespace ht
