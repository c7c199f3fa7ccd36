// Warm-start network: 24 contact features -> 128 -> 128 (ReLU) -> 3 impulses.
// BF16 operands on the tensor cores (mma.sync m16n8k16) with FP32
// accumulation.  Shared by the episode kernel (inference per contact) and the
// training kernels.
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

namespace jbk {

constexpr int kFeat = 24;       // input features
constexpr int kFeatPad = 32;    // padded to two k-steps
constexpr int kHid = 128;
constexpr int kOut = 3;
constexpr int kOutPad = 8;      // one n-tile
constexpr int kOutPadK = 16;    // outputs as a k-step (backward)

// Packed B-fragment counts (uint2 per lane per (k-tile, n-tile)).
constexpr int kW1Tiles = (kFeatPad / 16) * (kHid / 8);   // 32
constexpr int kW2Tiles = (kHid / 16) * (kHid / 8);       // 128
constexpr int kW3Tiles = (kHid / 16) * (kOutPad / 8);    // 8
// transposed packs for the backward pass: W3^T [16 x 128], W2^T [128 x 128]
constexpr int kW3TTiles = (kOutPadK / 16) * (kHid / 8);  // 16
constexpr int kW2TTiles = (kHid / 16) * (kHid / 8);      // 128

// BF16 image of the weights in the shared-memory layout of the tensor-core
// kernel (jb_mlp_tc.cu), written by the pack kernel after every parameter
// change and copied to shared memory in one bulk transfer.  Tiles are
// K-major without swizzle: element (r, k) of a [R][K] tile at byte
// (r / 8) * K * 16 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2.
constexpr int kImgW1T = 0;                          // W1^T [128 hidden][32 features]
constexpr int kImgW2T = kImgW1T + 128 * 32 * 2;     // W2^T [128 out][128 in]
constexpr int kImgW2 = kImgW2T + 128 * 128 * 2;     // W2 [128 in][128 out]
constexpr int kImgW3T = kImgW2 + 128 * 128 * 2;     // W3^T [16 outputs][128 hidden]
constexpr int kImgW3 = kImgW3T + 16 * 128 * 2;      // W3 [128 hidden][16 outputs]
constexpr int kImgBytes = kImgW3 + 128 * 16 * 2;    // 81,920
__host__ __device__ inline uint32_t kmaj_off(int r, int k, int K) {
  return (uint32_t)((r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// The tensor-core kernel's gradient: at most kTcMaxGrid CTAs, each writing
// its partial sums (parameters, then the loss) to a row of the scratch, which
// a second kernel sums in CTA order.
constexpr int kTcMaxGrid = 160;

// Layout of the network block in device memory (FP32 unless noted).
struct MlpLayout {
  // master weights, row-major [in][out]
  int w1, b1, w2, b2, w3, b3;
  int nparam;                 // floats of one parameter set
  int m, v;                   // AdamW moments (nparam floats each)
  int step;                   // float holding the step count
  // packed BF16 B fragments (uint2 per lane per tile, 8 bytes)
  int p1, p2, p3, p3t, p2t;   // offsets in uint2 units from pack_base
  int pack_base;              // byte offset of the packed block
  int img;                    // byte offset of the BF16 weight image (kImgBytes)
  int bytes;
};

__host__ __device__ inline MlpLayout mlp_layout() {
  MlpLayout L;
  int o = 0;
  L.w1 = o; o += kFeat * kHid;
  L.b1 = o; o += kHid;
  L.w2 = o; o += kHid * kHid;
  L.b2 = o; o += kHid;
  L.w3 = o; o += kHid * kOut;
  L.b3 = o; o += kOut;
  L.nparam = o;
  L.m = o; o += L.nparam;
  L.v = o; o += L.nparam;
  L.step = o; o += 1;
  int bytes = ((o * 4) + 255) & ~255;
  L.pack_base = bytes;
  int u = 0;
  L.p1 = u; u += kW1Tiles * 32;
  L.p2 = u; u += kW2Tiles * 32;
  L.p3 = u; u += kW3Tiles * 32;
  L.p3t = u; u += kW3TTiles * 32;
  L.p2t = u; u += kW2TTiles * 32;
  L.img = ((bytes + u * 8) + 255) & ~255;
  L.bytes = (L.img + kImgBytes + 255) & ~255;
  return L;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ float2 unpack_bf16x2(uint32_t u) {
  __nv_bfloat162 v = *reinterpret_cast<__nv_bfloat162*>(&u);
  return __bfloat1622float2(v);
}

// D = A (16x16, row) * B (16x8, col) + C, BF16 inputs, FP32 accumulate.
__device__ __forceinline__ void mma_16816(float c[4], const uint32_t a[4], uint2 b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

// Hidden layer from a 16 x 16*KS A operand held as fragments: acc = A W + b,
// then ReLU and conversion to the next layer's A fragments.
// Fragment conventions (g = lane / 4, t = lane % 4):
//   A: a0 = A[g][2t,2t+1], a1 = A[g+8][2t,2t+1], a2 = A[g][2t+8,+9], a3 = A[g+8][2t+8,+9]
//   B: b.x = B[2t,2t+1][g], b.y = B[2t+8,+9][g]
//   C: c0,c1 = C[g][2t,2t+1], c2,c3 = C[g+8][2t,2t+1]
template <int KS>
__device__ __forceinline__ void dense_relu_128(const uint32_t (&a)[KS][4], const uint2* __restrict__ wp,
                                               const float* __restrict__ bias, int lane, uint32_t (&h)[8][4]) {
  const int t = lane & 3;
#pragma unroll
  for (int j = 0; j < 8; ++j) {   // pairs of n-tiles -> one k-step of the next layer
    float c0[4], c1[4];
    const int n0 = (2 * j) * 8 + 2 * t, n1 = (2 * j + 1) * 8 + 2 * t;
    c0[0] = c0[2] = bias[n0]; c0[1] = c0[3] = bias[n0 + 1];
    c1[0] = c1[2] = bias[n1]; c1[1] = c1[3] = bias[n1 + 1];
#pragma unroll
    for (int k = 0; k < KS; ++k) {
      mma_16816(c0, a[k], wp[(k * 16 + 2 * j) * 32 + lane]);
      mma_16816(c1, a[k], wp[(k * 16 + 2 * j + 1) * 32 + lane]);
    }
    h[j][0] = pack_bf16x2(fmaxf(c0[0], 0.f), fmaxf(c0[1], 0.f));
    h[j][1] = pack_bf16x2(fmaxf(c0[2], 0.f), fmaxf(c0[3], 0.f));
    h[j][2] = pack_bf16x2(fmaxf(c1[0], 0.f), fmaxf(c1[1], 0.f));
    h[j][3] = pack_bf16x2(fmaxf(c1[2], 0.f), fmaxf(c1[3], 0.f));
  }
}

// Output layer: out = H2 W3 + b3 (16 x 8, columns 0..2 used).
__device__ __forceinline__ void dense_out(const uint32_t (&h)[8][4], const uint2* __restrict__ wp,
                                          const float* __restrict__ bias, int lane, float c[4]) {
  const int t = lane & 3;
  const int n = 2 * t;
  c[0] = c[2] = n < kOut ? bias[n] : 0.f;
  c[1] = c[3] = n + 1 < kOut ? bias[n + 1] : 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) mma_16816(c, h[k], wp[k * 32 + lane]);
}

}  // namespace jbk
