// Warm-start network: host entry points, packing (the BF16 fragments of the
// episode kernel's in-warp inference and the BF16 weight image of the
// tensor-core kernel), and AdamW on the FP32 master weights.  Batch
// inference and the training gradient run in the fused tcgen05 kernel of
// jb_mlp_tc.cu.  The contact features and targets come from the episode
// kernel's recorder.
#include <cstdarg>
#include <cstdio>

#include "jb_internal.cuh"
#include "jb_mlp.cuh"

namespace jbk {

#define FULLM 0xffffffffu

// ------------------------------------------------------------------ packing
// B fragment of the (k-tile, n-tile) of B[k][n] = src(k, n) for every lane.
template <class F>
__device__ void pack_tiles(uint2* dst, int KT, int NT, F src, int i) {
  int lane = i & 31, tile = i >> 5;
  if (tile >= KT * NT) return;
  int kt = tile / NT, nt = tile % NT;
  int g = lane >> 2, t = lane & 3;
  int k0 = kt * 16 + 2 * t, n = nt * 8 + g;
  dst[i] = make_uint2(pack_bf16x2(src(k0, n), src(k0 + 1, n)), pack_bf16x2(src(k0 + 8, n), src(k0 + 9, n)));
}

__global__ void mlp_pack_kernel(unsigned char* mlp) {
  const MlpLayout L = mlp_layout();
  const float* P = reinterpret_cast<const float*>(mlp);
  uint2* pk = reinterpret_cast<uint2*>(mlp + L.pack_base);
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  const float* W1 = P + L.w1;
  const float* W2 = P + L.w2;
  const float* W3 = P + L.w3;
  auto w1 = [&](int k, int n) { return k < kFeat ? W1[k * kHid + n] : 0.f; };
  auto w2 = [&](int k, int n) { return W2[k * kHid + n]; };
  auto w3 = [&](int k, int n) { return n < kOut ? W3[k * kOut + n] : 0.f; };
  auto w3t = [&](int k, int n) { return k < kOut ? W3[n * kOut + k] : 0.f; };   // W3^T [16 x 128]
  auto w2t = [&](int k, int n) { return W2[n * kHid + k]; };                    // W2^T
  if (i < kW1Tiles * 32) { pack_tiles(pk + L.p1, kFeatPad / 16, kHid / 8, w1, i); return; }
  i -= kW1Tiles * 32;
  if (i < kW2Tiles * 32) { pack_tiles(pk + L.p2, kHid / 16, kHid / 8, w2, i); return; }
  i -= kW2Tiles * 32;
  if (i < kW3Tiles * 32) { pack_tiles(pk + L.p3, kHid / 16, kOutPad / 8, w3, i); return; }
  i -= kW3Tiles * 32;
  if (i < kW3TTiles * 32) { pack_tiles(pk + L.p3t, kOutPadK / 16, kHid / 8, w3t, i); return; }
  i -= kW3TTiles * 32;
  if (i < kW2TTiles * 32) { pack_tiles(pk + L.p2t, kHid / 16, kHid / 8, w2t, i); return; }
  i -= kW2TTiles * 32;
  // the tensor-core kernel's weight image, 8 BF16 (16 bytes) per thread
  if (i < kImgBytes / 16) {
    unsigned char* img = mlp + L.img;
    int base, K;
    auto src = [&](int r, int k) -> float {
      switch (base) {
        case kImgW1T: return w1(k, r);            // W1^T[j][f] = W1[f][j]
        case kImgW2T: return W2[k * kHid + r];    // W2^T[o][i] = W2[i][o]
        case kImgW2: return W2[r * kHid + k];
        case kImgW3T: return w3(k, r);            // W3^T[o][k] = W3[k][o]
        default: return w3(r, k);                 // W3[k][o]
      }
    };
    int c = i;
    // chunks per tile: [128][32] 512, [128][128] 2048 twice, [16][128] 256, [128][16] 256
    if (c < 512) { base = kImgW1T; K = 32; }
    else if ((c -= 512) < 2048) { base = kImgW2T; K = kHid; }
    else if ((c -= 2048) < 2048) { base = kImgW2; K = kHid; }
    else if ((c -= 2048) < 256) { base = kImgW3T; K = kHid; }
    else { c -= 256; base = kImgW3; K = 16; }
    const int r = c / (K / 8), k = (c % (K / 8)) * 8;
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) w[q] = pack_bf16x2(src(r, k + 2 * q), src(r, k + 2 * q + 1));
    *reinterpret_cast<uint4*>(img + base + kmaj_off(r, k, K)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

constexpr int kPackThreads = (kW1Tiles + kW2Tiles + kW3Tiles + kW3TTiles + kW2TTiles) * 32 + kImgBytes / 16;

// AdamW on the master weights (decoupled weight decay on the matrices only).
__global__ void mlp_adamw_kernel(unsigned char* mlp, const float* __restrict__ grad, float lr, float b1, float b2,
                                 float eps, float wd, float bc1, float bc2) {
  const MlpLayout L = mlp_layout();
  float* P = reinterpret_cast<float*>(mlp);
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.nparam) return;
  bool is_bias = (i >= L.b1 && i < L.w2) || (i >= L.b2 && i < L.w3) || i >= L.b3;
  float g = grad[i];
  float m = P[L.m + i] = b1 * P[L.m + i] + (1.f - b1) * g;
  float v = P[L.v + i] = b2 * P[L.v + i] + (1.f - b2) * g * g;
  float w = P[i];
  if (!is_bias) w -= lr * wd * w;
  w -= lr * (m / bc1) / (sqrtf(v / bc2) + eps);
  P[i] = w;
}

}  // namespace jbk

using namespace jbk;

cudaError_t jbk_mlp_tc_launch(const unsigned char* mlp, const float* X, const float* T, int n, int mode, float* Y,
                              float* part, int pstride, float* grad, float* loss, int* err, cudaStream_t s);

namespace {
#define MCU(call)                                                                                    \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) return fail(JB_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

struct Scratch {
  float *grad, *loss, *part;
  int* err;
  int pstride;
  size_t bytes;
};

// gradient, loss, error flag, and the per-CTA partial sums of the gradient
// kernel (one row of pstride floats per CTA, min(tiles, kTcMaxGrid) rows)
Scratch carve_scratch(unsigned char* base, int n) {
  Scratch s;
  size_t o = 0;
  auto take = [&](size_t b) { unsigned char* p = base ? base + o : nullptr; o = (o + b + 255) & ~size_t(255); return p; };
  const int nparam = mlp_layout().nparam;
  s.pstride = (nparam + 1 + 63) & ~63;
  const int tiles = (n + 127) / 128;
  const int rows = tiles < kTcMaxGrid ? tiles : kTcMaxGrid;
  s.grad = (float*)take((size_t)nparam * 4);
  s.loss = (float*)take(4);
  s.err = (int*)take(4);
  s.part = (float*)take((size_t)rows * s.pstride * 4);
  s.bytes = o;
  return s;
}

unsigned blocks_for(int threads, int per) { return (unsigned)((threads + per - 1) / per); }
}  // namespace

extern "C" {

size_t jb_mlp_bytes(void) { return (size_t)mlp_layout().bytes; }
int32_t jb_mlp_param_count(void) { return mlp_layout().nparam; }
size_t jb_mlp_scratch_bytes(int32_t n) { return n > 0 ? carve_scratch(nullptr, n).bytes : 0; }

jb_status jb_mlp_load(void* d_mlp, const float* params, void* stream) {
  if (!d_mlp || !params) return fail(JB_EINVAL, "jb_mlp_load: null argument");
  const MlpLayout L = mlp_layout();
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* m = static_cast<unsigned char*>(d_mlp);
  MCU(cudaMemcpyAsync(m, params, sizeof(float) * L.nparam, cudaMemcpyHostToDevice, s));
  MCU(cudaMemsetAsync(m + sizeof(float) * L.m, 0, sizeof(float) * (2 * L.nparam + 1), s));
  mlp_pack_kernel<<<blocks_for(kPackThreads, 256), 256, 0, s>>>(m);
  MCU(cudaGetLastError());
  MCU(cudaStreamSynchronize(s));
  return JB_OK;
}

jb_status jb_mlp_save(const void* d_mlp, float* params, void* stream) {
  if (!d_mlp || !params) return fail(JB_EINVAL, "jb_mlp_save: null argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  MCU(cudaMemcpyAsync(params, d_mlp, sizeof(float) * mlp_layout().nparam, cudaMemcpyDeviceToHost, s));
  MCU(cudaStreamSynchronize(s));
  return JB_OK;
}

jb_status jb_mlp_forward(const void* d_mlp, const float* d_x, int32_t n, float* d_y, void* d_scratch,
                         size_t bytes, void* stream) {
  if (!d_mlp || !d_x || !d_y || n < 0) return fail(JB_EINVAL, "jb_mlp_forward: bad argument");
  if (n == 0) return JB_OK;
  if (!d_scratch || bytes < jb_mlp_scratch_bytes(n)) return fail(JB_ENOMEM, "jb_mlp_forward: scratch too small");
  Scratch sc = carve_scratch(static_cast<unsigned char*>(d_scratch), n);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  MCU(cudaMemsetAsync(sc.err, 0, sizeof(int), s));
  MCU(jbk_mlp_tc_launch(static_cast<const unsigned char*>(d_mlp), d_x, nullptr, n, 0, d_y, nullptr, 0, nullptr,
                        nullptr, sc.err, s));
  return JB_OK;
}

// Gradient of the loss (1/n) sum (y - t)^2 with respect to all parameters
// (FP32, in the master-weight layout) and the loss itself: one launch of the
// fused tensor-core kernel (forward, backward and the weight and bias sums).
jb_status jb_mlp_grad(const void* d_mlp, const float* d_x, const float* d_t, int32_t n, float* d_grad, float* d_loss,
                      void* d_scratch, size_t bytes, void* stream) {
  if (!d_mlp || !d_x || !d_t || !d_grad || n <= 0) return fail(JB_EINVAL, "jb_mlp_grad: bad argument");
  if (!d_scratch || bytes < jb_mlp_scratch_bytes(n)) return fail(JB_ENOMEM, "jb_mlp_grad: scratch too small");
  Scratch sc = carve_scratch(static_cast<unsigned char*>(d_scratch), n);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  MCU(cudaMemsetAsync(sc.err, 0, sizeof(int), s));
  MCU(jbk_mlp_tc_launch(static_cast<const unsigned char*>(d_mlp), d_x, d_t, n, 1, nullptr, sc.part, sc.pstride,
                        d_grad, d_loss, sc.err, s));
  return JB_OK;
}

jb_status jb_mlp_scratch_error(const void* d_scratch, size_t bytes, void* stream, int32_t* out) {
  if (!d_scratch || !out || bytes < jb_mlp_scratch_bytes(1)) return fail(JB_EINVAL, "jb_mlp_scratch_error: bad argument");
  Scratch sc = carve_scratch(static_cast<unsigned char*>(const_cast<void*>(d_scratch)), 1);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int v = 0;
  MCU(cudaMemcpyAsync(&v, sc.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  MCU(cudaStreamSynchronize(s));
  *out = v;
  return JB_OK;
}

jb_status jb_mlp_adamw(void* d_mlp, const float* d_grad, int32_t step, float lr, float beta1, float beta2, float eps,
                       float weight_decay, void* stream) {
  if (!d_mlp || !d_grad || step < 1) return fail(JB_EINVAL, "jb_mlp_adamw: bad argument");
  const MlpLayout L = mlp_layout();
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* m = static_cast<unsigned char*>(d_mlp);
  float bc1 = 1.f - powf(beta1, (float)step), bc2 = 1.f - powf(beta2, (float)step);
  mlp_adamw_kernel<<<blocks_for(L.nparam, 256), 256, 0, s>>>(m, d_grad, lr, beta1, beta2, eps, weight_decay, bc1, bc2);
  mlp_pack_kernel<<<blocks_for(kPackThreads, 256), 256, 0, s>>>(m);
  MCU(cudaGetLastError());
  return JB_OK;
}

// One training step on rows [0, n) of (X, T): gradient, then AdamW.
jb_status jb_mlp_train_step(void* d_mlp, const float* d_x, const float* d_t, int32_t n, int32_t step, float lr,
                            float beta1, float beta2, float eps, float weight_decay, float* d_loss, void* d_scratch,
                            size_t bytes, void* stream) {
  if (n <= 0) return fail(JB_EINVAL, "jb_mlp_train_step: n must be > 0");
  if (!d_scratch || bytes < jb_mlp_scratch_bytes(n)) return fail(JB_ENOMEM, "jb_mlp_train_step: scratch too small");
  Scratch sc = carve_scratch(static_cast<unsigned char*>(d_scratch), n);
  if (jb_status st = jb_mlp_grad(d_mlp, d_x, d_t, n, sc.grad, d_loss, d_scratch, bytes, stream)) return st;
  return jb_mlp_adamw(d_mlp, sc.grad, step, lr, beta1, beta2, eps, weight_decay, stream);
}

}  // extern "C"
