// Warm-start network kernels: fragment packing, batched forward, backward
// (data and weight gradients) and AdamW, BF16 tensor-core operands with FP32
// accumulation, FP32 master weights.  The contact features and targets come
// from the episode kernel's recorder; the packed weights feed its inference.
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
}

constexpr int kPackThreads = (kW1Tiles + kW2Tiles + kW3Tiles + kW3TTiles + kW2TTiles) * 32;

// ------------------------------------------------------------------ forward
// One warp per 16 rows.  Writes X as BF16 [n][32], H1 and H2 as BF16
// [n][128] (pre-activation masks follow from H > 0) and Y as FP32 [n][4].
__global__ void mlp_forward_kernel(const unsigned char* mlp, const float* __restrict__ X, int n,
                                   __nv_bfloat16* Xb, __nv_bfloat16* H1, __nv_bfloat16* H2, float* Y) {
  const MlpLayout L = mlp_layout();
  const float* P = reinterpret_cast<const float*>(mlp);
  const uint2* pk = reinterpret_cast<const uint2*>(mlp + L.pack_base);
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int r0 = warp * 16;
  if (r0 >= n) return;
  const int g = lane >> 2, t = lane & 3;
  const int ra = r0 + g, rb = r0 + g + 8;
  auto x = [&](int r, int c) { return (r < n && c < kFeat) ? X[(size_t)r * kFeat + c] : 0.f; };
  uint32_t a[2][4];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    int c = k * 16 + 2 * t;
    a[k][0] = pack_bf16x2(x(ra, c), x(ra, c + 1));
    a[k][1] = pack_bf16x2(x(rb, c), x(rb, c + 1));
    a[k][2] = pack_bf16x2(x(ra, c + 8), x(ra, c + 9));
    a[k][3] = pack_bf16x2(x(rb, c + 8), x(rb, c + 9));
    if (Xb) {
      if (ra < n) {
        *reinterpret_cast<uint32_t*>(Xb + (size_t)ra * kFeatPad + c) = a[k][0];
        *reinterpret_cast<uint32_t*>(Xb + (size_t)ra * kFeatPad + c + 8) = a[k][2];
      }
      if (rb < n) {
        *reinterpret_cast<uint32_t*>(Xb + (size_t)rb * kFeatPad + c) = a[k][1];
        *reinterpret_cast<uint32_t*>(Xb + (size_t)rb * kFeatPad + c + 8) = a[k][3];
      }
    }
  }
  uint32_t h1[8][4], h2[8][4];
  dense_relu_128<2>(a, pk + L.p1, P + L.b1, lane, h1);
  dense_relu_128<8>(h1, pk + L.p2, P + L.b2, lane, h2);
  float y[4];
  dense_out(h2, pk + L.p3, P + L.b3, lane, y);
  auto store_h = [&](__nv_bfloat16* H, const uint32_t (&h)[8][4]) {
    if (!H) return;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      int c = 16 * j + 2 * t;
      if (ra < n) {
        *reinterpret_cast<uint32_t*>(H + (size_t)ra * kHid + c) = h[j][0];
        *reinterpret_cast<uint32_t*>(H + (size_t)ra * kHid + c + 8) = h[j][2];
      }
      if (rb < n) {
        *reinterpret_cast<uint32_t*>(H + (size_t)rb * kHid + c) = h[j][1];
        *reinterpret_cast<uint32_t*>(H + (size_t)rb * kHid + c + 8) = h[j][3];
      }
    }
  };
  store_h(H1, h1);
  store_h(H2, h2);
  // outputs: lanes with t = 0 hold columns 0, 1; t = 1 holds column 2
  if (t < 2) {
    int c = 2 * t;
    if (ra < n) { Y[(size_t)ra * 4 + c] = y[0]; if (c + 1 < 4) Y[(size_t)ra * 4 + c + 1] = y[1]; }
    if (rb < n) { Y[(size_t)rb * 4 + c] = y[2]; if (c + 1 < 4) Y[(size_t)rb * 4 + c + 1] = y[3]; }
  }
}

// --------------------------------------------------------- backward (data)
// Loss = (1/n) sum_rows sum_c (y - t)^2.  One warp per 16 rows: dY, then
// dH2 = (dY W3^T) * [H2 > 0] and dH1 = (dH2 W2^T) * [H1 > 0], BF16 stores.
__global__ void mlp_backward_data_kernel(const unsigned char* mlp, const float* __restrict__ Y,
                                         const float* __restrict__ T, int n, const __nv_bfloat16* H1,
                                         const __nv_bfloat16* H2, __nv_bfloat16* dY, __nv_bfloat16* dH2,
                                         __nv_bfloat16* dH1, float* loss) {
  const MlpLayout L = mlp_layout();
  const uint2* pk = reinterpret_cast<const uint2*>(mlp + L.pack_base);
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int r0 = warp * 16;
  if (r0 >= n) return;
  const int g = lane >> 2, t = lane & 3;
  const int ra = r0 + g, rb = r0 + g + 8;
  const float s = 2.f / (float)n;
  auto err = [&](int r, int c) {
    return (r < n && c < kOut) ? Y[(size_t)r * 4 + c] - T[(size_t)r * kOut + c] : 0.f;
  };
  // dY as one k-step (16 columns, 3 used)
  uint32_t a[4];
  int c = 2 * t;
  float e0 = err(ra, c), e1 = err(ra, c + 1), e2 = err(rb, c), e3 = err(rb, c + 1);
  a[0] = pack_bf16x2(s * e0, s * e1);
  a[1] = pack_bf16x2(s * e2, s * e3);
  a[2] = 0u;
  a[3] = 0u;
  float l = (e0 * e0 + e1 * e1 + e2 * e2 + e3 * e3) / (float)n;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(FULLM, l, o);
  if (lane == 0 && loss) atomicAdd(loss, l);
  if (t < 4) {   // dY stored [n][8]
    if (ra < n) *reinterpret_cast<uint32_t*>(dY + (size_t)ra * kOutPad + c) = a[0];
    if (rb < n) *reinterpret_cast<uint32_t*>(dY + (size_t)rb * kOutPad + c) = a[1];
  }
  auto relu_mask = [&](const __nv_bfloat16* H, int r, int col) {
    if (r >= n) return make_float2(0.f, 0.f);
    float2 h = unpack_bf16x2(*reinterpret_cast<const uint32_t*>(H + (size_t)r * kHid + col));
    return make_float2(h.x > 0.f ? 1.f : 0.f, h.y > 0.f ? 1.f : 0.f);
  };
  // dH2 = dY W3^T, one k-step over 16 n-tiles
  uint32_t d2[8][4];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float c0[4] = {0.f, 0.f, 0.f, 0.f}, c1[4] = {0.f, 0.f, 0.f, 0.f};
    mma_16816(c0, a, pk[L.p3t + (2 * j) * 32 + lane]);
    mma_16816(c1, a, pk[L.p3t + (2 * j + 1) * 32 + lane]);
    int n0 = 16 * j + 2 * t, n1 = n0 + 8;
    float2 m0a = relu_mask(H2, ra, n0), m0b = relu_mask(H2, rb, n0);
    float2 m1a = relu_mask(H2, ra, n1), m1b = relu_mask(H2, rb, n1);
    d2[j][0] = pack_bf16x2(c0[0] * m0a.x, c0[1] * m0a.y);
    d2[j][1] = pack_bf16x2(c0[2] * m0b.x, c0[3] * m0b.y);
    d2[j][2] = pack_bf16x2(c1[0] * m1a.x, c1[1] * m1a.y);
    d2[j][3] = pack_bf16x2(c1[2] * m1b.x, c1[3] * m1b.y);
    if (ra < n) {
      *reinterpret_cast<uint32_t*>(dH2 + (size_t)ra * kHid + n0) = d2[j][0];
      *reinterpret_cast<uint32_t*>(dH2 + (size_t)ra * kHid + n1) = d2[j][2];
    }
    if (rb < n) {
      *reinterpret_cast<uint32_t*>(dH2 + (size_t)rb * kHid + n0) = d2[j][1];
      *reinterpret_cast<uint32_t*>(dH2 + (size_t)rb * kHid + n1) = d2[j][3];
    }
  }
  // dH1 = dH2 W2^T
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float c0[4] = {0.f, 0.f, 0.f, 0.f}, c1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      mma_16816(c0, d2[k], pk[L.p2t + (k * 16 + 2 * j) * 32 + lane]);
      mma_16816(c1, d2[k], pk[L.p2t + (k * 16 + 2 * j + 1) * 32 + lane]);
    }
    int n0 = 16 * j + 2 * t, n1 = n0 + 8;
    float2 m0a = relu_mask(H1, ra, n0), m0b = relu_mask(H1, rb, n0);
    float2 m1a = relu_mask(H1, ra, n1), m1b = relu_mask(H1, rb, n1);
    if (ra < n) {
      *reinterpret_cast<uint32_t*>(dH1 + (size_t)ra * kHid + n0) = pack_bf16x2(c0[0] * m0a.x, c0[1] * m0a.y);
      *reinterpret_cast<uint32_t*>(dH1 + (size_t)ra * kHid + n1) = pack_bf16x2(c1[0] * m1a.x, c1[1] * m1a.y);
    }
    if (rb < n) {
      *reinterpret_cast<uint32_t*>(dH1 + (size_t)rb * kHid + n0) = pack_bf16x2(c0[2] * m0b.x, c0[3] * m0b.y);
      *reinterpret_cast<uint32_t*>(dH1 + (size_t)rb * kHid + n1) = pack_bf16x2(c1[2] * m1b.x, c1[3] * m1b.y);
    }
  }
}

// ------------------------------------------------------ backward (weights)
// dW[m][j] += sum_b A[b][m] G[b][j] over a chunk of rows; A [n][lda] and
// G [n][ldg] BF16 row-major.  One warp per (16 x 8) tile and row chunk;
// partial tiles are added into the FP32 gradient with atomics.
__global__ void mlp_wgrad_kernel(const __nv_bfloat16* A, int lda, int M, const __nv_bfloat16* G, int ldg, int N,
                                 int n, int chunk, float* dW, int ldw, int mmax, int nmax) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int mt = M / 16, nt = N / 8;
  const int tile = warp % (mt * nt), ck = warp / (mt * nt);
  const int k_begin = ck * chunk;
  if (k_begin >= n) return;
  const int k_end = min(n, k_begin + chunk);
  const int m0 = (tile / nt) * 16, n0 = (tile % nt) * 8;
  const int g = lane >> 2, t = lane & 3;
  const unsigned short* Au = reinterpret_cast<const unsigned short*>(A);
  const unsigned short* Gu = reinterpret_cast<const unsigned short*>(G);
  auto av = [&](int k, int m) -> uint32_t { return k < k_end ? Au[(size_t)k * lda + m] : 0u; };
  auto gv = [&](int k, int j) -> uint32_t { return k < k_end ? Gu[(size_t)k * ldg + j] : 0u; };
  float c[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k0 = k_begin; k0 < k_end; k0 += 16) {
    uint32_t a[4];
    int ka = k0 + 2 * t;
    a[0] = av(ka, m0 + g) | (av(ka + 1, m0 + g) << 16);
    a[1] = av(ka, m0 + g + 8) | (av(ka + 1, m0 + g + 8) << 16);
    a[2] = av(ka + 8, m0 + g) | (av(ka + 9, m0 + g) << 16);
    a[3] = av(ka + 8, m0 + g + 8) | (av(ka + 9, m0 + g + 8) << 16);
    uint2 b;
    b.x = gv(ka, n0 + g) | (gv(ka + 1, n0 + g) << 16);
    b.y = gv(ka + 8, n0 + g) | (gv(ka + 9, n0 + g) << 16);
    mma_16816(c, a, b);
  }
  const int row0 = m0 + g, row1 = m0 + g + 8, col = n0 + 2 * t;
  if (row0 < mmax) {
    if (col < nmax) atomicAdd(dW + row0 * ldw + col, c[0]);
    if (col + 1 < nmax) atomicAdd(dW + row0 * ldw + col + 1, c[1]);
  }
  if (row1 < mmax) {
    if (col < nmax) atomicAdd(dW + row1 * ldw + col, c[2]);
    if (col + 1 < nmax) atomicAdd(dW + row1 * ldw + col + 1, c[3]);
  }
}

// Bias gradient: db[j] += sum over a chunk of rows of G[b][j] (FP32 accumulate).
__global__ void mlp_bgrad_kernel(const __nv_bfloat16* G, int ldg, int N, int nmax, int n, int chunk, float* db) {
  int j = threadIdx.x;
  int k0 = blockIdx.x * chunk;
  if (j >= nmax || k0 >= n) return;
  int k1 = min(n, k0 + chunk);
  float s = 0.f;
  for (int k = k0; k < k1; ++k) s += __bfloat162float(G[(size_t)k * ldg + j]);
  atomicAdd(db + j, s);
  (void)N;
}

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

namespace {
#define MCU(call)                                                                                    \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) return fail(JB_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

struct Scratch {
  __nv_bfloat16 *xb, *h1, *h2, *dy, *dh2, *dh1;
  float *y, *grad, *loss;
  size_t bytes;
};

Scratch carve_scratch(unsigned char* base, int n) {
  Scratch s;
  size_t o = 0;
  auto take = [&](size_t b) { unsigned char* p = base ? base + o : nullptr; o = (o + b + 255) & ~size_t(255); return p; };
  s.xb = (__nv_bfloat16*)take((size_t)n * kFeatPad * 2);
  s.h1 = (__nv_bfloat16*)take((size_t)n * kHid * 2);
  s.h2 = (__nv_bfloat16*)take((size_t)n * kHid * 2);
  s.dy = (__nv_bfloat16*)take((size_t)n * kOutPad * 2);
  s.dh2 = (__nv_bfloat16*)take((size_t)n * kHid * 2);
  s.dh1 = (__nv_bfloat16*)take((size_t)n * kHid * 2);
  s.y = (float*)take((size_t)n * 4 * 4);
  s.grad = (float*)take((size_t)mlp_layout().nparam * 4);
  s.loss = (float*)take(4);
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
  int warps = (n + 15) / 16;
  mlp_forward_kernel<<<blocks_for(warps * 32, 128), 128, 0, s>>>(static_cast<const unsigned char*>(d_mlp), d_x, n,
                                                                nullptr, nullptr, nullptr, sc.y);
  MCU(cudaGetLastError());
  // compact [n][4] -> [n][3]
  MCU(cudaMemcpy2DAsync(d_y, 3 * sizeof(float), sc.y, 4 * sizeof(float), 3 * sizeof(float), n,
                        cudaMemcpyDeviceToDevice, s));
  return JB_OK;
}

// Gradient of the loss (1/n) sum (y - t)^2 with respect to all parameters
// (FP32, in the master-weight layout) and the loss itself.
jb_status jb_mlp_grad(const void* d_mlp, const float* d_x, const float* d_t, int32_t n, float* d_grad, float* d_loss,
                      void* d_scratch, size_t bytes, void* stream) {
  if (!d_mlp || !d_x || !d_t || !d_grad || n <= 0) return fail(JB_EINVAL, "jb_mlp_grad: bad argument");
  if (!d_scratch || bytes < jb_mlp_scratch_bytes(n)) return fail(JB_ENOMEM, "jb_mlp_grad: scratch too small");
  const MlpLayout L = mlp_layout();
  Scratch sc = carve_scratch(static_cast<unsigned char*>(d_scratch), n);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const unsigned char* m = static_cast<const unsigned char*>(d_mlp);
  int warps = (n + 15) / 16;
  mlp_forward_kernel<<<blocks_for(warps * 32, 128), 128, 0, s>>>(m, d_x, n, sc.xb, sc.h1, sc.h2, sc.y);
  MCU(cudaMemsetAsync(d_grad, 0, sizeof(float) * L.nparam, s));
  if (d_loss) MCU(cudaMemsetAsync(d_loss, 0, sizeof(float), s));
  mlp_backward_data_kernel<<<blocks_for(warps * 32, 128), 128, 0, s>>>(m, sc.y, d_t, n, sc.h1, sc.h2, sc.dy, sc.dh2,
                                                                      sc.dh1, d_loss);
  const int chunk = 1024;
  const int nck = (n + chunk - 1) / chunk;
  auto wgrad = [&](const __nv_bfloat16* A, int lda, int M, const __nv_bfloat16* G, int ldg, int N, float* dW,
                   int ldw, int mmax, int nmax) {
    int w = (M / 16) * (N / 8) * nck;
    mlp_wgrad_kernel<<<blocks_for(w * 32, 128), 128, 0, s>>>(A, lda, M, G, ldg, N, n, chunk, dW, ldw, mmax, nmax);
  };
  wgrad(sc.xb, kFeatPad, kFeatPad, sc.dh1, kHid, kHid, d_grad + L.w1, kHid, kFeat, kHid);
  wgrad(sc.h1, kHid, kHid, sc.dh2, kHid, kHid, d_grad + L.w2, kHid, kHid, kHid);
  wgrad(sc.h2, kHid, kHid, sc.dy, kOutPad, kOutPad, d_grad + L.w3, kOut, kHid, kOut);
  mlp_bgrad_kernel<<<nck, 128, 0, s>>>(sc.dh1, kHid, kHid, kHid, n, chunk, d_grad + L.b1);
  mlp_bgrad_kernel<<<nck, 128, 0, s>>>(sc.dh2, kHid, kHid, kHid, n, chunk, d_grad + L.b2);
  mlp_bgrad_kernel<<<nck, 128, 0, s>>>(sc.dy, kOutPad, kOutPad, kOut, n, chunk, d_grad + L.b3);
  MCU(cudaGetLastError());
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
  Scratch sc = carve_scratch(static_cast<unsigned char*>(d_scratch), n);
  if (jb_status st = jb_mlp_grad(d_mlp, d_x, d_t, n, sc.grad, d_loss, d_scratch, bytes, stream)) return st;
  return jb_mlp_adamw(d_mlp, sc.grad, step, lr, beta1, beta2, eps, weight_decay, stream);
}

}  // extern "C"
