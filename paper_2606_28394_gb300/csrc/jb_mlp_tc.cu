// Warm-start network on the fifth-generation tensor cores (tcgen05): batch
// inference and the training gradient, one fused kernel.
//
// A CTA of 128 threads owns a tile of 128 rows (contact samples); thread t is
// row t of the tile and lane t of tensor memory (TMEM).  Per tile:
//   forward   D1 = X W1, H1 = relu(D1 + b1); D2 = H1 W2, H2 = relu(D2 + b2);
//             D3 = H2 W3, y = D3 + b3
//   backward  dY = (2/n)(y - t); dH2 = (dY W3^T) . [H2 > 0];
//             dH1 = (dH2 W2^T) . [H1 > 0]
//   gradients dW2 += H1^T dH2, dW3 += H2^T dY, dW1^T += dH1^T X,
//             db2 += dH2^T 1, db1 += dH1^T 1 (a matrix of ones as B)
// Every product is one tcgen05.mma sequence issued by thread 0 (M = 128, K =
// 16 per instruction, BF16 operands, FP32 accumulators in TMEM), completion
// signalled through an mbarrier.  The epilogues read the accumulators back
// with tcgen05.ld (one TMEM lane per thread), apply bias, ReLU or the ReLU
// mask, round to BF16 and write the next operands to shared memory.  The
// weight-gradient accumulators stay in TMEM across the CTA's tiles; at the
// end each CTA writes them as one row of partial sums, and a second kernel
// adds the rows in CTA order, so the gradient repeats bit for bit.
//
// Operands live in shared memory in the K-major layout without swizzle:
// 8 x 8 BF16 core matrices (8 rows of 16 bytes, contiguous), the core
// matrices of a row group adjacent along K (leading byte offset 128 B), row
// groups K * 16 B apart (stride byte offset).  Every activation is needed
// K-major along both of its dimensions (the forward contracts over features,
// the weight gradient over rows), so the epilogues write it twice: as the
// thread's own row, and transposed as the thread's own column.
//
// The weights arrive in one bulk copy (cp.async.bulk, the TMA engine) of
// the BF16 image that the pack kernel keeps in the network block in exactly
// this layout; the rows are read by the threads (24 FP32 features each).
//
// Waits on the mbarrier are bounded (about one second); a wait that runs out
// sets the error flag, and the CTA frees its TMEM and returns.
#include <cuda_bf16.h>

#include "jb_internal.cuh"
#include "jb_mlp.cuh"

namespace jbk {
namespace tc {

constexpr int kRows = 128;        // rows per tile = MMA M = threads = TMEM lanes
constexpr int kTmemCols = 512;
// TMEM columns
constexpr int kColWork = 0;       // D1, D2, D3, dH2 and dH1 pre-activations in turn (128)
constexpr int kColDW2 = 128;      // dW2 [128 in][128 out]
constexpr int kColDW1 = 256;      // dW1^T [128 hidden][32 features]
constexpr int kColDW3 = 288;      // dW3 [128 hidden][16 outputs]
constexpr int kColDB1 = 304;      // db1, replicated over 16 columns
constexpr int kColDB2 = 320;      // db2
// dynamic shared memory (bytes); K-major BF16 tiles [rows][K]
constexpr int kSzW1T = 128 * 32 * 2;    // W1^T [128 hidden][32 features]
constexpr int kSzH = 128 * 128 * 2;     // any [128][128] tile
constexpr int kSzW3T = 16 * 128 * 2;    // W3^T [16 outputs][128 hidden]
constexpr int kSzW3 = 128 * 16 * 2;     // W3 [128 hidden][16 outputs]
constexpr int kSzX = 128 * 32 * 2;      // X [128 rows][32 features]
constexpr int oW1T = 0;
constexpr int oW2T = oW1T + kSzW1T;     // W2^T [128 out][128 in]  (B of D2 = H1 W2)
constexpr int oW2 = oW2T + kSzH;        // W2 [128 in][128 out]    (B of dH1 = dH2 W2^T)
constexpr int oW3T = oW2 + kSzH;
constexpr int oW3 = oW3T + kSzW3T;
constexpr int oXR = oW3 + kSzW3;        // X; then dY [128][16] | dY^T [16][128]; then ones [16][128]
constexpr int oXT = oXR + kSzX;         // X^T [32 features][128 rows]
constexpr int oR1 = oXT + kSzX;         // H1 [rows][hidden]; then dH2 [rows][hidden]
constexpr int oH1T = oR1 + kSzH;        // H1^T [hidden][rows]
constexpr int oR2 = oH1T + kSzH;        // H2 [rows][hidden]; then dH1^T [hidden][rows]
constexpr int oR3 = oR2 + kSzH;         // H2^T [hidden][rows]; then dH2^T [hidden][rows]
constexpr int kSmemBytes = oR3 + kSzH;  // 229,376
static_assert(kSmemBytes <= 227 * 1024 - 2048, "fused tile must fit one CTA's shared memory");
static_assert(oW1T == kImgW1T && oW2T == kImgW2T && oW2 == kImgW2 && oW3T == kImgW3T && oW3 == kImgW3 &&
                  oXR == kImgBytes,
              "the weight tiles are the pack kernel's image, byte for byte");

// Byte offset of element (r, k) of a K-major tile with K columns.
__device__ __forceinline__ uint32_t kmaj(int r, int k, int K) { return kmaj_off(r, k, K); }

// Shared-memory matrix descriptor: K-major, no swizzle, leading byte offset
// 128 (the second core matrix of a K = 16 step), stride byte offset K * 16
// (the next group of 8 rows), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, int K) {
  const uint64_t lbo = 128u >> 4, sbo = (uint64_t)(K * 16) >> 4;
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | (lbo << 16) | (sbo << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

// D (+)= A B over `ksteps` K = 16 steps: A a K-major tile with Ka columns at
// a, B one with Kb columns at b (both advance 256 bytes = two core matrices
// per step).  acc = false overwrites D on the first step.
__device__ __forceinline__ void umma_seq(uint32_t d, uint32_t a, int Ka, uint32_t b, int Kb, int ksteps, uint32_t id,
                                         bool acc) {
  for (int s = 0; s < ksteps; ++s)
    umma(d, sdesc(a + 256u * s, Ka), sdesc(b + 256u * s, Kb), id, (s > 0 || acc) ? 1u : 0u);
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory stores become visible to the tensor cores
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > (2ll << 30)) return false;   // about one second
  }
}

// 16 consecutive FP32 columns of this thread's TMEM lane (taddr carries the
// warp's lane quadrant).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void st16(unsigned char* sm, uint32_t off, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  *reinterpret_cast<uint4*>(sm + off) = make_uint4(a, b, c, d);
}
__device__ __forceinline__ void st_bf16(unsigned char* sm, uint32_t off, float v) {
  *reinterpret_cast<__nv_bfloat16*>(sm + off) = __float2bfloat16_rn(v);
}

// Epilogue of a [128 x 128] accumulator: value(c, v) of each column of this
// thread's row, rounded to BF16, stored as row `tid` of the tile at `row_off`
// (if >= 0) and as column `tid` of the tile at `col_off` (if >= 0); bit c of
// mask is set where the BF16 value is positive.
template <class F>
__device__ __forceinline__ void epilogue128(unsigned char* sm, uint32_t taddr, int tid, int row_off, int col_off,
                                            uint32_t (&mask)[4], F value) {
#pragma unroll
  for (int i = 0; i < 4; ++i) mask[i] = 0u;
  for (int c0 = 0; c0 < 128; c0 += 16) {
    float v[16];
    tmem_ld16(taddr + c0, v);
    uint32_t w[8];
#pragma unroll
    for (int i = 0; i < 16; i += 2) {
      const __nv_bfloat16 lo = __float2bfloat16_rn(value(c0 + i, v[i]));
      const __nv_bfloat16 hi = __float2bfloat16_rn(value(c0 + i + 1, v[i + 1]));
      const float flo = __bfloat162float(lo), fhi = __bfloat162float(hi);
      if (flo > 0.f) mask[(c0 + i) >> 5] |= 1u << ((c0 + i) & 31);
      if (fhi > 0.f) mask[(c0 + i + 1) >> 5] |= 1u << ((c0 + i + 1) & 31);
      w[i >> 1] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
      if (col_off >= 0) {
        *reinterpret_cast<__nv_bfloat16*>(sm + col_off + kmaj(c0 + i, tid, 128)) = lo;
        *reinterpret_cast<__nv_bfloat16*>(sm + col_off + kmaj(c0 + i + 1, tid, 128)) = hi;
      }
    }
    if (row_off >= 0) {
      st16(sm, row_off + kmaj(tid, c0, 128), w[0], w[1], w[2], w[3]);
      st16(sm, row_off + kmaj(tid, c0 + 8, 128), w[4], w[5], w[6], w[7]);
    }
  }
}

__device__ __forceinline__ bool bit(const uint32_t (&m)[4], int c) { return (m[c >> 5] >> (c & 31)) & 1u; }

// mode 0: forward only, Y [n][3]; mode 1: loss and gradient (grad and loss
// accumulated with atomics, zeroed by the caller).
__global__ void __launch_bounds__(kRows, 1)
    mlp_tc_kernel(const unsigned char* __restrict__ mlp, const float* __restrict__ X, const float* __restrict__ T,
                  int n, int mode, float* __restrict__ Y, float* __restrict__ part, int pstride,
                  int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ float b1s[kHid], b2s[kHid], b3s[4];
  __shared__ float red_s[4][4];   // per warp: the three output-bias sums and the loss
  __shared__ int bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const MlpLayout L = mlp_layout();
  const float* P = reinterpret_cast<const float*>(mlp);
  const int ntiles = (n + kRows - 1) / kRows;
  if ((int)blockIdx.x >= ntiles) return;
  const uint32_t mb = smem_u32(&mbar);

  b1s[tid] = P[L.b1 + tid];
  b2s[tid] = P[L.b2 + tid];
  if (tid < 4) b3s[tid] = tid < kOut ? P[L.b3 + tid] : 0.f;
  if (tid < 16) red_s[tid >> 2][tid & 3] = 0.f;
  if (tid == 0) {
    bad = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // the weights: one bulk copy (TMA) of the BF16 image the pack kernel keeps
  // in the block, in exactly this shared-memory layout
  if (tid == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(kImgBytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(sm + oW1T)),
                 "l"(mlp + L.img), "r"(kImgBytes), "r"(mb)
                 : "memory");
  }
  if (mode == 1)
    // X^T rows of the padding features stay zero
    for (int f = kFeat; f < 32; ++f) st_bf16(sm, oXT + kmaj(f, tid, 128), 0.f);
  fence_async_smem();
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tb = tmem_base;
  const uint32_t tl = tb + ((uint32_t)(warp * 32) << 16);   // this warp's TMEM lanes
  const uint32_t s0 = smem_u32(sm);
  uint32_t phase = 0;
  if (!mbar_wait(mb, phase)) bad = 1;   // the weight image
  phase ^= 1u;
  __syncthreads();

  // the issuing thread orders its MMAs after the epilogue's stores and TMEM
  // reads; every thread then waits for their completion
  auto issue_begin = [&]() {
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
  };
  auto wait_done = [&]() -> bool {
    if (!mbar_wait(mb, phase)) bad = 1;
    phase ^= 1u;
    tc_after_sync();
    __syncthreads();
    return bad == 0;
  };

  bool first = true;
  for (int tile = bad ? ntiles : (int)blockIdx.x; tile < ntiles; tile += gridDim.x, first = false) {
    const int row = tile * kRows + tid;
    const bool live = row < n;
    // X row -> X [rows][32] (A of D1) and, for the gradient, X^T [32][rows]
    {
      float x[32];
#pragma unroll
      for (int f = 0; f < 32; ++f) x[f] = (live && f < kFeat) ? X[(size_t)row * kFeat + f] : 0.f;
#pragma unroll
      for (int k = 0; k < 32; k += 8)
        st16(sm, oXR + kmaj(tid, k, 32), pack_bf16x2(x[k], x[k + 1]), pack_bf16x2(x[k + 2], x[k + 3]),
             pack_bf16x2(x[k + 4], x[k + 5]), pack_bf16x2(x[k + 6], x[k + 7]));
      if (mode == 1)
#pragma unroll
        for (int f = 0; f < kFeat; ++f) st_bf16(sm, oXT + kmaj(f, tid, 128), x[f]);
    }
    issue_begin();
    if (tid == 0) {
      tc_after_sync();
      umma_seq(tb + kColWork, s0 + oXR, 32, s0 + oW1T, 32, 2, idesc(128, 128), false);
      umma_commit(mb);
    }
    if (!wait_done()) break;
    uint32_t m1[4], m2[4];
    // H1 = relu(D1 + b1): rows (A of D2) and, for the gradient, columns (A of dW2)
    epilogue128(sm, tl + kColWork, tid, oR1, mode == 1 ? oH1T : -1, m1,
                [&](int c, float v) { return fmaxf(v + b1s[c], 0.f); });
    issue_begin();
    if (tid == 0) {
      tc_after_sync();
      umma_seq(tb + kColWork, s0 + oR1, 128, s0 + oW2T, 128, 8, idesc(128, 128), false);
      umma_commit(mb);
    }
    if (!wait_done()) break;
    // H2 = relu(D2 + b2)
    epilogue128(sm, tl + kColWork, tid, oR2, mode == 1 ? oR3 : -1, m2,
                [&](int c, float v) { return fmaxf(v + b2s[c], 0.f); });
    issue_begin();
    if (tid == 0) {
      tc_after_sync();
      umma_seq(tb + kColWork, s0 + oR2, 128, s0 + oW3T, 128, 8, idesc(128, 16), false);
      umma_commit(mb);
    }
    if (!wait_done()) break;
    // y = D3 + b3
    float y[3];
    {
      float v[16];
      tmem_ld16(tl + kColWork, v);
#pragma unroll
      for (int o = 0; o < kOut; ++o) y[o] = v[o] + b3s[o];
    }
    if (mode == 0) {
      if (live)
#pragma unroll
        for (int o = 0; o < kOut; ++o) Y[(size_t)row * kOut + o] = y[o];
      // the next tile's D1 overwrites the accumulator this thread just read
      tc_before_sync();
      __syncthreads();
      continue;
    }
    // dY = (2/n)(y - t) as rows [rows][16] (A of dH2) and columns [16][rows]
    // (B of dW3); the loss and db3 from the same values
    {
      const float s = 2.f / (float)n;
      float e[3], d[3], l2 = 0.f;
#pragma unroll
      for (int o = 0; o < kOut; ++o) {
        e[o] = live ? y[o] - T[(size_t)row * kOut + o] : 0.f;
        l2 += e[o] * e[o];
        d[o] = __bfloat162float(__float2bfloat16_rn(s * e[o]));
      }
      st16(sm, oXR + kmaj(tid, 0, 16), pack_bf16x2(d[0], d[1]), pack_bf16x2(d[2], 0.f), 0u, 0u);
      st16(sm, oXR + kmaj(tid, 8, 16), 0u, 0u, 0u, 0u);
#pragma unroll
      for (int o = 0; o < 16; ++o) st_bf16(sm, oXR + kSzW3 + kmaj(o, tid, 128), o < kOut ? d[o] : 0.f);
      float red[4] = {d[0], d[1], d[2], l2 / (float)n};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) red[i] += __shfl_xor_sync(0xffffffffu, red[i], o);
      if (lane == 0)
#pragma unroll
        for (int i = 0; i < 4; ++i) red_s[warp][i] += red[i];
    }
    issue_begin();
    if (tid == 0) {
      tc_after_sync();
      // dH2 pre-mask = dY W3^T; dW3 += H2^T dY
      umma_seq(tb + kColWork, s0 + oXR, 16, s0 + oW3, 16, 1, idesc(128, 128), false);
      umma_seq(tb + kColDW3, s0 + oR3, 128, s0 + oXR + kSzW3, 128, 8, idesc(128, 16), !first);
      umma_commit(mb);
    }
    if (!wait_done()) break;
    // dH2 = D . [H2 > 0]: rows (A of dH1) and columns (B of dW2, A of db2);
    // a [16][rows] tile of ones for the bias sums
    {
      uint32_t unused[4];
      epilogue128(sm, tl + kColWork, tid, oR1, oR3, unused,
                  [&](int c, float v) { return bit(m2, c) ? v : 0.f; });
#pragma unroll
      for (int o = 0; o < 16; ++o) st_bf16(sm, oXR + kmaj(o, tid, 128), 1.f);
    }
    issue_begin();
    if (tid == 0) {
      tc_after_sync();
      // dH1 pre-mask = dH2 W2^T; dW2 += H1^T dH2; db2 += dH2^T 1
      umma_seq(tb + kColWork, s0 + oR1, 128, s0 + oW2, 128, 8, idesc(128, 128), false);
      umma_seq(tb + kColDW2, s0 + oH1T, 128, s0 + oR3, 128, 8, idesc(128, 128), !first);
      umma_seq(tb + kColDB2, s0 + oR3, 128, s0 + oXR, 128, 8, idesc(128, 16), !first);
      umma_commit(mb);
    }
    if (!wait_done()) break;
    // dH1 = D . [H1 > 0] as columns [hidden][rows] (A of dW1^T and db1)
    {
      uint32_t unused[4];
      epilogue128(sm, tl + kColWork, tid, -1, oR2, unused, [&](int c, float v) { return bit(m1, c) ? v : 0.f; });
    }
    issue_begin();
    if (tid == 0) {
      tc_after_sync();
      // dW1^T += dH1^T X; db1 += dH1^T 1
      umma_seq(tb + kColDW1, s0 + oR2, 128, s0 + oXT, 128, 8, idesc(128, 32), !first);
      umma_seq(tb + kColDB1, s0 + oR2, 128, s0 + oXR, 128, 8, idesc(128, 16), !first);
      umma_commit(mb);
    }
    if (!wait_done()) break;
  }

  if (mode == 1 && bad == 0) {
    // this CTA's partial sums, in the parameter layout, at row blockIdx.x of
    // the partials (summed over CTAs in a fixed order by the next kernel, so
    // that the gradient is bitwise reproducible); this thread's TMEM lane is
    // hidden unit tid of every accumulator
    float* g = part + (size_t)blockIdx.x * pstride;
    float v[16];
    for (int c0 = 0; c0 < kHid; c0 += 16) {
      tmem_ld16(tl + kColDW2 + c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) g[L.w2 + tid * kHid + c0 + i] = v[i];
    }
    for (int c0 = 0; c0 < 32; c0 += 16) {
      tmem_ld16(tl + kColDW1 + c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (c0 + i < kFeat) g[L.w1 + (c0 + i) * kHid + tid] = v[i];
    }
    tmem_ld16(tl + kColDW3, v);
#pragma unroll
    for (int o = 0; o < kOut; ++o) g[L.w3 + tid * kOut + o] = v[o];
    tmem_ld16(tl + kColDB1, v);
    g[L.b1 + tid] = v[0];
    tmem_ld16(tl + kColDB2, v);
    g[L.b2 + tid] = v[0];
    if (tid < 4) {
      const float r = ((red_s[0][tid] + red_s[1][tid]) + red_s[2][tid]) + red_s[3][tid];
      if (tid < kOut) g[L.b3 + tid] = r;
      else g[L.nparam] = r;   // the loss
    }
  }
  if (bad && tid == 0) {
    atomicExch(err, 1);
    // let MMAs still in flight finish (bounded) before the TMEM goes
    mbar_wait(mb, phase);
  }
  tc_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tb), "r"(kTmemCols));
  }
}

// grad[i] = sum over the G CTA partials of entry i, in CTA order (entry
// nparam is the loss).
__global__ void mlp_partial_sum_kernel(const float* __restrict__ part, int G, int pstride, float* __restrict__ grad,
                                       float* __restrict__ loss) {
  const MlpLayout L = mlp_layout();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > L.nparam) return;
  float s = 0.f;
  for (int b = 0; b < G; ++b) s += part[(size_t)b * pstride + i];
  if (i < L.nparam) grad[i] = s;
  else if (loss) *loss = s;
}

}  // namespace tc
}  // namespace jbk

// Launches the fused kernel over n rows: grid = min(tiles, SMs, kTcMaxGrid),
// one CTA per SM (its shared memory fills the SM); for the gradient, then the
// fixed-order sum of the CTAs' partials (part holds kTcMaxGrid rows of
// pstride floats).  Returns a CUDA error code.
cudaError_t jbk_mlp_tc_launch(const unsigned char* mlp, const float* X, const float* T, int n, int mode, float* Y,
                              float* part, int pstride, float* grad, float* loss, int* err, cudaStream_t s) {
  using namespace jbk::tc;
  static int configured_device = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (configured_device != dev) {
    e = cudaFuncSetAttribute(mlp_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e != cudaSuccess) return e;
    configured_device = dev;
  }
  int nsm = 0;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int tiles = (n + kRows - 1) / kRows;
  int grid = tiles < nsm ? tiles : nsm;
  if (grid > jbk::kTcMaxGrid) grid = jbk::kTcMaxGrid;
  if (grid <= 0) return cudaSuccess;
  mlp_tc_kernel<<<grid, kRows, kSmemBytes, s>>>(mlp, X, T, n, mode, Y, part, pstride, err);
  e = cudaGetLastError();
  if (e != cudaSuccess || mode != 1) return e;
  const int nsum = jbk::mlp_layout().nparam + 1;
  mlp_partial_sum_kernel<<<(nsum + 255) / 256, 256, 0, s>>>(part, grid, pstride, grad, loss);
  return cudaGetLastError();
}
