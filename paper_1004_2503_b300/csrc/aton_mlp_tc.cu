// aton_mlp_tc.cu -- training step of the chemistry-surrogate MLP (5 -> 64 -> 64 -> 3, SiLU) on the
// 5th-generation tensor cores (tcgen05): forward and backward of 128 rows per CTA with BF16
// operands in shared memory and FP32 accumulators in tensor memory (TMEM).
//
// One CTA of 256 threads takes 128 rows; row r is TMEM lane r of every accumulator (M = 128,
// one row per lane). Warp w may read TMEM lanes 32 (w mod 4) .. +31, so warps w and w + 4 share
// the rows of a lane quadrant and split the columns of each accumulator between them. Thread 0
// brings the weight operands in with one bulk copy (they sit in device memory already in the
// shared-memory layout, refreshed by every Adam step), issues the products (tcgen05.mma,
// kind::f16, BF16 x BF16 -> FP32) and commits each group to an mbarrier; the threads read the
// accumulators back with tcgen05.ld, apply the bias and the activation in registers and write
// the next operands to shared memory, a row's 8 consecutive features as one 16-byte store.
// Every activation buffer holds [row][feature] in the canonical layout without swizzle: 8 x 8
// BF16 "core matrices" of 128 bytes (8 rows of 16 bytes, one row's 8 consecutive features),
// the core matrices of an 8-row group 128 bytes apart along the features, the 8-row groups
// (pitch x 16) bytes apart. A product reads such a buffer either K-major (its rows are the
// product's M or N rows, its features the contraction) or, for the weight gradients, MN-major
// (its features are the product's rows and the contraction runs over the 128 rows): the same
// bytes, the transposed copy never written.
//
//   forward   Z1 = X W1^T (K 16), H1 = silu(Z1 + b1); Z2 = H1 W2^T (K 64), H2 = silu(Z2 + b2);
//             Y = H2 W3^T + b3 (N padded to 16)
//   backward  dY = 2 (Y - T) / (rows x 3); dZ2 = (dY W3) * silu'(Z2 + b2) (K 16);
//             dZ1 = (dZ2 W2) * silu'(Z1 + b1) (K 64)
//   weights   [dZ2 | dZ1]^T [H1 | X | 1]  (M 128, N 96, K = the 128 rows): dW2 in the upper left
//             block, dW1 in the lower middle, the bias gradients db2, db1 in the column of ones;
//             H2^T dY (M 128, N 16; rows 64..127 unused): dW3^T. (Both keep M = 128.)
//
// db3 and the loss are summed over the rows in a fixed order. Each CTA writes one FP32 partial
// gradient (the layout of the parameter vector) and its loss; k_mlp_adam sums them.
// Every mbarrier wait is bounded (2 s): a wait that gives up sets *err, the CTA issues no further
// products and frees its tensor memory at the end.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "aton_internal.h"
#include "aton_mlp.cuh"

namespace aton {

namespace {

constexpr int kTcRows = 128;          // rows per CTA = TMEM lanes
constexpr int kTcThreads = kMlpTcThreads;   // two warps per lane quadrant
constexpr unsigned kTmemCols = 256;   // columns allocated (power of two >= 32)
constexpr unsigned kWaitPolls = 1u << 24;
static_assert(kTcThreads == 2 * kTcRows, "two threads per row");

// shared-memory buffers (byte offsets; every block 1024-aligned), [row][feature] canonical
constexpr int kPHX = 96;                             // HX: H1 0..63, X 64..79, 1 at 80, 0 81..95
constexpr int kPH2 = 64, kPDZ = 128, kPDY = 16;      // H2; dZ2 0..63 and dZ1 64..127; dY (3 used)
constexpr uint32_t kSmHX = 0;
constexpr uint32_t kSmH2 = kSmHX + 128 * kPHX * 2;
constexpr uint32_t kSmDZ = kSmH2 + 128 * kPH2 * 2;
constexpr uint32_t kSmDY = kSmDZ + 128 * kPDZ * 2;
constexpr uint32_t kSmW = kSmDY + 128 * kPDY * 2;     // the weight operands (an MlpTcImage)
constexpr uint32_t kSmW1 = kSmW + offsetof(MlpTcImage, W1);
constexpr uint32_t kSmW2 = kSmW + offsetof(MlpTcImage, W2);
constexpr uint32_t kSmW3 = kSmW + offsetof(MlpTcImage, W3);
constexpr uint32_t kSmW2T = kSmW + offsetof(MlpTcImage, W2T);
constexpr uint32_t kSmW3T = kSmW + offsetof(MlpTcImage, W3T);
constexpr uint32_t kSmBias = kSmW + offsetof(MlpTcImage, bias);   // b1[64], b2[64], b3[16]
constexpr uint32_t kSmRed = kSmW + sizeof(MlpTcImage);   // per-warp dy sums [4][16], loss [4]
constexpr uint32_t kSmBar = kSmRed + (4 * 16 + 4) * 4;   // mbarrier of the products
constexpr uint32_t kSmWBar = kSmBar + 8;                 // mbarrier of the weight copy
constexpr uint32_t kSmTmem = kSmWBar + 8;                // TMEM base written by tcgen05.alloc
constexpr uint32_t kTcSmem = kSmTmem + 8 + 1024;         // (+ alignment slack of the base)
static_assert(kSmW % 16 == 0 && sizeof(MlpTcImage) % 16 == 0, "bulk copy alignment");
static_assert(kSmBar % 8 == 0 && kSmWBar % 8 == 0, "mbarrier alignment");
static_assert(kSmDZ - kSmH2 + 128 * kPDZ * 2 >= 17280, "the M = 128 view of H2 stays in bounds");

// byte offset of element (r, c) in a [row][feature] buffer of pitch P features (canonical)
__device__ __forceinline__ uint32_t cano(int r, int c, int P) { return tc_cano(r, c, P); }

// shared-memory matrix descriptor, no swizzle, descriptor version 1: start address, leading
// byte offset (between core matrices adjacent along the contraction) and stride byte offset
// (between core matrices adjacent along the product's rows)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// a [row][feature] buffer of pitch P read K-major (the features are the contraction: 128 bytes
// between feature groups, P x 16 between 8-row groups) or MN-major (the rows are the
// contraction: the same two offsets in the other roles)
__device__ __forceinline__ uint64_t sdesc_k(uint32_t saddr, int P) {
  return sdesc(saddr, 128u, (uint32_t)P * 16u);
}
__device__ __forceinline__ uint64_t sdesc_mn(uint32_t saddr, int P) {
  return sdesc(saddr, (uint32_t)P * 16u, 128u);
}

// instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, M x N; tA / tB set: the
// operand is MN-major
__host__ __device__ constexpr uint32_t idesc(int M, int N, bool tA = false, bool tB = false) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)tA << 15) | ((uint32_t)tB << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// D[tmem] (+)= A B^T for one K = 16 slice
__device__ __forceinline__ void mma16(uint32_t d, uint64_t a, uint64_t b, uint32_t id, bool acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"((uint32_t)acc)
      : "memory");
}

// D = A B^T over K (a multiple of 16), both operands K-major: a, b are their first elements,
// pa, pb their buffers' pitches (a K = 16 slice is two core matrices along the features)
__device__ __forceinline__ void gemm_k(uint32_t d, uint32_t a, int pa, uint32_t b, int pb, int K,
                                       uint32_t id) {
  for (int ks = 0; ks < K / 16; ++ks)
    mma16(d, sdesc_k(a + ks * 256u, pa), sdesc_k(b + ks * 256u, pb), id, ks > 0);
}
// D = A B^T over the 128 rows of both buffers, both MN-major (their features are the product's
// rows): a K = 16 slice is two 8-row groups
__device__ __forceinline__ void gemm_mn(uint32_t d, uint32_t a, int pa, uint32_t b, int pb,
                                        uint32_t id) {
  for (int ks = 0; ks < 128 / 16; ++ks)
    mma16(d, sdesc_mn(a + ks * 32u * pa, pa), sdesc_mn(b + ks * 32u * pb, pb), id, ks > 0);
}

__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}

// bounded wait for the given phase parity of the mbarrier: gives up after kWaitPolls polls or
// 2 s (each poll may suspend the thread for up to 2 us until the phase completes)
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  unsigned long long t0 = 0;
  for (unsigned i = 0; i < kWaitPolls; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity), "r"(2000u)
        : "memory");
    if (done) return true;
    unsigned long long now;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
    if (i == 0) t0 = now;
    else if (now - t0 > 2000000000ull) return false;
  }
  return false;
}

__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 8 consecutive features of a row (one 16-byte store)
__device__ __forceinline__ void put8(unsigned char* sm, uint32_t off, const float* v) {
  uint4 q;
  q.x = pack_bf16(v[0], v[1]);
  q.y = pack_bf16(v[2], v[3]);
  q.z = pack_bf16(v[4], v[5]);
  q.w = pack_bf16(v[6], v[7]);
  *reinterpret_cast<uint4*>(sm + off) = q;
}

// bulk copy (TMA engine) of `bytes` from global to shared memory, completion counted on `bar`
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

}  // namespace

__global__ void __launch_bounds__(kTcThreads, 2)
    k_mlp_train_tc(const MlpTcImage* __restrict__ img, const float* __restrict__ X,
                   const float* __restrict__ T, int n, float inv_count, float* partial,
                   float* loss_part, unsigned int* err) {
  extern __shared__ __align__(1024) unsigned char tc_raw[];
  unsigned char* sm = tc_raw + ((1024u - (su32(tc_raw) & 1023u)) & 1023u);
  const uint32_t sb = su32(sm);
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int r = t & (kTcRows - 1);   // this thread's row (TMEM lane)
  const int hf = t >> 7;             // which half of the accumulator columns it reads
  const int row = blockIdx.x * kTcRows + r;
  const bool valid = row < n;
  float* bias = reinterpret_cast<float*>(sm + kSmBias);
  float* red = reinterpret_cast<float*>(sm + kSmRed);
  const uint32_t bar = sb + kSmBar, wbar = sb + kSmWBar;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kSmTmem);

  if (t == 0) {   // the weight operands: one bulk copy, already in the shared-memory layout
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(wbar));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    bulk_load(sb + kSmW, img, (uint32_t)sizeof(MlpTcImage), wbar);
  }
  float tg[kMlpOut];
  if (hf == 0) {   // this row's input into HX features 64..79 (5 used); its targets
    float v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = valid && k < kMlpIn ? X[(size_t)row * kMlpIn + k] : 0.f;
    put8(sm, kSmHX + cano(r, 64, kPHX), v);
    put8(sm, kSmHX + cano(r, 72, kPHX), v + 8);
#pragma unroll
    for (int k = 0; k < kMlpOut; ++k) tg[k] = valid ? T[(size_t)row * kMlpOut + k] : 0.f;
  } else {         // the column of ones (80) and zeros (81..95)
    float v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = k == 0 ? 1.f : 0.f;
    put8(sm, kSmHX + cano(r, 80, kPHX), v);
    put8(sm, kSmHX + cano(r, 88, kPHX), v + 8);
#pragma unroll
    for (int k = 0; k < kMlpOut; ++k) tg[k] = 0.f;
  }
  if (w == 0) {   // TMEM: 256 columns x 128 lanes of FP32
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     sb + kSmTmem),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const bool wok = bar_wait(wbar, 0);   // the weights have landed
  bool ok = wok;
  const uint32_t tm = *tmem_slot;
  const uint32_t lane_base = tm + ((uint32_t)(32 * (w & 3)) << 16);   // this warp's TMEM lanes
  // TMEM columns: Z1 [0, 64), Z2 then dH1 [64, 128), Y [128, 144), dH2 [144, 208);
  // afterwards the weight products: D' [0, 96), D'' [128, 144)
  const uint32_t cZ1 = 0, cZ2 = 64, cY = 128, cH2 = 144;
  uint32_t phase = 0;
  // issue (thread 0) a group of products and wait for it (every thread)
  auto run = [&](auto issue) {
    if (t == 0) {
      fence_after();
      if (ok) issue();
      commit(bar);
    }
    if (!bar_wait(bar, phase & 1)) ok = false;
    ++phase;
    fence_after();
  };
  // operands written by the threads -> visible to the tensor cores; TMEM reads done
  auto handoff = [&]() {
    fence_async_smem();
    fence_before();
    __syncthreads();
  };
  float z[16], g[16], v[16];
  const int c0 = 32 * hf;   // this thread's 32 of the 64 hidden columns

  // ---- layer 1: Z1 = X W1^T
  run([&] { gemm_k(tm + cZ1, sb + kSmHX + 8 * 128, kPHX, sb + kSmW1, 16, 16, idesc(128, 64)); });
  for (int c = c0; c < c0 + 32; c += 16) {
    tld16(lane_base + cZ1 + c, z);
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = silu(z[j] + bias[c + j]);
    put8(sm, kSmHX + cano(r, c, kPHX), v);
    put8(sm, kSmHX + cano(r, c + 8, kPHX), v + 8);
  }
  handoff();
  // ---- layer 2: Z2 = H1 W2^T
  run([&] { gemm_k(tm + cZ2, sb + kSmHX, kPHX, sb + kSmW2, 64, 64, idesc(128, 64)); });
  for (int c = c0; c < c0 + 32; c += 16) {
    tld16(lane_base + cZ2 + c, z);
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = silu(z[j] + bias[64 + c + j]);
    put8(sm, kSmH2 + cano(r, c, kPH2), v);
    put8(sm, kSmH2 + cano(r, c + 8, kPH2), v + 8);
  }
  handoff();
  // ---- layer 3: Y = H2 W3^T + b3; dY = 2 (Y - T) / (rows x 3); the loss (first half only)
  run([&] { gemm_k(tm + cY, sb + kSmH2, kPH2, sb + kSmW3, 64, 64, idesc(128, 16)); });
  if (hf == 0) {
    float dy[kMlpOut], sq = 0.f;
    tld16(lane_base + cY, z);
#pragma unroll
    for (int k = 0; k < kMlpOut; ++k) {
      const float d = valid ? z[k] + bias[128 + k] - tg[k] : 0.f;
      dy[k] = 2.f * d * inv_count;
      sq += d * d;
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = k < kMlpOut ? dy[k] : 0.f;
    put8(sm, kSmDY + cano(r, 0, kPDY), v);
    put8(sm, kSmDY + cano(r, 8, kPDY), v + 8);
    // per-warp sums of dy (db3) and of the squared error, in lane order
#pragma unroll
    for (int k = 0; k < kMlpOut; ++k) {
      float s = dy[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) red[w * 16 + k] = s;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if (lane == 0) red[64 + w] = sq;
  }
  handoff();
  // ---- dH2 = dY W3 (B = W3^T, K = 16 outputs)
  run([&] { gemm_k(tm + cH2, sb + kSmDY, kPDY, sb + kSmW3T, 16, 16, idesc(128, 64)); });
  // dZ2 = dH2 * silu'(Z2 + b2) into DZ features 0..63
  for (int c = c0; c < c0 + 32; c += 16) {
    tld16(lane_base + cZ2 + c, z);
    tld16(lane_base + cH2 + c, g);
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = g[j] * dsilu(z[j] + bias[64 + c + j]);
    put8(sm, kSmDZ + cano(r, c, kPDZ), v);
    put8(sm, kSmDZ + cano(r, c + 8, kPDZ), v + 8);
  }
  handoff();
  // ---- dH1 = dZ2 W2 (B = W2^T, K = 64) into the columns of Z2
  run([&] { gemm_k(tm + cZ2, sb + kSmDZ, kPDZ, sb + kSmW2T, 64, 64, idesc(128, 64)); });
  // dZ1 = dH1 * silu'(Z1 + b1) into DZ features 64..127
  for (int c = c0; c < c0 + 32; c += 16) {
    tld16(lane_base + cZ1 + c, z);
    tld16(lane_base + cZ2 + c, g);
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = g[j] * dsilu(z[j] + bias[c + j]);
    put8(sm, kSmDZ + cano(r, 64 + c, kPDZ), v);
    put8(sm, kSmDZ + cano(r, 64 + c + 8, kPDZ), v + 8);
  }
  handoff();
  // ---- weight and bias gradients over the rows: [dZ2 | dZ1]^T [H1 | X | 1], H2^T dY
  run([&] {
    gemm_mn(tm + 0, sb + kSmDZ, kPDZ, sb + kSmHX, kPHX, idesc(128, 96, true, true));
    gemm_mn(tm + cY, sb + kSmH2, kPH2, sb + kSmDY, kPDY, idesc(128, 16, true, true));
  });
  float* P = partial + (size_t)blockIdx.x * kMlpPartStride;
  // D' columns: the first half reads 0..47, the second 48..95; lane r < 64 holds row r of dW2
  // (columns 0..63, 16-byte stores), lane r >= 64 row r - 64 of dW1 (columns 64..68); column 80
  // holds db2 (r < 64) and db1 (r >= 64)
  for (int c = 48 * hf; c < 48 * hf + 48; c += 16) {
    tld16(lane_base + c, z);
    if (!ok)
#pragma unroll
      for (int j = 0; j < 16; ++j) z[j] = 0.f;
    if (c < 64) {
      if (r < 64)
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *reinterpret_cast<float4*>(P + kOffW2 + r * kMlpH + c + j) =
              make_float4(z[j], z[j + 1], z[j + 2], z[j + 3]);
    } else if (c == 64) {
      if (r >= 64)
#pragma unroll
        for (int j = 0; j < kMlpIn; ++j) P[kOffW1 + (r - 64) * kMlpIn + j] = z[j];
    } else {   // c == 80
      P[r < 64 ? kOffB2 + r : kOffB1 + (r - 64)] = z[0];
    }
  }
  if (hf == 1) {   // D'': dW3[k][r] for r < 64
    tld16(lane_base + cY, z);
    if (r < 64)
#pragma unroll
      for (int k = 0; k < kMlpOut; ++k) P[kOffW3 + k * kMlpH + r] = ok ? z[k] : 0.f;
  }
  if (t < kMlpOut) P[kOffB3 + t] = red[t] + red[16 + t] + red[32 + t] + red[48 + t];
  if (t == 0) loss_part[blockIdx.x] = red[64] + red[65] + red[66] + red[67];
  if (!ok && t == 0) atomicAdd(err, 1u);
  // if the weight copy did not complete in time, wait (bounded) once more before the CTA exits,
  // so that the copy does not write into shared memory afterwards
  if (!wok && t == 0) bar_wait(wbar, 0);
  fence_before();
  __syncthreads();
  if (w == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(kTmemCols)
                 : "memory");
  }
}

size_t mlp_train_tc_smem() { return kTcSmem; }

}  // namespace aton
