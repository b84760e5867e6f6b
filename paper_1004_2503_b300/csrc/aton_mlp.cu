// aton_mlp.cu -- training and inference kernels of the chemistry-surrogate MLP and its C ABI.
//
// The surrogate replaces the sub-cycled chemistry operator Phi (Appendix Eq. A4) for cells that
// would sub-cycle heavily. Features of a cell are (log10 nH, log10 y, log10 T, log10 N, log10 dt);
// targets are the changes (log10 y' - log10 y, log10 T' - log10 T, log10 N' - log10 N), both
// standardised with statistics of the training set. Training pairs come from the exact
// operator (the plain step's chemistry kernel writes them through a pair sink).
//
// Kernels:
//   k_mlp_train   -- forward and backward of 128 rows per CTA on BF16 tensor cores (mma.sync
//                    m16n8k16, FP32 accumulation); the weight gradients are tensor-core products
//                    over the CTA's rows of transposed BF16 copies held in shared memory; one FP32
//                    partial gradient per CTA (summed later in a fixed order: deterministic).
//   k_mlp_adam    -- sums the partials, Adam update of the FP32 master weights, refreshes the
//                    BF16 weight image.
//   k_mlp_forward -- inference (normalised features -> normalised outputs).
//   k_mlp_features, k_mlp_stats, k_mlp_norm_final -- features/targets of pair records and their
//                    standardisation.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>

#include "aton_internal.h"
#include "aton_mlp.cuh"

namespace aton {

namespace {

constexpr int kRows = 128;          // rows per training CTA (8 warps x 16)
constexpr int kTP = kRows + 8;      // row pitch of the transposed activation copies
constexpr int kThreads = 256;
constexpr int kRecLen = 8;          // pair record: nH, N, y, T, N', y', T', sub-steps

struct TrainSmem {
  MlpImage W;
  __nv_bfloat16 XT[16 * kTP];       // [input][row]
  __nv_bfloat16 H1T[kMlpH * kTP];   // [unit][row]
  __nv_bfloat16 H2T[kMlpH * kTP];
  __nv_bfloat16 D1T[kMlpH * kTP];   // dL/dz1, [unit][row]
  __nv_bfloat16 D2T[kMlpH * kTP];
  __nv_bfloat16 DYT[16 * kTP];      // dL/dy, [output][row] (rows 8..15 stay zero)
  float db1[8][kMlpH], db2[8][kMlpH], db3[8][8];
  float loss[8];
};

__device__ __forceinline__ void copy_image(MlpImage* dst, const MlpImage* src, bool full) {
  const size_t nbytes = full ? sizeof(MlpImage) : offsetof(MlpImage, W2T);
  const uint4* s = reinterpret_cast<const uint4*>(src);
  uint4* d = reinterpret_cast<uint4*>(dst);
  for (size_t i = threadIdx.x; i < nbytes / 16; i += blockDim.x) d[i] = s[i];
  if (!full) {  // the biases follow the transposed blocks
    const float* sb = src->b1;
    float* db = dst->b1;
    for (int i = threadIdx.x; i < 2 * kMlpH + 8; i += blockDim.x) db[i] = sb[i];
  }
}

// A fragment of rows r0..r0+15, k0..k0+15 from a transposed [m][k] array (pitch kTP)
__device__ __forceinline__ void frag_a_T(const __nv_bfloat16* AT, int m0, int k0, unsigned a[4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  a[0] = ld_pair(AT + (m0 + g) * kTP + k0 + 2 * t);
  a[1] = ld_pair(AT + (m0 + g + 8) * kTP + k0 + 2 * t);
  a[2] = ld_pair(AT + (m0 + g) * kTP + k0 + 2 * t + 8);
  a[3] = ld_pair(AT + (m0 + g + 8) * kTP + k0 + 2 * t + 8);
}

// sum over the 8 lanes that share t (lanes g = 0..7): result valid in lanes with g == 0
__device__ __forceinline__ float sum_over_g(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 8);
  v += __shfl_xor_sync(0xffffffffu, v, 16);
  return v;
}

__global__ void __launch_bounds__(kThreads) k_mlp_train(const MlpImage* __restrict__ img,
                                                        const float* __restrict__ X,
                                                        const float* __restrict__ T, int n,
                                                        float inv_count, float* partial,
                                                        float* loss_part) {
  extern __shared__ __align__(16) unsigned char smraw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(smraw);
  copy_image(&S.W, img, true);
  // zero the padded rows of XT (inputs 5..15) and DYT (outputs 3..15)
  for (int i = threadIdx.x; i < 16 * kTP; i += kThreads) {
    S.XT[i] = __float2bfloat16(0.f);
    S.DYT[i] = __float2bfloat16(0.f);
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int rl0 = w * 16;                       // first row of the warp inside the CTA
  const int rg0 = blockIdx.x * kRows + rl0;     // first global row
  const int ra = rg0 + g, rb = rg0 + g + 8;
  const bool va = ra < n, vb = rb < n;
  // input fragment (features 5..7 and 8..15 are zero)
  float xa0 = 0.f, xa1 = 0.f, xb0 = 0.f, xb1 = 0.f;
  if (2 * t < kMlpIn) {
    if (va) xa0 = X[(size_t)ra * kMlpIn + 2 * t];
    if (vb) xb0 = X[(size_t)rb * kMlpIn + 2 * t];
  }
  if (2 * t + 1 < kMlpIn) {
    if (va) xa1 = X[(size_t)ra * kMlpIn + 2 * t + 1];
    if (vb) xb1 = X[(size_t)rb * kMlpIn + 2 * t + 1];
  }
  const unsigned xa[4] = {pack_bf16(xa0, xa1), pack_bf16(xb0, xb1), 0u, 0u};
  S.XT[(2 * t) * kTP + rl0 + g] = __float2bfloat16(xa0);
  S.XT[(2 * t + 1) * kTP + rl0 + g] = __float2bfloat16(xa1);
  S.XT[(2 * t) * kTP + rl0 + g + 8] = __float2bfloat16(xb0);
  S.XT[(2 * t + 1) * kTP + rl0 + g + 8] = __float2bfloat16(xb1);

  float z1[8][4], z2[8][4], y[4];
  mlp_forward16<true>(S.W, xa, z1, z2, y);

  // dL/dy = 2 (y - target) / (rows * 3) on the three used outputs
  float dy[4] = {0.f, 0.f, 0.f, 0.f}, sq = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int col = 2 * t + (q & 1);
    const bool v = (q < 2 ? va : vb) && col < kMlpOut;
    if (v) {
      const float tg = T[(size_t)(q < 2 ? ra : rb) * kMlpOut + col];
      const float d = y[q] - tg;
      dy[q] = 2.f * d * inv_count;
      sq += d * d;
    }
  }
  // loss and db3 partials
  sq += __shfl_xor_sync(0xffffffffu, sq, 1);
  sq += __shfl_xor_sync(0xffffffffu, sq, 2);
  sq = sum_over_g(sq);
  if (lane == 0) S.loss[w] = sq;
  {
    const float s0 = sum_over_g(dy[0] + dy[2]), s1 = sum_over_g(dy[1] + dy[3]);
    if (g == 0) { S.db3[w][2 * t] = s0; S.db3[w][2 * t + 1] = s1; }
  }
  // transposed copies: dy, h1, h2
  S.DYT[(2 * t) * kTP + rl0 + g] = __float2bfloat16(dy[0]);
  S.DYT[(2 * t + 1) * kTP + rl0 + g] = __float2bfloat16(dy[1]);
  S.DYT[(2 * t) * kTP + rl0 + g + 8] = __float2bfloat16(dy[2]);
  S.DYT[(2 * t + 1) * kTP + rl0 + g + 8] = __float2bfloat16(dy[3]);
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int c = nt * 8 + 2 * t;
    S.H1T[c * kTP + rl0 + g] = __float2bfloat16(silu(z1[nt][0]));
    S.H1T[(c + 1) * kTP + rl0 + g] = __float2bfloat16(silu(z1[nt][1]));
    S.H1T[c * kTP + rl0 + g + 8] = __float2bfloat16(silu(z1[nt][2]));
    S.H1T[(c + 1) * kTP + rl0 + g + 8] = __float2bfloat16(silu(z1[nt][3]));
    S.H2T[c * kTP + rl0 + g] = __float2bfloat16(silu(z2[nt][0]));
    S.H2T[(c + 1) * kTP + rl0 + g] = __float2bfloat16(silu(z2[nt][1]));
    S.H2T[c * kTP + rl0 + g + 8] = __float2bfloat16(silu(z2[nt][2]));
    S.H2T[(c + 1) * kTP + rl0 + g + 8] = __float2bfloat16(silu(z2[nt][3]));
  }
  // dh2 = dy W3 (K = outputs, padded to 16), dz2 = dh2 * silu'(z2)
  const unsigned dya[4] = {pack_bf16(dy[0], dy[1]), pack_bf16(dy[2], dy[3]), 0u, 0u};
  unsigned da[4][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    mma_bf16(c, dya, ld_pair(S.W.W3T + (nt * 8 + g) * kP3T + 2 * t), 0u);
#pragma unroll
    for (int q = 0; q < 4; ++q) c[q] *= dsilu(z2[nt][q]);
    const int col = nt * 8 + 2 * t;
    S.D2T[col * kTP + rl0 + g] = __float2bfloat16(c[0]);
    S.D2T[(col + 1) * kTP + rl0 + g] = __float2bfloat16(c[1]);
    S.D2T[col * kTP + rl0 + g + 8] = __float2bfloat16(c[2]);
    S.D2T[(col + 1) * kTP + rl0 + g + 8] = __float2bfloat16(c[3]);
    const float s0 = sum_over_g(c[0] + c[2]), s1 = sum_over_g(c[1] + c[3]);
    if (g == 0) { S.db2[w][col] = s0; S.db2[w][col + 1] = s1; }
    const int ks = nt >> 1;
    if ((nt & 1) == 0) { da[ks][0] = pack_bf16(c[0], c[1]); da[ks][1] = pack_bf16(c[2], c[3]); }
    else { da[ks][2] = pack_bf16(c[0], c[1]); da[ks][3] = pack_bf16(c[2], c[3]); }
  }
  // dh1 = dz2 W2, dz1 = dh1 * silu'(z1)
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    const __nv_bfloat16* wt = S.W.W2T + (nt * 8 + g) * kP2 + 2 * t;
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) mma_bf16(c, da[ks], ld_pair(wt + ks * 16), ld_pair(wt + ks * 16 + 8));
#pragma unroll
    for (int q = 0; q < 4; ++q) c[q] *= dsilu(z1[nt][q]);
    const int col = nt * 8 + 2 * t;
    S.D1T[col * kTP + rl0 + g] = __float2bfloat16(c[0]);
    S.D1T[(col + 1) * kTP + rl0 + g] = __float2bfloat16(c[1]);
    S.D1T[col * kTP + rl0 + g + 8] = __float2bfloat16(c[2]);
    S.D1T[(col + 1) * kTP + rl0 + g + 8] = __float2bfloat16(c[3]);
    const float s0 = sum_over_g(c[0] + c[2]), s1 = sum_over_g(c[1] + c[3]);
    if (g == 0) { S.db1[w][col] = s0; S.db1[w][col + 1] = s1; }
  }
  __syncthreads();

  float* P = partial + (size_t)blockIdx.x * kMlpParams;
  // dW2 = dZ2^T H1 over the CTA's rows: warp w owns out-tile w/2 and in-tiles 4(w%2)..+3
  {
    const int m0 = (w >> 1) * 16;
    float c[4][4] = {};
    for (int ks = 0; ks < kRows / 16; ++ks) {
      unsigned a[4];
      frag_a_T(S.D2T, m0, ks * 16, a);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int n0 = ((w & 1) * 4 + j) * 8;
        const __nv_bfloat16* b = S.H1T + (n0 + g) * kTP + ks * 16 + 2 * t;
        mma_bf16(c[j], a, ld_pair(b), ld_pair(b + 8));
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n0 = ((w & 1) * 4 + j) * 8 + 2 * t;
      P[kOffW2 + (m0 + g) * kMlpH + n0] = c[j][0];
      P[kOffW2 + (m0 + g) * kMlpH + n0 + 1] = c[j][1];
      P[kOffW2 + (m0 + g + 8) * kMlpH + n0] = c[j][2];
      P[kOffW2 + (m0 + g + 8) * kMlpH + n0 + 1] = c[j][3];
    }
  }
  // dW1 = dZ1^T X: warp w owns out-tile w/2 and in-tile w%2 (inputs 0..4 kept)
  {
    const int m0 = (w >> 1) * 16, n0 = (w & 1) * 8;
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    for (int ks = 0; ks < kRows / 16; ++ks) {
      unsigned a[4];
      frag_a_T(S.D1T, m0, ks * 16, a);
      const __nv_bfloat16* b = S.XT + (n0 + g) * kTP + ks * 16 + 2 * t;
      mma_bf16(c, a, ld_pair(b), ld_pair(b + 8));
    }
    const int i0 = n0 + 2 * t;
    if (i0 < kMlpIn) {
      P[kOffW1 + (m0 + g) * kMlpIn + i0] = c[0];
      P[kOffW1 + (m0 + g + 8) * kMlpIn + i0] = c[2];
    }
    if (i0 + 1 < kMlpIn) {
      P[kOffW1 + (m0 + g) * kMlpIn + i0 + 1] = c[1];
      P[kOffW1 + (m0 + g + 8) * kMlpIn + i0 + 1] = c[3];
    }
  }
  // dW3 = dY^T H2: warp w owns in-tile w (outputs 0..2 kept)
  {
    const int n0 = w * 8;
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    for (int ks = 0; ks < kRows / 16; ++ks) {
      unsigned a[4];
      frag_a_T(S.DYT, 0, ks * 16, a);
      const __nv_bfloat16* b = S.H2T + (n0 + g) * kTP + ks * 16 + 2 * t;
      mma_bf16(c, a, ld_pair(b), ld_pair(b + 8));
    }
    if (g < kMlpOut) {
      P[kOffW3 + g * kMlpH + n0 + 2 * t] = c[0];
      P[kOffW3 + g * kMlpH + n0 + 2 * t + 1] = c[1];
    }
  }
  // biases (fixed order over warps) and the loss
  for (int i = threadIdx.x; i < kMlpH; i += kThreads) {
    float s1 = 0.f, s2 = 0.f;
    for (int ww = 0; ww < 8; ++ww) { s1 += S.db1[ww][i]; s2 += S.db2[ww][i]; }
    P[kOffB1 + i] = s1;
    P[kOffB2 + i] = s2;
  }
  if (threadIdx.x < kMlpOut) {
    float s = 0.f;
    for (int ww = 0; ww < 8; ++ww) s += S.db3[ww][threadIdx.x];
    P[kOffB3 + threadIdx.x] = s;
  }
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int ww = 0; ww < 8; ++ww) s += S.loss[ww];
    loss_part[blockIdx.x] = s;
  }
}

// Places parameter p (value v) into the BF16 image (and its transposed copy).
__device__ __forceinline__ void image_put(MlpImage* img, int p, float v) {
  const __nv_bfloat16 b = __float2bfloat16(v);
  if (p < kOffB1) {
    const int o = p / kMlpIn, i = p % kMlpIn;
    img->W1[o * kP1 + i] = b;
  } else if (p < kOffW2) {
    img->b1[p - kOffB1] = v;
  } else if (p < kOffB2) {
    const int q = p - kOffW2, o = q / kMlpH, i = q % kMlpH;
    img->W2[o * kP2 + i] = b;
    img->W2T[i * kP2 + o] = b;
  } else if (p < kOffW3) {
    img->b2[p - kOffB2] = v;
  } else if (p < kOffB3) {
    const int q = p - kOffW3, o = q / kMlpH, i = q % kMlpH;
    img->W3[o * kP2 + i] = b;
    img->W3T[i * kP3T + o] = b;
  } else {
    img->b3[p - kOffB3] = v;
  }
}

// Sums the per-CTA partial gradients (fixed order, FP64); with adam set, updates the master
// weights and moments and refreshes the image; otherwise writes the gradient to `grad`.
__global__ void k_mlp_adam(const float* __restrict__ partial, int nblk, float* theta, float* m,
                           float* v, float lr, float b1, float b2, float eps, float bc1, float bc2,
                           MlpImage* img, float* grad, int adam) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kMlpParams) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += (double)partial[(size_t)b * kMlpParams + p];
  const float gr = (float)s;
  if (!adam) {
    grad[p] = gr;
    return;
  }
  const float mm = b1 * m[p] + (1.f - b1) * gr;
  const float vv = b2 * v[p] + (1.f - b2) * gr * gr;
  m[p] = mm;
  v[p] = vv;
  const float th = theta[p] - lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
  theta[p] = th;
  image_put(img, p, th);
}

__global__ void k_mlp_loss(const float* loss_part, int nblk, float inv_count, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += loss_part[b];
    *out = s * inv_count;
  }
}

__global__ void k_mlp_image(const float* theta, MlpImage* img) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kMlpParams) image_put(img, p, theta[p]);
}

// Deterministic initialisation: uniform in +-sqrt(6/fan_in) for weights (counter hash of the
// seed and index, splitmix64), zero biases.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void k_mlp_init(float* theta, unsigned long long seed) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kMlpParams) return;
  float fan = 0.f;
  if (p < kOffB1) fan = kMlpIn;
  else if (p >= kOffW2 && p < kOffB2) fan = kMlpH;
  else if (p >= kOffW3 && p < kOffB3) fan = kMlpH;
  if (fan == 0.f) { theta[p] = 0.f; return; }
  const double u = (splitmix64(seed * 0x100000001B3ull + (unsigned long long)p) >> 11) *
                   (1.0 / 9007199254740992.0);
  theta[p] = (float)((2.0 * u - 1.0) * sqrt(6.0 / fan));
}

__global__ void __launch_bounds__(kThreads) k_mlp_forward(const MlpImage* __restrict__ img,
                                                          const float* __restrict__ X, long long n,
                                                          float* __restrict__ Y) {
  __shared__ __align__(16) MlpImage W;
  copy_image(&W, img, false);
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  for (long long r0 = ((long long)blockIdx.x * 8 + w) * 16; r0 < n; r0 += (long long)gridDim.x * 128) {
    const long long ra = r0 + g, rb = r0 + g + 8;
    float x[4] = {0.f, 0.f, 0.f, 0.f};
    if (2 * t < kMlpIn) {
      if (ra < n) x[0] = X[ra * kMlpIn + 2 * t];
      if (rb < n) x[2] = X[rb * kMlpIn + 2 * t];
    }
    if (2 * t + 1 < kMlpIn) {
      if (ra < n) x[1] = X[ra * kMlpIn + 2 * t + 1];
      if (rb < n) x[3] = X[rb * kMlpIn + 2 * t + 1];
    }
    const unsigned xa[4] = {pack_bf16(x[0], x[1]), pack_bf16(x[2], x[3]), 0u, 0u};
    float z1[8][4], z2[8][4], y[4];
    mlp_forward16<false>(W, xa, z1, z2, y);
    for (int q = 0; q < 4; ++q) {
      const int col = 2 * t + (q & 1);
      const long long r = q < 2 ? ra : rb;
      if (col < kMlpOut && r < n) Y[r * kMlpOut + col] = y[q];
    }
  }
}

// raw features and target changes of one pair record
__device__ __forceinline__ void rec_feats(const float* rec, float dt, float f[kMlpIn], float tg[kMlpOut]) {
  const float nH = rec[0], N = rec[1], y = rec[2], T = rec[3], N1 = rec[4], y1 = rec[5], T1 = rec[6];
  f[0] = log10f(nH);
  f[1] = log10f(fmaxf(y, 1e-10f));
  f[2] = log10f(T);
  f[3] = log10f(fmaxf(N, 1e-30f));
  f[4] = log10f(dt);
  tg[0] = fminf(fmaxf(log10f(fmaxf(y1, 1e-10f)) - f[1], -kDlyMax), kDlyMax);
  tg[1] = fminf(fmaxf(log10f(T1) - f[2], -kDlTMax), kDlTMax);
  tg[2] = fminf(fmaxf(log10f(fmaxf(N1, 1e-30f)) - f[3], -kDlNMax), 0.f);
}

// sums for the standardisation: per feature/target sum, sum of squares; per feature min, max
__global__ void k_mlp_stats(const float* rec, long long n, float dt, double* acc) {
  __shared__ double s[16][kThreads];
  double a[16];
  for (int i = 0; i < 16; ++i) a[i] = 0.0;
  for (long long r = blockIdx.x * (long long)kThreads + threadIdx.x; r < n; r += (long long)gridDim.x * kThreads) {
    float f[kMlpIn], tg[kMlpOut];
    rec_feats(rec + r * kRecLen, dt, f, tg);
    for (int i = 0; i < kMlpIn; ++i) { a[i] += f[i]; a[kMlpIn + i] += (double)f[i] * f[i]; }
    for (int i = 0; i < kMlpOut; ++i) { a[10 + i] += tg[i]; a[13 + i] += (double)tg[i] * tg[i]; }
  }
  for (int i = 0; i < 16; ++i) s[i][threadIdx.x] = a[i];
  __syncthreads();
  if (threadIdx.x < 16) {
    double t = 0.0;
    for (int j = 0; j < kThreads; ++j) t += s[threadIdx.x][j];
    acc[blockIdx.x * 16 + threadIdx.x] = t;
  }
}

__global__ void k_mlp_minmax(const float* rec, long long n, float dt, float* mm) {
  __shared__ float lo[kMlpIn][kThreads], hi[kMlpIn][kThreads];
  float l[kMlpIn], h[kMlpIn];
  for (int i = 0; i < kMlpIn; ++i) { l[i] = 3e38f; h[i] = -3e38f; }
  for (long long r = threadIdx.x; r < n; r += kThreads) {
    float f[kMlpIn], tg[kMlpOut];
    rec_feats(rec + r * kRecLen, dt, f, tg);
    for (int i = 0; i < kMlpIn; ++i) { l[i] = fminf(l[i], f[i]); h[i] = fmaxf(h[i], f[i]); }
  }
  for (int i = 0; i < kMlpIn; ++i) { lo[i][threadIdx.x] = l[i]; hi[i][threadIdx.x] = h[i]; }
  __syncthreads();
  if (threadIdx.x < kMlpIn) {
    float a = 3e38f, b = -3e38f;
    for (int j = 0; j < kThreads; ++j) { a = fminf(a, lo[threadIdx.x][j]); b = fmaxf(b, hi[threadIdx.x][j]); }
    mm[threadIdx.x] = a;
    mm[kMlpIn + threadIdx.x] = b;
  }
}

__global__ void k_mlp_norm_final(const double* acc, int nblk, long long n, const float* mm,
                                 MlpNorm* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s[16];
  for (int i = 0; i < 16; ++i) {
    s[i] = 0.0;
    for (int b = 0; b < nblk; ++b) s[i] += acc[b * 16 + i];
  }
  for (int i = 0; i < kMlpIn; ++i) {
    const double mu = s[i] / n, var = s[kMlpIn + i] / n - mu * mu;
    out->in_mean[i] = (float)mu;
    out->in_scale[i] = (float)(var > 1e-12 ? 1.0 / sqrt(var) : 1.0);
    out->in_min[i] = mm[i];
    out->in_max[i] = mm[kMlpIn + i];
  }
  for (int i = 0; i < kMlpOut; ++i) {
    const double mu = s[10 + i] / n, var = s[13 + i] / n - mu * mu;
    out->out_mean[i] = (float)mu;
    out->out_scale[i] = (float)(var > 1e-12 ? 1.0 / sqrt(var) : 1.0);
  }
}

__global__ void k_mlp_features(const float* rec, long long n, float dt, const MlpNorm* nm,
                               float* X, float* T) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
    float f[kMlpIn], tg[kMlpOut];
    rec_feats(rec + r * kRecLen, dt, f, tg);
    for (int i = 0; i < kMlpIn; ++i) X[r * kMlpIn + i] = (f[i] - nm->in_mean[i]) * nm->in_scale[i];
    if (T)
      for (int i = 0; i < kMlpOut; ++i) T[r * kMlpOut + i] = (tg[i] - nm->out_mean[i]) * nm->out_scale[i];
  }
}

}  // namespace

size_t mlp_train_smem() { return sizeof(TrainSmem); }

}  // namespace aton

// ===========================================================================================
// C ABI of the surrogate network
// ===========================================================================================
using namespace aton;

struct aton_mlp {
  float* theta = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  MlpImage* img = nullptr;
  MlpNorm* norm = nullptr;
  float* partial = nullptr;
  float* loss_part = nullptr;
  double* d_loss = nullptr;
  double* d_acc = nullptr;
  float* d_mm = nullptr;
  int cap_blocks = 0;
  long long step = 0;
  cudaStream_t stream = nullptr;
};

static int mfail(int code, const char* msg, cudaError_t e = cudaSuccess) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s%s%s", msg, e != cudaSuccess ? ": " : "",
           e != cudaSuccess ? cudaGetErrorString(e) : "");
  set_last_message(buf);
  return code;
}
#define MCU(call)                                                        \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) return mfail(ATON_ERR_CUDA, #call, e_);       \
  } while (0)

static int ensure_blocks(aton_mlp* h, int nblk) {
  if (nblk <= h->cap_blocks) return ATON_OK;
  cudaFree(h->partial);
  cudaFree(h->loss_part);
  h->partial = nullptr;
  h->loss_part = nullptr;
  MCU(cudaMalloc(&h->partial, sizeof(float) * (size_t)nblk * kMlpParams));
  MCU(cudaMalloc(&h->loss_part, sizeof(float) * nblk));
  h->cap_blocks = nblk;
  return ATON_OK;
}

extern "C" {

int aton_mlp_create(aton_mlp_handle* out, unsigned long long seed) {
  if (!out) return mfail(ATON_ERR_BADARG, "out is NULL");
  *out = nullptr;
  aton_mlp* h = new aton_mlp();
  auto bail = [&](int rc) { aton_mlp_destroy(h); return rc; };
  if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess)
    return bail(mfail(ATON_ERR_CUDA, "stream"));
  if (cudaMalloc(&h->theta, sizeof(float) * kMlpParams) != cudaSuccess ||
      cudaMalloc(&h->m, sizeof(float) * kMlpParams) != cudaSuccess ||
      cudaMalloc(&h->v, sizeof(float) * kMlpParams) != cudaSuccess ||
      cudaMalloc(&h->img, sizeof(MlpImage)) != cudaSuccess ||
      cudaMalloc(&h->norm, sizeof(MlpNorm)) != cudaSuccess ||
      cudaMalloc(&h->d_loss, sizeof(double)) != cudaSuccess ||
      cudaMalloc(&h->d_acc, sizeof(double) * 16 * 148) != cudaSuccess ||
      cudaMalloc(&h->d_mm, sizeof(float) * 2 * kMlpIn) != cudaSuccess)
    return bail(mfail(ATON_ERR_NOMEM, "cudaMalloc"));
  if (cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(TrainSmem)) != cudaSuccess)
    return bail(mfail(ATON_ERR_CUDA, "train kernel attribute"));
  cudaStream_t s = h->stream;
  cudaMemsetAsync(h->m, 0, sizeof(float) * kMlpParams, s);
  cudaMemsetAsync(h->v, 0, sizeof(float) * kMlpParams, s);
  cudaMemsetAsync(h->img, 0, sizeof(MlpImage), s);   // padding stays zero
  MlpNorm id{};
  for (int i = 0; i < kMlpIn; ++i) { id.in_scale[i] = 1.f; id.in_min[i] = -3e38f; id.in_max[i] = 3e38f; }
  for (int i = 0; i < kMlpOut; ++i) id.out_scale[i] = 1.f;
  cudaMemcpyAsync(h->norm, &id, sizeof(id), cudaMemcpyHostToDevice, s);
  k_mlp_init<<<(kMlpParams + 255) / 256, 256, 0, s>>>(h->theta, seed);
  k_mlp_image<<<(kMlpParams + 255) / 256, 256, 0, s>>>(h->theta, h->img);
  if (cudaStreamSynchronize(s) != cudaSuccess) return bail(mfail(ATON_ERR_CUDA, "init"));
  *out = h;
  return ATON_OK;
}

void aton_mlp_destroy(aton_mlp_handle h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  cudaFree(h->theta); cudaFree(h->m); cudaFree(h->v); cudaFree(h->img); cudaFree(h->norm);
  cudaFree(h->partial); cudaFree(h->loss_part); cudaFree(h->d_loss); cudaFree(h->d_acc);
  cudaFree(h->d_mm);
  if (h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

int aton_mlp_num_params(void) { return kMlpParams; }

int aton_mlp_set_params(aton_mlp_handle h, const float* theta, int where) {
  if (!h || !theta) return mfail(ATON_ERR_BADARG, "NULL argument");
  MCU(cudaMemcpyAsync(h->theta, theta, sizeof(float) * kMlpParams,
                      where == ATON_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, h->stream));
  MCU(cudaMemsetAsync(h->m, 0, sizeof(float) * kMlpParams, h->stream));
  MCU(cudaMemsetAsync(h->v, 0, sizeof(float) * kMlpParams, h->stream));
  h->step = 0;
  k_mlp_image<<<(kMlpParams + 255) / 256, 256, 0, h->stream>>>(h->theta, h->img);
  MCU(cudaGetLastError());
  MCU(cudaStreamSynchronize(h->stream));
  return ATON_OK;
}

int aton_mlp_get_params(aton_mlp_handle h, float* theta, int where) {
  if (!h || !theta) return mfail(ATON_ERR_BADARG, "NULL argument");
  MCU(cudaMemcpyAsync(theta, h->theta, sizeof(float) * kMlpParams,
                      where == ATON_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->stream));
  MCU(cudaStreamSynchronize(h->stream));
  return ATON_OK;
}

int aton_mlp_fit_norm(aton_mlp_handle h, const float* records, int64_t n, double dt) {
  if (!h || !records || n < 1 || !(dt > 0)) return mfail(ATON_ERR_BADARG, "bad argument");
  const int nblk = 148;
  k_mlp_stats<<<nblk, kThreads, 0, h->stream>>>(records, n, (float)dt, h->d_acc);
  k_mlp_minmax<<<1, kThreads, 0, h->stream>>>(records, n, (float)dt, h->d_mm);
  k_mlp_norm_final<<<1, 32, 0, h->stream>>>(h->d_acc, nblk, n, h->d_mm, h->norm);
  MCU(cudaGetLastError());
  MCU(cudaStreamSynchronize(h->stream));
  return ATON_OK;
}

int aton_mlp_get_norm(aton_mlp_handle h, float* out) {
  if (!h || !out) return mfail(ATON_ERR_BADARG, "NULL argument");
  MCU(cudaMemcpyAsync(out, h->norm, sizeof(MlpNorm), cudaMemcpyDeviceToHost, h->stream));
  MCU(cudaStreamSynchronize(h->stream));
  return ATON_OK;
}

int aton_mlp_set_norm(aton_mlp_handle h, const float* in) {
  if (!h || !in) return mfail(ATON_ERR_BADARG, "NULL argument");
  MCU(cudaMemcpyAsync(h->norm, in, sizeof(MlpNorm), cudaMemcpyHostToDevice, h->stream));
  MCU(cudaStreamSynchronize(h->stream));
  return ATON_OK;
}

int aton_mlp_features(aton_mlp_handle h, const float* records, int64_t n, double dt, float* X,
                      float* T) {
  if (!h || !records || !X || n < 0 || !(dt > 0)) return mfail(ATON_ERR_BADARG, "bad argument");
  if (n == 0) return ATON_OK;
  k_mlp_features<<<148 * 4, 256, 0, h->stream>>>(records, n, (float)dt, h->norm, X, T);
  MCU(cudaGetLastError());
  MCU(cudaStreamSynchronize(h->stream));
  return ATON_OK;
}

int aton_mlp_forward(aton_mlp_handle h, const float* X, int64_t n, float* Y) {
  if (!h || !X || !Y || n < 0) return mfail(ATON_ERR_BADARG, "bad argument");
  if (n == 0) return ATON_OK;
  const long long blocks = std::min<long long>((n + kRows - 1) / kRows, 148 * 8);
  k_mlp_forward<<<(int)blocks, kThreads, 0, h->stream>>>(h->img, X, n, Y);
  MCU(cudaGetLastError());
  MCU(cudaStreamSynchronize(h->stream));
  return ATON_OK;
}

static int train_common(aton_mlp* h, const float* X, const float* T, int n, int adam, float lr,
                        float* grad, double* loss) {
  if (!X || !T || n < 1) return mfail(ATON_ERR_BADARG, "bad argument");
  const int nblk = (n + kRows - 1) / kRows;
  if (int rc = ensure_blocks(h, nblk)) return rc;
  const float inv = 1.f / (float)((double)n * kMlpOut);
  k_mlp_train<<<nblk, kThreads, sizeof(TrainSmem), h->stream>>>(h->img, X, T, n, inv, h->partial,
                                                               h->loss_part);
  MCU(cudaGetLastError());
  float bc1 = 1.f, bc2 = 1.f;
  if (adam) {
    h->step += 1;
    bc1 = (float)(1.0 - pow(0.9, (double)h->step));
    bc2 = (float)(1.0 - pow(0.999, (double)h->step));
  }
  k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, h->stream>>>(h->partial, nblk, h->theta, h->m,
                                                              h->v, lr, 0.9f, 0.999f, 1e-8f, bc1,
                                                              bc2, h->img, grad, adam);
  k_mlp_loss<<<1, 32, 0, h->stream>>>(h->loss_part, nblk, 1.0 / ((double)n * kMlpOut), h->d_loss);
  MCU(cudaGetLastError());
  if (loss) {
    MCU(cudaMemcpyAsync(loss, h->d_loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    MCU(cudaStreamSynchronize(h->stream));
  }
  return ATON_OK;
}

int aton_mlp_loss_grad(aton_mlp_handle h, const float* X, const float* T, int n, float* grad,
                       double* loss) {
  if (!h || !grad) return mfail(ATON_ERR_BADARG, "NULL argument");
  int rc = train_common(h, X, T, n, 0, 0.f, grad, loss);
  if (rc) return rc;
  MCU(cudaStreamSynchronize(h->stream));
  return ATON_OK;
}

int aton_mlp_train_step(aton_mlp_handle h, const float* X, const float* T, int n, float lr,
                        double* loss) {
  if (!h || !(lr > 0)) return mfail(ATON_ERR_BADARG, "bad argument");
  return train_common(h, X, T, n, 1, lr, nullptr, loss);
}

int aton_mlp_synchronize(aton_mlp_handle h) {
  if (!h) return mfail(ATON_ERR_BADARG, "NULL handle");
  MCU(cudaStreamSynchronize(h->stream));
  return ATON_OK;
}

}  // extern "C"

namespace aton {
const MlpImage* mlp_image(const aton_mlp* h) { return h->img; }
const MlpNorm* mlp_norm(const aton_mlp* h) { return h->norm; }
}  // namespace aton
