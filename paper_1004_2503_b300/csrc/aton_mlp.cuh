// aton_mlp.cuh -- the chemistry-surrogate MLP (5 -> 64 -> 64 -> 3, SiLU): its parameter layout
// and BF16 weight image, and the inference of a few scattered cells on BF16 tensor cores with
// FP32 accumulation (warp-level mma.sync m16n8k16: the surrogate kernels run the network for
// 32 listed cells at a time, far below a 128-row tcgen05 tile; training, on full 128-row tiles,
// uses tcgen05 in aton_mlp_tc.cu).
//
// One warp carries 16 rows through a layer as m16n8k16 products: the accumulator fragments of
// one layer (16 x 8 tiles, FP32) become, after the activation and a BF16 conversion, the A
// fragments of the next layer's product (two adjacent 16 x 8 tiles form one 16 x 16 A tile), so
// activations never leave registers. Weights sit in shared memory as a packed image (rows padded
// by 8 BF16 so the B-fragment loads of a warp fall in distinct banks).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace aton {

constexpr int kMlpIn = 5, kMlpH = 64, kMlpOut = 3;
constexpr int kMlpParams = kMlpH * kMlpIn + kMlpH + kMlpH * kMlpH + kMlpH + kMlpOut * kMlpH + kMlpOut;
// flat parameter offsets (W1 64x5, b1, W2 64x64, b2, W3 3x64, b3)
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kMlpH * kMlpIn, kOffW2 = kOffB1 + kMlpH;
constexpr int kOffB2 = kOffW2 + kMlpH * kMlpH, kOffW3 = kOffB2 + kMlpH;
constexpr int kOffB3 = kOffW3 + kMlpOut * kMlpH;

// Row pitches (BF16 elements) of the shared-memory weight image.
constexpr int kP1 = 16 + 8;   // W1 rows: 16 inputs (5 used) + pad
constexpr int kP2 = 64 + 8;   // W2, W3, W2T rows
constexpr int kP3T = 8 + 8;   // W3T rows: 8 outputs (3 used) + pad

struct MlpImage {
  __nv_bfloat16 W1[kMlpH * kP1];     // [out][in]
  __nv_bfloat16 W2[kMlpH * kP2];     // [out][in]
  __nv_bfloat16 W3[8 * kP2];         // [out (3 used)][in]
  __nv_bfloat16 W2T[kMlpH * kP2];    // [in][out]  (backward)
  __nv_bfloat16 W3T[kMlpH * kP3T];   // [in][out]  (backward)
  float b1[kMlpH], b2[kMlpH], b3[8];
};
// bytes of the image needed by the forward pass (W1, W2, W3 and the biases are copied; the
// transposed blocks only for training)
constexpr size_t kImgBytes = sizeof(MlpImage);

// Byte offset of element (r, c) of a [row][column] BF16 matrix of pitch P columns in the
// canonical no-swizzle layout of the tcgen05 operands: 8 x 8 core matrices of 128 bytes (8 rows
// of 16 bytes, a row's 8 consecutive columns), core matrices adjacent along the columns 128
// bytes apart, 8-row groups P x 16 bytes apart.
__host__ __device__ constexpr unsigned tc_cano(int r, int c, int P) {
  return (unsigned)((r >> 3) * (P * 16) + (c >> 3) * 128 + (r & 7) * 16 + (c & 7) * 2);
}

// The training kernel's weight operands, byte for byte as they sit in its shared memory (one
// bulk copy per CTA): each matrix [row][column] in the canonical layout, padding zero.
struct MlpTcImage {
  unsigned char W1[64 * 16 * 2];    // W1    [out][in]   64 x 16 (inputs 5..15 zero)
  unsigned char W2[64 * 64 * 2];    // W2    [out][in]   64 x 64
  unsigned char W3[16 * 64 * 2];    // W3    [out][in]   16 x 64 (outputs 3..15 zero)
  unsigned char W2T[64 * 64 * 2];   // W2^T  [in][out]   64 x 64
  unsigned char W3T[64 * 16 * 2];   // W3^T  [in][out]   64 x 16 (outputs 3..15 zero)
  float bias[144];                  // b1 [0, 64), b2 [64, 128), b3 [128, 131)
};
static_assert(sizeof(MlpTcImage) % 16 == 0, "bulk copies move multiples of 16 bytes");

// Ranges of the targets (changes of log10 y, log10 T, log10 N over one step), applied to the
// training targets and to the decoded predictions alike.
constexpr float kDlyMax = 6.f, kDlTMax = 3.f, kDlNMax = 6.f;

// Normalisation and training range of the surrogate.
struct MlpNorm {
  float in_mean[kMlpIn], in_scale[kMlpIn];      // feature -> (f - mean) * scale
  float out_mean[kMlpOut], out_scale[kMlpOut];  // target = mean + out / scale
  float in_min[kMlpIn], in_max[kMlpIn];         // raw feature range seen in training
};

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<unsigned*>(&v);
}

__device__ __forceinline__ unsigned ld_pair(const __nv_bfloat16* p) {
  return *reinterpret_cast<const unsigned*>(p);
}

// D = A(16x16, bf16) * B(16x8, bf16) + C, FP32 accumulate.
__device__ __forceinline__ void mma_bf16(float c[4], const unsigned a[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// SiLU z * sigmoid(z) with sigmoid(z) = (1 + tanh(z/2)) / 2 (one hardware tanh).
__device__ __forceinline__ float tanh_hw(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float silu(float z) {
  const float h = 0.5f * z;
  return h + h * tanh_hw(h);
}
// d silu / dz = s (1 + z (1 - s)), s = sigmoid(z)
__device__ __forceinline__ float dsilu(float z) {
  const float s = 0.5f + 0.5f * tanh_hw(0.5f * z);
  return s * (1.f + z * (1.f - s));
}

// Forward of 16 rows held by one warp. xa: the A fragment of the (padded) input tile, i.e. lane
// (g = lane/4, t = lane%4) holds x[g][2t..2t+1] in xa[0], x[g+8][2t..2t+1] in xa[1] (columns
// 8..15 are zero: xa[2] = xa[3] = 0). Outputs: z1, z2 (pre-activations, C layout, 8 tiles x 4)
// when keep is set (training), and y (C layout of the single 16 x 8 output tile).
template <bool KEEP>
__device__ __forceinline__ void mlp_forward16(const MlpImage& W, const unsigned xa[4], float z1[8][4],
                                              float z2[8][4], float y[4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float acc[8][4];
  // layer 1: 8 output tiles, one k step
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int col = nt * 8 + 2 * t;
    acc[nt][0] = W.b1[col]; acc[nt][1] = W.b1[col + 1];
    acc[nt][2] = W.b1[col]; acc[nt][3] = W.b1[col + 1];
    const __nv_bfloat16* w = W.W1 + (nt * 8 + g) * kP1 + 2 * t;
    mma_bf16(acc[nt], xa, ld_pair(w), 0u);
  }
  unsigned ha[4][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    if (KEEP) {
#pragma unroll
      for (int q = 0; q < 4; ++q) z1[nt][q] = acc[nt][q];
    }
    const float h0 = silu(acc[nt][0]), h1 = silu(acc[nt][1]), h2 = silu(acc[nt][2]),
                h3 = silu(acc[nt][3]);
    const int ks = nt >> 1;
    if ((nt & 1) == 0) { ha[ks][0] = pack_bf16(h0, h1); ha[ks][1] = pack_bf16(h2, h3); }
    else { ha[ks][2] = pack_bf16(h0, h1); ha[ks][3] = pack_bf16(h2, h3); }
  }
  // layer 2: 8 output tiles, four k steps
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int col = nt * 8 + 2 * t;
    acc[nt][0] = W.b2[col]; acc[nt][1] = W.b2[col + 1];
    acc[nt][2] = W.b2[col]; acc[nt][3] = W.b2[col + 1];
    const __nv_bfloat16* w = W.W2 + (nt * 8 + g) * kP2 + 2 * t;
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) mma_bf16(acc[nt], ha[ks], ld_pair(w + ks * 16), ld_pair(w + ks * 16 + 8));
  }
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    if (KEEP) {
#pragma unroll
      for (int q = 0; q < 4; ++q) z2[nt][q] = acc[nt][q];
    }
    const float h0 = silu(acc[nt][0]), h1 = silu(acc[nt][1]), h2 = silu(acc[nt][2]),
                h3 = silu(acc[nt][3]);
    const int ks = nt >> 1;
    if ((nt & 1) == 0) { ha[ks][0] = pack_bf16(h0, h1); ha[ks][1] = pack_bf16(h2, h3); }
    else { ha[ks][2] = pack_bf16(h0, h1); ha[ks][3] = pack_bf16(h2, h3); }
  }
  // layer 3: one output tile (3 of 8 columns used), four k steps
  y[0] = W.b3[2 * t]; y[1] = W.b3[2 * t + 1]; y[2] = y[0]; y[3] = y[1];
  const __nv_bfloat16* w = W.W3 + g * kP2 + 2 * t;
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) mma_bf16(y, ha[ks], ld_pair(w + ks * 16), ld_pair(w + ks * 16 + 8));
}

// Inference of 16 rows with few registers (bitwise the outputs of mlp_forward16: the same
// products in the same order): the activations of each layer go to a per-warp shared-memory
// tile H (16 rows x kP2 BF16, twice: layer 1 and layer 2) instead of registers, and the output
// tiles are not unrolled, so only one accumulator tile and one operand set are live. For the
// fused step kernel, whose register count the rarely used network must not raise. W may sit in
// shared memory (the fused kernel's tail copies it there) or in global memory (read through L1).
__device__ __forceinline__ void mlp_infer16_sh(const MlpImage& W, const unsigned xa[4],
                                               __nv_bfloat16* H1, __nv_bfloat16* H2, float y[4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  // C tile (rows g, g+8; columns col, col+1) after SiLU into H as BF16 pairs
  auto put = [&](__nv_bfloat16* H, int col, const float c[4]) {
    *reinterpret_cast<unsigned*>(H + g * kP2 + col) = pack_bf16(silu(c[0]), silu(c[1]));
    *reinterpret_cast<unsigned*>(H + (g + 8) * kP2 + col) = pack_bf16(silu(c[2]), silu(c[3]));
  };
  // A fragment of k step ks from H
  auto frag = [&](const __nv_bfloat16* H, int ks, unsigned a[4]) {
    const int c = ks * 16 + 2 * t;
    a[0] = ld_pair(H + g * kP2 + c);
    a[1] = ld_pair(H + (g + 8) * kP2 + c);
    a[2] = ld_pair(H + g * kP2 + c + 8);
    a[3] = ld_pair(H + (g + 8) * kP2 + c + 8);
  };
#pragma unroll 1
  for (int nt = 0; nt < 8; ++nt) {
    const int col = nt * 8 + 2 * t;
    float acc[4] = {W.b1[col], W.b1[col + 1], W.b1[col], W.b1[col + 1]};
    mma_bf16(acc, xa, ld_pair(W.W1 + (nt * 8 + g) * kP1 + 2 * t), 0u);
    put(H1, col, acc);
  }
  __syncwarp();
#pragma unroll 1
  for (int nt = 0; nt < 8; ++nt) {
    const int col = nt * 8 + 2 * t;
    float acc[4] = {W.b2[col], W.b2[col + 1], W.b2[col], W.b2[col + 1]};
    const __nv_bfloat16* w = W.W2 + (nt * 8 + g) * kP2 + 2 * t;
#pragma unroll 1
    for (int ks = 0; ks < 4; ++ks) {
      unsigned a[4];
      frag(H1, ks, a);
      mma_bf16(acc, a, ld_pair(w + ks * 16), ld_pair(w + ks * 16 + 8));
    }
    put(H2, col, acc);
  }
  __syncwarp();
  y[0] = W.b3[2 * t]; y[1] = W.b3[2 * t + 1]; y[2] = y[0]; y[3] = y[1];
  const __nv_bfloat16* w = W.W3 + g * kP2 + 2 * t;
#pragma unroll 1
  for (int ks = 0; ks < 4; ++ks) {
    unsigned a[4];
    frag(H2, ks, a);
    mma_bf16(y, a, ld_pair(w + ks * 16), ld_pair(w + ks * 16 + 8));
  }
  __syncwarp();   // (H may be reused by the warp's next call)
}

}  // namespace aton
