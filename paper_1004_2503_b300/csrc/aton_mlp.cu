// aton_mlp.cu -- training and inference kernels of the chemistry-surrogate MLP and its C ABI.
//
// The surrogate replaces the sub-cycled chemistry operator Phi (Appendix Eq. A4) for cells that
// would sub-cycle heavily. Features of a cell are (log10 nH, log10 y, log10 T, log10 N, log10 dt);
// targets are the changes (log10 y' - log10 y, log10 T' - log10 T, log10 N' - log10 N), both
// standardised with statistics of the training set. Training pairs come from the exact
// operator (the plain step's chemistry kernel writes them through a pair sink).
//
// Kernels:
//   k_mlp_train_tc -- (aton_mlp_tc.cu) forward and backward of 128 rows per CTA on the tcgen05
//                    tensor cores, accumulators in tensor memory; one FP32 partial gradient per
//                    CTA (summed later in a fixed order: deterministic).
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

constexpr int kRows = 128;          // rows per CTA (training: one per thread; inference: 8 x 16)
constexpr int kThreads = 256;
constexpr int kRecLen = 8;          // pair record: nH, N, y, T, N', y', T', sub-steps

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

// Places parameter p (value v) into the BF16 image (and its transposed copy) and into the
// training kernel's canonical image.
__device__ __forceinline__ void image_put(MlpImage* img, MlpTcImage* tc, int p, float v) {
  const __nv_bfloat16 b = __float2bfloat16(v);
  auto tcw = [&](unsigned char* m, int r, int c, int P) {
    *reinterpret_cast<__nv_bfloat16*>(m + tc_cano(r, c, P)) = b;
  };
  if (p < kOffB1) {
    const int o = p / kMlpIn, i = p % kMlpIn;
    img->W1[o * kP1 + i] = b;
    tcw(tc->W1, o, i, 16);
  } else if (p < kOffW2) {
    img->b1[p - kOffB1] = v;
    tc->bias[p - kOffB1] = v;
  } else if (p < kOffB2) {
    const int q = p - kOffW2, o = q / kMlpH, i = q % kMlpH;
    img->W2[o * kP2 + i] = b;
    img->W2T[i * kP2 + o] = b;
    tcw(tc->W2, o, i, 64);
    tcw(tc->W2T, i, o, 64);
  } else if (p < kOffW3) {
    img->b2[p - kOffB2] = v;
    tc->bias[64 + p - kOffB2] = v;
  } else if (p < kOffB3) {
    const int q = p - kOffW3, o = q / kMlpH, i = q % kMlpH;
    img->W3[o * kP2 + i] = b;
    img->W3T[i * kP3T + o] = b;
    tcw(tc->W3, o, i, 64);
    tcw(tc->W3T, i, o, 16);
  } else {
    img->b3[p - kOffB3] = v;
    tc->bias[128 + p - kOffB3] = v;
  }
}

// Sums the per-CTA partial gradients (fixed order, FP64); with adam set, updates the master
// weights and moments and refreshes the image; otherwise writes the gradient to `grad`.
__global__ void k_mlp_adam(const float* __restrict__ partial, int nblk, float* theta, float* m,
                           float* v, float lr, float b1, float b2, float eps, float bc1, float bc2,
                           MlpImage* img, MlpTcImage* tc, float* grad, int adam) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kMlpParams) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += (double)partial[(size_t)b * kMlpPartStride + p];
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
  image_put(img, tc, p, th);
}

__global__ void k_mlp_loss(const float* loss_part, int nblk, float inv_count, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += loss_part[b];
    *out = s * inv_count;
  }
}

__global__ void k_mlp_image(const float* theta, MlpImage* img, MlpTcImage* tc) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kMlpParams) image_put(img, tc, p, theta[p]);
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
  MlpTcImage* tcimg = nullptr;   // the training kernel's canonical copy of the weights
  MlpNorm* norm = nullptr;
  float* partial = nullptr;
  float* loss_part = nullptr;
  double* d_loss = nullptr;
  double* d_acc = nullptr;
  float* d_mm = nullptr;
  unsigned int* d_err = nullptr;   // tensor-core pipeline waits that gave up (must stay 0)
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
  MCU(cudaMalloc(&h->partial, sizeof(float) * (size_t)nblk * kMlpPartStride));
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
      cudaMalloc(&h->tcimg, sizeof(MlpTcImage)) != cudaSuccess ||
      cudaMalloc(&h->norm, sizeof(MlpNorm)) != cudaSuccess ||
      cudaMalloc(&h->d_loss, sizeof(double)) != cudaSuccess ||
      cudaMalloc(&h->d_acc, sizeof(double) * 16 * 148) != cudaSuccess ||
      cudaMalloc(&h->d_mm, sizeof(float) * 2 * kMlpIn) != cudaSuccess ||
      cudaMalloc(&h->d_err, sizeof(unsigned int)) != cudaSuccess)
    return bail(mfail(ATON_ERR_NOMEM, "cudaMalloc"));
  if (cudaFuncSetAttribute(k_mlp_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)mlp_train_tc_smem()) != cudaSuccess)
    return bail(mfail(ATON_ERR_CUDA, "train kernel attribute"));
  cudaStream_t s = h->stream;
  cudaMemsetAsync(h->d_err, 0, sizeof(unsigned int), s);
  cudaMemsetAsync(h->m, 0, sizeof(float) * kMlpParams, s);
  cudaMemsetAsync(h->v, 0, sizeof(float) * kMlpParams, s);
  cudaMemsetAsync(h->img, 0, sizeof(MlpImage), s);   // padding stays zero
  cudaMemsetAsync(h->tcimg, 0, sizeof(MlpTcImage), s);
  MlpNorm id{};
  for (int i = 0; i < kMlpIn; ++i) { id.in_scale[i] = 1.f; id.in_min[i] = -3e38f; id.in_max[i] = 3e38f; }
  for (int i = 0; i < kMlpOut; ++i) id.out_scale[i] = 1.f;
  cudaMemcpyAsync(h->norm, &id, sizeof(id), cudaMemcpyHostToDevice, s);
  k_mlp_init<<<(kMlpParams + 255) / 256, 256, 0, s>>>(h->theta, seed);
  k_mlp_image<<<(kMlpParams + 255) / 256, 256, 0, s>>>(h->theta, h->img, h->tcimg);
  if (cudaStreamSynchronize(s) != cudaSuccess) return bail(mfail(ATON_ERR_CUDA, "init"));
  *out = h;
  return ATON_OK;
}

void aton_mlp_destroy(aton_mlp_handle h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  cudaFree(h->theta); cudaFree(h->m); cudaFree(h->v); cudaFree(h->img); cudaFree(h->tcimg);
  cudaFree(h->norm);
  cudaFree(h->partial); cudaFree(h->loss_part); cudaFree(h->d_loss); cudaFree(h->d_acc);
  cudaFree(h->d_mm); cudaFree(h->d_err);
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
  k_mlp_image<<<(kMlpParams + 255) / 256, 256, 0, h->stream>>>(h->theta, h->img, h->tcimg);
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

// the training kernel's error word (a tensor-core pipeline wait that gave up); call after a sync
static int check_err(aton_mlp* h) {
  unsigned int e = 0;
  MCU(cudaMemcpy(&e, h->d_err, sizeof(e), cudaMemcpyDeviceToHost));
  if (e) return mfail(ATON_ERR_CUDA, "training kernel: a tensor-core wait gave up");
  return ATON_OK;
}

static int train_common(aton_mlp* h, const float* X, const float* T, int n, int adam, float lr,
                        float* grad, double* loss) {
  if (!X || !T || n < 1) return mfail(ATON_ERR_BADARG, "bad argument");
  const int nblk = (n + kRows - 1) / kRows;
  if (int rc = ensure_blocks(h, nblk)) return rc;
  const float inv = 1.f / (float)((double)n * kMlpOut);
  k_mlp_train_tc<<<nblk, kMlpTcThreads, mlp_train_tc_smem(), h->stream>>>(
      h->tcimg, X, T, n, inv, h->partial, h->loss_part, h->d_err);
  MCU(cudaGetLastError());
  float bc1 = 1.f, bc2 = 1.f;
  if (adam) {
    h->step += 1;
    bc1 = (float)(1.0 - pow(0.9, (double)h->step));
    bc2 = (float)(1.0 - pow(0.999, (double)h->step));
  }
  k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, h->stream>>>(h->partial, nblk, h->theta, h->m,
                                                              h->v, lr, 0.9f, 0.999f, 1e-8f, bc1,
                                                              bc2, h->img, h->tcimg, grad, adam);
  k_mlp_loss<<<1, 32, 0, h->stream>>>(h->loss_part, nblk, 1.0 / ((double)n * kMlpOut), h->d_loss);
  MCU(cudaGetLastError());
  if (loss) {
    MCU(cudaMemcpyAsync(loss, h->d_loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    MCU(cudaStreamSynchronize(h->stream));
    return check_err(h);
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
  return check_err(h);
}

}  // extern "C"

namespace aton {
const MlpImage* mlp_image(const aton_mlp* h) { return h->img; }
const MlpNorm* mlp_norm(const aton_mlp* h) { return h->norm; }
}  // namespace aton
