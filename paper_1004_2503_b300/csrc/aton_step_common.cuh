// aton_step_common.cuh -- device helpers shared by the fused step kernels and the plain
// step: boundary index map, per-thread tallies and their FP64 block reduction, and the
// realisability clamp.
#pragma once
#include "aton_internal.h"

namespace aton {

__device__ __forceinline__ int bc_map(int v, int n, bool periodic) {
  if (periodic) {
    v %= n;
    return v < 0 ? v + n : v;
  }
  return v < 0 ? 0 : (v >= n ? n - 1 : v);
}

// Per-thread tallies of one step.
struct Tally {
  KahanF absorbed, escaped;
  float clipped = 0.f;
  unsigned int sub = 0, mx = 0, err = 0, nan = 0, sur = 0;
};

// Block reduction of the tallies (FP64 for the photon sums) into slot `slot`.
template <int NWARP>
__device__ __forceinline__ void flush_tally(const Tally& t, const Slots& S, int slot) {
  __shared__ double s_acc[NWARP][3];
  __shared__ unsigned long long s_sub[NWARP];
  __shared__ unsigned int s_u[NWARP][4];
  double a0 = t.absorbed.value(), a1 = t.escaped.value(), a2 = (double)t.clipped;
  unsigned long long sb = t.sub;
  unsigned int mx = t.mx, er = t.err, na = t.nan, su = t.sur;
  const unsigned full = 0xffffffffu;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_down_sync(full, a0, o);
    a1 += __shfl_down_sync(full, a1, o);
    a2 += __shfl_down_sync(full, a2, o);
    sb += __shfl_down_sync(full, sb, o);
    mx = max(mx, __shfl_down_sync(full, mx, o));
    er += __shfl_down_sync(full, er, o);
    na += __shfl_down_sync(full, na, o);
    su += __shfl_down_sync(full, su, o);
  }
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int w = tid >> 5, lane = tid & 31;
  if (lane == 0) {
    s_acc[w][0] = a0; s_acc[w][1] = a1; s_acc[w][2] = a2;
    s_sub[w] = sb; s_u[w][0] = mx; s_u[w][1] = er; s_u[w][2] = na; s_u[w][3] = su;
  }
  __syncthreads();
  if (tid == 0) {
    double b0 = 0, b1 = 0, b2 = 0;
    unsigned long long bs = 0;
    unsigned int bm = 0, be = 0, bn = 0, bu = 0;
    for (int i = 0; i < NWARP; ++i) {
      b0 += s_acc[i][0]; b1 += s_acc[i][1]; b2 += s_acc[i][2];
      bs += s_sub[i]; bm = max(bm, s_u[i][0]); be += s_u[i][1]; bn += s_u[i][2]; bu += s_u[i][3];
    }
    S.acc[3 * slot + 0] += b0;
    S.acc[3 * slot + 1] += b1;
    S.acc[3 * slot + 2] += b2;
    S.sub[slot] += bs;
    S.mx[slot] = max(S.mx[slot], bm);
    S.err[slot] += be;
    S.nan[slot] += bn;
    S.sur[slot] += bu;
  }
}

// Realisability after transport: N >= 0 (the removed amount is tallied), |Fh| <= N.
__device__ __forceinline__ void clamp_state(float& N, float& X, float& Y, float& Z, float& clipped) {
  if (N < 0.f) {
    clipped += N;
    N = 0.f; X = 0.f; Y = 0.f; Z = 0.f;
  } else {
    const float F2 = X * X + Y * Y + Z * Z;
    if (F2 > N * N) {   // IEEE sqrt and division: F2 may be denormal, N may be 0
      const float s = N > 0.f ? N / sqrtf(F2) : 0.f;
      X *= s; Y *= s; Z *= s;
    }
  }
}

}  // namespace aton
