// aton_stats.cu -- statistics of the ionisation state and of the radiation field (section 4:
// volume- and mass-weighted ionised fraction, Gamma12 and J21 averages, the distributions
// (1-x)(nH) and J21(nH) with the mean per density bin).
//
// One pass over N, y, T, nH with a fixed grid, so every sum has a fixed order:
//  - histogram counts in shared-memory integer atomics, added to global 64-bit counters per CTA
//    (integer sums: exact in any order);
//  - the scalar sums in per-thread compensated FP32 accumulators (error-free TwoSum), reduced in
//    FP64 per CTA into a
//    per-CTA slot, then summed over the slots in index order;
//  - the per-density-bin sums of y and N: within each group of 32 consecutive cells (a warp),
//    runs of equal density bin are summed in FP32 by a segmented tree, and each run's sum is
//    added with an error-free TwoSum to the warp's own row of FP32 (sum, error) pairs (runs of
//    the same bin in lane order; FP64 arithmetic, a slow pipe on this part, stays out of the
//    loop), reduced in FP64 at the end.
// Bin decisions compare the stored floats with float edges prepared on the host (a log2 guess
// then an exact fix-up), so they are exact and reproducible.
#include "aton_internal.h"
#include "aton_stats.cuh"

namespace aton {

namespace {

constexpr int kMB = kStatsMaxBins;
constexpr int kWarps = kStatsThreads / 32;

// bin b with E[b] <= v < E[b+1]; below E[1] -> 0, at or above E[nb-1] -> nb-1; NaN -> 0
__device__ __forceinline__ int find_bin(float v, const float* E, int nb, float g0, float gs) {
  float t = (log2f(v) - g0) * gs;                  // a guess: log2 is approximate
  t = fminf(fmaxf(t, 0.f), (float)(nb - 1));       // -inf, NaN -> 0
  int b = (int)t;
  while (b > 0 && !(v >= E[b])) --b;               // exact fix-up against the edges
  while (b < nb - 1 && v >= E[b + 1]) ++b;
  return b;
}

using Kf = TwoSumF;   // compensated FP32 sum

// (sum, error) pair += v with Knuth's TwoSum (valid whatever the magnitudes)
__device__ __forceinline__ void pair_add(float2& p, float v) {
  const float t = p.x + v;
  const float bp = t - p.x;
  p.y += (p.x - (t - bp)) + (v - bp);
  p.x = t;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kStatsThreads) k_stats(const StatsArgs a) {
  __shared__ float E[3][kMB + 1];
  __shared__ unsigned int Hy[kMB * kMB];
  __shared__ unsigned int HJ[kMB * kMB];
  __shared__ unsigned int Cn[kMB];
  __shared__ unsigned int Cp;
  __shared__ float2 Wb[kWarps][kMB][2];   // (sum, error) of y and of N per density bin
  __shared__ double Ws[kWarps][kStatsScalars];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int nb_n = a.nb_n, nb_y = a.nb_y, nb_J = a.nb_J;
  for (int i = t; i < 3 * (kMB + 1); i += kStatsThreads) (&E[0][0])[i] = a.edges[i];
  for (int i = t; i < kMB * kMB; i += kStatsThreads) { Hy[i] = 0u; HJ[i] = 0u; }
  if (t < kMB) Cn[t] = 0u;
  if (t == 0) Cp = 0u;
  __syncthreads();

  // scalar sums: y, nH, nH y, N, T, nH T, N on the plateau
  Kf sy, sn, sny, sN, sT, snT, sNp;
  unsigned int cp = 0;
  for (int i = lane; i < kMB; i += 32) {
    Wb[w][i][0] = make_float2(0.f, 0.f);
    Wb[w][i][1] = make_float2(0.f, 0.f);
  }
  __syncwarp();
  const long long ncell = a.ncell;
  const long long stride = (long long)gridDim.x * kStatsThreads;
  const unsigned full = 0xffffffffu;
  for (long long base = (long long)blockIdx.x * kStatsThreads + (t & ~31); base < ncell;
       base += stride) {
    const long long i = base + lane;
    int bn = -1, ky = 0, kJ = 0;
    float yv = 0.f, Nv = 0.f;
    if (i < ncell) {
      const float n = __ldg(a.nH + i), yy = __ldg(a.y + i), NN = __ldg(a.N + i), TT = __ldg(a.T + i);
      bn = find_bin(n, E[0], nb_n, a.g[0], a.g[1]);
      ky = bn * nb_y + find_bin(yy, E[1], nb_y, a.g[2], a.g[3]);
      kJ = bn * nb_J + find_bin(NN, E[2], nb_J, a.g[4], a.g[5]);
      sy.add(yy); sn.add(n); sny.add(n * yy); sN.add(NN); sT.add(TT); snT.add(n * TT);
      if (n < a.n_plateau) { sNp.add(NN); ++cp; }
      yv = yy;
      Nv = NN;
    }
    // (aggregating the counts over the warp, with match-any rounds or run lengths, measured
    // slower than the contended shared-memory atomics)
    if (i < ncell) {
      atomicAdd(&Hy[ky], 1u);
      atomicAdd(&HJ[kJ], 1u);
      atomicAdd(&Cn[bn], 1u);
    }
    // per-density-bin sums: runs of consecutive lanes with the same bin are summed by a
    // segmented tree (lane L adds lane L+o while no run starts in (L, L+o]), then each run's
    // first lane adds its sum to the warp's FP64 row; runs of the same bin add in lane order
    const int bprev = __shfl_up_sync(full, bn, 1);
    const bool head = lane == 0 || bprev != bn;
    const unsigned heads = __ballot_sync(full, head);
    float ry = yv, rN = Nv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float uy = __shfl_down_sync(full, ry, o);
      const float uN = __shfl_down_sync(full, rN, o);
      if (lane + o < 32 && !(heads & (((1u << o) - 1u) << (lane + 1)))) { ry += uy; rN += uN; }
    }
    bool pending = head && bn >= 0;
    unsigned grp = __match_any_sync(full, pending ? bn : -1 - lane);
    while (__any_sync(full, pending)) {
      if (pending && lane == __ffs(grp) - 1) {
        pair_add(Wb[w][bn][0], ry);
        pair_add(Wb[w][bn][1], rN);
        pending = false;
      }
      grp &= grp - 1u;
      __syncwarp();
    }
  }
  // per-CTA reductions (fixed order)
  const double v[kStatsScalars] = {sy.value(), sn.value(), sny.value(), sN.value(), sT.value(),
                                   snT.value(), sNp.value()};
#pragma unroll
  for (int k = 0; k < kStatsScalars; ++k) {
    const double r = warp_sum(v[k]);
    if (lane == 0) Ws[w][k] = r;
  }
  if (cp) atomicAdd(&Cp, cp);
  __syncthreads();
  double* ps = a.part_scalar + (size_t)blockIdx.x * kStatsScalars;
  if (t < kStatsScalars) {
    double r = 0.0;
    for (int k = 0; k < kWarps; ++k) r += Ws[k][t];
    ps[t] = r;
  }
  double* pb = a.part_bins + (size_t)blockIdx.x * kMB * 2;
  if (t < 2 * kMB) {
    const int b = t >> 1, q = t & 1;
    double r = 0.0;
    for (int k = 0; k < kWarps; ++k) r += (double)Wb[k][b][q].x + (double)Wb[k][b][q].y;
    pb[t] = r;
  }
  for (int i = t; i < nb_n * nb_y; i += kStatsThreads)
    if (Hy[i]) atomicAdd(a.hist_y + i, (unsigned long long)Hy[i]);
  for (int i = t; i < nb_n * nb_J; i += kStatsThreads)
    if (HJ[i]) atomicAdd(a.hist_J + i, (unsigned long long)HJ[i]);
  if (t < nb_n && Cn[t]) atomicAdd(a.bin_count + t, (unsigned long long)Cn[t]);
  if (t == 0 && Cp) atomicAdd(a.plateau_count, (unsigned long long)Cp);
}

// Sums of the per-CTA slots in index order: out[0..S) scalars, out[S..S+2*kMB) bin sums.
__global__ void k_stats_final(const double* part_scalar, const double* part_bins, int nblocks,
                              double* out) {
  const int t = threadIdx.x;
  if (t < kStatsScalars) {
    double r = 0.0;
    for (int b = 0; b < nblocks; ++b) r += part_scalar[(size_t)b * kStatsScalars + t];
    out[t] = r;
  } else if (t < kStatsScalars + 2 * kMB) {
    const int k = t - kStatsScalars;
    double r = 0.0;
    for (int b = 0; b < nblocks; ++b) r += part_bins[(size_t)b * kMB * 2 + k];
    out[t] = r;
  }
}

}  // namespace

cudaError_t launch_stats(const StatsArgs& a, double* out, cudaStream_t s) {
  k_stats<<<kStatsBlocks, kStatsThreads, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_stats_final<<<1, 256, 0, s>>>(a.part_scalar, a.part_bins, kStatsBlocks, out);
  return cudaGetLastError();
}

}  // namespace aton
