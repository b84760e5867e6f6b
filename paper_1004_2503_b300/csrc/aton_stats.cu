// aton_stats.cu -- statistics of the ionisation state and of the radiation field (section 4:
// volume- and mass-weighted ionised fraction, Gamma12 and J21 averages, the distributions
// (1-x)(nH) and J21(nH) with the mean per density bin).
//
// One pass over N, y, T, nH with a fixed grid. Each thread takes four consecutive cells per
// iteration (one 16-byte load per field; a warp covers 128 consecutive cells). Every result is
// reproducible bit for bit:
//  - histogram counts in shared-memory integer atomics (equal keys of a thread's four cells
//    merged), added to global 64-bit counters per CTA (integer sums: exact in any order); the
//    count per density bin is the row sum of the (1-x) histogram;
//  - the scalar sums: the four cells' values summed pairwise in FP32, then added to per-thread
//    compensated FP32 accumulators (error-free TwoSum), reduced in FP64 per CTA into a per-CTA
//    slot, then summed over the slots in index order;
//  - the per-density-bin sums of y and N are exact: a float m 2^(e-150) (m its 24-bit
//    significand, e its biased exponent) is added as the integer m 2^(e mod 8) (below 2^31) to
//    a 64-bit shared-memory accumulator of its density bin and exponent band e / 8, kept as two
//    32-bit words: the low word takes the term with a 32-bit atomic add (64-bit shared atomics
//    are several times slower here) and the returned old value shows a carry, which the adding
//    thread then adds to the high word. Integer sums commute, so the order in which the lanes
//    add does not matter. At the end each CTA turns its bands into one FP64 value per bin (band
//    by band in a fixed order) for its slot. A CTA's sum stays below 2^63 for up to 2^32 cells
//    per CTA. (A valid state holds no negative or non-finite y or N; such a value makes its
//    bin's sum NaN.)
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
  float t = (__log2f(v) - g0) * gs;                // a guess (hardware log2, approximate)
  t = fminf(fmaxf(t, 0.f), (float)(nb - 1));       // -inf, NaN -> 0
  int b = (int)t;
  while (b > 0 && !(v >= E[b])) --b;               // exact fix-up against the edges
  while (b < nb - 1 && v >= E[b + 1]) ++b;
  return b;
}

using Kf = TwoSumF;   // compensated FP32 sum

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// counts of four keys into H, equal neighbours merged (one atomic per run of equal keys)
__device__ __forceinline__ void count4(unsigned int* H, int k0, int k1, int k2, int k3) {
  unsigned c = 1u;
  if (k1 == k0) ++c; else { atomicAdd(&H[k0], c); c = 1u; }
  if (k2 == k1) ++c; else { atomicAdd(&H[k1], c); c = 1u; }
  if (k3 == k2) ++c; else { atomicAdd(&H[k2], c); c = 1u; }
  atomicAdd(&H[k3], c);
}

constexpr int kBands = 32;   // exponent bands of the exact per-bin sums (8 exponents each)

// four (bin, value) pairs into the exact accumulators (lo, hi)[bin][band], equal neighbouring
// keys merged; a negative or non-finite value marks its bin in *bad instead
__device__ __forceinline__ void exact4(unsigned int* lo, unsigned int* hi, unsigned long long* bad,
                                       const int b[4], const float v[4]) {
  auto flush = [&](int key, unsigned long long acc) {
    const unsigned a0 = (unsigned)acc, a1 = (unsigned)(acc >> 32);
    const unsigned old = atomicAdd(&lo[key], a0);
    const unsigned c = a1 + (old + a0 < a0 ? 1u : 0u);   // the carry out of the low word
    if (c) atomicAdd(&hi[key], c);
  };
  int key = -1;
  unsigned long long acc = 0ull;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const unsigned u = __float_as_uint(v[j]), a = u & 0x7FFFFFFFu;
    if (a >= 0x7F800000u || (u != a && a != 0u)) {   // Inf, NaN or below zero (-0 is zero)
      atomicOr(bad, 1ull << b[j]);
      continue;
    }
    const int ef = (int)(a >> 23);
    const unsigned m = (a & 0x7FFFFFu) | (ef ? 0x800000u : 0u);
    const int e = max(ef, 1);                      // a subnormal: m 2^(1-150)
    const int k = b[j] * kBands + (e >> 3);
    if (k != key) {
      if (key >= 0 && acc) flush(key, acc);
      key = k;
      acc = 0ull;
    }
    acc += m << (e & 7);
  }
  if (key >= 0 && acc) flush(key, acc);
}

// shared memory of k_stats (dynamic: above the 48 KB static limit)
struct StatsSmem {
  unsigned int Alo[2][kMB * kBands];        // exact sums of y (0) and N (1) per bin and band:
  unsigned int Ahi[2][kMB * kBands];        // low and high 32-bit words
  unsigned long long bad[2];                // bins with a non-finite y (0) or N (1)
  double Ws[kWarps][kStatsScalars];
  unsigned int Hy[kMB * kMB];
  unsigned int HJ[kMB * kMB];
  float E[3][kMB + 1];
  unsigned int Cp;
};

__global__ void __launch_bounds__(kStatsThreads, kStatsBlocks / 148) k_stats(const StatsArgs a) {
  extern __shared__ __align__(16) unsigned char st_raw[];
  StatsSmem& S = *reinterpret_cast<StatsSmem*>(st_raw);
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int nb_n = a.nb_n, nb_y = a.nb_y, nb_J = a.nb_J;
  for (int i = t; i < 3 * (kMB + 1); i += kStatsThreads) (&S.E[0][0])[i] = a.edges[i];
  for (int i = t; i < kMB * kMB; i += kStatsThreads) { S.Hy[i] = 0u; S.HJ[i] = 0u; }
  for (int i = t; i < 2 * kMB * kBands; i += kStatsThreads) {
    (&S.Alo[0][0])[i] = 0u;
    (&S.Ahi[0][0])[i] = 0u;
  }
  if (t < 2) S.bad[t] = 0ull;
  if (t == 0) S.Cp = 0u;
  __syncthreads();

  // scalar sums: y, nH, nH y, N, T, nH T, N on the plateau
  Kf sy, sn, sny, sN, sT, snT, sNp;
  unsigned int cp = 0;
  const float npl = a.n_plateau;
  auto bins = [&](float n, float yy, float NN, int& ky, int& kJ) {
    const int b = find_bin(n, S.E[0], nb_n, a.g[0], a.g[1]);
    ky = b * nb_y + find_bin(yy, S.E[1], nb_y, a.g[2], a.g[3]);
    kJ = b * nb_J + find_bin(NN, S.E[2], nb_J, a.g[4], a.g[5]);
    return b;
  };
  const long long ncell = a.ncell;
  const long long n4 = ncell >> 2;                // groups of four cells (16-byte loads)
  const float4* __restrict__ gn = reinterpret_cast<const float4*>(a.nH);
  const float4* __restrict__ gy = reinterpret_cast<const float4*>(a.y);
  const float4* __restrict__ gN = reinterpret_cast<const float4*>(a.N);
  const float4* __restrict__ gT = reinterpret_cast<const float4*>(a.T);
  const long long stride = (long long)gridDim.x * kStatsThreads;
  // software-pipelined: the next group's four loads are issued before this group's bins and
  // sums, so the loads of one iteration overlap the shared-memory work of the previous one
  long long g = (long long)blockIdx.x * kStatsThreads + t;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 qn = z4, qy = z4, qN = z4, qT = z4;
  if (g < n4) { qn = __ldg(gn + g); qy = __ldg(gy + g); qN = __ldg(gN + g); qT = __ldg(gT + g); }
  for (; g < n4; g += stride) {
    const float4 n = qn, yy = qy, NN = qN, TT = qT;
    const long long gq = g + stride;
    if (gq < n4) { qn = __ldg(gn + gq); qy = __ldg(gy + gq); qN = __ldg(gN + gq); qT = __ldg(gT + gq); }
    int b[4], ky[4], kJ[4];
    b[0] = bins(n.x, yy.x, NN.x, ky[0], kJ[0]);
    b[1] = bins(n.y, yy.y, NN.y, ky[1], kJ[1]);
    b[2] = bins(n.z, yy.z, NN.z, ky[2], kJ[2]);
    b[3] = bins(n.w, yy.w, NN.w, ky[3], kJ[3]);
    count4(S.Hy, ky[0], ky[1], ky[2], ky[3]);
    count4(S.HJ, kJ[0], kJ[1], kJ[2], kJ[3]);
    const float vy[4] = {yy.x, yy.y, yy.z, yy.w}, vN[4] = {NN.x, NN.y, NN.z, NN.w};
    exact4(S.Alo[0], S.Ahi[0], &S.bad[0], b, vy);
    exact4(S.Alo[1], S.Ahi[1], &S.bad[1], b, vN);
    // (pairwise FP32 sums of the four cells: relative error at most 2^-23 for these
    // non-negative values, before the compensated accumulation)
    sy.add((yy.x + yy.y) + (yy.z + yy.w));
    sn.add((n.x + n.y) + (n.z + n.w));
    sny.add((n.x * yy.x + n.y * yy.y) + (n.z * yy.z + n.w * yy.w));
    sN.add((NN.x + NN.y) + (NN.z + NN.w));
    sT.add((TT.x + TT.y) + (TT.z + TT.w));
    snT.add((n.x * TT.x + n.y * TT.y) + (n.z * TT.z + n.w * TT.w));
    const bool p0 = n.x < npl, p1 = n.y < npl, p2 = n.z < npl, p3 = n.w < npl;
    if (p0 | p1 | p2 | p3) {
      sNp.add(((p0 ? NN.x : 0.f) + (p1 ? NN.y : 0.f)) + ((p2 ? NN.z : 0.f) + (p3 ? NN.w : 0.f)));
      cp += (unsigned)p0 + (unsigned)p1 + (unsigned)p2 + (unsigned)p3;
    }
  }
  // the last ncell % 4 cells: thread 0 of the first CTA, one by one
  if (blockIdx.x == 0 && t == 0) {
    for (long long i = 4 * n4; i < ncell; ++i) {
      const float n = a.nH[i], y1 = a.y[i], N1 = a.N[i], T1 = a.T[i];
      int ky, kJ;
      const int b1[4] = {bins(n, y1, N1, ky, kJ), 0, 0, 0};
      atomicAdd(&S.Hy[ky], 1u);
      atomicAdd(&S.HJ[kJ], 1u);
      const float vy[4] = {y1, 0.f, 0.f, 0.f}, vN[4] = {N1, 0.f, 0.f, 0.f};
      exact4(S.Alo[0], S.Ahi[0], &S.bad[0], b1, vy);   // (the zeros add nothing)
      exact4(S.Alo[1], S.Ahi[1], &S.bad[1], b1, vN);
      sy.add(y1); sn.add(n); sny.add(n * y1); sN.add(N1); sT.add(T1); snT.add(n * T1);
      if (n < npl) { sNp.add(N1); ++cp; }
    }
  }
  // per-CTA reductions (fixed order)
  const double v[kStatsScalars] = {sy.value(), sn.value(), sny.value(), sN.value(), sT.value(),
                                   snT.value(), sNp.value()};
#pragma unroll
  for (int k = 0; k < kStatsScalars; ++k) {
    const double r = warp_sum(v[k]);
    if (lane == 0) S.Ws[w][k] = r;
  }
  if (cp) atomicAdd(&S.Cp, cp);
  __syncthreads();
  double* ps = a.part_scalar + (size_t)blockIdx.x * kStatsScalars;
  if (t < kStatsScalars) {
    double r = 0.0;
    for (int k = 0; k < kWarps; ++k) r += S.Ws[k][t];
    ps[t] = r;
  }
  double* pb = a.part_bins + (size_t)blockIdx.x * kMB * 2;
  if (t < 2 * kMB) {   // the exact band sums of (bin, quantity) as one FP64 value
    const int bb = t >> 1, q = t & 1;
    double r = 0.0;
    for (int k = 0; k < kBands; ++k) {
      const int i = bb * kBands + k;
      const unsigned long long a = ((unsigned long long)S.Ahi[q][i] << 32) | S.Alo[q][i];
      // a 2^(8k - 150): the power of two built from its bit pattern (a normal double)
      if (a) r += (double)a * __longlong_as_double((long long)(1023 + 8 * k - 150) << 52);
    }
    pb[t] = (S.bad[q] >> bb) & 1ull ? __longlong_as_double(0x7FF8000000000000ll) : r;
  }
  for (int i = t; i < nb_n * nb_y; i += kStatsThreads)
    if (S.Hy[i]) atomicAdd(a.hist_y + i, (unsigned long long)S.Hy[i]);
  for (int i = t; i < nb_n * nb_J; i += kStatsThreads)
    if (S.HJ[i]) atomicAdd(a.hist_J + i, (unsigned long long)S.HJ[i]);
  if (t < nb_n) {   // cells per density bin: the row sum of the (1-x) histogram
    unsigned long long c = 0;
    for (int j = 0; j < nb_y; ++j) c += S.Hy[t * nb_y + j];
    if (c) atomicAdd(a.bin_count + t, c);
  }
  if (t == 0 && S.Cp) atomicAdd(a.plateau_count, (unsigned long long)S.Cp);
}

// Sums of the per-CTA slots in index order: out[0..S) scalars, out[S..S+2*kMB) bin sums.
__global__ void k_stats_final(const double* part_scalar, const double* part_bins, int nblocks,
                              double* out) {
  const int t = threadIdx.x;
  // (the loads are unrolled ahead of the additions, which stay in slot order)
  if (t < kStatsScalars) {
    double r = 0.0;
#pragma unroll 16
    for (int b = 0; b < nblocks; ++b) r += part_scalar[(size_t)b * kStatsScalars + t];
    out[t] = r;
  } else if (t < kStatsScalars + 2 * kMB) {
    const int k = t - kStatsScalars;
    double r = 0.0;
#pragma unroll 16
    for (int b = 0; b < nblocks; ++b) r += part_bins[(size_t)b * kMB * 2 + k];
    out[t] = r;
  }
}

}  // namespace

cudaError_t init_stats_attributes() {
  return cudaFuncSetAttribute(k_stats, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(StatsSmem));
}

cudaError_t launch_stats(const StatsArgs& a, double* out, cudaStream_t s) {
  k_stats<<<kStatsBlocks, kStatsThreads, sizeof(StatsSmem), s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_stats_final<<<1, 256, 0, s>>>(a.part_scalar, a.part_bins, kStatsBlocks, out);
  return cudaGetLastError();
}

}  // namespace aton
