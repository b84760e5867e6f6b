// aton_stats.cuh -- arguments and launcher of the ionisation/radiation statistics pass.
#pragma once
#include <cuda_runtime.h>

namespace aton {

constexpr int kStatsMaxBins = 64;          // per histogram axis (ATON_STATS_MAX_BINS)
constexpr int kStatsThreads = 256;
constexpr int kStatsBlocks = 148 * 3;      // fixed grid (three CTAs per SM): fixed summation order
constexpr int kStatsScalars = 7;           // sums of y, nH, nH y, N, T, nH T, N on the plateau

struct StatsArgs {
  const float* N;
  const float* y;
  const float* T;
  const float* nH;
  long long ncell;
  int nb_n, nb_y, nb_J;
  const float* edges;        // [3][kStatsMaxBins + 1]: nH edges, y edges, N edges of the J21 bins
  float g[6];                // bin guesses: (log2 v - g[2q]) * g[2q+1] for q = nH, y, N
  float n_plateau;
  double* part_scalar;       // [kStatsBlocks][kStatsScalars]
  double* part_bins;         // [kStatsBlocks][kStatsMaxBins][2]: sums of y and N per density bin
  unsigned long long* hist_y;         // [nb_n][nb_y]
  unsigned long long* hist_J;         // [nb_n][nb_J]
  unsigned long long* bin_count;      // [nb_n]
  unsigned long long* plateau_count;  // [1]
};

// The shared-memory attribute of k_stats on the current device (once per device, before the
// first launch there).
cudaError_t init_stats_attributes();

// k_stats then the fixed-order sum of its slots into out[kStatsScalars + 2 kStatsMaxBins].
cudaError_t launch_stats(const StatsArgs& a, double* out, cudaStream_t s);

}  // namespace aton
