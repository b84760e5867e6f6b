// aton_internal.h -- shared declarations of the libaton.so host code and kernels (not part
// of the public C ABI, which is include/aton.h).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <utility>
#include <vector>

#include "aton.h"
#include "aton_device.cuh"
#include "aton_mlp.cuh"

namespace aton {

constexpr int kTileX = 32;          // cells per CTA row in x (one warp)
constexpr int kPlainBlocks = 148 * 8;  // fixed grid of the unfused kernels (deterministic slots)
constexpr int kPlainThreads = 256;
constexpr int kSurBlocks = kPlainBlocks;  // grid of the surrogate pass (CTAs without candidates exit)

// One point source of a fused tile: plane z, cell (tx + 32*ty) inside the tile, dN added.
struct TileSrc {
  int z;
  int cell;
  float dN;
  int pad;
};

// Per-slot tallies written by the kernels (one slot per fused tile or unfused block).
struct Slots {
  double* acc = nullptr;              // [n][3]: absorbed, escaped, clipped (density units)
  unsigned long long* sub = nullptr;  // [n]: sub-steps
  unsigned int* mx = nullptr;         // [n]: max sub-steps of a cell
  unsigned int* err = nullptr;        // [n]: cells at the sub-cycle cap
  unsigned int* nan = nullptr;        // [n]: non-finite cells
  unsigned int* timeout = nullptr;    // [1]: pipeline waits that gave up (must stay 0)
  unsigned int* sur = nullptr;        // [n]: cells whose chemistry the surrogate replaced
  int n = 0;
};

// Tensor maps of the TMA-staged fused kernel (one set per tile height).
struct TmaMaps {
  CUtensorMap u[2][4];   // ping-pong buffer x (N, Fx, Fy, Fz), box (32+8) x (ty+2) x 1
};

struct Fields {
  float* N;
  float* Fx;
  float* Fy;
  float* Fz;
};

// A cell the fused kernel's surrogate gate selected, kept until the end of its CTA (F as F / c).
struct SurRec {
  float N, X, Y, Z, y, T, n;
  int o;
};
constexpr int kSurCap = 64;   // cells per CTA; a cell beyond them takes the exact operator at once

// The chemistry surrogate in the fused kernel (surrogate instance only).
struct SurList {
  const MlpImage* img = nullptr;   // BF16 weight image of the network (device)
  const MlpNorm* norm = nullptr;   // normalisation and training range (device)
  float gate = 0.f;                // sub-step estimate at which a cell is offered
  float resid = 0.f;               // photon residual up to which a prediction is accepted
  SurRec* buf = nullptr;           // [tile][kSurCap] selected cells (device)
  int* cnt = nullptr;              // [tile] cells listed (zero between steps)
};

struct FusedArgs {
  StepParams P;
  Fields in, out;
  float* y;
  float* T;
  const float* nH;
  const int* tsrc_start;  // [ntile + 1]
  const TileSrc* tsrc;
  Slots slots;
  int tz;
  int in_buf;   // ping-pong index of `in` (selects the TMA maps)
  SurList sur;  // (surrogate instance only: img != nullptr)
};

struct PlainArgs {
  StepParams P;
  Fields in, out;
  float* y;
  float* T;
  const float* nH;
  const int* src_idx;   // merged sources
  const float* src_dN;
  int nsrc;
  Slots slots;
  // pair sink: every `sink_stride`-th cell (offset rotating with the step) writes a record
  float* sink;
  long long sink_cap, sink_base;
  int sink_stride, sink_phase;
  // surrogate chemistry
  const MlpImage* sur_img;
  const MlpNorm* sur_norm;
  float sur_gate, sur_resid;
  int* sur_list;        // candidate cells of the step (capacity ncell)
  int* sur_count;       // number of candidates (reset before every chemistry pass)
  bool transported;     // the transport pass already ran (launch_transport_tma): sources and
                        // chemistry only
};

// The standard chemistry configuration (evolving temperature, cooling and collisional
// ionisation on, no clumping): the fused kernels have a compile-time instance for it.
inline bool standard_chemistry(const StepParams& P) {
  return !P.fixed_T && P.cooling && P.coll_ion && !(P.clR_A > 0.f) && !(P.clI_A > 0.f);
}

// ---- training step of the surrogate MLP on tcgen05 (aton_mlp_tc.cu) ----
// 128 rows per CTA of kMlpTcThreads threads; one partial gradient per CTA, kMlpPartStride floats
// apart (the parameter vector padded to a multiple of four floats: 16-byte stores)
constexpr int kMlpTcThreads = 256;
constexpr int kMlpPartStride = (kMlpParams + 3) & ~3;
__global__ void k_mlp_train_tc(const MlpTcImage* __restrict__ img, const float* __restrict__ X,
                               const float* __restrict__ T, int n, float inv_count, float* partial,
                               float* loss_part, unsigned int* err);
size_t mlp_train_tc_smem();

// ---- last-failure message of the calling thread (aton_capi.cu) ----
void set_last_message(const char* msg);

// ---- launchers (aton_kernels.cu) ----
cudaError_t init_kernel_attributes();
cudaError_t init_tma_attributes();
cudaError_t launch_fused_tma(int ty, int rpt, const FusedArgs& a, const TmaMaps& m,
                             cudaStream_t s);
// the transport pass of the plain step on the TMA-staged kernel (tile 32 x 8; GLF flux)
cudaError_t launch_transport_tma(const FusedArgs& a, const TmaMaps& m8, cudaStream_t s);
bool make_tma_maps(int nx, int ny, int nz, int ty, float* const u[2][4], TmaMaps* out);
cudaError_t launch_fused(int ty, const FusedArgs& a, cudaStream_t s);
int fused_tiles(int nx, int ny, int nz, int ty, int tz);
cudaError_t launch_plain_step(const PlainArgs& a, cudaStream_t s);
const MlpImage* mlp_image(const struct ::aton_mlp* h);
const MlpNorm* mlp_norm(const struct ::aton_mlp* h);
int plain_launches();
cudaError_t launch_scale(float* dst, const float* src, float k, int64_t n, cudaStream_t s);
cudaError_t launch_max_f2(const float* N, const float* Fx, const float* Fy, const float* Fz,
                          float rc, int64_t n, unsigned int* out, cudaStream_t s);
cudaError_t launch_one_minus(float* dst, const float* src, int64_t n, cudaStream_t s);
cudaError_t launch_validate(const float* N, const float* y, const float* T, const float* nH,
                            int64_t n, unsigned int* bad, cudaStream_t s);
cudaError_t launch_reduce_slots(const Slots& sl, double* out_acc3, unsigned long long* out_u64_4,
                                cudaStream_t s);
cudaError_t launch_sum_field(const float* f, int64_t n, double* partial, double* out,
                             cudaStream_t s);
constexpr int kSumBlocks = 148 * 4;

}  // namespace aton
