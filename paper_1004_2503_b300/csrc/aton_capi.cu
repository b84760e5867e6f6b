// aton_capi.cu -- host implementation of the C ABI declared in include/aton.h.
//
// The handle owns the device state (double-buffered N, F; y = 1 - x, T, nH in place),
// the per-tile tally slots, the point-source lists (merged per cell, and bucketed per fused
// tile), and a cache of CUDA graphs that each replay a batch of steps. The host only queues
// work (section 2.2 and the Appendix: the host drives the time loop and never computes on the
// data); it reads back only when a call returns data.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "aton_internal.h"
#include "aton_stats.cuh"

using namespace aton;

static thread_local std::string g_msg;
static constexpr int kMaxDevices = 64;
static std::mutex g_attr_mutex;            // guards g_attr_done
static bool g_attr_done[kMaxDevices] = {};  // kernel attributes set on device d

static int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_msg = buf;
  return code;
}

void aton::set_last_message(const char* msg) { g_msg = msg ? msg : ""; }

#define CU(call)                                                                    \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return fail(e_ == cudaErrorMemoryAllocation ? ATON_ERR_NOMEM : ATON_ERR_CUDA, \
                  "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

static constexpr double kEV = 1.602176634e-12;
static constexpr double kKBh = 1.380649e-16;
static constexpr double kIH = 13.6;  // eV

struct aton_ctx {
  int nx = 0, ny = 0, nz = 0;
  int64_t ncell = 0;
  double dx = 0, c = 0, dt = 0, V = 0;
  aton_params prm{};
  int device = 0;
  cudaStream_t own = nullptr, user = nullptr;
  float* f[2][4] = {{nullptr}};
  float *y = nullptr, *T = nullptr, *nH = nullptr;
  int cur = 0;
  bool fields_set = false;
  // reductions
  double* d_part = nullptr;
  double* d_out = nullptr;            // [4]: acc3 + stored
  unsigned long long* d_u64 = nullptr;  // [5]
  unsigned int* d_bad = nullptr;
  Slots slots;
  // folded tallies (density units for the photon sums)
  double fold_acc[3] = {0, 0, 0};
  unsigned long long fold_u[5] = {0, 0, 0, 0, 0};
  double emitted = 0, stored0 = 0;
  double offs[ATON_BUDGET_LEN] = {0};
  int64_t steps = 0;
  int latched = ATON_OK;
  // sources
  std::vector<std::pair<int64_t, double>> src;  // merged (cell, rate), sorted by cell
  // pinned staging of the source upload (two buffers, each free again once its event has
  // completed), so the per-step upload is an asynchronous copy
  char* src_pin[2] = {nullptr, nullptr};
  size_t src_pin_cap = 0;
  cudaEvent_t src_ev[2] = {nullptr, nullptr};
  int src_pin_i = 0;
  double emit_per_step = 0;       // photons actually injected per step
  // device copy of the staging layout (one upload per change): the merged list (cell index,
  // photons per step) and the per-tile records with their tile offsets
  char* d_srcbuf = nullptr;
  size_t srcbuf_cap = 0;
  int* d_src_idx = nullptr;
  float* d_src_dN = nullptr;
  int src_n = 0;
  int* d_tstart = nullptr;
  TileSrc* d_tsrc = nullptr;
  bool tiles_dirty = true;
  // execution
  int mode = ATON_MODE_FUSED;
  int graph_batch = 100;
  int ty = 8, tz = 64;
  int rpt = 2;         // rows of the fused tile per thread (2: TMA kernel, ty >= 8, GLF flux)
  std::map<std::pair<int, int>, cudaGraphExec_t> graphs;
  TmaMaps tma[3];          // tile heights 4, 8, 16
  bool tma_ok[3] = {false, false, false};
  // pair sink and surrogate
  float* sink = nullptr;
  long long sink_cap = 0, sink_steps = 0;
  int sink_stride = 1;
  aton_mlp_handle sur = nullptr;
  aton_surrogate_params sur_p{};
  int* sur_list = nullptr;
  int* sur_count = nullptr;
  // the fused kernel's per-tile surrogate lists (sized for sur_tiles tiles)
  SurRec* sur_buf = nullptr;
  int* sur_cnt = nullptr;
  int sur_tiles = 0;
  double quiet_k = 0.0;   // rate bound of the chemistry's cold-gas shortcut (set with prm)
  // asynchronous budget read: pinned landing area [acc3, stored, timeout word], event, and the
  // host-side terms as of the request
  double* bud_pin = nullptr;
  cudaEvent_t bud_ev = nullptr;
  bool bud_pending = false;
  double bud_fold[3] = {0, 0, 0};
  double bud_emitted = 0, bud_stored0 = 0;
  double bud_offs[ATON_BUDGET_LEN] = {0};
  // statistics pass
  float* st_edges = nullptr;
  double* st_part = nullptr;
  double* st_out = nullptr;
  unsigned long long* st_u64 = nullptr;

  cudaStream_t stream() const { return user ? user : own; }
};

static int check_h(aton_handle h) {
  if (!h) return fail(ATON_ERR_BADARG, "null handle");
  return ATON_OK;
}

static void drop_graphs(aton_handle h) {
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
}

// Upper bound over T in [T_floor, 1300 K] of alpha_B(T) and of the recombination plus free-free
// cooling coefficients over 1.5 T (both / kB), with a 25 % margin over the maximum on a fine
// grid: the kernels skip those rates in cold gas where this bound makes their effect on y and T
// smaller than 2^-26 relatively.
static double quiet_bound(double T_floor) {
  double m = 0.0;
  const double lo = std::log(T_floor), hi = std::log(1300.0);
  for (int i = 0; i <= 4000; ++i) {
    const double T = std::exp(lo + (hi - lo) * i / 4000.0);
    const double lam = 2.0 * 157807.0 / T;
    const double alpha = 2.753e-14 * std::pow(lam, 1.5) / std::pow(1.0 + std::pow(lam / 2.740, 0.407), 2.242);
    const double rec = 3.435e-30 * T * std::pow(lam, 1.970) / std::pow(1.0 + std::pow(lam / 2.250, 0.376), 3.720);
    const double d = std::log10(T) - 5.5;
    const double ff = 1.42e-27 * (1.1 + 0.34 * std::exp(-d * d / 3.0)) * std::sqrt(T);
    m = std::fmax(m, std::fmax(alpha, (rec + ff) / kKBh / (1.5 * T)));
  }
  return 1.25 * m;
}

static StepParams step_params(const aton_ctx* h) {
  StepParams P{};
  P.nx = h->nx; P.ny = h->ny; P.nz = h->nz;
  P.bc = h->prm.bc;
  P.lam = (float)(h->c * h->dt / h->dx);
  P.c = (float)h->c;
  P.rc = (float)(1.0 / h->c);
  P.dt = (float)h->dt;
  P.csig = (float)(h->c * h->prm.sigma_n);
  const double eheat = (h->prm.sigma_e * h->prm.e_gamma_eV - h->prm.sigma_n * kIH) / h->prm.sigma_n;
  P.eheat_K = (float)(eheat * kEV / kKBh);
  P.fixed_T = h->prm.fixed_T != 0;
  P.coll_ion = h->prm.coll_ion != 0;
  P.cooling = h->prm.cooling != 0;
  P.max_sub = h->prm.max_sub;
  P.T_floor = (float)h->prm.T_floor;
  P.sub_eps = (float)h->prm.sub_eps;
  P.y_floor = (float)h->prm.y_floor;
  P.clR_A = (float)h->prm.clump_R_A; P.clR_b = (float)h->prm.clump_R_b;
  P.clI_A = (float)h->prm.clump_I_A; P.clI_b = (float)h->prm.clump_I_b;
  P.hll = h->prm.flux == ATON_FLUX_HLL;
  P.quiet_k = (float)h->quiet_k;
  P.quiet_dt = (float)(h->dt * h->quiet_k * 67108864.0);
  P.heat_eps = (float)(eheat * kEV / kKBh / (1.5 * h->prm.sub_eps));
  P.eheat15 = (float)(eheat * kEV / kKBh / 1.5);
  return P;
}

static int slots_needed(const aton_ctx* h) {
  // the plain path with the surrogate uses two slot ranges of kPlainBlocks, its transport pass
  // on the TMA-staged kernel one slot per 32 x 8 tile
  return std::max({fused_tiles(h->nx, h->ny, h->nz, h->ty, h->tz),
                   fused_tiles(h->nx, h->ny, h->nz, 8, h->tz), 2 * kPlainBlocks});
}

static void free_slots(Slots& s) {
  cudaFree(s.acc); cudaFree(s.sub); cudaFree(s.mx); cudaFree(s.err); cudaFree(s.nan);
  cudaFree(s.timeout); cudaFree(s.sur);
  s = Slots{};
}

static int ty_index(int ty) { return ty == 4 ? 0 : (ty == 8 ? 1 : 2); }

// Adds the slot tallies into the host fold (FP64, fixed order) and clears the slots.
static int fold_slots(aton_handle h) {
  if (h->slots.n == 0) return ATON_OK;
  cudaStream_t s = h->stream();
  CU(launch_reduce_slots(h->slots, h->d_out, h->d_u64, s));
  double a[3];
  unsigned long long u[5];
  CU(cudaMemcpyAsync(a, h->d_out, sizeof(a), cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(u, h->d_u64, sizeof(u), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  for (int i = 0; i < 3; ++i) h->fold_acc[i] += a[i];
  h->fold_u[0] += u[0];
  h->fold_u[1] = std::max(h->fold_u[1], u[1]);
  h->fold_u[2] += u[2];
  h->fold_u[3] += u[3];
  h->fold_u[4] += u[4];
  const int n = h->slots.n;
  CU(cudaMemsetAsync(h->slots.acc, 0, sizeof(double) * 3 * n, s));
  CU(cudaMemsetAsync(h->slots.sub, 0, sizeof(unsigned long long) * n, s));
  CU(cudaMemsetAsync(h->slots.mx, 0, sizeof(unsigned int) * n, s));
  CU(cudaMemsetAsync(h->slots.err, 0, sizeof(unsigned int) * n, s));
  CU(cudaMemsetAsync(h->slots.nan, 0, sizeof(unsigned int) * n, s));
  CU(cudaMemsetAsync(h->slots.sur, 0, sizeof(unsigned int) * n, s));
  return ATON_OK;
}

static int ensure_slots_n(aton_handle h, int need) {
  if (h->slots.n >= need) return ATON_OK;
  int rc = fold_slots(h);
  if (rc) return rc;
  free_slots(h->slots);
  drop_graphs(h);
  Slots s;
  cudaError_t e;
  if ((e = cudaMalloc(&s.acc, sizeof(double) * 3 * need)) != cudaSuccess ||
      (e = cudaMalloc(&s.sub, sizeof(unsigned long long) * need)) != cudaSuccess ||
      (e = cudaMalloc(&s.mx, sizeof(unsigned int) * need)) != cudaSuccess ||
      (e = cudaMalloc(&s.err, sizeof(unsigned int) * need)) != cudaSuccess ||
      (e = cudaMalloc(&s.nan, sizeof(unsigned int) * need)) != cudaSuccess ||
      (e = cudaMalloc(&s.timeout, sizeof(unsigned int))) != cudaSuccess ||
      (e = cudaMalloc(&s.sur, sizeof(unsigned int) * need)) != cudaSuccess) {
    free_slots(s);   // (what was allocated before the failure)
    return fail(e == cudaErrorMemoryAllocation ? ATON_ERR_NOMEM : ATON_ERR_CUDA,
                "tally slots: %s", cudaGetErrorString(e));
  }
  s.n = need;
  h->slots = s;
  cudaStream_t st = h->stream();
  CU(cudaMemsetAsync(s.acc, 0, sizeof(double) * 3 * need, st));
  CU(cudaMemsetAsync(s.sub, 0, sizeof(unsigned long long) * need, st));
  CU(cudaMemsetAsync(s.mx, 0, sizeof(unsigned int) * need, st));
  CU(cudaMemsetAsync(s.err, 0, sizeof(unsigned int) * need, st));
  CU(cudaMemsetAsync(s.nan, 0, sizeof(unsigned int) * need, st));
  CU(cudaMemsetAsync(s.timeout, 0, sizeof(unsigned int), st));
  CU(cudaMemsetAsync(s.sur, 0, sizeof(unsigned int) * need, st));
  return ATON_OK;
}

static int ensure_slots(aton_handle h) { return ensure_slots_n(h, slots_needed(h)); }

// Uploads the merged source list and the per-tile buckets of the current fused tile.
static size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

static int upload_sources(aton_handle h) {
  cudaStream_t s = h->stream();
  const int n = (int)h->src.size();
  const int gxn = (h->nx + kTileX - 1) / kTileX, gyn = (h->ny + h->ty - 1) / h->ty;
  const int ntile = fused_tiles(h->nx, h->ny, h->nz, h->ty, h->tz);
  // staging layout: idx[n] int, dN[n] float, start[ntile+1] int, tile records[n]
  const size_t o_dN = align16(sizeof(int) * n), o_st = o_dN + align16(sizeof(float) * n);
  const size_t o_ts = o_st + align16(sizeof(int) * (ntile + 1));
  const size_t need = o_ts + sizeof(TileSrc) * std::max(n, 1);
  const int b = h->src_pin_i;
  for (int q = 0; q < 2; ++q)
    if (!h->src_ev[q] && cudaEventCreateWithFlags(&h->src_ev[q], cudaEventDisableTiming) != cudaSuccess)
      return fail(ATON_ERR_CUDA, "cudaEventCreate failed");
  if (need > h->src_pin_cap) {
    for (int q = 0; q < 2; ++q) {
      CU(cudaEventSynchronize(h->src_ev[q]));
      if (h->src_pin[q]) cudaFreeHost(h->src_pin[q]);
      h->src_pin[q] = nullptr;
    }
    const size_t cap = std::max(need + need / 2, (size_t)65536);
    for (int q = 0; q < 2; ++q)
      if (cudaMallocHost(&h->src_pin[q], cap) != cudaSuccess) {
        h->src_pin_cap = 0;
        return fail(ATON_ERR_NOMEM, "pinned staging of %zu bytes failed", cap);
      }
    h->src_pin_cap = cap;
  }
  // the buffer's previous upload has been copied (in practice long ago)
  CU(cudaEventSynchronize(h->src_ev[b]));
  char* pb = h->src_pin[b];
  int* idx = reinterpret_cast<int*>(pb);
  float* dN = reinterpret_cast<float*>(pb + o_dN);
  int* start = reinterpret_cast<int*>(pb + o_st);
  TileSrc* ts = reinterpret_cast<TileSrc*>(pb + o_ts);
  double emit = 0;
  for (int k = 0; k < n; ++k) {
    idx[k] = (int)h->src[k].first;
    dN[k] = (float)(h->src[k].second * h->dt / h->V);
    emit += (double)dN[k] * h->V;
  }
  h->emit_per_step = emit;
  if (need > h->srcbuf_cap) {
    cudaFree(h->d_srcbuf);   // (synchronises: no step still reads it)
    h->d_srcbuf = nullptr;
    h->srcbuf_cap = 0;
    const size_t cap = h->src_pin_cap;
    CU(cudaMalloc(&h->d_srcbuf, cap));
    h->srcbuf_cap = cap;
  }
  // the kernels' pointers into the buffer move with n and the tile count: captured graphs
  // hold them (and the unfused source launch size), so they are dropped when these change
  int* const p_idx = reinterpret_cast<int*>(h->d_srcbuf);
  float* const p_dN = reinterpret_cast<float*>(h->d_srcbuf + o_dN);
  int* const p_st = reinterpret_cast<int*>(h->d_srcbuf + o_st);
  TileSrc* const p_ts = reinterpret_cast<TileSrc*>(h->d_srcbuf + o_ts);
  if (p_idx != h->d_src_idx || p_dN != h->d_src_dN || p_st != h->d_tstart ||
      p_ts != h->d_tsrc || h->src_n != n)
    drop_graphs(h);
  h->d_src_idx = p_idx; h->d_src_dN = p_dN; h->d_tstart = p_st; h->d_tsrc = p_ts;
  h->src_n = n;
  // per-tile records ordered by (tile, z, cell): the merged list is sorted by cell index, so
  // within a tile it is already in (z, cell) order and a stable counting sort by tile suffices
  std::vector<int> tile_of(n);
  std::fill(start, start + ntile + 1, 0);
  for (int k = 0; k < n; ++k) {
    const int64_t c = h->src[k].first;
    const int i = (int)(c % h->nx), j = (int)((c / h->nx) % h->ny), z = (int)(c / ((int64_t)h->nx * h->ny));
    const int bx = i / kTileX, by = j / h->ty, bz = z / h->tz;
    tile_of[k] = bx + gxn * (by + gyn * bz);
    start[tile_of[k] + 1] += 1;
  }
  for (int t = 0; t < ntile; ++t) start[t + 1] += start[t];
  {
    std::vector<int> fill(start, start + ntile);
    for (int k = 0; k < n; ++k) {
      const int64_t c = h->src[k].first;
      const int i = (int)(c % h->nx), j = (int)((c / h->nx) % h->ny), z = (int)(c / ((int64_t)h->nx * h->ny));
      ts[fill[tile_of[k]]++] = TileSrc{z, (i % kTileX) + kTileX * (j % h->ty), dN[k], 0};
    }
  }
  CU(cudaMemcpyAsync(h->d_srcbuf, pb, need, cudaMemcpyHostToDevice, s));
  CU(cudaEventRecord(h->src_ev[b], s));
  h->src_pin_i = 1 - b;
  h->tiles_dirty = false;
  return ATON_OK;
}

static bool sur_on(const aton_ctx* h) { return h->sur && h->sur_p.enabled; }

// Steps that take the plain three-kernel path whatever the execution mode: with the pair sink,
// with the HLL flux unless the TMA-staged fused kernel can run it, and with the surrogate unless
// the TMA-staged fused kernel can run the network (GLF flux).
static bool plain_only(const aton_ctx* h) {
  const bool tma_fused = h->mode == ATON_MODE_FUSED && h->tma_ok[ty_index(h->ty)];
  return h->sink != nullptr || (h->prm.flux == ATON_FLUX_HLL && !tma_fused) ||
         (sur_on(h) && (!tma_fused || h->prm.flux == ATON_FLUX_HLL));
}

static int enqueue_step(aton_handle h, cudaStream_t s) {
  const int nxt = 1 - h->cur;
  const Fields in{h->f[h->cur][0], h->f[h->cur][1], h->f[h->cur][2], h->f[h->cur][3]};
  const Fields out{h->f[nxt][0], h->f[nxt][1], h->f[nxt][2], h->f[nxt][3]};
  cudaError_t e;
  if (!plain_only(h) && (h->mode == ATON_MODE_FUSED || h->mode == ATON_MODE_FUSED_LDG)) {
    FusedArgs a{};
    a.P = step_params(h);
    a.in = in; a.out = out;
    a.y = h->y; a.T = h->T; a.nH = h->nH;
    a.tsrc_start = h->d_tstart; a.tsrc = h->d_tsrc;
    a.slots = h->slots;
    a.tz = h->tz;
    a.in_buf = h->cur;
    const int ti = ty_index(h->ty);
    if (sur_on(h)) {
      // (plain_only routes every other surrogate case to the plain step: here the TMA kernel
      // with the GLF flux runs the network for the cells its gate selects)
      a.sur.img = mlp_image(h->sur);
      a.sur.norm = mlp_norm(h->sur);
      a.sur.gate = (float)h->sur_p.gate_substeps;
      a.sur.resid = (float)h->sur_p.residual_max;
      a.sur.buf = h->sur_buf;
      a.sur.cnt = h->sur_cnt;
      e = launch_fused_tma(h->ty, h->ty >= 8 ? h->rpt : 1, a, h->tma[ti], s);
    } else if (h->mode == ATON_MODE_FUSED && h->tma_ok[ti]) {
      // (two rows per thread: tile heights 8 and 16 with the GLF flux)
      const int rpt = h->ty >= 8 && h->prm.flux != ATON_FLUX_HLL ? h->rpt : 1;
      e = launch_fused_tma(h->ty, rpt, a, h->tma[ti], s);
    } else {
      e = launch_fused(h->ty, a, s);
    }
  } else {
    PlainArgs a{};
    a.P = step_params(h);
    a.in = in; a.out = out;
    a.y = h->y; a.T = h->T; a.nH = h->nH;
    a.src_idx = h->d_src_idx; a.src_dN = h->d_src_dN; a.nsrc = h->src_n;
    a.slots = h->slots;
    if (h->sink) {
      const long long per = (h->ncell + h->sink_stride - 1) / h->sink_stride;
      a.sink = h->sink;
      a.sink_cap = h->sink_cap;
      a.sink_stride = h->sink_stride;
      a.sink_phase = (int)(h->sink_steps % h->sink_stride);
      a.sink_base = h->sink_steps * per;
    }
    if (h->sur && h->sur_p.enabled) {
      a.sur_img = mlp_image(h->sur);
      a.sur_norm = mlp_norm(h->sur);
      a.sur_gate = (float)h->sur_p.gate_substeps;
      a.sur_resid = (float)h->sur_p.residual_max;
      a.sur_list = h->sur_list;
      a.sur_count = h->sur_count;
    }
    // the transport pass on the TMA-staged kernel (one closure per cell) where the grid allows
    // it and the flux is GLF; otherwise k_plain_transport
    if (h->prm.flux == ATON_FLUX_GLF && h->tma_ok[ty_index(8)]) {
      FusedArgs t{};
      t.P = a.P;
      t.in = in; t.out = out;
      t.y = h->y; t.T = h->T; t.nH = h->nH;
      t.slots = h->slots;
      t.tz = h->tz;
      t.in_buf = h->cur;
      e = launch_transport_tma(t, h->tma[ty_index(8)], s);
      if (e != cudaSuccess) return fail(ATON_ERR_CUDA, "transport launch: %s", cudaGetErrorString(e));
      a.transported = true;
    }
    e = launch_plain_step(a, s);
    if (h->sink) h->sink_steps += 1;
  }
  if (e != cudaSuccess) return fail(ATON_ERR_CUDA, "step launch: %s", cudaGetErrorString(e));
  h->cur = nxt;
  return ATON_OK;
}

// The fused kernel's per-tile surrogate lists for the current tiling (counts zeroed; the kernel
// leaves them zero). Captured graphs hold the pointers, so they are dropped on a reallocation.
static int ensure_sur_lists(aton_handle h) {
  const int need = fused_tiles(h->nx, h->ny, h->nz, h->ty, h->tz);
  if (h->sur_tiles >= need) return ATON_OK;
  CU(cudaStreamSynchronize(h->stream()));
  cudaFree(h->sur_buf); cudaFree(h->sur_cnt);
  h->sur_buf = nullptr; h->sur_cnt = nullptr; h->sur_tiles = 0;
  drop_graphs(h);
  CU(cudaMalloc(&h->sur_buf, sizeof(SurRec) * kSurCap * (size_t)need));
  CU(cudaMalloc(&h->sur_cnt, sizeof(int) * (size_t)need));
  CU(cudaMemsetAsync(h->sur_cnt, 0, sizeof(int) * (size_t)need, h->stream()));
  h->sur_tiles = need;
  return ATON_OK;
}

static int prepare(aton_handle h) {
  if (!h->fields_set) return fail(ATON_ERR_STATE, "aton_set_fields has not been called");
  int rc = ensure_slots(h);
  if (rc) return rc;
  if (sur_on(h) && !plain_only(h) && h->mode == ATON_MODE_FUSED) {
    rc = ensure_sur_lists(h);
    if (rc) return rc;
  }
  if (h->tiles_dirty) {
    rc = upload_sources(h);
    if (rc) return rc;
  }
  return ATON_OK;
}

extern "C" {

void aton_default_params(aton_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->sigma_n = 2.93e-18;
  p->sigma_e = 2.49e-18;
  p->e_gamma_eV = 20.27;
  p->bc = ATON_BC_PERIODIC;
  p->fixed_T = 0;
  p->coll_ion = 1;
  p->cooling = 1;
  p->max_sub = 10000;
  p->T_floor = 1.0;
  p->sub_eps = 0.1;
  p->y_floor = 1e-6;
}

// ---------------------------------------------------------------------------------------
// Ionisation and radiation statistics (section 4)
// ---------------------------------------------------------------------------------------
static constexpr double kHPlanck = 6.62607015e-27;  // erg s
static constexpr double kSigma0 = 6.30e-18;         // HI cross-section at the Lyman limit, cm^2
static constexpr double kPi = 3.14159265358979323846;

// Gamma per unit J21 under the power-law reading: Gamma = 4 pi J_0 sigma_0 / (h (alpha + 3))
static double gamma_per_J21(double alpha) {
  return 4.0 * kPi * kSigma0 * 1e-21 / (kHPlanck * (alpha + 3.0));
}

int aton_default_stats_params(aton_stats_params* p) {
  if (!p) return fail(ATON_ERR_BADARG, "p is NULL");
  p->nb_nH = 48; p->nb_y = 48; p->nb_J = 48;
  p->nH_lo = 1e-6; p->nH_hi = 1.0;
  p->y_lo = 1e-7; p->y_hi = 1.0;
  p->J21_lo = 1e-6; p->J21_hi = 1e4;
  p->spectral_index = 1.0;
  p->nH_plateau = 1e-3;
  return ATON_OK;
}

// edge k of nb log-spaced bins over [lo, hi], divided by div, rounded to float
static void log_edges(double lo, double hi, int nb, double div, float* E) {
  const double a = std::log10(lo), b = std::log10(hi);
  for (int k = 0; k <= nb; ++k) E[k] = (float)(std::pow(10.0, a + (b - a) * k / nb) / div);
}

static bool good_range(double lo, double hi) {
  return std::isfinite(lo) && std::isfinite(hi) && lo > 0.0 && hi > lo;
}

int aton_ionisation_stats(aton_handle h, const aton_stats_params* p, aton_stats* s,
                          uint64_t* hist_y, uint64_t* hist_J, uint64_t* bin_count,
                          double* bin_mean_y, double* bin_mean_J21) {
  if (int rc = check_h(h)) return rc;
  if (!p || !s) return fail(ATON_ERR_BADARG, "params or stats is NULL");
  if (!h->fields_set) return fail(ATON_ERR_STATE, "aton_set_fields has not been called");
  const int MB = kStatsMaxBins;
  if (p->nb_nH < 1 || p->nb_nH > MB || p->nb_y < 1 || p->nb_y > MB || p->nb_J < 1 || p->nb_J > MB)
    return fail(ATON_ERR_BADARG, "bins must be 1..%d", MB);
  if (!good_range(p->nH_lo, p->nH_hi) || !good_range(p->y_lo, p->y_hi) ||
      !good_range(p->J21_lo, p->J21_hi))
    return fail(ATON_ERR_BADARG, "a bin range has lo <= 0 or hi <= lo");
  if (!(p->spectral_index > -3.0) || !std::isfinite(p->spectral_index))
    return fail(ATON_ERR_BADARG, "spectral_index must be finite and > -3");
  const size_t n_u64 = 2 * (size_t)MB * MB + MB + 1;
  const size_t n_out = kStatsScalars + 2 * MB;
  if (!h->st_edges || !h->st_part || !h->st_out || !h->st_u64) {
    // (all four or none: a call after a failed allocation starts over)
    cudaFree(h->st_edges); cudaFree(h->st_part); cudaFree(h->st_out); cudaFree(h->st_u64);
    h->st_edges = nullptr; h->st_part = nullptr; h->st_out = nullptr; h->st_u64 = nullptr;
    CU(cudaMalloc(&h->st_edges, sizeof(float) * 3 * (MB + 1)));
    CU(cudaMalloc(&h->st_part, sizeof(double) * kStatsBlocks * (kStatsScalars + 2 * MB)));
    CU(cudaMalloc(&h->st_out, sizeof(double) * n_out));
    CU(cudaMalloc(&h->st_u64, sizeof(unsigned long long) * n_u64));
  }
  // J21 = kJ N: Gamma = c sigma_n N and Gamma per J21 from the reading
  const double kJ = h->c * h->prm.sigma_n / gamma_per_J21(p->spectral_index);
  std::vector<float> E(3 * (MB + 1), 0.f);
  log_edges(p->nH_lo, p->nH_hi, p->nb_nH, 1.0, &E[0]);
  log_edges(p->y_lo, p->y_hi, p->nb_y, 1.0, &E[MB + 1]);
  log_edges(p->J21_lo, p->J21_hi, p->nb_J, kJ, &E[2 * (MB + 1)]);
  cudaStream_t st = h->stream();
  CU(cudaMemcpyAsync(h->st_edges, E.data(), sizeof(float) * E.size(), cudaMemcpyHostToDevice, st));
  CU(cudaMemsetAsync(h->st_u64, 0, sizeof(unsigned long long) * n_u64, st));
  StatsArgs a{};
  a.N = h->f[h->cur][0];
  a.y = h->y;
  a.T = h->T;
  a.nH = h->nH;
  a.ncell = h->ncell;
  a.nb_n = p->nb_nH; a.nb_y = p->nb_y; a.nb_J = p->nb_J;
  a.edges = h->st_edges;
  const double lo[3] = {p->nH_lo, p->y_lo, p->J21_lo / kJ};
  const double hi[3] = {p->nH_hi, p->y_hi, p->J21_hi / kJ};
  const int nb[3] = {p->nb_nH, p->nb_y, p->nb_J};
  for (int q = 0; q < 3; ++q) {
    a.g[2 * q] = (float)std::log2(lo[q]);
    a.g[2 * q + 1] = (float)(nb[q] / std::log2(hi[q] / lo[q]));
  }
  a.n_plateau = (float)p->nH_plateau;
  a.part_scalar = h->st_part;
  a.part_bins = h->st_part + (size_t)kStatsBlocks * kStatsScalars;
  a.hist_y = h->st_u64;
  a.hist_J = h->st_u64 + (size_t)MB * MB;
  a.bin_count = h->st_u64 + 2 * (size_t)MB * MB;
  a.plateau_count = h->st_u64 + 2 * (size_t)MB * MB + MB;
  CU(launch_stats(a, h->st_out, st));
  std::vector<double> out(n_out);
  std::vector<unsigned long long> u(n_u64);
  CU(cudaMemcpyAsync(out.data(), h->st_out, sizeof(double) * n_out, cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(u.data(), h->st_u64, sizeof(unsigned long long) * n_u64,
                     cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  const double n = (double)h->ncell;
  const double sy = out[0], sn = out[1], sny = out[2], sN = out[3], sT = out[4], snT = out[5],
               sNp = out[6];
  const unsigned long long cp = u[2 * (size_t)MB * MB + MB];
  s->x_volume = 1.0 - sy / n;
  s->x_mass = 1.0 - sny / sn;
  s->gamma12_volume = h->c * h->prm.sigma_n * sN / n / 1e-12;
  s->J21_volume = kJ * sN / n;
  s->J21_plateau = cp ? kJ * sNp / (double)cp : 0.0;
  s->T_volume = sT / n;
  s->T_mass = snT / sn;
  s->photons = sN * h->V;
  s->cells = h->ncell;
  s->plateau_cells = (int64_t)cp;
  for (int b = 0; b < p->nb_nH; ++b) {
    if (hist_y)
      for (int k = 0; k < p->nb_y; ++k) hist_y[b * p->nb_y + k] = u[b * p->nb_y + k];
    if (hist_J)
      for (int k = 0; k < p->nb_J; ++k) hist_J[b * p->nb_J + k] = u[(size_t)MB * MB + b * p->nb_J + k];
    const unsigned long long c = u[2 * (size_t)MB * MB + b];
    if (bin_count) bin_count[b] = c;
    const double* bs = out.data() + kStatsScalars + 2 * b;
    if (bin_mean_y) bin_mean_y[b] = c ? bs[0] / (double)c : 0.0;
    if (bin_mean_J21) bin_mean_J21[b] = c ? kJ * bs[1] / (double)c : 0.0;
  }
  return ATON_OK;
}

// case-B recombination rate, Hui & Gnedin (1997), FP64 (host)
static double alpha_B_host(double T) {
  const double lam = 2.0 * 157807.0 / T;
  return 2.753e-14 * std::pow(lam, 1.5) / std::pow(1.0 + std::pow(lam / 2.740, 0.407), 2.242);
}

int aton_equilibrium_neutral_fraction(const double* nH, int n, double J21_0, double n_star,
                                      int power, double T, double spectral_index,
                                      double* y_out) {
  if ((!nH || !y_out) && n > 0) return fail(ATON_ERR_BADARG, "NULL array");
  if (n < 0) return fail(ATON_ERR_BADARG, "n < 0");
  if (!(J21_0 >= 0.0) || !(T > 0.0)) return fail(ATON_ERR_BADARG, "J21_0 < 0 or T <= 0");
  if (power != 0 && power != 1 && power != 4) return fail(ATON_ERR_BADARG, "power must be 0, 1 or 4");
  if (power > 0 && !(n_star > 0.0)) return fail(ATON_ERR_BADARG, "n_star <= 0");
  if (!(spectral_index > -3.0)) return fail(ATON_ERR_BADARG, "spectral_index <= -3");
  const double G0 = J21_0 * gamma_per_J21(spectral_index);
  const double al = alpha_B_host(T);
  for (int i = 0; i < n; ++i) {
    const double G = power == 0 ? G0 : G0 * std::exp(-std::pow(nH[i] / n_star, power));
    const double a = al * nH[i];
    if (!(G > 0.0)) {
      y_out[i] = 1.0;
      continue;
    }
    const double q = G + std::sqrt(G * G + 4.0 * a * G);
    y_out[i] = 4.0 * a * G / (q * q);   // a x^2 / G with x = 2G / q
  }
  return ATON_OK;
}

const char* aton_strerror(int code) {
  switch (code) {
    case ATON_OK: return "ok";
    case ATON_ERR_BADARG: return "invalid argument";
    case ATON_ERR_NOMEM: return "out of memory";
    case ATON_ERR_CUDA: return "CUDA error";
    case ATON_ERR_SUBCYCLE: return "chemistry sub-cycle cap reached in some cells";
    case ATON_ERR_NONFINITE: return "non-finite or out-of-range field values";
    case ATON_ERR_STATE: return "call out of order";
    default: return "unknown status";
  }
}

const char* aton_last_message(void) { return g_msg.c_str(); }

void aton_finalize(aton_handle h) {
  if (!h) return;
  int prev = -1;   // the caller's current device, made current again at the end
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  cudaSetDevice(h->device);
  if (h->stream()) cudaStreamSynchronize(h->stream());
  drop_graphs(h);
  for (int b = 0; b < 2; ++b)
    for (int q = 0; q < 4; ++q) cudaFree(h->f[b][q]);
  cudaFree(h->y); cudaFree(h->T); cudaFree(h->nH);
  cudaFree(h->d_part); cudaFree(h->d_out); cudaFree(h->d_u64); cudaFree(h->d_bad);
  free_slots(h->slots);
  cudaFree(h->d_srcbuf);
  cudaFree(h->sur_list); cudaFree(h->sur_count);
  cudaFree(h->sur_buf); cudaFree(h->sur_cnt);
  cudaFree(h->st_edges); cudaFree(h->st_part); cudaFree(h->st_out); cudaFree(h->st_u64);
  if (h->bud_pin) cudaFreeHost(h->bud_pin);
  for (int b = 0; b < 2; ++b) {
    if (h->src_ev[b]) cudaEventSynchronize(h->src_ev[b]);
    if (h->src_pin[b]) cudaFreeHost(h->src_pin[b]);
    if (h->src_ev[b]) cudaEventDestroy(h->src_ev[b]);
  }
  if (h->bud_ev) cudaEventDestroy(h->bud_ev);
  if (h->own) cudaStreamDestroy(h->own);
  delete h;
  if (prev >= 0) cudaSetDevice(prev);
}

int aton_init(int nx, int ny, int nz, double dx_cm, double c_cms, double dt_s, aton_handle* out) {
  if (!out) return fail(ATON_ERR_BADARG, "out is NULL");
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1) return fail(ATON_ERR_BADARG, "grid sizes must be >= 1");
  const int64_t ncell = (int64_t)nx * ny * nz;
  if (ncell > 2147483647LL) return fail(ATON_ERR_BADARG, "more than 2^31-1 cells");
  if (!(dx_cm > 0) || !(c_cms > 0) || !(dt_s > 0) || !std::isfinite(dx_cm) ||
      !std::isfinite(c_cms) || !std::isfinite(dt_s))
    return fail(ATON_ERR_BADARG, "dx, c and dt must be positive and finite");
  const double cfl = 3.0 * c_cms * dt_s / dx_cm;
  if (cfl > 1.0 + 1e-12)
    return fail(ATON_ERR_BADARG, "3 c dt / dx = %.6g exceeds 1 (unsplit 3-D Lax-Friedrichs limit)", cfl);
  aton_ctx* h = new aton_ctx();
  h->nx = nx; h->ny = ny; h->nz = nz; h->ncell = ncell;
  h->dx = dx_cm; h->c = c_cms; h->dt = dt_s; h->V = dx_cm * dx_cm * dx_cm;
  aton_default_params(&h->prm);
  h->quiet_k = quiet_bound(h->prm.T_floor);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    delete h;
    return fail(ATON_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  }
  h->device = dev;
  // kernel attributes are per device: set them the first time a handle is made on this device
  // (several host threads may create handles on different devices at once)
  if (dev < 0 || dev >= kMaxDevices) {
    delete h;
    return fail(ATON_ERR_BADARG, "device index %d out of range", dev);
  }
  {
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    if (!g_attr_done[dev]) {
      e = init_kernel_attributes();
      if (e == cudaSuccess) e = init_tma_attributes();
      if (e == cudaSuccess) e = init_stats_attributes();
      if (e != cudaSuccess) {
        delete h;
        return fail(ATON_ERR_CUDA, "kernel attributes: %s", cudaGetErrorString(e));
      }
      g_attr_done[dev] = true;
    }
  }
  auto bail = [&](int rc) { aton_finalize(h); return rc; };
  if (cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking) != cudaSuccess)
    return bail(fail(ATON_ERR_CUDA, "cudaStreamCreate failed"));
  // Failure injection on the host for tests: ATON_TEST_FAIL_ALLOC=k makes the k-th device
  // allocation below (counting from 0) report cudaErrorMemoryAllocation without allocating, so
  // the clean-up of a partly built handle can be checked without exhausting the device.
  const char* fa = std::getenv("ATON_TEST_FAIL_ALLOC");
  const int fail_at = fa ? std::atoi(fa) : -1;
  int nalloc = 0;
  auto dalloc = [&](void** p, size_t bytes) {
    if (nalloc++ == fail_at) {
      *p = nullptr;
      return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
  };
  const size_t fb = sizeof(float) * (size_t)ncell;
  for (int b = 0; b < 2; ++b)
    for (int q = 0; q < 4; ++q)
      if (dalloc((void**)&h->f[b][q], fb) != cudaSuccess)
        return bail(fail(ATON_ERR_NOMEM, "cudaMalloc of %zu bytes failed", fb));
  if (dalloc((void**)&h->y, fb) != cudaSuccess || dalloc((void**)&h->T, fb) != cudaSuccess ||
      dalloc((void**)&h->nH, fb) != cudaSuccess)
    return bail(fail(ATON_ERR_NOMEM, "cudaMalloc of %zu bytes failed", fb));
  if (dalloc((void**)&h->d_part, sizeof(double) * kSumBlocks) != cudaSuccess ||
      dalloc((void**)&h->d_out, sizeof(double) * 4) != cudaSuccess ||
      dalloc((void**)&h->d_u64, sizeof(unsigned long long) * 5) != cudaSuccess ||
      dalloc((void**)&h->d_bad, sizeof(unsigned int)) != cudaSuccess)
    return bail(fail(ATON_ERR_NOMEM, "cudaMalloc of reduction scratch failed"));
  h->tz = std::min(64, nz);
  // TMA maps of the fields (row pitch must be a multiple of 16 bytes: nx % 4 == 0)
  {
    const int tys[3] = {4, 8, 16};
    for (int i = 0; i < 3; ++i) h->tma_ok[i] = make_tma_maps(nx, ny, nz, tys[i], h->f, &h->tma[i]);
  }
  *out = h;
  return ATON_OK;
}

int aton_set_params(aton_handle h, const aton_params* p) {
  if (int rc = check_h(h)) return rc;
  if (!p) return fail(ATON_ERR_BADARG, "params is NULL");
  if (!(p->sigma_n > 0) || !(p->sigma_e >= 0) || !(p->e_gamma_eV >= 0))
    return fail(ATON_ERR_BADARG, "cross-sections / photon energy out of range");
  if (p->bc != ATON_BC_PERIODIC && p->bc != ATON_BC_TRANSMISSIVE)
    return fail(ATON_ERR_BADARG, "bc must be ATON_BC_PERIODIC or ATON_BC_TRANSMISSIVE");
  if (p->max_sub < 1) return fail(ATON_ERR_BADARG, "max_sub must be >= 1");
  if (!(p->T_floor > 0) || !(p->sub_eps > 0 && p->sub_eps <= 1) || !(p->y_floor > 0))
    return fail(ATON_ERR_BADARG, "T_floor, sub_eps or y_floor out of range");
  if (!(p->clump_R_A >= 0) || !(p->clump_I_A >= 0) || !std::isfinite(p->clump_R_b) ||
      !std::isfinite(p->clump_I_b))
    return fail(ATON_ERR_BADARG, "clumping parameters out of range");
  if (p->flux != ATON_FLUX_GLF && p->flux != ATON_FLUX_HLL)
    return fail(ATON_ERR_BADARG, "flux must be ATON_FLUX_GLF or ATON_FLUX_HLL");
  h->prm = *p;
  h->quiet_k = quiet_bound(p->T_floor);
  drop_graphs(h);  // parameters are baked into captured launches
  return ATON_OK;
}

int aton_get_params(aton_handle h, aton_params* p) {
  if (int rc = check_h(h)) return rc;
  if (!p) return fail(ATON_ERR_BADARG, "params is NULL");
  *p = h->prm;
  return ATON_OK;
}

int aton_set_stream(aton_handle h, void* stream) {
  if (int rc = check_h(h)) return rc;
  CU(cudaStreamSynchronize(h->stream()));
  h->user = (cudaStream_t)stream;
  return ATON_OK;
}

int aton_set_exec(aton_handle h, int mode, int graph_batch) {
  if (int rc = check_h(h)) return rc;
  if (mode != ATON_MODE_FUSED && mode != ATON_MODE_UNFUSED && mode != ATON_MODE_FUSED_LDG)
    return fail(ATON_ERR_BADARG, "mode must be ATON_MODE_FUSED, _UNFUSED or _FUSED_LDG");
  if (graph_batch < 0) return fail(ATON_ERR_BADARG, "graph_batch must be >= 0");
  if (mode != h->mode) {
    if (int rc = fold_slots(h)) return rc;
  }
  h->mode = mode;
  h->graph_batch = graph_batch;
  drop_graphs(h);
  return ATON_OK;
}

int aton_get_exec(aton_handle h, int* mode, int* graph_batch, int* ty, int* tz) {
  if (int rc = check_h(h)) return rc;
  if (mode) *mode = h->mode;
  if (graph_batch) *graph_batch = h->graph_batch;
  if (ty) *ty = h->ty;
  if (tz) *tz = h->tz;
  return ATON_OK;
}

int aton_set_tile(aton_handle h, int ty, int tz) {
  if (int rc = check_h(h)) return rc;
  if (ty != 4 && ty != 8 && ty != 16) return fail(ATON_ERR_BADARG, "ty must be 4, 8 or 16");
  if (tz < 1) return fail(ATON_ERR_BADARG, "tz must be >= 1");
  tz = std::min(tz, h->nz);
  if (ty == h->ty && tz == h->tz) return ATON_OK;
  if (int rc = fold_slots(h)) return rc;
  h->ty = ty;
  h->tz = tz;
  h->tiles_dirty = true;
  drop_graphs(h);
  return ATON_OK;
}

int aton_set_tile_rows(aton_handle h, int rows) {
  if (int rc = check_h(h)) return rc;
  if (rows != 1 && rows != 2) return fail(ATON_ERR_BADARG, "rows per thread must be 1 or 2");
  if (rows == h->rpt) return ATON_OK;
  h->rpt = rows;
  drop_graphs(h);
  return ATON_OK;
}

int aton_get_tile_rows(aton_handle h, int* rows) {
  if (int rc = check_h(h)) return rc;
  if (!rows) return fail(ATON_ERR_BADARG, "NULL rows");
  *rows = h->rpt;
  return ATON_OK;
}

int aton_set_fields(aton_handle h, const float* N, const float* Fx, const float* Fy,
                    const float* Fz, const float* x, const float* y, const float* T,
                    const float* nH, int where) {
  if (int rc = check_h(h)) return rc;
  if (!N || !Fx || !Fy || !Fz || !T || !nH) return fail(ATON_ERR_BADARG, "NULL field pointer");
  if ((x == nullptr) == (y == nullptr)) return fail(ATON_ERR_BADARG, "give exactly one of x, y");
  if (where != ATON_HOST && where != ATON_DEVICE) return fail(ATON_ERR_BADARG, "bad where");
  cudaStream_t s = h->stream();
  const cudaMemcpyKind k = where == ATON_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const size_t fb = sizeof(float) * (size_t)h->ncell;
  h->fields_set = false;
  float** d = h->f[h->cur];
  CU(cudaMemcpyAsync(d[0], N, fb, k, s));
  CU(cudaMemcpyAsync(d[1], Fx, fb, k, s));
  CU(cudaMemcpyAsync(d[2], Fy, fb, k, s));
  CU(cudaMemcpyAsync(d[3], Fz, fb, k, s));
  CU(cudaMemcpyAsync(h->y, x ? x : y, fb, k, s));
  CU(cudaMemcpyAsync(h->T, T, fb, k, s));
  CU(cudaMemcpyAsync(h->nH, nH, fb, k, s));
  if (x) CU(launch_one_minus(h->y, h->y, h->ncell, s));
  CU(cudaMemsetAsync(h->d_bad, 0, sizeof(unsigned int), s));
  CU(launch_validate(d[0], h->y, h->T, h->nH, h->ncell, h->d_bad, s));
  unsigned int bad = 0;
  CU(cudaMemcpyAsync(&bad, h->d_bad, sizeof(bad), cudaMemcpyDeviceToHost, s));
  CU(launch_sum_field(d[0], h->ncell, h->d_part, h->d_out + 3, s));
  double st = 0;
  CU(cudaMemcpyAsync(&st, h->d_out + 3, sizeof(st), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  if (bad) return fail(ATON_ERR_NONFINITE, "%u cells have non-finite or out-of-range values", bad);
  // reset tallies
  if (h->slots.n) {
    if (int rc = fold_slots(h)) return rc;
  }
  std::memset(h->fold_acc, 0, sizeof(h->fold_acc));
  std::memset(h->fold_u, 0, sizeof(h->fold_u));
  h->sink_steps = 0;
  std::memset(h->offs, 0, sizeof(h->offs));
  h->emitted = 0;
  h->steps = 0;
  h->stored0 = st * h->V;
  h->latched = ATON_OK;
  h->fields_set = true;
  return ATON_OK;
}

int aton_get_fields(aton_handle h, float* N, float* Fx, float* Fy, float* Fz, float* x, float* y,
                    float* T, int where) {
  if (int rc = check_h(h)) return rc;
  if (where != ATON_HOST && where != ATON_DEVICE) return fail(ATON_ERR_BADARG, "bad where");
  if (!h->fields_set) return fail(ATON_ERR_STATE, "aton_set_fields has not been called");
  cudaStream_t s = h->stream();
  const cudaMemcpyKind k = where == ATON_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  const size_t fb = sizeof(float) * (size_t)h->ncell;
  float** d = h->f[h->cur];
  float* scratch = h->f[1 - h->cur][0];  // the spare buffer is dead between steps
  if (N) CU(cudaMemcpyAsync(N, d[0], fb, k, s));
  float* outs[3] = {Fx, Fy, Fz};
  for (int q = 0; q < 3; ++q)
    if (outs[q]) CU(cudaMemcpyAsync(outs[q], d[q + 1], fb, k, s));
  if (y) CU(cudaMemcpyAsync(y, h->y, fb, k, s));
  if (x) {
    CU(launch_one_minus(scratch, h->y, h->ncell, s));
    CU(cudaMemcpyAsync(x, scratch, fb, k, s));
  }
  if (T) CU(cudaMemcpyAsync(T, h->T, fb, k, s));
  CU(cudaStreamSynchronize(s));
  return ATON_OK;
}

int aton_add_sources(aton_handle h, const int64_t* cell_idx, const double* rate, int64_t n, int mode) {
  if (int rc = check_h(h)) return rc;
  if (n < 0) return fail(ATON_ERR_BADARG, "n < 0");
  if (n > 0 && (!cell_idx || !rate)) return fail(ATON_ERR_BADARG, "NULL source arrays");
  if (mode != ATON_SRC_REPLACE && mode != ATON_SRC_APPEND) return fail(ATON_ERR_BADARG, "bad mode");
  for (int64_t i = 0; i < n; ++i) {
    if (cell_idx[i] < 0 || cell_idx[i] >= h->ncell)
      return fail(ATON_ERR_BADARG, "source %lld: cell index %lld out of range", (long long)i,
                  (long long)cell_idx[i]);
    if (!(rate[i] >= 0) || !std::isfinite(rate[i]))
      return fail(ATON_ERR_BADARG, "source %lld: rate must be finite and >= 0", (long long)i);
  }
  // merged list sorted by cell; a cell listed more than once (or already present, when
  // appending) gets its rates summed in the order given
  std::vector<std::pair<int64_t, double>> all;
  all.reserve((mode == ATON_SRC_APPEND ? h->src.size() : 0) + (size_t)n);
  if (mode == ATON_SRC_APPEND) all = h->src;
  for (int64_t i = 0; i < n; ++i) all.emplace_back(cell_idx[i], rate[i]);
  std::stable_sort(all.begin(), all.end(),
                   [](const auto& a, const auto& b) { return a.first < b.first; });
  h->src.clear();
  for (const auto& e : all) {
    if (!h->src.empty() && h->src.back().first == e.first) h->src.back().second += e.second;
    else h->src.push_back(e);
  }
  return upload_sources(h);
}

int aton_step(aton_handle h, int nsteps) {
  if (int rc = check_h(h)) return rc;
  if (nsteps < 0) return fail(ATON_ERR_BADARG, "nsteps < 0");
  if (h->latched != ATON_OK) return h->latched;
  if (int rc = prepare(h)) return rc;
  cudaStream_t s = h->stream();
  int left = nsteps;
  while (left > 0) {
    const bool graphs = h->graph_batch > 0 && h->sink == nullptr;
    const int b = graphs ? std::min(left, h->graph_batch) : 1;
    if (graphs) {
      auto key = std::make_pair(b, h->cur);
      auto it = h->graphs.find(key);
      if (it == h->graphs.end()) {
        const int cur0 = h->cur;
        CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        int rc = ATON_OK;
        for (int i = 0; i < b && rc == ATON_OK; ++i) rc = enqueue_step(h, s);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(s, &g);
        h->cur = cur0;
        if (rc) { if (g) cudaGraphDestroy(g); return rc; }
        if (e != cudaSuccess) return fail(ATON_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        cudaGraphExec_t ge = nullptr;
        e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(ATON_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
        it = h->graphs.emplace(key, ge).first;
      }
      CU(cudaGraphLaunch(it->second, s));
      if (b & 1) h->cur = 1 - h->cur;
    } else {
      if (int rc = enqueue_step(h, s)) return rc;
    }
    h->steps += b;
    h->emitted += h->emit_per_step * b;
    left -= b;
  }
  return ATON_OK;
}

static int read_tallies(aton_handle h, double acc[3], unsigned long long u[5], double* stored) {
  cudaStream_t s = h->stream();
  double a[4] = {0, 0, 0, 0};
  unsigned long long uu[5] = {0, 0, 0, 0, 0};
  if (h->slots.n) {
    CU(launch_reduce_slots(h->slots, h->d_out, h->d_u64, s));
  }
  if (stored) CU(launch_sum_field(h->f[h->cur][0], h->ncell, h->d_part, h->d_out + 3, s));
  CU(cudaMemcpyAsync(a, h->d_out, sizeof(a), cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(uu, h->d_u64, sizeof(uu), cudaMemcpyDeviceToHost, s));
  unsigned int tmo = 0;
  if (h->slots.timeout) CU(cudaMemcpyAsync(&tmo, h->slots.timeout, sizeof(tmo), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  if (tmo) {
    h->latched = ATON_ERR_CUDA;
    return fail(ATON_ERR_CUDA, "%u CTAs gave up waiting on a pipeline barrier", tmo);
  }
  if (!h->slots.n) { a[0] = a[1] = a[2] = 0; uu[0] = uu[1] = uu[2] = uu[3] = uu[4] = 0; }
  for (int i = 0; i < 3; ++i) acc[i] = h->fold_acc[i] + a[i];
  u[0] = h->fold_u[0] + uu[0];
  u[1] = std::max(h->fold_u[1], uu[1]);
  u[2] = h->fold_u[2] + uu[2];
  u[3] = h->fold_u[3] + uu[3];
  u[4] = h->fold_u[4] + uu[4];
  if (stored) *stored = a[3];
  if (u[3]) h->latched = ATON_ERR_NONFINITE;
  else if (u[2]) h->latched = ATON_ERR_SUBCYCLE;
  return ATON_OK;
}

int aton_synchronize(aton_handle h) {
  if (int rc = check_h(h)) return rc;
  CU(cudaStreamSynchronize(h->stream()));
  if (!h->fields_set) return ATON_OK;
  double acc[3];
  unsigned long long u[5];
  if (int rc = read_tallies(h, acc, u, nullptr)) return rc;
  return h->latched;
}

int aton_photon_budget(aton_handle h, double* out) {
  if (int rc = check_h(h)) return rc;
  if (!out) return fail(ATON_ERR_BADARG, "out is NULL");
  if (!h->fields_set) return fail(ATON_ERR_STATE, "aton_set_fields has not been called");
  double acc[3], st = 0;
  unsigned long long u[5];
  if (int rc = read_tallies(h, acc, u, &st)) return rc;
  out[ATON_B_EMITTED] = h->emitted + h->offs[ATON_B_EMITTED];
  out[ATON_B_STORED] = st * h->V;
  out[ATON_B_ABSORBED] = acc[0] * h->V + h->offs[ATON_B_ABSORBED];
  out[ATON_B_ESCAPED] = acc[1] * h->V + h->offs[ATON_B_ESCAPED];
  out[ATON_B_CLIPPED] = acc[2] * h->V + h->offs[ATON_B_CLIPPED];
  out[ATON_B_STORED0] = h->stored0 + h->offs[ATON_B_STORED0];
  return ATON_OK;
}

int aton_budget_request(aton_handle h) {
  if (int rc = check_h(h)) return rc;
  if (!h->fields_set) return fail(ATON_ERR_STATE, "aton_set_fields has not been called");
  if (!h->bud_pin) {
    CU(cudaMallocHost(&h->bud_pin, sizeof(double) * 5));
    CU(cudaEventCreateWithFlags(&h->bud_ev, cudaEventDisableTiming));
  }
  // a request not collected is replaced: its copy must land before the buffer is reused
  if (h->bud_pending) CU(cudaEventSynchronize(h->bud_ev));
  cudaStream_t s = h->stream();
  if (h->slots.n) {
    CU(launch_reduce_slots(h->slots, h->d_out, h->d_u64, s));
  } else {
    CU(cudaMemsetAsync(h->d_out, 0, sizeof(double) * 3, s));
  }
  CU(launch_sum_field(h->f[h->cur][0], h->ncell, h->d_part, h->d_out + 3, s));
  CU(cudaMemcpyAsync(h->bud_pin, h->d_out, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
  h->bud_pin[4] = 0.0;
  if (h->slots.timeout) {
    CU(cudaMemcpyAsync(reinterpret_cast<unsigned int*>(h->bud_pin + 4), h->slots.timeout,
                       sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
  }
  CU(cudaEventRecord(h->bud_ev, s));
  for (int i = 0; i < 3; ++i) h->bud_fold[i] = h->fold_acc[i];
  h->bud_emitted = h->emitted;
  h->bud_stored0 = h->stored0;
  std::memcpy(h->bud_offs, h->offs, sizeof(h->offs));
  h->bud_pending = true;
  return ATON_OK;
}

int aton_budget_collect(aton_handle h, double* out) {
  if (int rc = check_h(h)) return rc;
  if (!out) return fail(ATON_ERR_BADARG, "out is NULL");
  if (!h->bud_pending) return fail(ATON_ERR_STATE, "no budget request is outstanding");
  h->bud_pending = false;
  CU(cudaEventSynchronize(h->bud_ev));
  unsigned int tmo = 0;
  std::memcpy(&tmo, h->bud_pin + 4, sizeof(tmo));
  if (tmo) {
    h->latched = ATON_ERR_CUDA;
    return fail(ATON_ERR_CUDA, "%u CTAs gave up waiting on a pipeline barrier", tmo);
  }
  const double* a = h->bud_pin;
  out[ATON_B_EMITTED] = h->bud_emitted + h->bud_offs[ATON_B_EMITTED];
  out[ATON_B_STORED] = a[3] * h->V;
  out[ATON_B_ABSORBED] = (h->bud_fold[0] + a[0]) * h->V + h->bud_offs[ATON_B_ABSORBED];
  out[ATON_B_ESCAPED] = (h->bud_fold[1] + a[1]) * h->V + h->bud_offs[ATON_B_ESCAPED];
  out[ATON_B_CLIPPED] = (h->bud_fold[2] + a[2]) * h->V + h->bud_offs[ATON_B_CLIPPED];
  out[ATON_B_STORED0] = h->bud_stored0 + h->bud_offs[ATON_B_STORED0];
  return ATON_OK;
}

int aton_set_budget(aton_handle h, const double* in) {
  if (int rc = check_h(h)) return rc;
  if (!in) return fail(ATON_ERR_BADARG, "in is NULL");
  if (!h->fields_set) return fail(ATON_ERR_STATE, "aton_set_fields has not been called");
  double cur[ATON_BUDGET_LEN];
  if (int rc = aton_photon_budget(h, cur)) return rc;
  for (int i = 0; i < ATON_BUDGET_LEN; ++i)
    if (i != ATON_B_STORED) h->offs[i] += in[i] - cur[i];
  return ATON_OK;
}

int aton_get_diag(aton_handle h, aton_diag* out) {
  if (int rc = check_h(h)) return rc;
  if (!out) return fail(ATON_ERR_BADARG, "out is NULL");
  if (!h->fields_set) return fail(ATON_ERR_STATE, "aton_set_fields has not been called");
  double acc[3];
  unsigned long long u[5];
  if (int rc = read_tallies(h, acc, u, nullptr)) return rc;
  out->steps = h->steps;
  out->surrogate_cells = (int64_t)u[4];
  out->substeps_total = (int64_t)u[0];
  out->substeps_max = (int64_t)u[1];
  out->error_cells = (int64_t)u[2];
  out->nonfinite_cells = (int64_t)u[3];
  // largest reduced flux of the current state (a reduction over N, F on demand)
  cudaStream_t s = h->stream();
  CU(cudaMemsetAsync(h->d_bad, 0, sizeof(unsigned int), s));
  CU(launch_max_f2(h->f[h->cur][0], h->f[h->cur][1], h->f[h->cur][2], h->f[h->cur][3],
                   (float)(1.0 / h->c), h->ncell, h->d_bad, s));
  unsigned int bits = 0;
  CU(cudaMemcpyAsync(&bits, h->d_bad, sizeof(bits), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  float f2;
  std::memcpy(&f2, &bits, sizeof(f2));
  out->max_f = std::sqrt((double)f2);
  return ATON_OK;
}

int aton_last_error_cells(aton_handle h, int64_t* count) {
  if (int rc = check_h(h)) return rc;
  if (!count) return fail(ATON_ERR_BADARG, "count is NULL");
  aton_diag d;
  if (int rc = aton_get_diag(h, &d)) return rc;
  *count = d.error_cells + d.nonfinite_cells;
  return ATON_OK;
}

int aton_launches_per_step(aton_handle h, int* launches) {
  if (int rc = check_h(h)) return rc;
  if (!launches) return fail(ATON_ERR_BADARG, "launches is NULL");
  const bool fused = (h->mode == ATON_MODE_FUSED || h->mode == ATON_MODE_FUSED_LDG) && !plain_only(h);
  if (fused) {
    *launches = 1;   // (with the surrogate the fused kernel runs the network itself)
  } else {
    *launches = h->src_n > 0 ? plain_launches() : plain_launches() - 1;
    if (sur_on(h)) *launches += 1;   // the candidate pass (plus a counter reset)
  }
  return ATON_OK;
}

int aton_set_pair_sink(aton_handle h, float* records, int64_t capacity, int stride) {
  if (int rc = check_h(h)) return rc;
  if (records && (capacity < 1 || stride < 1))
    return fail(ATON_ERR_BADARG, "capacity and stride must be >= 1");
  h->sink = records;
  h->sink_cap = records ? capacity : 0;
  h->sink_stride = records ? stride : 1;
  h->sink_steps = 0;
  drop_graphs(h);
  return ATON_OK;
}

int aton_pair_count(aton_handle h, int64_t* count) {
  if (int rc = check_h(h)) return rc;
  if (!count) return fail(ATON_ERR_BADARG, "count is NULL");
  const long long per = (h->ncell + h->sink_stride - 1) / h->sink_stride;
  *count = h->sink ? std::min<long long>(h->sink_steps * per, h->sink_cap) : 0;
  return ATON_OK;
}

void aton_default_surrogate_params(aton_surrogate_params* p) {
  if (!p) return;
  p->enabled = 1;
  p->gate_substeps = 8.0;
  p->residual_max = 1e-4;
}

int aton_set_surrogate(aton_handle h, aton_mlp_handle m, const aton_surrogate_params* p) {
  if (int rc = check_h(h)) return rc;
  if (m && !p) return fail(ATON_ERR_BADARG, "params is NULL");
  if (p && (!(p->gate_substeps >= 0) || !(p->residual_max >= 0)))
    return fail(ATON_ERR_BADARG, "gate and residual must be >= 0");
  if (m && p->enabled && !h->sur_list) {
    CU(cudaMalloc(&h->sur_list, sizeof(int) * (size_t)h->ncell));
    CU(cudaMalloc(&h->sur_count, sizeof(int)));
  }
  h->sur = m;
  if (p) h->sur_p = *p;
  else h->sur_p = aton_surrogate_params{};
  drop_graphs(h);
  return ATON_OK;
}

int aton_autotune(aton_handle h, int steps, int* ty_out, int* tz_out, float* ms_out) {
  if (int rc = check_h(h)) return rc;
  if (steps < 1) return fail(ATON_ERR_BADARG, "steps must be >= 1");
  if (!h->fields_set) return fail(ATON_ERR_STATE, "aton_set_fields has not been called");
  cudaStream_t s = h->stream();
  if (int rc = fold_slots(h)) return rc;
  // room for the finest candidate tiling, so trial steps never fold into the real tallies
  if (int rc = ensure_slots_n(h, std::max(fused_tiles(h->nx, h->ny, h->nz, 4, std::min(16, h->nz)),
                                          kPlainBlocks)))
    return rc;
  const size_t fb = sizeof(float) * (size_t)h->ncell;
  // save the state the candidates start from
  std::vector<float*> save(6, nullptr);
  float* src[6] = {h->f[h->cur][0], h->f[h->cur][1], h->f[h->cur][2], h->f[h->cur][3], h->y, h->T};
  for (int q = 0; q < 6; ++q) {
    if (cudaMalloc(&save[q], fb) != cudaSuccess) {
      for (auto p : save) cudaFree(p);
      return fail(ATON_ERR_NOMEM, "autotune scratch allocation failed");
    }
    CU(cudaMemcpyAsync(save[q], src[q], fb, cudaMemcpyDeviceToDevice, s));
  }
  const int mode0 = h->mode, gb0 = h->graph_batch, ty0 = h->ty, tz0 = h->tz, cur0 = h->cur;
  const int rpt0 = h->rpt;
  h->graph_batch = 0;
  int best_ty = ty0, best_tz = tz0;
  float best = 1e30f;
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  const int tys[3] = {4, 8, 16};
  const int tzs[7] = {16, 32, 48, 64, 96, 128, 256};
  struct Cand {
    int mode, ty, tz, rows;
    float ms;
  };
  std::vector<Cand> cands;
  for (int kind = 0; kind < 2; ++kind)
    for (int a = 0; a < 3; ++a)
      for (int rows = 1; rows <= 2; ++rows)
        for (int b = 0; b < 7; ++b) {
          const int tz = std::min(tzs[b], h->nz);
          if (b > 0 && tz == std::min(tzs[b - 1], h->nz)) continue;
          // kind 0: the TMA-staged kernel (when the grid allows it), kind 1: plain loads; two
          // rows per thread with the TMA-staged kernel at tile heights 8 and 16, GLF flux
          if (kind == 0 && !h->tma_ok[ty_index(tys[a])]) continue;
          if (rows == 2 && (kind != 0 || tys[a] < 8 || h->prm.flux == ATON_FLUX_HLL)) continue;
          cands.push_back(Cand{kind == 0 ? ATON_MODE_FUSED : ATON_MODE_FUSED_LDG, tys[a], tz, rows,
                               1e30f});
        }
  // time a candidate over n steps from the saved state (after one untimed step)
  auto time_cand = [&](Cand& c, int n) -> int {
    h->mode = c.mode;
    h->ty = c.ty;
    h->tz = c.tz;
    h->rpt = c.rows;
    h->tiles_dirty = true;
    int rc = prepare(h);
    if (rc) return rc;
    for (int q = 0; q < 6; ++q) {
      float* dst = q < 4 ? h->f[cur0][q] : (q == 4 ? h->y : h->T);
      cudaMemcpyAsync(dst, save[q], fb, cudaMemcpyDeviceToDevice, s);
    }
    h->cur = cur0;
    if ((rc = enqueue_step(h, s))) return rc;  // warm-up
    cudaEventRecord(e0, s);
    for (int i = 0; i < n && rc == ATON_OK; ++i) rc = enqueue_step(h, s);
    cudaEventRecord(e1, s);
    if (rc) return rc;
    if (cudaEventSynchronize(e1) != cudaSuccess) return fail(ATON_ERR_CUDA, "autotune sync");
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    c.ms = ms / n;
    return ATON_OK;
  };
  int rc = ATON_OK;
  for (auto& c : cands)
    if ((rc = time_cand(c, steps))) break;
  // the three fastest again over three times the steps (the short first timing is noisy)
  if (rc == ATON_OK) {
    std::sort(cands.begin(), cands.end(), [](const Cand& x, const Cand& y) { return x.ms < y.ms; });
    const size_t top = std::min<size_t>(3, cands.size());
    for (size_t i = 0; i < top && rc == ATON_OK; ++i) rc = time_cand(cands[i], 3 * steps);
    if (rc == ATON_OK)
      std::sort(cands.begin(), cands.begin() + top,
                [](const Cand& x, const Cand& y) { return x.ms < y.ms; });
  }
  int best_mode = ATON_MODE_FUSED, best_rpt = rpt0;
  if (rc == ATON_OK && !cands.empty()) {
    best = cands[0].ms; best_ty = cands[0].ty; best_tz = cands[0].tz;
    best_mode = cands[0].mode; best_rpt = cands[0].rows;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // restore the state, drop the tallies of the trial steps
  for (int q = 0; q < 6; ++q) {
    float* dst = q < 4 ? h->f[cur0][q] : (q == 4 ? h->y : h->T);
    cudaMemcpyAsync(dst, save[q], fb, cudaMemcpyDeviceToDevice, s);
  }
  cudaStreamSynchronize(s);
  for (auto p : save) cudaFree(p);
  h->cur = cur0;
  if (h->slots.n) {
    cudaStream_t st = s;
    CU(cudaMemsetAsync(h->slots.acc, 0, sizeof(double) * 3 * h->slots.n, st));
    CU(cudaMemsetAsync(h->slots.sub, 0, sizeof(unsigned long long) * h->slots.n, st));
    CU(cudaMemsetAsync(h->slots.mx, 0, sizeof(unsigned int) * h->slots.n, st));
    CU(cudaMemsetAsync(h->slots.err, 0, sizeof(unsigned int) * h->slots.n, st));
    CU(cudaMemsetAsync(h->slots.nan, 0, sizeof(unsigned int) * h->slots.n, st));
  }
  // keep the caller's choice of the unfused path; otherwise take the faster fused kernel
  h->mode = mode0 == ATON_MODE_UNFUSED ? mode0 : best_mode;
  h->graph_batch = gb0;
  h->ty = best_ty;
  h->tz = best_tz;
  h->rpt = best_rpt;
  h->tiles_dirty = true;
  drop_graphs(h);
  if (rc) return rc;
  if (ty_out) *ty_out = best_ty;
  if (tz_out) *tz_out = best_tz;
  if (ms_out) *ms_out = best;
  return ATON_OK;
}

}  // extern "C"
