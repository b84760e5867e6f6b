// aton_tma.cu -- the fused step kernel with TMA-staged planes (sm_103a).
//
// Same step as k_fused (Lax-Friedrichs M1 transport, section 2.2 and Appendix Eqs. A2/A5;
// sources, section 2.3; chemistry operator Phi, Appendix Eq. A4), with the plane loads moved
// to the TMA engine. Thread 0 streams each z-plane of the CTA's 32 x TY column tile into a
// three-deep shared-memory stage ring with cp.async.bulk.tensor: a (32+8) x (TY+2) box of each
// of N, Fx, Fy, Fz (one-cell halo; the x origin is 4 cells left so it stays 16-byte aligned);
// one mbarrier per stage signals the landed bytes. A stage is refilled right after the CTA
// barrier that ends its use, three planes ahead of the next use, so no thread waits on a free
// stage and no warp is spent on producing. The chemistry fields y, T, nH of the own cell are
// loaded one plane ahead into registers. Every thread turns each landed plane into a
// three-plane ring of two vector records per slot, (N, F/c) and the closure pair (iso, w) with
// N D = iso I + w (F/c)(F/c)^T, patching the slots that lie outside the grid from global memory
// (boundary map; edge tiles only) and evaluating the closure once per slot; a neighbour then
// costs two vector loads, the z neighbours included (planes z-1, z, z+1 are all in the ring
// while plane z is updated). The cell update is the same as in k_fused.
//
// Used when nx is a multiple of 4 (the tensor-map row pitch must be a multiple of 16 bytes);
// otherwise the step falls back to k_fused.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "aton_internal.h"
#include "aton_step_common.cuh"

namespace aton {

namespace {

constexpr int kStages = 3;   // planes in flight: a stage is refilled three planes ahead
constexpr int kBoxX = kTileX + 8;          // x0-4 .. x0+35
constexpr unsigned kWaitLimit = 1u << 26;            // polls before a wait is declared failed
constexpr unsigned long long kWaitNs = 2000000000ull;  // or nanoseconds (2 s), whichever first
constexpr unsigned kSuspendNs = 4000;                  // suspend-time hint of one poll

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait on the phase with the given parity. Each poll may suspend the thread until the
// phase completes or kSuspendNs pass (so a waiting warp does not spin on the issue slots).
// Returns false (and the caller raises the error word) if the phase did not complete within
// kWaitLimit polls or kWaitNs nanoseconds.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  const unsigned a = smem_u32(bar);
  unsigned long long t0 = 0;
  for (unsigned i = 0; i < kWaitLimit; ++i) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity), "r"(kSuspendNs)
        : "memory");
    if (done) return true;
    if (i == 0) t0 = global_ns();
    else if (global_ns() - t0 > kWaitNs) return false;
  }
  return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

template <int TY, bool HLL = false>
struct Layout {
  static constexpr int PL = kBoxX * (TY + 2);             // floats per field-plane (with halo)
  static constexpr int PLP = (PL + 31) & ~31;             // padded to 128 bytes
  static constexpr int STAGE = 4 * PLP;                  // floats per stage
  static constexpr int RX = kTileX + 2;                   // ring row pitch (one-cell halo)
  static constexpr int PLR = RX * (TY + 2);               // ring slots per plane
  static constexpr unsigned U_BYTES = 4u * PL * 4u;       // bytes landed per plane (u)
  static constexpr size_t STAGE_BYTES = (size_t)kStages * STAGE * 4;
  // per slot: (N, F/c), the closure pair, and with HLL the x, y, z speed bounds
  static constexpr size_t RING_BYTES = (size_t)3 * PLR * (16 + 8 + (HLL ? 24 : 0));
  static constexpr size_t BYTES = STAGE_BYTES + RING_BYTES + kStages * 8 + 128;
};

}  // namespace

// (no minimum-blocks bound: the compiler's own allocation at TY = 4, 72 registers and seven
// CTAs per SM, is the fastest configuration; a cap at 64 for eight CTAs spilled and ran slower)
// FULL: every tile lies inside the grid (nx a multiple of 32, ny of TY), so every thread owns a
// cell and no own slot needs patching; the bounds tests fold away. HLL: the HLL intercell flux
// instead of global Lax-Friedrichs (the ring then also holds each cell's speed bounds). SUR:
// the chemistry surrogate; a cell the gate selects (off the one-sub-step shortcut) is listed in
// the CTA's region of a device buffer and, after the z-loop, runs through the network (sur_tail),
// the accepted predictions replacing the exact operator. RPT: rows of the tile per thread (the
// CTA has TY / RPT warps; thread row t owns the rows t RPT .. t RPT + RPT - 1), which spreads
// the per-plane work that does not depend on the cell count (the stage wait, the barrier, the
// loop) and the halo rows over more cells. TO: transport only (the first kernel of the plain
// three-kernel step): the transported and clamped (N, F) are stored, without sources or
// chemistry, and y, T, nH are not read.
// Launch bounds: the surrogate instance at tile 32 x 8 with two rows is held to five CTAs per SM,
// like the exact one (its network tail after the z-loop would otherwise raise the register
// count); the others declare no minimum (0): an explicit minimum of one CTA let the compiler
// spend 127 registers on the exact two-row instance, four CTAs per SM, where it takes 94.
template <int TY, bool PER, bool STD, bool FULL, bool HLL = false, bool SUR = false, int RPT = 1,
          bool TO = false>
__global__ void __launch_bounds__(kTileX * TY / RPT, (SUR && RPT == 2 && TY == 8) ? 5 : 0)
    k_fused_tma(const FusedArgs A, const __grid_constant__ TmaMaps M) {
  using L = Layout<TY, HLL>;
  constexpr int TX = kTileX, NH = 2 * TX + 2 * TY, TYT = TY / RPT;
  static_assert(TY % RPT == 0 && TX * TYT >= NH, "one halo slot per thread at most");
  static_assert(!(TO && SUR), "transport only: no chemistry");
  extern __shared__ __align__(128) float sm_raw[];
  // 128-byte aligned base for the TMA boxes, as an offset from the shared array (so every
  // access below stays a shared-memory access)
  float* sm = sm_raw + ((128u - (smem_u32(sm_raw) & 127u)) & 127u) / 4;
  float* stage0 = sm;
  // ring of prepared planes: (N, Fx/c, Fy/c, Fz/c) and the closure pair (iso, w)
  float4* RU = reinterpret_cast<float4*>(sm + kStages * L::STAGE);
  float2* RW = reinterpret_cast<float2*>(RU + 3 * L::PLR);
  // speed bounds (lo, hi) along x, y, z (HLL only; empty otherwise)
  float2* SX = RW + 3 * L::PLR;
  float2* SY = SX + (HLL ? 3 * L::PLR : 0);
  float2* SZ = SY + (HLL ? 3 * L::PLR : 0);
  unsigned long long* full = reinterpret_cast<unsigned long long*>(SZ + (HLL ? 3 * L::PLR : 0));

  const StepParams& P = A.P;
  const int tx = threadIdx.x, tid = tx + TX * threadIdx.y;
  const int nx = P.nx, ny = P.ny, nz = P.nz;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * A.tz;
  const int z1 = min(z0 + A.tz, nz);
  const int nplanes = z1 - z0 + 2;   // planes z0-1 .. z1
  const long long plane = (long long)nx * ny;
  const int tile = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  bool failed = false;
  auto plane_of = [&](int z) {   // z in [-1, nz]
    return z < 0 ? (PER ? nz - 1 : 0) : (z >= nz ? (PER ? 0 : nz - 1) : z);
  };
  // plane index k (plane z0 - 1 + k) into stage k % kStages; issued by thread 0 only
  auto issue = [&](int k) {
    const int s = k % kStages;
    const int p = plane_of(z0 - 1 + k);
    mbar_expect_tx(&full[s], L::U_BYTES);
    float* st = stage0 + s * L::STAGE;
    for (int q = 0; q < 4; ++q)
      tma_load_3d(st + q * L::PLP, &M.u[A.in_buf][q], x0 - 4, y0 - 1, p, &full[s]);
  };
  auto wait = [&](int k) {   // plane k landed (skipped once a wait has failed)
    if (!failed && !mbar_wait(&full[k % kStages], (k / kStages) & 1)) failed = true;
  };

  int issued = 0;   // planes issued so far (thread 0)
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (; issued < kStages && issued < nplanes; ++issued) issue(issued);
  }
  __syncthreads();

  Tally tl;
  const int gx = x0 + tx;
  // the thread's own rows ty = threadIdx.y RPT + r
  bool act[RPT], own_out[RPT];
  int oslot[RPT], orslot[RPT], gy[RPT], ocell[RPT];
  long long ocol[RPT];
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int ty = threadIdx.y * RPT + r;
    gy[r] = y0 + ty;
    act[r] = FULL || (gx < nx && gy[r] < ny);
    own_out[r] = !act[r];   // (false when FULL)
    oslot[r] = (ty + 1) * kBoxX + (tx + 4);       // stage slot
    orslot[r] = (ty + 1) * L::RX + (tx + 1);      // ring slot
    ocell[r] = tx + TX * ty;                      // cell index in the tile (source lists)
    ocol[r] = bc_map(gx, nx, PER) + (long long)nx * bc_map(gy[r], ny, PER);
  }
  // halo slot of this thread (if any) in tile coordinates
  int hx = 0, hy = 0, hslot = -1, hrslot = -1;
  if (tid < NH) {
    if (tid < TX) { hx = tid; hy = -1; }
    else if (tid < 2 * TX) { hx = tid - TX; hy = TY; }
    else if (tid < 2 * TX + TY) { hx = -1; hy = tid - 2 * TX; }
    else { hx = TX; hy = tid - 2 * TX - TY; }
    hslot = (hy + 1) * kBoxX + (hx + 4);
    hrslot = (hy + 1) * L::RX + (hx + 1);
  }
  const bool halo_out = hslot >= 0 && (x0 + hx < 0 || x0 + hx >= nx || y0 + hy < 0 || y0 + hy >= ny);
  const long long hcol = hslot >= 0 ? bc_map(x0 + hx, nx, PER) + (long long)nx * bc_map(y0 + hy, ny, PER) : 0;
  const float rc = P.rc, lam = P.lam;
  const float hl = 0.5f * lam, cu = 1.f - 3.f * lam;
  const float* __restrict__ gN = A.in.N;
  const float* __restrict__ gX = A.in.Fx;
  const float* __restrict__ gY = A.in.Fy;
  const float* __restrict__ gZ = A.in.Fz;

  // (N, F/c) of a slot of stage `st`: patched from global memory (boundary map) when the slot
  // lies outside the grid, read from the TMA box otherwise.
  auto prep = [&](const float* st, int slot, bool out, long long col, int p) {
    float4 u;
    if (out) {
      const long long o = (long long)p * plane + col;
      u = make_float4(__ldg(gN + o), __ldg(gX + o) * rc, __ldg(gY + o) * rc, __ldg(gZ + o) * rc);
    } else {
      u = make_float4(st[slot], st[L::PLP + slot] * rc, st[2 * L::PLP + slot] * rc,
                      st[3 * L::PLP + slot] * rc);
    }
    return u;
  };
  // the prepared own slot into ring plane r; returns the z flux (Fz/c, Dxz, Dyz, Dzz) N
  auto put = [&](int r, int rslot, const float4& u) {
    if (HLL)
      return ring_put_hll<7>(RU + r * L::PLR, RW + r * L::PLR, SX + r * L::PLR, SY + r * L::PLR,
                             SZ + r * L::PLR, rslot, u);
    return ring_put(RU + r * L::PLR, RW + r * L::PLR, rslot, u);
  };
  // the prepared halo slot: with HLL a halo row needs its speeds along y only, a halo column
  // along x only (warps 0 and 1 hold the rows, warp 2 the columns: no divergence)
  const bool hrow = hy < 0 || hy >= TY;
  auto put_halo = [&](int r, const float4& u) {
    if (HLL) {
      float4* U = RU + r * L::PLR;
      float2* W = RW + r * L::PLR;
      if (hrow)
        ring_put_hll<2>(U, W, SX + r * L::PLR, SY + r * L::PLR, SZ + r * L::PLR, hrslot, u);
      else
        ring_put_hll<1>(U, W, SX + r * L::PLR, SY + r * L::PLR, SZ + r * L::PLR, hrslot, u);
    } else {
      ring_put(RU + r * L::PLR, RW + r * L::PLR, hrslot, u);
    }
  };

  // plane z0-1 (own slots only) into ring plane 0, plane z0 into ring plane 1
  wait(0);
#pragma unroll
  for (int r = 0; r < RPT; ++r)
    put(0, orslot[r], prep(stage0, oslot[r], own_out[r], ocol[r], plane_of(z0 - 1)));
  {
    wait(1);
    const float* st = stage0 + (1 % kStages) * L::STAGE;
    const int p = plane_of(z0);
#pragma unroll
    for (int r = 0; r < RPT; ++r) put(1, orslot[r], prep(st, oslot[r], own_out[r], ocol[r], p));
    if (hslot >= 0) put_halo(1, prep(st, hslot, halo_out, hcol, p));
  }
  int sp = TO ? 0 : A.tsrc_start[tile];   // (the transport-only pass has no source lists)
  const int se = TO ? 0 : A.tsrc_start[tile + 1];
  TileSrc src{nz, 0, 0.f, 0};
  if (sp < se) src = A.tsrc[sp];
  long long o = (long long)z0 * plane;   // plane offset of z (a row adds ocol[r])
  float cy[RPT], cT[RPT], cn[RPT];
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    cy[r] = 0.f; cT[r] = 1.f; cn[r] = 1.f;
    if (!TO && act[r]) { cy[r] = A.y[o + ocol[r]]; cT[r] = A.T[o + ocol[r]]; cn[r] = __ldg(A.nH + o + ocol[r]); }
  }
  // HLL: the flux through each own cell's lower z face, carried from plane to plane (the first
  // from ring planes 0 and 1, planes z0-1 and z0)
  float4 fzm[RPT];
  if (HLL) {
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int c0 = orslot[r], c1 = L::PLR + orslot[r];
      fzm[r] = hll_zface(RU[c0], RW[c0], SZ[c0], RU[c1], RW[c1], SZ[c1]);
    }
  }
  int rkm = 0, rk = 1, rkn = 2;         // ring planes of z-1, z and z+1 (plane index mod 3)
  // stages of z and z+1 (plane index mod kStages) and the phase parity of the latter
  int skn = 2 % kStages;
  unsigned pkn = (2 / kStages) & 1;

  for (int z = z0; z < z1; ++z, o += plane) {
    const int k = z - z0 + 1;           // plane index of z
    float4 up[RPT], pp[RPT];
    {
      if (!failed && !mbar_wait(&full[skn], pkn)) failed = true;
      const float* st = stage0 + skn * L::STAGE;
      const int p = plane_of(z + 1);
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        up[r] = prep(st, oslot[r], own_out[r], ocol[r], p);
        pp[r] = put(rkn, orslot[r], up[r]);
      }
      if (hslot >= 0) put_halo(rkn, prep(st, hslot, halo_out, hcol, p));
    }
    // chemistry fields of the own cells, one plane ahead
    float ny_[RPT], nT_[RPT], nn_[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      ny_[r] = 0.f; nT_[r] = 1.f; nn_[r] = 1.f;
      if (!TO && act[r] && z + 1 < z1) {
        const long long on = o + plane + ocol[r];
        ny_[r] = A.y[on]; nT_[r] = A.T[on]; nn_[r] = __ldg(A.nH + on);
      }
    }
    __syncthreads();
    // every thread has turned plane k+1 into ring records (before this barrier), so the stages
    // of planes up to k+1 are free: keep planes k+2 .. k+1+kStages in flight
    if (tid == 0 && !failed && issued < nplanes && issued <= k + 1 + kStages) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      while (issued < nplanes && issued <= k + 1 + kStages) issue(issued++);
    }
    float4 u[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      if (!act[r]) continue;
      const int c0 = rk * L::PLR + orslot[r], cm = rkm * L::PLR + orslot[r];
      const float4 uc = RU[c0], um = RU[cm];   // (um: GLF only)
      if (HLL) {
        const int cp = rkn * L::PLR + orslot[r];
        float4 fzp;
        u[r] = hll_update_zc(RU + c0, RW + c0, SX + c0, SY + c0, SZ + c0, uc, up[r], RW[cp],
                             SZ[cp], fzm[r], fzp, lam);
        fzm[r] = fzp;
      } else {
        const float4 pm = z_flux_q(um, RW[cm]);
        u[r] = lf_update(RU + c0, RW + c0, uc, um, pm, up[r], pp[r], cu, hl);
      }
      if (!PER) {
        float e = 0.f;
        if (gx == 0) e -= uc.y;
        if (gx == nx - 1) e += uc.y;
        if (gy[r] == 0) e -= uc.z;
        if (gy[r] == ny - 1) e += uc.z;
        if (z == 0) e -= uc.w;
        if (z == nz - 1) e += uc.w;
        if (e != 0.f) tl.escaped.add(lam * e);
      }
      clamp_state(u[r].x, u[r].y, u[r].z, u[r].w, tl.clipped);
    }
    while (!TO && src.z == z) {
#pragma unroll
      for (int r = 0; r < RPT; ++r)
        if (src.cell == ocell[r]) u[r].x += src.dN;
      src.z = nz;
      if (++sp < se) src = A.tsrc[sp];
    }
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      if (!act[r]) continue;
      const long long oc = o + ocol[r];
      if (TO) {   // the transported state, physical F
        A.out.N[oc] = u[r].x;
        A.out.Fx[oc] = u[r].y * P.c; A.out.Fy[oc] = u[r].z * P.c; A.out.Fz[oc] = u[r].w * P.c;
      } else if (SUR)
        chem_tally_store<STD>(P, tl, cn[r], u[r], cy[r], cT[r], A.out, A.y, A.T, oc, false, 0.f,
                              0.f, 0.f,
                              SurDefer{P, A.sur, A.sur.buf + (size_t)tile * kSurCap,
                                       A.sur.cnt + tile, (int)oc});
      else
        chem_tally_store<STD>(P, tl, cn[r], u[r], cy[r], cT[r], A.out, A.y, A.T, oc);
      cy[r] = ny_[r]; cT[r] = nT_[r]; cn[r] = nn_[r];
    }
    rkm = rk;
    rk = rkn;
    rkn = rkn == 2 ? 0 : rkn + 1;
    if (++skn == kStages) { skn = 0; pkn ^= 1u; }
  }
  if (failed) atomicAdd(A.slots.timeout, 1u);
  // if a wait gave up, thread 0 waits (bounded) for the planes it issued last before the CTA
  // exits, so no copy writes into shared memory afterwards
  if (__syncthreads_or(failed) && tid == 0)
    for (int k = max(0, issued - kStages); k < issued; ++k)
      mbar_wait(&full[k % kStages], (k / kStages) & 1);
  if (SUR) {
    static_assert(!SUR || L::STAGE_BYTES + L::RING_BYTES >= kSurScratchBytes,
                  "stage and plane rings too small for the network");
    sur_tail<STD>(P, A.sur, A.sur.buf + (size_t)tile * kSurCap, A.sur.cnt + tile, tl, A.out,
                  A.y, A.T, sm);
  }
  flush_tally<TYT>(tl, A.slots, tile);
}

namespace {

template <int TY, bool PER, bool STD, bool FULL, bool HLL, bool SUR, int RPT>
cudaError_t set_smem() {
  return cudaFuncSetAttribute(k_fused_tma<TY, PER, STD, FULL, HLL, SUR, RPT>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Layout<TY, HLL>::BYTES);
}

template <int TY, bool PER>
cudaError_t set_tma_attr() {
  const cudaError_t es[] = {
      set_smem<TY, PER, false, false, false, false, 1>(),
      set_smem<TY, PER, true, false, false, false, 1>(),
      set_smem<TY, PER, true, true, false, false, 1>(),
      set_smem<TY, PER, false, false, false, true, 1>(),
      set_smem<TY, PER, true, false, false, true, 1>(),
      set_smem<TY, PER, true, true, false, true, 1>(),
      set_smem<TY, PER, false, false, true, false, 1>(),
      set_smem<TY, PER, true, false, true, false, 1>(),
      set_smem<TY, PER, true, true, true, false, 1>(),
  };
  for (cudaError_t e : es)
    if (e != cudaSuccess) return e;
  if constexpr (TY >= 8) {   // two rows per thread (GLF; with HLL one row measured faster)
    const cudaError_t e2[] = {
        set_smem<TY, PER, false, false, false, false, 2>(),
        set_smem<TY, PER, true, false, false, false, 2>(),
        set_smem<TY, PER, true, true, false, false, 2>(),
        set_smem<TY, PER, false, false, false, true, 2>(),
        set_smem<TY, PER, true, false, false, true, 2>(),
        set_smem<TY, PER, true, true, false, true, 2>(),
    };
    for (cudaError_t e : e2)
      if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int TY, bool PER, int RPT>
cudaError_t launch_tma_t(const FusedArgs& a, const TmaMaps& m, cudaStream_t s) {
  dim3 grid((a.P.nx + kTileX - 1) / kTileX, (a.P.ny + TY - 1) / TY, (a.P.nz + a.tz - 1) / a.tz);
  dim3 block(kTileX, TY / RPT);
  const bool full = a.P.nx % kTileX == 0 && a.P.ny % TY == 0;
  const bool std_ = standard_chemistry(a.P);
  if (a.P.hll) {   // (the standard-chemistry and full-tile instances as for GLF; one row per
                   // thread: the HLL ring of 48 bytes per slot leaves three CTAs per SM at
                   // tile height 8, too few warps for two rows each)
    if (RPT != 1) return cudaErrorInvalidConfiguration;
    constexpr size_t B = Layout<TY, true>::BYTES;
    if (!std_)
      k_fused_tma<TY, PER, false, false, true><<<grid, block, B, s>>>(a, m);
    else if (full)
      k_fused_tma<TY, PER, true, true, true><<<grid, block, B, s>>>(a, m);
    else
      k_fused_tma<TY, PER, true, false, true><<<grid, block, B, s>>>(a, m);
  } else if (a.sur.img) {   // the surrogate instances
    constexpr size_t B = Layout<TY>::BYTES;
    if (!std_)
      k_fused_tma<TY, PER, false, false, false, true, RPT><<<grid, block, B, s>>>(a, m);
    else if (full)
      k_fused_tma<TY, PER, true, true, false, true, RPT><<<grid, block, B, s>>>(a, m);
    else
      k_fused_tma<TY, PER, true, false, false, true, RPT><<<grid, block, B, s>>>(a, m);
  } else {
    constexpr size_t B = Layout<TY>::BYTES;
    if (!std_)
      k_fused_tma<TY, PER, false, false, false, false, RPT><<<grid, block, B, s>>>(a, m);
    else if (full)
      k_fused_tma<TY, PER, true, true, false, false, RPT><<<grid, block, B, s>>>(a, m);
    else
      k_fused_tma<TY, PER, true, false, false, false, RPT><<<grid, block, B, s>>>(a, m);
  }
  return cudaGetLastError();
}

}  // namespace


cudaError_t launch_fused_tma(int ty, int rpt, const FusedArgs& a, const TmaMaps& m,
                             cudaStream_t s) {
  const bool per = a.P.bc == 0;
  if (rpt == 2) {
    switch (ty) {
      case 8: return per ? launch_tma_t<8, true, 2>(a, m, s) : launch_tma_t<8, false, 2>(a, m, s);
      case 16: return per ? launch_tma_t<16, true, 2>(a, m, s) : launch_tma_t<16, false, 2>(a, m, s);
      default: return cudaErrorInvalidValue;
    }
  }
  if (rpt != 1) return cudaErrorInvalidValue;
  switch (ty) {
    case 4: return per ? launch_tma_t<4, true, 1>(a, m, s) : launch_tma_t<4, false, 1>(a, m, s);
    case 8: return per ? launch_tma_t<8, true, 1>(a, m, s) : launch_tma_t<8, false, 1>(a, m, s);
    case 16: return per ? launch_tma_t<16, true, 1>(a, m, s) : launch_tma_t<16, false, 1>(a, m, s);
    default: return cudaErrorInvalidValue;
  }
}

// The transport-only instance (tile 32 x 8, two rows per thread, GLF flux) of the plain
// three-kernel step: the plain step's transport pass, with one closure evaluation per cell.
namespace {
template <bool PER, bool FULL>
cudaError_t set_to_attr() {
  return cudaFuncSetAttribute(k_fused_tma<8, PER, false, FULL, false, false, 2, true>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Layout<8>::BYTES);
}

// (its shared-memory attribute is set per device with the others, init_tma_attributes)
template <bool PER, bool FULL>
cudaError_t launch_to(const FusedArgs& a, const TmaMaps& m, cudaStream_t s) {
  using K = Layout<8>;
  dim3 grid((a.P.nx + kTileX - 1) / kTileX, (a.P.ny + 7) / 8, (a.P.nz + a.tz - 1) / a.tz);
  k_fused_tma<8, PER, false, FULL, false, false, 2, true><<<grid, dim3(kTileX, 4), K::BYTES, s>>>(a, m);
  return cudaGetLastError();
}
}  // namespace

// Shared-memory attributes of every instance of the TMA-staged kernel on the current device.
cudaError_t init_tma_attributes() {
  cudaError_t e;
  if ((e = set_tma_attr<4, true>()) != cudaSuccess) return e;
  if ((e = set_tma_attr<4, false>()) != cudaSuccess) return e;
  if ((e = set_tma_attr<8, true>()) != cudaSuccess) return e;
  if ((e = set_tma_attr<8, false>()) != cudaSuccess) return e;
  if ((e = set_tma_attr<16, true>()) != cudaSuccess) return e;
  if ((e = set_tma_attr<16, false>()) != cudaSuccess) return e;
  if ((e = set_to_attr<true, true>()) != cudaSuccess) return e;
  if ((e = set_to_attr<true, false>()) != cudaSuccess) return e;
  if ((e = set_to_attr<false, true>()) != cudaSuccess) return e;
  return set_to_attr<false, false>();
}

cudaError_t launch_transport_tma(const FusedArgs& a, const TmaMaps& m8, cudaStream_t s) {
  if (a.P.hll) return cudaErrorInvalidConfiguration;
  const bool full = a.P.nx % kTileX == 0 && a.P.ny % 8 == 0;
  if (a.P.bc == 0) return full ? launch_to<true, true>(a, m8, s) : launch_to<true, false>(a, m8, s);
  return full ? launch_to<false, true>(a, m8, s) : launch_to<false, false>(a, m8, s);
}

// Tensor maps of the radiation fields for a tile height ty: for each ping-pong buffer and each
// of N, Fx, Fy, Fz a (32+8) x (ty+2) x 1 box. Returns false if the driver entry point is
// unavailable or an encode fails (the caller then uses k_fused).
bool make_tma_maps(int nx, int ny, int nz, int ty, float* const u[2][4], TmaMaps* out) {
  if (nx % 4 != 0) return false;
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return false;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4};
  const cuuint32_t estr[3] = {1, 1, 1};
  const cuuint32_t box_u[3] = {(cuuint32_t)kBoxX, (cuuint32_t)(ty + 2), 1};
  for (int b = 0; b < 2; ++b)
    for (int q = 0; q < 4; ++q)
      if (encode(&out->u[b][q], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, u[b][q], dims, strides, box_u,
                 estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
          CUDA_SUCCESS)
        return false;
  return true;
}

}  // namespace aton
