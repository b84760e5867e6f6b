// aton_kernels.cu -- sm_103a kernels of one ATON radiative step.
//
// Device memory holds the physical flux F; every load scales it to Fh = F/c and every store
// back to F, so a saved state reloads bit for bit.
//
// Fused path (one kernel per step): each CTA owns a 32 x TY column tile of the grid and a
// z-slab of tz planes, and marches through the slab plane by plane. The (N, Fh) plane with a
// one-cell halo and the M1 closure pair (iso, w) of each of its cells (N D = iso I + w Fh Fh^T,
// evaluated once per cell) sit in a three-deep shared-memory ring; the z neighbours of the own
// column stay in registers. For
// every cell of a plane the kernel then does the Lax-Friedrichs transport (section 2.2;
// Appendix Eqs. A2, A5), the realisability clamp, the point-source injection (section 2.3)
// and the chemistry/cooling/absorption operator Phi (Appendix Eq. A4), and stores N, Fh, y,
// T once. Loads of plane z+2 are issued before plane z is computed.
//
// Plain path (three kernels per step): transport to the other buffer, source scatter,
// chemistry in place; the comparison baseline.
//
// Tallies (absorbed, escaped, clipped photons in density units; sub-step counts; error
// counts) are reduced per CTA in FP64 and added to a per-tile slot, so sums are deterministic.
#include "aton_internal.h"
#include "aton_step_common.cuh"

namespace aton {

// =========================================================================================
// Fused step kernel
// =========================================================================================
template <int TY, bool PER, bool STD>
__global__ void __launch_bounds__(kTileX * TY) k_fused(const FusedArgs A) {
  constexpr int TX = kTileX, RX = kRingRX, PLR = RX * (TY + 2);
  constexpr int NH = 2 * TX + 2 * TY;
  // three-plane ring: [3][PLR] (N, F/c), [3][PLR] closure pairs (iso, w)
  extern __shared__ float4 ring[];
  float4* RU = ring;
  float2* RW = reinterpret_cast<float2*>(RU + 3 * PLR);
  const StepParams& P = A.P;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + TX * ty;
  const int nx = P.nx, ny = P.ny, nz = P.nz;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * A.tz;
  const int z1 = min(z0 + A.tz, nz);
  const long long plane = (long long)nx * ny;
  const int gx = x0 + tx, gy = y0 + ty;
  const bool act = (gx < nx) && (gy < ny);
  const long long ocol = bc_map(gx, nx, PER) + (long long)nx * bc_map(gy, ny, PER);
  const int oslot = (ty + 1) * RX + (tx + 1);
  int hslot = -1;
  long long hcol = 0;
  if (tid < NH) {   // the halo ring of the tile: rows y0-1 and y0+TY, columns x0-1 and x0+TX
    int hx, hy;
    if (tid < TX) { hx = tid; hy = -1; }
    else if (tid < 2 * TX) { hx = tid - TX; hy = TY; }
    else if (tid < 2 * TX + TY) { hx = -1; hy = tid - 2 * TX; }
    else { hx = TX; hy = tid - 2 * TX - TY; }
    hslot = (hy + 1) * RX + (hx + 1);
    hcol = bc_map(x0 + hx, nx, PER) + (long long)nx * bc_map(y0 + hy, ny, PER);
  }
  const float* __restrict__ iN = A.in.N;
  const float* __restrict__ iX = A.in.Fx;
  const float* __restrict__ iY = A.in.Fy;
  const float* __restrict__ iZ = A.in.Fz;
  const float rc = P.rc, lam = P.lam;
  const float hl = 0.5f * lam, cu = 1.f - 3.f * lam;
  auto pz = [&](int z) { return (long long)bc_map(z, nz, PER) * plane; };
  auto ld = [&](long long o) {
    return make_float4(__ldg(iN + o), __ldg(iX + o) * rc, __ldg(iY + o) * rc, __ldg(iZ + o) * rc);
  };

  // prologue: plane z0-1 (own column, registers), plane z0 (ring slot 0), plane z0+1 (registers)
  float4 um = ld(pz(z0 - 1) + ocol);
  float4 pm = z_flux(um);
  float4 uc = ld(pz(z0) + ocol);
  float4 pc = ring_put(RU, RW, oslot, uc);
  if (hslot >= 0) ring_put(RU, RW, hslot, ld(pz(z0) + hcol));
  float4 nu = ld(pz(z0 + 1) + ocol);
  float4 nh = make_float4(0.f, 0.f, 0.f, 0.f);
  if (hslot >= 0) nh = ld(pz(z0 + 1) + hcol);
  float cy = 0.f, cT = 1.f, cn = 1.f;
  long long o = (long long)z0 * plane + ocol;
  if (act) { cy = A.y[o]; cT = A.T[o]; cn = __ldg(A.nH + o); }

  // the tile's next point source (host-merged, sorted by plane, at most one entry per cell)
  const int tile = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  int sp = A.tsrc_start[tile];
  const int se = A.tsrc_start[tile + 1];
  TileSrc src{nz, 0, 0.f, 0};
  if (sp < se) src = A.tsrc[sp];
  Tally tl;

  // offset of plane z+2 (boundary-mapped), advanced without an integer modulo
  int zz2 = bc_map(z0 + 2, nz, PER);
  long long p2 = (long long)zz2 * plane;
  int rcur = 0;
  for (int z = z0; z < z1; ++z, o += plane) {
    const int rnx = rcur == 2 ? 0 : rcur + 1;
    // plane z+1 into the ring (own and halo slot); its z flux kept in registers
    const float4 up = nu;
    const float4 pp = ring_put(RU + rnx * PLR, RW + rnx * PLR, oslot, up);
    if (hslot >= 0) ring_put(RU + rnx * PLR, RW + rnx * PLR, hslot, nh);
    // prefetch plane z+2 and the chemistry fields of plane z+1
    float ny_ = 0.f, nT_ = 1.f, nn_ = 1.f;
    if (z + 1 < z1) {
      nu = ld(p2 + ocol);
      if (hslot >= 0) nh = ld(p2 + hcol);
      if (act) { ny_ = A.y[o + plane]; nT_ = A.T[o + plane]; nn_ = __ldg(A.nH + o + plane); }
    }
    __syncthreads();
    if (act) {
      const int c0 = rcur * PLR + oslot;
      float4 u = lf_update(RU + c0, RW + c0, uc, um, pm, up, pp, cu, hl);
      if (!PER) {  // transmissive faces: outward photon flux through the boundary
        float e = 0.f;
        if (gx == 0) e -= uc.y;
        if (gx == nx - 1) e += uc.y;
        if (gy == 0) e -= uc.z;
        if (gy == ny - 1) e += uc.z;
        if (z == 0) e -= uc.w;
        if (z == nz - 1) e += uc.w;
        if (e != 0.f) tl.escaped.add(lam * e);
      }
      clamp_state(u.x, u.y, u.z, u.w, tl.clipped);
      while (src.z == z) {
        if (src.cell == tid) u.x += src.dN;
        src.z = nz;
        if (++sp < se) src = A.tsrc[sp];
      }
      chem_tally_store<STD>(P, tl, cn, u, cy, cT, A.out, A.y, A.T, o);
    }
    um = uc; pm = pc; uc = up; pc = pp;
    cy = ny_; cT = nT_; cn = nn_;
    rcur = rnx;
    // z+3 (boundary-mapped) for the next plane's prefetch
    if (++zz2 >= nz) { zz2 = PER ? zz2 - nz : nz - 1; }
    p2 = (long long)zz2 * plane;
  }
  flush_tally<TY>(tl, A.slots, tile);
}

int fused_tiles(int nx, int ny, int nz, int ty, int tz) {
  return ((nx + kTileX - 1) / kTileX) * ((ny + ty - 1) / ty) * ((nz + tz - 1) / tz);
}

template <int TY>
static constexpr size_t fused_smem() {
  return (size_t)3 * kRingRX * (TY + 2) * (sizeof(float4) + sizeof(float2));
}

template <int TY, bool PER>
static cudaError_t set_fused_attr() {
  cudaError_t e = cudaFuncSetAttribute(k_fused<TY, PER, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fused_smem<TY>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_fused<TY, PER, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)fused_smem<TY>());
}

cudaError_t init_kernel_attributes() {
  cudaError_t e;
  if ((e = set_fused_attr<4, true>()) != cudaSuccess) return e;
  if ((e = set_fused_attr<4, false>()) != cudaSuccess) return e;
  if ((e = set_fused_attr<8, true>()) != cudaSuccess) return e;
  if ((e = set_fused_attr<8, false>()) != cudaSuccess) return e;
  if ((e = set_fused_attr<16, true>()) != cudaSuccess) return e;
  return set_fused_attr<16, false>();
}

template <int TY, bool PER>
static cudaError_t launch_fused_t(const FusedArgs& a, cudaStream_t s) {
  const size_t smem = fused_smem<TY>();
  dim3 grid((a.P.nx + kTileX - 1) / kTileX, (a.P.ny + TY - 1) / TY, (a.P.nz + a.tz - 1) / a.tz);
  dim3 block(kTileX, TY);
  if (standard_chemistry(a.P)) k_fused<TY, PER, true><<<grid, block, smem, s>>>(a);
  else k_fused<TY, PER, false><<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fused(int ty, const FusedArgs& a, cudaStream_t s) {
  const bool per = a.P.bc == 0;
  switch (ty) {
    case 4: return per ? launch_fused_t<4, true>(a, s) : launch_fused_t<4, false>(a, s);
    case 8: return per ? launch_fused_t<8, true>(a, s) : launch_fused_t<8, false>(a, s);
    case 16: return per ? launch_fused_t<16, true>(a, s) : launch_fused_t<16, false>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

// =========================================================================================
// Plain (unfused) step: transport kernel, source kernel, chemistry kernel
// =========================================================================================
__device__ __forceinline__ void load_u(const Fields& f, long long o, float rc, float u[4]) {
  u[0] = __ldg(f.N + o); u[1] = __ldg(f.Fx + o) * rc; u[2] = __ldg(f.Fy + o) * rc;
  u[3] = __ldg(f.Fz + o) * rc;
}

template <bool PER, bool HLL>
__global__ void __launch_bounds__(kPlainThreads) k_plain_transport(const PlainArgs A) {
  const StepParams& P = A.P;
  const int nx = P.nx, ny = P.ny, nz = P.nz;
  const long long ncell = (long long)nx * ny * nz;
  Tally tl;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < ncell;
       id += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(id % nx);
    const int j = (int)((id / nx) % ny);
    const int k = (int)(id / ((long long)nx * ny));
    float u[4];
    load_u(A.in, id, P.rc, u);
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    ND6 dc{};
    M1Speeds mc{};
    if (HLL) {
      dc = m1_pressure(u[0], u[1], u[2], u[3]);
      mc = m1_speeds(u[0], u[1], u[2], u[3]);
    }
    for (int d = 0; d < 3; ++d) {
      int ip[3] = {i, j, k}, im[3] = {i, j, k};
      ip[d] += 1; im[d] -= 1;
      const int n3[3] = {nx, ny, nz};
      ip[d] = bc_map(ip[d], n3[d], PER);
      im[d] = bc_map(im[d], n3[d], PER);
      const long long op = ip[0] + (long long)nx * (ip[1] + (long long)ny * ip[2]);
      const long long om = im[0] + (long long)nx * (im[1] + (long long)ny * im[2]);
      float a[4], b[4];
      load_u(A.in, op, P.rc, a);
      load_u(A.in, om, P.rc, b);
      const ND6 da = m1_pressure(a[0], a[1], a[2], a[3]);
      const ND6 db = m1_pressure(b[0], b[1], b[2], b[3]);
      float fa[4], fb[4], fc[4];
      if (d == 0) {
        fa[0] = a[1]; fa[1] = da.xx; fa[2] = da.xy; fa[3] = da.xz;
        fb[0] = b[1]; fb[1] = db.xx; fb[2] = db.xy; fb[3] = db.xz;
        fc[0] = u[1]; fc[1] = dc.xx; fc[2] = dc.xy; fc[3] = dc.xz;
      } else if (d == 1) {
        fa[0] = a[2]; fa[1] = da.xy; fa[2] = da.yy; fa[3] = da.yz;
        fb[0] = b[2]; fb[1] = db.xy; fb[2] = db.yy; fb[3] = db.yz;
        fc[0] = u[2]; fc[1] = dc.xy; fc[2] = dc.yy; fc[3] = dc.yz;
      } else {
        fa[0] = a[3]; fa[1] = da.xz; fa[2] = da.yz; fa[3] = da.zz;
        fb[0] = b[3]; fb[1] = db.xz; fb[2] = db.yz; fb[3] = db.zz;
        fc[0] = u[3]; fc[1] = dc.xz; fc[2] = dc.yz; fc[3] = dc.zz;
      }
      if (!HLL) {
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] += 0.5f * (fa[q] - fb[q]) - 0.5f * (a[q] - 2.f * u[q] + b[q]);
      } else {
        // wave-speed bounds of the two faces from the three cells' speeds along d
        const M1Speeds ma = m1_speeds(a[0], a[1], a[2], a[3]);
        const M1Speeds mb = m1_speeds(b[0], b[1], b[2], b[3]);
        const float gc = d == 0 ? mc.gx : (d == 1 ? mc.gy : mc.gz);
        const float ga = d == 0 ? ma.gx : (d == 1 ? ma.gy : ma.gz);
        const float gb = d == 0 ? mb.gx : (d == 1 ? mb.gy : mb.gz);
        float lc, hc, la, ha, lb, hb;
        m1_axis_speeds(mc, gc, lc, hc);
        m1_axis_speeds(ma, ga, la, ha);
        m1_axis_speeds(mb, gb, lb, hb);
        // face + between the centre and a, face - between b and the centre (hll_coef: l+ - l-
        // >= 1/sqrt(3) unless both cells stream at f = 1 parallel to the face, where the two
        // fluxes vanish and their mean is taken)
        const HllCoef kp = hll_coef(fminf(0.f, fminf(lc, la)), fmaxf(0.f, fmaxf(hc, ha)));
        const HllCoef km = hll_coef(fminf(0.f, fminf(lb, lc)), fmaxf(0.f, fmaxf(hb, hc)));
#pragma unroll
        for (int q = 0; q < 4; ++q)
          acc[q] += hll_face(kp, fc[q], fa[q], u[q], a[q]) - hll_face(km, fb[q], fc[q], b[q], u[q]);
      }
    }
    // acc is the sum over the three axes of (flux at the high face - flux at the low face)
    float Nn = u[0] - P.lam * acc[0];
    float Xn = u[1] - P.lam * acc[1];
    float Yn = u[2] - P.lam * acc[2];
    float Zn = u[3] - P.lam * acc[3];
    if (!PER) {
      float e = 0.f;
      if (i == 0) e -= u[1];
      if (i == nx - 1) e += u[1];
      if (j == 0) e -= u[2];
      if (j == ny - 1) e += u[2];
      if (k == 0) e -= u[3];
      if (k == nz - 1) e += u[3];
      if (e != 0.f) tl.escaped.add(P.lam * e);
    }
    clamp_state(Nn, Xn, Yn, Zn, tl.clipped);
    A.out.N[id] = Nn; A.out.Fx[id] = Xn * P.c; A.out.Fy[id] = Yn * P.c; A.out.Fz[id] = Zn * P.c;
  }
  flush_tally<kPlainThreads / 32>(tl, A.slots, blockIdx.x);
}

__global__ void k_plain_sources(const PlainArgs A) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < A.nsrc) A.out.N[A.src_idx[s]] += A.src_dN[s];
}

// pair record of the chemistry operator: nH, N, y, T in; N', y', T' out; sub-steps
__device__ __forceinline__ void sink_record(const PlainArgs& A, long long id, float n, float N0,
                                            float y0, float T0, float N1, float y1, float T1,
                                            int nsub) {
  if (A.sink && (id + A.sink_phase) % A.sink_stride == 0) {
    const long long r = A.sink_base + id / A.sink_stride;
    if (r < A.sink_cap) {
      float* o = A.sink + r * 8;
      o[0] = n; o[1] = N0; o[2] = y0; o[3] = T0; o[4] = N1; o[5] = y1; o[6] = T1; o[7] = (float)nsub;
    }
  }
}

__global__ void __launch_bounds__(kPlainThreads) k_plain_chem(const PlainArgs A) {
  const StepParams& P = A.P;
  const long long ncell = (long long)P.nx * P.ny * P.nz;
  Tally tl;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < ncell;
       id += (long long)gridDim.x * blockDim.x) {
    float N = A.out.N[id], X = A.out.Fx[id] * P.rc, Y = A.out.Fy[id] * P.rc, Z = A.out.Fz[id] * P.rc;
    float y = A.y[id], T = A.T[id];
    const float n = __ldg(A.nH + id);
    const float N0 = N, y0 = y, T0 = T;
    const ChemOut co = chem_cell(P, n, N, X, Y, Z, y, T);
    sink_record(A, id, n, N0, y0, T0, N, y, T, co.nsub);
    tl.absorbed.add(N0 - N);
    tl.sub += co.nsub;
    tl.mx = max(tl.mx, (unsigned)co.nsub);
    tl.err += co.err;
    if (!isfinite(N) || !isfinite(T) || !isfinite(X + Y + Z)) tl.nan += 1;
    A.out.N[id] = N; A.out.Fx[id] = X * P.c; A.out.Fy[id] = Y * P.c; A.out.Fz[id] = Z * P.c;
    A.y[id] = y; A.T[id] = T;
  }
  flush_tally<kPlainThreads / 32>(tl, A.slots, blockIdx.x);
}

// Chemistry with the learned surrogate, pass 1: the exact operator for every cell except the
// candidates, which are appended to a list. A cell is a candidate when the exact operator would
// sub-cycle heavily -- the explicit estimate of the sub-step count from photo-ionisation
// (Gamma y dt over eps max(y, y_floor)) and photo-heating (over eps T) is at least sur_gate --
// and its features lie inside the training range. (The network's registers stay out of this
// kernel, which keeps the occupancy of the plain chemistry kernel.)
__global__ void __launch_bounds__(kPlainThreads) k_plain_chem_gate(const PlainArgs A) {
  const StepParams& P = A.P;
  const long long ncell = (long long)P.nx * P.ny * P.nz;
  Tally tl;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < ncell;
       id += (long long)gridDim.x * blockDim.x) {
    float N = A.out.N[id];
    float y = A.y[id], T = A.T[id];
    const float n = __ldg(A.nH + id);
    if (sur_candidate(P, A.sur_gate, *A.sur_norm, n, N, y, T)) {
      A.sur_list[atomicAdd(A.sur_count, 1)] = (int)id;
      continue;
    }
    float X = A.out.Fx[id] * P.rc, Y = A.out.Fy[id] * P.rc, Z = A.out.Fz[id] * P.rc;
    const float N0 = N;
    const ChemOut co = chem_cell(P, n, N, X, Y, Z, y, T);
    tl.absorbed.add(N0 - N);
    tl.sub += co.nsub;
    tl.mx = max(tl.mx, (unsigned)co.nsub);
    tl.err += co.err;
    if (!isfinite(N) || !isfinite(T) || !isfinite(X + Y + Z)) tl.nan += 1;
    A.out.N[id] = N; A.out.Fx[id] = X * P.c; A.out.Fy[id] = Y * P.c; A.out.Fz[id] = Z * P.c;
    A.y[id] = y; A.T[id] = T;
  }
  flush_tally<kPlainThreads / 32>(tl, A.slots, blockIdx.x);
}

// Pass 2: the listed candidates, 32 per warp. The warp runs the MLP for its 32 cells on tensor
// cores; a prediction is accepted only if its photons absorbed per atom, (N - N')/nH, match
// the atoms ionised, (y - y') plus the recombinations over dt at the mean state, within
// sur_resid of max(y, 1e-8) (sur_accept); rejected cells take the exact operator. Tallies go to
// the slots after the first pass's.
__global__ void __launch_bounds__(kPlainThreads) k_plain_chem_sur(const PlainArgs A) {
  __shared__ __align__(16) MlpImage W;
  __shared__ float xs[kPlainThreads / 32][32][8];
  __shared__ float ys[kPlainThreads / 32][32][4];
  const int count = *A.sur_count;
  Tally tl;
  // blocks without a chunk of candidates skip the weight copy
  if (blockIdx.x * (kPlainThreads / 32) < (count + 31) / 32) {
    {
      const uint4* s = reinterpret_cast<const uint4*>(A.sur_img);
      uint4* d = reinterpret_cast<uint4*>(&W);
      const int nb = (int)(offsetof(MlpImage, W2T) / 16);
      for (int i = threadIdx.x; i < nb; i += blockDim.x) d[i] = s[i];
      for (int i = threadIdx.x; i < 2 * kMlpH + 8; i += blockDim.x) W.b1[i] = A.sur_img->b1[i];
    }
    __syncthreads();
    const MlpNorm nm = *A.sur_norm;
    const StepParams& P = A.P;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const float l10dt = log10f(P.dt);
    const int nchunk = (count + 31) / 32;
    for (int ch = blockIdx.x * (kPlainThreads / 32) + w; ch < nchunk; ch += gridDim.x * (kPlainThreads / 32)) {
      const int k = ch * 32 + lane;
      const bool valid = k < count;
      const long long id = valid ? A.sur_list[k] : 0;
      float N = 0.f, X = 0.f, Y = 0.f, Z = 0.f, y = 1.f, T = 1e4f, n = 1.f;
      if (valid) {
        N = A.out.N[id]; X = A.out.Fx[id] * P.rc; Y = A.out.Fy[id] * P.rc; Z = A.out.Fz[id] * P.rc;
        y = A.y[id]; T = A.T[id]; n = __ldg(A.nH + id);
      }
      const float N0 = N;
      const float f[kMlpIn] = {log10f(n), log10f(fmaxf(y, 1e-10f)), log10f(T), log10f(fmaxf(N, 1e-30f)), l10dt};
#pragma unroll
      for (int i = 0; i < kMlpIn; ++i) xs[w][lane][i] = (f[i] - nm.in_mean[i]) * nm.in_scale[i];
      __syncwarp();
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int r0 = half * 16;
        const float* xa = xs[w][r0 + g];
        const float* xb = xs[w][r0 + g + 8];
        const unsigned a[4] = {pack_bf16(2 * t < kMlpIn ? xa[2 * t] : 0.f, 2 * t + 1 < kMlpIn ? xa[2 * t + 1] : 0.f),
                               pack_bf16(2 * t < kMlpIn ? xb[2 * t] : 0.f, 2 * t + 1 < kMlpIn ? xb[2 * t + 1] : 0.f),
                               0u, 0u};
        float z1[8][4], z2[8][4], yo[4];
        mlp_forward16<false>(W, a, z1, z2, yo);
        if (2 * t < 4) {
          ys[w][r0 + g][2 * t] = yo[0]; ys[w][r0 + g][2 * t + 1] = yo[1];
          ys[w][r0 + g + 8][2 * t] = yo[2]; ys[w][r0 + g + 8][2 * t + 1] = yo[3];
        }
      }
      __syncwarp();
      bool done = false;
      if (valid) {
        const float o3[3] = {ys[w][lane][0], ys[w][lane][1], ys[w][lane][2]};
        float N1, y1, T1;
        if (sur_accept(P, nm, A.sur_resid, o3, n, N, y, T, N1, y1, T1)) {
          const float fr = N > 0.f ? N1 / N : 1.f;
          N = N1; X *= fr; Y *= fr; Z *= fr; y = y1; T = T1;
          done = true;
          tl.sur += 1;
        }
        int nsub = 0;
        if (!done) {
          const ChemOut co = chem_cell(P, n, N, X, Y, Z, y, T);
          nsub = co.nsub;
          tl.err += co.err;
        }
        tl.absorbed.add(N0 - N);
        tl.sub += nsub;
        tl.mx = max(tl.mx, (unsigned)nsub);
        if (!isfinite(N) || !isfinite(T) || !isfinite(X + Y + Z)) tl.nan += 1;
        A.out.N[id] = N; A.out.Fx[id] = X * P.c; A.out.Fy[id] = Y * P.c; A.out.Fz[id] = Z * P.c;
        A.y[id] = y; A.T[id] = T;
      }
      __syncwarp();
    }
  }
  flush_tally<kPlainThreads / 32>(tl, A.slots, kPlainBlocks + blockIdx.x);
}

int plain_launches() { return 3; }

cudaError_t launch_plain_step(const PlainArgs& a, cudaStream_t s) {
  if (a.transported) {
  } else if (a.P.hll) {
    if (a.P.bc == 0) k_plain_transport<true, true><<<kPlainBlocks, kPlainThreads, 0, s>>>(a);
    else k_plain_transport<false, true><<<kPlainBlocks, kPlainThreads, 0, s>>>(a);
  } else {
    if (a.P.bc == 0) k_plain_transport<true, false><<<kPlainBlocks, kPlainThreads, 0, s>>>(a);
    else k_plain_transport<false, false><<<kPlainBlocks, kPlainThreads, 0, s>>>(a);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (a.nsrc > 0) {
    k_plain_sources<<<(a.nsrc + 255) / 256, 256, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (a.sur_img) {
    e = cudaMemsetAsync(a.sur_count, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_plain_chem_gate<<<kPlainBlocks, kPlainThreads, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_plain_chem_sur<<<kSurBlocks, kPlainThreads, 0, s>>>(a);
  } else {
    k_plain_chem<<<kPlainBlocks, kPlainThreads, 0, s>>>(a);
  }
  return cudaGetLastError();
}

// =========================================================================================
// Utility kernels
// =========================================================================================
__global__ void k_scale(float* dst, const float* src, float k, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i] * k;
}

__global__ void k_one_minus(float* dst, const float* src, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = 1.f - src[i];
}

__global__ void k_validate(const float* N, const float* y, const float* T, const float* nH,
                           long long n, unsigned int* bad) {
  unsigned int b = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float a = N[i], yy = y[i], t = T[i], h = nH[i];
    const bool ok = isfinite(a) && a >= 0.f && isfinite(yy) && yy >= 0.f && yy <= 1.f &&
                    isfinite(t) && t > 0.f && isfinite(h) && h >= 1.17549435e-38f;
    b += ok ? 0u : 1u;
  }
  if (b) atomicAdd(bad, b);
}

// Largest f^2 = |F|^2 / (cN)^2 of a state (cells with N > kNTiny), as the bits of a float:
// non-negative floats order like their bit patterns, so an integer atomicMax finds it.
__global__ void k_max_f2(const float* N, const float* Fx, const float* Fy, const float* Fz,
                         float rc, long long n, unsigned int* out) {
  float m = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float a = __ldg(N + i);
    if (a > kNTiny) {
      const float x = __ldg(Fx + i) * rc, y = __ldg(Fy + i) * rc, z = __ldg(Fz + i) * rc;
      m = fmaxf(m, div_fast(x * x + y * y + z * z, a * a));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(out, __float_as_uint(m));
}

cudaError_t launch_max_f2(const float* N, const float* Fx, const float* Fy, const float* Fz,
                          float rc, int64_t n, unsigned int* out, cudaStream_t s) {
  k_max_f2<<<148 * 4, 256, 0, s>>>(N, Fx, Fy, Fz, rc, n, out);
  return cudaGetLastError();
}

cudaError_t launch_scale(float* dst, const float* src, float k, int64_t n, cudaStream_t s) {
  k_scale<<<148 * 4, 256, 0, s>>>(dst, src, k, n);
  return cudaGetLastError();
}

cudaError_t launch_one_minus(float* dst, const float* src, int64_t n, cudaStream_t s) {
  k_one_minus<<<148 * 4, 256, 0, s>>>(dst, src, n);
  return cudaGetLastError();
}

cudaError_t launch_validate(const float* N, const float* y, const float* T, const float* nH,
                            int64_t n, unsigned int* bad, cudaStream_t s) {
  k_validate<<<148 * 4, 256, 0, s>>>(N, y, T, nH, n, bad);
  return cudaGetLastError();
}

// Fixed-order FP64 reduction of the slots: out_acc3 = sums of the three photon tallies,
// out_u64_4 = {sum sub-steps, max sub-steps, sum error cells, sum non-finite cells}.
__global__ void __launch_bounds__(512) k_reduce_slots(const Slots S, double* out_acc3,
                                                      unsigned long long* out4) {
  constexpr int NT = 512;
  __shared__ double sa[3][NT];
  __shared__ unsigned long long su[5][NT];
  const int t = threadIdx.x;
  double a0 = 0, a1 = 0, a2 = 0;
  unsigned long long sb = 0, mx = 0, er = 0, na = 0, us = 0;
  for (int i = t; i < S.n; i += NT) {
    a0 += S.acc[3 * i]; a1 += S.acc[3 * i + 1]; a2 += S.acc[3 * i + 2];
    sb += S.sub[i];
    mx = max(mx, (unsigned long long)S.mx[i]);
    er += S.err[i]; na += S.nan[i]; us += S.sur[i];
  }
  sa[0][t] = a0; sa[1][t] = a1; sa[2][t] = a2;
  su[0][t] = sb; su[1][t] = mx; su[2][t] = er; su[3][t] = na; su[4][t] = us;
  __syncthreads();
  for (int w = NT / 2; w > 0; w >>= 1) {
    if (t < w) {
      sa[0][t] += sa[0][t + w]; sa[1][t] += sa[1][t + w]; sa[2][t] += sa[2][t + w];
      su[0][t] += su[0][t + w]; su[1][t] = max(su[1][t], su[1][t + w]);
      su[2][t] += su[2][t + w]; su[3][t] += su[3][t + w]; su[4][t] += su[4][t + w];
    }
    __syncthreads();
  }
  if (t == 0) {
    out_acc3[0] = sa[0][0]; out_acc3[1] = sa[1][0]; out_acc3[2] = sa[2][0];
    out4[0] = su[0][0]; out4[1] = su[1][0]; out4[2] = su[2][0]; out4[3] = su[3][0];
    out4[4] = su[4][0];
  }
}

cudaError_t launch_reduce_slots(const Slots& sl, double* out_acc3, unsigned long long* out4,
                                cudaStream_t s) {
  k_reduce_slots<<<1, 512, 0, s>>>(sl, out_acc3, out4);
  return cudaGetLastError();
}

// Sum of a float field in FP64, fixed order: per-block partials then one block.
// Sum of a float field (the stored photons): each thread sums its float4 groups (grid-stride,
// fixed grid) in a compensated FP32 accumulator (error-free TwoSum) whose value s + c is taken
// in FP64, then the CTA reduces in FP64. FP32 arithmetic keeps the pass at memory speed (an FP64 add per element
// is throughput-bound on this part); the compensation keeps the per-thread sums to FP64 quality.
__global__ void __launch_bounds__(256) k_sum_partial(const float* f, long long n, double* part) {
  __shared__ double s[256];
  TwoSumF k;
  const long long n4 = n >> 2;
  const float4* f4 = reinterpret_cast<const float4*>(f);   // cudaMalloc'd: 16-byte aligned
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n4; i += (long long)gridDim.x * 256) {
    const float4 v = __ldg(f4 + i);
    k.add(v.x); k.add(v.y); k.add(v.z); k.add(v.w);
  }
  if (blockIdx.x == 0 && threadIdx.x < (n & 3)) k.add(f[(n4 << 2) + threadIdx.x]);
  s[threadIdx.x] = k.value();
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void __launch_bounds__(256) k_sum_final(const double* part, int n, double* out) {
  __shared__ double s[256];
  double a = 0;
  for (int i = threadIdx.x; i < n; i += 256) a += part[i];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

cudaError_t launch_sum_field(const float* f, int64_t n, double* partial, double* out,
                             cudaStream_t s) {
  k_sum_partial<<<kSumBlocks, 256, 0, s>>>(f, n, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sum_final<<<1, 256, 0, s>>>(partial, kSumBlocks, out);
  return cudaGetLastError();
}

}  // namespace aton
