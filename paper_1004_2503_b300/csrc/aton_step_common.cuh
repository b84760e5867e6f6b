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

// ---------------------------------------------------------------------------------------
// Cell update shared by the fused kernels. A plane of the three-plane ring holds, per slot
// (row pitch kTileX + 2, one-cell halo), the records (N, Fx/c, Fy/c, Fz/c) and the closure pair
// (iso, w) of m1_iso_w, so a neighbour costs two vector loads and the pressure components a face
// needs, N D_ij = iso delta_ij + w Fh_i Fh_j, are formed from them. Each product is rounded on
// its own (no contraction), so a face value is the same number in both cells that use it.
// ---------------------------------------------------------------------------------------
constexpr int kRingRX = kTileX + 2;

// Paired FP32 arithmetic (one instruction for two lanes on sm_100 and later; each lane rounds
// like the scalar operation).
__device__ __forceinline__ float2 lo2(const float4& v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4& v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 add2(const float2& a, const float2& b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(const float2& a, const float2& b) {
  return __fadd2_rn(a, make_float2(-b.x, -b.y));
}

// z flux (Fz/c, Dxz, Dyz, Dzz) N of a state and its closure pair.
__device__ __forceinline__ float4 z_flux_q(const float4& u, const float2& q) {
  const float wz = __fmul_rn(q.y, u.w);
  return make_float4(u.w, __fmul_rn(wz, u.y), __fmul_rn(wz, u.z), fmaf(wz, u.w, q.x));
}

// Store the record of a slot; returns the cell's z flux.
__device__ __forceinline__ float4 ring_put(float4* RU, float2* RW, int slot, const float4& u) {
  const float2 q = m1_iso_w(u.x, u.y, u.z, u.w);
  RU[slot] = u;
  RW[slot] = q;
  return z_flux_q(u, q);
}

// z flux of a state held in registers.
__device__ __forceinline__ float4 z_flux(const float4& u) {
  return z_flux_q(u, m1_iso_w(u.x, u.y, u.z, u.w));
}

// Global Lax-Friedrichs update of the centre cell (section 2.2; Appendix Eqs. A2, A5) from its
// x and y neighbours in the ring (U, W point at the centre slot) and its z neighbours in
// registers (um, pm below; up, pp above): with the face flux (Phi_L + Phi_R)/2 - (u_R - u_L)/2
// (wave speed c, Fh = F/c units), the update sums, over the six faces, the flux difference
// minus the neighbour values and is written around the centre value:
//   u' = (1 - 3 lam) u - lam/2 [sum_d (Phi_d(u_{+d}) - Phi_d(u_{-d})) - sum_nb u_nb].
// x faces carry (Fx, Dxx, Dxy, Dxz) N, y faces (Fy, Dxy, Dyy, Dyz) N, z faces (Fz, Dxz, Dyz, Dzz) N.
__device__ __forceinline__ float4 lf_update(const float4* U, const float2* W, const float4& uc,
                                            const float4& um, const float4& pm, const float4& up,
                                            const float4& pp, float cu, float hl) {
  constexpr int RX = kRingRX;
  const float4 uL = U[-1], uR = U[1], uD = U[-RX], uU = U[RX];
  const float2 qL = W[-1], qR = W[1], qD = W[-RX], qU = W[RX];
  const float wL = __fmul_rn(qL.y, uL.y), wR = __fmul_rn(qR.y, uR.y);   // w Fx (x neighbours)
  const float wD = __fmul_rn(qD.y, uD.z), wU = __fmul_rn(qU.y, uU.z);   // w Fy (y neighbours)
  // flux differences per component
  const float fN = (uR.y - uL.y) + (uU.z - uD.z) + (pp.x - pm.x);
  const float fX = (fmaf(wR, uR.y, qR.x) - fmaf(wL, uL.y, qL.x)) +
                   (__fmul_rn(wU, uU.y) - __fmul_rn(wD, uD.y)) + (pp.y - pm.y);
  const float fY = (__fmul_rn(wR, uR.z) - __fmul_rn(wL, uL.z)) +
                   (fmaf(wU, uU.z, qU.x) - fmaf(wD, uD.z, qD.x)) + (pp.z - pm.z);
  const float fZ = (__fmul_rn(wR, uR.w) - __fmul_rn(wL, uL.w)) +
                   (__fmul_rn(wU, uU.w) - __fmul_rn(wD, uD.w)) + (pp.w - pm.w);
  // the neighbour sums and the update in paired FP32 arithmetic (two components per
  // instruction, (N, Fx/c) and (Fy/c, Fz/c), the halves of the vector records)
  const float2 nA = add2(add2(add2(lo2(uR), lo2(uL)), add2(lo2(uU), lo2(uD))),
                         add2(lo2(up), lo2(um)));
  const float2 nB = add2(add2(add2(hi2(uR), hi2(uL)), add2(hi2(uU), hi2(uD))),
                         add2(hi2(up), hi2(um)));
  const float2 mh = make_float2(-hl, -hl), c2 = make_float2(cu, cu);
  const float2 rA = __ffma2_rn(mh, sub2(make_float2(fN, fX), nA), __fmul2_rn(c2, lo2(uc)));
  const float2 rB = __ffma2_rn(mh, sub2(make_float2(fY, fZ), nB), __fmul2_rn(c2, hi2(uc)));
  return make_float4(rA.x, rA.y, rB.x, rB.y);
}

// ---------------------------------------------------------------------------------------
// HLL intercell flux in the fused kernel (section 2.2 offers HLL beside Lax-Friedrichs). Each
// ring slot also keeps its cell's wave-speed bounds (units of c) along x, y and z: the extreme
// eigenvalues of the M1 flux Jacobian (m1_speeds, m1_axis_speeds). The face flux is
//   (l+ Phi_L - l- Phi_R + l+ l- (u_R - u_L)) / (l+ - l-),
//   l- = min(0, lo_L, lo_R), l+ = max(0, hi_L, hi_R),
// with the mean of the two fluxes where l+ - l- vanishes (both cells streaming at f = 1
// parallel to the face, where those fluxes vanish too).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void ring_put_speeds(float2* SX, float2* SY, float2* SZ, int slot,
                                                const float4& u) {
  const M1Speeds m = m1_speeds(u.x, u.y, u.z, u.w);
  float lo, hi;
  m1_axis_speeds(m, m.gx, lo, hi);
  SX[slot] = make_float2(lo, hi);
  m1_axis_speeds(m, m.gy, lo, hi);
  SY[slot] = make_float2(lo, hi);
  m1_axis_speeds(m, m.gz, lo, hi);
  SZ[slot] = make_float2(lo, hi);
}

// Store the record of a slot with its speed bounds along the axes in AX (the fused HLL kernel:
// x, y and z for the tile's own slots, only x or only y for a halo column or row); returns the
// cell's z flux.
template <int AX>
__device__ __forceinline__ float4 ring_put_hll(float4* RU, float2* RW, float2* SX, float2* SY,
                                               float2* SZ, int slot, const float4& u) {
  const float2 q = m1_iso_w_speeds<AX>(u.x, u.y, u.z, u.w, SX + slot, SY + slot, SZ + slot);
  RU[slot] = u;
  RW[slot] = q;
  return z_flux_q(u, q);
}

// fluxes along x and y of a state and its closure pair (along z: z_flux_q)
__device__ __forceinline__ float4 x_flux_q(const float4& u, const float2& q) {
  const float w = __fmul_rn(q.y, u.y);
  return make_float4(u.y, fmaf(w, u.y, q.x), __fmul_rn(w, u.z), __fmul_rn(w, u.w));
}
__device__ __forceinline__ float4 y_flux_q(const float4& u, const float2& q) {
  const float w = __fmul_rn(q.y, u.z);
  return make_float4(u.z, __fmul_rn(w, u.y), fmaf(w, u.z, q.x), __fmul_rn(w, u.w));
}

// Coefficients of the HLL face flux F = a Phi_L + b Phi_R + c (u_R - u_L) for the bounds
// l- <= 0 <= l+ of a face: a = l+ / (l+ - l-), b = -l- / (l+ - l-), c = l+ l- / (l+ - l-); where
// l+ - l- vanishes (both cells streaming at f = 1 parallel to the face, whose fluxes then vanish
// too) the mean, a = b = 1/2, c = 0. Taken once per face, so a component costs three operations.
struct HllCoef {
  float a, b, c;
};
__device__ __forceinline__ HllCoef hll_coef(float lm, float lp) {
  const float d = lp - lm;
  const bool g = d > 1e-6f;
  const float r = rcp_fast(g ? d : 1.f);   // d <= 2
  return g ? HllCoef{lp * r, -lm * r, lp * lm * r} : HllCoef{0.5f, 0.5f, 0.f};
}
__device__ __forceinline__ float hll_face(const HllCoef& k, float PL, float PR, float uL, float uR) {
  return fmaf(k.c, uR - uL, fmaf(k.a, PL, k.b * PR));
}

// (flux through the high face) - (flux through the low face) along one axis, for the centre c
// between its low (l) and high (h) neighbours
__device__ __forceinline__ float4 hll_axis(const float4& fl, const float4& fc, const float4& fh,
                                           const float4& ul, const float4& uc, const float4& uh,
                                           const float2& sl, const float2& sc, const float2& sh) {
  const HllCoef kp = hll_coef(fminf(0.f, fminf(sc.x, sh.x)), fmaxf(0.f, fmaxf(sc.y, sh.y)));
  const HllCoef km = hll_coef(fminf(0.f, fminf(sl.x, sc.x)), fmaxf(0.f, fmaxf(sl.y, sc.y)));
  return make_float4(hll_face(kp, fc.x, fh.x, uc.x, uh.x) - hll_face(km, fl.x, fc.x, ul.x, uc.x),
                     hll_face(kp, fc.y, fh.y, uc.y, uh.y) - hll_face(km, fl.y, fc.y, ul.y, uc.y),
                     hll_face(kp, fc.z, fh.z, uc.z, uh.z) - hll_face(km, fl.z, fc.z, ul.z, uc.z),
                     hll_face(kp, fc.w, fh.w, uc.w, uh.w) - hll_face(km, fl.w, fc.w, ul.w, uc.w));
}

// HLL flux through the face between a cell L and the cell R above it along z (the same numbers
// as hll_axis's faces along z, so that the flux a plane's update computes for its upper face is
// the one the next plane's update needs for its lower face)
__device__ __forceinline__ float4 hll_zface(const float4& uL, const float2& qL, const float2& sL,
                                            const float4& uR, const float2& qR, const float2& sR) {
  const HllCoef k = hll_coef(fminf(0.f, fminf(sL.x, sR.x)), fmaxf(0.f, fmaxf(sL.y, sR.y)));
  const float4 fL = z_flux_q(uL, qL), fR = z_flux_q(uR, qR);
  return make_float4(hll_face(k, fL.x, fR.x, uL.x, uR.x), hll_face(k, fL.y, fR.y, uL.y, uR.y),
                     hll_face(k, fL.z, fR.z, uL.z, uR.z), hll_face(k, fL.w, fR.w, uL.w, uR.w));
}

// HLL update of the centre cell: u' = u - lam sum_d (F_{d,+} - F_{d,-}). U, W, SX, SY, SZ point
// at the centre slot of plane z; the z neighbour above comes as (state, closure pair, z speeds),
// the lower z face's flux fm as carried from the previous plane's update (its upper face, which
// this update returns in fp): one z face evaluated per cell instead of two.
__device__ __forceinline__ float4 hll_update_zc(const float4* U, const float2* W, const float2* SX,
                                                const float2* SY, const float2* SZ,
                                                const float4& uc, const float4& up,
                                                const float2& qp, const float2& szp,
                                                const float4& fm, float4& fp, float lam) {
  constexpr int RX = kRingRX;
  const float2 qc = W[0];
  const float4 uL = U[-1], uR = U[1], uD = U[-RX], uU = U[RX];
  const float4 ax = hll_axis(x_flux_q(uL, W[-1]), x_flux_q(uc, qc), x_flux_q(uR, W[1]), uL, uc,
                             uR, SX[-1], SX[0], SX[1]);
  const float4 ay = hll_axis(y_flux_q(uD, W[-RX]), y_flux_q(uc, qc), y_flux_q(uU, W[RX]), uD,
                             uc, uU, SY[-RX], SY[0], SY[RX]);
  fp = hll_zface(uc, qc, SZ[0], up, qp, szp);
  const float4 az = make_float4(fp.x - fm.x, fp.y - fm.y, fp.z - fm.z, fp.w - fm.w);
  return make_float4(uc.x - lam * ((ax.x + ay.x) + az.x), uc.y - lam * ((ax.y + ay.y) + az.y),
                     uc.z - lam * ((ax.z + ay.z) + az.z), uc.w - lam * ((ax.w + ay.w) + az.w));
}

// ---------------------------------------------------------------------------------------
// Learned chemistry surrogate (a replacement of the operator Phi, Appendix Eq. A4, for cells
// the exact operator sub-cycles heavily).
//
// Gate: a cell is offered to the network when the explicit estimate of its sub-step count from
// photo-ionisation (Gamma y dt over eps max(y, y_floor)) or from photo-heating (over eps T) is
// at least `gate` -- written without quotients -- and its features (log10 nH, log10 y, log10 T,
// log10 N, log10 dt) lie inside the training range. The plain step's gate pass and the fused
// kernel take the same decision with this function.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ bool sur_candidate(const StepParams& P, float gate, const MlpNorm& nm,
                                              float n, float N, float y, float T) {
  const float gy = P.csig * N * y * P.dt;                  // Gamma y dt
  const float lim = gate * P.sub_eps;
  const bool heavy = gy >= lim * fmaxf(y, P.y_floor) ||
                     (!P.fixed_T && gy * P.eheat_K >= lim * T * 1.5f * (2.f - y));
  if (!heavy) return false;
  const float f[kMlpIn] = {log10f(n), log10f(fmaxf(y, 1e-10f)), log10f(T), log10f(fmaxf(N, 1e-30f)),
                           log10f(P.dt)};
  bool inr = true;
#pragma unroll
  for (int i = 0; i < kMlpIn; ++i) inr = inr && f[i] >= nm.in_min[i] && f[i] <= nm.in_max[i];
  return inr;
}

// Decodes the network's normalised outputs o (changes of log10 y, log10 T, log10 N over dt,
// clipped to their training ranges) into (N', y', T') and accepts them only if the photons
// absorbed per atom, (N - N')/nH, match the atoms ionised (y - y') plus the recombinations over
// dt at the mean state within `resid` of max(y, 1e-8).
__device__ __forceinline__ bool sur_accept(const StepParams& P, const MlpNorm& nm, float resid,
                                           const float o[3], float n, float N, float y, float T,
                                           float& N1, float& y1, float& T1) {
  const float dly = fminf(fmaxf(nm.out_mean[0] + o[0] / nm.out_scale[0], -kDlyMax), kDlyMax);
  const float dlT = fminf(fmaxf(nm.out_mean[1] + o[1] / nm.out_scale[1], -kDlTMax), kDlTMax);
  const float dlN = fminf(fmaxf(nm.out_mean[2] + o[2] / nm.out_scale[2], -kDlNMax), 0.f);
  y1 = fminf(fmaxf(fmaxf(y, 1e-10f) * exp2f(3.321928f * dly), 0.f), 1.f);
  T1 = fmaxf(T * exp2f(3.321928f * dlT), P.T_floor);
  N1 = fminf(fmaxf(N, 1e-30f) * exp2f(3.321928f * dlN), N);
  const float xm = 1.f - 0.5f * (y + y1);
  const float am = alpha_B(kLog2TwoTHI - log2f(0.5f * (T + T1)));
  const float rec = am * n * xm * xm * P.dt;
  const float r = fabsf((N - N1) / n - ((y - y1) + rec)) / fmaxf(y, 1e-8f);
  return r <= resid && isfinite(y1) && isfinite(T1) && isfinite(N1);
}

// The network for the cells of one warp (all 32 lanes call this together): the MLP for the
// warp's 32 cells on tensor cores (two 16-row m16n8k16 passes of mlp_infer16_sh with the weights
// W, a shared-memory copy in the fused kernel's tail, activations in the warp's shared-memory
// tiles H1, H2);
// each lane with `cand` set decodes and checks its own prediction. Returns whether this lane's prediction
// was accepted (then N1, y1, T1 hold it). Features are exchanged with shuffles: lane (g, t) of a
// 16-row pass needs features 2t, 2t+1 of rows g and g+8, and a row's three outputs sit in the
// lanes 4 (row mod 8) and 4 (row mod 8) + 1.
__device__ __forceinline__ bool sur_warp(const StepParams& P, const SurList& S, const MlpImage& W,
                                         bool cand, float n, float N, float y, float T, float& N1,
                                         float& y1, float& T1, __nv_bfloat16* H1,
                                         __nv_bfloat16* H2) {
  const unsigned full = 0xffffffffu;
  const MlpNorm& nm = *S.norm;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float f[kMlpIn] = {log10f(n), log10f(fmaxf(y, 1e-10f)), log10f(T), log10f(fmaxf(N, 1e-30f)),
                     log10f(P.dt)};
#pragma unroll
  for (int i = 0; i < kMlpIn; ++i) f[i] = (f[i] - nm.in_mean[i]) * nm.in_scale[i];
  float o[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int ra = half * 16 + g, rb = ra + 8;
    float fa[kMlpIn], fb[kMlpIn];
#pragma unroll
    for (int i = 0; i < kMlpIn; ++i) {
      fa[i] = __shfl_sync(full, f[i], ra);
      fb[i] = __shfl_sync(full, f[i], rb);
    }
    // columns 2t, 2t+1 of the 16-wide (5 used) input tile
    const float a0 = t == 0 ? fa[0] : (t == 1 ? fa[2] : (t == 2 ? fa[4] : 0.f));
    const float a1 = t == 0 ? fa[1] : (t == 1 ? fa[3] : 0.f);
    const float b0 = t == 0 ? fb[0] : (t == 1 ? fb[2] : (t == 2 ? fb[4] : 0.f));
    const float b1 = t == 0 ? fb[1] : (t == 1 ? fb[3] : 0.f);
    const unsigned a[4] = {pack_bf16(a0, a1), pack_bf16(b0, b1), 0u, 0u};
    float yo[4];
    mlp_infer16_sh(W, a, H1, H2, yo);
    const int r = lane - half * 16;
    const int s0 = 4 * (r & 7);
    const float c0 = __shfl_sync(full, yo[0], s0), c1 = __shfl_sync(full, yo[1], s0);
    const float c2 = __shfl_sync(full, yo[2], s0), c3 = __shfl_sync(full, yo[3], s0);
    const float d0 = __shfl_sync(full, yo[0], s0 + 1), d2 = __shfl_sync(full, yo[2], s0 + 1);
    if (r >= 0 && r < 16) {
      const bool hi = r >= 8;
      o[0] = hi ? c2 : c0;
      o[1] = hi ? c3 : c1;
      o[2] = hi ? d2 : d0;
    }
  }
  return cand && sur_accept(P, nm, S.resid, o, n, N, y, T, N1, y1, T1);
}

// The fused kernel's deferral (the chem_cell hook): a candidate goes to the CTA's list, a region
// of device memory of its own (global atomics on a rare path: shared-memory atomics in the plane
// loop would tie the compiler's hands on the ring accesses, which measured 12 % slower).
struct SurDefer {
  const StepParams& P;
  const SurList& S;
  SurRec* buf;
  int* cnt;
  int o;
  __device__ __forceinline__ bool operator()(float n, float N, float fx, float fy, float fz,
                                             float y, float T) const {
    if (!sur_candidate(P, S.gate, *S.norm, n, N, y, T)) return false;
    const int k = atomicAdd(cnt, 1);
    if (k >= kSurCap) return false;
    buf[k] = SurRec{N, fx, fy, fz, y, T, n, o};
    return true;
  }
};

// Chemistry of the transported cell, its tallies and the store of the new state (physical F:
// the chemistry scales F / c by its photon ratio times c). With `sur` set the cell takes the
// network's accepted prediction (N1, y1, T1; F scaled with N) instead of the exact operator.
// With a deferral `defer` (SurDefer) a selected cell is listed (and overwritten later).
template <bool STD, class Defer = NoDefer>
__device__ __forceinline__ void chem_tally_store(const StepParams& P, Tally& tl, float cn, float4 u,
                                                 float cy, float cT, const Fields& out, float* Yf,
                                                 float* Tf, long long o, bool sur = false,
                                                 float N1 = 0.f, float y1 = 0.f, float T1 = 0.f,
                                                 const Defer& defer = Defer()) {
  float Nn = u.x, Xn = u.y, Yn = u.z, Zn = u.w;
  const float N0 = Nn;
  ChemOut co{0, 0};
  if (sur) {
    const float fr = (N0 > 0.f ? N1 / N0 : 1.f) * P.c;
    Nn = N1; Xn *= fr; Yn *= fr; Zn *= fr; cy = y1; cT = T1;
    tl.sur += 1;
  } else {
    // (a deferred cell comes back untouched, F still as F / c, with no sub-steps: it is stored
    // and tallied like that -- no absorption -- and its CTA's surrogate pass overwrites it; an
    // early return here made every store and tally conditional and cost 12 % of the step)
    co = chem_cell<STD>(P, cn, Nn, Xn, Yn, Zn, cy, cT, P.c, defer);
  }
  tl.absorbed.add(N0 - Nn);
  tl.sub += co.nsub;
  tl.mx = max(tl.mx, (unsigned)co.nsub);
  tl.err += co.err;
  // one test: a NaN or an infinity in any of them makes the sum non-finite
  if (!isfinite(Nn + cT + (Xn + Yn + Zn))) tl.nan += 1;
  out.N[o] = Nn; out.Fx[o] = Xn; out.Fy[o] = Yn; out.Fz[o] = Zn;
  Yf[o] = cy; Tf[o] = cT;
}

// The end of a fused CTA with the surrogate: its listed cells, 32 per warp (warps 0 and 1),
// run through the network; accepted predictions are stored, the others take the exact operator
// (their latency overlaps with the other CTAs on the SM). Called by every thread of the CTA
// after its z-loop. `scratch`: shared memory free by then (the stage and plane rings), 16-byte
// aligned, at least sizeof(MlpImage) bytes. A CTA with listed cells first copies the forward
// weights and biases into it with one coalesced pass (the network's weight reads would otherwise
// be dependent round trips to L2, about 44 per 16 rows), laid out as an MlpImage whose backward
// blocks (W2T, W3T) are not copied and hold the two warps' activation tiles instead.
constexpr int kSurScratchBytes = (int)sizeof(MlpImage);
static_assert(2 * 2 * 16 * kP2 * 2 <= sizeof(MlpImage::W2T) + sizeof(MlpImage::W3T),
              "activation tiles fit in the backward blocks");
template <bool STD>
__device__ __forceinline__ void sur_tail(const StepParams& P, const SurList& S, const SurRec* buf,
                                         int* cnt, Tally& tl, const Fields& out, float* Yf,
                                         float* Tf, void* scratch) {
  static_assert(kSurCap <= 64, "two warps run the list");
  __syncthreads();   // (orders the list's writes, global memory included, before its reads)
  const int nc = min(*reinterpret_cast<volatile int*>(cnt), kSurCap);
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  if (nc == 0) return;   // (uniform over the CTA)
  MlpImage& Ws = *reinterpret_cast<MlpImage*>(scratch);
  {
    constexpr int kFwd = (int)(offsetof(MlpImage, W2T) / 16);            // W1, W2, W3
    constexpr int kBias0 = (int)(offsetof(MlpImage, b1) / 16);
    constexpr int kBias1 = (int)((sizeof(MlpImage) + 15) / 16);
    const uint4* src = reinterpret_cast<const uint4*>(S.img);
    uint4* dst = reinterpret_cast<uint4*>(&Ws);
    for (int i = tid; i < kFwd; i += nthr) dst[i] = src[i];
    for (int i = kBias0 + tid; i < kBias1; i += nthr) dst[i] = src[i];
  }
  __syncthreads();
  const int w = tid >> 5, lane = tid & 31;
  if (w < 2 && w * 32 < nc) {   // (uniform within the warp)
    __nv_bfloat16* H1 = reinterpret_cast<__nv_bfloat16*>(&Ws.W2T[0]) + w * 2 * 16 * kP2;
    __nv_bfloat16* H2 = H1 + 16 * kP2;
    const int k = w * 32 + lane;
    const bool valid = k < nc;
    const SurRec r = valid ? buf[k] : SurRec{0.f, 0.f, 0.f, 0.f, 1.f, 1e4f, 1.f, 0};
    float N1 = 0.f, y1 = 0.f, T1 = 0.f;
    const bool acc = sur_warp(P, S, Ws, valid, r.n, r.N, r.y, r.T, N1, y1, T1, H1, H2);
    if (valid)
      chem_tally_store<STD>(P, tl, r.n, make_float4(r.N, r.X, r.Y, r.Z), r.y, r.T, out, Yf, Tf,
                            r.o, acc, N1, y1, T1);
  }
  // the next step's list starts empty (every thread has read the count)
  __syncthreads();
  if (tid == 0) *cnt = 0;
}

}  // namespace aton
