// aton_device.cuh -- FP32 device arithmetic of one ATON step: the M1 closure, the rate fits
// and the sub-cycled chemistry/cooling/absorption operator of one cell.
//
// Device memory holds the physical flux F; the kernels scale it to Fh = F / c in registers so
// that N and Fh share units and the transport needs the single constant lambda = c dt / dx.
// Per-atom energies are carried in kelvin (energy / kB) so every quantity stays well inside
// the FP32 range for nH from 1e-9 to 1e3.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace aton {

// Parameters of one step, passed by value to the kernels.
struct StepParams {
  int nx, ny, nz;
  int bc;              // 0 periodic, 1 transmissive
  float lam;           // c dt / dx
  float c, rc;         // speed of light and its reciprocal (F <-> Fh in registers)
  float dt;            // radiative step [s]
  float csig;          // c sigma_n [cm^3 s^-1]
  float eheat_K;       // heat per photo-ionisation / kB [K]
  int fixed_T, coll_ion, cooling, max_sub;
  float T_floor, sub_eps, y_floor;
  float clR_A, clR_b, clI_A, clI_b;
  int hll;             // intercell flux: 0 global Lax-Friedrichs, 1 HLL (plain step only)
  float quiet_k;       // bound of alpha_B(T) and (rec(T) + ff(T)) / (1.5 T), T_floor..kTExcMin
  // constants of the one-sub-step chemistry shortcut, folded on the host:
  float quiet_dt;      // dt quiet_k 2^26
  float heat_eps;      // eheat_K / (1.5 sub_eps)
  float eheat15;       // eheat_K / 1.5
};

// ---------------------------------------------------------------------------------------
// M1 closure (section 2.2, Eqs. 5-6, chi from f = |F|/(cN) between 1/3 and 1; Levermore
// chi = (3 + 4f^2) / (5 + 2 s), s = sqrt(4 - 3 f^2); Eddington tensor read with the
// coefficients swapped relative to the printed Eq. 6 so that D = I/3 at chi = 1/3).
// Written without cancellation for small f: with g = Fh / N,
//   N D = N [ (1 - chi)/2 I + c2 g (x) g ],   (1 - chi)/2 = (1 + s - 2 f^2) / (5 + 2 s),
//   c2 = (3 chi - 1) / (2 f^2) = 3 (2 + 1/(2 + s)) / (5 + 2 s),
// which follows from 4 - 2 s = 6 f^2 / (2 + s).
// ---------------------------------------------------------------------------------------
struct ND6 {
  float xx, yy, zz, xy, xz, yz;
};

// Below kNTiny (photons cm^-3) the cell holds no radiation worth transporting and 1/N would
// leave the FP32 range (N reaches the denormals ahead of fronts through the scheme's
// diffusion); there D = I/3 (f = 0) is used. Unrealisable inputs with |Fh| > N take f = 1
// along Fh, as D = n (x) n requires.
constexpr float kNTiny = 1e-30f;

// Hardware reciprocal and quotient (a couple of ulp). Used only where the divisor is a
// positive normal FP32 number well inside the range (every call site states why).
__device__ __forceinline__ float rcp_fast(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float div_fast(float a, float b) { return __fdividef(a, b); }

__device__ __forceinline__ ND6 m1_pressure(float N, float fx, float fy, float fz) {
  ND6 r;
  if (N > kNTiny) {
    const float rN = rcp_fast(N);   // N in (1e-30, 8e37): the reciprocal stays normal
    float gx = fx * rN, gy = fy * rN, gz = fz * rN;
    float f2 = gx * gx + gy * gy + gz * gz;
    if (f2 > 1.f) {
      const float k = rsqrtf(f2);
      gx *= k; gy *= k; gz *= k;
      f2 = 1.f;
    }
    const float s = sqrtf(4.f - 3.f * f2);        // in [1, 2]
    const float r5N = rcp_fast(5.f + 2.f * s) * N;
    const float iso = (1.f + s - 2.f * f2) * r5N;
    const float Nc2 = fmaf(3.f, rcp_fast(2.f + s), 6.f) * r5N;
    const float ax = Nc2 * gx, ay = Nc2 * gy;
    r.xx = fmaf(ax, gx, iso);
    r.yy = fmaf(ay, gy, iso);
    r.zz = fmaf(Nc2 * gz, gz, iso);
    r.xy = ax * gy;
    r.xz = ax * gz;
    r.yz = ay * gz;
  } else {
    const float iso = N > 0.f ? N * (1.f / 3.f) : 0.f;
    r.xx = r.yy = r.zz = iso;
    r.xy = r.xz = r.yz = 0.f;
  }
  return r;
}

// The same closure as the pair (iso, w) with N D = iso I + w Fh (x) Fh: iso = N (1 - chi)/2 and
// w = c2 / N (c2 as above; divided by f^2 where |Fh| > N, since D then takes g = Fh / |Fh|).
// The fused kernels keep this pair per cell (two floats instead of six) and form the components
// they need from it. w stays normal for N below ~6e37 (c2 >= 3/4).
// Written without branches (the fused kernels evaluate it for every slot of a plane): the
// closure of an empty cell (N <= kNTiny) is evaluated on a stand-in N = 1 and replaced by the
// isotropic pair at the end, and the f > 1 rescaling is a selection.
__device__ __forceinline__ float2 m1_iso_w(float N, float fx, float fy, float fz) {
  const bool rad = N > kNTiny;
  const float rN = rcp_fast(rad ? N : 1.f);   // N in (1e-30, 8e37): the reciprocal stays normal
  const float gx = fx * rN, gy = fy * rN, gz = fz * rN;
  float f2 = gx * gx + gy * gy + gz * gz;
  const float k = f2 > 1.f ? rN * rcp_fast(f2) : rN;   // f2 in (1, 3e38]: a normal reciprocal
  f2 = fminf(f2, 1.f);
  const float s = sqrtf(4.f - 3.f * f2);        // in [1, 2]
  const float r5 = rcp_fast(5.f + 2.f * s);
  const float iso = (1.f + s - 2.f * f2) * (r5 * N);
  const float w = fmaf(3.f, rcp_fast(2.f + s), 6.f) * r5 * k;
  return rad ? make_float2(iso, w) : make_float2(N > 0.f ? N * (1.f / 3.f) : 0.f, 0.f);
}

// ---------------------------------------------------------------------------------------
// Extreme characteristic speeds (units of c) of the M1 flux Jacobian along an axis, the wave-
// speed bounds of the HLL flux (section 2.2). With f = |Fh|/N, mu the cosine between Fh and the
// axis, chi(f) and chi'(f) of the Levermore closure, the Jacobian's characteristic polynomial
// has the transverse root (3 chi - 1) mu / (2 f) and the pair
//   lambda = (chi' mu -/+ sqrt((chi' mu)^2 - C)) / 2,
//   C = (1 - mu^2)((3 chi - 1) chi'/f - 2) + 2 chi (1 - 3 mu^2) + 2 chi' f (3 mu^2 - 1),
// which bound all four (+-1/sqrt(3) at f = 0, mu at f = 1). Written without division by f:
// chi'/f = (8 (5 + 2s) + 6 (3 + 4 f^2)/s) / (5 + 2s)^2 and 3 chi - 1 = f^2 (6/(2 + s) + 12)/(5 + 2s)
// with s = sqrt(4 - 3 f^2), and chi' mu = (chi'/f) g_axis for g = Fh/N (g_axis = f mu).
// ---------------------------------------------------------------------------------------
struct M1Speeds {
  float gx, gy, gz;   // Fh / N, |g| <= 1 (0 below kNTiny)
  float f2;           // |g|^2
  float chi, dcf, P1; // chi, chi'/f, (3 chi - 1) chi'/f - 2
};

__device__ __forceinline__ M1Speeds m1_speeds(float N, float fx, float fy, float fz) {
  M1Speeds m;
  m.gx = m.gy = m.gz = 0.f;
  m.f2 = 0.f;
  if (N > kNTiny) {
    const float rN = rcp_fast(N);
    m.gx = fx * rN; m.gy = fy * rN; m.gz = fz * rN;
    m.f2 = m.gx * m.gx + m.gy * m.gy + m.gz * m.gz;
    if (m.f2 > 1.f) {
      const float k = rsqrtf(m.f2);
      m.gx *= k; m.gy *= k; m.gz *= k;
      m.f2 = 1.f;
    }
  }
  const float s = sqrtf(4.f - 3.f * m.f2);          // in [1, 2]
  const float r5 = rcp_fast(5.f + 2.f * s);
  m.chi = (3.f + 4.f * m.f2) * r5;
  m.dcf = fmaf(6.f * (3.f + 4.f * m.f2), rcp_fast(s), 8.f * (5.f + 2.f * s)) * r5 * r5;
  const float tcm1 = m.f2 * fmaf(6.f, rcp_fast(2.f + s), 12.f) * r5;   // 3 chi - 1
  m.P1 = tcm1 * m.dcf - 2.f;
  return m;
}

// speeds along the axis whose component of g is gd
__device__ __forceinline__ void m1_axis_speeds(const M1Speeds& m, float gd, float& lo, float& hi) {
  const float mu2 = m.f2 > 1e-30f ? fminf(div_fast(gd * gd, m.f2), 1.f) : 0.f;
  const float C = (1.f - mu2) * m.P1 + 2.f * m.chi * (1.f - 3.f * mu2) +
                  2.f * m.dcf * m.f2 * (3.f * mu2 - 1.f);
  const float b = m.dcf * gd;
  const float r = sqrtf(fmaxf(b * b - C, 0.f));
  lo = 0.5f * (b - r);
  hi = 0.5f * (b + r);
}

// The closure pair of m1_iso_w and the HLL wave-speed bounds (lo, hi) of m1_speeds /
// m1_axis_speeds along the axes in the mask AX (bit 0 x, bit 1 y, bit 2 z) in one pass: the
// reciprocal of N, f^2, s = sqrt(4 - 3 f^2) and 1/(5 + 2 s) serve both (the fused HLL kernel
// evaluates it for every ring slot; a halo slot needs the speeds along one axis only). An empty
// cell (N <= kNTiny) takes the isotropic pair and the speeds of f = 0, +-1/sqrt(3).
template <int AX>
__device__ __forceinline__ float2 m1_iso_w_speeds(float N, float fx, float fy, float fz,
                                                  float2* sx, float2* sy, float2* sz) {
  const bool rad = N > kNTiny;
  const float rN = rcp_fast(rad ? N : 1.f);   // N in (1e-30, 8e37): the reciprocal stays normal
  float gx = fx * rN, gy = fy * rN, gz = fz * rN;
  const float f2r = gx * gx + gy * gy + gz * gz;
  const bool over = f2r > 1.f;
  const float k = over ? rN * rcp_fast(f2r) : rN;   // f2 in (1, 3e38]: a normal reciprocal
  const float f2 = rad ? fminf(f2r, 1.f) : 0.f;
  const float s = sqrtf(4.f - 3.f * f2);        // in [1, 2]
  const float r5 = rcp_fast(5.f + 2.f * s);
  const float r2 = rcp_fast(2.f + s);
  const float iso = (1.f + s - 2.f * f2) * (r5 * N);
  const float w = fmaf(3.f, r2, 6.f) * r5 * k;
  // speeds: g on the unit sphere where |g| > 1, zero for an empty cell
  const float gs = rad ? (over ? rsqrtf(f2r) : 1.f) : 0.f;
  gx *= gs; gy *= gs; gz *= gs;
  const float chi = (3.f + 4.f * f2) * r5;
  const float dcf = fmaf(6.f * (3.f + 4.f * f2), rcp_fast(s), 8.f * (5.f + 2.f * s)) * r5 * r5;
  const float P1 = f2 * fmaf(6.f, r2, 12.f) * r5 * dcf - 2.f;   // (3 chi - 1) chi'/f - 2
  const float rf2 = f2 > 1e-30f ? rcp_fast(f2) : 0.f;          // f2 in (1e-30, 1]
  auto axis = [&](float gd) {
    const float mu2 = fminf(gd * gd * rf2, 1.f);
    const float C = (1.f - mu2) * P1 + 2.f * chi * (1.f - 3.f * mu2) +
                    2.f * dcf * f2 * (3.f * mu2 - 1.f);
    const float b = dcf * gd;
    const float r = sqrtf(fmaxf(b * b - C, 0.f));
    return make_float2(0.5f * (b - r), 0.5f * (b + r));
  };
  if (AX & 1) *sx = axis(gx);
  if (AX & 2) *sy = axis(gy);
  if (AX & 4) *sz = axis(gz);
  return rad ? make_float2(iso, w) : make_float2(N > 0.f ? N * (1.f / 3.f) : 0.f, 0.f);
}

// ---------------------------------------------------------------------------------------
// Rate fits (the paper defers to Anninos et al. 1997 and Cen 1992; section 2.2). Hui & Gnedin
// (1997) fits in lambda = 2 T_HI / T, evaluated in log2 form, plus Cen (1992) collisional
// excitation and bremsstrahlung. Cooling coefficients are returned divided by kB.
// ---------------------------------------------------------------------------------------
constexpr float kLog2TwoTHI = 18.267801676f;   // log2(2 * 157807 K)
constexpr float kLog2e = 1.442695041f;
constexpr float kLog10of2 = 0.301029996f;
constexpr float kTHI = 157807.f;
constexpr double kKB = 1.380649e-16;           // erg / K
// Below these temperatures exp(-157807/T) (collisional ionisation) and exp(-118348/T)
// (collisional excitation) are under the smallest normal FP32 number and flush to exactly 0.
constexpr float kTBetaMin = 1700.f;
constexpr float kTExcMin = 1300.f;

// case-B recombination rate [cm^3 s^-1]; l = log2(lambda)
__device__ __forceinline__ float alpha_B(float l) {
  const float q = exp2f(0.407f * (l - 1.454175893f));              // (lambda / 2.740)^0.407
  return 2.753e-14f * exp2f(1.5f * l - 2.242f * log2f(1.f + q));
}

// collisional ionisation rate of HI [cm^3 s^-1]; l = log2(lambda), l2T = log2(T), rT = 1/T
__device__ __forceinline__ float beta_coll(float l, float l2T, float rT) {
  const float q = exp2f(0.874f * (l + 1.498178735f));              // (lambda / 0.354)^0.874
  return 21.11f * exp2f(-1.5f * l2T - (kTHI * kLog2e) * rT - 1.089f * l - 1.101f * log2f(1.f + q));
}

// net cooling per H atom / kB [K s^-1] at (T, x, y = 1 - x, nH), with recombination clumping CR
__device__ __forceinline__ float cooling_K(float T, float l, float l2T, float rT, float x, float y,
                                           float n, float CR, bool coll_ion) {
  // case-B recombination cooling (Hui & Gnedin 1997), times n_e n_HII; the factor T enters the
  // exponent as log2 T
  const float qr = exp2f(0.376f * (l - 1.169925001f));
  const float rec = (float)(3.435e-30 / kKB) * exp2f(1.970f * l + l2T - 3.720f * log2f(1.f + qr));
  // collisional excitation (Cen 1992), times n_e n_HI (exactly 0 in FP32 below kTExcMin);
  // the divisor is in [1, 1 + sqrt(T/1e5)]
  const float ce = T > kTExcMin ? div_fast((float)(7.5e-19 / kKB) * exp2f(-(118348.f * kLog2e) * rT),
                                           1.f + sqrtf(T * 1e-5f))
                                 : 0.f;
  // bremsstrahlung with the Cen (1992) Gaunt factor, times n_e n_HII; sqrt T = 2^(l2T / 2)
  const float d = l2T * kLog10of2 - 5.5f;
  const float gff = 1.1f + 0.34f * exp2f(-(kLog2e / 3.f) * d * d);
  const float ff = (float)(1.42e-27 / kKB) * gff * exp2f(0.5f * l2T);
  float lx2 = CR * rec + ff;
  float lxy = ce;
  if (coll_ion && T > kTBetaMin) lxy += kTHI * beta_coll(l, l2T, rT);   // 13.6 eV each
  return n * x * (x * lx2 + y * lxy);
}

// ---------------------------------------------------------------------------------------
// Chemistry, photo-heating, cooling and absorption of one cell over dt: the operator Phi of
// Appendix Eq. A4, sub-cycled (section 2.2, chemistry paragraph) with backward-difference
// creation/destruction updates in the spirit of Anninos et al. (1997), for the balance of
// section 3.2.1 Eq. 14 in y = 1 - x:
//   y' - y = h [CR alpha nH x'^2 - CI c sigma_n N' y' - beta nH x y'],
//   N' = N / (1 + nH k y'),  k = CI c sigma_n h   (photons removed = photo-ionisations).
// g(y') = y' - y - a (1-y')^2 + k N y'/(1 + m y') + b y' is concave and increasing on [0,1]
// with g(0) <= 0 <= g(1); Newton from y converges monotonically after at most one step.
// Energy per atom / kB: e = 1.5 (1+x) T; e' = e + (N - N')/nH * eheat_K - h L(T) T'/T.
// The sub-step is the largest h <= remaining with |dy/dt| h <= eps max(y, y_floor) and
// (heating + cooling) h <= eps T (gross rates; dropped for gas at the floor that would cool)
// at the start of the sub-step; the last sub-step ends exactly at dt.
// ---------------------------------------------------------------------------------------
struct ChemOut {
  int nsub;
  int err;
  int deferred = 0;   // the cell was handed to a later pass (its state untouched)
};

// Hook of chem_cell for a cell that does not take the one-sub-step shortcut: returning true
// hands the cell, with its state untouched, to a later pass (the surrogate's, in the fused
// kernel). The default hands nothing on.
struct NoDefer {
  __device__ __forceinline__ bool operator()(float, float, float, float, float, float,
                                             float) const {
    return false;
  }
};

// STD selects the standard configuration at compile time (evolving temperature with cooling
// and collisional ionisation, no clumping), so its flag tests and clumping factors fold away;
// the kernels take it when the step's parameters are that configuration.
// F (any units) decays with N; fs is an extra factor applied with that ratio (a unit change the
// caller wants on the way out, e.g. c to turn F / c back into F).
// `defer(n, N, fx, fy, fz, y, T)` is asked once for a cell off the one-sub-step shortcut.
template <bool STD = false, class Defer = NoDefer>
__device__ __forceinline__ ChemOut chem_cell(const StepParams& P, float n, float& N, float& fx,
                                             float& fy, float& fz, float& y, float& T,
                                             float fs = 1.f, const Defer& defer = Defer()) {
  const bool fixedT = STD ? false : P.fixed_T != 0;
  const bool cool = STD ? true : P.cooling != 0;
  const bool coll = STD ? true : P.coll_ion != 0;
  float CR = 1.f, CI = 1.f;
  if (!STD && P.clR_A > 0.f) CR = fmaxf(1.f, P.clR_A * exp2f(P.clR_b * log2f(n)));
  if (!STD && P.clI_A > 0.f) CI = fmaxf(1.f, P.clI_A * exp2f(P.clI_b * log2f(n)));
  const float ksig = CI * P.csig;
  const float CRn = CR * n;
  // Remaining time as an unevaluated float pair rh + rl (error-free TwoSum updates): a plain
  // FP32 "rem -= h" stalls once h < ulp(rem)/2 (about 4e3 s for dt ~ 1e11 s, while dense gas
  // can need sub-steps of 1e3 s), and rounding h to coarse ticks would change the sequence.
  float rh = P.dt, rl = 0.f;
  const float N0 = N;
  float Nc = N, Tc = T, yc = fminf(fmaxf(y, 0.f), 1.f);
  float Nh = N, Nl = 0.f;   // N as an unevaluated pair Nh + Nl
  ChemOut o{0, 0};
  // One-sub-step shortcut: the step the loop below takes when its first sub-step is quiet and
  // spans the whole step: cold gas (T_floor to kTExcMin, no collisional terms) passing the
  // loop's quiet test with rem = dt, and neither sub-step limit binding. The loop then takes
  // one sub-step h = dt with a = b = 0, whose balance g = kN y'/(1 + m y') - d = 0 (y' = y - d,
  // m = nH c sigma dt, kN = c sigma N dt = Gam dt) is the quadratic
  //   m y'^2 + (1 + kN - m y) y' - y = 0,
  // solved here in closed form (its root in [0, y], written without cancellation for either
  // sign of B = 1 + kN - m y), with d taken back from the balance so that it keeps its full
  // relative precision. Where kN <= 2^-26, d <= kN y is under half an ulp of y and y' = y.
  // The absorption N' = N / (1 + m y') and the temperature update are the loop's own.
  {
    const float xi = 1.f - yc, dt = P.dt;
    constexpr float kHalfUlp = 1.4901161e-8f;   // 2^-26
    const float kk = ksig * dt;
    const float kN = kk * Nc;
    const float gr = fminf(kN, 1.f);
    const float xm = fmaf(gr, yc, xi);
    const float gy = kN * yc;
    // (the quiet test and the heating limit with their constants folded on the host)
    if (Tc < kTExcMin && Tc >= P.T_floor && CRn * P.quiet_dt * xm * xm <= yc * (1.f - gr) &&
        gy <= P.sub_eps * fmaxf(yc, P.y_floor) &&
        (fixedT || gy * P.heat_eps <= Tc * (1.f + xi))) {
      // (here kN < 1: the quiet test fails at gr = 1)
      const float m = n * kk;
      float Y = yc;
      if (kN > kHalfUlp) {
        const float B = 1.f + kN - m * yc;
        const float sD = sqrtf(fmaf(B, B, 4.f * m * yc));
        // B >= 0: B + sD in [1, 4]; B < 0: m y > 1 + kN, so m > 0
        const float Yq = B >= 0.f ? div_fast(2.f * yc, B + sD) : div_fast(sD - B, 2.f * m);
        Y = yc - div_fast(kN * Yq, fmaf(m, Yq, 1.f));
      }
      const float mY = m * Y;
      const float q = rcp_fast(1.f + mY);   // 1 + mY >= 1
      const float r = mY * q;
      const float dN = Nc * r;
      // N' / N = 1 - r, or 1 / (1 + m y') for a large absorbed fraction
      const float fN = r > 0.5f ? q : 1.f - r;
      const float Nn = r > 0.5f ? Nc * q : Nc - dN;
      if (!fixedT)   // T' = e' / (1.5 (1 + x')): the loop's update with the 1.5 folded
        T = fmaxf(div_fast(fmaf(div_fast(dN, n), P.eheat15, (1.f + xi) * Tc), 2.f - Y),
                  P.T_floor);
      const float fr = fN * fs;
      N = Nn;
      fx *= fr;
      fy *= fr;
      fz *= fr;
      y = Y;
      return ChemOut{1, 0};
    }
  }
  if (defer(n, Nc, fx, fy, fz, yc, Tc)) return ChemOut{0, 0, 1};
  while (rh > 0.f) {
    if (o.nsub >= P.max_sub) {
      o.err = 1;
      break;
    }
    const float rem = rh;
    const float xi = 1.f - yc;
    const float Gam = ksig * Nc;
    // Cold gas (T_floor to kTExcMin, where the collisional terms are exactly 0 in FP32) whose
    // recombinations and cooling over the rest of the step would change y and T by less than
    // 2^-26 relatively: those rates are not evaluated, their terms are below half an ulp of
    // the float result (quiet_k bounds alpha_B(T) and (rec(T) + ff(T)) / (1.5 T) there). The
    // recombinations enter the implicit update at the end state, whose ionised fraction the
    // photo-ionisations may raise to at most xm = x + min(Gam rem, 1) y (and y' >= (1 - that) y),
    // so the test takes xm: the dropped term a xm^2 stays under 2^-26 y'. (Cooling enters at the
    // start state x.)
    const float gr = fminf(Gam * rem, 1.f);
    const float xm = fmaf(gr, yc, xi);
    const bool quiet = Tc < kTExcMin && Tc >= P.T_floor &&
                       rem * CRn * xm * xm * P.quiet_k <=
                           1.4901161e-8f * yc * (1.f - gr);
    float l2T = 0.f, rT = 0.f, l = 0.f, an = 0.f, bn = 0.f;
    if (!quiet) {
      l2T = log2f(Tc);
      rT = rcp_fast(Tc);   // T_floor <= Tc < FP32 max (validated input, floored update)
      l = kLog2TwoTHI - l2T;
      an = CRn * alpha_B(l);   // C_R alpha nH
      // the collisional rate is exactly 0 in FP32 below kTBetaMin, so it is not evaluated there
      bn = (coll && Tc > kTBetaMin) ? n * beta_coll(l, l2T, rT) : 0.f;
    }
    const float dydt = an * xi * xi - (Gam + bn * xi) * yc;
    float h = rem;
    const float ymax = fmaxf(yc, P.y_floor);
    const float ady = fabsf(dydt);
    // (the quotients below are taken only when the limit binds: the divisor is then positive
    // and finite)
    if (ady * h > P.sub_eps * ymax) h = div_fast(P.sub_eps * ymax, ady);
    float LK = 0.f;
    if (!fixedT) {
      if (cool && !quiet) LK = cooling_K(Tc, l, l2T, rT, xi, yc, n, CR, coll);
      // gross rate: heating and cooling each bounded (no cancellation near thermal balance);
      // (heat + LK) / (1.5 (1 + x)) h <= eps T written without the quotient
      const float heat = Gam * yc * P.eheat_K;
      const float gross = heat + LK;
      const float cap = P.sub_eps * Tc * (1.5f * (1.f + xi));
      const bool pinned = Tc <= P.T_floor && heat < LK;   // cannot cool below the floor
      if (!pinned && gross * h > cap) h = div_fast(cap, gross);
    }
    const bool last = !(h < rem);   // the last sub-step ends exactly at dt
    const float a = h * an;
    const float b = h * bn * xi;
    const float kk = ksig * h;
    const float m = n * kk;
    const float kN = kk * Nc;
    // Newton on the change d = y - y' (no cancellation in y' - y when the change is small):
    // g = -d - a (x + d)^2 + kN y'/(1 + m y') + b y', dg/dd = -(1 + 2a(x+d) + kN/(1+my')^2 + b)
    // <= -1, |d2g/dd2| <= 2 (a + kN m). The iteration stops when the step just taken, or the
    // next one predicted from it (at most (a + kN m) step^2), is below 3e-7 |d|.
    const float Mq = a + kN * m;
    float d = 0.f;
    for (int it = 0; it < 40; ++it) {
      const float Yv = yc - d;
      const float omY = xi + d;
      const float rd = rcp_fast(1.f + m * Yv);   // 1 + m y' >= 1
      const float kNr = kN * rd;
      const float g = (kNr + b) * Yv - d - a * omY * omY;
      const float gp = 1.f + 2.f * a * omY + kNr * rd + b;
      const float dn = fminf(fmaxf(d + div_fast(g, gp), yc - 1.f), yc);   // gp >= 1
      const float dd = fabsf(dn - d);
      d = dn;
      if (fminf(Mq * dd, 1.f) * dd <= 3e-7f * fabsf(d)) break;
    }
    const float Y = yc - d;
    // photons absorbed in the sub-step: N r with r = m y'/(1 + m y'). N keeps full relative
    // precision either way: a large fraction is applied as N/(1 + m y') (no cancellation), a
    // small one (down to r << ulp(1)) is subtracted from the pair with an error-free TwoSum.
    const float mY = m * Y;
    const float r = div_fast(mY, 1.f + mY);
    const float dN = Nc * r;
    if (r > 0.5f) {
      Nh = div_fast(Nc, 1.f + mY);
      Nl = 0.f;
    } else {
      const float sm = Nh - dN;
      const float bv = sm - Nh;
      const float er = (Nh - (sm - bv)) + (-dN - bv);
      const float lo = Nl + er;
      Nh = sm + lo;
      Nl = lo - (Nh - sm);
    }
    Nh = fmaxf(Nh, 0.f);
    const float Nn = Nh + Nl;
    if (!fixedT) {
      // den >= 1.5 and bounded by the sub-step rule
      const float num = 1.5f * (1.f + xi) * Tc + div_fast(dN, n) * P.eheat_K;
      const float den = 1.5f * (2.f - Y) + h * LK * rT;
      Tc = fmaxf(div_fast(num, den), P.T_floor);
    }
    Nc = Nn;
    yc = Y;
    ++o.nsub;
    if (last) {
      rh = 0.f;
    } else {  // rh + rl -= h, TwoSum then renormalise
      const float sm = rh - h;
      const float bv = sm - rh;
      const float er = (rh - (sm - bv)) + (-h - bv);
      const float lo = rl + er;
      rh = sm + lo;
      rl = lo - (rh - sm);
    }
  }
  // F decays by the same factor as N in every sub-step, so by N_final / N_0 overall (after the
  // realisability clamp N = 0 implies F = 0)
  const float fr = (N0 > 0.f ? div_fast(Nc, N0) : 1.f) * fs;
  N = Nc;
  fx *= fr;
  fy *= fr;
  fz *= fr;
  y = yc;
  T = Tc;
  return o;
}

// Kahan-compensated FP32 accumulator (per-thread tallies of the step kernels before the FP64
// block reduction; its few extra registers matter there).
struct KahanF {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float yv = v - c;
    const float t = s + yv;
    c = (t - s) - yv;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Compensated FP32 accumulator for the reduction passes: every addition is split exactly into
// its rounded sum and rounding error (Knuth's TwoSum, valid whatever the magnitudes, where
// Kahan's form loses accuracy once a term exceeds the running sum, as photon densities
// spanning many decades make common), the errors gathered in c; value = s + c.
struct TwoSumF {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float t = s + v;
    const float bp = t - s;
    c += (s - (t - bp)) + (v - bp);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

}  // namespace aton
