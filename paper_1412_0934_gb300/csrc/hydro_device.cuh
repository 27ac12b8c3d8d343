// Device-side arithmetic of one MUSCL-Hancock/HLLC step of the 3D ideal-gas Euler equations
// (the hydro path of the paper, Sec. 2 and Sec. 4; textbook scheme, see include/hydro.h):
// primitive recovery, limited PLM slopes, the unsplit primitive Hancock predictor, floored face
// states, HLLC fluxes and the per-cell CFL speed.  Three precision policies:
//   PolF64   double state, double arithmetic;
//   PolF32   float state, float arithmetic, pressure recovery by error-free transformations;
//   PolMixed double state, double pressure recovery and update accumulation, float bulk;
//   PolDF    double state, double-float arithmetic (about 48 bits, on the FP32 pipes), double
//            update accumulation.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "df.cuh"
#include "hydro.h"

namespace hydro {

constexpr int NG = 2;  // ghost layers of the stencil

struct Params {
  double gamma, cfl, rho_floor, p_floor;
  int limiter;
  // Derived constants, precomputed on the host so kernels never convert or divide them:
  // index 0 gamma, 1 1/(gamma-1), 2 gamma-1, 3 rho_floor, 4 p_floor, 5 1/6; as doubles, as
  // floats, and as (hi, lo) float pairs.
  double kd[6];
  float kf[6];
  float kh[6], kl[6];
};

enum { K_GAMMA = 0, K_IGM1 = 1, K_GM1 = 2, K_RHOF = 3, K_PF = 4, K_SIXTH = 5 };

inline Params make_params(double gamma, double cfl, double rho_floor, double p_floor, int limiter) {
  Params p{gamma, cfl, rho_floor, p_floor, limiter, {}, {}, {}, {}};
  const double k[6] = {gamma, 1.0 / (gamma - 1.0), gamma - 1.0, rho_floor, p_floor, 1.0 / 6.0};
  for (int i = 0; i < 6; ++i) {
    p.kd[i] = k[i];
    p.kf[i] = (float)k[i];
    p.kh[i] = (float)k[i];
    p.kl[i] = (float)(k[i] - (double)p.kh[i]);
  }
  return p;
}

// ------------------------------------------------------------------ small helpers
template <class R>
__device__ __forceinline__ R rabs(R x) {
  return x < R(0) ? -x : x;
}
// Float policies use the SFU approximations (relative error a few ulp of float); double uses
// correctly rounded IEEE operations.
__device__ __forceinline__ float rcp_(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsqrt_(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float div_(float a, float b) { return a * rcp_(b); }
__device__ __forceinline__ double rsqrt_(double x) { return sqrt(x); }
__device__ __forceinline__ double rcp_(double x) { return 1.0 / x; }
__device__ __forceinline__ double div_(double a, double b) { return a / b; }

// Constant i of the parameters in arithmetic type R.
template <class R>
struct KC;
template <>
struct KC<float> {
  static __device__ __forceinline__ float get(const Params& P, int i) { return P.kf[i]; }
};
template <>
struct KC<double> {
  static __device__ __forceinline__ double get(const Params& P, int i) { return P.kd[i]; }
};
template <>
struct KC<df> {
  static __device__ __forceinline__ df get(const Params& P, int i) { return df(P.kh[i], P.kl[i]); }
};
template <class R>
__device__ __forceinline__ R kc(const Params& P, int i) {
  return KC<R>::get(P, i);
}

// a - b where cancellation is the point (internal energy from total minus kinetic energy): the
// plain difference in float and double, the accurate double-word sum in double-float.
__device__ __forceinline__ float sub_acc(float a, float b) { return a - b; }
__device__ __forceinline__ double sub_acc(double a, double b) { return a - b; }
__device__ __forceinline__ df sub_acc(const df& a, const df& b) { return add_acc(a, -b); }

// 0.5 x, 2 x and x f for a float constant f (exact scalings; df overloads in df.cuh).
__device__ __forceinline__ float half_(float x) { return 0.5f * x; }
__device__ __forceinline__ double half_(double x) { return 0.5 * x; }
__device__ __forceinline__ float twice_(float x) { return 2.f * x; }
__device__ __forceinline__ double twice_(double x) { return 2.0 * x; }
__device__ __forceinline__ float mulf_(float x, float f) { return x * f; }
__device__ __forceinline__ double mulf_(double x, float f) { return x * (double)f; }

__device__ __forceinline__ float shfl_xor_(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_xor_(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ bool isfinite_(float x) { return isfinite(x); }
__device__ __forceinline__ bool isfinite_(double x) { return isfinite(x); }

// Order-preserving 64-bit key of a non-negative double (IEEE bits compare as unsigned ints).
__device__ __forceinline__ unsigned long long dkey(double x) { return (unsigned long long)__double_as_longlong(x); }

// ------------------------------------------------------------------ comparisons
// For doubles the tests below run on the integer pipe over the IEEE bit patterns (GB300's FP64
// pipe is 1/73 of its FP32 rate, and comparisons would occupy it); they give the same result as
// the floating-point comparison for every non-NaN operand.  Floats use plain comparisons.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ bool cmp_lt_floor(double x, double f) {  // x < f for f > 0
  const long long X = dbits(x);
  return X < 0 ? (X & 0x7fffffffffffffffLL) != 0 || dbits(f) > 0 : X < dbits(f);
}
__device__ __forceinline__ bool cmp_lt_floor(float x, float f) { return x < f; }
__device__ __forceinline__ bool cmp_neg(double x) {  // x < 0
  const long long X = dbits(x);
  return X < 0 && (X & 0x7fffffffffffffffLL) != 0;
}
__device__ __forceinline__ bool cmp_neg(float x) { return x < 0.f; }
__device__ __forceinline__ bool cmp_pos(double x) { return dbits(x) > 0; }  // x > 0
__device__ __forceinline__ bool cmp_pos(float x) { return x > 0.f; }
// |a| <= |b|
__device__ __forceinline__ bool abs_le(double a, double b) {
  return (unsigned long long)(dbits(a) & 0x7fffffffffffffffLL) <= (unsigned long long)(dbits(b) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ bool abs_le(float a, float b) { return fabsf(a) <= fabsf(b); }
__device__ __forceinline__ bool abs_lt(double a, double b) { return !abs_le(b, a); }
__device__ __forceinline__ bool abs_lt(float a, float b) { return fabsf(a) < fabsf(b); }
// a * b <= 0: opposite signs or a zero factor.  (Differs from the rounded product only when
// |a b| underflows below 1e-308, where either limiter result is below 1e-154.)
__device__ __forceinline__ bool prod_nonpos(double a, double b) {
  const long long A = dbits(a), B = dbits(b);
  return ((A ^ B) < 0) || (A & 0x7fffffffffffffffLL) == 0 || (B & 0x7fffffffffffffffLL) == 0;
}
__device__ __forceinline__ bool prod_nonpos(float a, float b) { return a * b <= 0.f; }

// ------------------------------------------------------------------ slope limiter
// MinMod: 0 if a*b <= 0, else the argument of smaller magnitude (tie -> a).
// MC: 0 if a*b <= 0, else the smallest magnitude of 2a, 2b, (a+b)/2 (ties -> earlier).
// None: the centred difference (a+b)/2.
template <class R>
__device__ __forceinline__ R limited(R a, R b, int lim) {
  if (lim == HYDRO_NOLIMIT) return half_(a + b);
  if (prod_nonpos(a, b)) return R(0);
  if (lim == HYDRO_MINMOD) return abs_le(a, b) ? a : b;
  R ta = twice_(a), tb = twice_(b), m = half_(a + b);
  R best = ta;
  if (abs_lt(tb, best)) best = tb;
  if (abs_lt(m, best)) best = m;
  return best;
}

// MinMod alone (the same values as limited(a, b, HYDRO_MINMOD)), for kernels that fix the limiter at
// compile time.  Double-float: once the signs agree, |a| <= |b| is a <= b for positive values and
// b <= a for negative ones (one lexicographic comparison instead of two absolute values).
template <class R>
__device__ __forceinline__ R minmod(R a, R b) {
  if (prod_nonpos(a, b)) return R(0);
  return abs_le(a, b) ? a : b;
}
__device__ __forceinline__ df minmod(const df& a, const df& b) {
  if (prod_nonpos(a, b)) return df(0.f, 0.f);
  const bool le = a.h > 0.f ? !(b < a) : !(a < b);
  return le ? a : b;
}

// ------------------------------------------------------------------ Hancock predictor
// qh = q - hdt * (A_x dqx + A_y dqy + A_z dqz), A_d the primitive Jacobian of direction d.
template <class R>
__device__ __forceinline__ void hancock(const R q[5], const R dqx[5], const R dqy[5], const R dqz[5], R gamma, R hdt,
                                        R qh[5]) {
  const R ir = rcp_(q[0]);
  const R gp = gamma * q[4];
  // x: normal u
  R tx0 = q[1] * dqx[0] + q[0] * dqx[1];
  R tx1 = q[1] * dqx[1] + dqx[4] * ir;
  R tx2 = q[1] * dqx[2];
  R tx3 = q[1] * dqx[3];
  R tx4 = gp * dqx[1] + q[1] * dqx[4];
  // y: normal v
  R ty0 = q[2] * dqy[0] + q[0] * dqy[2];
  R ty1 = q[2] * dqy[1];
  R ty2 = q[2] * dqy[2] + dqy[4] * ir;
  R ty3 = q[2] * dqy[3];
  R ty4 = gp * dqy[2] + q[2] * dqy[4];
  // z: normal w
  R tz0 = q[3] * dqz[0] + q[0] * dqz[3];
  R tz1 = q[3] * dqz[1];
  R tz2 = q[3] * dqz[2];
  R tz3 = q[3] * dqz[3] + dqz[4] * ir;
  R tz4 = gp * dqz[3] + q[3] * dqz[4];
  qh[0] = q[0] - hdt * ((tx0 + ty0) + tz0);
  qh[1] = q[1] - hdt * ((tx1 + ty1) + tz1);
  qh[2] = q[2] - hdt * ((tx2 + ty2) + tz2);
  qh[3] = q[3] - hdt * ((tx3 + ty3) + tz3);
  qh[4] = q[4] - hdt * ((tx4 + ty4) + tz4);
}

template <class R>
__device__ __forceinline__ void floor_state(R q[5], R rho_floor, R p_floor) {
  q[0] = cmp_lt_floor(q[0], rho_floor) ? rho_floor : q[0];
  q[4] = cmp_lt_floor(q[4], p_floor) ? p_floor : q[4];
}

// ------------------------------------------------------------------ HLLC
// Flux through a face between floored states, in face-normal components: q = (rho, u_n, u_t1,
// u_t2, p); ke = u^2 + v^2 + w^2 summed in x, y, z order.  F = F_L if 0 <= S_L; F_R if S_R <= 0;
// else F_K + S_K (U*_K - U_K) with K = L if S* >= 0 else R (Davis speeds, Batten et al. star
// state).  Only the upwind side's physical flux is formed; branches are selected, not multiplied.
// 1/a and 1/b.  In double, where a division is a long sequence on the FP64 pipe, both come from
// one division, 1/a = b/(ab), 1/b = a/(ab) (the operands here are positive densities, or a mass
// flux and a speed difference, whose products stay far inside the exponent range).  A float
// reciprocal is one SFU instruction, and a double-float one costs about what the two extra
// double-float products would: two reciprocals.
__device__ __forceinline__ void rcp2(float a, float b, float& ra, float& rb) {
  ra = rcp_(a);
  rb = rcp_(b);
}
__device__ __forceinline__ void rcp2(double a, double b, double& ra, double& rb) {
  const double i = 1.0 / (a * b);
  ra = b * i;
  rb = a * i;
}
__device__ __forceinline__ void rcp2(const df& a, const df& b, df& ra, df& rb) {
  ra = rcp_(a);
  rb = rcp_(b);
}

// zn: the face normal is z.  The upwind side's kinetic sum |u|^2 is formed after the side is chosen,
// from its face-normal components (u_n, u_t1, u_t2), in the x, y, z order of the velocity: (u_n^2 +
// u_t1^2) + u_t2^2 for x and y normals (for y, u_n^2 + u_t1^2 = v^2 + u^2 = u^2 + v^2 exactly),
// (u_t1^2 + u_t2^2) + u_n^2 for a z normal.
template <class R>
__device__ __forceinline__ void hllc_core(const R qL[5], const R qR[5], bool zn, R gamma, R inv_gm1, R F[5]) {
  R irL, irR;
  rcp2(qL[0], qR[0], irL, irR);
  const R cL = rsqrt_(gamma * qL[4] * irL);
  const R cR = rsqrt_(gamma * qR[4] * irR);
  const R uL = qL[1], uR = qR[1];
  const R aL = uL - cL, bL = uR - cR;
  const R SL = aL <= bL ? aL : bL;
  const R aR = uL + cL, bR = uR + cR;
  const R SR = aR >= bR ? aR : bR;
  const R mL = qL[0] * (SL - uL);
  const R mR = qR[0] * (SR - uR);
  const R Ss = div_(qR[4] - qL[4] + uL * mL - uR * mR, mL - mR);
  const bool SLneg = cmp_neg(SL), SRpos = cmp_pos(SR);
  const bool star = SLneg && SRpos;
  const bool left = !SLneg || (SRpos && !cmp_neg(Ss));
  const R rK = left ? qL[0] : qR[0];
  const R uK = left ? uL : uR;
  const R t1 = left ? qL[2] : qR[2];
  const R t2 = left ? qL[3] : qR[3];
  const R pK = left ? qL[4] : qR[4];
  const R irK = left ? irL : irR;
  const R SK = left ? SL : SR;
  const R mK = left ? mL : mR;
  const R un2 = uK * uK, a2 = t1 * t1, b2 = t2 * t2;
  const R keK = zn ? (a2 + b2) + un2 : (un2 + a2) + b2;
  const R EK = pK * inv_gm1 + half_(rK * keK);
  // Star state of side K: density r* = m_K/(S_K - S*), velocity S*, pressure p* = p_K + m_K (S* - u_K),
  // energy E* = r* (E_K/rho_K + (S* - u_K)(S* + p_K/m_K)).  F*_K = F_K + S_K (U*_K - U_K) equals the
  // physical flux of that state, so one flux formula serves every branch.
  R iD, imK;
  rcp2(SK - Ss, mK, iD, imK);
  const R rs = mK * iD;
  const R ps = pK + mK * (Ss - uK);
  const R Es = rs * (EK * irK + (Ss - uK) * (Ss + pK * imK));
  const R re = star ? rs : rK;
  const R ue = star ? Ss : uK;
  const R pe = star ? ps : pK;
  const R Ee = star ? Es : EK;
  const R mn = re * ue;
  F[0] = mn;
  F[1] = mn * ue + pe;
  F[2] = mn * t1;
  F[3] = mn * t2;
  F[4] = ue * (Ee + pe);
}

template <class R>
__device__ __forceinline__ R kinetic_sum(const R q[5]) {
  return (q[1] * q[1] + q[2] * q[2]) + q[3] * q[3];
}

// Face of compile-time normal D (0 x, 1 y, 2 z); q, F in (rho, u, v, w, p) / (rho, m_x, m_y, m_z, E).
template <int D, class R>
__device__ __forceinline__ void hllc(const R qL[5], const R qR[5], R gamma, R inv_gm1, R F[5]) {
  constexpr int N = 1 + D;
  constexpr int T1 = (D == 0) ? 2 : 1;
  constexpr int T2 = (D == 2) ? 2 : 3;
  const R a[5] = {qL[0], qL[N], qL[T1], qL[T2], qL[4]};
  const R b[5] = {qR[0], qR[N], qR[T1], qR[T2], qR[4]};
  R Fr[5];
  hllc_core(a, b, D == 2, gamma, inv_gm1, Fr);
  F[0] = Fr[0];
  F[N] = Fr[1];
  F[T1] = Fr[2];
  F[T2] = Fr[3];
  F[4] = Fr[4];
}

// Same flux for a runtime normal d (selects instead of register indexing).
template <class R>
__device__ __forceinline__ void hllc_dyn(int d, const R qL[5], const R qR[5], R gamma, R inv_gm1, R F[5]) {
  const R a[5] = {qL[0], d == 0 ? qL[1] : (d == 1 ? qL[2] : qL[3]), d == 0 ? qL[2] : qL[1],
                  d == 2 ? qL[2] : qL[3], qL[4]};
  const R b[5] = {qR[0], d == 0 ? qR[1] : (d == 1 ? qR[2] : qR[3]), d == 0 ? qR[2] : qR[1],
                  d == 2 ? qR[2] : qR[3], qR[4]};
  R Fr[5];
  hllc_core(a, b, d == 2, gamma, inv_gm1, Fr);
  F[0] = Fr[0];
  F[1] = d == 0 ? Fr[1] : Fr[2];
  F[2] = d == 1 ? Fr[1] : (d == 0 ? Fr[2] : Fr[3]);
  F[3] = d == 2 ? Fr[1] : Fr[3];
  F[4] = Fr[4];
}

// ------------------------------------------------------------------ error-free transformations
__device__ __forceinline__ float two_sum_err(float a, float b, float s) {
  float bb = s - a;
  return (a - (s - bb)) + (b - bb);
}

// Conversions for the mixed and double-float policies without conversion instructions, which
// share GB300's narrow FP64 pipe with the double arithmetic.
// Exact float of an integer 0 <= n < 2^23: the bits of 2^23 + n read as a float, minus 2^23.
__device__ __forceinline__ float small_uint_to_float(unsigned n) {
  return __uint_as_float(0x4B000000u | n) - 8388608.f;
}
// Double -> float pair (hi, lo), hi + lo = x to 2^-47 relative, by rearranging IEEE-754 bit fields
// on the integer pipe and exact float arithmetic: hi is x cut to its leading 24 significant bits,
// lo the remaining 29-bit integer rounded once to a float (its top 23 bits times 64 plus its low 6
// bits, one FMA) and scaled by the power of two 2^(E-52), then one Fast2Sum.  Zero and |x|
// outside [2^-74, 2^99) take the conversion instructions instead.
// The rare cases out of line, so that the common path carries no conversion instruction (an
// inlined branch this short would be predicated, and its conversions issued for every value).
static __device__ __noinline__ float2 split_double_cvt(double x) {
  const float hi = (float)x;
  return make_float2(hi, (float)(x - (double)hi));
}
static __device__ __noinline__ double float_to_double_cvt(float f) { return (double)f; }

__device__ __forceinline__ void split_double(double x, float& hi, float& lo) {
  const unsigned xh = (unsigned)__double2hiint(x), xl = (unsigned)__double2loint(x);
  const unsigned ex = (xh >> 20) & 0x7FFu;  // biased exponent, E = ex - 1023
  if (__builtin_expect(ex - 949u >= 173u, 0)) {
    const float2 c = split_double_cvt(x);  // returned in registers: no stack frame on the common path
    hi = c.x;
    lo = c.y;
    return;
  }
  const unsigned sign = xh & 0x80000000u;
  const float ht = __uint_as_float(sign | ((ex - 896u) << 23) | ((xh & 0xFFFFFu) << 3) | (xl >> 29));
  const unsigned r = xl & 0x1FFFFFFFu;
  const float rf = fmaf(small_uint_to_float(r >> 6), 64.f, small_uint_to_float(r & 63u));
  const float lt = __uint_as_float(__float_as_uint(rf * __uint_as_float((ex - 948u) << 23)) | sign);
  hi = ht + lt;
  lo = lt - (hi - ht);
}
// Exact float -> double: sign kept, exponent rebiased by 1023 - 127, the 23 fraction bits placed
// at the top of the 52.  Zero maps to zero; subnormal, infinite and NaN floats take the cvt.
__device__ __forceinline__ double float_to_double(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xFFu;
  if (__builtin_expect(e == 0u || e == 0xFFu, 0))
    return (b & 0x7FFFFFFFu) == 0u ? __hiloint2double((int)(b & 0x80000000u), 0) : float_to_double_cvt(f);
  return __hiloint2double((int)((b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7FFFFFu) >> 3)), (int)(b << 29));
}

// ------------------------------------------------------------------ precision policies
// recover(): U (storage) -> q (arithmetic), floors applied, flags set on floors / non-finite.
// speed():   |u| + |v| + |w| + 3c of a stored state (CFL), in the arithmetic type.
// update():  U_old - dtdx * div in the policy's accumulation precision.

struct PolF64 {
  using S = double;
  using R = double;
  static __device__ __forceinline__ void recover(const double U[5], const Params& P, double q[5], unsigned& flags) {
    double rho = U[0];
    if (rho < P.rho_floor) { flags |= HYDRO_EBIT_RHO_FLOOR; rho = P.rho_floor; }
    const double ir = 1.0 / rho;
    const double kin = 0.5 * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) * ir;
    const double eint = U[4] - kin;
    if (eint < 0.0) flags |= HYDRO_EBIT_P_FLOOR;
    double p = P.kd[K_GM1] * eint;
    if (!(isfinite(p) && isfinite(rho))) flags |= HYDRO_EBIT_NONFINITE;
    q[0] = rho;
    q[1] = U[1] * ir;
    q[2] = U[2] * ir;
    q[3] = U[3] * ir;
    q[4] = p < P.p_floor ? P.p_floor : p;
  }
  static __device__ __forceinline__ double update(double Uold, double dtdx, double div) { return Uold - dtdx * div; }
  static __device__ __forceinline__ double speed(const double U[5], const Params& P, unsigned& flags);
};

struct PolF32 {
  using S = float;
  using R = float;
  // p = (gamma-1)(E - K/(2 rho)), K = |m|^2, with K formed exactly as a float pair (two-product
  // and two-sum), K/rho as a float pair (exact FMA residual), and E - K/(2 rho) by two-sum: the
  // cancellation between E and the kinetic energy loses nothing beyond the final rounding.
  static __device__ __forceinline__ void recover(const float U[5], const Params& P, float q[5], unsigned& flags) {
    float rho = U[0];
    const float rf = P.kf[K_RHOF];
    if (rho < rf) { flags |= HYDRO_EBIT_RHO_FLOOR; rho = rf; }
    const float ir = __frcp_rn(rho);
    const float mx = U[1], my = U[2], mz = U[3];
    const float a1 = mx * mx, e1 = fmaf(mx, mx, -a1);
    const float a2 = my * my, e2 = fmaf(my, my, -a2);
    const float a3 = mz * mz, e3 = fmaf(mz, mz, -a3);
    const float s1 = a1 + a2;
    const float t1 = two_sum_err(a1, a2, s1);
    const float Kh = s1 + a3;
    const float t2 = two_sum_err(s1, a3, Kh);
    const float Kl = ((e1 + e2) + e3) + (t1 + t2);
    // kinetic energy (K/rho)/2 = (kh + kl)/2
    const float kh = Kh * ir;
    const float r = fmaf(-kh, rho, Kh);
    const float kl = (r + Kl) * ir;
    const float hk = 0.5f * kh;
    const float d = U[4] - hk;
    const float de = two_sum_err(U[4], -hk, d);
    const float eint = d + (de - 0.5f * kl);
    if (eint < 0.f) flags |= HYDRO_EBIT_P_FLOOR;
    float p = P.kf[K_GM1] * eint;
    if (!(isfinite(p) && isfinite(rho))) flags |= HYDRO_EBIT_NONFINITE;
    const float pf = P.kf[K_PF];
    q[0] = rho;
    q[1] = mx * ir;
    q[2] = my * ir;
    q[3] = mz * ir;
    q[4] = p < pf ? pf : p;
  }
  static __device__ __forceinline__ float update(float Uold, float dtdx, float div) { return Uold - dtdx * div; }
  // CFL speed of a stored state: plain float recovery (the dt only needs float accuracy).
  static __device__ __forceinline__ float speed(const float U[5], const Params& P, unsigned& flags) {
    float rho = U[0];
    const float rf = P.kf[K_RHOF];
    if (rho < rf) { flags |= HYDRO_EBIT_RHO_FLOOR; rho = rf; }
    const float ir = rcp_(rho);
    const float u = U[1] * ir, v = U[2] * ir, w = U[3] * ir;
    const float eint = U[4] - 0.5f * rho * ((u * u + v * v) + w * w);
    float p = P.kf[K_GM1] * eint;
    if (!(isfinite(p) && isfinite(rho))) flags |= HYDRO_EBIT_NONFINITE;
    const float pf = P.kf[K_PF];
    p = p < pf ? pf : p;
    const float c = rsqrt_(P.kf[K_GAMMA] * p * ir);
    return ((fabsf(u) + fabsf(v)) + fabsf(w)) + 3.0f * c;
  }
};

struct PolMixed {
  using S = double;
  using R = float;
  // Recovery from the double state split into float pairs (split_double): |m|^2 as a float pair
  // (exact squares of the high parts, their exact sum errors, the cross terms 2 m_hi m_lo; the
  // m_lo^2 terms are below 2^-47 |m|^2), |m|^2/rho as a float pair (quotient of the high parts
  // plus the FMA residual and the rho_lo term over rho), and E - |m|^2/(2 rho) by a two-sum with
  // E's low part: the internal energy to float accuracy unless the kinetic energy exceeds it by
  // ~2^20, with no FP64 instruction.
  static __device__ __forceinline__ void recover(const double U[5], const Params& P, float q[5], unsigned& flags) {
    float rh, rl;
    if (cmp_lt_floor(U[0], P.kd[K_RHOF])) {
      flags |= HYDRO_EBIT_RHO_FLOOR;
      rh = P.kh[K_RHOF];
      rl = P.kl[K_RHOF];
    } else {
      split_double(U[0], rh, rl);
    }
    float xh, xl, yh, yl, zh, zl, eh, el;
    split_double(U[1], xh, xl);
    split_double(U[2], yh, yl);
    split_double(U[3], zh, zl);
    split_double(U[4], eh, el);
    const float ir = __frcp_rn(rh);
    const float a1 = xh * xh, e1 = fmaf(xh, xh, -a1);
    const float a2 = yh * yh, e2 = fmaf(yh, yh, -a2);
    const float a3 = zh * zh, e3 = fmaf(zh, zh, -a3);
    const float s1 = a1 + a2;
    const float t1 = two_sum_err(a1, a2, s1);
    const float Kh = s1 + a3;
    const float t2 = two_sum_err(s1, a3, Kh);
    const float Kl = (((e1 + e2) + e3) + (t1 + t2)) + 2.f * ((xh * xl + yh * yl) + zh * zl);
    const float kh = Kh * ir;
    const float kl = ((fmaf(-kh, rh, Kh) + Kl) - kh * rl) * ir;
    const float hk = 0.5f * kh;
    const float d = eh - hk;
    const float de = two_sum_err(eh, -hk, d);
    const float eint = d + ((de + el) - 0.5f * kl);
    if (eint < 0.f) flags |= HYDRO_EBIT_P_FLOOR;
    float p = P.kf[K_GM1] * eint;
    if (!(isfinite(p) && isfinite(rh))) flags |= HYDRO_EBIT_NONFINITE;
    const float pf = P.kf[K_PF];
    q[0] = rh;
    q[1] = xh * ir;
    q[2] = yh * ir;
    q[3] = zh * ir;
    q[4] = p < pf ? pf : p;
  }
  // dU = dtdx * div in float, accumulated into the double state (one FP64 add per field).
  static __device__ __forceinline__ double update(double Uold, float dtdx, float div) {
    return Uold - float_to_double(dtdx * div);
  }
  static __device__ __forceinline__ float speed(const double U[5], const Params& P, unsigned& flags);
};

struct PolDF {
  using S = double;
  using R = df;
  // The same recovery as PolF64, in double-float from the double state (split into float pairs on
  // the integer pipe, split_double).
  static __device__ __forceinline__ void recover(const double U[5], const Params& P, df q[5], unsigned& flags) {
    df rho, mx, my, mz, E;
    split_double(U[0], rho.h, rho.l);
    split_double(U[1], mx.h, mx.l);
    split_double(U[2], my.h, my.l);
    split_double(U[3], mz.h, mz.l);
    split_double(U[4], E.h, E.l);
    const df rf = kc<df>(P, K_RHOF);
    if (rho < rf) { flags |= HYDRO_EBIT_RHO_FLOOR; rho = rf; }
    const df ir = rcp_(rho);
    const df kin = half_(((mx * mx + my * my) + mz * mz) * ir);
    const df eint = sub_acc(E, kin);
    if (cmp_neg(eint)) flags |= HYDRO_EBIT_P_FLOOR;
    df p = kc<df>(P, K_GM1) * eint;
    if (!(isfinite(p.h) && isfinite(rho.h))) flags |= HYDRO_EBIT_NONFINITE;
    const df pf = kc<df>(P, K_PF);
    q[0] = rho;
    q[1] = mx * ir;
    q[2] = my * ir;
    q[3] = mz * ir;
    q[4] = p < pf ? pf : p;
  }
  // U_old - dtdx * div: the double-float increment made a double exactly (float_to_double) and
  // subtracted from the double state in double.
  static __device__ __forceinline__ double update(double Uold, const df& dtdx, const df& div) {
    const df d = dtdx * div;
    return Uold - (float_to_double(d.h) + float_to_double(d.l));
  }
  static __device__ __forceinline__ df speed(const double U[5], const Params& P, unsigned& flags);
};

// CFL speed of a recovered state.
template <class R>
__device__ __forceinline__ R cfl_speed(const R q[5], R gamma) {
  const R c = rsqrt_(gamma * q[4] * rcp_(q[0]));
  return ((rabs(q[1]) + rabs(q[2])) + rabs(q[3])) + mulf_(c, 3.f);
}

// CFL speed of a stored state (the step's epilogue and the standalone dt kernel share it, so
// both produce the same bits): FP64 and mixed through their recovery, FP32 through a plain one.
__device__ __forceinline__ double PolF64::speed(const double U[5], const Params& P, unsigned& flags) {
  double q[5];
  recover(U, P, q, flags);
  return cfl_speed(q, P.kd[K_GAMMA]);
}
// The mixed policy's arithmetic is float, and so is the accuracy its dt needs: each field is rounded
// to float by its IEEE bit fields (fields outside [2^-40, 2^40), other than zero, take the pair
// recovery instead) and recovered plainly in float.
__device__ __forceinline__ float round_float(double x, bool& ok) {
  const unsigned h = (unsigned)__double2hiint(x), l = (unsigned)__double2loint(x);
  const unsigned ex = (h >> 20) & 0x7FFu;
  const bool zero = (h & 0x7FFFFFFFu) == 0u && l == 0u;
  ok = ok && (zero || ex - 983u < 80u);
  const unsigned b = (h & 0x80000000u) | ((ex - 896u) << 23) | ((h & 0xFFFFFu) << 3) | (l >> 29);
  return zero ? 0.f : __uint_as_float(b + ((l >> 28) & 1u));  // round half away from zero
}
__device__ __forceinline__ float PolMixed::speed(const double U[5], const Params& P, unsigned& flags) {
  bool ok = true;
  float f[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) f[v] = round_float(U[v], ok);
  if (!ok) {
    float q[5];
    recover(U, P, q, flags);
    return cfl_speed(q, P.kf[K_GAMMA]);
  }
  float rho = f[0];
  const float rf = P.kf[K_RHOF];
  if (rho < rf) { flags |= HYDRO_EBIT_RHO_FLOOR; rho = rf; }
  const float ir = rcp_(rho);
  const float u = f[1] * ir, v = f[2] * ir, w = f[3] * ir;
  const float eint = f[4] - 0.5f * rho * ((u * u + v * v) + w * w);
  if (eint < 0.f) flags |= HYDRO_EBIT_P_FLOOR;
  float p = P.kf[K_GM1] * eint;
  const float pf = P.kf[K_PF];
  p = p < pf ? pf : p;
  const float c = rsqrt_(P.kf[K_GAMMA] * p * ir);
  return ((fabsf(u) + fabsf(v)) + fabsf(w)) + 3.0f * c;
}
__device__ __forceinline__ df PolDF::speed(const double U[5], const Params& P, unsigned& flags) {
  df q[5];
  recover(U, P, q, flags);
  return cfl_speed(q, kc<df>(P, K_GAMMA));
}

// ------------------------------------------------------------------ CFL candidates
// A float estimate of the CFL speed of a double state, with which the step's fused CFL maximum
// skips the exact speed of cells that cannot hold it.  Each field is cut to the float of its
// leading 24 significant bits (relative error below 2^-23), recovered in float with the SFU
// reciprocal and square root.  Returns false -- the cell then takes the exact speed -- unless every
// field is zero or of magnitude in [2^-40, 2^40), the density exceeds twice its floor and the
// internal energy exceeds 1e-3 of E + |m|^2/(2 rho).  When it returns true the exact recovery floors
// nothing and flags nothing, the float internal energy is within ~1.1e-6 (E + |m|^2/(2 rho)), i.e.
// 1.1e-3 of itself, so the sound speed is within ~6e-4 and s within 1e-3 of the exact speed.
__device__ __forceinline__ float cut_float(double x, bool& ok) {
  const unsigned h = (unsigned)__double2hiint(x), l = (unsigned)__double2loint(x);
  const unsigned ex = (h >> 20) & 0x7FFu;
  const bool zero = (h & 0x7FFFFFFFu) == 0u && l == 0u;
  ok = ok && (zero || ex - 983u < 80u);
  return zero ? 0.f : __uint_as_float((h & 0x80000000u) | ((ex - 896u) << 23) | ((h & 0xFFFFFu) << 3) | (l >> 29));
}
__device__ __forceinline__ bool speed_estimate(const double U[5], const Params& P, float& s) {
  bool ok = true;
  const float r = cut_float(U[0], ok), mx = cut_float(U[1], ok), my = cut_float(U[2], ok);
  const float mz = cut_float(U[3], ok), e = cut_float(U[4], ok);
  const float ir = rcp_(r);
  const float kin = 0.5f * (((mx * mx + my * my) + mz * mz) * ir);
  const float eint = e - kin;
  ok = ok && r > 2.f * P.kf[K_RHOF] && eint > 1e-3f * (e + kin);
  float p = P.kf[K_GM1] * eint;
  p = p < P.kf[K_PF] ? P.kf[K_PF] : p;
  s = ((fabsf(mx) + fabsf(my)) + fabsf(mz)) * ir + 3.f * rsqrt_(P.kf[K_GAMMA] * p * ir);
  return ok;
}

}  // namespace hydro
