// Reverse-mode pieces of the MUSCL-Hancock/HLLC step (dt held fixed): HLLC, the Hancock
// predictor, the limited slope (through the branch its forward values select, recorded as a
// 2-bit code), and the primitive recovery.  Each function recomputes the forward values it needs
// and returns adjoints with respect to its inputs.
#pragma once
#include "hydro_device.cuh"

namespace hydro {

// ------------------------------------------------------------------ limiter with branch code
// Code: 0 zero slope, 1 the first argument (a, or 2a for MC), 2 the second (b, or 2b for MC),
// 3 the centred (a+b)/2.  Same comparisons as limited().
template <class R>
__device__ __forceinline__ R limited_code(R a, R b, int lim, unsigned& code) {
  if (lim == HYDRO_NOLIMIT) { code = 3; return half_(a + b); }
  if (prod_nonpos(a, b)) { code = 0; return R(0); }
  if (lim == HYDRO_MINMOD) {
    if (abs_le(a, b)) { code = 1; return a; }
    code = 2;
    return b;
  }
  R ta = twice_(a), tb = twice_(b), m = half_(a + b);
  R best = ta;
  code = 1;
  if (abs_lt(tb, best)) { best = tb; code = 2; }
  if (abs_lt(m, best)) { best = m; code = 3; }
  return best;
}

// Partial derivatives (alpha, beta) of the limited slope with respect to (a, b) for a code
// (0, 1/2, 1 or 2: exact in any arithmetic type).
__device__ __forceinline__ void code_weights(unsigned code, int lim, float& alpha, float& beta) {
  const float w = (lim == HYDRO_MC) ? 2.f : 1.f;
  alpha = code == 1 ? w : (code == 3 ? 0.5f : 0.f);
  beta = code == 2 ? w : (code == 3 ? 0.5f : 0.f);
}

// ------------------------------------------------------------------ HLLC reverse
// Given the face-normal states (as in hllc_core) and lamF, accumulate lamqL, lamqR (5 each) and
// the adjoints of the kinetic sums keL, keR.
template <class R>
__device__ __forceinline__ void hllc_core_adj(const R qL[5], const R qR[5], R keL, R keR, R gamma, R inv_gm1,
                                              const R lamF[5], R lqL[5], R lqR[5], R& lkeL, R& lkeR) {
  // ---- forward recomputation (the values that select branches exactly as hllc_core forms them)
  R irL, irR;
  rcp2(qL[0], qR[0], irL, irR);
  const R cL = rsqrt_(gamma * qL[4] * irL);
  const R cR = rsqrt_(gamma * qR[4] * irR);
  const R uL = qL[1], uR = qR[1];
  const R aL = uL - cL, bL = uR - cR;
  const bool selL = aL <= bL;
  const R SL = selL ? aL : bL;
  const R aR = uL + cL, bR = uR + cR;
  const bool selR = aR >= bR;
  const R SR = selR ? aR : bR;
  const R mL = qL[0] * (SL - uL);
  const R mR = qR[0] * (SR - uR);
  const R num = qR[4] - qL[4] + uL * mL - uR * mR;
  const R den = mL - mR;
  const R iden = rcp_(den);  // S* = num / den; its sign (the only branch it decides) is exact
  const R Ss = num * iden;
  const bool SLneg = cmp_neg(SL), SRpos = cmp_pos(SR);
  const bool star = SLneg && SRpos;
  const bool left = !SLneg || (SRpos && !cmp_neg(Ss));
  const R rK = left ? qL[0] : qR[0];
  const R uK = left ? uL : uR;
  const R t1 = left ? qL[2] : qR[2];
  const R t2 = left ? qL[3] : qR[3];
  const R pK = left ? qL[4] : qR[4];
  const R keK = left ? keL : keR;
  const R irK = left ? irL : irR;
  const R SK = left ? SL : SR;
  const R mK = left ? mL : mR;
  const R EK = pK * inv_gm1 + half_(rK * keK);
  const R mn = rK * uK;
  // ---- reverse
  R lrK = 0, luK = 0, lt1 = 0, lt2 = 0, lpK = 0, lkeK = 0, lirK = 0, lSK = 0, lmK = 0, lSs = 0, lEK = 0, lmn = 0;
  if (star) {
    // star state of side K: fac = m_K / D (its density), D = S_K - S*, w = p_K / m_K
    const R Dd = SK - Ss;
    R iDd, imK;
    rcp2(Dd, mK, iDd, imK);
    const R fac = mK * iDd;
    const R w = pK * imK;
    const R Y = Ss - uK, Z = Ss + w;
    const R X = EK * irK + Y * Z;
    const R UK[5] = {rK, mn, rK * t1, rK * t2, EK};
    const R Us[5] = {fac, fac * Ss, fac * t1, fac * t2, fac * X};
    R lUs[5], lUK[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      lSK += lamF[v] * (Us[v] - UK[v]);
      lUs[v] = SK * lamF[v];
      lUK[v] = -SK * lamF[v];
    }
    const R lfac = lUs[0] + Ss * lUs[1] + t1 * lUs[2] + t2 * lUs[3] + X * lUs[4];
    lSs += fac * lUs[1];
    lt1 += fac * lUs[2];
    lt2 += fac * lUs[3];
    const R lX = fac * lUs[4];
    lEK += irK * lX;
    lirK += EK * lX;
    lSs += (Z + Y) * lX;
    luK -= Z * lX;
    const R lwm = (Y * lX) * imK;  // adjoint of w = p_K / m_K, over m_K
    lpK += lwm;
    lmK -= lwm * w;
    const R lfd = lfac * iDd;  // adjoint of fac = m_K / D, over D
    lmK += lfd;
    const R lD = -(lfd * fac);
    lSK += lD;
    lSs -= lD;
    lrK += lUK[0] + t1 * lUK[2] + t2 * lUK[3];
    lmn += lUK[1];
    lt1 += rK * lUK[2];
    lt2 += rK * lUK[3];
    lEK += lUK[4];
  }
  // F_K
  lmn += lamF[0] + uK * lamF[1] + t1 * lamF[2] + t2 * lamF[3];
  luK += mn * lamF[1] + (EK + pK) * lamF[4];
  lpK += lamF[1] + uK * lamF[4];
  lt1 += mn * lamF[2];
  lt2 += mn * lamF[3];
  lEK += uK * lamF[4];
  lrK += uK * lmn;
  luK += rK * lmn;
  lpK += inv_gm1 * lEK;
  lrK += half_(keK * lEK);
  lkeK += half_(rK * lEK);
  // scatter the upwind side's adjoints
  R lrL = 0, luL = 0, lpL = 0, lirL = 0, lSL = 0, lmL = 0;
  R lrR = 0, luR = 0, lpR = 0, lirR = 0, lSR = 0, lmR = 0;
  if (left) {
    lrL += lrK; luL += luK; lqL[2] += lt1; lqL[3] += lt2; lpL += lpK; lkeL += lkeK; lirL += lirK;
    lSL += lSK; lmL += lmK;
  } else {
    lrR += lrK; luR += luK; lqR[2] += lt1; lqR[3] += lt2; lpR += lpK; lkeR += lkeK; lirR += lirK;
    lSR += lSK; lmR += lmK;
  }
  // S* = num / den
  const R lnum = lSs * iden;
  const R lden = -(lnum * Ss);
  lpR += lnum;
  lpL -= lnum;
  luL += mL * lnum;
  lmL += uL * lnum + lden;
  luR -= mR * lnum;
  lmR -= uR * lnum + lden;
  // m_K = rho_K (S_K - u_K)
  lrL += (SL - uL) * lmL;
  lSL += qL[0] * lmL;
  luL -= qL[0] * lmL;
  lrR += (SR - uR) * lmR;
  lSR += qR[0] * lmR;
  luR -= qR[0] * lmR;
  // Davis speeds
  R lcL = 0, lcR = 0;
  if (selL) { luL += lSL; lcL -= lSL; } else { luR += lSL; lcR -= lSL; }
  if (selR) { luL += lSR; lcL += lSR; } else { luR += lSR; lcR += lSR; }
  // c = sqrt(gamma p ir), ir = 1/rho
  const R icc = rcp_(cL * cR);  // 1/c_L = c_R icc, 1/c_R = c_L icc
  const R lxL = half_(lcL) * (cR * icc), lxR = half_(lcR) * (cL * icc);
  lpL += gamma * irL * lxL;
  lirL += gamma * qL[4] * lxL;
  lpR += gamma * irR * lxR;
  lirR += gamma * qR[4] * lxR;
  lrL -= irL * irL * lirL;
  lrR -= irR * irR * lirR;
  lqL[0] += lrL;
  lqL[1] += luL;
  lqL[4] += lpL;
  lqR[0] += lrR;
  lqR[1] += luR;
  lqR[4] += lpR;
}

// Reverse of hllc<D> on (rho, u, v, w, p) states: accumulates lqL, lqR.
template <int D, class R>
__device__ __forceinline__ void hllc_adj(const R qL[5], const R qR[5], R gamma, R inv_gm1, const R lamF[5], R lqL[5],
                                         R lqR[5]) {
  constexpr int N = 1 + D;
  constexpr int T1 = (D == 0) ? 2 : 1;
  constexpr int T2 = (D == 2) ? 2 : 3;
  const R a[5] = {qL[0], qL[N], qL[T1], qL[T2], qL[4]};
  const R b[5] = {qR[0], qR[N], qR[T1], qR[T2], qR[4]};
  const R lF[5] = {lamF[0], lamF[N], lamF[T1], lamF[T2], lamF[4]};
  R la[5] = {0, 0, 0, 0, 0}, lb[5] = {0, 0, 0, 0, 0};
  R lkeL = 0, lkeR = 0;
  hllc_core_adj(a, b, kinetic_sum(qL), kinetic_sum(qR), gamma, inv_gm1, lF, la, lb, lkeL, lkeR);
  lqL[0] += la[0];
  lqL[N] += la[1];
  lqL[T1] += la[2];
  lqL[T2] += la[3];
  lqL[4] += la[4];
  lqR[0] += lb[0];
  lqR[N] += lb[1];
  lqR[T1] += lb[2];
  lqR[T2] += lb[3];
  lqR[4] += lb[4];
#pragma unroll
  for (int m = 1; m <= 3; ++m) {
    lqL[m] += twice_(qL[m] * lkeL);
    lqR[m] += twice_(qR[m] * lkeR);
  }
}

// ------------------------------------------------------------------ Hancock predictor reverse
// qh = q - hdt ((t_x + t_y) + t_z), t_d = A_d(q) dq_d.  Given lqh, adds to lq (including the
// identity) and to ldq[d].
template <class R>
__device__ __forceinline__ void hancock_adj(const R q[5], const R dq[3][5], R gamma, R hdt, const R lqh[5], R lq[5],
                                            R ldq[3][5]) {
  const R ir = rcp_(q[0]);
  const R gp = gamma * q[4];
  R g[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    lq[v] += lqh[v];
    g[v] = -hdt * lqh[v];
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int n = 1 + d;
    const R un = q[n];
    const R* D = dq[d];
    // adjoint with respect to the slopes
    ldq[d][0] += un * g[0];
#pragma unroll
    for (int m = 1; m <= 3; ++m)
      if (m != n) ldq[d][m] += un * g[m];
    ldq[d][n] += q[0] * g[0] + un * g[n] + gp * g[4];
    ldq[d][4] += g[n] * ir + un * g[4];
    // adjoint with respect to the state
    lq[0] += D[n] * g[0] - D[4] * ir * ir * g[n];
    lq[n] += D[0] * g[0] + (D[1] * g[1] + D[2] * g[2] + D[3] * g[3]) + D[4] * g[4];
    lq[4] += gamma * D[n] * g[4];
  }
}

// Reverse of floor_state: zero the adjoint of a floored density / pressure (pre: unfloored).
template <class R>
__device__ __forceinline__ void floor_mask(const R pre[5], R lq[5], R rho_floor, R p_floor) {
  if (cmp_lt_floor(pre[0], rho_floor)) lq[0] = R(0);
  if (cmp_lt_floor(pre[4], p_floor)) lq[4] = R(0);
}

// ------------------------------------------------------------------ recovery reverse
// q = recover(U) with floors; given lq returns lU (same arithmetic type throughout).
template <class R>
__device__ __forceinline__ void recover_adj(const R U[5], const Params& P, const R lq[5], R lU[5]) {
  const R rf = kc<R>(P, K_RHOF);
  const bool rho_free = !(U[0] < rf);
  const R rho = rho_free ? U[0] : rf;
  const R ir = rcp_(rho);
  const R K = (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]);
  const R kin = half_(K * ir);
  const R gm1 = kc<R>(P, K_GM1);
  const R praw = gm1 * (U[4] - kin);
  const R lpr = (praw < kc<R>(P, K_PF)) ? R(0) : lq[4];
  lU[4] = gm1 * lpr;
  const R lkin = -gm1 * lpr;
  R lir = half_(lkin * K);
#pragma unroll
  for (int m = 1; m <= 3; ++m) {
    lU[m] = lq[m] * ir + lkin * U[m] * ir;
    lir += lq[m] * U[m];
  }
  const R lrho = lq[0] - lir * ir * ir;
  lU[0] = rho_free ? lrho : R(0);
}

}  // namespace hydro
