// Ideal MHD with hyperbolic (GLM) divergence cleaning on a periodic box or on AMR patches with two
// ghost layers: the paper's second code
// runs magnetohydrodynamics on the GPU (Enzo MHD, Sec. 4); it prints no equations, so the scheme
// is the textbook one below.
//   U = (rho, m_x, m_y, m_z, E, B_x, B_y, B_z, psi), E = p/(gamma-1) + |m|^2/(2 rho) + |B|^2/2.
//   Primitive w = (rho, u, v, w, p, B, psi) reconstructed with the PLM limiter of the hydro step.
//   Conservative Hancock predictor (Toro, Sec. 14.4, unsplit): each of a cell's six extrapolated
//   states, as conserved, minus dt/(2dx) times the sum over axes of the flux differences of the
//   cell's own extrapolated states; recovered and floored.
//   HLL flux with Davis bounds from the fast magnetosonic speed; the normal field and psi at the
//   face from the 2x2 cleaning system (Dedner et al. 2002): B_n* = (B_nL + B_nR)/2 -
//   (psi_R - psi_L)/(2 c_h), psi* = (psi_L + psi_R)/2 - c_h (B_nR - B_nL)/2; fluxes psi* and
//   c_h^2 B_n*.  c_h = (cfl/3) dx/dt; after the update psi decays by exp(-alpha c_h dt/dx), alpha 0.4.
//
// Float arithmetic (FP32, mixed) steps a periodic box or a batch of patches in one fused launch, a
// column tile marching in z through shared memory (k_mhd_tile / k_mhdp_tile, below), with no
// per-cell scratch.  The 8-byte arithmetic takes three launches, one thread per cell each: predict
// (the cell's six face states into scratch), flux (the HLL flux through the cell's three low faces
// into scratch), update (flux divergence, damping, and the CFL speed of the new state folded into
// dt_next); the scratch holds 6 x 9 face states and 3 x 9 fluxes per cell, structure of arrays, in
// the arithmetic type (its shared-memory tile state would leave one 8-warp block per SM).
// Precision policies as the hydro step: FP64 (double), FP32 (float, SFU reciprocal and square
// root), FP64_DF (double state, double-float arithmetic on the FP32 pipes, the update summed in
// double), MIXED (double state read as float, float arithmetic, the update summed in double).
#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

#include "hydro_device.cuh"
#include "internal.h"
#include "step_tile.cuh"

namespace hydro {
namespace {

constexpr int NV = 9;
constexpr double kMhdAlpha = 0.4;  // psi damping: exp(-alpha c_h dt / dx) per step

template <class Pol>
struct MhdBox {
  using S = typename Pol::S;
  using R = typename Pol::R;
  const S* in[NV];
  S* out[NV];
  R* face;  // [6][NV][cells]: face 2d + h, h = 0 the low, 1 the high face along axis d
  R* flux;  // [3][NV][cells]: the flux through the cell's low face along each axis
  int nx, ny, nz;
  long long cells;
};

template <class R>
struct MhdConst {
  R gamma, gm1, igm1, rf, pf, ch, ch2, ich, hdt, dtdx, damp;  // ich = 1/c_h
  int limiter;
  int valid;  // 0: the step's dt was not positive and finite (nothing is updated)
};

// A stored value in the arithmetic type (double -> double-float exactly, by the IEEE bit fields).
__device__ __forceinline__ double to_r(double x, double*) { return x; }
__device__ __forceinline__ float to_r(float x, float*) { return x; }
__device__ __forceinline__ df to_r(double x, df*) {
  df r;
  split_double(x, r.h, r.l);
  return r;
}
__device__ __forceinline__ double to_double(double x) { return x; }
__device__ __forceinline__ double to_double(float x) { return (double)x; }
__device__ __forceinline__ double to_double(const df& x) { return (double)x; }

// Primitive state of a conserved one, rho and p floored; flags as the hydro recovery.
template <class R>
__device__ __forceinline__ void mhd_recover(const R U[NV], const MhdConst<R>& c, R q[NV], unsigned& flags) {
  if (!isfinite_(U[0])) flags |= HYDRO_EBIT_NONFINITE;
  const bool low = cmp_lt_floor(U[0], c.rf);
  if (low) flags |= HYDRO_EBIT_RHO_FLOOR;
  const R rho = low ? c.rf : U[0];
  const R ir = rcp_(rho);
  const R kin = half_((U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) * ir);
  const R mag = half_(U[5] * U[5] + U[6] * U[6] + U[7] * U[7]);
  const R eint = sub_acc(sub_acc(U[4], kin), mag);
  if (cmp_neg(eint)) flags |= HYDRO_EBIT_P_FLOOR;
  if (!isfinite_(eint)) flags |= HYDRO_EBIT_NONFINITE;
  const R p = c.gm1 * eint;
  q[0] = rho;
  q[1] = U[1] * ir;
  q[2] = U[2] * ir;
  q[3] = U[3] * ir;
  q[4] = cmp_lt_floor(p, c.pf) ? c.pf : p;
  q[5] = U[5];
  q[6] = U[6];
  q[7] = U[7];
  q[8] = U[8];
}

template <class R>
__device__ __forceinline__ void mhd_conserved(const R q[NV], const MhdConst<R>& c, R U[NV]) {
  const R rho = q[0];
  U[0] = rho;
  U[1] = rho * q[1];
  U[2] = rho * q[2];
  U[3] = rho * q[3];
  U[4] = (q[4] * c.igm1 + half_(rho * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]))) +
         half_(q[5] * q[5] + q[6] * q[6] + q[7] * q[7]);
  U[5] = q[5];
  U[6] = q[6];
  U[7] = q[7];
  U[8] = q[8];
}

// Physical flux along axis D with the GLM terms (B_n's flux psi, psi's flux c_h^2 B_n).
template <int D, class R>
__device__ __forceinline__ void mhd_flux(const R q[NV], const MhdConst<R>& c, R F[NV]) {
  constexpr int N = 1 + D;
  const R rho = q[0], p = q[4], un = q[N], Bn = q[5 + D];
  const R B2 = q[5] * q[5] + q[6] * q[6] + q[7] * q[7];
  const R pt = p + half_(B2);
  const R uB = q[1] * q[5] + q[2] * q[6] + q[3] * q[7];
  const R E = (p * c.igm1 + half_(rho * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]))) + half_(B2);
  const R mn = rho * un;
  F[0] = mn;
#pragma unroll
  for (int k = 0; k < 3; ++k) F[1 + k] = mn * q[1 + k] - Bn * q[5 + k];
  F[N] = F[N] + pt;
  F[4] = (E + pt) * un - Bn * uB;
#pragma unroll
  for (int k = 0; k < 3; ++k) F[5 + k] = un * q[5 + k] - q[1 + k] * Bn;
  F[5 + D] = q[8];
  F[8] = c.ch2 * Bn;
}

// Fast magnetosonic speed along an axis from a^2 = gamma p / rho, b^2 = |B|^2 / rho and b_n^2 / rho.
template <class R>
__device__ __forceinline__ R mhd_fast_ab(R a2, R b2, R bn2) {
  const R s = a2 + b2;
  R r = s * s - mulf_(a2 * bn2, 4.f);
  r = cmp_pos(r) ? r : R(0);
  return rsqrt_(half_(s + rsqrt_(r)));
}

template <class R>
__device__ __forceinline__ R mhd_fast(const R q[NV], int d, const MhdConst<R>& c) {
  const R ir = rcp_(q[0]);
  const R bn = d == 0 ? q[5] : (d == 1 ? q[6] : q[7]);
  return mhd_fast_ab(c.gamma * q[4] * ir, (q[5] * q[5] + q[6] * q[6] + q[7] * q[7]) * ir, bn * bn * ir);
}

// CFL speed sum over axes of |u_d| + c_f,d (the same function for the fused and standalone dt);
// 1/rho, a^2 and b^2 formed once for the three axes.
template <class R>
__device__ __forceinline__ R mhd_speed(const R q[NV], const MhdConst<R>& c) {
  const R ir = rcp_(q[0]);
  const R a2 = c.gamma * q[4] * ir;
  const R b2 = (q[5] * q[5] + q[6] * q[6] + q[7] * q[7]) * ir;
  return ((rabs(q[1]) + mhd_fast_ab(a2, b2, q[5] * q[5] * ir)) + (rabs(q[2]) + mhd_fast_ab(a2, b2, q[6] * q[6] * ir))) +
         (rabs(q[3]) + mhd_fast_ab(a2, b2, q[7] * q[7] * ir));
}

template <int D, class R>
__device__ __forceinline__ void mhd_hll(R qL[NV], R qR[NV], const MhdConst<R>& c, R F[NV]) {
  const R Bm = half_(qL[5 + D] + qR[5 + D]) - half_((qR[8] - qL[8]) * c.ich);
  const R pm = half_(qL[8] + qR[8]) - half_(c.ch * (qR[5 + D] - qL[5 + D]));
  qL[5 + D] = qR[5 + D] = Bm;
  qL[8] = qR[8] = pm;
  constexpr int N = 1 + D;
  const R cL = mhd_fast(qL, D, c), cR = mhd_fast(qR, D, c);
  const R a = qL[N] - cL, b = qR[N] - cR, e = qL[N] + cL, f = qR[N] + cR;
  const R SL = a < b ? a : b, SR = e > f ? e : f;
  if (!cmp_neg(SL)) {
    mhd_flux<D>(qL, c, F);
  } else if (!cmp_pos(SR)) {
    mhd_flux<D>(qR, c, F);
  } else {
    // (SR F_L - SL F_R + SL SR (U_R - U_L)) / (SR - SL), accumulated one side at a time so that
    // only one side's flux and state are live
    const R is = rcp_(SR - SL);
    const R ss = SL * SR;
    {
      R Fs[NV], Us[NV];
      mhd_flux<D>(qL, c, Fs);
      mhd_conserved(qL, c, Us);
#pragma unroll
      for (int v = 0; v < NV; ++v) F[v] = SR * Fs[v] - ss * Us[v];
    }
    {
      R Fs[NV], Us[NV];
      mhd_flux<D>(qR, c, Fs);
      mhd_conserved(qR, c, Us);
#pragma unroll
      for (int v = 0; v < NV; ++v) F[v] = ((F[v] - SL * Fs[v]) + ss * Us[v]) * is;
    }
  }
  F[5 + D] = pm;
  F[8] = c.ch2 * Bm;
}

// The same flux and HLL flux for a run-time normal d (one inlined copy serves the x and y faces):
// the components of the normal axis picked by selects, the same operations in the same order.
template <class R>
__device__ __forceinline__ R pick3(int d, R a, R b, R c) {
  return d == 0 ? a : (d == 1 ? b : c);
}

template <class R>
__device__ __forceinline__ void mhd_flux_dyn(int d, const R q[NV], const MhdConst<R>& c, R F[NV]) {
  const R rho = q[0], p = q[4], un = pick3(d, q[1], q[2], q[3]), Bn = pick3(d, q[5], q[6], q[7]);
  const R B2 = q[5] * q[5] + q[6] * q[6] + q[7] * q[7];
  const R pt = p + half_(B2);
  const R uB = q[1] * q[5] + q[2] * q[6] + q[3] * q[7];
  const R E = (p * c.igm1 + half_(rho * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]))) + half_(B2);
  const R mn = rho * un;
  F[0] = mn;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const R m = mn * q[1 + k] - Bn * q[5 + k];
    F[1 + k] = k == d ? m + pt : m;
  }
  F[4] = (E + pt) * un - Bn * uB;
#pragma unroll
  for (int k = 0; k < 3; ++k) F[5 + k] = k == d ? q[8] : un * q[5 + k] - q[1 + k] * Bn;
  F[8] = c.ch2 * Bn;
}

template <class R>
__device__ __forceinline__ void mhd_hll_dyn(int d, R qL[NV], R qR[NV], const MhdConst<R>& c, R F[NV]) {
  const R bL = pick3(d, qL[5], qL[6], qL[7]), bR = pick3(d, qR[5], qR[6], qR[7]);
  const R Bm = half_(bL + bR) - half_((qR[8] - qL[8]) * c.ich);
  const R pm = half_(qL[8] + qR[8]) - half_(c.ch * (bR - bL));
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (k == d) qL[5 + k] = qR[5 + k] = Bm;
  }
  qL[8] = qR[8] = pm;
  const R cL = mhd_fast(qL, d, c), cR = mhd_fast(qR, d, c);
  const R uL = pick3(d, qL[1], qL[2], qL[3]), uR = pick3(d, qR[1], qR[2], qR[3]);
  const R a = uL - cL, b = uR - cR, e = uL + cL, f = uR + cR;
  const R SL = a < b ? a : b, SR = e > f ? e : f;
  if (!cmp_neg(SL)) {
    mhd_flux_dyn(d, qL, c, F);
  } else if (!cmp_pos(SR)) {
    mhd_flux_dyn(d, qR, c, F);
  } else {
    const R is = rcp_(SR - SL);
    const R ss = SL * SR;
    {
      R Fs[NV], Us[NV];
      mhd_flux_dyn(d, qL, c, Fs);
      mhd_conserved(qL, c, Us);
#pragma unroll
      for (int v = 0; v < NV; ++v) F[v] = SR * Fs[v] - ss * Us[v];
    }
    {
      R Fs[NV], Us[NV];
      mhd_flux_dyn(d, qR, c, Fs);
      mhd_conserved(qR, c, Us);
#pragma unroll
      for (int v = 0; v < NV; ++v) F[v] = ((F[v] - SL * Fs[v]) + ss * Us[v]) * is;
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (k == d) F[5 + k] = pm;
  }
  F[8] = c.ch2 * Bm;
}

__device__ __forceinline__ void cell_of(long long a, int nx, int ny, int& i, int& j, int& k) {
  const int t = (int)a;  // cells < 2^31
  const int row = t / nx;
  i = t - row * nx;
  k = row / ny;
  j = row - k * ny;
}

template <class Pol>
__device__ __forceinline__ void load_q(const MhdBox<Pol>& B, long long a, const MhdConst<typename Pol::R>& c,
                                       typename Pol::R q[NV], unsigned& flags) {
  using R = typename Pol::R;
  R U[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) U[v] = to_r(__ldg(B.in[v] + a), (R*)nullptr);
  mhd_recover(U, c, q, flags);
}

// The three-launch form (8-byte arithmetic): a cell's two extrapolated states along axis D into the
// scratch (read back for their advance: no registers to spare for the 27 slopes) and the flux
// difference of those states added into dF.
template <int D, class Pol>
__device__ __forceinline__ void axis_states(const MhdBox<Pol>& B, long long a, long long am, long long ap,
                                            const typename Pol::R q[NV], const MhdConst<typename Pol::R>& c,
                                            typename Pol::R dF[NV]) {
  using R = typename Pol::R;
  unsigned nf = 0;  // neighbours are flagged by their own threads
  R lo[NV], hi[NV];
  {
    R qm[NV], qp[NV];
    load_q(B, am, c, qm, nf);
    load_q(B, ap, c, qp, nf);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const R s = limited(q[v] - qm[v], qp[v] - q[v], c.limiter);
      lo[v] = q[v] - half_(s);
      hi[v] = q[v] + half_(s);
      B.face[((long long)(2 * D) * NV + v) * B.cells + a] = lo[v];
      B.face[((long long)(2 * D + 1) * NV + v) * B.cells + a] = hi[v];
    }
  }
  R Fh[NV];
  mhd_flux<D>(hi, c, Fh);
  {
    R Fl[NV];
    mhd_flux<D>(lo, c, Fl);
#pragma unroll
    for (int v = 0; v < NV; ++v) dF[v] = D == 0 ? Fh[v] - Fl[v] : dF[v] + (Fh[v] - Fl[v]);
  }
}

// Two resident blocks of 256 threads per SM at least (the register budget of 128 per thread): the
// double-float kernels otherwise take ~170 registers and leave 8 warps per SM for long dependent
// chains.
template <class Pol>
__global__ void __launch_bounds__(256, 2) k_mhd_predict(MhdBox<Pol> B, const MhdConst<typename Pol::R>* cp, unsigned* err) {
  using R = typename Pol::R;
  const MhdConst<R> c = *cp;
  if (!c.valid) return;
  unsigned flags = 0;
  for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < B.cells;
       a += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    cell_of(a, B.nx, B.ny, i, j, k);
    const long long sy = B.nx, sz = (long long)B.nx * B.ny;
    const long long axm = a + (i == 0 ? B.nx - 1 : -1), axp = a + (i == B.nx - 1 ? -(B.nx - 1) : 1);
    const long long aym = a + (j == 0 ? (B.ny - 1) * sy : -sy), ayp = a + (j == B.ny - 1 ? -(B.ny - 1) * sy : sy);
    const long long azm = a + (k == 0 ? (B.nz - 1) * sz : -sz), azp = a + (k == B.nz - 1 ? -(B.nz - 1) * sz : sz);
    R q[NV], dF[NV];
    load_q(B, a, c, q, flags);
    axis_states<0>(B, a, axm, axp, q, c, dF);
    axis_states<1>(B, a, aym, ayp, q, c, dF);
    axis_states<2>(B, a, azm, azp, q, c, dF);
    // the six extrapolated states advanced by half a step, recovered and floored (this thread's
    // own scratch entries written just above)
    unsigned nf = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        const int f = 2 * d + h;
        R w[NV], U[NV], r[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) w[v] = B.face[((long long)f * NV + v) * B.cells + a];
        mhd_conserved(w, c, U);
#pragma unroll
        for (int v = 0; v < NV; ++v) U[v] = U[v] - c.hdt * dF[v];
        mhd_recover(U, c, r, nf);
#pragma unroll
        for (int v = 0; v < NV; ++v) B.face[((long long)f * NV + v) * B.cells + a] = r[v];
      }
    }
  }
  flush_flags(flags, err);
}

template <int D, class Pol>
__device__ __forceinline__ void low_face_flux(const MhdBox<Pol>& B, long long a, long long am,
                                              const MhdConst<typename Pol::R>& c) {
  using R = typename Pol::R;
  R qL[NV], qR[NV], F[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    qL[v] = B.face[((long long)(2 * D + 1) * NV + v) * B.cells + am];  // high face of the cell below
    qR[v] = B.face[((long long)(2 * D) * NV + v) * B.cells + a];       // low face of this cell
  }
  mhd_hll<D>(qL, qR, c, F);
#pragma unroll
  for (int v = 0; v < NV; ++v) B.flux[((long long)D * NV + v) * B.cells + a] = F[v];
}

template <class Pol>
__global__ void __launch_bounds__(256, 2) k_mhd_flux(MhdBox<Pol> B, const MhdConst<typename Pol::R>* cp) {
  const MhdConst<typename Pol::R> c = *cp;
  if (!c.valid) return;
  for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < B.cells;
       a += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    cell_of(a, B.nx, B.ny, i, j, k);
    const long long sy = B.nx, sz = (long long)B.nx * B.ny;
    low_face_flux<0>(B, a, a + (i == 0 ? B.nx - 1 : -1), c);
    low_face_flux<1>(B, a, a + (j == 0 ? (B.ny - 1) * sy : -sy), c);
    low_face_flux<2>(B, a, a + (k == 0 ? (B.nz - 1) * sz : -sz), c);
  }
}

template <class R>
__device__ __forceinline__ R block_max_r(R v) {
  __shared__ R red[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const R w = shfl_xor_(v, o);
    v = w > v ? w : v;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = red[w] > v ? red[w] : v;
  return v;
}

// The update of cell a from its flux divergence div (x, y, z summed in that order), psi damping, and
// the CFL speed of the new state folded into smax when dt_next is wanted.
template <class Pol>
__device__ __forceinline__ void mhd_update_cell(const MhdBox<Pol>& B, long long a, const MhdConst<typename Pol::R>& c,
                                                const typename Pol::R div[NV], bool want_cfl, unsigned& flags,
                                                typename Pol::R& smax) {
  using S = typename Pol::S;
  using R = typename Pol::R;
  S Un[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) Un[v] = Pol::update(__ldg(B.in[v] + a), c.dtdx, div[v]);
  Un[8] = Un[8] * (S)to_double(c.damp);
#pragma unroll
  for (int v = 0; v < NV; ++v) B.out[v][a] = Un[v];
  if (want_cfl) {
    R U[NV], q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) U[v] = to_r(Un[v], (R*)nullptr);
    mhd_recover(U, c, q, flags);
    const R s = mhd_speed(q, c);
    smax = s > smax ? s : smax;
  }
}

template <class Pol>
__global__ void __launch_bounds__(256, 2) k_mhd_update(MhdBox<Pol> B, const MhdConst<typename Pol::R>* cp, double cfl,
                                                    double dx, double* dt_next, unsigned* err) {
  using R = typename Pol::R;
  const MhdConst<R> c = *cp;
  if (!c.valid) return;
  unsigned flags = 0;
  R smax = R(0);
  for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < B.cells;
       a += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    cell_of(a, B.nx, B.ny, i, j, k);
    const long long sy = B.nx, sz = (long long)B.nx * B.ny;
    const long long bx = a + (i == B.nx - 1 ? -(B.nx - 1) : 1);
    const long long by = a + (j == B.ny - 1 ? -(B.ny - 1) * sy : sy);
    const long long bz = a + (k == B.nz - 1 ? -(B.nz - 1) * sz : sz);
    R div[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const R* fx = B.flux + (long long)(0 * NV + v) * B.cells;
      const R* fy = B.flux + (long long)(1 * NV + v) * B.cells;
      const R* fz = B.flux + (long long)(2 * NV + v) * B.cells;
      div[v] = ((fx[bx] - fx[a]) + (fy[by] - fy[a])) + (fz[bz] - fz[a]);
    }
    mhd_update_cell(B, a, c, div, dt_next != nullptr, flags, smax);
  }
  if (dt_next) {
    const R m = block_max_r(smax);
    if (threadIdx.x == 0) publish_dt(cfl, dx, to_double(m), dt_next);
  }
  flush_flags(flags, err);
}

// ------------------------------------------------------------------ fused tile step
// One launch per step: a TX x TY column tile marching in z, the structure of the hydro step.  The
// primitive planes p-1, p, p+1 of the tile plus two halo cells per side sit in a shared-memory ring.
// Per plane p, two phases between block barriers:
//   1  each column predicts its cell of plane p (slopes, the six extrapolated states advanced by the
//      conservative Hancock half step and recovered): the four in-plane face states go to shared
//      memory, the low z state meets the high z state of plane p-1 (kept in registers) in the HLL
//      flux of face p-1/2, and the column's cell of plane p-1 is updated from its x/y fluxes (shared
//      memory) and its two z fluxes; the last warps then predict one ring cell per thread, for its
//      face state toward the tile
//   2  the HLL fluxes of plane p's x and y faces, each once, into shared memory, and the load of
//      plane p+2 (recovered) into the slot of plane p-1; split named barriers let the ring warps
//      take the tile-edge faces while the other warps take the interior faces and the load
// No global scratch: each cell is read once per plane (halo re-reads from L2) and written once; the
// operations and their order per cell are those of the three-launch form.
template <class R, int TX, int TY, class Off>
struct MhdTileShared {
  R q[3][NV][TY + 4][TX + 4];  // primitive planes, slot (p + 3) % 3
  R lx[NV][TY][TX + 1];        // low x face state of cell i, i = 0 .. TX (TX: the right ring cell)
  R hx[NV][TY][TX + 1];        // high x face state of cell i - 1 (i = 0: the left ring cell)
  R ly[NV][TY + 1][TX];        // low y face state of cell j, j = 0 .. TY
  R hy[NV][TY + 1][TX];        // high y face state of cell j - 1
  R fx[NV][TY][TX + 1];        // HLL flux through the x face between cells i - 1 and i
  R fy[NV][TY + 1][TX];        // HLL flux through the y face between cells j - 1 and j
  Off yoff[TY + 4];            // y offset (stored y index x its stride) of the halo rows
  int xoff[TX + 4];            // stored x index of the halo columns
};


constexpr int kMhdTX = 32, kMhdTY = 8;  // one row per warp: conflict-free shared rows
constexpr int kMhdPatchZChunk = 32;     // planes per tile record of a patch

// The policies whose periodic step runs the fused tile kernel: float arithmetic (FP32, mixed; at
// 256^3 +15% and +35% over the three-launch form).  The 8-byte arithmetic's tile state fills an SM
// with one 8-warp block (FP64 -21%, double-float -39%): those keep the three launches.
template <class Pol>
constexpr bool kMhdFused = sizeof(typename Pol::R) == 4;

// Resident blocks per SM: float arithmetic fits two tiles' shared memory per SM, 8-byte one.
template <class Pol>
constexpr int mhd_tile_blocks() {
  return sizeof(typename Pol::R) == 4 ? 2 : 1;
}

// Slopes of the cell (ci, cj) of plane p (tile coordinates; the ring at -1 and TX / TY) and the
// sum over axes of the flux differences of its extrapolated states, as axis_states.
template <class Pol, class Sh>
__device__ __forceinline__ void mhd_tile_predict(const Sh& sm, int ci, int cj,
                                                 int sm1, int s0, int sp1, const MhdConst<typename Pol::R>& c,
                                                 typename Pol::R q[NV], typename Pol::R sl[3][NV],
                                                 typename Pol::R dF[NV]) {
  using R = typename Pol::R;
  const int x = ci + 2, y = cj + 2;
#pragma unroll
  for (int v = 0; v < NV; ++v) q[v] = sm.q[s0][v][y][x];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    R lo[NV], hi[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const R qm = d == 0 ? sm.q[s0][v][y][x - 1] : (d == 1 ? sm.q[s0][v][y - 1][x] : sm.q[sm1][v][y][x]);
      const R qp = d == 0 ? sm.q[s0][v][y][x + 1] : (d == 1 ? sm.q[s0][v][y + 1][x] : sm.q[sp1][v][y][x]);
      const R s = limited(q[v] - qm, qp - q[v], c.limiter);
      sl[d][v] = s;
      lo[v] = q[v] - half_(s);
      hi[v] = q[v] + half_(s);
    }
    R Fh[NV], Fl[NV];
    if (d == 0) {
      mhd_flux<0>(hi, c, Fh);
      mhd_flux<0>(lo, c, Fl);
    } else if (d == 1) {
      mhd_flux<1>(hi, c, Fh);
      mhd_flux<1>(lo, c, Fl);
    } else {
      mhd_flux<2>(hi, c, Fh);
      mhd_flux<2>(lo, c, Fl);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) dF[v] = d == 0 ? Fh[v] - Fl[v] : dF[v] + (Fh[v] - Fl[v]);
  }
}

// One extrapolated state (low, h = 0, or high, h = 1, along the axis of the slopes sl) advanced by
// half a step and recovered (floored; its flags belong to no cell and are dropped).
template <class R>
__device__ __forceinline__ void mhd_face_state(const R q[NV], const R sl[NV], const R dF[NV], int h,
                                               const MhdConst<R>& c, R r[NV]) {
  R w[NV], U[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) w[v] = h ? q[v] + half_(sl[v]) : q[v] - half_(sl[v]);
  mhd_conserved(w, c, U);
#pragma unroll
  for (int v = 0; v < NV; ++v) U[v] = U[v] - c.hdt * dF[v];
  unsigned nf = 0;
  mhd_recover(U, c, r, nf);
}

// The tile [x0, x0+TX) x [y0, y0+TY) x [z0, z1) of box B advanced by one step (want_cfl: the
// largest CFL speed of its new cells into smax); every thread of the block calls it.  GH: B is an
// AMR patch (HostMhdPatch) whose input carries two ghost layers filled by the caller and whose
// output carries B.gout (left as they are); else B is a periodic box (MhdBox: indices wrap, the
// fields contiguous).  Fixed at compile time, so that the periodic kernel carries no strides.
// Offsets of the halo rows: int on a periodic box (fewer than 2^31 cells), 64-bit on a patch.
template <bool GH>
using MhdOff = typename std::conditional<GH, long long, int>::type;
template <class Pol, int TX, int TY, bool GH>
using MhdTileSh = MhdTileShared<typename Pol::R, TX, TY, MhdOff<GH>>;

template <class Pol, int TX, int TY, bool GH, class Box>
__device__ __forceinline__ void mhd_tile_body(MhdTileSh<Pol, TX, TY, GH>& sm, const Box& B,
                                              const MhdConst<typename Pol::R>& c,
                                              int x0, int y0, int z0, int z1, bool want_cfl, unsigned& flags,
                                              typename Pol::R& smax) {
  using S = typename Pol::S;
  using R = typename Pol::R;
  constexpr int NT = TX * TY, QW = TX + 4, QH = TY + 4, QN = QW * QH;
  // ring cells, taken by the last RW whole warps (NTI threads before them); faces between two
  // tile cells: NIX in x, NIF in all
  constexpr int NR = 2 * (TX + TY), RW = (NR + 31) / 32, NTI = NT - 32 * RW;
  constexpr int NIX = (TX - 1) * TY, NIF = NIX + TX * (TY - 1);
  static_assert(NTI > 0 && NT % 32 == 0, "whole warps on both sides of the split");
  const int tid = threadIdx.x, ti = tid % TX, tj = tid / TX;
  const int nx = B.nx, ny = B.ny, nz = B.nz;
  // field pointers, read where used (a periodic box's from the kernel parameters)
  auto fin = [&](int v) -> const S* { return static_cast<const S*>(B.in[v]); };
  auto fout = [&](int v) -> S* { return static_cast<S*>(B.out[v]); };
  constexpr bool periodic = !GH;
  constexpr int gin = GH ? 2 : 0;
  long long isy = nx, isz = (long long)nx * ny, osy = isy, osz = isz;
  int gout = 0;
  if constexpr (GH) {
    isy = B.isy; isz = B.isz; osy = B.osy; osz = B.osz;
    gout = B.gout;
  }
  __syncthreads();  // the previous tile of this block is done with the offsets
  for (int k = tid; k < QW; k += NT) {
    const int x = x0 - 2 + k;
    sm.xoff[k] = periodic ? wrapi(x, nx) : min(max(x, -2), nx + 1) + 2;
  }
  for (int k = tid; k < QH; k += NT) {
    const int y = y0 - 2 + k;
    sm.yoff[k] = (MhdOff<GH>)(periodic ? wrapi(y, ny) : min(max(y, -2), ny + 1) + 2) * (MhdOff<GH>)isy;
  }
  __syncthreads();

  // extents of the input and output arrays (elements per field), for the bounds-checked build
  const long long in_extent = (long long)(nz + 2 * gin) * isz, out_extent = (long long)(nz + 2 * gout) * osz;
  // plane z of the tile and its halo, recovered into its ring slot, cells first, first + stride,
  // ...; the flags of a cell count once, in the tile that updates it
  auto load_plane = [&](int z, int first, int stride) {
    R(&qs)[NV][TY + 4][TX + 4] = sm.q[ring_slot(z)];
    const long long zo = (long long)(periodic ? wrapi(z, nz) : z + 2) * isz;
    const bool zmine = z >= z0 && z < z1;
    for (int k = first; k < QN; k += stride) {
      const int cy = k / QW, cx = k - cy * QW;
      const long long a = zo + sm.yoff[cy] + sm.xoff[cx];
      const bool ok = index_ok(a, in_extent, flags);  // (always true outside the checked build)
      R U[NV], w[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) U[v] = ok ? to_r(__ldg(fin(v) + a), (R*)nullptr) : R(0);
      unsigned f = 0;
      mhd_recover(U, c, w, f);
      if (zmine && cx >= 2 && cx < TX + 2 && cy >= 2 && cy < TY + 2 && x0 + cx - 2 < nx && y0 + cy - 2 < ny) flags |= f;
#pragma unroll
      for (int v = 0; v < NV; ++v) qs[v][cy][cx] = w[v];
    }
  };

  const bool own = (x0 + ti < nx) && (y0 + tj < ny);
  const bool ringw = tid >= NTI;
  const int r = tid - NTI;  // ring cell of a ring-warp thread (r < NR)
  R LzPrev[NV], FzPrev[NV], Fz[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) LzPrev[v] = FzPrev[v] = Fz[v] = R(0);

  // the column's cell of plane k: the x/y flux differences of plane k and its two z fluxes
  auto update = [&](int k) {
    R div[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v)
      div[v] = ((sm.fx[v][tj][ti + 1] - sm.fx[v][tj][ti]) + (sm.fy[v][tj + 1][ti] - sm.fy[v][tj][ti])) +
               (Fz[v] - FzPrev[v]);
    const int gx = x0 + ti, gy = y0 + tj;
    const long long ai = (long long)(k + gin) * isz + (long long)(gy + gin) * isy + (gx + gin);
    const long long ao = GH ? (long long)(k + gout) * osz + (long long)(gy + gout) * osy + (gx + gout) : ai;
    if (!index_ok(ai, in_extent, flags) || !index_ok(ao, out_extent, flags)) return;
    S Un[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Un[v] = Pol::update(__ldg(fin(v) + ai), c.dtdx, div[v]);
    Un[8] = Un[8] * (S)to_double(c.damp);
#pragma unroll
    for (int v = 0; v < NV; ++v) fout(v)[ao] = Un[v];
    if (want_cfl) {
      R U[NV], w[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) U[v] = to_r(Un[v], (R*)nullptr);
      mhd_recover(U, c, w, flags);
      const R s = mhd_speed(w, c);
      smax = s > smax ? s : smax;
    }
  };
  // the HLL flux through the x face between cells i - 1 and i of row j (d = 0), or the y face
  // between rows j - 1 and j of column i (d = 1)
  auto face = [&](int d, int i, int j) {
    constexpr int XS = TY * (TX + 1), YS = (TY + 1) * TX;  // field strides of the x / y arrays
    const int o = d == 0 ? j * (TX + 1) + i : j * TX + i, st = d == 0 ? XS : YS;
    const R* hs = d == 0 ? &sm.hx[0][0][0] : &sm.hy[0][0][0];
    const R* ls = d == 0 ? &sm.lx[0][0][0] : &sm.ly[0][0][0];
    R* fs = d == 0 ? &sm.fx[0][0][0] : &sm.fy[0][0][0];
    R qL[NV], qR[NV], F[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      qL[v] = hs[v * st + o];
      qR[v] = ls[v * st + o];
    }
    mhd_hll_dyn(d, qL, qR, c, F);
#pragma unroll
    for (int v = 0; v < NV; ++v) fs[v * st + o] = F[v];
  };
  auto ring_cell = [&](int& ci, int& cj, unsigned& mask) {
    if (r < TX) { ci = r; cj = -1; mask = 8u; }                       // below the tile: high y state
    else if (r < 2 * TX) { ci = r - TX; cj = TY; mask = 4u; }         // above: low y
    else if (r < 2 * TX + TY) { ci = -1; cj = r - 2 * TX; mask = 2u; }  // left: high x
    else { ci = TX; cj = r - 2 * TX - TY; mask = 1u; }                // right: low x
  };

  load_plane(z0 - 2, NT - 1 - tid, NT);
  load_plane(z0 - 1, NT - 1 - tid, NT);
  load_plane(z0, NT - 1 - tid, NT);
  __syncthreads();
  // Per plane p:
  //   1  every thread predicts its column's cell (its z face p-1/2 and the update of plane p-1
  //      follow); on x/y planes the ring warps then signal barrier 1 and predict their ring cells
  //   2  (x/y planes) the other warps, once every tile cell is predicted (barrier 1), signal
  //      barrier 2 and take the faces between two tile cells, then, once the ring cells are
  //      predicted (barrier 3: plane p-1 no longer read), load plane p+2 into its slot; the ring
  //      warps, after barrier 2, take the faces between their ring cell and the tile
  for (int p = z0 - 1; p <= z1; ++p) {
    const int sm1 = ring_slot(p - 1), s0 = ring_slot(p), sp1 = ring_slot(p + 1);
    const bool xy = p >= z0 && p < z1;
    // ---- phase 1: the column's cell (it = 0), then a ring cell (it = 1), through one call site
    for (int it = 0; it < 2; ++it) {
      int ci = ti, cj = tj;
      unsigned mask;  // face states wanted: bit 2d + h, h = 0 low, 1 high along axis d
      if (it == 0) {
        mask = (xy ? 0xFu : 0u) | (p >= z0 && own ? 0x10u : 0u) | (p < z1 ? 0x20u : 0u);
      } else {
        if (!xy || !ringw || r >= NR) break;
        ring_cell(ci, cj, mask);
      }
      R q[NV], sl[3][NV], dF[NV];
      mhd_tile_predict<Pol>(sm, ci, cj, sm1, s0, sp1, c, q, sl, dF);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          if (!((mask >> (2 * d + h)) & 1u)) continue;
          R rs[NV];
          mhd_face_state(q, sl[d], dF, h, c, rs);
          if (d == 0) {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              if (h) sm.hx[v][cj][ci + 1] = rs[v];
              else sm.lx[v][cj][ci] = rs[v];
            }
          } else if (d == 1) {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              if (h) sm.hy[v][cj + 1][ci] = rs[v];
              else sm.ly[v][cj][ci] = rs[v];
            }
          } else if (h == 0) {
            mhd_hll<2>(LzPrev, rs, c, Fz);  // face p-1/2
          } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) LzPrev[v] = rs[v];
          }
        }
      }
      if (it == 0) {
        if (p >= z0 + 1 && own) update(p - 1);
#pragma unroll
        for (int v = 0; v < NV; ++v) FzPrev[v] = Fz[v];
        if (xy && ringw) bar_arrive(1, NT);
      }
    }
    if (!xy) {
      __syncthreads();
      if (p + 2 <= z1 + 1) load_plane(p + 2, NT - 1 - tid, NT);
      __syncthreads();
      continue;
    }
    // ---- phase 2 (x/y plane; p + 2 <= z1 + 1): faces f < NIF between two tile cells (x, then
    // y), f = NIF + r between ring cell r and the tile, through one call site
    if (ringw) {
      bar_arrive(3, NT);
      bar_sync(2, NT);
    } else {
      bar_sync(1, NT);
      bar_arrive(2, NT);
    }
    const int fend = ringw ? (r < NR ? NIF + r + 1 : 0) : NIF;
    for (int f = ringw ? NIF + r : tid; f < fend; f += NTI) {
      int d, i, j;
      if (f < NIX) {
        d = 0; j = f / (TX - 1); i = f - j * (TX - 1) + 1;
      } else if (f < NIF) {
        const int g = f - NIX;
        d = 1; j = g / TX; i = g - j * TX; j += 1;
      } else {
        const int e = f - NIF;
        if (e < TX) { d = 1; i = e; j = 0; }
        else if (e < 2 * TX) { d = 1; i = e - TX; j = TY; }
        else if (e < 2 * TX + TY) { d = 0; i = 0; j = e - 2 * TX; }
        else { d = 0; i = TX; j = e - 2 * TX - TY; }
      }
      face(d, i, j);
    }
    if (!ringw) {
      bar_sync(3, NT);
      load_plane(p + 2, NTI - 1 - tid, NTI);
    }
    __syncthreads();
  }
}

// Periodic box: one tile per block, tiles from the block index.
template <class Pol, int TX, int TY>
__global__ void __launch_bounds__(TX* TY, (mhd_tile_blocks<Pol>()))
    k_mhd_tile(MhdBox<Pol> B, const MhdConst<typename Pol::R>* cp, double cfl, double dx, double* dt_next, int zchunk,
               unsigned* err) {
  using R = typename Pol::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& sm = *reinterpret_cast<MhdTileSh<Pol, TX, TY, false>*>(smem_raw);
  const MhdConst<R> c = *cp;
  if (!c.valid) return;
  const int z0 = blockIdx.z * zchunk;
  unsigned flags = 0;
  R smax = R(0);
  mhd_tile_body<Pol, TX, TY, false>(sm, B, c, blockIdx.x * TX, blockIdx.y * TY, z0, min(z0 + zchunk, B.nz),
                                    dt_next != nullptr, flags, smax);
  if (dt_next) {
    const R m = block_max_r(smax);
    if (threadIdx.x == 0) publish_dt(cfl, dx, to_double(m), dt_next);
  }
  flush_flags(flags, err);
}

// AMR patches with two ghost layers: one tile record (patch, x0, y0, z0) per block, each patch's
// constants and dt slot its own.
template <class Pol, int TX, int TY>
__global__ void __launch_bounds__(TX* TY, (mhd_tile_blocks<Pol>()))
    k_mhdp_tile(const HostMhdPatch* patches, const int4* tiles, const MhdConst<typename Pol::R>* consts, double cfl,
                double* dt_next, int zchunk, unsigned* err) {
  using R = typename Pol::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& sm = *reinterpret_cast<MhdTileSh<Pol, TX, TY, true>*>(smem_raw);
  const int4 t = tiles[blockIdx.x];
  const HostMhdPatch H = patches[t.x];  // in registers: its pointers are read at every load
  const MhdConst<R> c = consts[t.x];
  if (!c.valid) return;  // (block-uniform)
  unsigned flags = 0;
  R smax = R(0);
  mhd_tile_body<Pol, TX, TY, true>(sm, H, c, t.y, t.z, t.w, min(t.w + zchunk, H.nz), dt_next != nullptr, flags, smax);
  if (dt_next) {
    const R m = block_max_r(smax);
    if (threadIdx.x == 0) publish_dt(cfl, H.dx, to_double(m), dt_next + t.x);
  }
  flush_flags(flags, err);
}

// Planes per z chunk: the fewest waves of resident blocks times the planes a block marches (its
// chunk plus the plane below it, predicted for its z face, and the two halo loads of each end).
inline int mhd_zchunk(int nx, int ny, int nz, int resident) {
  const long long cols = (long long)((nx + kMhdTX - 1) / kMhdTX) * ((ny + kMhdTY - 1) / kMhdTY);
  int best = nz;
  double best_cost = 1e300;
  for (int zc = 8; zc <= 128; zc *= 2) {
    const int z = zc < nz ? zc : nz;
    const long long blocks = cols * ((nz + z - 1) / z);
    const long long waves = (blocks + resident - 1) / resident;
    const double cost = (double)waves * (z + 1.5);
    if (cost < best_cost) {
      best_cost = cost;
      best = z;
    }
    if (z == nz) break;
  }
  return best;
}

template <class Pol>
cudaError_t mhd_tile_launch(const MhdBox<Pol>& B, const MhdConst<typename Pol::R>* cp, double cfl, double dx,
                            double* dt_next, unsigned* err, cudaStream_t s) {
  using R = typename Pol::R;
  constexpr int TX = kMhdTX, TY = kMhdTY;
  const size_t smem = sizeof(MhdTileSh<Pol, TX, TY, false>);
  static PerDeviceOnce attr;
  cudaError_t e = attr.call([&] {
    return cudaFuncSetAttribute(k_mhd_tile<Pol, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int zc = mhd_zchunk(B.nx, B.ny, B.nz, sms * mhd_tile_blocks<Pol>());
  dim3 grid((B.nx + TX - 1) / TX, (B.ny + TY - 1) / TY, (B.nz + zc - 1) / zc);
  k_mhd_tile<Pol, TX, TY><<<grid, TX * TY, smem, s>>>(B, cp, cfl, dx, dt_next, zc, err);
  return cudaGetLastError();
}

template <class Pol>
__global__ void __launch_bounds__(256) k_mhd_cfl(MhdBox<Pol> B, MhdConst<typename Pol::R> c, double cfl, double dx,
                                                 double* dt, unsigned* err) {
  using R = typename Pol::R;
  unsigned flags = 0;
  R smax = R(0);
  for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < B.cells;
       a += (long long)gridDim.x * blockDim.x) {
    R q[NV];
    load_q(B, a, c, q, flags);
    const R s = mhd_speed(q, c);
    smax = s > smax ? s : smax;
  }
  const R m = block_max_r(smax);
  if (threadIdx.x == 0) publish_dt(cfl, dx, to_double(m), dt);
  flush_flags(flags, err);
}

// c_h and the half-step factors need dt, which lives on the device: a one-thread kernel turns it
// into the constants the three step kernels read.
template <class R>
__global__ void k_mhd_consts(MhdConst<R> base, double cfl, double dx, double alpha, const double* dt_dev,
                             MhdConst<R>* out, unsigned* err) {
  const double dt = dt_dev[0];
  MhdConst<R> c = base;
  c.valid = dt > 0.0 && dt <= 1e300;
  if (!c.valid) {
    atomicOr(err, HYDRO_EBIT_BAD_DT);
  } else {
    const double ch = (cfl / 3.0) * dx / dt;
    c.ch = R(ch);
    c.ch2 = R(ch * ch);
    c.ich = R(1.0 / ch);
    c.hdt = R(0.5 * dt / dx);
    c.dtdx = R(dt / dx);
    c.damp = R(exp(-alpha * ch * dt / dx));
  }
  *out = c;
}

template <class Pol>
MhdBox<Pol> box_of(const HostMhdBox& h, void* scratch) {
  using S = typename Pol::S;
  using R = typename Pol::R;
  MhdBox<Pol> b;
  for (int v = 0; v < NV; ++v) {
    b.in[v] = static_cast<const S*>(h.in[v]);
    b.out[v] = static_cast<S*>(h.out[v]);
  }
  b.nx = h.nx;
  b.ny = h.ny;
  b.nz = h.nz;
  b.cells = (long long)h.nx * h.ny * h.nz;
  // scratch: the step's constants in the first 256 bytes, then the face states and the fluxes
  b.face = scratch ? reinterpret_cast<R*>(static_cast<char*>(scratch) + 256) : nullptr;
  b.flux = b.face ? b.face + 6LL * NV * b.cells : nullptr;
  return b;
}

template <class R>
MhdConst<R> consts_of(const Params& prm) {
  MhdConst<R> c{};
  c.gamma = R(prm.gamma);
  c.gm1 = R(prm.gamma - 1.0);
  c.igm1 = R(1.0 / (prm.gamma - 1.0));
  c.rf = R(prm.rho_floor);
  c.pf = R(prm.p_floor);
  c.limiter = prm.limiter;
  c.valid = 1;
  return c;
}

int grid_for(long long cells) {
  const long long b = (cells + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 152LL * 64 ? 152LL * 64 : b));
}

template <class Pol>
cudaError_t mhd_step_t(const HostMhdBox& h, const Params& prm, const double* dt, double* dt_next, void* scratch,
                       unsigned* err, cudaStream_t s) {
  using R = typename Pol::R;
  MhdBox<Pol> B = box_of<Pol>(h, scratch);
  static_assert(sizeof(MhdConst<R>) <= 256, "the constants fit before the face states");
  auto* cp = static_cast<MhdConst<R>*>(scratch);
  k_mhd_consts<R><<<1, 1, 0, s>>>(consts_of<R>(prm), prm.cfl, h.dx, kMhdAlpha, dt, cp, err);
  if constexpr (kMhdFused<Pol>) {
    B.face = B.flux = nullptr;  // no per-cell scratch
    return mhd_tile_launch<Pol>(B, cp, prm.cfl, h.dx, dt_next, err, s);
  } else {
    const int g = grid_for(B.cells);
    k_mhd_predict<Pol><<<g, 256, 0, s>>>(B, cp, err);
    k_mhd_flux<Pol><<<g, 256, 0, s>>>(B, cp);
    k_mhd_update<Pol><<<g, 256, 0, s>>>(B, cp, prm.cfl, h.dx, dt_next, err);
    return cudaGetLastError();
  }
}

template <class Pol>
cudaError_t mhd_cfl_t(const HostMhdBox& h, const Params& prm, double* dt, unsigned* err, cudaStream_t s) {
  MhdBox<Pol> B = box_of<Pol>(h, nullptr);
  k_mhd_cfl<Pol><<<grid_for(B.cells), 256, 0, s>>>(B, consts_of<typename Pol::R>(prm), prm.cfl, h.dx, dt, err);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ patches with two ghost layers
// The same step on many patches in one set of launches.  Each patch's extended box is its interior
// and one ring cell beyond each face, (nx+2)(ny+2)(nz+2) cells: the face states are formed there
// (the ring cells' from the ghost layers), the low-face fluxes on the cells [0, n] of each axis,
// the update on the interior.  Block b of every launch takes extended cells blocks[b].y ..
// blocks[b].y + 255 of patch blocks[b].x; a patch's scratch starts at its own element offset.
struct ExtCell {
  int i, j, k;  // -1 .. n per axis
  bool ring;    // outside the interior
};

__device__ __forceinline__ bool ext_cell(const HostMhdPatch& P, int t, ExtCell& e) {
  const int ex = P.nx + 2, ey = P.ny + 2;
  if (t >= ex * ey * (P.nz + 2)) return false;
  const int row = t / ex, z = row / ey;
  e.i = t - row * ex - 1;
  e.j = row - z * ey - 1;
  e.k = z - 1;
  e.ring = e.i < 0 || e.j < 0 || e.k < 0 || e.i >= P.nx || e.j >= P.ny || e.k >= P.nz;
  return true;
}

__device__ __forceinline__ long long in_addr(const HostMhdPatch& P, int i, int j, int k) {
  return (long long)(k + 2) * P.isz + (long long)(j + 2) * P.isy + (i + 2);
}

template <class Pol>
__device__ __forceinline__ void load_qp(const HostMhdPatch& P, long long a, const MhdConst<typename Pol::R>& c,
                                        typename Pol::R q[NV], unsigned& flags) {
  using S = typename Pol::S;
  using R = typename Pol::R;
  R U[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) U[v] = to_r(__ldg(static_cast<const S*>(P.in[v]) + a), (R*)nullptr);
  mhd_recover(U, c, q, flags);
}

template <class R>
__global__ void k_mhdp_consts(const HostMhdPatch* patches, int npatch, MhdConst<R> base, double cfl, double alpha,
                              const double* dt_dev, MhdConst<R>* out, unsigned* err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npatch) return;
  const double dt = dt_dev[p], dx = patches[p].dx;
  MhdConst<R> c = base;
  c.valid = dt > 0.0 && dt <= 1e300;
  if (!c.valid) {
    atomicOr(err, HYDRO_EBIT_BAD_DT);
  } else {
    const double ch = (cfl / 3.0) * dx / dt;
    c.ch = R(ch);
    c.ch2 = R(ch * ch);
    c.ich = R(1.0 / ch);
    c.hdt = R(0.5 * dt / dx);
    c.dtdx = R(dt / dx);
    c.damp = R(exp(-alpha * ch * dt / dx));
  }
  out[p] = c;
}

template <int D, class Pol>
__device__ __forceinline__ void axis_states_p(const HostMhdPatch& P, typename Pol::R* face, long long ec, long long e,
                                              const ExtCell& x, const typename Pol::R q[NV],
                                              const MhdConst<typename Pol::R>& c, typename Pol::R dF[NV]) {
  using R = typename Pol::R;
  unsigned nf = 0;  // neighbours are flagged by their own threads
  const int di = D == 0, dj = D == 1, dk = D == 2;
  R lo[NV], hi[NV];
  {
    R qm[NV], qp[NV];
    load_qp<Pol>(P, in_addr(P, x.i - di, x.j - dj, x.k - dk), c, qm, nf);
    load_qp<Pol>(P, in_addr(P, x.i + di, x.j + dj, x.k + dk), c, qp, nf);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const R s = limited(q[v] - qm[v], qp[v] - q[v], c.limiter);
      lo[v] = q[v] - half_(s);
      hi[v] = q[v] + half_(s);
      face[((long long)(2 * D) * NV + v) * ec + e] = lo[v];
      face[((long long)(2 * D + 1) * NV + v) * ec + e] = hi[v];
    }
  }
  R Fh[NV];
  mhd_flux<D>(hi, c, Fh);
  {
    R Fl[NV];
    mhd_flux<D>(lo, c, Fl);
#pragma unroll
    for (int v = 0; v < NV; ++v) dF[v] = D == 0 ? Fh[v] - Fl[v] : dF[v] + (Fh[v] - Fl[v]);
  }
}

template <class Pol>
__global__ void __launch_bounds__(256, 2) k_mhdp_predict(const HostMhdPatch* patches, const int2* blocks,
                                                         const MhdConst<typename Pol::R>* consts, void* scratch,
                                                         unsigned* err) {
  using R = typename Pol::R;
  const int2 b = blocks[blockIdx.x];
  const HostMhdPatch P = patches[b.x];
  const MhdConst<R> c = consts[b.x];
  ExtCell x;
  if (!c.valid || !ext_cell(P, b.y + threadIdx.x, x)) return;
  const long long ec = (long long)(P.nx + 2) * (P.ny + 2) * (P.nz + 2), e = b.y + threadIdx.x;
  R* face = static_cast<R*>(scratch) + P.scratch;
  unsigned flags = 0;
  R q[NV], dF[NV];
  load_qp<Pol>(P, in_addr(P, x.i, x.j, x.k), c, q, flags);
  axis_states_p<0, Pol>(P, face, ec, e, x, q, c, dF);
  axis_states_p<1, Pol>(P, face, ec, e, x, q, c, dF);
  axis_states_p<2, Pol>(P, face, ec, e, x, q, c, dF);
  unsigned nf = 0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      const int f = 2 * d + h;
      R w[NV], U[NV], r[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) w[v] = face[((long long)f * NV + v) * ec + e];
      mhd_conserved(w, c, U);
#pragma unroll
      for (int v = 0; v < NV; ++v) U[v] = U[v] - c.hdt * dF[v];
      mhd_recover(U, c, r, nf);
#pragma unroll
      for (int v = 0; v < NV; ++v) face[((long long)f * NV + v) * ec + e] = r[v];
    }
  }
  if (!x.ring && flags) atomicOr(err, flags);  // the interior's own recovery; ghosts are flagged by their owners
}

template <int D, class Pol>
__device__ __forceinline__ void low_face_flux_p(const typename Pol::R* face, typename Pol::R* flux, long long ec,
                                                long long e, long long em, const MhdConst<typename Pol::R>& c) {
  using R = typename Pol::R;
  R qL[NV], qR[NV], F[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    qL[v] = face[((long long)(2 * D + 1) * NV + v) * ec + em];  // high face of the cell below
    qR[v] = face[((long long)(2 * D) * NV + v) * ec + e];       // low face of this cell
  }
  mhd_hll<D>(qL, qR, c, F);
#pragma unroll
  for (int v = 0; v < NV; ++v) flux[((long long)D * NV + v) * ec + e] = F[v];
}

template <class Pol>
__global__ void __launch_bounds__(256, 2) k_mhdp_flux(const HostMhdPatch* patches, const int2* blocks,
                                                      const MhdConst<typename Pol::R>* consts, void* scratch) {
  using R = typename Pol::R;
  const int2 b = blocks[blockIdx.x];
  const HostMhdPatch P = patches[b.x];
  const MhdConst<R> c = consts[b.x];
  ExtCell x;
  if (!c.valid || !ext_cell(P, b.y + threadIdx.x, x)) return;
  if (x.i < 0 || x.j < 0 || x.k < 0) return;  // low faces of the cells 0 .. n per axis
  const long long ex = P.nx + 2, ey = P.ny + 2, ec = ex * ey * (P.nz + 2), e = b.y + threadIdx.x;
  const R* face = static_cast<const R*>(scratch) + P.scratch;
  R* flux = static_cast<R*>(scratch) + P.scratch + 6LL * NV * ec;
  if (x.j < P.ny && x.k < P.nz) low_face_flux_p<0, Pol>(face, flux, ec, e, e - 1, c);
  if (x.i < P.nx && x.k < P.nz) low_face_flux_p<1, Pol>(face, flux, ec, e, e - ex, c);
  if (x.i < P.nx && x.j < P.ny) low_face_flux_p<2, Pol>(face, flux, ec, e, e - ex * ey, c);
}

template <class Pol>
__global__ void __launch_bounds__(256, 2) k_mhdp_update(const HostMhdPatch* patches, const int2* blocks,
                                                        const MhdConst<typename Pol::R>* consts, void* scratch,
                                                        double cfl, double* dt_next, unsigned* err) {
  using S = typename Pol::S;
  using R = typename Pol::R;
  const int2 b = blocks[blockIdx.x];
  const HostMhdPatch P = patches[b.x];
  const MhdConst<R> c = consts[b.x];
  if (!c.valid) return;  // (block-uniform)
  ExtCell x;
  const bool live = ext_cell(P, b.y + threadIdx.x, x) && !x.ring;
  unsigned flags = 0;
  R smax = R(0);
  if (live) {
    const long long ex = P.nx + 2, ey = P.ny + 2, ec = ex * ey * (P.nz + 2), e = b.y + threadIdx.x;
    const R* flux = static_cast<const R*>(scratch) + P.scratch + 6LL * NV * ec;
    const long long ai = in_addr(P, x.i, x.j, x.k);
    const long long ao = (long long)(x.k + P.gout) * P.osz + (long long)(x.j + P.gout) * P.osy + (x.i + P.gout);
    S Un[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const R* fx = flux + (long long)(0 * NV + v) * ec;
      const R* fy = flux + (long long)(1 * NV + v) * ec;
      const R* fz = flux + (long long)(2 * NV + v) * ec;
      const R div = ((fx[e + 1] - fx[e]) + (fy[e + ex] - fy[e])) + (fz[e + ex * ey] - fz[e]);
      Un[v] = Pol::update(__ldg(static_cast<const S*>(P.in[v]) + ai), c.dtdx, div);
    }
    Un[8] = Un[8] * (S)to_double(c.damp);
#pragma unroll
    for (int v = 0; v < NV; ++v) static_cast<S*>(P.out[v])[ao] = Un[v];
    if (dt_next) {
      R U[NV], q[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) U[v] = to_r(Un[v], (R*)nullptr);
      mhd_recover(U, c, q, flags);
      smax = mhd_speed(q, c);
    }
  }
  if (dt_next) {
    const R m = block_max_r(smax);
    if (threadIdx.x == 0) publish_dt(cfl, P.dx, to_double(m), dt_next + b.x);
  }
  flush_flags(flags, err);
}

template <class Pol>
__global__ void __launch_bounds__(256) k_mhdp_cfl(const HostMhdPatch* patches, const int2* blocks,
                                                  MhdConst<typename Pol::R> c, double cfl, double* dt, unsigned* err) {
  using R = typename Pol::R;
  const int2 b = blocks[blockIdx.x];
  const HostMhdPatch P = patches[b.x];
  ExtCell x;
  unsigned flags = 0;
  R smax = R(0);
  if (ext_cell(P, b.y + threadIdx.x, x) && !x.ring) {
    R q[NV];
    load_qp<Pol>(P, in_addr(P, x.i, x.j, x.k), c, q, flags);
    smax = mhd_speed(q, c);
  }
  const R m = block_max_r(smax);
  if (threadIdx.x == 0) publish_dt(cfl, P.dx, to_double(m), dt + b.x);
  flush_flags(flags, err);
}

template <class Pol>
cudaError_t mhd_patches_t(const HostMhdPatch* d_patches, const void* d_table, int ntable, int npatch,
                          const Params& prm, const double* dt, double* dt_next, void* scratch, unsigned* err,
                          cudaStream_t s) {
  using R = typename Pol::R;
  auto* consts = static_cast<MhdConst<R>*>(scratch);
  void* body = static_cast<char*>(scratch) + mhd_patch_consts_bytes(npatch);
  k_mhdp_consts<R><<<(npatch + 127) / 128, 128, 0, s>>>(d_patches, npatch, consts_of<R>(prm), prm.cfl, kMhdAlpha, dt,
                                                        consts, err);
  if constexpr (kMhdFused<Pol>) {
    constexpr int TX = kMhdTX, TY = kMhdTY;
    const size_t smem = sizeof(MhdTileSh<Pol, TX, TY, true>);
    static PerDeviceOnce attr;
    cudaError_t e = attr.call([&] {
      return cudaFuncSetAttribute(k_mhdp_tile<Pol, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (e != cudaSuccess) return e;
    k_mhdp_tile<Pol, TX, TY><<<ntable, TX * TY, smem, s>>>(d_patches, static_cast<const int4*>(d_table), consts,
                                                           prm.cfl, dt_next, kMhdPatchZChunk, err);
    return cudaGetLastError();
  } else {
    const int nblocks = ntable;
    const int2* d_blocks = static_cast<const int2*>(d_table);
    k_mhdp_predict<Pol><<<nblocks, 256, 0, s>>>(d_patches, d_blocks, consts, body, err);
    k_mhdp_flux<Pol><<<nblocks, 256, 0, s>>>(d_patches, d_blocks, consts, body);
    k_mhdp_update<Pol><<<nblocks, 256, 0, s>>>(d_patches, d_blocks, consts, body, prm.cfl, dt_next, err);
    return cudaGetLastError();
  }
}

template <class Pol>
cudaError_t mhd_patches_cfl_t(const HostMhdPatch* d_patches, const int2* d_blocks, int nblocks, const Params& prm,
                              double* dt, unsigned* err, cudaStream_t s) {
  k_mhdp_cfl<Pol><<<nblocks, 256, 0, s>>>(d_patches, d_blocks, consts_of<typename Pol::R>(prm), prm.cfl, dt, err);
  return cudaGetLastError();
}

}  // namespace

size_t mhd_patch_consts_bytes(int npatch) { return ((size_t)npatch * 128 + 255) / 256 * 256; }

cudaError_t launch_mhd_patches(int precision, const HostMhdPatch* d_patches, const void* d_blocks, int nblocks,
                               int npatch, const Params& prm, const double* dt, double* dt_next, void* scratch,
                               unsigned* err, cudaStream_t s) {
  static_assert(sizeof(MhdConst<double>) <= 128 && sizeof(MhdConst<df>) <= 128, "per-patch constants slot");
  switch (precision) {
    case HYDRO_FP64: return mhd_patches_t<PolF64>(d_patches, d_blocks, nblocks, npatch, prm, dt, dt_next, scratch, err, s);
    case HYDRO_FP32: return mhd_patches_t<PolF32>(d_patches, d_blocks, nblocks, npatch, prm, dt, dt_next, scratch, err, s);
    case HYDRO_FP64_DF: return mhd_patches_t<PolDF>(d_patches, d_blocks, nblocks, npatch, prm, dt, dt_next, scratch, err, s);
    case HYDRO_MIXED: return mhd_patches_t<PolMixed>(d_patches, d_blocks, nblocks, npatch, prm, dt, dt_next, scratch, err, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_mhd_patches_cfl(int precision, const HostMhdPatch* d_patches, const int2* d_blocks, int nblocks,
                                   const Params& prm, double* dt, unsigned* err, cudaStream_t s) {
  switch (precision) {
    case HYDRO_FP64: return mhd_patches_cfl_t<PolF64>(d_patches, d_blocks, nblocks, prm, dt, err, s);
    case HYDRO_FP32: return mhd_patches_cfl_t<PolF32>(d_patches, d_blocks, nblocks, prm, dt, err, s);
    case HYDRO_FP64_DF: return mhd_patches_cfl_t<PolDF>(d_patches, d_blocks, nblocks, prm, dt, err, s);
    case HYDRO_MIXED: return mhd_patches_cfl_t<PolMixed>(d_patches, d_blocks, nblocks, prm, dt, err, s);
  }
  return cudaErrorInvalidValue;
}

static bool mhd_fused(int precision) {
  switch (precision) {
    case HYDRO_FP64: return kMhdFused<PolF64>;
    case HYDRO_FP32: return kMhdFused<PolF32>;
    case HYDRO_FP64_DF: return kMhdFused<PolDF>;
    case HYDRO_MIXED: return kMhdFused<PolMixed>;
  }
  return false;
}

size_t mhd_scratch_bytes(int precision, int nx, int ny, int nz, int elem_size) {
  if (mhd_fused(precision)) return 256;  // the step's constants alone
  return (size_t)9 * NV * (size_t)nx * ny * nz * elem_size + 256;
}

int mhd_step_launches(int precision) { return mhd_fused(precision) ? 2 : 4; }

bool mhd_patch_tiles(int precision, int* tx, int* ty, int* zc) {
  if (!mhd_fused(precision)) return false;
  *tx = kMhdTX;
  *ty = kMhdTY;
  *zc = kMhdPatchZChunk;
  return true;
}

cudaError_t launch_mhd_step(int precision, const HostMhdBox& h, const Params& prm, const double* dt, double* dt_next,
                            void* scratch, unsigned* err, cudaStream_t s) {
  switch (precision) {
    case HYDRO_FP64: return mhd_step_t<PolF64>(h, prm, dt, dt_next, scratch, err, s);
    case HYDRO_FP32: return mhd_step_t<PolF32>(h, prm, dt, dt_next, scratch, err, s);
    case HYDRO_FP64_DF: return mhd_step_t<PolDF>(h, prm, dt, dt_next, scratch, err, s);
    case HYDRO_MIXED: return mhd_step_t<PolMixed>(h, prm, dt, dt_next, scratch, err, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_mhd_cfl(int precision, const HostMhdBox& h, const Params& prm, double* dt, unsigned* err,
                           cudaStream_t s) {
  switch (precision) {
    case HYDRO_FP64: return mhd_cfl_t<PolF64>(h, prm, dt, err, s);
    case HYDRO_FP32: return mhd_cfl_t<PolF32>(h, prm, dt, err, s);
    case HYDRO_FP64_DF: return mhd_cfl_t<PolDF>(h, prm, dt, err, s);
    case HYDRO_MIXED: return mhd_cfl_t<PolMixed>(h, prm, dt, err, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hydro
