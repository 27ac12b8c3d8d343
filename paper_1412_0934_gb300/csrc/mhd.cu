// Ideal MHD with hyperbolic (GLM) divergence cleaning on a periodic box: the paper's second code
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
// Three launches per step, one thread per cell each: predict (the cell's six face states into
// scratch), flux (the HLL flux through the cell's three low faces into scratch), update (flux
// divergence, damping, and the CFL speed of the new state folded into dt_next).  The scratch holds
// 6 x 9 face states and 3 x 9 fluxes per cell, structure of arrays.
#include <cuda_runtime.h>

#include <cmath>

#include "hydro_device.cuh"
#include "internal.h"
#include "step_tile.cuh"

namespace hydro {
namespace {

constexpr int NV = 9;
constexpr double kMhdAlpha = 0.4;  // psi damping: exp(-alpha c_h dt / dx) per step

template <class T>
struct MhdBox {
  const T* in[NV];
  T* out[NV];
  T* face;  // [6][NV][cells]: face 2d + h, h = 0 the low, 1 the high face along axis d
  T* flux;  // [3][NV][cells]: the flux through the cell's low face along each axis
  int nx, ny, nz;
  long long cells;
};

template <class T>
struct MhdConst {
  T gamma, gm1, igm1, rf, pf, ch, hdt, dtdx, damp;
  int limiter;
  int valid;  // 0: the step's dt was not positive and finite (nothing is updated)
};

// Limited slope of left and right differences (the hydro step's limiter, in T).
template <class T>
__device__ __forceinline__ T mhd_slope(T a, T b, int lim) {
  if (lim == HYDRO_NOLIMIT) return T(0.5) * (a + b);
  if (a * b <= T(0)) return T(0);
  if (lim == HYDRO_MINMOD) return fabs(a) <= fabs(b) ? a : b;
  T ta = T(2) * a, tb = T(2) * b, m = T(0.5) * (a + b);
  T best = ta;
  if (fabs(tb) < fabs(best)) best = tb;
  if (fabs(m) < fabs(best)) best = m;
  return best;
}

// Primitive state of a conserved one, rho and p floored; flags as the hydro recovery.
template <class T>
__device__ __forceinline__ void mhd_recover(const T U[NV], const MhdConst<T>& c, T q[NV], unsigned& flags) {
  if (!(U[0] >= c.rf)) flags |= isfinite(U[0]) ? HYDRO_EBIT_RHO_FLOOR : HYDRO_EBIT_NONFINITE;
  const T rho = U[0] < c.rf ? c.rf : U[0];
  const T ir = T(1) / rho;
  const T kin = T(0.5) * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) * ir;
  const T mag = T(0.5) * (U[5] * U[5] + U[6] * U[6] + U[7] * U[7]);
  const T eint = (U[4] - kin) - mag;
  if (eint < T(0)) flags |= HYDRO_EBIT_P_FLOOR;
  if (!isfinite(eint)) flags |= HYDRO_EBIT_NONFINITE;
  const T p = c.gm1 * eint;
  q[0] = rho;
  q[1] = U[1] * ir;
  q[2] = U[2] * ir;
  q[3] = U[3] * ir;
  q[4] = p < c.pf ? c.pf : p;
  q[5] = U[5];
  q[6] = U[6];
  q[7] = U[7];
  q[8] = U[8];
}

template <class T>
__device__ __forceinline__ void mhd_conserved(const T q[NV], const MhdConst<T>& c, T U[NV]) {
  const T rho = q[0];
  U[0] = rho;
  U[1] = rho * q[1];
  U[2] = rho * q[2];
  U[3] = rho * q[3];
  U[4] = q[4] * c.igm1 + T(0.5) * rho * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) +
         T(0.5) * (q[5] * q[5] + q[6] * q[6] + q[7] * q[7]);
  U[5] = q[5];
  U[6] = q[6];
  U[7] = q[7];
  U[8] = q[8];
}

// Physical flux along axis D with the GLM terms (B_n's flux psi, psi's flux c_h^2 B_n).
template <int D, class T>
__device__ __forceinline__ void mhd_flux(const T q[NV], const MhdConst<T>& c, T F[NV]) {
  constexpr int N = 1 + D;
  const T rho = q[0], p = q[4], un = q[N], Bn = q[5 + D];
  const T B2 = q[5] * q[5] + q[6] * q[6] + q[7] * q[7];
  const T pt = p + T(0.5) * B2;
  const T uB = q[1] * q[5] + q[2] * q[6] + q[3] * q[7];
  const T E = p * c.igm1 + T(0.5) * rho * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) + T(0.5) * B2;
  const T mn = rho * un;
  F[0] = mn;
#pragma unroll
  for (int k = 0; k < 3; ++k) F[1 + k] = mn * q[1 + k] - Bn * q[5 + k];
  F[N] += pt;
  F[4] = (E + pt) * un - Bn * uB;
#pragma unroll
  for (int k = 0; k < 3; ++k) F[5 + k] = un * q[5 + k] - q[1 + k] * Bn;
  F[5 + D] = q[8];
  F[8] = c.ch * c.ch * Bn;
}

template <class T>
__device__ __forceinline__ T mhd_fast(const T q[NV], int d, const MhdConst<T>& c) {
  const T ir = T(1) / q[0];
  const T a2 = c.gamma * q[4] * ir;
  const T b2 = (q[5] * q[5] + q[6] * q[6] + q[7] * q[7]) * ir;
  const T bn = q[5 + d];
  const T bn2 = bn * bn * ir;
  const T s = a2 + b2;
  T r = s * s - T(4) * a2 * bn2;
  r = r > T(0) ? r : T(0);
  return sqrt(T(0.5) * (s + sqrt(r)));
}

// CFL speed sum over axes of |u_d| + c_f,d (the same function for the fused and standalone dt).
template <class T>
__device__ __forceinline__ T mhd_speed(const T q[NV], const MhdConst<T>& c) {
  return ((fabs(q[1]) + mhd_fast(q, 0, c)) + (fabs(q[2]) + mhd_fast(q, 1, c))) + (fabs(q[3]) + mhd_fast(q, 2, c));
}

template <int D, class T>
__device__ __forceinline__ void mhd_hll(T qL[NV], T qR[NV], const MhdConst<T>& c, T F[NV]) {
  const T Bm = T(0.5) * (qL[5 + D] + qR[5 + D]) - (qR[8] - qL[8]) / (T(2) * c.ch);
  const T pm = T(0.5) * (qL[8] + qR[8]) - T(0.5) * c.ch * (qR[5 + D] - qL[5 + D]);
  qL[5 + D] = qR[5 + D] = Bm;
  qL[8] = qR[8] = pm;
  constexpr int N = 1 + D;
  const T cL = mhd_fast(qL, D, c), cR = mhd_fast(qR, D, c);
  const T a = qL[N] - cL, b = qR[N] - cR, e = qL[N] + cL, f = qR[N] + cR;
  const T SL = a < b ? a : b, SR = e > f ? e : f;
  if (SL >= T(0)) {
    mhd_flux<D>(qL, c, F);
  } else if (SR <= T(0)) {
    mhd_flux<D>(qR, c, F);
  } else {
    T FL[NV], FR[NV], UL[NV], UR[NV];
    mhd_flux<D>(qL, c, FL);
    mhd_flux<D>(qR, c, FR);
    mhd_conserved(qL, c, UL);
    mhd_conserved(qR, c, UR);
    const T is = T(1) / (SR - SL);
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = ((SR * FL[v] - SL * FR[v]) + SL * SR * (UR[v] - UL[v])) * is;
  }
  F[5 + D] = pm;
  F[8] = c.ch * c.ch * Bm;
}

__device__ __forceinline__ void cell_of(long long a, int nx, int ny, int& i, int& j, int& k) {
  const int t = (int)a;  // cells < 2^31
  const int row = t / nx;
  i = t - row * nx;
  k = row / ny;
  j = row - k * ny;
}

template <class T>
__device__ __forceinline__ void load_q(const MhdBox<T>& B, long long a, const MhdConst<T>& c, T q[NV],
                                       unsigned& flags) {
  T U[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) U[v] = __ldg(B.in[v] + a);
  mhd_recover(U, c, q, flags);
}

template <int D, class T>
__device__ __forceinline__ void axis_states(const MhdBox<T>& B, long long a, long long am, long long ap,
                                            const T q[NV], const MhdConst<T>& c, T dF[NV]) {
  unsigned nf = 0;  // neighbours are flagged by their own threads
  T qm[NV], qp[NV], lo[NV], hi[NV], Fl[NV], Fh[NV];
  load_q(B, am, c, qm, nf);
  load_q(B, ap, c, qp, nf);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const T s = mhd_slope(q[v] - qm[v], qp[v] - q[v], c.limiter);
    lo[v] = q[v] - T(0.5) * s;
    hi[v] = q[v] + T(0.5) * s;
  }
  mhd_flux<D>(hi, c, Fh);
  mhd_flux<D>(lo, c, Fl);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    dF[v] = D == 0 ? Fh[v] - Fl[v] : dF[v] + (Fh[v] - Fl[v]);
    B.face[((long long)(2 * D) * NV + v) * B.cells + a] = lo[v];
    B.face[((long long)(2 * D + 1) * NV + v) * B.cells + a] = hi[v];
  }
}

template <class T>
__global__ void __launch_bounds__(256) k_mhd_predict(MhdBox<T> B, const MhdConst<T>* cp, unsigned* err) {
  const MhdConst<T> c = *cp;
  if (!c.valid) return;
  unsigned flags = 0;
  for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < B.cells;
       a += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    cell_of(a, B.nx, B.ny, i, j, k);
    const long long sx = 1, sy = B.nx, sz = (long long)B.nx * B.ny;
    const long long axm = a + (i == 0 ? (B.nx - 1) * sx : -sx), axp = a + (i == B.nx - 1 ? -(B.nx - 1) * sx : sx);
    const long long aym = a + (j == 0 ? (B.ny - 1) * sy : -sy), ayp = a + (j == B.ny - 1 ? -(B.ny - 1) * sy : sy);
    const long long azm = a + (k == 0 ? (B.nz - 1) * sz : -sz), azp = a + (k == B.nz - 1 ? -(B.nz - 1) * sz : sz);
    T q[NV], dF[NV];
    load_q(B, a, c, q, flags);
    axis_states<0>(B, a, axm, axp, q, c, dF);
    axis_states<1>(B, a, aym, ayp, q, c, dF);
    axis_states<2>(B, a, azm, azp, q, c, dF);
    // the six extrapolated states advanced by half a step, recovered and floored (this thread's
    // own scratch entries, written just above)
    unsigned nf = 0;
#pragma unroll 1
    for (int f = 0; f < 6; ++f) {
      T w[NV], U[NV], r[NV];
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
  flush_flags(flags, err);
}

template <int D, class T>
__device__ __forceinline__ void low_face_flux(const MhdBox<T>& B, long long a, long long am, const MhdConst<T>& c) {
  T qL[NV], qR[NV], F[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    qL[v] = B.face[((long long)(2 * D + 1) * NV + v) * B.cells + am];  // high face of the cell below
    qR[v] = B.face[((long long)(2 * D) * NV + v) * B.cells + a];       // low face of this cell
  }
  mhd_hll<D>(qL, qR, c, F);
#pragma unroll
  for (int v = 0; v < NV; ++v) B.flux[((long long)D * NV + v) * B.cells + a] = F[v];
}

template <class T>
__global__ void __launch_bounds__(256) k_mhd_flux(MhdBox<T> B, const MhdConst<T>* cp) {
  const MhdConst<T> c = *cp;
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

template <class T>
__device__ __forceinline__ T block_max_t(T v) {
  __shared__ T red[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = red[w] > v ? red[w] : v;
  return v;
}

template <class T>
__global__ void __launch_bounds__(256) k_mhd_update(MhdBox<T> B, const MhdConst<T>* cp, double cfl, double dx,
                                                    double* dt_next, unsigned* err) {
  const MhdConst<T> c = *cp;
  if (!c.valid) return;
  unsigned flags = 0;
  T smax = T(0);
  for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < B.cells;
       a += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    cell_of(a, B.nx, B.ny, i, j, k);
    const long long sy = B.nx, sz = (long long)B.nx * B.ny;
    const long long bx = a + (i == B.nx - 1 ? -(B.nx - 1) : 1);
    const long long by = a + (j == B.ny - 1 ? -(B.ny - 1) * sy : sy);
    const long long bz = a + (k == B.nz - 1 ? -(B.nz - 1) * sz : sz);
    T Un[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const T* fx = B.flux + (long long)(0 * NV + v) * B.cells;
      const T* fy = B.flux + (long long)(1 * NV + v) * B.cells;
      const T* fz = B.flux + (long long)(2 * NV + v) * B.cells;
      const T div = ((fx[bx] - fx[a]) + (fy[by] - fy[a])) + (fz[bz] - fz[a]);
      Un[v] = __ldg(B.in[v] + a) - c.dtdx * div;
    }
    Un[8] = Un[8] * c.damp;
#pragma unroll
    for (int v = 0; v < NV; ++v) B.out[v][a] = Un[v];
    if (dt_next) {
      T q[NV];
      mhd_recover(Un, c, q, flags);
      const T s = mhd_speed(q, c);
      smax = s > smax ? s : smax;
    }
  }
  if (dt_next) {
    const T m = block_max_t(smax);
    if (threadIdx.x == 0) publish_dt(cfl, dx, (double)m, dt_next);
  }
  flush_flags(flags, err);
}

template <class T>
__global__ void __launch_bounds__(256) k_mhd_cfl(MhdBox<T> B, MhdConst<T> c, double cfl, double dx, double* dt,
                                                 unsigned* err) {
  unsigned flags = 0;
  T smax = T(0);
  for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < B.cells;
       a += (long long)gridDim.x * blockDim.x) {
    T q[NV];
    load_q(B, a, c, q, flags);
    const T s = mhd_speed(q, c);
    smax = s > smax ? s : smax;
  }
  const T m = block_max_t(smax);
  if (threadIdx.x == 0) publish_dt(cfl, dx, (double)m, dt);
  flush_flags(flags, err);
}

// c_h and the half-step factors need dt, which lives on the device: a one-thread kernel turns it
// into the constants the three step kernels read.
template <class T>
__global__ void k_mhd_consts(MhdConst<T> base, double cfl, double dx, double alpha, const double* dt_dev,
                             MhdConst<T>* out, unsigned* err) {
  const double dt = dt_dev[0];
  MhdConst<T> c = base;
  c.valid = dt > 0.0 && dt <= 1e300;
  if (!c.valid) {
    atomicOr(err, HYDRO_EBIT_BAD_DT);
  } else {
    const double ch = (cfl / 3.0) * dx / dt;
    c.ch = (T)ch;
    c.hdt = (T)(0.5 * dt / dx);
    c.dtdx = (T)(dt / dx);
    c.damp = (T)exp(-alpha * ch * dt / dx);
  }
  *out = c;
}

template <class T>
MhdBox<T> box_of(const HostMhdBox& h, void* scratch) {
  MhdBox<T> b;
  for (int v = 0; v < NV; ++v) {
    b.in[v] = static_cast<const T*>(h.in[v]);
    b.out[v] = static_cast<T*>(h.out[v]);
  }
  b.nx = h.nx;
  b.ny = h.ny;
  b.nz = h.nz;
  b.cells = (long long)h.nx * h.ny * h.nz;
  // scratch: the step's constants in the first 256 bytes, then the face states and the fluxes
  b.face = scratch ? reinterpret_cast<T*>(static_cast<char*>(scratch) + 256) : nullptr;
  b.flux = b.face ? b.face + 6LL * NV * b.cells : nullptr;
  return b;
}

template <class T>
MhdConst<T> consts_of(const Params& prm) {
  MhdConst<T> c{};
  c.gamma = (T)prm.gamma;
  c.gm1 = (T)(prm.gamma - 1.0);
  c.igm1 = (T)(1.0 / (prm.gamma - 1.0));
  c.rf = (T)prm.rho_floor;
  c.pf = (T)prm.p_floor;
  c.limiter = prm.limiter;
  c.valid = 1;
  return c;
}

int grid_for(long long cells) {
  const long long b = (cells + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 152LL * 64 ? 152LL * 64 : b));
}

template <class T>
cudaError_t mhd_step_t(const HostMhdBox& h, const Params& prm, const double* dt, double* dt_next, void* scratch,
                       unsigned* err, cudaStream_t s) {
  MhdBox<T> B = box_of<T>(h, scratch);
  static_assert(sizeof(MhdConst<T>) <= 256, "the constants fit before the face states");
  auto* cp = static_cast<MhdConst<T>*>(scratch);
  k_mhd_consts<T><<<1, 1, 0, s>>>(consts_of<T>(prm), prm.cfl, h.dx, kMhdAlpha, dt, cp, err);
  const int g = grid_for(B.cells);
  k_mhd_predict<T><<<g, 256, 0, s>>>(B, cp, err);
  k_mhd_flux<T><<<g, 256, 0, s>>>(B, cp);
  k_mhd_update<T><<<g, 256, 0, s>>>(B, cp, prm.cfl, h.dx, dt_next, err);
  return cudaGetLastError();
}

template <class T>
cudaError_t mhd_cfl_t(const HostMhdBox& h, const Params& prm, double* dt, unsigned* err, cudaStream_t s) {
  MhdBox<T> B = box_of<T>(h, nullptr);
  k_mhd_cfl<T><<<grid_for(B.cells), 256, 0, s>>>(B, consts_of<T>(prm), prm.cfl, h.dx, dt, err);
  return cudaGetLastError();
}

}  // namespace

size_t mhd_scratch_bytes(int nx, int ny, int nz, int elem_size) {
  return (size_t)9 * NV * (size_t)nx * ny * nz * elem_size + 256;
}

cudaError_t launch_mhd_step(int elem_size, const HostMhdBox& h, const Params& prm, const double* dt, double* dt_next,
                            void* scratch, unsigned* err, cudaStream_t s) {
  return elem_size == 4 ? mhd_step_t<float>(h, prm, dt, dt_next, scratch, err, s)
                        : mhd_step_t<double>(h, prm, dt, dt_next, scratch, err, s);
}

cudaError_t launch_mhd_cfl(int elem_size, const HostMhdBox& h, const Params& prm, double* dt, unsigned* err,
                           cudaStream_t s) {
  return elem_size == 4 ? mhd_cfl_t<float>(h, prm, dt, err, s) : mhd_cfl_t<double>(h, prm, dt, err, s);
}

}  // namespace hydro
