// Test infrastructure: the plain, slow FP64 CPU oracle of one MUSCL-Hancock/HLLC step of the
// 3D ideal-gas Euler equations on a patch with 2 ghost layers.
//
// What it computes: the Euler equations of an ideal fluid on the mesh (paper Sec. 2, where the
// baryonic component is an ideal fluid and the Euler equations are solved with PLM among other
// methods, the PLM reference being Colella & Glaz 1985); the fluxes that update a patch's cells
// (Sec. 4, Enzo: the GPU computes every flux that updates a patch's cells); and the
// adaptive time step (Sec. 2 and Sec. 4).  The paper prints no equations, so each step below is
// the textbook method (Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics":
// MUSCL-Hancock in primitive variables, HLLC of Toro, Spruce & Speares with the star states of
// Batten et al. 1997, Davis wave-speed bounds), with these readings where the paper is silent:
//   * reconstruction in primitive variables q = (rho, u, v, w, p), component by component;
//   * limiter minmod(a,b) = 0 if a*b <= 0 else the argument of smaller magnitude (tie -> a);
//     MC: 0 if a*b <= 0 else the smallest-magnitude of 2a, 2b, (a+b)/2 (ties -> earlier);
//     "none": the centred difference (a+b)/2;
//   * unsplit Hancock predictor q_h = q - dt/(2 dx) * sum_{d=x,y,z} A_d(q) dq_d, summed x, y, z;
//   * face states q_h +- dq_d / 2, floored: rho >= rho_floor, p >= p_floor; the same floors after
//     recovery (rho floored before dividing, p floored after);
//   * HLLC flux chosen by 0 <= S_L -> F_L, else 0 <= S* -> F*_L, else 0 < S_R -> F*_R, else F_R;
//   * update U' = U - dt/dx * ((Fx+ - Fx-) + (Fy+ - Fy-) + (Fz+ - Fz-));
//   * CFL dt = C * dx / max_cells(|u| + |v| + |w| + 3c), c = sqrt(gamma p / rho).
// The stages run one after another over the whole box with full-size temporaries: recovery,
// slopes, predictor, face states, fluxes, update.  Nothing is fused or reordered.
//
// The code is generic over the scalar type T (double, Dual, TVar, Counted; see scalars.hpp).
// It shares no code with the CUDA library.  Only tests/, the smoke check and the timed CPU
// baseline use anything under oracle/.
#pragma once
#include <cmath>
#include <cstdint>
#include <vector>
#include <type_traits>

#include "scalars.hpp"

namespace oracle {

struct Config {
  double gamma;
  double cfl;
  double rho_floor;
  double p_floor;
  int limiter;  // 0 = MinMod, 1 = MC, 2 = none (centred)
};

constexpr int G = 2;  // ghost layers

// Five fields over a box of nx*ny*nz cells, x fastest.
template <class T>
struct Fields {
  int nx = 0, ny = 0, nz = 0;
  std::vector<T> f[5];
  Fields() {}
  Fields(int x, int y, int z) { resize(x, y, z); }
  void resize(int x, int y, int z) {
    nx = x; ny = y; nz = z;
    for (int v = 0; v < 5; ++v) f[v].assign((size_t)x * y * z, T(0.0));
  }
  size_t at(int i, int j, int k) const { return ((size_t)k * ny + j) * nx + i; }
};

// max(x, floor) taken on the value; the floor is a constant.
template <class T>
inline T floor_at(const T& x, double fl) {
  return (value(x) < fl) ? T(fl) : x;
}
template <class T>
inline T tabs(const T& x) {
  return (value(x) < 0.0) ? -x : x;
}

// ------------------------------------------------------------------ a2: primitive recovery
template <class T>
inline void recover(const Config& c, const T U[5], T q[5]) {
  T rho = floor_at(U[0], c.rho_floor);
  T kin = T(0.5) * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / rho;
  T p = T(c.gamma - 1.0) * (U[4] - kin);
  q[0] = rho;
  q[1] = U[1] / rho;
  q[2] = U[2] / rho;
  q[3] = U[3] / rho;
  q[4] = floor_at(p, c.p_floor);
}

// ------------------------------------------------------------------ a3: limited slope
template <class T>
inline T limited_slope(const T& a, const T& b, int limiter) {
  if (limiter == 2) return T(0.5) * (a + b);
  if (value(a) * value(b) <= 0.0) return T(0.0);
  if (limiter == 0) {
    return (std::fabs(value(a)) <= std::fabs(value(b))) ? a : b;
  }
  T two_a = T(2.0) * a;
  T two_b = T(2.0) * b;
  T mid = T(0.5) * (a + b);
  T best = two_a;
  if (std::fabs(value(two_b)) < std::fabs(value(best))) best = two_b;
  if (std::fabs(value(mid)) < std::fabs(value(best))) best = mid;
  return best;
}

// ------------------------------------------------------------------ a4: Hancock term A_d(q) dq
// Primitive-variable Jacobian of direction d (normal velocity component n = 1 + d) applied to dq.
template <class T>
inline void hancock_term(const Config& c, const T q[5], const T dq[5], int d, T out[5]) {
  const int n = 1 + d;
  const T& un = q[n];
  out[0] = un * dq[0] + q[0] * dq[n];
  out[1] = un * dq[1];
  out[2] = un * dq[2];
  out[3] = un * dq[3];
  out[n] = out[n] + dq[4] / q[0];
  out[4] = T(c.gamma) * q[4] * dq[n] + un * dq[4];
}

// ------------------------------------------------------------------ a6: HLLC flux
// Physical flux and conserved state of primitive state q through a face of normal d.
template <class T>
inline void physical_flux(const Config& c, const T q[5], int d, T F[5], T U[5]) {
  const int n = 1 + d;
  T E = q[4] / T(c.gamma - 1.0) + T(0.5) * q[0] * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  T mn = q[0] * q[n];
  U[0] = q[0];
  U[1] = q[0] * q[1];
  U[2] = q[0] * q[2];
  U[3] = q[0] * q[3];
  U[4] = E;
  F[0] = mn;
  F[1] = mn * q[1];
  F[2] = mn * q[2];
  F[3] = mn * q[3];
  F[n] = F[n] + q[4];
  F[4] = q[n] * (E + q[4]);
}

template <class T>
inline void hllc_flux(const Config& c, const T qL[5], const T qR[5], int d, T F[5]) {
  const int n = 1 + d;
  T cL = sqrt(T(c.gamma) * qL[4] / qL[0]);
  T cR = sqrt(T(c.gamma) * qR[4] / qR[0]);
  // Davis estimates of the extreme wave speeds.
  T aL = qL[n] - cL, bL = qR[n] - cR;
  T SL = (value(aL) <= value(bL)) ? aL : bL;
  T aR = qL[n] + cL, bR = qR[n] + cR;
  T SR = (value(aR) >= value(bR)) ? aR : bR;
  T FL[5], UL[5], FR[5], UR[5];
  physical_flux(c, qL, d, FL, UL);
  physical_flux(c, qR, d, FR, UR);
  if (0.0 <= value(SL)) {
    for (int v = 0; v < 5; ++v) F[v] = FL[v];
    return;
  }
  if (value(SR) <= 0.0) {
    for (int v = 0; v < 5; ++v) F[v] = FR[v];
    return;
  }
  // Contact speed S*.
  T mL = qL[0] * (SL - qL[n]);
  T mR = qR[0] * (SR - qR[n]);
  T Sstar = (qR[4] - qL[4] + qL[n] * mL - qR[n] * mR) / (mL - mR);
  // Star state of side K: rho_K (S_K - u_K)/(S_K - S*) * [1, S*, u_t, u_t', E_K/rho_K
  //   + (S* - u_K)(S* + p_K/(rho_K (S_K - u_K)))], then F*_K = F_K + S_K (U*_K - U_K).
  const bool left = (0.0 <= value(Sstar));
  const T* q = left ? qL : qR;
  const T* FK = left ? FL : FR;
  const T* UK = left ? UL : UR;
  T SK = left ? SL : SR;
  T mK = left ? mL : mR;
  T fac = mK / (SK - Sstar);
  T Us[5];
  Us[0] = fac;
  Us[1] = fac * q[1];
  Us[2] = fac * q[2];
  Us[3] = fac * q[3];
  Us[n] = fac * Sstar;
  Us[4] = fac * (UK[4] / q[0] + (Sstar - q[n]) * (Sstar + q[4] / mK));
  for (int v = 0; v < 5; ++v) F[v] = FK[v] + SK * (Us[v] - UK[v]);
}

// ------------------------------------------------------------------ one step on a ghosted patch
// The box Ug is (nx+2G) x (ny+2G) x (nz+2G) cells with ghosts filled by the caller.  Each stage
// below runs over the whole box (or the part of it the next stage reads) into a full-size
// temporary; step_patch runs them in order.

// a2: recovery over the whole ghosted box.  Returns the number of cells processed.
template <class T>
size_t stage_recover(const Config& c, const Fields<T>& Ug, Fields<T>& q) {
  const int NX = Ug.nx, NY = Ug.ny, NZ = Ug.nz;
  const bool par = std::is_same<T, double>::value;
  q.resize(NX, NY, NZ);
#pragma omp parallel for if (par)
  for (int k = 0; k < NZ; ++k)
    for (int j = 0; j < NY; ++j)
      for (int i = 0; i < NX; ++i) {
        size_t a = Ug.at(i, j, k);
        T U[5], w[5];
        for (int v = 0; v < 5; ++v) U[v] = Ug.f[v][a];
        recover(c, U, w);
        for (int v = 0; v < 5; ++v) q.f[v][a] = w[v];
      }
  return (size_t)NX * NY * NZ;
}

// a3: limited slopes of every cell one layer inside the box, each direction.
template <class T>
size_t stage_slopes(const Config& c, const Fields<T>& q, Fields<T> slope[3]) {
  const int NX = q.nx, NY = q.ny, NZ = q.nz;
  const bool par = std::is_same<T, double>::value;
  for (int d = 0; d < 3; ++d) slope[d].resize(NX, NY, NZ);
#pragma omp parallel for if (par)
  for (int k = 1; k < NZ - 1; ++k)
    for (int j = 1; j < NY - 1; ++j)
      for (int i = 1; i < NX - 1; ++i) {
        size_t a = q.at(i, j, k);
        size_t lo[3] = {q.at(i - 1, j, k), q.at(i, j - 1, k), q.at(i, j, k - 1)};
        size_t hi[3] = {q.at(i + 1, j, k), q.at(i, j + 1, k), q.at(i, j, k + 1)};
        for (int d = 0; d < 3; ++d)
          for (int v = 0; v < 5; ++v) {
            T dl = q.f[v][a] - q.f[v][lo[d]];
            T dr = q.f[v][hi[d]] - q.f[v][a];
            slope[d].f[v][a] = limited_slope(dl, dr, c.limiter);
          }
      }
  return (size_t)(NX - 2) * (NY - 2) * (NZ - 2);
}

// a4: Hancock half-step predictor on the same cells as the slopes.
template <class T>
size_t stage_predict(const Config& c, const Fields<T>& q, const Fields<T> slope[3], Fields<T>& qh,
                     double dx, double dt) {
  const int NX = q.nx, NY = q.ny, NZ = q.nz;
  const bool par = std::is_same<T, double>::value;
  const double hdt = 0.5 * dt / dx;
  qh.resize(NX, NY, NZ);
#pragma omp parallel for if (par)
  for (int k = 1; k < NZ - 1; ++k)
    for (int j = 1; j < NY - 1; ++j)
      for (int i = 1; i < NX - 1; ++i) {
        size_t a = q.at(i, j, k);
        T w[5], dq[3][5], t[3][5];
        for (int v = 0; v < 5; ++v) w[v] = q.f[v][a];
        for (int d = 0; d < 3; ++d) {
          for (int v = 0; v < 5; ++v) dq[d][v] = slope[d].f[v][a];
          hancock_term(c, w, dq[d], d, t[d]);
        }
        for (int v = 0; v < 5; ++v) qh.f[v][a] = w[v] - T(hdt) * ((t[0][v] + t[1][v]) + t[2][v]);
      }
  return (size_t)(NX - 2) * (NY - 2) * (NZ - 2);
}

// a5 + a6: floored face states and the HLLC flux through every face of the interior cells.
// flux[d] at cell (i,j,k) is the flux through the face between that cell and its +d neighbour.
template <class T>
size_t stage_fluxes(const Config& c, const Fields<T>& qh, const Fields<T> slope[3], Fields<T> flux[3]) {
  const int NX = qh.nx, NY = qh.ny, NZ = qh.nz;
  const int nx = NX - 2 * G, ny = NY - 2 * G, nz = NZ - 2 * G;
  const bool par = std::is_same<T, double>::value;
  size_t faces = 0;
  for (int d = 0; d < 3; ++d) {
    flux[d].resize(NX, NY, NZ);
    const int i0 = G - (d == 0), j0 = G - (d == 1), k0 = G - (d == 2);
    faces += (size_t)(G + nx - i0) * (G + ny - j0) * (G + nz - k0);
#pragma omp parallel for if (par)
    for (int k = k0; k < G + nz; ++k)
      for (int j = j0; j < G + ny; ++j)
        for (int i = i0; i < G + nx; ++i) {
          size_t a = qh.at(i, j, k);
          size_t b = qh.at(i + (d == 0), j + (d == 1), k + (d == 2));
          T qL[5], qR[5], F[5];
          for (int v = 0; v < 5; ++v) {
            qL[v] = qh.f[v][a] + T(0.5) * slope[d].f[v][a];
            qR[v] = qh.f[v][b] - T(0.5) * slope[d].f[v][b];
          }
          qL[0] = floor_at(qL[0], c.rho_floor);
          qL[4] = floor_at(qL[4], c.p_floor);
          qR[0] = floor_at(qR[0], c.rho_floor);
          qR[4] = floor_at(qR[4], c.p_floor);
          hllc_flux(c, qL, qR, d, F);
          for (int v = 0; v < 5; ++v) flux[d].f[v][a] = F[v];
        }
  }
  return faces;
}

// a7: conservative update of the interior cells.
template <class T>
size_t stage_update(const Fields<T>& Ug, const Fields<T> flux[3], Fields<T>& Unew, double dx, double dt) {
  const int nx = Ug.nx - 2 * G, ny = Ug.ny - 2 * G, nz = Ug.nz - 2 * G;
  const bool par = std::is_same<T, double>::value;
  const double dtdx = dt / dx;
  Unew.resize(nx, ny, nz);
#pragma omp parallel for if (par)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t a = Ug.at(i + G, j + G, k + G);
        size_t mx = Ug.at(i + G - 1, j + G, k + G);
        size_t my = Ug.at(i + G, j + G - 1, k + G);
        size_t mz = Ug.at(i + G, j + G, k + G - 1);
        size_t o = Unew.at(i, j, k);
        for (int v = 0; v < 5; ++v) {
          T div = ((flux[0].f[v][a] - flux[0].f[v][mx]) + (flux[1].f[v][a] - flux[1].f[v][my])) +
                  (flux[2].f[v][a] - flux[2].f[v][mz]);
          Unew.f[v][o] = Ug.f[v][a] - T(dtdx) * div;
        }
      }
  return (size_t)nx * ny * nz;
}

// Returns U^{n+1} on the nx*ny*nz interior cells.
template <class T>
void step_patch(const Config& c, const Fields<T>& Ug, Fields<T>& Unew, double dx, double dt) {
  Fields<T> q, qh, slope[3], flux[3];
  stage_recover(c, Ug, q);
  stage_slopes(c, q, slope);
  stage_predict(c, q, slope, qh, dx, dt);
  stage_fluxes(c, qh, slope, flux);
  stage_update(Ug, flux, Unew, dx, dt);
}

// ------------------------------------------------------------------ periodic ghosts
template <class T>
void fill_periodic(const Fields<T>& U, Fields<T>& Ug) {
  const int nx = U.nx, ny = U.ny, nz = U.nz;
  Ug.resize(nx + 2 * G, ny + 2 * G, nz + 2 * G);
  for (int k = 0; k < nz + 2 * G; ++k)
    for (int j = 0; j < ny + 2 * G; ++j)
      for (int i = 0; i < nx + 2 * G; ++i) {
        int si = ((i - G) % nx + nx) % nx;
        int sj = ((j - G) % ny + ny) % ny;
        int sk = ((k - G) % nz + nz) % nz;
        for (int v = 0; v < 5; ++v) Ug.f[v][Ug.at(i, j, k)] = U.f[v][U.at(si, sj, sk)];
      }
}

template <class T>
void step_periodic(const Config& c, const Fields<T>& U, Fields<T>& Unew, double dx, double dt) {
  Fields<T> Ug;
  fill_periodic(U, Ug);
  step_patch(c, Ug, Unew, dx, dt);
}

// ------------------------------------------------------------------ a8: CFL time step
// Over the cells [i0,i0+nx) x [j0,j0+ny) x [k0,k0+nz) of U.
inline double cfl_dt(const Config& c, const Fields<double>& U, int i0, int j0, int k0, int nx, int ny,
                     int nz, double dx) {
  double smax = 0.0;
  for (int k = k0; k < k0 + nz; ++k)
    for (int j = j0; j < j0 + ny; ++j)
      for (int i = i0; i < i0 + nx; ++i) {
        size_t a = U.at(i, j, k);
        double Uc[5], q[5];
        for (int v = 0; v < 5; ++v) Uc[v] = U.f[v][a];
        recover(c, Uc, q);
        double cs = std::sqrt(c.gamma * q[4] / q[0]);
        double s = ((std::fabs(q[1]) + std::fabs(q[2])) + std::fabs(q[3])) + 3.0 * cs;
        if (s > smax) smax = s;
      }
  return c.cfl * (dx / smax);
}

// ------------------------------------------------------------------ initial map q -> U
template <class T>
inline void prim_to_cons(const Config& c, const T q[5], T U[5]) {
  U[0] = q[0];
  U[1] = q[0] * q[1];
  U[2] = q[0] * q[2];
  U[3] = q[0] * q[3];
  U[4] = q[4] / T(c.gamma - 1.0) + T(0.5) * q[0] * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
}

}  // namespace oracle
