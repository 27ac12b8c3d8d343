// Test infrastructure: C entry points of the FP64 CPU oracle, called through ctypes by the
// tests, the smoke check and the timed CPU baseline.  Nothing in the CUDA library links this.
//
// Array layout of every U argument: five fields (rho, m_x, m_y, m_z, E) one after another,
// each nz*ny*nx doubles with x fastest; "ghosted" arrays have (nz+4)*(ny+4)*(nx+4) cells per
// field.  Entry points return 0 on success and -1 on a bad argument.
#include <algorithm>
#include <cstring>
#include <vector>

#include <omp.h>

#include "euler_oracle.hpp"

using namespace oracle;

extern "C" {

typedef struct {
  double gamma, cfl, rho_floor, p_floor;
  int limiter;
} oracle_config;

}  // extern "C"

namespace {

Config to_cfg(const oracle_config* c) { return Config{c->gamma, c->cfl, c->rho_floor, c->p_floor, c->limiter}; }

template <class T>
void load(Fields<T>& F, const double* src, int nx, int ny, int nz) {
  F.resize(nx, ny, nz);
  const size_t n = (size_t)nx * ny * nz;
  for (int v = 0; v < 5; ++v)
    for (size_t a = 0; a < n; ++a) F.f[v][a] = T(src[(size_t)v * n + a]);
}
template <class T>
void store(const Fields<T>& F, double* dst) {
  const size_t n = (size_t)F.nx * F.ny * F.nz;
  for (int v = 0; v < 5; ++v)
    for (size_t a = 0; a < n; ++a) dst[(size_t)v * n + a] = value(F.f[v][a]);
}
bool bad_dims(int nx, int ny, int nz) { return nx <= 0 || ny <= 0 || nz <= 0; }

// J^T lam for a ghosted patch, through one tape: lam_out on the interior, result on the ghosted box.
void patch_adjoint(const Config& c, const Fields<double>& Ug, const Fields<double>& lam_out,
                   Fields<double>& lam_in, double dx, double dt) {
  Tape tape;
  active_tape() = &tape;
  const size_t n = (size_t)Ug.nx * Ug.ny * Ug.nz;
  Fields<TVar> X(Ug.nx, Ug.ny, Ug.nz), Y;
  for (int v = 0; v < 5; ++v)
    for (size_t a = 0; a < n; ++a) X.f[v][a] = TVar(Ug.f[v][a], tape.leaf());
  step_patch(c, X, Y, dx, dt);
  std::vector<double> adj(tape.nodes.size(), 0.0);
  const size_t m = (size_t)Y.nx * Y.ny * Y.nz;
  for (int v = 0; v < 5; ++v)
    for (size_t a = 0; a < m; ++a)
      if (Y.f[v][a].i >= 0) adj[(size_t)Y.f[v][a].i] += lam_out.f[v][a];
  tape.reverse(adj);
  lam_in.resize(Ug.nx, Ug.ny, Ug.nz);
  for (int v = 0; v < 5; ++v)
    for (size_t a = 0; a < n; ++a) lam_in.f[v][a] = adj[(size_t)X.f[v][a].i];
  active_tape() = nullptr;
}

}  // namespace

extern "C" {

// One step on a periodic box: U, out are [5][nz][ny][nx].
int oracle_step_periodic(const oracle_config* cfg, const double* U, double* out, int nx, int ny, int nz,
                         double dx, double dt) {
  if (!cfg || !U || !out || bad_dims(nx, ny, nz)) return -1;
  Fields<double> A, B;
  load(A, U, nx, ny, nz);
  step_periodic(to_cfg(cfg), A, B, dx, dt);
  store(B, out);
  return 0;
}

// One step on a ghosted patch: Ug is [5][nz+4][ny+4][nx+4], out is [5][nz][ny][nx].
int oracle_step_patch(const oracle_config* cfg, const double* Ug, double* out, int nx, int ny, int nz,
                      double dx, double dt) {
  if (!cfg || !Ug || !out || bad_dims(nx, ny, nz)) return -1;
  Fields<double> A, B;
  load(A, Ug, nx + 2 * G, ny + 2 * G, nz + 2 * G);
  step_patch(to_cfg(cfg), A, B, dx, dt);
  store(B, out);
  return 0;
}

// The fluxes through the six boundary faces of a ghosted patch's interior, the ones step_patch
// applies there (for the flux registers of AMR refluxing).  out per field v, in this order:
// x-low [nz][ny], x-high [nz][ny], y-low [nz][nx], y-high [nz][nx], z-low [ny][nx], z-high [ny][nx]
// (faces i = 0 and i = nx of the interior, and so on).
int oracle_patch_boundary_fluxes(const oracle_config* cfg, const double* Ug, int nx, int ny, int nz, double dx,
                                 double dt, double* out) {
  if (!cfg || !Ug || !out || bad_dims(nx, ny, nz)) return -1;
  const Config c = to_cfg(cfg);
  Fields<double> A, q, qh, slope[3], flux[3];
  load(A, Ug, nx + 2 * G, ny + 2 * G, nz + 2 * G);
  stage_recover(c, A, q);
  stage_slopes(c, q, slope);
  stage_predict(c, q, slope, qh, dx, dt);
  stage_fluxes(c, qh, slope, flux);
  const size_t R = 2 * ((size_t)ny * nz + (size_t)nx * nz + (size_t)nx * ny);
  for (int v = 0; v < 5; ++v) {
    double* o = out + v * R;
    for (int side = 0; side < 2; ++side) {
      const int i = side ? G + nx - 1 : G - 1;
      for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j) *o++ = flux[0].f[v][A.at(i, G + j, G + k)];
    }
    for (int side = 0; side < 2; ++side) {
      const int j = side ? G + ny - 1 : G - 1;
      for (int k = 0; k < nz; ++k)
        for (int i = 0; i < nx; ++i) *o++ = flux[1].f[v][A.at(G + i, j, G + k)];
    }
    for (int side = 0; side < 2; ++side) {
      const int k = side ? G + nz - 1 : G - 1;
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) *o++ = flux[2].f[v][A.at(G + i, G + j, k)];
    }
  }
  return 0;
}

// CFL dt of a periodic box ([5][nz][ny][nx]) or of the interior of a ghosted patch.
double oracle_cfl_periodic(const oracle_config* cfg, const double* U, int nx, int ny, int nz, double dx) {
  if (!cfg || !U || bad_dims(nx, ny, nz)) return -1.0;
  Fields<double> A;
  load(A, U, nx, ny, nz);
  return cfl_dt(to_cfg(cfg), A, 0, 0, 0, nx, ny, nz, dx);
}
double oracle_cfl_patch(const oracle_config* cfg, const double* Ug, int nx, int ny, int nz, double dx) {
  if (!cfg || !Ug || bad_dims(nx, ny, nz)) return -1.0;
  Fields<double> A;
  load(A, Ug, nx + 2 * G, ny + 2 * G, nz + 2 * G);
  return cfl_dt(to_cfg(cfg), A, G, G, G, nx, ny, nz, dx);
}

// Tangent (J v) of one periodic step by dual numbers: dU is v, dout receives J v.
int oracle_step_periodic_tangent(const oracle_config* cfg, const double* U, const double* dU, double* out,
                                 double* dout, int nx, int ny, int nz, double dx, double dt) {
  if (!cfg || !U || !dU || !out || !dout || bad_dims(nx, ny, nz)) return -1;
  const size_t n = (size_t)nx * ny * nz;
  Fields<Dual> A(nx, ny, nz), B;
  for (int v = 0; v < 5; ++v)
    for (size_t a = 0; a < n; ++a) A.f[v][a] = Dual(U[(size_t)v * n + a], dU[(size_t)v * n + a]);
  step_periodic(to_cfg(cfg), A, B, dx, dt);
  for (int v = 0; v < 5; ++v)
    for (size_t a = 0; a < n; ++a) {
      out[(size_t)v * n + a] = B.f[v][a].v;
      dout[(size_t)v * n + a] = B.f[v][a].d;
    }
  return 0;
}

// Adjoint (J^T w) of one periodic step by reverse-mode tape.  The output cells are split into
// blocks of at most `block` cells per axis; for each block the step of the block's ghosted
// sub-box is taped and reversed, and the input adjoints are summed back with periodic wrap.
// Because every output cell lies in exactly one block, the sum is J^T w.
int oracle_step_periodic_adjoint(const oracle_config* cfg, const double* U, const double* lam_out,
                                 double* lam_in, int nx, int ny, int nz, double dx, double dt, int block) {
  if (!cfg || !U || !lam_out || !lam_in || bad_dims(nx, ny, nz) || block <= 0) return -1;
  const Config c = to_cfg(cfg);
  Fields<double> A, L, R(nx, ny, nz);
  load(A, U, nx, ny, nz);
  load(L, lam_out, nx, ny, nz);
  for (int k0 = 0; k0 < nz; k0 += block)
    for (int j0 = 0; j0 < ny; j0 += block)
      for (int i0 = 0; i0 < nx; i0 += block) {
        const int bx = std::min(block, nx - i0), by = std::min(block, ny - j0), bz = std::min(block, nz - k0);
        Fields<double> Ug(bx + 2 * G, by + 2 * G, bz + 2 * G), Lb(bx, by, bz), Lg;
        auto wrap = [](int i, int n) { return ((i % n) + n) % n; };
        for (int k = 0; k < bz + 2 * G; ++k)
          for (int j = 0; j < by + 2 * G; ++j)
            for (int i = 0; i < bx + 2 * G; ++i) {
              size_t s = A.at(wrap(i0 + i - G, nx), wrap(j0 + j - G, ny), wrap(k0 + k - G, nz));
              for (int v = 0; v < 5; ++v) Ug.f[v][Ug.at(i, j, k)] = A.f[v][s];
            }
        for (int k = 0; k < bz; ++k)
          for (int j = 0; j < by; ++j)
            for (int i = 0; i < bx; ++i)
              for (int v = 0; v < 5; ++v) Lb.f[v][Lb.at(i, j, k)] = L.f[v][L.at(i0 + i, j0 + j, k0 + k)];
        patch_adjoint(c, Ug, Lb, Lg, dx, dt);
        for (int k = 0; k < bz + 2 * G; ++k)
          for (int j = 0; j < by + 2 * G; ++j)
            for (int i = 0; i < bx + 2 * G; ++i) {
              size_t d = R.at(wrap(i0 + i - G, nx), wrap(j0 + j - G, ny), wrap(k0 + k - G, nz));
              for (int v = 0; v < 5; ++v) R.f[v][d] += Lg.f[v][Lg.at(i, j, k)];
            }
      }
  store(R, lam_in);
  return 0;
}

// Adjoint of one step on a ghosted patch: lam_out on the interior ([5][nz][ny][nx]), lam_in on
// the ghosted box ([5][nz+4][ny+4][nx+4]).
int oracle_step_patch_adjoint(const oracle_config* cfg, const double* Ug, const double* lam_out, double* lam_in,
                              int nx, int ny, int nz, double dx, double dt) {
  if (!cfg || !Ug || !lam_out || !lam_in || bad_dims(nx, ny, nz)) return -1;
  Fields<double> A, L, R;
  load(A, Ug, nx + 2 * G, ny + 2 * G, nz + 2 * G);
  load(L, lam_out, nx, ny, nz);
  patch_adjoint(to_cfg(cfg), A, L, R, dx, dt);
  store(R, lam_in);
  return 0;
}

// HLLC flux of one face with normal d (0, 1, 2); q = (rho, u, v, w, p), F = flux of (rho, m, E).
int oracle_hllc(const oracle_config* cfg, const double* qL, const double* qR, int d, double* F) {
  if (!cfg || !qL || !qR || !F || d < 0 || d > 2) return -1;
  hllc_flux(to_cfg(cfg), qL, qR, d, F);
  return 0;
}

// HLLC fluxes of n faces of normal d: qL, qR and F are [5][n].
int oracle_hllc_n(const oracle_config* cfg, const double* qL, const double* qR, int d, double* F, long n) {
  if (!cfg || !qL || !qR || !F || d < 0 || d > 2 || n < 0) return -1;
  const Config c = to_cfg(cfg);
  for (long a = 0; a < n; ++a) {
    double l[5], r[5], f[5];
    for (int v = 0; v < 5; ++v) {
      l[v] = qL[(size_t)v * n + a];
      r[v] = qR[(size_t)v * n + a];
    }
    hllc_flux(c, l, r, d, f);
    for (int v = 0; v < 5; ++v) F[(size_t)v * n + a] = f[v];
  }
  return 0;
}

// Recovery of n cells: U and q are [5][n].
int oracle_recover(const oracle_config* cfg, const double* U, double* q, long n) {
  if (!cfg || !U || !q || n < 0) return -1;
  const Config c = to_cfg(cfg);
  for (long a = 0; a < n; ++a) {
    double Uc[5], w[5];
    for (int v = 0; v < 5; ++v) Uc[v] = U[(size_t)v * n + a];
    recover(c, Uc, w);
    for (int v = 0; v < 5; ++v) q[(size_t)v * n + a] = w[v];
  }
  return 0;
}

// Primitive -> conservative map of n cells ([5][n] each), and its adjoint: given lamU, the
// gradient with respect to q (rho, u, v, w, p) by the tape.
int oracle_prim_to_cons(const oracle_config* cfg, const double* q, double* U, long n) {
  if (!cfg || !q || !U || n < 0) return -1;
  const Config c = to_cfg(cfg);
  for (long a = 0; a < n; ++a) {
    double w[5], Uc[5];
    for (int v = 0; v < 5; ++v) w[v] = q[(size_t)v * n + a];
    prim_to_cons(c, w, Uc);
    for (int v = 0; v < 5; ++v) U[(size_t)v * n + a] = Uc[v];
  }
  return 0;
}
int oracle_prim_to_cons_adjoint(const oracle_config* cfg, const double* q, const double* lamU, double* lamq,
                                long n) {
  if (!cfg || !q || !lamU || !lamq || n < 0) return -1;
  const Config c = to_cfg(cfg);
  for (long a = 0; a < n; ++a) {
    Tape tape;
    active_tape() = &tape;
    TVar w[5], Uc[5];
    for (int v = 0; v < 5; ++v) w[v] = TVar(q[(size_t)v * n + a], tape.leaf());
    prim_to_cons(c, w, Uc);
    std::vector<double> adj(tape.nodes.size(), 0.0);
    for (int v = 0; v < 5; ++v)
      if (Uc[v].i >= 0) adj[(size_t)Uc[v].i] += lamU[(size_t)v * n + a];
    tape.reverse(adj);
    for (int v = 0; v < 5; ++v) lamq[(size_t)v * n + a] = adj[(size_t)w[v].i];
    active_tape() = nullptr;
  }
  return 0;
}

// Operation counts of one periodic step, per unit of each stage: out[0] recovery per cell,
// out[1] slopes per cell (3 directions), out[2] predictor per cell, out[3] face states + HLLC
// per face, out[4] update per cell (binary +, -, *, / and sqrt); out[5..24] the same by kind.
// out must hold 25 doubles.
int oracle_count_ops(const oracle_config* cfg, const double* U, int nx, int ny, int nz, double dx, double dt,
                     double* out) {
  if (!cfg || !U || !out || bad_dims(nx, ny, nz)) return -1;
  const Config c = to_cfg(cfg);
  Fields<Counted> A, Ug, q, qh, slope[3], flux[3], B;
  load(A, U, nx, ny, nz);
  fill_periodic(A, Ug);
  // out[0..4]: all operations per unit of each stage; out[5 + 4*s + k]: operations of kind k
  // (+-, *, /, sqrt) per unit of stage s.
  uint64_t& cnt = op_counter();
  uint64_t* kinds = op_kinds();
  auto reset = [&]() { cnt = 0; for (int k = 0; k < 4; ++k) kinds[k] = 0; };
  auto record = [&](int s, size_t units) {
    out[s] = (double)cnt / (double)units;
    for (int k = 0; k < 4; ++k) out[5 + 4 * s + k] = (double)kinds[k] / (double)units;
  };
  reset();
  record(0, stage_recover(c, Ug, q));
  reset();
  record(1, stage_slopes(c, q, slope));
  reset();
  record(2, stage_predict(c, q, slope, qh, dx, dt));
  reset();
  record(3, stage_fluxes(c, qh, slope, flux));
  reset();
  record(4, stage_update(Ug, flux, B, dx, dt));
  return 0;
}

// The number of OpenMP threads the oracle's parallel stages run with on this host.
int oracle_threads() { return omp_get_max_threads(); }

}  // extern "C"
