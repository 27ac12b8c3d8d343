// The step with piecewise-parabolic reconstruction (PPM; the paper lists it among its hydro
// methods, Sec. 2) on a periodic box.  Per axis and primitive variable (Colella & Woodward 1984):
//   dq_i    = MC-limited slope (the PLM MC limiter of q_i - q_{i-1} and q_{i+1} - q_i);
//   q_{i+h} = q_i + (q_{i+1} - q_i)/2 - (dq_{i+1} - dq_i)/6      (h = 1/2);
//   edges qL = q_{i-h}, qR = q_{i+h}, then: both set to q_i at a local extremum
//   ((qR - q)(q - qL) <= 0); else with D = qR - qL, Q6 = 6 (q - (qL + qR)/2): qL = 3q - 2qR if
//   D Q6 > D^2, qR = 3q - 2qL if -D^2 > D Q6.
// The rest is the PLM step with the parabola's centre slope D in the Hancock predictor and face
// states q_h + (qR - q), q_h + (qL - q) in place of q_h +- dq/2.  The stencil radius is 3.
//
// Kernel layout: one thread per column of a TX x TY tile marching up z (as the PLM kernel), on a
// periodic box (indices wrapped) or on a patch carrying three ghost layers filled by the caller.
// Shared memory holds a ring of five recovered planes (p-2 .. p+2) over the tile and three halo
// cells each side, the x- and y-face states of plane p (the tile's cells and one ring cell beyond
// each edge) and the x and y fluxes of plane p.  The z reconstruction of a column reads its own
// five ring entries; the z-face state of the plane below, the z flux below and the x/y flux
// difference of the plane below stay in registers until the plane is updated one plane later.
#pragma once

#include <algorithm>

#include "adjoint.cuh"
#include "hydro_device.cuh"
#include "internal.h"
#include "step_tile.cuh"

namespace hydro {

constexpr int kPpmHalo = 3;

template <class R, int TX, int TY>
struct PpmShared {
  static constexpr int QX = TX + 2 * kPpmHalo, QY = TY + 2 * kPpmHalo;
  R q[5][5][QY][QX];       // ring of recovered planes: [slot][var][y + 3][x + 3]
  R wx[2][5][TY][TX + 2];  // x-face states at n+1/2: [0: low face, 1: high face][var][y][x + 1]
  R wy[2][5][TY + 2][TX];  // y-face states: [low/high][var][y + 1][x]
  R fx[5][TY][TX + 1];     // flux through the low x face of cell x, x = 0 .. TX
  R fy[5][TY + 1][TX];     // flux through the low y face of cell y, y = 0 .. TY
  int sx[QX], sy[QY];      // stored index of each tile column / row (wrapped, or clamped to the ghosts)
  R red[TX * TY / 32];     // per-warp maxima of the CFL speed
  int tile;                // batched kernel: the tile taken from the work-list
};

__device__ __forceinline__ int wrap_index(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// Edges (qL, qR) of the middle one of five consecutive cell values a .. e.
template <class R>
__device__ __forceinline__ void ppm_edges(R a, R b, R c, R d, R e, R sixth, R& qL, R& qR) {
  const R sb = limited(b - a, c - b, HYDRO_MC);
  const R sc = limited(c - b, d - c, HYDRO_MC);
  const R sd = limited(d - c, e - d, HYDRO_MC);
  qL = (b + half_(c - b)) - (sc - sb) * sixth;
  qR = (c + half_(d - c)) - (sd - sc) * sixth;
  if (prod_nonpos(qR - c, c - qL)) {
    qL = c;
    qR = c;
    return;
  }
  const R D = qR - qL;
  const R Q6 = mulf_(c - half_(qL + qR), 6.f);
  const R DQ = D * Q6, DD = D * D;
  if (DQ > DD)
    qL = mulf_(c, 3.f) - twice_(qR);
  else if (-DD > DQ)
    qR = mulf_(c, 3.f) - twice_(qL);
}

// Edge offsets (edge - q) of tile cell (i, j) of the middle plane along x, y and z, and the
// Hancock-predicted state qh.  sl: ring slots of planes p-2 .. p+2.
template <class R, int TX, int TY>
__device__ __forceinline__ void ppm_cell(const PpmShared<R, TX, TY>& sm, const int sl[5], int i, int j, R gamma,
                                         R hdt, R sixth, R lo[3][5], R hi[3][5], R qh[5]) {
  const int X = i + kPpmHalo, Y = j + kPpmHalo;
  R q[5], D[3][5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const R c = sm.q[sl[2]][v][Y][X];
    q[v] = c;
    R l, r;
    ppm_edges(sm.q[sl[2]][v][Y][X - 2], sm.q[sl[2]][v][Y][X - 1], c, sm.q[sl[2]][v][Y][X + 1],
              sm.q[sl[2]][v][Y][X + 2], sixth, l, r);
    D[0][v] = r - l;
    lo[0][v] = l - c;
    hi[0][v] = r - c;
    ppm_edges(sm.q[sl[2]][v][Y - 2][X], sm.q[sl[2]][v][Y - 1][X], c, sm.q[sl[2]][v][Y + 1][X],
              sm.q[sl[2]][v][Y + 2][X], sixth, l, r);
    D[1][v] = r - l;
    lo[1][v] = l - c;
    hi[1][v] = r - c;
    ppm_edges(sm.q[sl[0]][v][Y][X], sm.q[sl[1]][v][Y][X], c, sm.q[sl[3]][v][Y][X], sm.q[sl[4]][v][Y][X], sixth, l,
              r);
    D[2][v] = r - l;
    lo[2][v] = l - c;
    hi[2][v] = r - c;
  }
  hancock(q, D[0], D[1], D[2], gamma, hdt, qh);
}

// The same reconstruction and prediction with the three axes in a loop, for double-float arithmetic,
// whose fifteen inlined edge reconstructions per cell overflow the instruction cache: one copy of
// the five per-variable reconstructions serves all axes (the stencil addresses per axis as offsets
// in the ring), the Hancock terms are summed axis by axis in the x, y, z order of ppm_cell, and the
// edge offsets (edge - q) go where the caller wants them: out(d, v, lo, hi) for axis d.
template <class R, int TX, int TY, class Out>
__device__ __forceinline__ void ppm_cell_axes(const PpmShared<R, TX, TY>& sm, const int sl[5], int i, int j, R gamma,
                                              R hdt, R sixth, R qh[5], Out out) {
  constexpr int QX = TX + 2 * kPpmHalo;
  constexpr int SLOT = 5 * (TY + 2 * kPpmHalo) * QX;  // elements per ring slot
  const R* c0 = &sm.q[sl[2]][0][j + kPpmHalo][i + kPpmHalo];
  constexpr int VAR = (TY + 2 * kPpmHalo) * QX;  // elements per variable within a slot
  R q[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) q[v] = c0[v * VAR];
  const R ir = rcp_(q[0]);
  const R gp = gamma * q[4];
  R acc[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) acc[v] = R(0);
#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
    int off[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) off[k] = d == 2 ? (sl[k] - sl[2]) * SLOT : (k - 2) * (d == 0 ? 1 : QX);
    R D[5], lo[5], hi[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const R* b = c0 + v * VAR;
      R l, r;
      ppm_edges(b[off[0]], b[off[1]], q[v], b[off[3]], b[off[4]], sixth, l, r);
      D[v] = r - l;
      lo[v] = l - q[v];
      hi[v] = r - q[v];
    }
    out(d, lo, hi);
    // Hancock terms of axis d (normal velocity q[1 + d]), as in hancock()
    const R un = d == 0 ? q[1] : (d == 1 ? q[2] : q[3]);
    const R Dn = d == 0 ? D[1] : (d == 1 ? D[2] : D[3]);
    R t[5];
    t[0] = un * D[0] + q[0] * Dn;
    t[1] = un * D[1];
    t[2] = un * D[2];
    t[3] = un * D[3];
    const R tn = (d == 0 ? t[1] : (d == 1 ? t[2] : t[3])) + D[4] * ir;
    if (d == 0) t[1] = tn;
    else if (d == 1) t[2] = tn;
    else t[3] = tn;
    t[4] = gp * Dn + un * D[4];
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] = d == 0 ? t[v] : acc[v] + t[v];
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) qh[v] = q[v] - hdt * acc[v];
}

// Resident blocks per SM: the 8-byte ring and face arrays take ~165 KB of shared memory.
template <class Pol>
constexpr int ppm_min_blocks() { return sizeof(typename Pol::R) >= 8 ? 1 : 2; }

// Block-wide maximum of v (all threads call); the result is valid in thread 0.
template <class R, int TX, int TY>
__device__ __forceinline__ R ppm_block_max(PpmShared<R, TX, TY>& sm, R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    R w = shfl_xor_(v, o);
    v = w > v ? w : v;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sm.red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < TX * TY / 32; ++w) v = sm.red[w] > v ? sm.red[w] : v;
  return v;
}

// Columns [x0, x0+TX) x rows [y0, y0+TY) x planes [z0, z1) of patch P (P.gin == 0: a periodic box;
// P.gin == 3: ghost layers filled by the caller) stepped by dt; with want_cfl the largest CFL speed
// of the updated cells of this thread is folded into smax.
template <class Pol, int TX, int TY>
__device__ __forceinline__ void ppm_tile(PpmShared<typename Pol::R, TX, TY>& sm, const PatchIO<typename Pol::S>& P,
                                         int x0, int y0, int z0, int z1, const Params& prm, double dtv, bool want_cfl,
                                         unsigned& flags, typename Pol::R& smax) {
  using S = typename Pol::S;
  using R = typename Pol::R;
  constexpr int QX = TX + 2 * kPpmHalo, QY = TY + 2 * kPpmHalo, NT = TX * TY;
  constexpr bool kCompactPpm = std::is_same<R, df>::value;  // double-float arithmetic
  const int tid = threadIdx.x;
  const bool periodic = P.gin == 0;
  __syncthreads();  // the previous tile's last reads of the index tables are done
  for (int k = tid; k < QX; k += NT)
    sm.sx[k] = periodic ? wrap_index(x0 + k - kPpmHalo, P.nx) : min(x0 + k - kPpmHalo + P.gin, P.nx + 2 * P.gin - 1);
  for (int k = tid; k < QY; k += NT)
    sm.sy[k] = periodic ? wrap_index(y0 + k - kPpmHalo, P.ny) : min(y0 + k - kPpmHalo + P.gin, P.ny + 2 * P.gin - 1);
  __syncthreads();
  const R gamma = kc<R>(prm, K_GAMMA), igm1 = kc<R>(prm, K_IGM1), sixth = kc<R>(prm, K_SIXTH);
  const R rf = kc<R>(prm, K_RHOF), pf = kc<R>(prm, K_PF);
  const R hdt = (R)(0.5 * dtv / P.dx);
  const R dtdx = (R)(dtv / P.dx);

  // plane z of the patch (wrapped, or within the ghost layers), recovered into ring slot s over
  // the tile and its halo
  auto load_plane = [&](int z, int s, int first, int stride) {
    const long long zo = (long long)(periodic ? wrap_index(z, P.nz) : z + P.gin) * P.isz;
    for (int c = first; c < QX * QY; c += stride) {
      const int y = c / QX, x = c - y * QX;
      const long long a = zo + (long long)sm.sy[y] * P.isy + sm.sx[x];
      S U[5];
      R q[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) U[v] = __ldg(P.in[v] + a);
      Pol::recover(U, prm, q, flags);
#pragma unroll
      for (int v = 0; v < 5; ++v) sm.q[s][v][y][x] = q[v];
    }
  };
  // slot of plane z: (z - z0 + 3) mod 5
  for (int k = 0; k < 5; ++k) load_plane(z0 - kPpmHalo + k, k, tid, NT);
  __syncthreads();

  const int i = tid % TX, j = tid / TX;
  const bool own = x0 + i < P.nx && y0 + j < P.ny;
  // ring cell of this thread: x-low (i = -1), x-high (i = TX), y-low (j = -1), y-high (j = TY)
  int rk = -1, ri = 0, rj = 0;
  if (tid < TY) { rk = 0; ri = -1; rj = tid; }
  else if (tid < 2 * TY) { rk = 1; ri = TX; rj = tid - TY; }
  else if (tid < 2 * TY + TX) { rk = 2; ri = tid - 2 * TY; rj = -1; }
  else if (tid < 2 * TY + 2 * TX) { rk = 3; ri = tid - 2 * TY - TX; rj = TY; }

  // Split barriers (ids 1-3), in double-float arithmetic, whose block is alone on its SM: the
  // ring cells belong to the first NR threads, whole warps, which signal barrier 1 once their tile
  // cells are predicted, predict the ring, signal barrier 3 and take the faces between ring and
  // tile after barrier 2; the other warps wait for every tile cell (barrier 1), signal barrier 2,
  // take the faces between two tile cells and, once the ring cells no longer read plane p-2
  // (barrier 3), load plane p+3 into its slot.  The ring cells' full reconstructions then overlap
  // the interior faces instead of holding the other warps at one block barrier (+4.5% at 512^3).
  // Float arithmetic keeps one block barrier per phase: with two resident blocks the other block
  // fills the waits, and the split (FP32 -6.5%, the batched mixed step -5%) or one call site for
  // the tile and ring reconstructions (FP32 -10%) cost more.
  constexpr int NR = 2 * (TX + TY), NIX = (TX - 1) * TY, NIF = NIX + TX * (TY - 1);
  constexpr bool kSplit = kCompactPpm && NR % 32 == 0 && NR < NT;
  const bool ringw = tid < NR;

  R zhi[5], fzb[5], dxy[5];  // z-high face state, z flux below, x/y flux difference: plane p-1
#pragma unroll
  for (int v = 0; v < 5; ++v) zhi[v] = fzb[v] = dxy[v] = R(0);
  for (int p = z0 - 1; p <= z1; ++p) {
    const int base = p - z0 + 1;
    int sl[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) sl[k] = (base + k) % 5;
    const bool xy = p >= z0 && p < z1;  // plane p is updated: its x and y faces are needed
    R zlo[5], znew[5];
    // z face p - 1/2, then the update of plane p - 1 (its faces p - 3/2 and p - 1/2 are known)
    auto zface_update = [&]() {
      if (p > z0 - 1) {
        R ql[5], qr[5], F[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          ql[v] = zhi[v];
          qr[v] = zlo[v];
        }
        floor_state(ql, rf, pf);
        floor_state(qr, rf, pf);
        hllc<2>(ql, qr, gamma, igm1, F);
        if (p > z0 && own) {
          const int z = p - 1;
          const long long ai = (long long)(z + P.gin) * P.isz + (long long)(y0 + j + P.gin) * P.isy + (x0 + i + P.gin);
          const long long ao = (long long)(z + P.gout) * P.osz + (long long)(y0 + j + P.gout) * P.osy + (x0 + i + P.gout);
          S Un[5];
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            Un[v] = Pol::update(__ldg(P.in[v] + ai), dtdx, dxy[v] + (F[v] - fzb[v]));
            P.out[v][ao] = Un[v];
          }
          if (want_cfl) {
            const R sp = Pol::speed(Un, prm, flags);
            smax = sp > smax ? sp : smax;
          }
        }
#pragma unroll
        for (int v = 0; v < 5; ++v) fzb[v] = F[v];
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) zhi[v] = znew[v];
    };
    if constexpr (kCompactPpm) {
      // double-float: the tile cell (it 0) and this thread's ring cell (it 1) through one inlined
      // copy of the reconstruction; the x/y edge offsets are stored and completed with qh after it
      for (int it = 0; it < 2; ++it) {
        if (it == 1 && !(xy && rk >= 0)) break;
        const int ci = it == 0 ? i : ri, cj = it == 0 ? j : rj;
        R qh[5];
        ppm_cell_axes(sm, sl, ci, cj, gamma, hdt, sixth, qh, [&](int d, const R lo[5], const R hi[5]) {
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            if (it == 0) {
              if (d == 2) {
                zlo[v] = lo[v];
                znew[v] = hi[v];
              } else if (xy && d == 0) {
                sm.wx[0][v][j][i + 1] = lo[v];
                sm.wx[1][v][j][i + 1] = hi[v];
              } else if (xy) {
                sm.wy[0][v][j + 1][i] = lo[v];
                sm.wy[1][v][j + 1][i] = hi[v];
              }
            } else if (d == (rk >> 1)) {
              if (rk == 0) sm.wx[1][v][rj][0] = hi[v];
              else if (rk == 1) sm.wx[0][v][rj][TX + 1] = lo[v];
              else if (rk == 2) sm.wy[1][v][0][ri] = hi[v];
              else sm.wy[0][v][TY + 1][ri] = lo[v];
            }
          }
        });
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          if (it == 0) {
            zlo[v] = qh[v] + zlo[v];
            znew[v] = qh[v] + znew[v];
            if (xy) {
              sm.wx[0][v][j][i + 1] = qh[v] + sm.wx[0][v][j][i + 1];
              sm.wx[1][v][j][i + 1] = qh[v] + sm.wx[1][v][j][i + 1];
              sm.wy[0][v][j + 1][i] = qh[v] + sm.wy[0][v][j + 1][i];
              sm.wy[1][v][j + 1][i] = qh[v] + sm.wy[1][v][j + 1][i];
            }
          } else if (rk == 0) sm.wx[1][v][rj][0] = qh[v] + sm.wx[1][v][rj][0];
          else if (rk == 1) sm.wx[0][v][rj][TX + 1] = qh[v] + sm.wx[0][v][rj][TX + 1];
          else if (rk == 2) sm.wy[1][v][0][ri] = qh[v] + sm.wy[1][v][0][ri];
          else sm.wy[0][v][TY + 1][ri] = qh[v] + sm.wy[0][v][TY + 1][ri];
        }
        if (it == 0) {
          zface_update();
          if (kSplit && xy && ringw) bar_arrive(1, NT);
        }
      }
    } else {
      R lo[3][5], hi[3][5], qh[5];
      ppm_cell(sm, sl, i, j, gamma, hdt, sixth, lo, hi, qh);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        zlo[v] = qh[v] + lo[2][v];
        znew[v] = qh[v] + hi[2][v];
        if (xy) {
          sm.wx[0][v][j][i + 1] = qh[v] + lo[0][v];
          sm.wx[1][v][j][i + 1] = qh[v] + hi[0][v];
          sm.wy[0][v][j + 1][i] = qh[v] + lo[1][v];
          sm.wy[1][v][j + 1][i] = qh[v] + hi[1][v];
        }
      }
    }
    if (!kCompactPpm && xy && rk >= 0) {
      R lo[3][5], hi[3][5], qh[5];
      ppm_cell(sm, sl, ri, rj, gamma, hdt, sixth, lo, hi, qh);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        if (rk == 0) sm.wx[1][v][rj][0] = qh[v] + hi[0][v];
        else if (rk == 1) sm.wx[0][v][rj][TX + 1] = qh[v] + lo[0][v];
        else if (rk == 2) sm.wy[1][v][0][ri] = qh[v] + hi[1][v];
        else sm.wy[0][v][TY + 1][ri] = qh[v] + lo[1][v];
      }
    }
    if constexpr (!kCompactPpm) zface_update();
    if (kSplit && xy) {
      if (ringw) {
        bar_arrive(3, NT);
        bar_sync(2, NT);
      } else {
        bar_sync(1, NT);
        bar_arrive(2, NT);
      }
      // faces f < NIF between two tile cells (x, then y) by the other warps; face NIF + tid
      // between this thread's ring cell and the tile by a ring thread; one HLLC call site
      const int fend = ringw ? NIF + tid + 1 : NIF;
      for (int f = ringw ? NIF + tid : tid - NR; f < fend; f += NT - NR) {
        int d, fx, fy;
        if (f < NIX) {
          d = 0; fy = f / (TX - 1); fx = f - fy * (TX - 1) + 1;
        } else if (f < NIF) {
          const int g = f - NIX;
          d = 1; fy = g / TX; fx = g - fy * TX; fy += 1;
        } else if (rk == 0) { d = 0; fx = 0; fy = rj; }
        else if (rk == 1) { d = 0; fx = TX; fy = rj; }
        else if (rk == 2) { d = 1; fx = ri; fy = 0; }
        else { d = 1; fx = ri; fy = TY; }
        R ql[5], qr[5], F[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          ql[v] = d == 0 ? sm.wx[1][v][fy][fx] : sm.wy[1][v][fy][fx];
          qr[v] = d == 0 ? sm.wx[0][v][fy][fx + 1] : sm.wy[0][v][fy + 1][fx];
        }
        floor_state(ql, rf, pf);
        floor_state(qr, rf, pf);
        hllc_dyn(d, ql, qr, gamma, igm1, F);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          if (d == 0) sm.fx[v][fy][fx] = F[v];
          else sm.fy[v][fy][fx] = F[v];
        }
      }
      if (!ringw) {
        bar_sync(3, NT);
        load_plane(p + kPpmHalo, sl[0], tid - NR, NT - NR);  // (p < z1 on an x/y plane)
      }
      __syncthreads();  // fluxes and plane p+3 in place
      if (xy) {
#pragma unroll
        for (int v = 0; v < 5; ++v)
          dxy[v] = (sm.fx[v][j][i + 1] - sm.fx[v][j][i]) + (sm.fy[v][j + 1][i] - sm.fy[v][j][i]);
      }
      continue;
    }
    __syncthreads();  // face states written; ring slot of plane p-2 free
    if (kCompactPpm && xy) {
      // double-float: x and y faces through one inlined copy of HLLC (runtime normal)
      constexpr int NXF = (TX + 1) * TY;
      for (int f = tid; f < NXF + TX * (TY + 1); f += NT) {
        const int d = f < NXF ? 0 : 1;
        const int g = d == 0 ? f : f - NXF;
        const int w = d == 0 ? TX + 1 : TX;
        const int fy = g / w, fx = g - fy * w;
        R ql[5], qr[5], F[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          ql[v] = d == 0 ? sm.wx[1][v][fy][fx] : sm.wy[1][v][fy][fx];
          qr[v] = d == 0 ? sm.wx[0][v][fy][fx + 1] : sm.wy[0][v][fy + 1][fx];
        }
        floor_state(ql, rf, pf);
        floor_state(qr, rf, pf);
        hllc_dyn(d, ql, qr, gamma, igm1, F);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          if (d == 0) sm.fx[v][fy][fx] = F[v];
          else sm.fy[v][fy][fx] = F[v];
        }
      }
    } else if (xy) {
      for (int f = tid; f < (TX + 1) * TY; f += NT) {
        const int fy = f / (TX + 1), fx = f - fy * (TX + 1);
        R ql[5], qr[5], F[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          ql[v] = sm.wx[1][v][fy][fx];
          qr[v] = sm.wx[0][v][fy][fx + 1];
        }
        floor_state(ql, rf, pf);
        floor_state(qr, rf, pf);
        hllc<0>(ql, qr, gamma, igm1, F);
#pragma unroll
        for (int v = 0; v < 5; ++v) sm.fx[v][fy][fx] = F[v];
      }
      for (int f = tid; f < TX * (TY + 1); f += NT) {
        const int fy = f / TX, fx = f - fy * TX;
        R ql[5], qr[5], F[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          ql[v] = sm.wy[1][v][fy][fx];
          qr[v] = sm.wy[0][v][fy + 1][fx];
        }
        floor_state(ql, rf, pf);
        floor_state(qr, rf, pf);
        hllc<1>(ql, qr, gamma, igm1, F);
#pragma unroll
        for (int v = 0; v < 5; ++v) sm.fy[v][fy][fx] = F[v];
      }
    }
    if (p < z1) load_plane(p + kPpmHalo, sl[0], tid, NT);
    __syncthreads();  // fluxes and plane p+3 in place
    if (xy) {
#pragma unroll
      for (int v = 0; v < 5; ++v)
        dxy[v] = (sm.fx[v][j][i + 1] - sm.fx[v][j][i]) + (sm.fy[v][j + 1][i] - sm.fy[v][j][i]);
    }
  }
}

// Periodic box: one tile per block, tiles from the block index.
template <class Pol, int TX, int TY>
__global__ void __launch_bounds__(TX * TY, ppm_min_blocks<Pol>())
    k_step_ppm(PatchIO<typename Pol::S> P, Params prm, const double* dt_dev, double* dt_next, int zchunk,
               unsigned* err) {
  using R = typename Pol::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& sm = *reinterpret_cast<PpmShared<R, TX, TY>*>(smem_raw);
  const double dt = dt_dev[0];
  if (!(dt > 0.0 && dt <= 1e300)) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) atomicOr(err, HYDRO_EBIT_BAD_DT);
    return;
  }
  unsigned flags = 0;
  R smax = 0;
  const int z0 = blockIdx.z * zchunk;
  ppm_tile<Pol, TX, TY>(sm, P, blockIdx.x * TX, blockIdx.y * TY, z0, min(z0 + zchunk, P.nz), prm, dt,
                        dt_next != nullptr, flags, smax);
  if (dt_next) {
    const R m = ppm_block_max(sm, smax);
    if (threadIdx.x == 0) publish_dt(prm.cfl, P.dx, (double)m, dt_next);
  }
  flush_flags(flags, err);
}

// Patches with three ghost layers: a persistent grid taking tiles from the device work-list by an
// atomic counter (as the PLM batched kernel); per-patch dt, dx and dt_next.
template <class Pol, int TX, int TY>
__global__ void __launch_bounds__(TX * TY, ppm_min_blocks<Pol>())
    k_step_ppm_batched(const PatchIO<typename Pol::S>* patches, const TileRec* tiles, int ntiles, int* counter,
                       Params prm, const double* dt_dev, double* dt_next, int zchunk, unsigned* err) {
  using R = typename Pol::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& sm = *reinterpret_cast<PpmShared<R, TX, TY>*>(smem_raw);
  unsigned flags = 0;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) sm.tile = atomicAdd(counter, 1);
    __syncthreads();
    const int t = sm.tile;
    if (t >= ntiles) break;
    const TileRec r = tiles[t];
    const PatchIO<typename Pol::S> P = patches[r.patch];
    if (r.x0 < 0 || r.y0 < 0 || r.z0 < 0 || r.x0 >= P.nx || r.y0 >= P.ny || r.z0 >= P.nz || P.gin != kPpmHalo) {
      flags |= HYDRO_EBIT_BAD_TILE;
      continue;
    }
    const double dt = dt_dev[r.patch];
    if (!(dt > 0.0 && dt <= 1e300)) {
      flags |= HYDRO_EBIT_BAD_DT;
      continue;
    }
    R smax = 0;
    ppm_tile<Pol, TX, TY>(sm, P, r.x0, r.y0, r.z0, min(r.z0 + zchunk, P.nz), prm, dt, dt_next != nullptr, flags,
                          smax);
    if (dt_next) {
      const R m = ppm_block_max(sm, smax);
      if (threadIdx.x == 0) publish_dt(prm.cfl, P.dx, (double)m, dt_next + r.patch);
    }
  }
  flush_flags(flags, err);
}

constexpr int kPpmTX = 16, kPpmTY = 16;
static_assert(kTileX[0] == kPpmTX && kTileY[0] == kPpmTY, "the PPM work-list is built with tile shape 0");

template <class Pol>
cudaError_t ppm_attr(const void* fn) {
  const size_t smem = sizeof(PpmShared<typename Pol::R, kPpmTX, kPpmTY>);
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <class Pol>
cudaError_t launch_ppm(const HostPatchIO& P, const Params& prm, const double* dt, double* dt_next, int zchunk,
                       unsigned* err, cudaStream_t s) {
  static PerDeviceOnce attr;
  cudaError_t ea = attr.call([&] { return ppm_attr<Pol>(reinterpret_cast<const void*>(k_step_ppm<Pol, kPpmTX, kPpmTY>)); });
  if (ea != cudaSuccess) return ea;
  const size_t smem = sizeof(PpmShared<typename Pol::R, kPpmTX, kPpmTY>);
  dim3 grid((P.nx + kPpmTX - 1) / kPpmTX, (P.ny + kPpmTY - 1) / kPpmTY, (P.nz + zchunk - 1) / zchunk);
  k_step_ppm<Pol, kPpmTX, kPpmTY><<<grid, kPpmTX * kPpmTY, smem, s>>>(to_dev<Pol>(P), prm, dt, dt_next, zchunk, err);
  return cudaGetLastError();
}

template <class Pol>
cudaError_t launch_ppm_batched(const HostPatchIO* d_patches, const HostTileRec* d_tiles, int ntiles, int* d_counter,
                               const Params& prm, const double* dt, double* dt_next, int zchunk, unsigned* err,
                               int sm_count, cudaStream_t s) {
  using K = decltype(&k_step_ppm_batched<Pol, kPpmTX, kPpmTY>);
  const K fn = &k_step_ppm_batched<Pol, kPpmTX, kPpmTY>;
  static PerDeviceOnce attr;
  cudaError_t ea = attr.call([&] { return ppm_attr<Pol>(reinterpret_cast<const void*>(fn)); });
  if (ea != cudaSuccess) return ea;
  const size_t smem = sizeof(PpmShared<typename Pol::R, kPpmTX, kPpmTY>);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPpmTX * kPpmTY, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  const int grid = std::max(1, std::min(ntiles, sm_count * per_sm));
  fn<<<grid, kPpmTX * kPpmTY, smem, s>>>(reinterpret_cast<const PatchIO<typename Pol::S>*>(d_patches),
                                         reinterpret_cast<const TileRec*>(d_tiles), ntiles, d_counter, prm, dt,
                                         dt_next, zchunk, err);
  return cudaGetLastError();
}

}  // namespace hydro
