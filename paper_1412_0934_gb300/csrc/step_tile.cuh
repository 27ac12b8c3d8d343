// One MUSCL-Hancock/HLLC step of a TX x TY column tile of a patch, marching in z through
// shared memory (the GPU solves hydro on chunks of patches carrying their boundary cells,
// Sec. 3; every flux that updates a patch's cells is computed on the GPU, Sec. 4).
//
// Per plane p of the march (p = z0-1 .. z1), with a 3-plane ring of primitive planes, two phases
// separated by block barriers:
//   1  slopes (x, y, z) and Hancock predictor of plane p over the tile (plus a 1-cell ring when
//      plane p's x/y faces are needed); each interior column forms its z face states and the HLLC
//      flux of face p-1/2, then updates plane p-1:  U - dt/dx ((dFx + dFy) + dFz) from the x/y
//      fluxes of plane p-1 in shared memory, writes it, and folds the CFL speed of the new state
//      into a running maximum
//   2  HLLC fluxes of the x and y faces of plane p (each face once), and the load of U of plane
//      p+2 over the tile plus 2 halo cells per side, recovered to q into the ring
// Global memory is read once per cell per plane (halo re-reads come from L2) and written once.
// In double-float arithmetic with one block per SM (32x16 tiles, or the one-block build), the
// ring cells' predictions of phase 1 overlap the interior faces of phase 2 through named barriers:
// the ring warps signal that their tile cells are predicted, predict the ring, and take the faces
// between ring and tile, while the other warps take the faces between tile cells and the load.
#pragma once
#include <type_traits>

#include "hydro_device.cuh"

namespace hydro {

// Device view of one (input, output) patch pair.
template <class S>
struct PatchIO {
  const S* in[5];
  S* out[5];
  int nx, ny, nz;
  int gin, gout;  // ghost layers of in / out; gin == 0 means a periodic box
  long long isy, isz, osy, osz;
  double dx;
};

// One tile of the work-list: columns [x0, x0+TX) x [y0, y0+TY), planes [z0, min(z0+zchunk, nz)).
struct TileRec {
  int patch, x0, y0, z0;
};

// Five values per cell of an H x W plane, packed for wide shared-memory accesses:
// float: (v0..v3) as one float4 + v4; double: (v0,v1), (v2,v3) as double2 + v4.
template <class R, int H, int W>
struct Plane5;
template <int H, int W>
struct Plane5<float, H, W> {
  float4 a[H][W];
  float b[H][W];
  __device__ __forceinline__ void st(int j, int i, const float v[5]) {
    a[j][i] = make_float4(v[0], v[1], v[2], v[3]);
    b[j][i] = v[4];
  }
  __device__ __forceinline__ void ld(int j, int i, float v[5]) const {
    const float4 t = a[j][i];
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    v[4] = b[j][i];
  }
};
template <int H, int W>
struct Plane5<double, H, W> {
  double2 a[H][W];
  double2 b[H][W];
  double c[H][W];
  __device__ __forceinline__ void st(int j, int i, const double v[5]) {
    a[j][i] = make_double2(v[0], v[1]);
    b[j][i] = make_double2(v[2], v[3]);
    c[j][i] = v[4];
  }
  __device__ __forceinline__ void ld(int j, int i, double v[5]) const {
    const double2 t = a[j][i], u = b[j][i];
    v[0] = t.x; v[1] = t.y; v[2] = u.x; v[3] = u.y;
    v[4] = c[j][i];
  }
};

template <int H, int W>
struct Plane5<df, H, W> {
  float4 a[H][W];  // (h0, l0, h1, l1)
  float4 b[H][W];  // (h2, l2, h3, l3)
  float2 c[H][W];  // (h4, l4)
  __device__ __forceinline__ void st(int j, int i, const df v[5]) {
    a[j][i] = make_float4(v[0].h, v[0].l, v[1].h, v[1].l);
    b[j][i] = make_float4(v[2].h, v[2].l, v[3].h, v[3].l);
    c[j][i] = make_float2(v[4].h, v[4].l);
  }
  __device__ __forceinline__ void ld(int j, int i, df v[5]) const {
    const float4 t = a[j][i], u = b[j][i];
    const float2 w = c[j][i];
    v[0] = df(t.x, t.y); v[1] = df(t.z, t.w); v[2] = df(u.x, u.y); v[3] = df(u.z, u.w);
    v[4] = df(w.x, w.y);
  }
};

template <class Pol, int TX, int TY>
struct TileShared {
  using R = typename Pol::R;
  Plane5<R, TY + 4, TX + 4> q[3];  // primitive planes p-1, p, p+1 (ring)
  Plane5<R, TY + 2, TX + 2> qh;    // predicted state of plane p (tile + 1 ring)
  Plane5<R, TY + 2, TX + 2> sx;    // x slopes of plane p
  Plane5<R, TY + 2, TX + 2> sy;    // y slopes of plane p
  Plane5<R, TY, TX + 1> fx;        // x-face fluxes of plane p, index i+1 for face i+1/2
  Plane5<R, TY + 1, TX> fy;        // y-face fluxes of plane p, index j+1 for face j+1/2
  long long yoff[TY + 4];          // y offset (y index * stride) of the halo rows
  int xoff[TX + 4];                // x index of the halo columns
  int pairok[(TX + 4) / 2];        // halo columns 2k, 2k+1 adjacent in memory, the first even
  R red[TX * TY / 32];
  int tile;
};

__device__ __forceinline__ int wrapi(int x, int n) {
  x %= n;
  return x < 0 ? x + n : x;
}
__device__ __forceinline__ int ring_slot(int p) { return (p + 3) % 3; }

// Limited slope of a cell from its backward and forward differences, the limiter fixed at compile
// time (the step kernels are compiled once per limiter: its tests and selections then cost no
// branches on a run-time value); the same values as limited(a, b, LIM).
template <int LIM, class R>
__device__ __forceinline__ R limited_t(R a, R b, int) {
  if constexpr (LIM == HYDRO_MINMOD) return minmod(a, b);
  else return limited(a, b, LIM);
}

template <int LIM, class Pol, int TX, int TY>
__device__ __forceinline__ void predict_cell(TileShared<Pol, TX, TY>& sm, int i, int j, int sm1, int s0, int sp1,
                                             const Params& prm, typename Pol::R hdt, typename Pol::R qh[5],
                                             typename Pol::R dqz[5]) {
  using R = typename Pol::R;
  const int ci = i + 2, cj = j + 2;
  R c[5], xm[5], xp[5], ym[5], yp[5], zm[5], zp[5], dqx[5], dqy[5];
  sm.q[s0].ld(cj, ci, c);
  sm.q[s0].ld(cj, ci - 1, xm);
  sm.q[s0].ld(cj, ci + 1, xp);
  sm.q[s0].ld(cj - 1, ci, ym);
  sm.q[s0].ld(cj + 1, ci, yp);
  sm.q[sm1].ld(cj, ci, zm);
  sm.q[sp1].ld(cj, ci, zp);
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    dqx[v] = limited_t<LIM>(c[v] - xm[v], xp[v] - c[v], prm.limiter);
    dqy[v] = limited_t<LIM>(c[v] - ym[v], yp[v] - c[v], prm.limiter);
    dqz[v] = limited_t<LIM>(c[v] - zm[v], zp[v] - c[v], prm.limiter);
  }
  hancock(c, dqx, dqy, dqz, kc<R>(prm, K_GAMMA), hdt, qh);
  sm.qh.st(j + 1, i + 1, qh);
  sm.sx.st(j + 1, i + 1, dqx);
  sm.sy.st(j + 1, i + 1, dqy);
}

// Flux of the x face between tile cells (i, j) and (i+1, j) (D = 0) or the y face between
// (i, j) and (i, j+1) (D = 1), from the predicted states and slopes of plane p.
template <int D, class Pol, int TX, int TY>
__device__ __forceinline__ void face_flux(TileShared<Pol, TX, TY>& sm, int i, int j, const Params& prm,
                                          typename Pol::R F[5]) {
  using R = typename Pol::R;
  const int li = i + 1, lj = j + 1;
  const int ri = li + (D == 0), rj = lj + (D == 1);
  R qL[5], qR[5], sL[5], sR[5];
  sm.qh.ld(lj, li, qL);
  sm.qh.ld(rj, ri, qR);
  if (D == 0) {
    sm.sx.ld(lj, li, sL);
    sm.sx.ld(rj, ri, sR);
  } else {
    sm.sy.ld(lj, li, sL);
    sm.sy.ld(rj, ri, sR);
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    qL[v] = qL[v] + half_(sL[v]);
    qR[v] = qR[v] - half_(sR[v]);
  }
  floor_state(qL, kc<R>(prm, K_RHOF), kc<R>(prm, K_PF));
  floor_state(qR, kc<R>(prm, K_RHOF), kc<R>(prm, K_PF));
  hllc<D>(qL, qR, kc<R>(prm, K_GAMMA), kc<R>(prm, K_IGM1), F);
}

// The same for a runtime direction d (one inlined copy serves both x and y faces).
template <class Pol, int TX, int TY>
__device__ __forceinline__ void face_flux_dyn(TileShared<Pol, TX, TY>& sm, int d, int i, int j, const Params& prm,
                                              typename Pol::R F[5]) {
  using R = typename Pol::R;
  const int li = i + 1, lj = j + 1;
  const int ri = li + (d == 0), rj = lj + (d == 1);
  R qL[5], qR[5], sL[5], sR[5];
  sm.qh.ld(lj, li, qL);
  sm.qh.ld(rj, ri, qR);
  const auto& sl = d == 0 ? sm.sx : sm.sy;
  sl.ld(lj, li, sL);
  sl.ld(rj, ri, sR);
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    qL[v] = qL[v] + half_(sL[v]);
    qR[v] = qR[v] - half_(sR[v]);
  }
  floor_state(qL, kc<R>(prm, K_RHOF), kc<R>(prm, K_PF));
  floor_state(qR, kc<R>(prm, K_RHOF), kc<R>(prm, K_PF));
  hllc_dyn(d, qL, qR, kc<R>(prm, K_GAMMA), kc<R>(prm, K_IGM1), F);
}

// Bounds-checked build (compiled with -DHYDRO_CHECK_BOUNDS; the library's default build has no
// checks): every global index of the step is tested against the extent of its patch's array,
// (nz + 2 ghost layers) z strides, before the access; an index outside sets HYDRO_EBIT_OOB and the
// access is skipped (a load then reads zero).
#ifdef HYDRO_CHECK_BOUNDS
constexpr bool kCheckBounds = true;
#else
constexpr bool kCheckBounds = false;
#endif
__device__ __forceinline__ bool index_ok(long long a, long long extent, unsigned& flags) {
  if (!kCheckBounds) return true;
  const bool ok = a >= 0 && a < extent;
  if (!ok) flags |= HYDRO_EBIT_OOB;
  return ok;
}

// Two x-adjacent stored values at an even, vector-aligned address (one 16-byte load for double,
// 8-byte for float), read through the read-only path.
__device__ __forceinline__ void ldg_pair(const double* p, double& a, double& b) {
  const double2 t = __ldg(reinterpret_cast<const double2*>(p));
  a = t.x;
  b = t.y;
}
__device__ __forceinline__ void ldg_pair(const float* p, float& a, float& b) {
  const float2 t = __ldg(reinterpret_cast<const float2*>(p));
  a = t.x;
  b = t.y;
}

// Named block barriers 1-3 (0 is __syncthreads), in their non-aligned form: a thread that arrives does
// not wait; a thread that syncs waits until `count` threads have arrived (arrive or sync).  Memory
// accesses before an arrive or a sync are visible to the threads that return from the sync.
__device__ __forceinline__ void bar_arrive(int id, int count) {
  asm volatile("barrier.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_sync(int id, int count) {
  asm volatile("barrier.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Resident blocks per SM the register allocation must allow: 2 x 256 threads for 8-byte
// arithmetic (its shared memory allows 2), 3 x 256 for float arithmetic (4 x 256, a 64-register
// budget, spills more than the extra warps gain: measured -8% for FP32, 0..-2% for mixed).
template <class Pol, int NT, int MINB>
constexpr int min_blocks() {
  constexpr int b = (sizeof(typename Pol::R) >= 8 ? 2 : 3) * 256 / NT;
  return MINB > 0 ? MINB : (b < 1 ? 1 : b);
}

// Advances the tile; returns (through smax) the largest CFL speed of the updated cells.
template <int LIM, int MINB, class Pol, int TX, int TY>
__device__ void step_tile(TileShared<Pol, TX, TY>& sm, const PatchIO<typename Pol::S>& P, int x0, int y0, int z0,
                          int z1, const Params& prm, double dt, bool want_cfl, unsigned& flags,
                          typename Pol::R& smax) {
  using S = typename Pol::S;
  using R = typename Pol::R;
  constexpr int NT = TX * TY;
  constexpr int QW = TX + 4, QH = TY + 4, QN = QW * QH;
  const int tid = threadIdx.x;
  const int ti = tid % TX, tj = tid / TX;
  const bool periodic = (P.gin == 0);

  for (int c = tid; c < QW; c += NT) {
    int x = x0 - 2 + c;
    sm.xoff[c] = periodic ? wrapi(x, P.nx) : min(max(x, -2), P.nx + 1) + 2;
  }
  for (int c = tid; c < QH; c += NT) {
    int y = y0 - 2 + c;
    y = periodic ? wrapi(y, P.ny) : min(max(y, -2), P.ny + 1) + 2;
    sm.yoff[c] = (long long)y * P.isy;
  }
  // Vector loads of cell pairs need even strides and field pointers aligned to the pair's size.
  bool vec = (P.isy % 2 == 0) && (P.isz % 2 == 0);
#pragma unroll
  for (int v = 0; v < 5; ++v) vec = vec && (reinterpret_cast<uintptr_t>(P.in[v]) % (2 * sizeof(S)) == 0);
  __syncthreads();
  for (int k = tid; k < QW / 2; k += NT) {
    const int a = sm.xoff[2 * k], b = sm.xoff[2 * k + 1];
    sm.pairok[k] = vec && b == a + 1 && (a & 1) == 0;
  }
  __syncthreads();

  auto plane_offset = [&](int z) {
    const int zi = periodic ? wrapi(z, P.nz) : z + 2;
    return (long long)zi * P.isz;
  };
  // Plane loads, two x-adjacent cells per thread: pair c of the (TX+4) x (TY+4) halo plane (cells
  // 2 (c mod QP), +1 of row c / QP) goes to thread NT-1-c (mod NT), so the threads left without a
  // pair (or with one pair where others take two) are the first ones, the warps that also take the
  // tile's edge faces.  A pair adjacent in memory (pairok: no wrap or clamp between its columns, the
  // first column even) is read with one vector load per field, else with two.
  constexpr int QP = QW / 2, QNP = QH * QP;
  const long long in_extent = (long long)(P.nz + 2 * P.gin) * P.isz;
  auto fetch_pair = [&](long long zo, int c, S U0[5], S U1[5]) {
    const int cy = c / QP, px = c - cy * QP;
    const long long a = zo + sm.yoff[cy] + sm.xoff[2 * px];
    if (sm.pairok[px]) {
      if (!index_ok(a, in_extent, flags) || !index_ok(a + 1, in_extent, flags)) {
#pragma unroll
        for (int v = 0; v < 5; ++v) U0[v] = U1[v] = S(0);
        return;
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) ldg_pair(P.in[v] + a, U0[v], U1[v]);
    } else {
      const long long a1 = zo + sm.yoff[cy] + sm.xoff[2 * px + 1];
      if (!index_ok(a, in_extent, flags) || !index_ok(a1, in_extent, flags)) {
#pragma unroll
        for (int v = 0; v < 5; ++v) U0[v] = U1[v] = S(0);
        return;
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        U0[v] = __ldg(P.in[v] + a);
        U1[v] = __ldg(P.in[v] + a1);
      }
    }
  };
  auto store_pair = [&](int slot, int c, const S U0[5], const S U1[5]) {
    const int cy = c / QP, cx = 2 * (c - cy * QP);
    R q[5];
    Pol::recover(U0, prm, q, flags);
    sm.q[slot].st(cy, cx, q);
    Pol::recover(U1, prm, q, flags);
    sm.q[slot].st(cy, cx + 1, q);
  };
  auto load_plane = [&](int z) {
    const int slot = ring_slot(z);
    const long long zo = plane_offset(z);
    for (int c = NT - 1 - tid; c < QNP; c += NT) {
      S U0[5], U1[5];
      fetch_pair(zo, c, U0, U1);
      store_pair(slot, c, U0, U1);
    }
  };
  // Float arithmetic: phase 2 issues the next plane's loads into registers before its face fluxes
  // and recovers them after, so the load latency overlaps the fluxes (8-byte arithmetic has no
  // registers to spare for it).
  constexpr bool kPrefetch = std::is_same<R, float>::value;
  constexpr int NPF = kPrefetch ? (QNP + NT - 1) / NT : 1;
  S pre0[NPF][5], pre1[NPF][5];
  auto fetch_plane = [&](int z) {
    const long long zo = plane_offset(z);
#pragma unroll
    for (int k = 0; k < NPF; ++k) {
      const int c = NT - 1 - tid + k * NT;
      if (c < QNP) fetch_pair(zo, c, pre0[k], pre1[k]);
    }
  };
  auto commit_plane = [&](int z) {
    const int slot = ring_slot(z);
#pragma unroll
    for (int k = 0; k < NPF; ++k) {
      const int c = NT - 1 - tid + k * NT;
      if (c < QNP) store_pair(slot, c, pre0[k], pre1[k]);
    }
  };
  constexpr bool kCompact = std::is_same<R, df>::value;  // double-float arithmetic

  const R hdt = (R)(0.5 * dt / P.dx);
  const R dtdx = (R)(dt / P.dx);
  const int gx = x0 + ti, gy = y0 + tj;
  const bool own = (gx < P.nx) && (gy < P.ny);
  const R gamma = kc<R>(prm, K_GAMMA);

  // Carried across planes: the lower z state of the next face, the flux through the lower z face of
  // the plane awaiting its update, and the warp's running maximum of the sure CFL speed estimates.
  constexpr bool kEstimate = std::is_same<R, double>::value;
  float thr = 0.f;
  R LzPrev[5], FzPrev[5], Fz[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) { LzPrev[v] = FzPrev[v] = Fz[v] = R(0); }

  auto z_faces = [&](int p, const R qh[5], const R dqz[5]) {
    R Lz[5], Rz[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      Lz[v] = qh[v] + half_(dqz[v]);
      Rz[v] = qh[v] - half_(dqz[v]);
    }
    floor_state(Lz, kc<R>(prm, K_RHOF), kc<R>(prm, K_PF));
    floor_state(Rz, kc<R>(prm, K_RHOF), kc<R>(prm, K_PF));
    if (p >= z0) hllc<2>(LzPrev, Rz, gamma, kc<R>(prm, K_IGM1), Fz);
#pragma unroll
    for (int v = 0; v < 5; ++v) LzPrev[v] = Lz[v];
  };
  // Update of plane k = p-1 by this column: the x and y flux differences of plane k (written to
  // shared memory by the previous plane's phase 2) and its two z fluxes.
  auto update = [&](int k) {
    R xp[5], xm[5], yp[5], ym[5], dF[5];
    sm.fx.ld(tj, ti + 1, xp);
    sm.fx.ld(tj, ti, xm);
    sm.fy.ld(tj + 1, ti, yp);
    sm.fy.ld(tj, ti, ym);
#pragma unroll
    for (int v = 0; v < 5; ++v) dF[v] = (xp[v] - xm[v]) + (yp[v] - ym[v]);
    // the updated cell of this column, written to the output; false where the column lies outside
    // the patch (or, in the bounds-checked build, an index lies outside its array)
    auto write_cell = [&](S Un[5]) -> bool {
      if (!own) return false;
      const long long ai = (long long)(k + P.gin) * P.isz + (long long)(gy + P.gin) * P.isy + (gx + P.gin);
      const long long ao = (long long)(k + P.gout) * P.osz + (long long)(gy + P.gout) * P.osy + (gx + P.gout);
      if (!index_ok(ai, in_extent, flags) || !index_ok(ao, (long long)(P.nz + 2 * P.gout) * P.osz, flags)) return false;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const R div = (dF[v] - FzPrev[v]) + Fz[v];
        Un[v] = Pol::update(__ldg(P.in[v] + ai), dtdx, div);
        P.out[v][ao] = Un[v];
      }
      return true;
    };
    S Un[5];
    if constexpr (!kEstimate) {
      if (write_cell(Un) && want_cfl) {
        const R sp = Pol::speed(Un, prm, flags);
        smax = sp > smax ? sp : smax;
      }
    } else {
      bool have = write_cell(Un);
      if (!want_cfl) return;
      // CFL maximum of the updated cells.  In double arithmetic the exact speed occupies the narrow
      // FP64 pipe: every cell first takes the float estimate speed_estimate (FP32 and integer
      // pipes), the warp keeps the running maximum T of the estimates it is sure of, and only cells
      // whose estimate is unsure or at least 0.99 T take the exact speed.  The cell with the tile's
      // largest exact speed always does (its estimate is at least 0.999 of that speed, T at most
      // 1.001 of it), so the maximum, the dt and the flags are those of taking every cell's exact
      // speed.  (+6.5% for the FP64 step at 512^3; the double-float step, whose exact speed runs on
      // the FP32 pipes like the estimate, lost 4.7% with it.)
      float se = 0.f;
      bool sure = true;
      if (have) sure = speed_estimate(Un, prm, se);
      float w = sure ? se : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) w = fmaxf(w, __shfl_xor_sync(0xffffffffu, w, o));
      thr = fmaxf(thr, w);
      if (have && (!sure || se >= 0.99f * thr)) {
        const R sp = Pol::speed(Un, prm, flags);
        smax = sp > smax ? sp : smax;
      }
    }
  };
  auto ring_cell = [&](int r, int& ci, int& cj) {
    if (r < TX) { ci = r; cj = -1; }
    else if (r < 2 * TX) { ci = r - TX; cj = TY; }
    else if (r < 2 * TX + TY) { ci = -1; cj = r - 2 * TX; }
    else { ci = TX; cj = r - 2 * TX - TY; }
  };
  constexpr int NR = 2 * (TX + TY);  // ring cells
  constexpr int NXF = (TX + 1) * TY, NYF = TX * (TY + 1);
  // Double-float: the ring cells go to the last RW warps (whole warps, for the split barriers);
  // NIX + NIY faces lie between two tile cells.  The split barriers pay where a block is alone on
  // its SM (512 threads, or the one-block-per-SM build): with two resident blocks the other block
  // already fills the barrier waits, and interleaving the predictor with the faces costs more
  // (measured at 16x16: 37.0 vs 31.7 ms per 512^3 step; at 32x16: 31.5 vs 32.7 ms).
  constexpr bool kSplit = kCompact && min_blocks<Pol, NT, MINB>() == 1;
  constexpr int RW = (NR + 31) / 32, NTI = kSplit ? NT - 32 * RW : NT - NR;
  constexpr int NIX = (TX - 1) * TY, NIF = NIX + TX * (TY - 1);
  const bool ringw = tid >= NTI;

  load_plane(z0 - 2);
  load_plane(z0 - 1);
  load_plane(z0);
  __syncthreads();
  // Per plane p, two phases separated by barriers:
  //   1  predict plane p (tile; its ring when its x/y faces are needed), the z face p-1/2 of each
  //      column, and the update of plane p-1 (x/y flux differences from shared memory)
  //   2  the x/y faces of plane p, and the load + recovery of plane p+2 into the ring slot that
  //      plane p-1 held
  for (int p = z0 - 1; p <= z1; ++p) {
    const int sm1 = ring_slot(p - 1), s0 = ring_slot(p), sp1 = ring_slot(p + 1);
    const bool xy = p >= z0 && p < z1;
    const bool upd = p >= z0 + 1;
    // ---- phase 1
    if constexpr (kCompact) {
      // One call site each for the predictor and the x/y face flux: double-float code is large
      // enough that several inlined copies overflow the instruction cache.  The ring cells go to
      // the last RW warps, which signal barrier 1 as soon as their tile cells are predicted and
      // predict their ring cells while the other warps go on to the interior faces.
      for (int it = 0; it < 2; ++it) {
        int ci = ti, cj = tj;
        if (it == 1) {
          if (!xy || !ringw || (kSplit && tid - NTI >= NR)) break;
          ring_cell(tid - NTI, ci, cj);
        }
        R qh[5], dqz[5];
        predict_cell<LIM>(sm, ci, cj, sm1, s0, sp1, prm, hdt, qh, dqz);
        if (it == 0) {
          z_faces(p, qh, dqz);
          if (upd) update(p - 1);
          if (kSplit && xy && ringw) bar_arrive(1, NT);
        }
      }
    } else {
      {
        R qh[5], dqz[5];
        predict_cell<LIM>(sm, ti, tj, sm1, s0, sp1, prm, hdt, qh, dqz);
        z_faces(p, qh, dqz);
      }
      if (upd) update(p - 1);
      if (xy && tid >= NT - NR) {
        int ci, cj;
        ring_cell(tid - (NT - NR), ci, cj);
        R qh[5], dqz[5];
        predict_cell<LIM>(sm, ci, cj, sm1, s0, sp1, prm, hdt, qh, dqz);
      }
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) FzPrev[v] = Fz[v];
    const bool ld2 = p + 2 <= z1 + 1;
    if (kSplit && xy) {
      // Split barriers.  Barrier 1: every tile cell predicted (the ring warps arrive before their
      // ring cells); barrier 2: the ring warps wait for it through the other warps' arrivals;
      // barrier 3: the ring cells predicted, so that plane p-1's slot may be overwritten.
      if (ringw) {
        bar_arrive(3, NT);
        bar_sync(2, NT);
      } else {
        bar_sync(1, NT);
        bar_arrive(2, NT);
      }
      // ---- phase 2, double-float: the other warps take the faces between two tile cells, each
      // ring thread the face between its ring cell and the tile (one call site for all of them)
      const int r = tid - NTI;
      int f = ringw ? NIF + r : tid;
      const int fend = ringw ? NIF + NR : NIF;
      const int fstep = ringw ? NR : NTI;
      for (; f < fend; f += fstep) {
        int d, i, j;
        if (f < NIX) { d = 0; i = f % (TX - 1); j = f / (TX - 1); }
        else if (f < NIF) { d = 1; i = (f - NIX) % TX; j = (f - NIX) / TX; }
        else {
          int ci, cj;
          ring_cell(f - NIF, ci, cj);
          d = (cj == -1 || cj == TY) ? 1 : 0;
          i = d == 0 ? (ci < 0 ? -1 : TX - 1) : ci;
          j = d == 1 ? (cj < 0 ? -1 : TY - 1) : cj;
        }
        R F[5];
        face_flux_dyn(sm, d, i, j, prm, F);
        if (d == 0) sm.fx.st(j, i + 1, F);
        else sm.fy.st(j + 1, i, F);
      }
      // plane p+2 (an x/y plane is never the last one: p + 2 <= z1 + 1) into plane p-1's slot by
      // the other warps, after barrier 3 (every thread of those warps syncs on it once per x/y
      // plane, completing the ring warps' arrival)
      if (!ringw) {
        bar_sync(3, NT);
        const int slot = ring_slot(p + 2);
        const long long zo = plane_offset(p + 2);
        for (int c = NTI - 1 - tid; ld2 && c < QNP; c += NTI) {
          S U0[5], U1[5];
          fetch_pair(zo, c, U0, U1);
          store_pair(slot, c, U0, U1);
        }
      }
      __syncthreads();
      continue;
    }
    __syncthreads();
    // ---- phase 2
    if (kPrefetch && ld2) fetch_plane(p + 2);
    if (xy) {
      if constexpr (kCompact) {
        for (int f = tid; f < NXF + NYF; f += NT) {
          int d, i, j;
          if (f < NXF) { d = 0; i = f % (TX + 1) - 1; j = f / (TX + 1); }
          else { d = 1; i = (f - NXF) % TX; j = (f - NXF) / TX - 1; }
          R F[5];
          face_flux_dyn(sm, d, i, j, prm, F);
          if (d == 0) sm.fx.st(j, i + 1, F);
          else sm.fy.st(j + 1, i, F);
        }
      } else {
        // the x face on this column's right and the y face above it; the first warps also take
        // the faces on the tile's left and bottom edges
        R F[5];
        face_flux<0>(sm, ti, tj, prm, F);
        sm.fx.st(tj, ti + 1, F);
        face_flux<1>(sm, ti, tj, prm, F);
        sm.fy.st(tj + 1, ti, F);
        if (tid < TY) {
          face_flux<0>(sm, -1, tid, prm, F);
          sm.fx.st(tid, 0, F);
        } else if (tid >= 32 && tid < 32 + TX) {
          face_flux<1>(sm, tid - 32, -1, prm, F);
          sm.fy.st(0, tid - 32, F);
        }
      }
    }
    if (ld2) {
      if constexpr (kPrefetch) commit_plane(p + 2);
      else load_plane(p + 2);
    }
    __syncthreads();
  }
}

// Block-wide maximum of v (all threads call); the result is valid in thread 0.
template <class Pol, int TX, int TY>
__device__ __forceinline__ typename Pol::R block_max(TileShared<Pol, TX, TY>& sm, typename Pol::R v) {
  using R = typename Pol::R;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    R w = shfl_xor_(v, o);
    v = w > v ? w : v;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sm.red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < TX * TY / 32; ++w) v = sm.red[w] > v ? sm.red[w] : v;
  }
  return v;
}

__device__ __forceinline__ void flush_flags(unsigned flags, unsigned* err) {
  const unsigned f = __reduce_or_sync(0xffffffffu, flags);
  if ((threadIdx.x & 31) == 0 && f) atomicOr(err, f);
}

// dt of a tile from its largest speed; folded into the patch's slot by an order-preserving min.
__device__ __forceinline__ void publish_dt(double cfl, double dx, double smax, double* slot) {
  if (smax > 0.0) {
    const double dt = cfl * (dx / smax);
    atomicMin(reinterpret_cast<unsigned long long*>(slot), dkey(dt));
  }
}

// ------------------------------------------------------------------ kernels
// Uniform grid: one tile per block, tiles from the block index.
template <class Pol, int TX, int TY, int MINB, int LIM>
__global__ void __launch_bounds__(TX* TY, (min_blocks<Pol, TX * TY, MINB>())) k_step_uniform(PatchIO<typename Pol::S> P, Params prm, const double* dt_dev,
                                                         double* dt_next, int zchunk, unsigned* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& sm = *reinterpret_cast<TileShared<Pol, TX, TY>*>(smem_raw);
  const double dt = dt_dev[0];
  if (!(dt > 0.0 && dt <= 1e300)) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) atomicOr(err, HYDRO_EBIT_BAD_DT);
    return;
  }
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * zchunk;
  const int z1 = min(z0 + zchunk, P.nz);
  unsigned flags = 0;
  typename Pol::R smax = 0;
  step_tile<LIM, MINB>(sm, P, x0, y0, z0, z1, prm, dt, dt_next != nullptr, flags, smax);
  if (dt_next) {
    const auto m = block_max(sm, smax);
    if (threadIdx.x == 0) publish_dt(prm.cfl, P.dx, (double)m, dt_next);
  }
  flush_flags(flags, err);
}

// Batched patches: a persistent grid pulls tiles from the work-list through an atomic counter.
template <class Pol, int TX, int TY, int MINB, int LIM>
__global__ void __launch_bounds__(TX* TY, (min_blocks<Pol, TX * TY, MINB>())) k_step_batched(const PatchIO<typename Pol::S>* patches, const TileRec* tiles,
                                                         int ntiles, int* counter, Params prm, const double* dt_dev,
                                                         double* dt_next, int zchunk, unsigned* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& sm = *reinterpret_cast<TileShared<Pol, TX, TY>*>(smem_raw);
  unsigned flags = 0;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) sm.tile = atomicAdd(counter, 1);
    __syncthreads();
    const int t = sm.tile;
    if (t >= ntiles) break;
    const TileRec r = tiles[t];
    const PatchIO<typename Pol::S> P = patches[r.patch];
    if (r.x0 < 0 || r.y0 < 0 || r.z0 < 0 || r.x0 >= P.nx || r.y0 >= P.ny || r.z0 >= P.nz) {
      flags |= HYDRO_EBIT_BAD_TILE;
      continue;
    }
    const double dt = dt_dev[r.patch];
    if (!(dt > 0.0 && dt <= 1e300)) {
      flags |= HYDRO_EBIT_BAD_DT;
      continue;
    }
    const int z1 = min(r.z0 + zchunk, P.nz);
    typename Pol::R smax = 0;
    step_tile<LIM, MINB>(sm, P, r.x0, r.y0, r.z0, z1, prm, dt, dt_next != nullptr, flags, smax);
    if (dt_next) {
      const auto m = block_max(sm, smax);
      if (threadIdx.x == 0) publish_dt(prm.cfl, P.dx, (double)m, dt_next + r.patch);
    }
  }
  flush_flags(flags, err);
}

}  // namespace hydro
