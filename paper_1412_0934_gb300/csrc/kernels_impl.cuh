// Kernels and launchers of one precision policy POL (included once per policy by kernels_*.cu):
// the step kernels of step_tile.cuh for every compiled tile shape, the PPM step of step_ppm.cuh,
// the standalone CFL dt
// reduction, the oct-group step, the primitive->conservative map and its adjoint, and the
// adjoint step (adjoint.cuh).
#pragma once
#include "adjoint.cuh"
#include "internal.h"
#include "step_ppm.cuh"
#include "step_tile.cuh"

namespace hydro {

// ------------------------------------------------------------------ step launchers
// The step kernels are compiled once per PLM limiter (LIM: HYDRO_MINMOD, HYDRO_MC, HYDRO_NOLIMIT).

template <class Pol, int TX, int TY, int MINB, int LIM>
cudaError_t launch_uniform_t(const HostPatchIO& P, const Params& prm, const double* dt, double* dt_next, int zchunk,
                             unsigned* err, cudaStream_t s) {
  const size_t smem = sizeof(TileShared<Pol, TX, TY>);
  static PerDeviceOnce attr;
  cudaError_t e = attr.call([&] {
    return cudaFuncSetAttribute(k_step_uniform<Pol, TX, TY, MINB, LIM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
  });
  if (e != cudaSuccess) return e;
  dim3 grid((P.nx + TX - 1) / TX, (P.ny + TY - 1) / TY, (P.nz + zchunk - 1) / zchunk);
  k_step_uniform<Pol, TX, TY, MINB, LIM><<<grid, TX * TY, smem, s>>>(to_dev<Pol>(P), prm, dt, dt_next, zchunk, err);
  return cudaGetLastError();
}

template <class Pol, int TX, int TY, int MINB, int LIM>
cudaError_t launch_batched_t(const HostPatchIO* d_patches, const HostTileRec* d_tiles, int ntiles, int* d_counter,
                             const Params& prm, const double* dt, double* dt_next, int zchunk, unsigned* err, int grid,
                             cudaStream_t s) {
  const size_t smem = sizeof(TileShared<Pol, TX, TY>);
  static PerDeviceOnce attr;
  cudaError_t e = attr.call([&] {
    return cudaFuncSetAttribute(k_step_batched<Pol, TX, TY, MINB, LIM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
  });
  if (e != cudaSuccess) return e;
  k_step_batched<Pol, TX, TY, MINB, LIM><<<grid, TX * TY, smem, s>>>(
      reinterpret_cast<const PatchIO<typename Pol::S>*>(d_patches), reinterpret_cast<const TileRec*>(d_tiles), ntiles,
      d_counter, prm, dt, dt_next, zchunk, err);
  return cudaGetLastError();
}

template <class Pol, int TX, int TY, int MINB, int LIM>
int blocks_per_sm_t() {
  const size_t smem = sizeof(TileShared<Pol, TX, TY>);
  cudaFuncSetAttribute(k_step_batched<Pol, TX, TY, MINB, LIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_batched<Pol, TX, TY, MINB, LIM>, TX * TY, smem) !=
      cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

// Tile id -> compiled shape, and the limiter -> compiled variant.
#define HYDRO_LIM_SWITCH(T, lim, CALL)                     \
  (lim == HYDRO_MINMOD ? CALL(T, HYDRO_MINMOD)             \
                       : lim == HYDRO_MC ? CALL(T, HYDRO_MC) : CALL(T, HYDRO_NOLIMIT))
#define HYDRO_TILE_SWITCH(tile, lim, CALL)                    \
  switch (tile) {                                             \
    case 0: return HYDRO_LIM_SWITCH(0, lim, CALL);           \
    case 1: return HYDRO_LIM_SWITCH(1, lim, CALL);           \
    case 2: return HYDRO_LIM_SWITCH(2, lim, CALL);           \
    case 3: return HYDRO_LIM_SWITCH(3, lim, CALL);           \
    case 4: return HYDRO_LIM_SWITCH(4, lim, CALL);           \
  }

template <class Pol>
cudaError_t launch_uniform(int tile, const HostPatchIO& P, const Params& prm, const double* dt, double* dt_next,
                           int zchunk, unsigned* err, cudaStream_t s) {
#define HYDRO_CALL(T, L) launch_uniform_t<Pol, kTileX[T], kTileY[T], kTileMinBlocks[T], L>(P, prm, dt, dt_next, zchunk, err, s)
  HYDRO_TILE_SWITCH(tile, prm.limiter, HYDRO_CALL)
#undef HYDRO_CALL
  return cudaErrorInvalidValue;
}

template <class Pol>
cudaError_t launch_batched(int tile, const HostPatchIO* d_patches, const HostTileRec* d_tiles, int ntiles,
                           int* d_counter, const Params& prm, const double* dt, double* dt_next, int zchunk,
                           unsigned* err, int grid, cudaStream_t s) {
#define HYDRO_CALL(T, L)                                                                                          \
  launch_batched_t<Pol, kTileX[T], kTileY[T], kTileMinBlocks[T], L>(d_patches, d_tiles, ntiles, d_counter, prm, dt, \
                                                                    dt_next, zchunk, err, grid, s)
  HYDRO_TILE_SWITCH(tile, prm.limiter, HYDRO_CALL)
#undef HYDRO_CALL
  return cudaErrorInvalidValue;
}

template <class Pol>
int batched_blocks_per_sm(int tile, int limiter) {
#define HYDRO_CALL(T, L) blocks_per_sm_t<Pol, kTileX[T], kTileY[T], kTileMinBlocks[T], L>()
  HYDRO_TILE_SWITCH(tile, limiter, HYDRO_CALL)
#undef HYDRO_CALL
  return 1;
}
#undef HYDRO_TILE_SWITCH
#undef HYDRO_LIM_SWITCH

// ------------------------------------------------------------------ CFL dt (standalone)
// blockIdx.y walks the patches, blockIdx.x the interior cells of one patch.  The per-block
// largest speed is reduced by warp shuffles and shared memory and folded into the patch's dt
// slot exactly as the step's fused epilogue does, so both give the same bits.
template <class Pol>
__global__ void __launch_bounds__(256) k_cfl(const PatchIO<typename Pol::S>* patches, PatchIO<typename Pol::S> single,
                                             int npatch, Params prm, double* dt_out, unsigned* err) {
  using S = typename Pol::S;
  using R = typename Pol::R;
  __shared__ R red[8];
  unsigned flags = 0;
  for (int pi = blockIdx.y; pi < npatch; pi += gridDim.y) {
    const PatchIO<S> P = patches ? patches[pi] : single;
    // cells by (row, x): rows = (z, y) pairs, one 32-bit division per row (64-bit integer division
    // is a long sequence that runs partly on the FP64 pipe)
    const int rows = P.ny * P.nz;
    R smax = 0;
    const int nxb = (P.nx + 31) / 32;  // 32-wide segments per row
    for (long long s = (long long)blockIdx.x * 8 + (threadIdx.x >> 5); s < (long long)rows * nxb;
         s += (long long)gridDim.x * 8) {
      const int row = (int)(s / nxb), i = (int)(s - (long long)row * nxb) * 32 + (threadIdx.x & 31);
      if (i >= P.nx) continue;
      const int k = row / P.ny, j = row - k * P.ny;
      const long long a = (long long)(k + P.gin) * P.isz + (long long)(j + P.gin) * P.isy + (i + P.gin);
      S U[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) U[v] = __ldg(P.in[v] + a);
      const R sp = Pol::speed(U, prm, flags);
      smax = sp > smax ? sp : smax;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      R w = shfl_xor_(smax, o);
      smax = w > smax ? w : smax;
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = smax;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < 8; ++w) smax = red[w] > smax ? red[w] : smax;
      publish_dt(prm.cfl, P.dx, (double)smax, dt_out + pi);
    }
  }
  flush_flags(flags, err);
}

template <class Pol>
cudaError_t launch_cfl(const HostPatchIO* d_patches, const HostPatchIO& single, int npatch, const Params& prm,
                       double* dt_out, unsigned* err, cudaStream_t s) {
  long long maxcells = (long long)single.nx * single.ny * single.nz;
  int gx;
  if (d_patches) {
    gx = 64;  // patches up to a few 10^5 cells
  } else {
    long long b = (maxcells + 256 * 4 - 1) / (256 * 4);
    gx = (int)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
  }
  dim3 grid(gx, npatch < 65535 ? npatch : 65535);
  k_cfl<Pol><<<grid, 256, 0, s>>>(reinterpret_cast<const PatchIO<typename Pol::S>*>(d_patches), to_dev<Pol>(single),
                                  npatch, prm, dt_out, err);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ oct groups
// One warp per group.  The 80 cells of the 6^3 stencil that the step reads are recovered into
// shared memory; the 32 cells next to the oct's faces (the oct and the 24 outside neighbours
// across its faces) are predicted; the 36 faces of the oct get HLLC fluxes; 8 lanes update the
// oct.  Local coordinates run from -2 to 3 (stored at +2).
__device__ __forceinline__ bool oct_needed(int x, int y, int z) {
  const int ox = (x < 0 || x > 1), oy = (y < 0 || y > 1), oz = (z < 0 || z > 1);
  const int nout = ox + oy + oz;
  const bool far = (x == -2 || x == 3 || y == -2 || y == 3 || z == -2 || z == 3);
  return nout <= 1 || (nout == 2 && !far);
}
// Coordinates of predicted cell e (0..31): 0..7 the oct, 8..31 the face neighbours.
__device__ __forceinline__ void oct_ecell(int e, int& x, int& y, int& z) {
  if (e < 8) { x = e & 1; y = (e >> 1) & 1; z = (e >> 2) & 1; return; }
  const int r = e - 8, f = r >> 2, a = r & 1, b = (r >> 1) & 1;
  const int out = (f & 1) ? 2 : -1;
  const int d = f >> 1;
  x = d == 0 ? out : a;
  y = d == 1 ? out : (d == 0 ? a : b);
  z = d == 2 ? out : b;
}
__device__ __forceinline__ int oct_eindex(int x, int y, int z) {
  const bool ix = (x == 0 || x == 1), iy = (y == 0 || y == 1), iz = (z == 0 || z == 1);
  if (ix && iy && iz) return x + 2 * y + 4 * z;
  int d, c, a, b;
  if (!ix) { d = 0; c = x; a = y; b = z; }
  else if (!iy) { d = 1; c = y; a = x; b = z; }
  else { d = 2; c = z; a = x; b = y; }
  const int f = 2 * d + (c == 2 ? 1 : 0);
  return 8 + 4 * f + a + 2 * b;
}

constexpr int kOctWarps = 4;

template <class Pol>
struct OctSmem {
  using R = typename Pol::R;
  R q[kOctWarps][5][216];
  R qh[kOctWarps][5][32];
  R sl[kOctWarps][3][5][32];
  R f[kOctWarps][5][36];
  short need[80];
};

// Where a group's 6^3 stencil comes from and where its 8 cells go.  OctGathered: the caller's
// gathered buffer, group g's cell c (z, y, x from -2) at g*216 + c.  OctLevel: a periodic level
// grid and the groups' origins (the oct's lowest cell, x, y, z), wrapped on the fly -- no gathered
// copy of the stencils.  Both write group g's cells at g*8 .. g*8+7.  OctTable: octs stored
// oct-major (cell (i, j, k) of oct o at o*8 + (k*2 + j)*2 + i) with their neighbour table; group g
// steps oct list[g] and writes it in place of that oct.
template <class S>
struct OctGathered {
  const S* f[5];
  __device__ __forceinline__ bool begin(long long, unsigned&) const { return true; }
  __device__ __forceinline__ long long cell(long long g, int c) const { return g * 216 + c; }
  __device__ __forceinline__ long long out_cell(long long g, int e) const { return g * 8 + e; }
};
template <class S>
struct OctLevel {
  const S* f[5];
  int nx, ny, nz;
  long long sy, sz;
  const int* origins;  // [ngroups][3]
  int ox, oy, oz;      // origin of the current group
  // Loads group g's origin; an origin outside the grid flags HYDRO_EBIT_BAD_TILE and the group
  // is skipped (nothing is read or written for it).
  __device__ __forceinline__ bool begin(long long g, unsigned& flags) {
    ox = __ldg(origins + 3 * g);
    oy = __ldg(origins + 3 * g + 1);
    oz = __ldg(origins + 3 * g + 2);
    if (ox < 0 || oy < 0 || oz < 0 || ox >= nx || oy >= ny || oz >= nz) {
      flags |= HYDRO_EBIT_BAD_TILE;
      return false;
    }
    return true;
  }
  __device__ __forceinline__ long long cell(long long, int c) const {
    int x = ox + c % 6 - 2, y = oy + (c / 6) % 6 - 2, z = oz + c / 36 - 2;
    x += x < 0 ? nx : (x >= nx ? -nx : 0);
    y += y < 0 ? ny : (y >= ny ? -ny : 0);
    z += z < 0 ? nz : (z >= nz ? -nz : 0);
    return z * sz + y * sy + x;
  }
  __device__ __forceinline__ long long out_cell(long long g, int e) const { return g * 8 + e; }
};
template <class S>
struct OctTable {
  const S* f[5];
  const int* nbr;   // [noct][27]: oct at offset (dx, dy, dz) in entry ((dz+1)*3 + dy+1)*3 + dx+1
  const int* list;  // [ngroups]: the octs to step
  int noct;
  int oct;          // the current group's oct
  // Loads group g's oct and checks it and its 27 neighbour entries (one per lane, warp-wide):
  // an index outside [0, noct) flags HYDRO_EBIT_BAD_TILE and the group is skipped.
  __device__ __forceinline__ bool begin(long long g, unsigned& flags) {
    oct = __ldg(list + g);
    bool bad = (unsigned)oct >= (unsigned)noct;
    const int lane = threadIdx.x & 31;
    if (!bad && lane < 27) bad = (unsigned)__ldg(nbr + 27LL * oct + lane) >= (unsigned)noct;
    if (__any_sync(0xffffffffu, bad)) {
      flags |= HYDRO_EBIT_BAD_TILE;
      return false;
    }
    return true;
  }
  // Stencil cell (x, y, z), each 0..5, is cell (x%2, y%2, z%2) of neighbour (x/2, y/2, z/2).
  __device__ __forceinline__ long long cell(long long, int c) const {
    const int x = c % 6, y = (c / 6) % 6, z = c / 36;
    const int n = __ldg(nbr + 27LL * oct + ((z >> 1) * 3 + (y >> 1)) * 3 + (x >> 1));
    return 8LL * n + ((z & 1) * 2 + (y & 1)) * 2 + (x & 1);
  }
  __device__ __forceinline__ long long out_cell(long long, int e) const { return 8LL * oct + e; }
};

// Resident blocks per SM: six (24 warps) for float arithmetic, measured fastest against the
// register budget of the prefetched next group; four for 8-byte arithmetic, whose larger
// registers would otherwise spill.
template <class Pol>
constexpr int oct_min_blocks() { return sizeof(typename Pol::R) >= 8 ? 4 : 6; }

template <class Pol, class Src>
__global__ void __launch_bounds__(32 * kOctWarps, oct_min_blocks<Pol>()) k_octs(Src src, typename Pol::S* o0, typename Pol::S* o1,
                                                         typename Pol::S* o2, typename Pol::S* o3,
                                                         typename Pol::S* o4, long long ngroups, double dx, Params prm,
                                                         const double* dt_dev, unsigned* err) {
  using S = typename Pol::S;
  using R = typename Pol::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& sm = *reinterpret_cast<OctSmem<Pol>*>(smem_raw);
  S* gout[5] = {o0, o1, o2, o3, o4};
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    int n = 0;
    for (int c = 0; c < 216; ++c) {
      const int x = c % 6 - 2, y = (c / 6) % 6 - 2, z = c / 36 - 2;
      if (oct_needed(x, y, z)) sm.need[n++] = (short)c;
    }
  }
  __syncthreads();
  const double dt = dt_dev[0];
  if (!(dt > 0.0 && dt <= 1e300)) {
    if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(err, HYDRO_EBIT_BAD_DT);
    return;
  }
  const R hdt = (R)(0.5 * dt / dx);
  const R dtdx = (R)(dt / dx);
  const R gamma = kc<R>(prm, K_GAMMA), igm1 = kc<R>(prm, K_IGM1);
  const R rf = kc<R>(prm, K_RHOF), pf = kc<R>(prm, K_PF);
  unsigned flags = 0;
  // The needed cells of the next group are loaded into registers while this group is computed.
  const long long gstride = (long long)gridDim.x * kOctWarps;
  S pre[3][5];
  Src nxt = src;  // source state of the prefetched group
  bool nxt_ok = false;
  auto fetch = [&](long long g) {
    nxt_ok = nxt.begin(g, flags);
    if (!nxt_ok) return;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const int k = lane + 32 * t;
      if (k < 80) {
        const long long a = nxt.cell(g, sm.need[k]);
#pragma unroll
        for (int v = 0; v < 5; ++v) pre[t][v] = __ldg(nxt.f[v] + a);
      }
    }
  };
  long long g = (long long)blockIdx.x * kOctWarps + w;
  if (g < ngroups) fetch(g);
  for (; g < ngroups; g += gstride) {
    const Src cur = nxt;
    const bool ok = nxt_ok;
    if (!ok) {  // (warp-uniform: one warp per group)
      if (g + gstride < ngroups) fetch(g + gstride);
      continue;
    }
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const int k = lane + 32 * t;
      if (k < 80) {
        R q[5];
        Pol::recover(pre[t], prm, q, flags);
        const int c = sm.need[k];
#pragma unroll
        for (int v = 0; v < 5; ++v) sm.q[w][v][c] = q[v];
      }
    }
    if (g + gstride < ngroups) fetch(g + gstride);
    __syncwarp();
    {
      int x, y, z;
      oct_ecell(lane, x, y, z);
      const int c = (z + 2) * 36 + (y + 2) * 6 + (x + 2);
      R q0[5], dqx[5], dqy[5], dqz[5], qh[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const R* Q = sm.q[w][v];
        const R cc = Q[c];
        q0[v] = cc;
        dqx[v] = limited(cc - Q[c - 1], Q[c + 1] - cc, prm.limiter);
        dqy[v] = limited(cc - Q[c - 6], Q[c + 6] - cc, prm.limiter);
        dqz[v] = limited(cc - Q[c - 36], Q[c + 36] - cc, prm.limiter);
      }
      hancock(q0, dqx, dqy, dqz, gamma, hdt, qh);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        sm.qh[w][v][lane] = qh[v];
        sm.sl[w][0][v][lane] = dqx[v];
        sm.sl[w][1][v][lane] = dqy[v];
        sm.sl[w][2][v][lane] = dqz[v];
      }
    }
    __syncwarp();
    for (int fi = lane; fi < 36; fi += 32) {
      const int d = fi / 12, m = fi % 12, s = m >> 2, a = m & 1, b = (m >> 1) & 1;
      // face between cells at coordinate s-1 and s along d; (a, b) the transverse coordinates
      int lx, ly, lz;
      if (d == 0) { lx = s - 1; ly = a; lz = b; }
      else if (d == 1) { lx = a; ly = s - 1; lz = b; }
      else { lx = a; ly = b; lz = s - 1; }
      const int eL = oct_eindex(lx, ly, lz);
      const int eR = oct_eindex(lx + (d == 0), ly + (d == 1), lz + (d == 2));
      R qL[5], qR[5], F[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        qL[v] = sm.qh[w][v][eL] + half_(sm.sl[w][d][v][eL]);
        qR[v] = sm.qh[w][v][eR] - half_(sm.sl[w][d][v][eR]);
      }
      floor_state(qL, rf, pf);
      floor_state(qR, rf, pf);
      hllc_dyn(d, qL, qR, gamma, igm1, F);
#pragma unroll
      for (int v = 0; v < 5; ++v) sm.f[w][v][fi] = F[v];
    }
    __syncwarp();
    if (lane < 8) {
      const int x = lane & 1, y = (lane >> 1) & 1, z = (lane >> 2) & 1;
      const int c = (z + 2) * 36 + (y + 2) * 6 + (x + 2);
      const int fxm = 0 * 12 + (x * 4 + y + 2 * z), fxp = fxm + 4;
      const int fym = 1 * 12 + (y * 4 + x + 2 * z), fyp = fym + 4;
      const int fzm = 2 * 12 + (z * 4 + x + 2 * y), fzp = fzm + 4;
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const R* F = sm.f[w][v];
        const R div = ((F[fxp] - F[fxm]) + (F[fyp] - F[fym])) + (F[fzp] - F[fzm]);
        gout[v][cur.out_cell(g, lane)] = Pol::update(__ldg(cur.f[v] + cur.cell(g, c)), dtdx, div);
      }
    }
    __syncwarp();
  }
  flush_flags(flags, err);
}

template <class Pol, class Src>
cudaError_t launch_octs_src(const Src& src, void* const out[5], long long ngroups, double dx, const Params& prm,
                            const double* dt, unsigned* err, cudaStream_t s) {
  using S = typename Pol::S;
  const size_t smem = sizeof(OctSmem<Pol>);
  static PerDeviceOnce attr;
  cudaError_t e = attr.call(
      [&] { return cudaFuncSetAttribute(k_octs<Pol, Src>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); });
  if (e != cudaSuccess) return e;
  long long blocks = (ngroups + kOctWarps - 1) / kOctWarps;
  const long long cap = 152LL * 64;
  if (blocks > cap) blocks = cap;
  k_octs<Pol, Src><<<(unsigned)blocks, 32 * kOctWarps, smem, s>>>(src, (S*)out[0], (S*)out[1], (S*)out[2], (S*)out[3],
                                                                   (S*)out[4], ngroups, dx, prm, dt, err);
  return cudaGetLastError();
}

template <class Pol>
cudaError_t launch_octs(void* const gathered[5], void* const out[5], long long ngroups, double dx, const Params& prm,
                        const double* dt, unsigned* err, cudaStream_t s) {
  using S = typename Pol::S;
  OctGathered<S> src;
  for (int v = 0; v < 5; ++v) src.f[v] = static_cast<const S*>(gathered[v]);
  return launch_octs_src<Pol>(src, out, ngroups, dx, prm, dt, err, s);
}

template <class Pol>
cudaError_t launch_octs_level(const HostPatchIO& level, const int* origins, void* const out[5], long long ngroups,
                              const Params& prm, const double* dt, unsigned* err, cudaStream_t s) {
  using S = typename Pol::S;
  OctLevel<S> src;
  for (int v = 0; v < 5; ++v) src.f[v] = static_cast<const S*>(level.in[v]);
  src.nx = level.nx; src.ny = level.ny; src.nz = level.nz;
  src.sy = level.isy; src.sz = level.isz;
  src.origins = origins;
  src.ox = src.oy = src.oz = 0;
  return launch_octs_src<Pol>(src, out, ngroups, level.dx, prm, dt, err, s);
}

template <class Pol>
cudaError_t launch_octs_table(void* const in[5], const int* nbr, int noct, const int* list, void* const out[5],
                              long long ngroups, double dx, const Params& prm, const double* dt, unsigned* err,
                              cudaStream_t s) {
  using S = typename Pol::S;
  OctTable<S> src;
  for (int v = 0; v < 5; ++v) src.f[v] = static_cast<const S*>(in[v]);
  src.nbr = nbr;
  src.list = list;
  src.noct = noct;
  src.oct = 0;
  return launch_octs_src<Pol>(src, out, ngroups, dx, prm, dt, err, s);
}

// ------------------------------------------------------------------ primitive <-> conservative
// Interior cell c -> (i, j, k), in 32-bit arithmetic when the patch has fewer than 2^31 cells (a
// 64-bit integer division is a long sequence that runs partly on the FP64 pipe).
template <class S>
__device__ __forceinline__ void cell_ijk(const PatchIO<S>& P, long long c, int& i, int& j, int& k) {
  const long long nxy = (long long)P.nx * P.ny;
  if (nxy * P.nz <= 0x7fffffffLL) {
    const int cc = (int)c, nxy32 = (int)nxy;
    k = cc / nxy32;
    const int r = cc - k * nxy32;
    j = r / P.nx;
    i = r - j * P.nx;
  } else {
    k = (int)(c / nxy);
    const long long r = c - (long long)k * nxy;
    j = (int)(r / P.nx);
    i = (int)(r - (long long)j * P.nx);
  }
}
template <class S>
__device__ __forceinline__ long long cell_offset(const PatchIO<S>& P, int i, int j, int k, bool out_side) {
  const int g = out_side ? P.gout : P.gin;
  const long long sy = out_side ? P.osy : P.isy, sz = out_side ? P.osz : P.isz;
  return (long long)(k + g) * sz + (long long)(j + g) * sy + (i + g);
}

// U = (rho, rho u, rho v, rho w, p/(gamma-1) + rho |u|^2 / 2), in the storage type.
template <class S>
__global__ void k_p2c(PatchIO<S> P, double gamma) {
  const long long n = (long long)P.nx * P.ny * P.nz;
  const S igm1 = (S)(1.0 / (gamma - 1.0));
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    cell_ijk(P, c, i, j, k);
    const long long a = cell_offset(P, i, j, k, false), b = cell_offset(P, i, j, k, true);
    const S r = P.in[0][a], u = P.in[1][a], v = P.in[2][a], w = P.in[3][a], p = P.in[4][a];
    P.out[0][b] = r;
    P.out[1][b] = r * u;
    P.out[2][b] = r * v;
    P.out[3][b] = r * w;
    P.out[4][b] = p * igm1 + S(0.5) * r * ((u * u + v * v) + w * w);
  }
}

// lamW = (dU/dW)^T lamU.  W and lamU share one layout (P.in / L.in); lamW uses P.out's layout.
template <class S>
__global__ void k_p2c_adjoint(PatchIO<S> P, PatchIO<S> L, double gamma) {
  const long long n = (long long)P.nx * P.ny * P.nz;
  const S igm1 = (S)(1.0 / (gamma - 1.0));
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    cell_ijk(P, c, i, j, k);
    const long long a = cell_offset(P, i, j, k, false), la = cell_offset(L, i, j, k, false),
                    b = cell_offset(P, i, j, k, true);
    const S r = P.in[0][a], u = P.in[1][a], v = P.in[2][a], w = P.in[3][a];
    const S l0 = L.in[0][la], l1 = L.in[1][la], l2 = L.in[2][la], l3 = L.in[3][la], l4 = L.in[4][la];
    P.out[0][b] = l0 + u * l1 + v * l2 + w * l3 + S(0.5) * ((u * u + v * v) + w * w) * l4;
    P.out[1][b] = r * l1 + r * u * l4;
    P.out[2][b] = r * l2 + r * v * l4;
    P.out[3][b] = r * l3 + r * w * l4;
    P.out[4][b] = igm1 * l4;
  }
}

template <class Pol>
cudaError_t launch_p2c(const HostPatchIO& W, void* const U[5], const Params& prm, cudaStream_t s) {
  HostPatchIO h = W;
  for (int v = 0; v < 5; ++v) h.out[v] = U[v];
  k_p2c<typename Pol::S><<<152 * 8, 256, 0, s>>>(to_dev<Pol>(h), prm.gamma);
  return cudaGetLastError();
}

template <class Pol>
cudaError_t launch_p2c_adjoint(const HostPatchIO& W, const HostPatchIO& lamU, void* const lamW[5], const Params& prm,
                               cudaStream_t s) {
  HostPatchIO h = W;
  for (int v = 0; v < 5; ++v) h.out[v] = lamW[v];
  k_p2c_adjoint<typename Pol::S><<<152 * 8, 256, 0, s>>>(to_dev<Pol>(h), to_dev<Pol>(lamU), prm.gamma);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ flux registers
// Fluxes through the six boundary faces of boxes (AMR refluxing, Berger & Colella 1989: the
// coarse level's fluxes at a fine patch's boundary are replaced by the fine ones): one thread per
// face; both adjacent cells predicted from their own 3^3-minus-corners stencil exactly as the step
// does (recovery, limited slopes, Hancock predictor), face states floored, HLLC.  A box is either
// a ghosted patch's interior or a box of a periodic level.  The register (storage type, layout
// x-low [nz][ny], x-high, y-low [nz][nx], y-high, z-low [ny][nx], z-high per field) receives
// dt * F, added to its contents when accumulating (the time integral over a patch's substeps).
// Face f of a box's register (32-bit arithmetic: a box has fewer than 2^31 boundary faces).
__device__ __forceinline__ void box_face(const HostBoxFluxes& B, int f, int& d, int& i, int& j, int& k) {
  const int nx = B.n[0], ny = B.n[1], nz = B.n[2];
  const int X = ny * nz, Y = nx * nz;
  if (f < 2 * X) {
    d = 0;
    const int side = f >= X, r = f - side * X;
    k = r / ny;
    j = r - k * ny;
    i = side ? nx - 1 : -1;
  } else if (f < 2 * X + 2 * Y) {
    d = 1;
    const int g = f - 2 * X, side = g >= Y, r = g - side * Y;
    k = r / nx;
    i = r - k * nx;
    j = side ? ny - 1 : -1;
  } else {
    d = 2;
    const int g = f - 2 * X - 2 * Y, Z = nx * ny, side = g >= Z, r = g - side * Z;
    j = r / nx;
    i = r - j * nx;
    k = side ? nz - 1 : -1;
  }
}

template <class Pol>
__global__ void __launch_bounds__(256) k_box_fluxes(const HostBoxFluxes* boxes, const int2* blocks, Params prm,
                                                    const double* dt_dev, int accumulate) {
  using S = typename Pol::S;
  using R = typename Pol::R;
  const int2 b = blocks[blockIdx.x];
  const HostBoxFluxes B = boxes[b.x];
  const int nface = 2 * (B.n[1] * B.n[2] + B.n[0] * B.n[2] + B.n[0] * B.n[1]);
  const int f = b.y * 256 + threadIdx.x;
  if (f >= nface) return;
  int d, i, j, k;
  box_face(B, f, d, i, j, k);  // the face between cell (i, j, k) and its +d neighbour
  const double dt = dt_dev[B.dt_index];
  unsigned flags = 0;
  // address of cell (x, y, z) in box coordinates (interior from 0; the stencil reaches -2 .. n+1)
  auto addr = [&](int x, int y, int z) -> long long {
    if (B.periodic) {  // origin in [0, N), box no larger than N: o + x in [-2, 2N + 2)
      auto wrap = [](int v, int n) {
        v += v < 0 ? n : 0;
        v -= v >= n ? n : 0;
        return v >= n ? v - n : v;
      };
      x = wrap(x + B.o[0], B.N[0]);
      y = wrap(y + B.o[1], B.N[1]);
      z = wrap(z + B.o[2], B.N[2]);
      return (long long)z * B.sz + (long long)y * B.sy + x;
    }
    return (long long)(z + 2) * B.sz + (long long)(y + 2) * B.sy + (x + 2);
  };
  auto q_at = [&](int x, int y, int z, R q[5]) {
    const long long a = addr(x, y, z);
    S U[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) U[v] = __ldg(static_cast<const S*>(B.U[v]) + a);
    Pol::recover(U, prm, q, flags);
  };
  const R hdt = (R)(0.5 * dt / B.dx);
  R st[2][5];  // face states: left then right
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const int x = i + (side && d == 0), y = j + (side && d == 1), z = k + (side && d == 2);
    R c[5], m[5], p[5], dq[3][5], qh[5];
    q_at(x, y, z, c);
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      q_at(x - (e == 0), y - (e == 1), z - (e == 2), m);
      q_at(x + (e == 0), y + (e == 1), z + (e == 2), p);
#pragma unroll
      for (int v = 0; v < 5; ++v) dq[e][v] = limited(c[v] - m[v], p[v] - c[v], prm.limiter);
    }
    hancock(c, dq[0], dq[1], dq[2], kc<R>(prm, K_GAMMA), hdt, qh);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const R sd = d == 0 ? dq[0][v] : (d == 1 ? dq[1][v] : dq[2][v]);
      st[side][v] = side ? qh[v] - half_(sd) : qh[v] + half_(sd);
    }
  }
  floor_state(st[0], kc<R>(prm, K_RHOF), kc<R>(prm, K_PF));
  floor_state(st[1], kc<R>(prm, K_RHOF), kc<R>(prm, K_PF));
  R F[5];
  hllc_dyn(d, st[0], st[1], kc<R>(prm, K_GAMMA), kc<R>(prm, K_IGM1), F);
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    S* reg = static_cast<S*>(B.reg) + (long long)v * nface + f;
    const S add = (S)(dt * (double)F[v]);
    *reg = accumulate ? *reg + add : add;
  }
}

template <class Pol>
cudaError_t launch_box_fluxes(const HostBoxFluxes* d_boxes, const int2* d_blocks, int nblocks, const Params& prm,
                              const double* dt, int accumulate, cudaStream_t s) {
  k_box_fluxes<Pol><<<nblocks, 256, 0, s>>>(d_boxes, d_blocks, prm, dt, accumulate);
  return cudaGetLastError();
}

template <class Pol>
const KernelOps& make_ops() {
  static const KernelOps ops = {
      &launch_uniform<Pol>,      &launch_batched<Pol>,      &batched_blocks_per_sm<Pol>,
      &launch_cfl<Pol>,          &launch_octs<Pol>,         &launch_octs_level<Pol>,   &launch_octs_table<Pol>,
      &launch_adjoint<Pol>,
      &adjoint_scratch_bytes<Pol>, &launch_p2c<Pol>,        &launch_p2c_adjoint<Pol>,
      &launch_box_fluxes<Pol>,   &launch_ppm<Pol>,          &launch_ppm_batched<Pol>,
      (int)sizeof(typename Pol::S), 1};
  return ops;
}

}  // namespace hydro
