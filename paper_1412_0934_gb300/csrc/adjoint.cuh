// Adjoint of one periodic MUSCL-Hancock/HLLC step with dt held fixed:
//   lam_n = lam_np1 + (dU^{n+1}/dU^n - I)^T lam_np1.
// Two kernels, both deterministic (every contribution is gathered, none atomically scattered):
//  k_adj_faces  z-marching tile: recomputes recovery, slopes and predictor in shared memory; for
//               every face, lamF = dt/dx (lam_{right} - lam_{left}) is pulled back through HLLC,
//               the floors and the face states onto the two cells' predicted states and slopes;
//               then each cell's predictor is reversed.  Writes per cell the adjoint of q from the
//               predictor, the adjoints of its three slopes and the limiter branch codes.
//  k_adj_cells  per cell: gathers the slope adjoints of the cell and its six neighbours through the
//               recorded branches, reverses the recovery, adds lam_np1.
#pragma once
#include <type_traits>

#include "adjoint_device.cuh"
#include "internal.h"
#include "step_tile.cuh"

namespace hydro {

template <class Pol>
PatchIO<typename Pol::S> to_dev(const HostPatchIO& h) {
  static_assert(sizeof(PatchIO<typename Pol::S>) == sizeof(HostPatchIO), "layout");
  PatchIO<typename Pol::S> d;
  for (int v = 0; v < 5; ++v) {
    d.in[v] = static_cast<const typename Pol::S*>(h.in[v]);
    d.out[v] = static_cast<typename Pol::S*>(h.out[v]);
  }
  d.nx = h.nx; d.ny = h.ny; d.nz = h.nz; d.gin = h.gin; d.gout = h.gout;
  d.isy = h.isy; d.isz = h.isz; d.osy = h.osy; d.osz = h.osz; d.dx = h.dx;
  return d;
}

template <class R, int TX, int TY>
struct AdjShared {
  R q[3][5][TY + 4][TX + 4];  // primitive planes k, k+1, k+2
  R qh[2][5][TY + 2][TX + 2];  // predicted planes k, k+1 (tile + ring)
  R sx[2][5][TY + 2][TX + 2];
  R sy[2][5][TY + 2][TX + 2];
  R sz[2][5][TY][TX];           // z slopes (interior)
  R lam[2][5][TY + 2][TX + 2];  // lam_np1 planes k, k+1 (tile + ring)
  R axL[5][TY][TX + 1], axR[5][TY][TX + 1];  // x faces: adjoint of the left / right face state
  R ayL[5][TY + 1][TX], ayR[5][TY + 1][TX];
  long long yoff[TY + 4];
  int xoff[TX + 4];
};

template <class R>
struct AdjScratch {
  R* lq;           // [5][N] adjoint of q from the predictor (identity included)
  R* ld;           // [15][N] adjoint of the slopes, index d*5+v
  unsigned* code;  // [N] limiter branch codes, 2 bits per (d, v)
};

template <class Pol, int TX, int TY, int LIM>
__device__ __forceinline__ void adj_predict(AdjShared<typename Pol::R, TX, TY>& sm, int i, int j, int sq0, int sq1,
                                            int sq2, int sp, bool interior, const Params& prm, typename Pol::R hdt,
                                            unsigned& code) {
  using R = typename Pol::R;
  const int ci = i + 2, cj = j + 2;
  R q0[5], dqx[5], dqy[5], dqz[5], qh[5];
  code = 0;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const R c = sm.q[sq1][v][cj][ci];
    unsigned cx, cy, cz;
    q0[v] = c;
    dqx[v] = limited_code(c - sm.q[sq1][v][cj][ci - 1], sm.q[sq1][v][cj][ci + 1] - c, LIM, cx);
    dqy[v] = limited_code(c - sm.q[sq1][v][cj - 1][ci], sm.q[sq1][v][cj + 1][ci] - c, LIM, cy);
    dqz[v] = limited_code(c - sm.q[sq0][v][cj][ci], sm.q[sq2][v][cj][ci] - c, LIM, cz);
    code |= (cx << (2 * v)) | (cy << (2 * (5 + v))) | (cz << (2 * (10 + v)));
  }
  hancock(q0, dqx, dqy, dqz, kc<R>(prm, K_GAMMA), hdt, qh);
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    sm.qh[sp][v][j + 1][i + 1] = qh[v];
    sm.sx[sp][v][j + 1][i + 1] = dqx[v];
    sm.sy[sp][v][j + 1][i + 1] = dqy[v];
    if (interior) sm.sz[sp][v][j][i] = dqz[v];
  }
}

// Adjoint of the face between (i, j) and its +D neighbour in plane slot sp (D = 0 x, 1 y).
template <int D, class Pol, int TX, int TY>
__device__ __forceinline__ void adj_face_xy(AdjShared<typename Pol::R, TX, TY>& sm, int i, int j, int sp,
                                            const Params& prm, typename Pol::R dtdx, typename Pol::R lL[5],
                                            typename Pol::R lR[5]) {
  using R = typename Pol::R;
  const int li = i + 1, lj = j + 1;
  const int ri = li + (D == 0), rj = lj + (D == 1);
  R pL[5], pR[5], qL[5], qR[5], lF[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const R sL = (D == 0) ? sm.sx[sp][v][lj][li] : sm.sy[sp][v][lj][li];
    const R sR = (D == 0) ? sm.sx[sp][v][rj][ri] : sm.sy[sp][v][rj][ri];
    pL[v] = sm.qh[sp][v][lj][li] + half_(sL);
    pR[v] = sm.qh[sp][v][rj][ri] - half_(sR);
    qL[v] = pL[v];
    qR[v] = pR[v];
    lF[v] = dtdx * (sm.lam[sp][v][rj][ri] - sm.lam[sp][v][lj][li]);
    lL[v] = R(0);
    lR[v] = R(0);
  }
  const R rf = kc<R>(prm, K_RHOF), pf = kc<R>(prm, K_PF);
  floor_state(qL, rf, pf);
  floor_state(qR, rf, pf);
  hllc_adj<D>(qL, qR, kc<R>(prm, K_GAMMA), kc<R>(prm, K_IGM1), lF, lL, lR);
  floor_mask(pL, lL, rf, pf);
  floor_mask(pR, lR, rf, pf);
}

// LIM: the PLM limiter, fixed at compile time (one kernel per limiter; prm.limiter is the same value).
template <class Pol, int TX, int TY, int LIM>
__global__ void __launch_bounds__(TX* TY) k_adj_faces(PatchIO<typename Pol::S> P, PatchIO<typename Pol::S> L,
                                                      Params prm, const double* dt_dev, int zchunk,
                                                      AdjScratch<typename Pol::R> scr, unsigned* err) {
  using S = typename Pol::S;
  using R = typename Pol::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& sm = *reinterpret_cast<AdjShared<R, TX, TY>*>(smem_raw);
  constexpr int NT = TX * TY;
  constexpr int QW = TX + 4, QH = TY + 4, QN = QW * QH;
  constexpr int EW = TX + 2, EN = (TX + 2) * (TY + 2);
  const int tid = threadIdx.x, ti = tid % TX, tj = tid / TX;
  const double dt = dt_dev[0];
  if (!(dt > 0.0 && dt <= 1e300)) {
    if (tid == 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) atomicOr(err, HYDRO_EBIT_BAD_DT);
    return;
  }
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * zchunk;
  const int z1 = min(z0 + zchunk, P.nz);
  const R hdt = (R)(0.5 * dt / P.dx), dtdx = (R)(dt / P.dx);
  const R gamma = kc<R>(prm, K_GAMMA), igm1 = kc<R>(prm, K_IGM1);
  const R rf = kc<R>(prm, K_RHOF), pf = kc<R>(prm, K_PF);
  unsigned flags = 0;
  for (int c = tid; c < QW; c += NT) sm.xoff[c] = wrapi(x0 - 2 + c, P.nx);
  for (int c = tid; c < QH; c += NT) sm.yoff[c] = (long long)wrapi(y0 - 2 + c, P.ny) * P.isy;
  __syncthreads();
  auto load_q = [&](int z) {
    const int slot = ring_slot(z);
    const long long zo = (long long)wrapi(z, P.nz) * P.isz;
    for (int c = tid; c < QN; c += NT) {
      const int cy = c / QW, cx = c - cy * QW;
      const long long a = zo + sm.yoff[cy] + sm.xoff[cx];
      S U[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) U[v] = __ldg(P.in[v] + a);
      R q[5];
      Pol::recover(U, prm, q, flags);
#pragma unroll
      for (int v = 0; v < 5; ++v) sm.q[slot][v][cy][cx] = q[v];
    }
  };
  auto load_lam = [&](int z) {
    const int slot = (z + 2) & 1;
    const long long zo = (long long)wrapi(z, L.nz) * L.isz;
    for (int c = tid; c < EN; c += NT) {
      const int cy = c / EW, cx = c - cy * EW;
      const long long a = zo + (long long)wrapi(y0 - 1 + cy, L.ny) * L.isy + sm.xoff[cx + 1];
#pragma unroll
      for (int v = 0; v < 5; ++v) sm.lam[slot][v][cy][cx] = (R)__ldg(L.in[v] + a);
    }
  };
  // predict plane z into slot (z+2)&1 over the tile and its ring (codes of the interior cell)
  auto predict = [&](int z, unsigned& code_interior) {
    const int sp = (z + 2) & 1;
    const int s0 = ring_slot(z - 1), s1 = ring_slot(z), s2 = ring_slot(z + 1);
    adj_predict<Pol, TX, TY, LIM>(sm, ti, tj, s0, s1, s2, sp, true, prm, hdt, code_interior);
    if (tid < 2 * (TX + TY)) {
      int ri, rj;
      const int r = tid;
      if (r < TX) { ri = r; rj = -1; }
      else if (r < 2 * TX) { ri = r - TX; rj = TY; }
      else if (r < 2 * TX + TY) { ri = -1; rj = r - 2 * TX; }
      else { ri = TX; rj = r - 2 * TX - TY; }
      unsigned dummy;
      adj_predict<Pol, TX, TY, LIM>(sm, ri, rj, s0, s1, s2, sp, false, prm, hdt, dummy);
    }
  };

  const int gx = x0 + ti, gy = y0 + tj;
  const bool own = gx < P.nx && gy < P.ny;
  const long long N = (long long)P.nx * P.ny * P.nz;
  R lRz[5] = {0, 0, 0, 0, 0};  // adjoint of the right state of face k - 1/2 (belongs to cell k)
  unsigned code_k = 0, code_next = 0;

  load_q(z0 - 2);
  load_q(z0 - 1);
  load_q(z0);
  load_lam(z0 - 1);
  __syncthreads();
  predict(z0 - 1, code_k);
  __syncthreads();
  for (int k = z0 - 1; k < z1; ++k) {
    // ---- A: plane k+2 of q, plane k+1 of lam
    load_q(k + 2);
    load_lam(k + 1);
    __syncthreads();
    // ---- B: predict plane k+1
    predict(k + 1, code_next);
    __syncthreads();
    const int pk = (k + 2) & 1, pk1 = (k + 3) & 1;
    // ---- C: z face k+1/2 (interior); x and y faces of plane k
    R lLz[5];
    {
      R pL[5], pR[5], qL[5], qR[5], lF[5], lL[5], lRn[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        pL[v] = sm.qh[pk][v][tj + 1][ti + 1] + half_(sm.sz[pk][v][tj][ti]);
        pR[v] = sm.qh[pk1][v][tj + 1][ti + 1] - half_(sm.sz[pk1][v][tj][ti]);
        qL[v] = pL[v];
        qR[v] = pR[v];
        lF[v] = dtdx * (sm.lam[pk1][v][tj + 1][ti + 1] - sm.lam[pk][v][tj + 1][ti + 1]);
        lL[v] = R(0);
        lRn[v] = R(0);
      }
      floor_state(qL, rf, pf);
      floor_state(qR, rf, pf);
      hllc_adj<2>(qL, qR, gamma, igm1, lF, lL, lRn);
      floor_mask(pL, lL, rf, pf);
      floor_mask(pR, lRn, rf, pf);
#pragma unroll
      for (int v = 0; v < 5; ++v) lLz[v] = lL[v];
      if (k >= z0) {
        R a[5], b[5];
        adj_face_xy<0, Pol, TX, TY>(sm, ti, tj, pk, prm, dtdx, a, b);
#pragma unroll
        for (int v = 0; v < 5; ++v) { sm.axL[v][tj][ti + 1] = a[v]; sm.axR[v][tj][ti + 1] = b[v]; }
        adj_face_xy<1, Pol, TX, TY>(sm, ti, tj, pk, prm, dtdx, a, b);
#pragma unroll
        for (int v = 0; v < 5; ++v) { sm.ayL[v][tj + 1][ti] = a[v]; sm.ayR[v][tj + 1][ti] = b[v]; }
        if (tid < TY) {
          adj_face_xy<0, Pol, TX, TY>(sm, -1, tid, pk, prm, dtdx, a, b);
#pragma unroll
          for (int v = 0; v < 5; ++v) { sm.axL[v][tid][0] = a[v]; sm.axR[v][tid][0] = b[v]; }
        } else if (tid >= 32 && tid < 32 + TX) {
          adj_face_xy<1, Pol, TX, TY>(sm, tid - 32, -1, pk, prm, dtdx, a, b);
#pragma unroll
          for (int v = 0; v < 5; ++v) { sm.ayL[v][0][tid - 32] = a[v]; sm.ayR[v][0][tid - 32] = b[v]; }
        }
      }
      __syncthreads();
      // ---- D: finalize cell (ti, tj, k)
      if (k >= z0 && own) {
        R lqh[5], ldq[3][5], q0[5], dq[3][5], lq[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const R xl = sm.axL[v][tj][ti + 1], xr = sm.axR[v][tj][ti];
          const R yl = sm.ayL[v][tj + 1][ti], yr = sm.ayR[v][tj][ti];
          lqh[v] = ((xl + xr) + (yl + yr)) + (lLz[v] + lRz[v]);
          ldq[0][v] = half_(xl - xr);
          ldq[1][v] = half_(yl - yr);
          ldq[2][v] = half_(lLz[v] - lRz[v]);
          q0[v] = sm.q[ring_slot(k)][v][tj + 2][ti + 2];
          dq[0][v] = sm.sx[pk][v][tj + 1][ti + 1];
          dq[1][v] = sm.sy[pk][v][tj + 1][ti + 1];
          dq[2][v] = sm.sz[pk][v][tj][ti];
          lq[v] = R(0);
        }
        hancock_adj(q0, dq, gamma, hdt, lqh, lq, ldq);
        const long long cidx = ((long long)k * P.ny + gy) * P.nx + gx;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          scr.lq[v * N + cidx] = lq[v];
          scr.ld[(0 * 5 + v) * N + cidx] = ldq[0][v];
          scr.ld[(1 * 5 + v) * N + cidx] = ldq[1][v];
          scr.ld[(2 * 5 + v) * N + cidx] = ldq[2][v];
        }
        scr.code[cidx] = code_k;
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) lRz[v] = lRn[v];
      code_k = code_next;
    }
    __syncthreads();
  }
  flush_flags(flags, err);
}

// Per cell: lam_n = lam_np1 + recover^T(lq_pred + slope gathers).  One thread per cell of a
// 32 x 8 x 1 block over (x, y, z): indices from the grid, periodic neighbours by one compare each.
template <class Pol, int LIM>
__global__ void __launch_bounds__(256) k_adj_cells(PatchIO<typename Pol::S> P, PatchIO<typename Pol::S> L,
                                                   Params prm, AdjScratch<typename Pol::R> scr,
                                                   typename Pol::S* o0, typename Pol::S* o1, typename Pol::S* o2,
                                                   typename Pol::S* o3, typename Pol::S* o4, int out_g,
                                                   long long osy, long long osz) {
  using S = typename Pol::S;
  using R = typename Pol::R;
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
  if (i >= P.nx || j >= P.ny) return;
  S* outp[5] = {o0, o1, o2, o3, o4};
  const long long nx = P.nx, nxy = nx * P.ny, N = nxy * P.nz;
  const long long c = k * nxy + j * nx + i;
  const long long nb[3][2] = {{c + (i == 0 ? nx - 1 : -1), c + (i == P.nx - 1 ? 1 - nx : 1)},
                              {c + (j == 0 ? nxy - nx : -nx), c + (j == P.ny - 1 ? nx - nxy : nx)},
                              {c + (k == 0 ? N - nxy : -nxy), c + (k == P.nz - 1 ? nxy - N : nxy)}};
  const unsigned cc = scr.code[c];
  R lq[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) lq[v] = scr.lq[v * N + c];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const unsigned cm = scr.code[nb[d][0]], cp = scr.code[nb[d][1]];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const int sh = 2 * (5 * d + v);
      float a0, b0, am, bm, ap, bp;
      code_weights((cc >> sh) & 3u, LIM, a0, b0);
      code_weights((cm >> sh) & 3u, LIM, am, bm);
      code_weights((cp >> sh) & 3u, LIM, ap, bp);
      const R* ld = scr.ld + (long long)(5 * d + v) * N;
      lq[v] += (mulf_(ld[c], a0 - b0) + mulf_(ld[nb[d][0]], bm)) - mulf_(ld[nb[d][1]], ap);
    }
  }
  const long long a = (long long)k * P.isz + (long long)j * P.isy + i;
  const long long la = (long long)k * L.isz + (long long)j * L.isy + i;
  R U[5], lU[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) U[v] = R(P.in[v][a]);
  recover_adj(U, prm, lq, lU);
  const long long o = (long long)(k + out_g) * osz + (long long)(j + out_g) * osy + (i + out_g);
#pragma unroll
  for (int v = 0; v < 5; ++v) outp[v][o] = (S)(R(L.in[v][la]) + lU[v]);
}

template <class Pol>
struct AdjTile;
template <>
struct AdjTile<PolF64> {
  static constexpr int TX = 8, TY = 8;
};
template <>
struct AdjTile<PolF32> {
  static constexpr int TX = 16, TY = 8;
};
template <>
struct AdjTile<PolMixed> {
  static constexpr int TX = 16, TY = 8;
};

template <class Pol>
size_t adjoint_scratch_bytes(int nx, int ny, int nz) {
  const size_t N = (size_t)nx * ny * nz;
  return N * 20 * sizeof(typename Pol::R) + N * sizeof(unsigned) + 256;
}

template <class Pol, int LIM>
cudaError_t launch_adjoint_t(const HostPatchIO& U, const HostPatchIO& lam, void* const lam_out[5], const Params& prm,
                             const double* dt, void* scratch, size_t scratch_bytes, unsigned* err, cudaStream_t s) {
  using R = typename Pol::R;
  using S = typename Pol::S;
  constexpr int TX = AdjTile<Pol>::TX, TY = AdjTile<Pol>::TY;
  if (scratch_bytes < adjoint_scratch_bytes<Pol>(U.nx, U.ny, U.nz)) return cudaErrorInvalidValue;
  const size_t N = (size_t)U.nx * U.ny * U.nz;
  AdjScratch<R> scr;
  scr.lq = static_cast<R*>(scratch);
  scr.ld = scr.lq + 5 * N;
  scr.code = reinterpret_cast<unsigned*>(scr.ld + 15 * N);
  const size_t smem = sizeof(AdjShared<R, TX, TY>);
  static PerDeviceOnce attr;
  cudaError_t ea = attr.call([&] {
    return cudaFuncSetAttribute(k_adj_faces<Pol, TX, TY, LIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (ea != cudaSuccess) return ea;
  // z chunk: FP32 takes the longest of 16, 8, 4, 2 planes whose grid still fills half of the SMs'
  // resident blocks (a small grid leaves SMs idle, a short march repeats halo planes; half is the
  // measured balance).  FP64 keeps 16: it is bound by the FP64 pipe, which a few warps per SM
  // already keep busy (8-plane chunks that fill every resident slot measured 3% slower at 64^3).
  static int resident = 0;
  if (!resident) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_adj_faces<Pol, TX, TY, LIM>, TX * TY,
                                                                  smem);
    if (e != cudaSuccess) return e;
    if (resident < 1) resident = 1;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return cudaErrorUnknown;
  const long long cols = (long long)((U.nx + TX - 1) / TX) * ((U.ny + TY - 1) / TY);
  int zc = 16;
  while (!std::is_same<R, double>::value && zc > 2 && 2 * cols * ((U.nz + zc - 1) / zc) < (long long)resident * sms)
    zc /= 2;
  if (zc > U.nz) zc = U.nz;
  dim3 grid((U.nx + TX - 1) / TX, (U.ny + TY - 1) / TY, (U.nz + zc - 1) / zc);
  k_adj_faces<Pol, TX, TY, LIM><<<grid, TX * TY, smem, s>>>(to_dev<Pol>(U), to_dev<Pol>(lam), prm, dt, zc, scr, err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const dim3 cgrid((U.nx + 31) / 32, (U.ny + 7) / 8, U.nz);
  k_adj_cells<Pol, LIM><<<cgrid, dim3(32, 8), 0, s>>>(to_dev<Pol>(U), to_dev<Pol>(lam), prm, scr,
                                                         (S*)lam_out[0], (S*)lam_out[1], (S*)lam_out[2],
                                                         (S*)lam_out[3], (S*)lam_out[4], lam.gout, lam.osy, lam.osz);
  return cudaGetLastError();
}

template <class Pol>
cudaError_t launch_adjoint(const HostPatchIO& U, const HostPatchIO& lam, void* const lam_out[5], const Params& prm,
                           const double* dt, void* scratch, size_t scratch_bytes, unsigned* err, cudaStream_t s) {
  if constexpr (std::is_same<Pol, PolMixed>::value || std::is_same<Pol, PolDF>::value) {
    return cudaErrorNotSupported;  // the adjoint kernels are FP64 and FP32 (double-float uses FP64's)
  } else {
    switch (prm.limiter) {
      case HYDRO_MINMOD: return launch_adjoint_t<Pol, HYDRO_MINMOD>(U, lam, lam_out, prm, dt, scratch, scratch_bytes, err, s);
      case HYDRO_MC: return launch_adjoint_t<Pol, HYDRO_MC>(U, lam, lam_out, prm, dt, scratch, scratch_bytes, err, s);
      case HYDRO_NOLIMIT: return launch_adjoint_t<Pol, HYDRO_NOLIMIT>(U, lam, lam_out, prm, dt, scratch, scratch_bytes, err, s);
    }
    return cudaErrorInvalidValue;
  }
}

}  // namespace hydro
