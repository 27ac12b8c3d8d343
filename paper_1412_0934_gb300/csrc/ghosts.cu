// Ghost cells of AMR patches.
// Coarse-to-fine ghost fill, refinement ratio 2 (the paper's Ramses GPU procedure
// builds chunks of patches whose boundary cells are interpolated from the coarser level, Sec. 3):
// conservative piecewise-linear prolongation of each conserved variable, MinMod-limited slopes.
// A fine cell with fine-level index f lies in coarse cell floor(f/2) (wrapped on the periodic
// coarse level), on its upper half when f is odd:
//     U_f = U_C + s_x D_x + s_y D_y + s_z D_z,  s_d = +-1/4,  D_d = minmod(U_C - U_{C-e_d}, U_{C+e_d} - U_C).
// One thread per ghost cell; each block takes up to 256 consecutive ghost cells of one patch (a
// block table built on the host: patch and first ghost index per block); the arithmetic is in
// the storage type.  The coarse level may be taken at a fraction theta of its step, linear in time
// between its states before and after the step (a finer level subcycles inside the coarse step:
// the paper's time refinement, Sec. 2).
#include <cuda_runtime.h>

#include "hydro_device.cuh"
#include "internal.h"

namespace hydro {

template <class S>
__device__ __forceinline__ S minmod_s(S a, S b) {
  if (prod_nonpos(a, b)) return S(0);
  return abs_le(a, b) ? a : b;
}

// One thread per coarse cell under a patch's ghost shell: it forms the cell's three limited
// slopes once and its eight children as ((U_C +- D_x/4) +- D_y/4) +- D_z/4 -- the two x partial
// sums, then four, then eight (the same operations in the same order as child by child, so the
// same bits) -- and writes the children that are ghost cells of the patch.  Coarse cells whose
// children are all interior return at once.  Each block takes up to 256 coarse cells of one patch
// (a block table built on the host).
// Coarse value at element a: the state after the coarse step, or with Blend the state at a
// fraction of the step, w0 U_old + w1 U_new with each product and the sum rounded once (no FMA).
__device__ __forceinline__ double blend_rn(double w0, double a, double w1, double b) {
  return __dadd_rn(__dmul_rn(w0, a), __dmul_rn(w1, b));
}
__device__ __forceinline__ float blend_rn(float w0, float a, float w1, float b) {
  return __fadd_rn(__fmul_rn(w0, a), __fmul_rn(w1, b));
}

template <class S, bool Blend>
__global__ void __launch_bounds__(256) k_fill_ghosts(const HostGhostPatch* patches, const int2* blocks,
                                                     HostPatchIO coarse, HostPatchIO coarse_old, S w0, S w1) {
  const int2 b = blocks[blockIdx.x];      // (patch, first coarse cell of this block)
  const HostGhostPatch P = patches[b.x];  // by value: the stores below cannot alias it
  const int t = b.y + threadIdx.x;
  const int ncell = P.cm[0] * P.cm[1] * P.cm[2];
  if (t >= ncell) return;
  const int cz = t / (P.cm[0] * P.cm[1]), r = t - cz * P.cm[0] * P.cm[1], cy = r / P.cm[0], cx = r - cy * P.cm[0];
  const int cc[3] = {P.clo[0] + cx, P.clo[1] + cy, P.clo[2] + cz};
  const int n[3] = {P.nx, P.ny, P.nz}, o[3] = {P.ox, P.oy, P.oz};
  // local ghosted index of child h (0, 1) along d, and whether it is in the box / in the interior
  int l[3][2];
  bool inb[3][2], inr[3][2];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      l[d][h] = 2 * cc[d] + h - (o[d] - 2);
      inb[d][h] = l[d][h] >= 0 && l[d][h] < n[d] + 4;
      inr[d][h] = l[d][h] >= 2 && l[d][h] < n[d] + 2;
    }
  bool any = false;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int hx = k & 1, hy = (k >> 1) & 1, hz = k >> 2;
    any |= inb[0][hx] && inb[1][hy] && inb[2][hz] && !(inr[0][hx] && inr[1][hy] && inr[2][hz]);
  }
  if (!any) return;
  const int nc[3] = {coarse.nx, coarse.ny, coarse.nz};
  int c[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int q = cc[d] % nc[d];
    c[d] = q < 0 ? q + nc[d] : q;
  }
  const long long a0 = c[2] * coarse.isz + c[1] * coarse.isy + c[0];
  const long long st[3] = {1, coarse.isy, coarse.isz};
  long long am[3], ap[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    am[d] = a0 + (c[d] == 0 ? (long long)(nc[d] - 1) * st[d] : -st[d]);
    ap[d] = a0 + (c[d] == nc[d] - 1 ? -(long long)(nc[d] - 1) * st[d] : st[d]);
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const S* U = static_cast<const S*>(coarse.in[v]);
    const S* Uo = static_cast<const S*>(coarse_old.in[v]);
    auto at = [&](long long a) { return Blend ? blend_rn(w0, __ldg(Uo + a), w1, __ldg(U + a)) : __ldg(U + a); };
    const S u0 = at(a0);
    S D[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) D[d] = minmod_s(u0 - at(am[d]), at(ap[d]) - u0);
    S ax[2], ay[4], az[8];
#pragma unroll
    for (int hx = 0; hx < 2; ++hx) ax[hx] = u0 + (hx ? S(0.25) : S(-0.25)) * D[0];
#pragma unroll
    for (int k = 0; k < 4; ++k) ay[k] = ax[k & 1] + ((k >> 1) ? S(0.25) : S(-0.25)) * D[1];
#pragma unroll
    for (int k = 0; k < 8; ++k) az[k] = ay[k & 3] + ((k >> 2) ? S(0.25) : S(-0.25)) * D[2];
    S* out = static_cast<S*>(P.U[v]);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int hx = k & 1, hy = (k >> 1) & 1, hz = k >> 2;
      if (inb[0][hx] && inb[1][hy] && inb[2][hz] && !(inr[0][hx] && inr[1][hy] && inr[2][hz]))
        out[(long long)l[2][hz] * P.sz + (long long)l[1][hy] * P.sy + l[0][hx]] = az[k];
    }
  }
}

// Same-level exchange: one block per copy task (a box of a source patch's interior into a box of a
// destination patch's ghost shell), threads over the box's cells, five fields each.
template <class S>
__global__ void __launch_bounds__(256) k_copy_boxes(const HostGhostPatch* patches, const HostCopyTask* tasks) {
  const HostCopyTask t = tasks[blockIdx.x];
  const HostGhostPatch D = patches[t.dst], Sp = patches[t.src];  // by value: the stores cannot alias them
  const int nxy = t.n[0] * t.n[1], total = nxy * t.n[2];
  for (int c = threadIdx.x; c < total; c += blockDim.x) {
    const int z = c / nxy, r = c - z * nxy, y = r / t.n[0], x = r - y * t.n[0];
    const long long d = (long long)(t.dlo[2] + z) * D.sz + (long long)(t.dlo[1] + y) * D.sy + (t.dlo[0] + x);
    const long long s = (long long)(t.slo[2] + z) * Sp.sz + (long long)(t.slo[1] + y) * Sp.sy + (t.slo[0] + x);
#pragma unroll
    for (int v = 0; v < 5; ++v) static_cast<S*>(D.U[v])[d] = static_cast<const S*>(Sp.U[v])[s];
  }
}

cudaError_t launch_copy_boxes(int elem_size, const HostGhostPatch* d_patches, const HostCopyTask* d_tasks, int ntasks,
                              cudaStream_t s) {
  if (elem_size == 4)
    k_copy_boxes<float><<<ntasks, 256, 0, s>>>(d_patches, d_tasks);
  else
    k_copy_boxes<double><<<ntasks, 256, 0, s>>>(d_patches, d_tasks);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ refluxing and average-down
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

// Faces of one kind (t = 2d + side: d the normal axis, side 0 the box's lower face) of every box:
// the coarse cell outside the box across the face gets s/dx (Rc - mean of the 4 fine faces' Rf),
// s = +1 on the lower side, -1 on the upper.  Boxes of a level do not overlap, so the cells one
// launch writes are distinct; the six kinds run in turn, so the result is deterministic.  The
// products and sums are kept unfused (explicitly rounded) in the order written.
template <class S>
__global__ void __launch_bounds__(256) k_reflux(const HostRefluxBox* boxes, const int2* blocks, int t, HostPatchIO coarse) {
  const int2 b = blocks[blockIdx.x];
  const HostRefluxBox B = boxes[b.x];
  const int d = t >> 1, side = t & 1;
  const int a1 = d == 0 ? 1 : 0, a2 = d == 2 ? 1 : 2;  // the face's (col, row) axes: x faces [k][j], y [k][i], z [j][i]
  const int ncol = B.n[a1], nrow = B.n[a2];
  const int f = b.y * 256 + threadIdx.x;
  if (f >= ncol * nrow) return;
  const int row = f / ncol, col = f - row * ncol;
  // register offsets: x-low, x-high [nz][ny]; y-low, y-high [nz][nx]; z-low, z-high [ny][nx]
  const long long nx = B.n[0], ny = B.n[1], nz = B.n[2];
  const long long base_c[3] = {0, 2 * ny * nz, 2 * ny * nz + 2 * nx * nz};
  const long long size_c[3] = {ny * nz, nx * nz, nx * ny};
  const long long RC = 2 * (ny * nz + nx * nz + nx * ny), RF = 4 * RC;
  const long long fcol = 2 * ncol;
  const long long base_f[3] = {0, 8 * ny * nz, 8 * ny * nz + 8 * nx * nz};
  const long long size_f[3] = {4 * ny * nz, 4 * nx * nz, 4 * nx * ny};
  const long long ic = base_c[d] + side * size_c[d] + (long long)row * ncol + col;
  const long long if0 = base_f[d] + side * size_f[d] + (long long)(2 * row) * fcol + 2 * col;
  int cell[3];
  cell[a1] = B.o[a1] + col;
  cell[a2] = B.o[a2] + row;
  cell[d] = side ? B.o[d] + B.n[d] : B.o[d] - 1;
  const int N[3] = {coarse.nx, coarse.ny, coarse.nz};
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    cell[e] %= N[e];
    cell[e] += cell[e] < 0 ? N[e] : 0;
  }
  const long long a = (long long)cell[2] * coarse.isz + (long long)cell[1] * coarse.isy + cell[0];
  const S sdx = (S)((side ? -1.0 : 1.0) / B.dx);
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const S* Rc = static_cast<const S*>(B.rc) + v * RC;
    const S* Rf = static_cast<const S*>(B.rf) + v * RF;
    const S p = Rf[if0], q = Rf[if0 + fcol], r = Rf[if0 + 1], u = Rf[if0 + fcol + 1];
    const S avg = mul_rn(S(0.25), add_rn(add_rn(add_rn(p, q), r), u));
    S* U = static_cast<S*>(coarse.out[v]);
    U[a] = add_rn(U[a], mul_rn(sdx, add_rn(Rc[ic], -avg)));
  }
}

// Coarse cells under a fine patch's interior (origin even, sizes even) <- mean of their children.
template <class S>
__global__ void __launch_bounds__(256) k_average_down(const HostGhostPatch* patches, const int2* blocks,
                                                      HostPatchIO coarse) {
  const int2 b = blocks[blockIdx.x];
  const HostGhostPatch P = patches[b.x];
  const int mx = P.nx / 2, my = P.ny / 2, mz = P.nz / 2;
  const int c = b.y * 256 + threadIdx.x;
  if (c >= mx * my * mz) return;
  const int cz = c / (mx * my), r = c - cz * mx * my, cy = r / mx, cx = r - cy * mx;
  int g[3] = {P.ox / 2 + cx, P.oy / 2 + cy, P.oz / 2 + cz};
  const int N[3] = {coarse.nx, coarse.ny, coarse.nz};
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    g[e] %= N[e];
    g[e] += g[e] < 0 ? N[e] : 0;
  }
  const long long a = (long long)g[2] * coarse.isz + (long long)g[1] * coarse.isy + g[0];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const S* F = static_cast<const S*>(P.U[v]);
    S sum = S(0);
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      const int x = 2 * cx + (h & 1) + 2, y = 2 * cy + ((h >> 1) & 1) + 2, z = 2 * cz + (h >> 2) + 2;
      sum = add_rn(sum, F[(long long)z * P.sz + (long long)y * P.sy + x]);
    }
    static_cast<S*>(coarse.out[v])[a] = mul_rn(S(0.125), sum);
  }
}

cudaError_t launch_reflux(int elem_size, const HostRefluxBox* d_boxes, const int2* const d_blocks[6],
                          const int nblocks[6], const HostPatchIO& coarse, cudaStream_t s) {
  for (int t = 0; t < 6; ++t) {
    if (nblocks[t] == 0) continue;
    if (elem_size == 4)
      k_reflux<float><<<nblocks[t], 256, 0, s>>>(d_boxes, d_blocks[t], t, coarse);
    else
      k_reflux<double><<<nblocks[t], 256, 0, s>>>(d_boxes, d_blocks[t], t, coarse);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_average_down(int elem_size, const HostGhostPatch* d_patches, const int2* d_blocks, int nblocks,
                                const HostPatchIO& coarse, cudaStream_t s) {
  if (elem_size == 4)
    k_average_down<float><<<nblocks, 256, 0, s>>>(d_patches, d_blocks, coarse);
  else
    k_average_down<double><<<nblocks, 256, 0, s>>>(d_patches, d_blocks, coarse);
  return cudaGetLastError();
}

cudaError_t launch_fill_ghosts(int elem_size, const HostGhostPatch* d_patches, const int2* d_blocks, int nblocks,
                               const HostPatchIO& coarse, const HostPatchIO* coarse_old, double theta,
                               cudaStream_t s) {
  const double w0 = 1.0 - theta, w1 = theta;
  const HostPatchIO& old = coarse_old ? *coarse_old : coarse;
  if (elem_size == 4) {
    if (coarse_old)
      k_fill_ghosts<float, true><<<nblocks, 256, 0, s>>>(d_patches, d_blocks, coarse, old, (float)w0, (float)w1);
    else
      k_fill_ghosts<float, false><<<nblocks, 256, 0, s>>>(d_patches, d_blocks, coarse, old, 0.f, 1.f);
  } else {
    if (coarse_old)
      k_fill_ghosts<double, true><<<nblocks, 256, 0, s>>>(d_patches, d_blocks, coarse, old, w0, w1);
    else
      k_fill_ghosts<double, false><<<nblocks, 256, 0, s>>>(d_patches, d_blocks, coarse, old, 0.0, 1.0);
  }
  return cudaGetLastError();
}

}  // namespace hydro
