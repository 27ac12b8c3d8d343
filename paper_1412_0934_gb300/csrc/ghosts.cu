// Ghost cells of AMR patches.
// Coarse-to-fine ghost fill, refinement ratio 2 (the paper's Ramses GPU procedure
// builds chunks of patches whose boundary cells are interpolated from the coarser level, Sec. 3):
// conservative piecewise-linear prolongation of each conserved variable, MinMod-limited slopes.
// A fine cell with fine-level index f lies in coarse cell floor(f/2) (wrapped on the periodic
// coarse level), on its upper half when f is odd:
//     U_f = U_C + s_x D_x + s_y D_y + s_z D_z,  s_d = +-1/4,  D_d = minmod(U_C - U_{C-e_d}, U_{C+e_d} - U_C).
// One thread per ghost cell; each block takes up to 256 consecutive ghost cells of one patch (a
// block table built on the host: patch and first ghost index per block); the arithmetic is in
// the storage type.
#include <cuda_runtime.h>

#include "hydro_device.cuh"
#include "internal.h"

namespace hydro {

template <class S>
__device__ __forceinline__ S minmod_s(S a, S b) {
  if (prod_nonpos(a, b)) return S(0);
  return abs_le(a, b) ? a : b;
}

// Ghost cell g (0 .. ghosts-1) of a ghosted box GX x GY x GZ (interior nx x ny x nz at offset 2):
// the 4 full z planes below/above, then the 4 full y rows per interior plane, then the 4 x cells
// per interior row.
__device__ __forceinline__ void ghost_cell(int g, int nx, int ny, int nz, int& i, int& j, int& k) {
  const int GX = nx + 4, GY = ny + 4;
  const int A = 4 * GX * GY, B = 4 * nz * GX;
  if (g < A) {
    const int zi = g / (GX * GY);
    const int r = g - zi * GX * GY;
    k = zi < 2 ? zi : nz + zi;
    j = r / GX;
    i = r - j * GX;
  } else if (g < A + B) {
    const int h = g - A;
    const int zi = h / (4 * GX);
    const int r = h - zi * 4 * GX;
    const int yi = r / GX;
    k = zi + 2;
    j = yi < 2 ? yi : ny + yi;
    i = r - yi * GX;
  } else {
    const int h = g - A - B;
    const int row = h >> 2;
    const int xi = h & 3;
    k = row / ny + 2;
    j = row - (k - 2) * ny + 2;
    i = xi < 2 ? xi : nx + xi;
  }
}

template <class S>
__global__ void __launch_bounds__(256) k_fill_ghosts(const HostGhostPatch* patches, const int2* blocks,
                                                     HostPatchIO coarse) {
  const int2 b = blocks[blockIdx.x];  // (patch, first ghost cell of this block)
  const HostGhostPatch P = patches[b.x];  // by value: the stores below cannot alias it
  const int g = b.y + threadIdx.x;
  if (g < P.nghost) {
    int i, j, k;
    ghost_cell(g, P.nx, P.ny, P.nz, i, j, k);
    const int f[3] = {P.ox + i - 2, P.oy + j - 2, P.oz + k - 2};
    const int n[3] = {coarse.nx, coarse.ny, coarse.nz};
    int c[3];
    S s[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      int q = f[d] >> 1;  // floor(f / 2)
      q %= n[d];
      c[d] = q < 0 ? q + n[d] : q;
      s[d] = (f[d] & 1) ? S(0.25) : S(-0.25);
    }
    const long long a0 = c[2] * coarse.isz + c[1] * coarse.isy + c[0];
    const long long st[3] = {1, coarse.isy, coarse.isz};
    long long am[3], ap[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      am[d] = a0 + (c[d] == 0 ? (long long)(n[d] - 1) * st[d] : -st[d]);
      ap[d] = a0 + (c[d] == n[d] - 1 ? -(long long)(n[d] - 1) * st[d] : st[d]);
    }
    const long long out = (long long)k * P.sz + (long long)j * P.sy + i;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const S* U = static_cast<const S*>(coarse.in[v]);
      const S u0 = __ldg(U + a0);
      S u = u0;
#pragma unroll
      for (int d = 0; d < 3; ++d) u = u + s[d] * minmod_s(u0 - __ldg(U + am[d]), __ldg(U + ap[d]) - u0);
      static_cast<S*>(P.U[v])[out] = u;
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

cudaError_t launch_fill_ghosts(int elem_size, const HostGhostPatch* d_patches, const int2* d_blocks, int nblocks,
                               const HostPatchIO& coarse, cudaStream_t s) {
  if (elem_size == 4)
    k_fill_ghosts<float><<<nblocks, 256, 0, s>>>(d_patches, d_blocks, coarse);
  else
    k_fill_ghosts<double><<<nblocks, 256, 0, s>>>(d_patches, d_blocks, coarse);
  return cudaGetLastError();
}

}  // namespace hydro
