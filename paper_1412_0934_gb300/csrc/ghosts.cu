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

// One thread per coarse cell under a patch's ghost shell: it forms the cell's three limited
// slopes once and its eight children as ((U_C +- D_x/4) +- D_y/4) +- D_z/4 -- the two x partial
// sums, then four, then eight (the same operations in the same order as child by child, so the
// same bits) -- and writes the children that are ghost cells of the patch.  Coarse cells whose
// children are all interior return at once.  Each block takes up to 256 coarse cells of one patch
// (a block table built on the host).
template <class S>
__global__ void __launch_bounds__(256) k_fill_ghosts(const HostGhostPatch* patches, const int2* blocks,
                                                     HostPatchIO coarse) {
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
    const S u0 = __ldg(U + a0);
    S D[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) D[d] = minmod_s(u0 - __ldg(U + am[d]), __ldg(U + ap[d]) - u0);
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

cudaError_t launch_fill_ghosts(int elem_size, const HostGhostPatch* d_patches, const int2* d_blocks, int nblocks,
                               const HostPatchIO& coarse, cudaStream_t s) {
  if (elem_size == 4)
    k_fill_ghosts<float><<<nblocks, 256, 0, s>>>(d_patches, d_blocks, coarse);
  else
    k_fill_ghosts<double><<<nblocks, 256, 0, s>>>(d_patches, d_blocks, coarse);
  return cudaGetLastError();
}

}  // namespace hydro
