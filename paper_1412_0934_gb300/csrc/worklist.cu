// Device-built tile work-list for the batched step (the paper's Ramses GPU procedure groups
// patches into large chunks that are solved together, Sec. 3; Enzo offloads patch by batch,
// Sec. 4): per-patch tile counts -> exclusive scan -> tile records (patch, x0, y0, z0), ordered
// patch by patch, z-chunk by z-chunk, then y and x so that concurrently running tiles share halos
// in L2.
#include "internal.h"

namespace hydro {

// idx: nullptr (entry k is patch k) or the patches of the list (entry k is patch idx[k]).
__global__ void k_tile_count(const HostPatchIO* patches, const int* idx, int npatch, int tx, int ty, int zc,
                             int* counts) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npatch; p += gridDim.x * blockDim.x) {
    const HostPatchIO& P = patches[idx ? idx[p] : p];
    counts[p] = ((P.nx + tx - 1) / tx) * ((P.ny + ty - 1) / ty) * ((P.nz + zc - 1) / zc);
  }
}

// Exclusive scan of counts[0..n) in place by one block of 1024 threads; counts[n] = total.
__global__ void __launch_bounds__(1024) k_scan(int* counts, int n) {
  __shared__ int part[1024];
  const int t = threadIdx.x;
  const int per = (n + 1023) / 1024;
  const int b = t * per, e = min(b + per, n);
  int s = 0;
  for (int i = b; i < e; ++i) s += counts[i];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int v = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int run = part[t] - s;  // exclusive prefix of this thread's chunk
  for (int i = b; i < e; ++i) {
    const int c = counts[i];
    counts[i] = run;
    run += c;
  }
  if (t == 1023) counts[n] = part[1023];
}

__global__ void k_tile_fill(const HostPatchIO* patches, const int* idx, int npatch, int tx, int ty, int zc,
                            const int* offsets, HostTileRec* tiles) {
  for (int p = blockIdx.x; p < npatch; p += gridDim.x) {
    const int pid = idx ? idx[p] : p;
    const HostPatchIO& P = patches[pid];
    const int ntx = (P.nx + tx - 1) / tx, nty = (P.ny + ty - 1) / ty, nzc = (P.nz + zc - 1) / zc;
    const int n = ntx * nty * nzc, base = offsets[p];
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const int ix = t % ntx, iy = (t / ntx) % nty, iz = t / (ntx * nty);
      tiles[base + t] = HostTileRec{pid, ix * tx, iy * ty, iz * zc};
    }
  }
}

cudaError_t build_worklist(const HostPatchIO* d_patches, int npatch, int tx, int ty, int zchunk, int* d_counts,
                           HostTileRec* d_tiles, cudaStream_t s, const int* d_idx) {
  k_tile_count<<<(npatch + 255) / 256, 256, 0, s>>>(d_patches, d_idx, npatch, tx, ty, zchunk, d_counts);
  k_scan<<<1, 1024, 0, s>>>(d_counts, npatch);
  k_tile_fill<<<npatch < 4096 ? npatch : 4096, 128, 0, s>>>(d_patches, d_idx, npatch, tx, ty, zchunk, d_counts,
                                                            d_tiles);
  return cudaGetLastError();
}

}  // namespace hydro
