// Host-side interface between the C ABI (hydro_api.cu) and the per-precision kernel files.
#pragma once
#include <cuda_runtime.h>

#include <atomic>

#include "hydro.h"

namespace hydro {

// A setting made once per device (a kernel's shared-memory opt-in is a property of the kernel on
// the device that is current when it is set): call() runs f the first time it is used with each
// device (ordinals 0-63) current, and again on later calls only if f failed.
struct PerDeviceOnce {
  std::atomic<unsigned long long> done{0};
  template <class F>
  cudaError_t call(F&& f) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = (dev >= 0 && dev < 64) ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = f();
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
    return e;
  }
};

struct Params;

// Layout-compatible host image of PatchIO<S> (pointers are untyped here).
struct HostPatchIO {
  const void* in[5];
  void* out[5];
  int nx, ny, nz;
  int gin, gout;
  long long isy, isz, osy, osz;
  double dx;
};

struct HostTileRec {
  int patch, x0, y0, z0;
};

// Compiled tile shapes of the step kernels (TX x TY columns per block) and the resident blocks
// per SM their register allocation targets (0: the policy default, 2 x 256 threads for 8-byte
// arithmetic, 3 x 256 for float; 1: a whole SM's registers for one block, no spills).
constexpr int kNumTiles = HYDRO_NUM_TILES;
constexpr int kTileX[kNumTiles] = {16, 32, 8, 32, 16};
constexpr int kTileY[kNumTiles] = {16, 8, 8, 16, 16};
constexpr int kTileMinBlocks[kNumTiles] = {0, 0, 0, 0, 1};

// A box whose boundary-face fluxes go to a register: a ghosted patch's interior (periodic == 0:
// cell (x, y, z) of the interior at (z+2) sz + (y+2) sy + x + 2) or the box at o of a periodic
// level of N cells per axis (periodic == 1).
struct HostBoxFluxes {
  const void* U[5];
  void* reg;         // 5 x 2 (ny nz + nx nz + nx ny) elements of the storage type
  int n[3];          // box cells (x, y, z)
  int o[3], N[3];    // periodic level: box origin and level size
  int periodic;
  int dt_index;      // dt_dev[dt_index] is this box's time step
  long long sy, sz;
  double dx;
};

struct KernelOps {
  // Uniform periodic grid (npatch == 1, gin == 0).
  cudaError_t (*step_uniform)(int tile, const HostPatchIO& P, const Params& prm, const double* dt, double* dt_next,
                              int zchunk, unsigned* err, cudaStream_t s);
  // Persistent batched step over a device work-list.
  cudaError_t (*step_batched)(int tile, const HostPatchIO* d_patches, const HostTileRec* d_tiles, int ntiles,
                              int* d_counter, const Params& prm, const double* dt, double* dt_next, int zchunk,
                              unsigned* err, int grid, cudaStream_t s);
  // Occupancy (blocks per SM) of the batched kernel for a tile shape and limiter.
  int (*batched_blocks_per_sm)(int tile, int limiter);
  // CFL dt per patch: d_patches (device) or a single patch by value when d_patches == nullptr.
  cudaError_t (*cfl)(const HostPatchIO* d_patches, const HostPatchIO& single, int npatch, const Params& prm,
                     double* dt_out, unsigned* err, cudaStream_t s);
  // Oct groups (6^3 gathered -> 2^3).
  cudaError_t (*octs)(void* const gathered[5], void* const out[5], long long ngroups, double dx, const Params& prm,
                      const double* dt, unsigned* err, cudaStream_t s);
  // Oct groups read in place from a periodic level grid at the given origins (-> 2^3 each).
  cudaError_t (*octs_level)(const HostPatchIO& level, const int* origins, void* const out[5], long long ngroups,
                            const Params& prm, const double* dt, unsigned* err, cudaStream_t s);
  // Oct groups of oct-major storage read through a neighbour table; group g steps oct list[g] and
  // writes its 8 cells in place of that oct in out.
  cudaError_t (*octs_table)(void* const in[5], const int* nbr, int noct, const int* list, void* const out[5],
                            long long ngroups, double dx, const Params& prm, const double* dt, unsigned* err,
                            cudaStream_t s);
  // Adjoint of one periodic step.
  cudaError_t (*adjoint)(const HostPatchIO& U, const HostPatchIO& lam, void* const lam_out[5], const Params& prm,
                         const double* dt, void* scratch, size_t scratch_bytes, unsigned* err, cudaStream_t s);
  size_t (*adjoint_scratch_bytes)(int nx, int ny, int nz);
  // Primitive -> conservative map and its adjoint, elementwise over a patch (interior).
  cudaError_t (*p2c)(const HostPatchIO& W, void* const U[5], const Params& prm, cudaStream_t s);
  cudaError_t (*p2c_adjoint)(const HostPatchIO& W, const HostPatchIO& lamU, void* const lamW[5], const Params& prm,
                             cudaStream_t s);
  // Boundary-face fluxes of boxes into registers (block b: faces 256 d_blocks[b].y ... of box d_blocks[b].x).
  cudaError_t (*box_fluxes)(const HostBoxFluxes* d_boxes, const int2* d_blocks, int nblocks, const Params& prm,
                            const double* dt, int accumulate, cudaStream_t s);
  // The PPM step of a periodic box (P.gin == 0), z chunks of zchunk planes; dt_next as step_uniform.
  cudaError_t (*step_ppm)(const HostPatchIO& P, const Params& prm, const double* dt, double* dt_next, int zchunk,
                          unsigned* err, cudaStream_t s);
  // The PPM step of patches with three ghost layers over a 16 x 16 tile work-list (persistent grid).
  cudaError_t (*step_ppm_batched)(const HostPatchIO* d_patches, const HostTileRec* d_tiles, int ntiles,
                                  int* d_counter, const Params& prm, const double* dt, double* dt_next, int zchunk,
                                  unsigned* err, int sm_count, cudaStream_t s);
  int elem_size;  // bytes per stored element
  int launches_per_step;
};

const KernelOps& ops_f64();
const KernelOps& ops_f32();
const KernelOps& ops_mixed();
const KernelOps& ops_df();
// Kernel set of a hydro_precision value (nullptr if out of range).
const KernelOps* ops_for(int precision);

// A fine patch whose ghost layers the coarse-to-fine fill writes: its fields, interior size,
// strides and the fine-level index of its first interior cell.
struct HostGhostPatch {
  void* U[5];
  int nx, ny, nz;
  int ox, oy, oz;
  int clo[3], cm[3];  // coarse cells under the ghosted box: lowest index and count per axis
  long long sy, sz;
};

// A box copied from patch src's interior (local ghosted coordinates slo) into patch dst's ghost
// shell (dlo), n cells per axis (x, y, z).
struct HostCopyTask {
  int dst, src;
  int dlo[3], slo[3], n[3];
};
cudaError_t launch_copy_boxes(int elem_size, const HostGhostPatch* d_patches, const HostCopyTask* d_tasks, int ntasks,
                              cudaStream_t s);

// A coarse box covered by a fine patch, with its coarse and fine flux registers (the fine one for
// the box refined by 2), for refluxing.
struct HostRefluxBox {
  int o[3], n[3];      // coarse box origin and cells (x, y, z)
  const void* rc;      // 5 x 2 (ny nz + nx nz + nx ny)
  const void* rf;      // 5 x 8 (ny nz + nx nz + nx ny)
  double dx;           // coarse cell size
};
cudaError_t launch_reflux(int elem_size, const HostRefluxBox* d_boxes, const int2* const d_blocks[6],
                          const int nblocks[6], const HostPatchIO& coarse, cudaStream_t s);
cudaError_t launch_average_down(int elem_size, const HostGhostPatch* d_patches, const int2* d_blocks, int nblocks,
                                const HostPatchIO& coarse, cudaStream_t s);

// Coarse-to-fine ghost fill (ghosts.cu): block b takes coarse cells d_blocks[b].y .. +255 under
// patch d_blocks[b].x.  coarse_old: nullptr, or the coarse state before its step (same layout), the
// coarse values then being (1 - theta) old + theta coarse.
cudaError_t launch_fill_ghosts(int elem_size, const HostGhostPatch* d_patches, const int2* d_blocks, int nblocks,
                               const HostPatchIO& coarse, const HostPatchIO* coarse_old, double theta,
                               cudaStream_t s);

// Morton order and neighbour table of a level's octs (octs_build.cu).  Scratch: bitmap and
// word_prefix of nwords words, block_prefix of (nwords + 1023) / 1024 words; nwords = max(1, 8^b / 32)
// for keys below 8^b.
cudaError_t launch_octs_build(const int* pos, int noct, const int dims[3], unsigned* bitmap, unsigned* word_prefix,
                              unsigned* block_prefix, size_t nwords, int* order, int* nbr, unsigned* err,
                              cudaStream_t s);

// Ideal MHD with GLM cleaning on a periodic box (mhd.cu): nine fields (rho, m, E, B, psi), each
// nx*ny*nz contiguous, x fastest; any precision.  The step needs mhd_scratch_bytes (elem_size: bytes
// of the arithmetic type) of device scratch: the step's constants, and for the 8-byte arithmetic the
// face states and fluxes of its three-launch form; mhd_step_launches kernels per step.
struct HostMhdBox {
  const void* in[9];
  void* out[9];
  int nx, ny, nz;
  double dx;
};
size_t mhd_scratch_bytes(int precision, int nx, int ny, int nz, int elem_size);
int mhd_step_launches(int precision);
// A patch of the batched MHD step (two ghost layers in, 0 or 2 out): its scratch, 81 elements per
// cell of its extended box (nx+2)(ny+2)(nz+2), starts at element offset `scratch` of the scratch
// body, which follows mhd_patch_consts_bytes(npatch) bytes of per-patch constants.
struct HostMhdPatch {
  const void* in[9];
  void* out[9];
  int nx, ny, nz, gout;
  long long isy, isz, osy, osz;
  double dx;
  long long scratch;
};
size_t mhd_patch_consts_bytes(int npatch);
// The step on patches: d_blocks is the int4 tile table (patch, x0, y0, z0) of mhd_patch_tiles'
// shape where that returns true (float arithmetic, one fused launch, no per-cell scratch), else the
// int2 block table (patch, first extended cell) of the three launches.
bool mhd_patch_tiles(int precision, int* tx, int* ty, int* zc);
cudaError_t launch_mhd_patches(int precision, const HostMhdPatch* d_patches, const void* d_blocks, int nblocks,
                               int npatch, const Params& prm, const double* dt, double* dt_next, void* scratch,
                               unsigned* err, cudaStream_t s);
cudaError_t launch_mhd_patches_cfl(int precision, const HostMhdPatch* d_patches, const int2* d_blocks, int nblocks,
                                   const Params& prm, double* dt, unsigned* err, cudaStream_t s);
cudaError_t launch_mhd_step(int precision, const HostMhdBox& h, const Params& prm, const double* dt, double* dt_next,
                            void* scratch, unsigned* err, cudaStream_t s);
cudaError_t launch_mhd_cfl(int precision, const HostMhdBox& h, const Params& prm, double* dt, unsigned* err,
                           cudaStream_t s);

// Work-list construction (precision-independent; descriptors read through HostPatchIO): the tiles of
// npatch patches -- patches 0 .. npatch-1, or d_idx[0 .. npatch-1] of d_patches when d_idx is given
// (the records carry the patch's own index).  d_counts: npatch + 1 ints of scratch.
cudaError_t build_worklist(const HostPatchIO* d_patches, int npatch, int tx, int ty, int zchunk, int* d_counts,
                           HostTileRec* d_tiles, cudaStream_t s, const int* d_idx = nullptr);

}  // namespace hydro
