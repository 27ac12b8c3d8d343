// hydro_step_batched_noalloc: the batched patch step for callers that cannot allocate device
// memory.  Some callers cannot call cudaMalloc -- code running inside another runtime's memory
// pool or under a strict memory budget, code that must not allocate after start-up, or a host
// program that only receives device pointers from elsewhere.  hydro_step needs a context, and
// hydro_init allocates; this entry point needs no context: the scratch that the batched step
// uses (uploaded patch descriptors, the prefix-sum counts, the tile work-list and the tile
// counter) lives in the file-scope __device__ arrays below, which every GPU that loads the library
// holds until the process exits (about 4.7 MB).  The caller passes the device word that receives
// the error bits, so that no fault the kernels detect goes unread.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "hydro.h"
#include "hydro_device.cuh"
#include "internal.h"

namespace {

constexpr int kMaxPatches = 4096;
constexpr int kMaxTiles = 262144;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) hydro::HostPatchIO g_patches[kMaxPatches];
static __device__ __align__(256) int g_counts[kMaxPatches + 1];
static __device__ __align__(256) hydro::HostTileRec g_tiles[kMaxTiles];
static __device__ __align__(256) int g_counter[1];

// Device addresses of the arrays above, looked up once per device (host code must not use the
// array names themselves: on the host they are stand-ins, not device addresses).
struct DeviceScratch {
  bool ready = false;
  hydro::HostPatchIO* patches = nullptr;
  int* counts = nullptr;
  hydro::HostTileRec* tiles = nullptr;
  int* counter = nullptr;
};
DeviceScratch g_scratch[kMaxDevices];
std::mutex g_setup_mutex;
// Host staging of the descriptors (pageable: cudaMemcpyAsync copies it out before returning).
hydro::HostPatchIO g_stage[kMaxPatches];
std::mutex g_stage_mutex;

int setup_device(int dev, DeviceScratch** out) {
  if (dev < 0 || dev >= kMaxDevices) return HYDRO_ERR_STATE;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceScratch& s = g_scratch[dev];
  if (!s.ready) {
    if (cudaGetSymbolAddress(reinterpret_cast<void**>(&s.patches), g_patches) != cudaSuccess ||
        cudaGetSymbolAddress(reinterpret_cast<void**>(&s.counts), g_counts) != cudaSuccess ||
        cudaGetSymbolAddress(reinterpret_cast<void**>(&s.tiles), g_tiles) != cudaSuccess ||
        cudaGetSymbolAddress(reinterpret_cast<void**>(&s.counter), g_counter) != cudaSuccess)
      return HYDRO_ERR_CUDA;
    s.ready = true;
  }
  *out = &s;
  return HYDRO_OK;
}

bool patch_ok(const hydro_patch& p, int es) {
  if (p.nx < 1 || p.ny < 1 || p.nz < 1 || (p.ng != 0 && p.ng != 2)) return false;
  if (!(std::isfinite(p.dx) && p.dx > 0.0)) return false;
  if (p.sy < p.nx + 2LL * p.ng || p.sz < p.sy * (p.ny + 2LL * p.ng)) return false;
  for (int v = 0; v < 5; ++v)
    if (!p.U[v] || reinterpret_cast<uintptr_t>(p.U[v]) % es) return false;
  return true;
}

bool disjoint(const hydro_patch& a, const hydro_patch& b, int es) {
  const size_t na = (size_t)(a.nz + 2 * a.ng) * (size_t)a.sz * es;
  const size_t nb = (size_t)(b.nz + 2 * b.ng) * (size_t)b.sz * es;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) {
      const char* x = static_cast<const char*>(a.U[i]);
      const char* y = static_cast<const char*>(b.U[j]);
      if (x < y + nb && y < x + na) return false;
    }
  return true;
}

}  // namespace

extern "C" int hydro_step_batched_noalloc(const hydro_config* cfg, const hydro_patch* in, const hydro_patch* out,
                                          int npatch, const double* dt_dev, double* dt_next_dev,
                                          unsigned* error_bits_dev) {
  if (!cfg || !in || !out || !dt_dev || !error_bits_dev || npatch < 1) return HYDRO_ERR_ARG;
  if (npatch > kMaxPatches) return HYDRO_ERR_ARG;
  if (!(cfg->gamma > 1.0 && std::isfinite(cfg->gamma)) || !(cfg->cfl > 0.0 && cfg->cfl <= 1.0) ||
      !(cfg->rho_floor >= 0.0 && cfg->p_floor >= 0.0) || cfg->limiter < HYDRO_MINMOD || cfg->limiter > HYDRO_NOLIMIT ||
      !hydro::ops_for(cfg->precision))
    return HYDRO_ERR_ARG;
  const int es = cfg->precision == HYDRO_FP32 ? 4 : 8;
  const int tile = 0;
  const int zchunk = 32;
  const int tx = hydro::kTileX[tile], ty = hydro::kTileY[tile];
  long long total = 0;
  for (int i = 0; i < npatch; ++i) {
    const hydro_patch &a = in[i], &b = out[i];
    if (!patch_ok(a, es) || !patch_ok(b, es)) return HYDRO_ERR_ARG;
    if (a.nx != b.nx || a.ny != b.ny || a.nz != b.nz || a.dx != b.dx || !disjoint(a, b, es)) return HYDRO_ERR_ARG;
    // the ghost layers hydro_step asks for: two per input patch, or none for a single periodic box
    if (a.ng != 2 && !(npatch == 1 && a.ng == 0)) return HYDRO_ERR_ARG;
    total += (long long)((a.nx + tx - 1) / tx) * ((a.ny + ty - 1) / ty) * ((a.nz + zchunk - 1) / zchunk);
  }
  if (total > kMaxTiles) return HYDRO_ERR_ARG;

  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HYDRO_ERR_CUDA;
  DeviceScratch* s = nullptr;
  int rc = setup_device(dev, &s);
  if (rc) return rc;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return HYDRO_ERR_CUDA;
  const hydro::KernelOps& ops = *hydro::ops_for(cfg->precision);
  const hydro::Params prm = hydro::make_params(cfg->gamma, cfg->cfl, cfg->rho_floor, cfg->p_floor, cfg->limiter);
  cudaStream_t st = static_cast<cudaStream_t>(cfg->cuda_stream);
  unsigned* err = error_bits_dev;
  {
    std::lock_guard<std::mutex> lock(g_stage_mutex);
    for (int i = 0; i < npatch; ++i) {
      hydro::HostPatchIO& h = g_stage[i];
      for (int v = 0; v < 5; ++v) {
        h.in[v] = in[i].U[v];
        h.out[v] = out[i].U[v];
      }
      h.nx = in[i].nx; h.ny = in[i].ny; h.nz = in[i].nz;
      h.gin = in[i].ng; h.gout = out[i].ng;
      h.isy = in[i].sy; h.isz = in[i].sz; h.osy = out[i].sy; h.osz = out[i].sz;
      h.dx = in[i].dx;
    }
    if (cudaMemcpyAsync(s->patches, g_stage, npatch * sizeof(hydro::HostPatchIO), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
      return HYDRO_ERR_CUDA;
  }
  if (hydro::build_worklist(s->patches, npatch, tx, ty, zchunk, s->counts, s->tiles, st) != cudaSuccess)
    return HYDRO_ERR_CUDA;
  if (cudaMemsetAsync(s->counter, 0, sizeof(int), st) != cudaSuccess) return HYDRO_ERR_CUDA;
  if (dt_next_dev && cudaMemsetAsync(dt_next_dev, 0xFF, (size_t)npatch * sizeof(double), st) != cudaSuccess)
    return HYDRO_ERR_CUDA;
  const int per_sm = ops.batched_blocks_per_sm(tile, cfg->limiter);
  long long grid = (long long)sms * per_sm;
  if (grid > total) grid = total;
  if (grid < 1) grid = 1;
  cudaError_t e = ops.step_batched(tile, s->patches, s->tiles, (int)total, s->counter, prm, dt_dev, dt_next_dev, zchunk,
                                   err, (int)grid, st);
  return e == cudaSuccess ? HYDRO_OK : HYDRO_ERR_CUDA;
}
