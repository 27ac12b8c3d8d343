// C ABI of the hydro library (include/hydro.h): argument validation, the context and its
// library-owned scratch, patch-set caching and work-list rebuilds, launch selection, the
// CUDA-graph multi-step runner and the autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "hydro.h"
#include "hydro_device.cuh"
#include "internal.h"

using hydro::HostPatchIO;
using hydro::HostTileRec;

struct hydro_ctx {
  hydro_config cfg;
  hydro::Params prm;
  cudaStream_t stream = nullptr;
  cudaStream_t capture = nullptr;  // private stream used to capture graphs
  const hydro::KernelOps* ops = nullptr;
  int device = 0, sm_count = 0;
  unsigned* d_err = nullptr;
  // batched step: cached patch set, device descriptors and work-list
  std::vector<hydro_patch> key_in, key_out;
  HostPatchIO* h_patches = nullptr;  // pinned staging
  HostPatchIO* d_patches = nullptr;
  size_t patches_cap = 0;
  int* d_counts = nullptr;
  size_t counts_cap = 0;
  HostTileRec* d_tiles = nullptr;
  size_t tiles_cap = 0;
  int ntiles = 0;
  int* d_counter = nullptr;  // 1 + HYDRO_NUM_PATCH_CLASSES tile counters
  int wl_tile = -1, wl_zchunk = -1;
  // tile shape per patch-shape class (-1: the context's tile_id / zchunk); the work-list of a batch
  // built per class: its entries' patches (d_cls_idx), their offsets in the work-list and counts
  int cls_tile[HYDRO_NUM_PATCH_CLASSES] = {-1, -1, -1}, cls_zc[HYDRO_NUM_PATCH_CLASSES] = {0, 0, 0};
  bool wl_per_class = false;
  int wl_cls[2 * HYDRO_NUM_PATCH_CLASSES] = {};
  int* d_cls_idx = nullptr;
  size_t cls_idx_cap = 0;
  int cls_off[HYDRO_NUM_PATCH_CLASSES] = {}, cls_ntiles[HYDRO_NUM_PATCH_CLASSES] = {};
  double* d_cls_dt = nullptr;  // the autotuner's per-class time steps
  size_t cls_dt_cap = 0;
  // CFL of many patches: cached descriptors
  std::vector<hydro_patch> cfl_key;
  HostPatchIO* h_cfl = nullptr;
  HostPatchIO* d_cfl = nullptr;
  size_t cfl_cap = 0;
  // tuning
  int tile_id = 0, zchunk = 32;
  // graph cache of hydro_run
  cudaGraphExec_t graph = nullptr;
  const void* g_a = nullptr;
  const void* g_b = nullptr;
  int g_n = -1;
  double* g_dt = nullptr;
  int g_tile = -1, g_zc = -1;
  // adjoint scratch
  void* d_adj = nullptr;
  size_t adj_cap = 0;
  // host-buffer step: device staging of one box (in and out), its descriptor and slab tile list,
  // per-slab tile counters, the two copy streams and the events that chain the pipeline
  char* d_stage = nullptr;
  size_t stage_cap = 0;
  HostPatchIO* d_stage_io = nullptr;
  HostTileRec* d_stage_tiles = nullptr;
  size_t stage_tiles_cap = 0;
  int* d_stage_counters = nullptr;
  size_t stage_counters_cap = 0;
  long long stage_key[7] = {-1, -1, -1, -1, -1, -1, -1};  // nx ny nz sy sz tile zc of the uploaded list
  double stage_dx = 0.0;
  cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
  cudaStream_t s_cmp2 = nullptr;  // second compute stream: consecutive slabs' kernels overlap
  cudaEvent_t ev_ready = nullptr;
  std::vector<cudaEvent_t> ev_copied, ev_stepped, ev_halo;
  cudaEvent_t ev_begin = nullptr, ev_end = nullptr;
  // coarse-to-fine ghost fill: uploaded patch descriptors and ghost-cell offsets of the last set
  std::vector<hydro::HostGhostPatch> ghost_key;
  hydro::HostGhostPatch* d_ghost = nullptr;
  size_t ghost_cap = 0;
  int2* d_ghost_blocks = nullptr;
  size_t ghost_blocks_cap = 0;
  int ghost_nblocks = 0;
  // same-level ghost exchange: uploaded patch descriptors and copy tasks of the last set
  std::vector<hydro::HostGhostPatch> xchg_key;
  int xchg_period[3] = {0, 0, 0};
  hydro::HostGhostPatch* d_xchg = nullptr;
  size_t xchg_cap = 0;
  hydro::HostCopyTask* d_tasks = nullptr;
  size_t tasks_cap = 0;
  int ntasks = 0;
  // flux registers (patch boxes, level boxes), refluxing, average-down: descriptors and block
  // tables of the last call of each kind (reused without an upload when unchanged)
  static constexpr int kAux = 6;  // 0, 1 box fluxes; 2 reflux; 3 average-down; 4 MHD step; 5 MHD CFL
  char* d_aux[kAux] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  size_t aux_cap[kAux] = {0, 0, 0, 0, 0, 0};
  std::vector<char> aux_last[kAux];
  // oct builder scratch: key bitmap, word prefix sums, block prefix sums
  unsigned* d_octs_scratch = nullptr;
  size_t octs_scratch_cap = 0;
  // MHD step scratch: constants, face states, fluxes
  char* d_mhd = nullptr;
  size_t mhd_cap = 0;
  long long launches = 0;
};

namespace hydro {
const KernelOps* ops_for(int precision) {
  switch (precision) {
    case HYDRO_FP64: return &ops_f64();
    case HYDRO_FP32: return &ops_f32();
    case HYDRO_MIXED: return &ops_mixed();
    case HYDRO_FP64_DF: return &ops_df();
  }
  return nullptr;
}
}  // namespace hydro

namespace {

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

int cuda_status(cudaError_t e) { return e == cudaSuccess ? HYDRO_OK : HYDRO_ERR_CUDA; }

int elem_size(const hydro_ctx* c) { return c->cfg.precision == HYDRO_FP32 ? 4 : 8; }

// PPM (stencil radius 3) steps periodic boxes and patches with three ghost layers; the calls built
// on the radius-2 PLM stencil alone (the host-buffer step, octs, boundary fluxes, the adjoint)
// reject a PPM context.
bool ppm(const hydro_ctx* c) { return c->cfg.limiter == HYDRO_PPM; }

bool valid_patch(const hydro_ctx* c, const hydro_patch& p) {
  if (p.nx < 1 || p.ny < 1 || p.nz < 1) return false;
  if (p.ng != 0 && p.ng != 2 && !(p.ng == 3 && ppm(c))) return false;
  if (!finite_pos(p.dx)) return false;
  const long long gx = p.nx + 2LL * p.ng, gy = p.ny + 2LL * p.ng;
  if (p.sy < gx || p.sz < p.sy * gy) return false;
  const int es = elem_size(c);
  for (int v = 0; v < 5; ++v) {
    if (!p.U[v]) return false;
    if (reinterpret_cast<uintptr_t>(p.U[v]) % es) return false;
  }
  return true;
}

// Byte extent of a field of patch p.
size_t field_bytes(const hydro_ctx* c, const hydro_patch& p) {
  return (size_t)(p.nz + 2 * p.ng) * (size_t)p.sz * elem_size(c);
}

bool overlaps(const hydro_ctx* c, const hydro_patch& a, const hydro_patch& b) {
  const size_t na = field_bytes(c, a), nb = field_bytes(c, b);
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) {
      const char* x = static_cast<const char*>(a.U[i]);
      const char* y = static_cast<const char*>(b.U[j]);
      if (x < y + nb && y < x + na) return true;
    }
  return false;
}

bool same_shape(const hydro_patch& a, const hydro_patch& b) {
  return a.nx == b.nx && a.ny == b.ny && a.nz == b.nz && a.dx == b.dx;
}

HostPatchIO make_io(const hydro_patch& in, const hydro_patch& out) {
  HostPatchIO h;
  for (int v = 0; v < 5; ++v) {
    h.in[v] = in.U[v];
    h.out[v] = out.U[v];
  }
  h.nx = in.nx; h.ny = in.ny; h.nz = in.nz;
  h.gin = in.ng; h.gout = out.ng;
  h.isy = in.sy; h.isz = in.sz; h.osy = out.sy; h.osz = out.sz;
  h.dx = in.dx;
  return h;
}

bool same_patch(const hydro_patch& a, const hydro_patch& b) { return std::memcmp(&a, &b, sizeof(hydro_patch)) == 0; }

bool same_set(const std::vector<hydro_patch>& key, const hydro_patch* p, int n) {
  if ((int)key.size() != n) return false;
  for (int i = 0; i < n; ++i)
    if (!same_patch(key[i], p[i])) return false;
  return true;
}

template <class T>
int ensure_device(T** d, size_t* cap, size_t n) {
  if (*cap >= n) return HYDRO_OK;
  if (*d) cudaFree(*d);
  *d = nullptr;
  *cap = 0;
  if (cudaMalloc(reinterpret_cast<void**>(d), n * sizeof(T)) != cudaSuccess) return HYDRO_ERR_NOMEM;
  *cap = n;
  return HYDRO_OK;
}

// Patch-shape class of a patch for the per-class tile choice (include/hydro.h): 0 an x or y edge
// of 8 cells or fewer, 1 an x or y edge not a multiple of 16, 2 both multiples of 16.
int patch_class(const hydro_patch& p) {
  if (p.nx <= 8 || p.ny <= 8) return 0;
  if (p.nx % 16 || p.ny % 16) return 1;
  return 2;
}

bool per_class(const hydro_ctx* c) {
  if (ppm(c)) return false;
  for (int k = 0; k < HYDRO_NUM_PATCH_CLASSES; ++k)
    if (c->cls_tile[k] >= 0) return true;
  return false;
}
int class_tile(const hydro_ctx* c, int k) { return c->cls_tile[k] >= 0 ? c->cls_tile[k] : c->tile_id; }
int class_zc(const hydro_ctx* c, int k) { return c->cls_tile[k] >= 0 ? c->cls_zc[k] : c->zchunk; }

// Upload the descriptors of (in, out) and build the tile work-list for the current tuning,
// unless the cached set and tuning are unchanged.  With a tile shape per patch-shape class the
// work-list holds one segment per class, each built with its class's tile shape and z chunk.
int prepare_batch(hydro_ctx* c, const hydro_patch* in, const hydro_patch* out, int n) {
  const bool set_same = same_set(c->key_in, in, n) && same_set(c->key_out, out, n);
  const int tile = ppm(c) ? 0 : c->tile_id;  // the PPM kernel's tiles are 16 x 16 (tile shape 0)
  const int tx = hydro::kTileX[tile], ty = hydro::kTileY[tile];
  const bool pc = per_class(c);
  int cls_key[2 * HYDRO_NUM_PATCH_CLASSES];
  for (int k = 0; k < HYDRO_NUM_PATCH_CLASSES; ++k) {
    cls_key[2 * k] = class_tile(c, k);
    cls_key[2 * k + 1] = class_zc(c, k);
  }
  if (set_same && pc == c->wl_per_class &&
      (pc ? std::memcmp(cls_key, c->wl_cls, sizeof(cls_key)) == 0 : (c->wl_tile == tile && c->wl_zchunk == c->zchunk)))
    return HYDRO_OK;
  if (!set_same) {
    size_t old = c->patches_cap;
    int rc = ensure_device(&c->d_patches, &c->patches_cap, (size_t)n);
    if (rc) return rc;
    if (c->patches_cap != old || !c->h_patches) {
      if (c->h_patches) cudaFreeHost(c->h_patches);
      if (cudaMallocHost(&c->h_patches, c->patches_cap * sizeof(HostPatchIO)) != cudaSuccess) return HYDRO_ERR_NOMEM;
    }
    // the staging buffer may still be read by an earlier copy on the stream
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return HYDRO_ERR_CUDA;
    for (int i = 0; i < n; ++i) c->h_patches[i] = make_io(in[i], out[i]);
    if (cudaMemcpyAsync(c->d_patches, c->h_patches, n * sizeof(HostPatchIO), cudaMemcpyHostToDevice, c->stream) !=
        cudaSuccess)
      return HYDRO_ERR_CUDA;
    c->key_in.assign(in, in + n);
    c->key_out.assign(out, out + n);
  }
  if (pc) {
    // patches by class (host), the index list uploaded, then one work-list segment per class
    std::vector<int> idx;
    idx.reserve(n);
    int cnt[HYDRO_NUM_PATCH_CLASSES] = {}, first[HYDRO_NUM_PATCH_CLASSES] = {};
    size_t tiles[HYDRO_NUM_PATCH_CLASSES] = {};
    for (int k = 0; k < HYDRO_NUM_PATCH_CLASSES; ++k) {
      first[k] = (int)idx.size();
      const int t = class_tile(c, k), z = class_zc(c, k), kx = hydro::kTileX[t], ky = hydro::kTileY[t];
      for (int i = 0; i < n; ++i)
        if (patch_class(in[i]) == k) {
          idx.push_back(i);
          tiles[k] += (size_t)((in[i].nx + kx - 1) / kx) * ((in[i].ny + ky - 1) / ky) * ((in[i].nz + z - 1) / z);
        }
      cnt[k] = (int)idx.size() - first[k];
    }
    size_t total = 0;
    for (int k = 0; k < HYDRO_NUM_PATCH_CLASSES; ++k) total += tiles[k];
    if (total > 0x7fffffff) return HYDRO_ERR_ARG;
    int rc = ensure_device(&c->d_counts, &c->counts_cap, (size_t)n + HYDRO_NUM_PATCH_CLASSES);
    if (rc) return rc;
    rc = ensure_device(&c->d_tiles, &c->tiles_cap, std::max<size_t>(total, 1));
    if (rc) return rc;
    rc = ensure_device(&c->d_cls_idx, &c->cls_idx_cap, (size_t)n);
    if (rc) return rc;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess ||
        cudaMemcpy(c->d_cls_idx, idx.data(), n * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
      return HYDRO_ERR_CUDA;
    size_t off = 0;
    for (int k = 0; k < HYDRO_NUM_PATCH_CLASSES; ++k) {
      c->cls_off[k] = (int)off;
      c->cls_ntiles[k] = (int)tiles[k];
      if (cnt[k]) {
        const int t = class_tile(c, k);
        if (hydro::build_worklist(c->d_patches, cnt[k], hydro::kTileX[t], hydro::kTileY[t], class_zc(c, k),
                                  c->d_counts + first[k] + k, c->d_tiles + off, c->stream,
                                  c->d_cls_idx + first[k]) != cudaSuccess)
          return HYDRO_ERR_CUDA;
        c->launches += 3;
      }
      off += tiles[k];
    }
    c->ntiles = (int)total;
    c->wl_per_class = true;
    std::memcpy(c->wl_cls, cls_key, sizeof(cls_key));
    c->wl_tile = -1;
    return HYDRO_OK;
  }
  // tile count on the host sizes the buffer; the device builds the list itself
  size_t total = 0;
  for (int i = 0; i < n; ++i)
    total += (size_t)((in[i].nx + tx - 1) / tx) * ((in[i].ny + ty - 1) / ty) * ((in[i].nz + c->zchunk - 1) / c->zchunk);
  if (total > 0x7fffffff) return HYDRO_ERR_ARG;
  int rc = ensure_device(&c->d_counts, &c->counts_cap, (size_t)n + 1);
  if (rc) return rc;
  rc = ensure_device(&c->d_tiles, &c->tiles_cap, total);
  if (rc) return rc;
  if (hydro::build_worklist(c->d_patches, n, tx, ty, c->zchunk, c->d_counts, c->d_tiles, c->stream) != cudaSuccess)
    return HYDRO_ERR_CUDA;
  c->launches += 3;
  c->ntiles = (int)total;
  c->wl_tile = tile;
  c->wl_zchunk = c->zchunk;
  c->wl_per_class = false;
  return HYDRO_OK;
}

int reset_slots(hydro_ctx* c, double* p, int n, cudaStream_t s) {
  // 0xFF.. is above the bits of every positive double: the neutral element of the min.
  return cuda_status(cudaMemsetAsync(p, 0xFF, (size_t)n * sizeof(double), s));
}

int step_one_uniform(hydro_ctx* c, const hydro_patch& in, const hydro_patch& out, const double* dt, double* dt_next,
                     cudaStream_t s) {
  if (dt_next) {
    int rc = reset_slots(c, dt_next, 1, s);
    if (rc) return rc;
  }
  int zc = std::min(c->zchunk, in.nz);
  cudaError_t e = ppm(c) ? c->ops->step_ppm(make_io(in, out), c->prm, dt, dt_next, zc, c->d_err, s)
                         : c->ops->step_uniform(c->tile_id, make_io(in, out), c->prm, dt, dt_next, zc, c->d_err, s);
  c->launches += 1;
  return cuda_status(e);
}

// Device copy of host descriptor bytes for a call kind: the buffer of the last call of that kind
// when the bytes are unchanged, else a fresh upload (after the stream has drained: earlier
// kernels may still read the buffer).  Returns the device address or nullptr.
char* upload_aux(hydro_ctx* c, int kind, const std::vector<char>& bytes) {
  if (c->d_aux[kind] && bytes == c->aux_last[kind]) return c->d_aux[kind];
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return nullptr;
  if (c->aux_cap[kind] < bytes.size() || !c->d_aux[kind]) {
    cudaFree(c->d_aux[kind]);
    c->d_aux[kind] = nullptr;
    c->aux_cap[kind] = 0;
    c->aux_last[kind].clear();
    const size_t n = std::max<size_t>(bytes.size(), 256);
    if (cudaMalloc(&c->d_aux[kind], n) != cudaSuccess) return nullptr;
    c->aux_cap[kind] = n;
  }
  if (!bytes.empty() && cudaMemcpy(c->d_aux[kind], bytes.data(), bytes.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return nullptr;
  c->aux_last[kind] = bytes;
  return c->d_aux[kind];
}
template <class T>
size_t append(std::vector<char>& bytes, const T* p, size_t n) {
  const size_t off = (bytes.size() + 255) / 256 * 256;
  bytes.resize(off + n * sizeof(T));
  if (n) std::memcpy(bytes.data() + off, p, n * sizeof(T));
  return off;
}

int box_fluxes(hydro_ctx* c, int kind, const std::vector<hydro::HostBoxFluxes>& boxes, const double* dt_dev,
               int accumulate) {
  std::vector<int2> blocks;
  for (size_t b = 0; b < boxes.size(); ++b) {
    const long long nx = boxes[b].n[0], ny = boxes[b].n[1], nz = boxes[b].n[2];
    const long long faces = 2 * (ny * nz + nx * nz + nx * ny);
    if (faces > 0x7fffffffLL) return HYDRO_ERR_ARG;
    for (long long k = 0; k * 256 < faces; ++k) blocks.push_back(make_int2((int)b, (int)k));
  }
  if (blocks.size() > 0x7fffffff) return HYDRO_ERR_ARG;
  std::vector<char> bytes;
  const size_t ob = append(bytes, boxes.data(), boxes.size());
  const size_t ok = append(bytes, blocks.data(), blocks.size());
  char* d = upload_aux(c, kind, bytes);
  if (!d) return HYDRO_ERR_CUDA;
  c->launches += 1;
  return cuda_status(c->ops->box_fluxes(reinterpret_cast<const hydro::HostBoxFluxes*>(d + ob),
                                        reinterpret_cast<const int2*>(d + ok), (int)blocks.size(), c->prm, dt_dev,
                                        accumulate, c->stream));
}

}  // namespace

extern "C" {

const char* hydro_status_string(int status) {
  switch (status) {
    case HYDRO_OK: return "ok";
    case HYDRO_ERR_ARG: return "invalid argument";
    case HYDRO_ERR_CUDA: return "CUDA error";
    case HYDRO_ERR_UNPHYSICAL: return "unphysical state flagged on the device";
    case HYDRO_ERR_TIMEOUT: return "bounded device wait timed out";
    case HYDRO_ERR_NOMEM: return "device allocation failed";
    case HYDRO_ERR_STATE: return "invalid context state";
  }
  return "unknown status";
}

int hydro_init(hydro_ctx** ctx, const hydro_config* cfg) {
  if (!ctx) return HYDRO_ERR_ARG;
  *ctx = nullptr;
  if (!cfg) return HYDRO_ERR_ARG;
  if (!(cfg->gamma > 1.0 && std::isfinite(cfg->gamma))) return HYDRO_ERR_ARG;
  if (!(cfg->cfl > 0.0 && cfg->cfl <= 1.0)) return HYDRO_ERR_ARG;
  if (!(cfg->rho_floor >= 0.0 && cfg->p_floor >= 0.0)) return HYDRO_ERR_ARG;
  if (cfg->limiter < HYDRO_MINMOD || cfg->limiter > HYDRO_PPM) return HYDRO_ERR_ARG;
  if (!hydro::ops_for(cfg->precision)) return HYDRO_ERR_ARG;
  hydro_ctx* c = new hydro_ctx();
  c->cfg = *cfg;
  c->prm = hydro::make_params(cfg->gamma, cfg->cfl, cfg->rho_floor, cfg->p_floor, cfg->limiter);
  c->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
  c->ops = hydro::ops_for(cfg->precision);
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    delete c;
    return HYDRO_ERR_CUDA;
  }
  if (cudaMalloc(&c->d_err, sizeof(unsigned)) != cudaSuccess || cudaMalloc(&c->d_counter, (1 + HYDRO_NUM_PATCH_CLASSES) * sizeof(int)) != cudaSuccess) {
    hydro_finalize(c);
    return HYDRO_ERR_NOMEM;
  }
  if (cudaMemsetAsync(c->d_err, 0, sizeof(unsigned), c->stream) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking) != cudaSuccess) {
    hydro_finalize(c);
    return HYDRO_ERR_CUDA;
  }
  // FP64 favours the square tile (fewest recomputed halo cells per update); others the wide one.
  c->tile_id = 0;
  c->zchunk = 32;
  *ctx = c;
  return HYDRO_OK;
}

int hydro_finalize(hydro_ctx* c) {
  if (!c) return HYDRO_OK;
  cudaStreamSynchronize(c->stream);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->capture) cudaStreamDestroy(c->capture);
  cudaFree(c->d_err);
  cudaFree(c->d_counter);
  cudaFree(c->d_cls_idx);
  cudaFree(c->d_cls_dt);
  cudaFree(c->d_patches);
  cudaFree(c->d_counts);
  cudaFree(c->d_tiles);
  cudaFree(c->d_cfl);
  cudaFree(c->d_adj);
  if (c->s_h2d) cudaStreamSynchronize(c->s_h2d);
  if (c->s_d2h) cudaStreamSynchronize(c->s_d2h);
  if (c->s_cmp2) cudaStreamSynchronize(c->s_cmp2);
  cudaFree(c->d_stage);
  cudaFree(c->d_stage_io);
  cudaFree(c->d_stage_tiles);
  cudaFree(c->d_stage_counters);
  cudaFree(c->d_ghost);
  cudaFree(c->d_ghost_blocks);
  cudaFree(c->d_xchg);
  cudaFree(c->d_tasks);
  for (int k = 0; k < hydro_ctx::kAux; ++k) cudaFree(c->d_aux[k]);
  cudaFree(c->d_octs_scratch);
  cudaFree(c->d_mhd);
  for (cudaEvent_t e : c->ev_copied) cudaEventDestroy(e);
  for (cudaEvent_t e : c->ev_stepped) cudaEventDestroy(e);
  for (cudaEvent_t e : c->ev_halo) cudaEventDestroy(e);
  if (c->ev_begin) cudaEventDestroy(c->ev_begin);
  if (c->ev_end) cudaEventDestroy(c->ev_end);
  if (c->s_h2d) cudaStreamDestroy(c->s_h2d);
  if (c->s_d2h) cudaStreamDestroy(c->s_d2h);
  if (c->s_cmp2) cudaStreamDestroy(c->s_cmp2);
  if (c->ev_ready) cudaEventDestroy(c->ev_ready);
  if (c->h_patches) cudaFreeHost(c->h_patches);
  if (c->h_cfl) cudaFreeHost(c->h_cfl);
  delete c;
  return HYDRO_OK;
}

int hydro_cfl_dt(hydro_ctx* c, const hydro_patch* p, int npatch, double* dt_dev) {
  if (!c || !p || npatch < 1 || !dt_dev) return HYDRO_ERR_ARG;
  for (int i = 0; i < npatch; ++i)
    if (!valid_patch(c, p[i])) return HYDRO_ERR_ARG;
  int rc = reset_slots(c, dt_dev, npatch, c->stream);
  if (rc) return rc;
  if (npatch == 1) {
    c->launches += 1;
    return cuda_status(c->ops->cfl(nullptr, make_io(p[0], p[0]), 1, c->prm, dt_dev, c->d_err, c->stream));
  }
  if (!same_set(c->cfl_key, p, npatch)) {
    size_t old = c->cfl_cap;
    rc = ensure_device(&c->d_cfl, &c->cfl_cap, (size_t)npatch);
    if (rc) return rc;
    if (c->cfl_cap != old || !c->h_cfl) {
      if (c->h_cfl) cudaFreeHost(c->h_cfl);
      if (cudaMallocHost(&c->h_cfl, c->cfl_cap * sizeof(HostPatchIO)) != cudaSuccess) return HYDRO_ERR_NOMEM;
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return HYDRO_ERR_CUDA;
    for (int i = 0; i < npatch; ++i) c->h_cfl[i] = make_io(p[i], p[i]);
    if (cudaMemcpyAsync(c->d_cfl, c->h_cfl, npatch * sizeof(HostPatchIO), cudaMemcpyHostToDevice, c->stream) !=
        cudaSuccess)
      return HYDRO_ERR_CUDA;
    c->cfl_key.assign(p, p + npatch);
  }
  HostPatchIO big = make_io(p[0], p[0]);
  c->launches += 1;
  return cuda_status(c->ops->cfl(c->d_cfl, big, npatch, c->prm, dt_dev, c->d_err, c->stream));
}

int hydro_step(hydro_ctx* c, const hydro_patch* in, const hydro_patch* out, int npatch, const double* dt_dev,
               double* dt_next_dev) {
  if (!c || !in || !out || npatch < 1 || !dt_dev) return HYDRO_ERR_ARG;
  for (int i = 0; i < npatch; ++i) {
    if (!valid_patch(c, in[i]) || !valid_patch(c, out[i])) return HYDRO_ERR_ARG;
    if (!same_shape(in[i], out[i])) return HYDRO_ERR_ARG;
    if (overlaps(c, in[i], out[i])) return HYDRO_ERR_ARG;
  }
  if (npatch == 1 && in[0].ng == 0) return step_one_uniform(c, in[0], out[0], dt_dev, dt_next_dev, c->stream);
  for (int i = 0; i < npatch; ++i)  // ghost layers the reconstruction's stencil needs
    if (in[i].ng != (ppm(c) ? 3 : 2)) return HYDRO_ERR_ARG;
  int rc = prepare_batch(c, in, out, npatch);
  if (rc) return rc;
  if (cudaMemsetAsync(c->d_counter, 0, (1 + HYDRO_NUM_PATCH_CLASSES) * sizeof(int), c->stream) != cudaSuccess)
    return HYDRO_ERR_CUDA;
  if (dt_next_dev) {
    rc = reset_slots(c, dt_next_dev, npatch, c->stream);
    if (rc) return rc;
  }
  if (c->wl_per_class) {
    // one persistent launch per class, each over its own work-list segment and counter
    for (int k = 0; k < HYDRO_NUM_PATCH_CLASSES; ++k) {
      if (!c->cls_ntiles[k]) continue;
      const int t = class_tile(c, k);
      const int per_sm = c->ops->batched_blocks_per_sm(t, c->cfg.limiter);
      const int grid = std::max(1, std::min(c->cls_ntiles[k], c->sm_count * per_sm));
      c->launches += 1;
      cudaError_t e = c->ops->step_batched(t, c->d_patches, c->d_tiles + c->cls_off[k], c->cls_ntiles[k],
                                           c->d_counter + 1 + k, c->prm, dt_dev, dt_next_dev, class_zc(c, k),
                                           c->d_err, grid, c->stream);
      if (e != cudaSuccess) return HYDRO_ERR_CUDA;
    }
    return HYDRO_OK;
  }
  c->launches += 1;
  if (ppm(c))
    return cuda_status(c->ops->step_ppm_batched(c->d_patches, c->d_tiles, c->ntiles, c->d_counter, c->prm, dt_dev,
                                                dt_next_dev, c->zchunk, c->d_err, c->sm_count, c->stream));
  const int per_sm = c->ops->batched_blocks_per_sm(c->tile_id, c->cfg.limiter);
  int grid = std::max(1, std::min(c->ntiles, c->sm_count * per_sm));
  return cuda_status(c->ops->step_batched(c->tile_id, c->d_patches, c->d_tiles, c->ntiles, c->d_counter, c->prm,
                                          dt_dev, dt_next_dev, c->zchunk, c->d_err, grid, c->stream));
}

// Host-buffer step of one periodic box: the state crosses the host link in z slabs on two copy
// streams while the step kernel runs on the slabs that have arrived (copies of a quarter of the
// GPU hydro time and more are the paper's data-movement cost, Sec. 3 and Table 1; here they
// overlap the compute instead of preceding and following it).
//   H2D:  planes nz-2, nz-1 (slab 0's lower halo), then slabs 0 .. S-1
//   step: slab k once slab k+1 has arrived (slab S-1 wraps onto slab 0, already there)
//   D2H:  slab k once its step has run
int hydro_step_host(hydro_ctx* c, const hydro_patch* in, const hydro_patch* out, const double* dt_dev,
                    double* dt_next_dev) {
  if (!c || !in || !out || !dt_dev || ppm(c)) return HYDRO_ERR_ARG;
  const hydro_patch &I = *in, &O = *out;
  if (!valid_patch(c, I) || !valid_patch(c, O) || !same_shape(I, O) || overlaps(c, I, O)) return HYDRO_ERR_ARG;
  if (I.ng != 0 || O.ng != 0 || I.sy != O.sy || I.sz != O.sz) return HYDRO_ERR_ARG;
  for (int v = 0; v < 5; ++v) {
    for (const void* ptr : {static_cast<const void*>(I.U[v]), static_cast<const void*>(O.U[v])}) {
      cudaPointerAttributes a;
      if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) return HYDRO_ERR_CUDA;
      if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return HYDRO_ERR_ARG;
    }
  }
  const int es = elem_size(c);
  const size_t plane = (size_t)I.sz * es;
  const size_t fb = (size_t)I.nz * plane;
  // slabs: the z chunk shortened until the box has >= 16 slabs (or 2-plane chunks)
  int zc = c->zchunk;
  while (zc > 2 && I.nz / zc < 16) zc /= 2;
  // at least two planes per slab: a slab's upper halo (two planes) then lies in the next slab
  zc = std::max(std::min(2, I.nz), std::min(zc, I.nz));
  // Slab boundaries: zc planes each, but ramped at both ends (zc/4, zc/2, ..., zc/2, zc/4, each at
  // least two planes) where the box is tall enough: the first step waits for the first slab and its
  // halo to arrive, and the last copy-out waits for the last slab's step, so short end slabs cut
  // the pipeline's fill and drain.
  std::vector<int> zs;  // slab k covers planes [zs[k], zs[k+1])
  {
    const int a = std::max(2, zc / 4), b = std::max(2, zc / 2);
    const int ends = 2 * (a + b);
    zs.push_back(0);
    if (zc >= 8 && I.nz >= ends + 2 * zc) {
      for (int h : {a, b}) zs.push_back(zs.back() + h);
      const int mid = I.nz - ends, nm = mid / zc, rem = mid - nm * zc;
      for (int k = 0; k < nm; ++k) zs.push_back(zs.back() + zc);
      if (rem >= 2) zs.push_back(zs.back() + rem);
      else if (rem > 0) zs.back() += rem;  // one plane left over: the last middle slab takes it
      for (int h : {b, a}) zs.push_back(zs.back() + h);
    } else {
      for (int z = zc; z < I.nz; z += zc) zs.push_back(z);
      zs.push_back(I.nz);
    }
  }
  const int S = (int)zs.size() - 1;
  const int tx = hydro::kTileX[c->tile_id], ty = hydro::kTileY[c->tile_id];
  const int ntx = (I.nx + tx - 1) / tx, nty = (I.ny + ty - 1) / ty, tps = ntx * nty;
  // staging, descriptors, tile list, counters, streams, events
  int rc = HYDRO_OK;
  if (c->stage_cap < 10 * fb) {
    if (c->s_h2d) cudaStreamSynchronize(c->s_h2d);
    if (c->s_d2h) cudaStreamSynchronize(c->s_d2h);
    if (c->s_cmp2) cudaStreamSynchronize(c->s_cmp2);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return HYDRO_ERR_CUDA;
    cudaFree(c->d_stage);
    c->d_stage = nullptr;
    c->stage_cap = 0;
    if (cudaMalloc(&c->d_stage, 10 * fb) != cudaSuccess) return HYDRO_ERR_NOMEM;
    c->stage_cap = 10 * fb;
    c->stage_key[0] = -1;
  }
  if (!c->d_stage_io && cudaMalloc(&c->d_stage_io, sizeof(HostPatchIO)) != cudaSuccess) return HYDRO_ERR_NOMEM;
  rc = ensure_device(&c->d_stage_tiles, &c->stage_tiles_cap, (size_t)S * tps);
  if (rc) return rc;
  rc = ensure_device(&c->d_stage_counters, &c->stage_counters_cap, (size_t)S);
  if (rc) return rc;
  if (!c->s_h2d && cudaStreamCreateWithFlags(&c->s_h2d, cudaStreamNonBlocking) != cudaSuccess) return HYDRO_ERR_CUDA;
  if (!c->s_d2h && cudaStreamCreateWithFlags(&c->s_d2h, cudaStreamNonBlocking) != cudaSuccess) return HYDRO_ERR_CUDA;
  if (!c->s_cmp2 && cudaStreamCreateWithFlags(&c->s_cmp2, cudaStreamNonBlocking) != cudaSuccess) return HYDRO_ERR_CUDA;
  if (!c->ev_ready && cudaEventCreateWithFlags(&c->ev_ready, cudaEventDisableTiming) != cudaSuccess)
    return HYDRO_ERR_CUDA;
  if (!c->ev_begin && (cudaEventCreateWithFlags(&c->ev_begin, cudaEventDisableTiming) != cudaSuccess ||
                       cudaEventCreateWithFlags(&c->ev_end, cudaEventDisableTiming) != cudaSuccess))
    return HYDRO_ERR_CUDA;
  while ((int)c->ev_copied.size() < S) {
    cudaEvent_t e[3];
    for (int k = 0; k < 3; ++k)
      if (cudaEventCreateWithFlags(&e[k], cudaEventDisableTiming) != cudaSuccess) {
        for (int m = 0; m < k; ++m) cudaEventDestroy(e[m]);
        return HYDRO_ERR_CUDA;
      }
    c->ev_copied.push_back(e[0]);
    c->ev_stepped.push_back(e[1]);
    c->ev_halo.push_back(e[2]);
  }
  char* din[5];
  char* dout[5];
  for (int v = 0; v < 5; ++v) {
    din[v] = c->d_stage + v * fb;
    dout[v] = c->d_stage + (5 + v) * fb;
  }
  const long long key[7] = {I.nx, I.ny, I.nz, I.sy, I.sz, c->tile_id, zc};
  if (std::memcmp(key, c->stage_key, sizeof(key)) != 0 || c->stage_dx != I.dx) {
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return HYDRO_ERR_CUDA;
    HostPatchIO h;
    for (int v = 0; v < 5; ++v) {
      h.in[v] = din[v];
      h.out[v] = dout[v];
    }
    h.nx = I.nx; h.ny = I.ny; h.nz = I.nz; h.gin = 0; h.gout = 0;
    h.isy = h.osy = I.sy; h.isz = h.osz = I.sz; h.dx = I.dx;
    std::vector<HostTileRec> t((size_t)S * tps);
    for (int k = 0; k < S; ++k)
      for (int j = 0; j < nty; ++j)
        for (int i = 0; i < ntx; ++i) t[(size_t)k * tps + j * ntx + i] = HostTileRec{0, i * tx, j * ty, zs[k]};
    if (cudaMemcpy(c->d_stage_io, &h, sizeof(h), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_stage_tiles, t.data(), t.size() * sizeof(HostTileRec), cudaMemcpyHostToDevice) != cudaSuccess)
      return HYDRO_ERR_CUDA;
    std::memcpy(c->stage_key, key, sizeof(key));
    c->stage_dx = I.dx;
  }
  // planes [za, zb) of the five fields, one copy per field (a z range of a field is contiguous)
  auto upload = [&](int za, int zb) -> bool {
    for (int v = 0; v < 5 && zb > za; ++v)
      if (cudaMemcpyAsync(din[v] + za * plane, static_cast<const char*>(I.U[v]) + za * plane, (zb - za) * plane,
                          cudaMemcpyHostToDevice, c->s_h2d) != cudaSuccess)
        return false;
    return true;
  };
  auto download = [&](int za, int zb) -> bool {
    for (int v = 0; v < 5 && zb > za; ++v)
      if (cudaMemcpyAsync(static_cast<char*>(O.U[v]) + za * plane, dout[v] + za * plane, (zb - za) * plane,
                          cudaMemcpyDeviceToHost, c->s_d2h) != cudaSuccess)
        return false;
    return true;
  };
  // the staging buffers may still be read or written by the previous call's work
  if (cudaEventRecord(c->ev_begin, c->stream) != cudaSuccess || cudaStreamWaitEvent(c->s_h2d, c->ev_begin) != cudaSuccess ||
      cudaStreamWaitEvent(c->s_d2h, c->ev_begin) != cudaSuccess)
    return HYDRO_ERR_CUDA;
  const int tail = S > 1 ? std::max(0, I.nz - 2) : I.nz;
  if (!upload(tail, I.nz)) return HYDRO_ERR_CUDA;
  for (int k = 0; k < S; ++k) {
    const int za = zs[k], zb = std::min(zs[k + 1], tail);
    // a slab's first two planes go first: with them the previous slab's step can start
    const int zh = std::min(za + 2, zb);
    if (!upload(za, zh) || cudaEventRecord(c->ev_halo[k], c->s_h2d) != cudaSuccess || !upload(zh, zb) ||
        cudaEventRecord(c->ev_copied[k], c->s_h2d) != cudaSuccess)
      return HYDRO_ERR_CUDA;
  }
  if (cudaMemsetAsync(c->d_stage_counters, 0, (size_t)S * sizeof(int), c->stream) != cudaSuccess) return HYDRO_ERR_CUDA;
  if (dt_next_dev) {
    rc = reset_slots(c, dt_next_dev, 1, c->stream);
    if (rc) return rc;
  }
  const int per_sm = c->ops->batched_blocks_per_sm(c->tile_id, c->cfg.limiter);
  const int grid = std::max(1, std::min(tps, c->sm_count * per_sm));
  // slabs alternate between two compute streams, so that a slab's last partial wave of tiles runs
  // beside the next slab's first (the slabs write disjoint planes; dt_next is an order-free min)
  if (cudaEventRecord(c->ev_ready, c->stream) != cudaSuccess || cudaStreamWaitEvent(c->s_cmp2, c->ev_ready) != cudaSuccess)
    return HYDRO_ERR_CUDA;
  for (int k = 0; k < S; ++k) {
    const int za = zs[k], zb = zs[k + 1];
    cudaStream_t sk = (k & 1) ? c->s_cmp2 : c->stream;
    // slab k and its upper halo: the first two planes of slab k+1 (the last slab's halo wraps onto
    // slab 0, uploaded before it)
    if (cudaStreamWaitEvent(sk, k + 1 < S ? c->ev_halo[k + 1] : c->ev_copied[S - 1]) != cudaSuccess)
      return HYDRO_ERR_CUDA;
    c->launches += 1;
    if (c->ops->step_batched(c->tile_id, c->d_stage_io, c->d_stage_tiles + (size_t)k * tps, tps,
                             c->d_stage_counters + k, c->prm, dt_dev, dt_next_dev, zb - za, c->d_err, grid,
                             sk) != cudaSuccess)
      return HYDRO_ERR_CUDA;
    if (cudaEventRecord(c->ev_stepped[k], sk) != cudaSuccess ||
        cudaStreamWaitEvent(c->s_d2h, c->ev_stepped[k]) != cudaSuccess)
      return HYDRO_ERR_CUDA;
    if (!download(za, zb)) return HYDRO_ERR_CUDA;
  }
  if (cudaEventRecord(c->ev_end, c->s_d2h) != cudaSuccess || cudaStreamWaitEvent(c->stream, c->ev_end) != cudaSuccess)
    return HYDRO_ERR_CUDA;
  return HYDRO_OK;
}

int hydro_step_octs(hydro_ctx* c, void* const gathered[5], void* const out[5], long long ngroups, double dx,
                    const double* dt_dev) {
  if (!c || !gathered || !out || ngroups < 1 || !finite_pos(dx) || !dt_dev || ppm(c)) return HYDRO_ERR_ARG;
  const int es = elem_size(c);
  for (int v = 0; v < 5; ++v) {
    if (!gathered[v] || !out[v]) return HYDRO_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(gathered[v]) % es || reinterpret_cast<uintptr_t>(out[v]) % es) return HYDRO_ERR_ARG;
  }
  c->launches += 1;
  return cuda_status(c->ops->octs(gathered, out, ngroups, dx, c->prm, dt_dev, c->d_err, c->stream));
}

// The ghost fill from the coarse level after its step (coarse_old == nullptr), or at the fraction
// theta of its step between coarse_old and coarse.
static int fill_ghosts_impl(hydro_ctx* c, const hydro_patch* coarse, const hydro_patch* coarse_old, double theta,
                            const hydro_patch* fine, const int* fine_origins, int npatch) {
  if (!c || !coarse || !fine || !fine_origins || npatch < 1) return HYDRO_ERR_ARG;
  const hydro_patch& C = *coarse;
  if (!valid_patch(c, C) || C.ng != 0) return HYDRO_ERR_ARG;
  if (coarse_old) {
    const hydro_patch& O = *coarse_old;
    if (!valid_patch(c, O) || O.ng != 0 || !same_shape(O, C) || O.sy != C.sy || O.sz != C.sz) return HYDRO_ERR_ARG;
    if (!(theta >= 0.0 && theta <= 1.0)) return HYDRO_ERR_ARG;
  }
  std::vector<hydro::HostGhostPatch> set((size_t)npatch);
  for (int i = 0; i < npatch; ++i) {
    const hydro_patch& F = fine[i];
    if (!valid_patch(c, F) || F.ng != 2 || F.dx != 0.5 * C.dx || overlaps(c, C, F)) return HYDRO_ERR_ARG;
    hydro::HostGhostPatch& g = set[i];
    for (int v = 0; v < 5; ++v) g.U[v] = F.U[v];
    g.nx = F.nx; g.ny = F.ny; g.nz = F.nz;
    g.ox = fine_origins[3 * i]; g.oy = fine_origins[3 * i + 1]; g.oz = fine_origins[3 * i + 2];
    g.sy = F.sy; g.sz = F.sz;
    const int o[3] = {g.ox, g.oy, g.oz}, nn[3] = {F.nx, F.ny, F.nz};
    long long cells = 1;
    for (int d = 0; d < 3; ++d) {  // coarse cells floor((o-2)/2) .. floor((o+n+1)/2)
      const long long lo = (long long)std::floor((o[d] - 2) / 2.0), hi = (long long)std::floor((o[d] + nn[d] + 1) / 2.0);
      if (lo < -0x3fffffffLL || hi > 0x3fffffffLL) return HYDRO_ERR_ARG;
      g.clo[d] = (int)lo;
      g.cm[d] = (int)(hi - lo + 1);
      cells *= g.cm[d];
    }
    if (cells > 0x7fffffff) return HYDRO_ERR_ARG;
  }
  const bool same = c->ghost_key.size() == set.size() &&
                    std::memcmp(c->ghost_key.data(), set.data(), set.size() * sizeof(set[0])) == 0;
  if (!same) {
    std::vector<int2> blocks;
    for (int i = 0; i < npatch; ++i)
      for (int first = 0; first < set[i].cm[0] * set[i].cm[1] * set[i].cm[2]; first += 256)
        blocks.push_back(make_int2(i, first));
    if (blocks.size() > 0x7fffffff) return HYDRO_ERR_ARG;
    int rc = ensure_device(&c->d_ghost, &c->ghost_cap, (size_t)npatch);
    if (rc) return rc;
    rc = ensure_device(&c->d_ghost_blocks, &c->ghost_blocks_cap, blocks.size());
    if (rc) return rc;
    // the descriptors may still be read by an earlier fill on the stream
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return HYDRO_ERR_CUDA;
    if (cudaMemcpy(c->d_ghost, set.data(), set.size() * sizeof(set[0]), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_ghost_blocks, blocks.data(), blocks.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess)
      return HYDRO_ERR_CUDA;
    c->ghost_key.swap(set);
    c->ghost_nblocks = (int)blocks.size();
  }
  c->launches += 1;
  const HostPatchIO old = coarse_old ? make_io(*coarse_old, *coarse_old) : make_io(C, C);
  return cuda_status(hydro::launch_fill_ghosts(elem_size(c), c->d_ghost, c->d_ghost_blocks, c->ghost_nblocks,
                                               make_io(C, C), coarse_old ? &old : nullptr, theta, c->stream));
}

int hydro_fill_ghosts(hydro_ctx* c, const hydro_patch* coarse, const hydro_patch* fine, const int* fine_origins,
                      int npatch) {
  return fill_ghosts_impl(c, coarse, nullptr, 1.0, fine, fine_origins, npatch);
}

int hydro_fill_ghosts_time(hydro_ctx* c, const hydro_patch* coarse_old, const hydro_patch* coarse_new, double theta,
                           const hydro_patch* fine, const int* fine_origins, int npatch) {
  if (!coarse_old) return HYDRO_ERR_ARG;
  return fill_ghosts_impl(c, coarse_new, coarse_old, theta, fine, fine_origins, npatch);
}

// Copy tasks of the same-level exchange: for each destination patch, every periodic image of every
// patch interior (its own included) that meets its ghosted box.  Candidate sources come from a
// coarse spatial hash of the interiors (64-cell bins over the period).
static std::vector<hydro::HostCopyTask> exchange_tasks(const std::vector<hydro::HostGhostPatch>& P, const int per[3]) {
  const int n = (int)P.size();
  const int B = 64;
  int nb[3];
  for (int d = 0; d < 3; ++d) nb[d] = std::max(1, (per[d] + B - 1) / B);
  auto org = [&](int p, int d) { const int o[3] = {P[p].ox, P[p].oy, P[p].oz}; return ((o[d] % per[d]) + per[d]) % per[d]; };
  auto dim = [&](int p, int d) { return d == 0 ? P[p].nx : (d == 1 ? P[p].ny : P[p].nz); };
  std::vector<std::vector<int>> bins((size_t)nb[0] * nb[1] * nb[2]);
  // bins met by the positions [lo, hi) of axis d, each position wrapped into [0, period) first
  auto bins_of = [&](int lo, int hi, int d) {
    std::vector<int> out;
    for (int x = lo; x < hi; ++x) {
      const int b = (((x % per[d]) + per[d]) % per[d]) / B;
      if (out.empty() || out.back() != b)
        if (std::find(out.begin(), out.end(), b) == out.end()) out.push_back(b);
    }
    return out;
  };
  for (int p = 0; p < n; ++p) {
    const std::vector<int> bx = bins_of(org(p, 0), org(p, 0) + dim(p, 0), 0);
    const std::vector<int> by = bins_of(org(p, 1), org(p, 1) + dim(p, 1), 1);
    const std::vector<int> bz = bins_of(org(p, 2), org(p, 2) + dim(p, 2), 2);
    for (int z : bz)
      for (int y : by)
        for (int x : bx) bins[((size_t)z * nb[1] + y) * nb[0] + x].push_back(p);
  }
  std::vector<hydro::HostCopyTask> tasks;
  std::vector<int> seen(n, -1);
  for (int a = 0; a < n; ++a) {
    int glo[3], ghi[3];
    for (int d = 0; d < 3; ++d) {
      glo[d] = org(a, d) - 2;
      ghi[d] = org(a, d) + dim(a, d) + 2;
    }
    const std::vector<int> bx = bins_of(glo[0], ghi[0], 0), by = bins_of(glo[1], ghi[1], 1), bz = bins_of(glo[2], ghi[2], 2);
    std::vector<int> cand;
    for (int z : bz)
      for (int y : by)
        for (int x : bx)
          for (int q : bins[((size_t)z * nb[1] + y) * nb[0] + x])
            if (seen[q] != a) { seen[q] = a; cand.push_back(q); }
    for (int b : cand) {
      for (int kz = -2; kz <= 2; ++kz)
        for (int ky = -2; ky <= 2; ++ky)
          for (int kx = -2; kx <= 2; ++kx) {
            const int k[3] = {kx, ky, kz};
            int lo[3], hi[3];
            bool empty = false, own = (b == a);
            for (int d = 0; d < 3; ++d) {
              const int s = org(b, d) + k[d] * per[d];
              lo[d] = std::max(glo[d], s);
              hi[d] = std::min(ghi[d], s + dim(b, d));
              if (lo[d] >= hi[d]) empty = true;
              if (k[d] != 0) own = false;
            }
            if (empty || own) continue;
            hydro::HostCopyTask t;
            t.dst = a;
            t.src = b;
            for (int d = 0; d < 3; ++d) {
              t.dlo[d] = lo[d] - glo[d];
              t.slo[d] = lo[d] - (org(b, d) + k[d] * per[d]) + 2;
              t.n[d] = hi[d] - lo[d];
            }
            tasks.push_back(t);
          }
    }
  }
  return tasks;
}

int hydro_patch_fluxes(hydro_ctx* c, const hydro_patch* patches, int npatch, const double* dt_dev,
                       void* const* registers, int accumulate) {
  if (!c || !patches || npatch < 1 || !dt_dev || !registers || ppm(c)) return HYDRO_ERR_ARG;
  std::vector<hydro::HostBoxFluxes> boxes((size_t)npatch);
  for (int i = 0; i < npatch; ++i) {
    const hydro_patch& P = patches[i];
    if (!valid_patch(c, P) || P.ng != 2 || !registers[i]) return HYDRO_ERR_ARG;
    hydro::HostBoxFluxes& b = boxes[i];
    for (int v = 0; v < 5; ++v) b.U[v] = P.U[v];
    b.reg = registers[i];
    b.n[0] = P.nx; b.n[1] = P.ny; b.n[2] = P.nz;
    for (int d = 0; d < 3; ++d) b.o[d] = b.N[d] = 0;
    b.periodic = 0;
    b.dt_index = i;
    b.sy = P.sy; b.sz = P.sz;
    b.dx = P.dx;
  }
  return box_fluxes(c, 0, boxes, dt_dev, accumulate);
}

int hydro_level_fluxes(hydro_ctx* c, const hydro_patch* level, const int* box_origins, const int* box_dims, int nbox,
                       const double* dt_dev, void* const* registers, int accumulate) {
  if (!c || !level || !box_origins || !box_dims || nbox < 1 || !dt_dev || !registers || ppm(c)) return HYDRO_ERR_ARG;
  const hydro_patch& L = *level;
  if (!valid_patch(c, L) || L.ng != 0) return HYDRO_ERR_ARG;
  std::vector<hydro::HostBoxFluxes> boxes((size_t)nbox);
  for (int i = 0; i < nbox; ++i) {
    hydro::HostBoxFluxes& b = boxes[i];
    for (int v = 0; v < 5; ++v) b.U[v] = L.U[v];
    b.reg = registers[i];
    b.N[0] = L.nx; b.N[1] = L.ny; b.N[2] = L.nz;
    for (int d = 0; d < 3; ++d) {
      b.n[d] = box_dims[3 * i + d];
      b.o[d] = ((box_origins[3 * i + d] % b.N[d]) + b.N[d]) % b.N[d];  // wrapped into [0, N)
      if (b.n[d] < 1 || b.n[d] > b.N[d]) return HYDRO_ERR_ARG;
    }
    if (!b.reg) return HYDRO_ERR_ARG;
    b.periodic = 1;
    b.dt_index = 0;
    b.sy = L.sy; b.sz = L.sz;
    b.dx = L.dx;
  }
  return box_fluxes(c, 1, boxes, dt_dev, accumulate);
}

int hydro_reflux(hydro_ctx* c, const hydro_patch* coarse, const int* box_origins, const int* box_dims, int nbox,
                 void* const* coarse_registers, void* const* fine_registers) {
  if (!c || !coarse || !box_origins || !box_dims || nbox < 1 || !coarse_registers || !fine_registers)
    return HYDRO_ERR_ARG;
  const hydro_patch& C = *coarse;
  if (!valid_patch(c, C) || C.ng != 0) return HYDRO_ERR_ARG;
  std::vector<hydro::HostRefluxBox> boxes((size_t)nbox);
  std::vector<int2> tables[6];
  for (int i = 0; i < nbox; ++i) {
    hydro::HostRefluxBox& b = boxes[i];
    for (int d = 0; d < 3; ++d) {
      b.o[d] = box_origins[3 * i + d];
      b.n[d] = box_dims[3 * i + d];
      if (b.n[d] < 1) return HYDRO_ERR_ARG;
    }
    b.rc = coarse_registers[i];
    b.rf = fine_registers[i];
    if (!b.rc || !b.rf) return HYDRO_ERR_ARG;
    b.dx = C.dx;
    const long long faces[3] = {(long long)b.n[1] * b.n[2], (long long)b.n[0] * b.n[2], (long long)b.n[0] * b.n[1]};
    for (int t = 0; t < 6; ++t)
      for (long long k = 0; k * 256 < faces[t >> 1]; ++k) tables[t].push_back(make_int2(i, (int)k));
  }
  std::vector<char> bytes;
  const size_t ob = append(bytes, boxes.data(), boxes.size());
  size_t ot[6];
  int nb[6];
  for (int t = 0; t < 6; ++t) {
    if (tables[t].size() > 0x7fffffff) return HYDRO_ERR_ARG;
    ot[t] = append(bytes, tables[t].data(), tables[t].size());
    nb[t] = (int)tables[t].size();
  }
  char* d = upload_aux(c, 2, bytes);
  if (!d) return HYDRO_ERR_CUDA;
  const int2* dt[6];
  for (int t = 0; t < 6; ++t) dt[t] = reinterpret_cast<const int2*>(d + ot[t]);
  c->launches += 6;
  return cuda_status(hydro::launch_reflux(elem_size(c), reinterpret_cast<const hydro::HostRefluxBox*>(d + ob), dt, nb,
                                          make_io(C, C), c->stream));
}

int hydro_average_down(hydro_ctx* c, const hydro_patch* coarse, const hydro_patch* fine, const int* fine_origins,
                       int npatch) {
  if (!c || !coarse || !fine || !fine_origins || npatch < 1) return HYDRO_ERR_ARG;
  const hydro_patch& C = *coarse;
  if (!valid_patch(c, C) || C.ng != 0) return HYDRO_ERR_ARG;
  std::vector<hydro::HostGhostPatch> set((size_t)npatch);
  std::vector<int2> blocks;
  for (int i = 0; i < npatch; ++i) {
    const hydro_patch& F = fine[i];
    const int o[3] = {fine_origins[3 * i], fine_origins[3 * i + 1], fine_origins[3 * i + 2]};
    if (!valid_patch(c, F) || F.ng != 2 || overlaps(c, C, F)) return HYDRO_ERR_ARG;
    if ((F.nx | F.ny | F.nz | o[0] | o[1] | o[2]) & 1) return HYDRO_ERR_ARG;  // aligned with coarse cells
    hydro::HostGhostPatch& g = set[i];
    for (int v = 0; v < 5; ++v) g.U[v] = F.U[v];
    g.nx = F.nx; g.ny = F.ny; g.nz = F.nz;
    g.ox = o[0]; g.oy = o[1]; g.oz = o[2];
    for (int d = 0; d < 3; ++d) g.clo[d] = g.cm[d] = 0;
    g.sy = F.sy; g.sz = F.sz;
    const long long cells = (long long)(F.nx / 2) * (F.ny / 2) * (F.nz / 2);
    for (long long k = 0; k * 256 < cells; ++k) blocks.push_back(make_int2(i, (int)k));
  }
  std::vector<char> bytes;
  const size_t op = append(bytes, set.data(), set.size());
  const size_t obk = append(bytes, blocks.data(), blocks.size());
  char* d = upload_aux(c, 3, bytes);
  if (!d) return HYDRO_ERR_CUDA;
  c->launches += 1;
  return cuda_status(hydro::launch_average_down(elem_size(c), reinterpret_cast<const hydro::HostGhostPatch*>(d + op),
                                                reinterpret_cast<const int2*>(d + obk), (int)blocks.size(),
                                                make_io(C, C), c->stream));
}

int hydro_exchange_ghosts(hydro_ctx* c, const hydro_patch* fine, const int* origins, int npatch, const int period[3]) {
  if (!c || !fine || !origins || !period || npatch < 1) return HYDRO_ERR_ARG;
  for (int d = 0; d < 3; ++d)
    if (period[d] < 1) return HYDRO_ERR_ARG;
  std::vector<hydro::HostGhostPatch> set((size_t)npatch);
  for (int i = 0; i < npatch; ++i) {
    const hydro_patch& F = fine[i];
    if (!valid_patch(c, F) || F.ng != 2 || F.nx > period[0] || F.ny > period[1] || F.nz > period[2])
      return HYDRO_ERR_ARG;
    hydro::HostGhostPatch& g = set[i];
    for (int v = 0; v < 5; ++v) g.U[v] = F.U[v];
    g.nx = F.nx; g.ny = F.ny; g.nz = F.nz;
    g.ox = origins[3 * i]; g.oy = origins[3 * i + 1]; g.oz = origins[3 * i + 2];
    for (int d = 0; d < 3; ++d) g.clo[d] = g.cm[d] = 0;
    g.sy = F.sy; g.sz = F.sz;
  }
  const bool same = c->xchg_key.size() == set.size() &&
                    std::memcmp(c->xchg_key.data(), set.data(), set.size() * sizeof(set[0])) == 0 &&
                    std::memcmp(c->xchg_period, period, sizeof(c->xchg_period)) == 0;
  if (!same) {
    const std::vector<hydro::HostCopyTask> tasks = exchange_tasks(set, period);
    if (tasks.size() > 0x7fffffff) return HYDRO_ERR_ARG;
    int rc = ensure_device(&c->d_xchg, &c->xchg_cap, (size_t)npatch);
    if (rc) return rc;
    rc = ensure_device(&c->d_tasks, &c->tasks_cap, std::max<size_t>(1, tasks.size()));
    if (rc) return rc;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return HYDRO_ERR_CUDA;
    if (cudaMemcpy(c->d_xchg, set.data(), set.size() * sizeof(set[0]), cudaMemcpyHostToDevice) != cudaSuccess ||
        (!tasks.empty() && cudaMemcpy(c->d_tasks, tasks.data(), tasks.size() * sizeof(tasks[0]),
                                      cudaMemcpyHostToDevice) != cudaSuccess))
      return HYDRO_ERR_CUDA;
    c->xchg_key.swap(set);
    std::memcpy(c->xchg_period, period, sizeof(c->xchg_period));
    c->ntasks = (int)tasks.size();
  }
  if (c->ntasks == 0) return HYDRO_OK;
  c->launches += 1;
  return cuda_status(hydro::launch_copy_boxes(elem_size(c), c->d_xchg, c->d_tasks, c->ntasks, c->stream));
}

int hydro_step_octs_level(hydro_ctx* c, const hydro_patch* level, const int* origins_dev, long long ngroups,
                          void* const out[5], const double* dt_dev) {
  if (!c || !level || !origins_dev || !out || ngroups < 1 || !dt_dev || ppm(c)) return HYDRO_ERR_ARG;
  const hydro_patch& L = *level;
  if (!valid_patch(c, L) || L.ng != 0 || L.nx < 4 || L.ny < 4 || L.nz < 4) return HYDRO_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(origins_dev) % sizeof(int)) return HYDRO_ERR_ARG;
  const int es = elem_size(c);
  for (int v = 0; v < 5; ++v)
    if (!out[v] || reinterpret_cast<uintptr_t>(out[v]) % es) return HYDRO_ERR_ARG;
  c->launches += 1;
  return cuda_status(c->ops->octs_level(make_io(L, L), origins_dev, out, ngroups, c->prm, dt_dev, c->d_err, c->stream));
}

int hydro_octs_build(hydro_ctx* c, const int* pos_dev, int noct, const int dims[3], int* order_dev, int* nbr_dev) {
  if (!c || !pos_dev || !dims || !order_dev || noct < 1 || noct > (1 << 28)) return HYDRO_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(pos_dev) % sizeof(int) || reinterpret_cast<uintptr_t>(order_dev) % sizeof(int) ||
      reinterpret_cast<uintptr_t>(nbr_dev) % sizeof(int))
    return HYDRO_ERR_ARG;
  int bits = 0;
  for (int d = 0; d < 3; ++d) {
    if (dims[d] < 1 || dims[d] > 1024) return HYDRO_ERR_ARG;
    while ((1 << bits) < dims[d]) ++bits;
  }
  const size_t nwords = std::max<size_t>(1, ((size_t)1 << (3 * bits)) >> 5);
  const size_t nblocks = (nwords + 1023) / 1024;
  int rc = ensure_device(&c->d_octs_scratch, &c->octs_scratch_cap, 2 * nwords + nblocks);
  if (rc) return rc;
  unsigned* bitmap = c->d_octs_scratch;
  c->launches += nbr_dev ? 5 : 4;
  return cuda_status(hydro::launch_octs_build(pos_dev, noct, dims, bitmap, bitmap + nwords, bitmap + 2 * nwords,
                                              nwords, order_dev, nbr_dev, c->d_err, c->stream));
}

int hydro_step_octs_table(hydro_ctx* c, void* const in[5], void* const out[5], int noct, const int* nbr_dev,
                          const int* list_dev, long long ngroups, double dx, const double* dt_dev) {
  if (!c || !in || !out || noct < 1 || !nbr_dev || !list_dev || ngroups < 1 || !finite_pos(dx) || !dt_dev || ppm(c))
    return HYDRO_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(nbr_dev) % sizeof(int) || reinterpret_cast<uintptr_t>(list_dev) % sizeof(int))
    return HYDRO_ERR_ARG;
  const int es = elem_size(c);
  const uintptr_t bytes = (uintptr_t)noct * 8 * es;
  for (int v = 0; v < 5; ++v) {
    if (!in[v] || !out[v]) return HYDRO_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(in[v]) % es || reinterpret_cast<uintptr_t>(out[v]) % es) return HYDRO_ERR_ARG;
  }
  for (int v = 0; v < 5; ++v)  // out is written while in is read as neighbours: no overlap
    for (int u = 0; u < 5; ++u) {
      const uintptr_t a = reinterpret_cast<uintptr_t>(out[v]), b = reinterpret_cast<uintptr_t>(in[u]);
      if (a < b + bytes && b < a + bytes) return HYDRO_ERR_ARG;
    }
  c->launches += 1;
  return cuda_status(
      c->ops->octs_table(in, nbr_dev, noct, list_dev, out, ngroups, dx, c->prm, dt_dev, c->d_err, c->stream));
}

// Arguments of the MHD calls: a periodic box of nine contiguous fields in a context with a PLM
// limiter.
static bool mhd_args(const hydro_ctx* c, void* const* U, int nx, int ny, int nz, double dx) {
  if (!c || !U || nx < 1 || ny < 1 || nz < 1 || !finite_pos(dx)) return false;
  if ((long long)nx * ny * nz > 0x7fffffffLL) return false;
  if (ppm(c)) return false;
  const int es = elem_size(c);
  for (int v = 0; v < 9; ++v)
    if (!U[v] || reinterpret_cast<uintptr_t>(U[v]) % es) return false;
  return true;
}

static hydro::HostMhdBox mhd_box(void* const* in, void* const* out, int nx, int ny, int nz, double dx) {
  hydro::HostMhdBox h;
  for (int v = 0; v < 9; ++v) {
    h.in[v] = in[v];
    h.out[v] = out ? out[v] : nullptr;
  }
  h.nx = nx; h.ny = ny; h.nz = nz;
  h.dx = dx;
  return h;
}

int hydro_mhd_step(hydro_ctx* c, void* const in[9], void* const out[9], int nx, int ny, int nz, double dx,
                   const double* dt_dev, double* dt_next_dev) {
  if (!mhd_args(c, in, nx, ny, nz, dx) || !mhd_args(c, out, nx, ny, nz, dx) || !dt_dev) return HYDRO_ERR_ARG;
  const uintptr_t bytes = (uintptr_t)nx * ny * nz * elem_size(c);
  for (int v = 0; v < 9; ++v)  // out is written while in is read by other cells: no overlap
    for (int u = 0; u < 9; ++u) {
      const uintptr_t a = reinterpret_cast<uintptr_t>(out[v]), b = reinterpret_cast<uintptr_t>(in[u]);
      if (a < b + bytes && b < a + bytes) return HYDRO_ERR_ARG;
    }
  int rc = ensure_device(&c->d_mhd, &c->mhd_cap,
                         hydro::mhd_scratch_bytes(c->cfg.precision, nx, ny, nz, elem_size(c)));
  if (rc) return rc;
  if (dt_next_dev) {
    rc = reset_slots(c, dt_next_dev, 1, c->stream);
    if (rc) return rc;
  }
  c->launches += hydro::mhd_step_launches(c->cfg.precision);
  return cuda_status(hydro::launch_mhd_step(c->cfg.precision, mhd_box(in, out, nx, ny, nz, dx), c->prm, dt_dev,
                                            dt_next_dev, c->d_mhd, c->d_err, c->stream));
}

int hydro_mhd_cfl_dt(hydro_ctx* c, void* const U[9], int nx, int ny, int nz, double dx, double* dt_dev) {
  if (!mhd_args(c, U, nx, ny, nz, dx) || !dt_dev) return HYDRO_ERR_ARG;
  int rc = reset_slots(c, dt_dev, 1, c->stream);
  if (rc) return rc;
  c->launches += 1;
  return cuda_status(
      hydro::launch_mhd_cfl(c->cfg.precision, mhd_box(U, nullptr, nx, ny, nz, dx), c->prm, dt_dev, c->d_err, c->stream));
}

// A patch of the batched MHD calls: sizes, ghost layers (2; 0 also allowed for an output unless
// ghosts_only), strides and pointers.
static bool mhd_patch_ok(const hydro_ctx* c, const hydro_mhd_patch& p, bool ghosts_only) {
  if (p.nx < 1 || p.ny < 1 || p.nz < 1 || !finite_pos(p.dx)) return false;
  if (p.ng != 2 && !(p.ng == 0 && !ghosts_only)) return false;
  const long long gx = p.nx + 2LL * p.ng, gy = p.ny + 2LL * p.ng;
  if (p.sy < gx || p.sz < p.sy * gy) return false;
  if ((long long)(p.nx + 2) * (p.ny + 2) * (p.nz + 2) > 0x7fffff00LL) return false;
  const int es = elem_size(c);
  for (int v = 0; v < 9; ++v)
    if (!p.U[v] || reinterpret_cast<uintptr_t>(p.U[v]) % es) return false;
  return true;
}

static size_t mhd_patch_bytes(const hydro_ctx* c, const hydro_mhd_patch& p) {
  return (size_t)(p.nz + 2 * p.ng) * (size_t)p.sz * elem_size(c);
}

// Descriptors and the block table of a patch set, uploaded (or reused) as aux kind `kind`: with
// tiles, the fused step's tile records (patch, x0, y0, z0) when the precision has them, else 256
// extended cells of one patch per block; returns the device descriptors, table, count and the
// per-cell scratch elements.
static int mhd_patch_tables(hydro_ctx* c, int kind, const hydro_mhd_patch* in, const hydro_mhd_patch* out, int npatch,
                            bool tiles, const hydro::HostMhdPatch** d_patches, const void** d_blocks, int* nblocks,
                            size_t* scratch_elems) {
  std::vector<hydro::HostMhdPatch> set((size_t)npatch);
  std::vector<int2> blocks;
  std::vector<int4> recs;
  int tx = 0, ty = 0, zc = 0;
  tiles = tiles && hydro::mhd_patch_tiles(c->cfg.precision, &tx, &ty, &zc);
  long long off = 0;
  for (int i = 0; i < npatch; ++i) {
    const hydro_mhd_patch& I = in[i];
    const hydro_mhd_patch& O = out ? out[i] : in[i];
    hydro::HostMhdPatch& h = set[i];
    for (int v = 0; v < 9; ++v) {
      h.in[v] = I.U[v];
      h.out[v] = O.U[v];
    }
    h.nx = I.nx; h.ny = I.ny; h.nz = I.nz; h.gout = O.ng;
    h.isy = I.sy; h.isz = I.sz; h.osy = O.sy; h.osz = O.sz;
    h.dx = I.dx;
    h.scratch = off;
    if (tiles) {
      h.scratch = 0;
      for (int z = 0; z < I.nz; z += zc)
        for (int y = 0; y < I.ny; y += ty)
          for (int x = 0; x < I.nx; x += tx) recs.push_back(make_int4(i, x, y, z));
      continue;
    }
    const long long ec = (long long)(I.nx + 2) * (I.ny + 2) * (I.nz + 2);
    off += 81 * ec;
    for (long long f = 0; f < ec; f += 256) blocks.push_back(make_int2(i, (int)f));
  }
  if (blocks.size() > 0x7fffffff || recs.size() > 0x7fffffff) return HYDRO_ERR_ARG;
  std::vector<char> bytes;
  const size_t op = append(bytes, set.data(), set.size());
  const size_t ob = tiles ? append(bytes, recs.data(), recs.size()) : append(bytes, blocks.data(), blocks.size());
  char* d = upload_aux(c, kind, bytes);
  if (!d) return HYDRO_ERR_CUDA;
  *d_patches = reinterpret_cast<const hydro::HostMhdPatch*>(d + op);
  *d_blocks = d + ob;
  *nblocks = (int)(tiles ? recs.size() : blocks.size());
  *scratch_elems = (size_t)off;
  return HYDRO_OK;
}

int hydro_mhd_step_patches(hydro_ctx* c, const hydro_mhd_patch* in, const hydro_mhd_patch* out, int npatch,
                           const double* dt_dev, double* dt_next_dev) {
  if (!c || !in || !out || npatch < 1 || !dt_dev) return HYDRO_ERR_ARG;
  if (ppm(c)) return HYDRO_ERR_ARG;
  for (int i = 0; i < npatch; ++i) {
    const hydro_mhd_patch &I = in[i], &O = out[i];
    if (!mhd_patch_ok(c, I, true) || !mhd_patch_ok(c, O, false)) return HYDRO_ERR_ARG;
    if (I.nx != O.nx || I.ny != O.ny || I.nz != O.nz || I.dx != O.dx) return HYDRO_ERR_ARG;
    const size_t bi = mhd_patch_bytes(c, I), bo = mhd_patch_bytes(c, O);
    for (int v = 0; v < 9; ++v)  // the output is written while the input is read: no overlap
      for (int u = 0; u < 9; ++u) {
        const uintptr_t a = reinterpret_cast<uintptr_t>(O.U[v]), b = reinterpret_cast<uintptr_t>(I.U[u]);
        if (a < b + bi && b < a + bo) return HYDRO_ERR_ARG;
      }
  }
  const hydro::HostMhdPatch* dp = nullptr;
  const void* db = nullptr;
  int nb = 0;
  size_t elems = 0;
  int rc = mhd_patch_tables(c, 4, in, out, npatch, true, &dp, &db, &nb, &elems);
  if (rc) return rc;
  rc = ensure_device(&c->d_mhd, &c->mhd_cap, hydro::mhd_patch_consts_bytes(npatch) + elems * elem_size(c));
  if (rc) return rc;
  if (dt_next_dev) {
    rc = reset_slots(c, dt_next_dev, npatch, c->stream);
    if (rc) return rc;
  }
  c->launches += hydro::mhd_step_launches(c->cfg.precision);
  return cuda_status(hydro::launch_mhd_patches(c->cfg.precision, dp, db, nb, npatch, c->prm, dt_dev, dt_next_dev,
                                               c->d_mhd, c->d_err, c->stream));
}

int hydro_mhd_cfl_patches(hydro_ctx* c, const hydro_mhd_patch* p, int npatch, double* dt_dev) {
  if (!c || !p || npatch < 1 || !dt_dev) return HYDRO_ERR_ARG;
  if (ppm(c)) return HYDRO_ERR_ARG;
  for (int i = 0; i < npatch; ++i)
    if (!mhd_patch_ok(c, p[i], true)) return HYDRO_ERR_ARG;
  const hydro::HostMhdPatch* dp = nullptr;
  const void* db = nullptr;
  int nb = 0;
  size_t elems = 0;
  int rc = mhd_patch_tables(c, 5, p, nullptr, npatch, false, &dp, &db, &nb, &elems);
  if (rc) return rc;
  rc = reset_slots(c, dt_dev, npatch, c->stream);
  if (rc) return rc;
  c->launches += 1;
  return cuda_status(hydro::launch_mhd_patches_cfl(c->cfg.precision, dp, static_cast<const int2*>(db), nb, c->prm,
                                                   dt_dev, c->d_err, c->stream));
}

int hydro_adjoint_step(hydro_ctx* c, const hydro_patch* U_n, const double* dt_dev, const hydro_patch* lam_np1,
                       const hydro_patch* lam_n, int npatch) {
  if (!c || !U_n || !dt_dev || !lam_np1 || !lam_n || npatch < 1 || ppm(c)) return HYDRO_ERR_ARG;
  if (c->cfg.precision == HYDRO_MIXED) return HYDRO_ERR_ARG;
  // The double-float context runs the FP64 reverse sweep: on GB300 it is faster than the same
  // sweep in double-float arithmetic, whose register footprint (~240 per thread) leaves too few
  // warps per SM to cover the FP32 pipes' dependent chains; both keep the FP64 accuracy.
  const hydro::KernelOps* aops = c->cfg.precision == HYDRO_FP64_DF ? hydro::ops_for(HYDRO_FP64) : c->ops;
  for (int i = 0; i < npatch; ++i) {
    const hydro_patch &U = U_n[i], &L = lam_np1[i], &O = lam_n[i];
    if (!valid_patch(c, U) || !valid_patch(c, L) || !valid_patch(c, O)) return HYDRO_ERR_ARG;
    if (U.ng != 0 || L.ng != 0 || O.ng != 0) return HYDRO_ERR_ARG;
    if (!same_shape(U, L) || !same_shape(U, O)) return HYDRO_ERR_ARG;
    if (overlaps(c, L, O) || overlaps(c, U, O)) return HYDRO_ERR_ARG;
  }
  for (int i = 0; i < npatch; ++i) {
    const hydro_patch &U = U_n[i], &L = lam_np1[i], &O = lam_n[i];
    const size_t need = aops->adjoint_scratch_bytes(U.nx, U.ny, U.nz);
    if (need > c->adj_cap) {
      cudaFree(c->d_adj);
      c->d_adj = nullptr;
      c->adj_cap = 0;
      if (cudaMalloc(&c->d_adj, need) != cudaSuccess) return HYDRO_ERR_NOMEM;
      c->adj_cap = need;
    }
    void* outp[5];
    for (int v = 0; v < 5; ++v) outp[v] = O.U[v];
    HostPatchIO lam = make_io(L, O);
    c->launches += 2;
    cudaError_t e = aops->adjoint(make_io(U, O), lam, outp, c->prm, dt_dev + i, c->d_adj, c->adj_cap, c->d_err,
                                  c->stream);
    if (e == cudaErrorNotSupported) return HYDRO_ERR_STATE;
    if (e != cudaSuccess) return HYDRO_ERR_CUDA;
  }
  return HYDRO_OK;
}

int hydro_prim_to_cons(hydro_ctx* c, const hydro_patch* W, const hydro_patch* U, int npatch) {
  if (!c || !W || !U || npatch < 1) return HYDRO_ERR_ARG;
  for (int i = 0; i < npatch; ++i) {
    if (!valid_patch(c, W[i]) || !valid_patch(c, U[i]) || !same_shape(W[i], U[i]) || overlaps(c, W[i], U[i]))
      return HYDRO_ERR_ARG;
  }
  for (int i = 0; i < npatch; ++i) {
    void* o[5];
    for (int v = 0; v < 5; ++v) o[v] = U[i].U[v];
    c->launches += 1;
    cudaError_t e = c->ops->p2c(make_io(W[i], U[i]), o, c->prm, c->stream);
    if (e != cudaSuccess) return HYDRO_ERR_CUDA;
  }
  return HYDRO_OK;
}

int hydro_prim_to_cons_adjoint(hydro_ctx* c, const hydro_patch* W, const hydro_patch* lamU, const hydro_patch* lamW,
                               int npatch) {
  if (!c || !W || !lamU || !lamW || npatch < 1) return HYDRO_ERR_ARG;
  for (int i = 0; i < npatch; ++i) {
    if (!valid_patch(c, W[i]) || !valid_patch(c, lamU[i]) || !valid_patch(c, lamW[i])) return HYDRO_ERR_ARG;
    if (!same_shape(W[i], lamU[i]) || !same_shape(W[i], lamW[i])) return HYDRO_ERR_ARG;
    if (overlaps(c, W[i], lamW[i]) || overlaps(c, lamU[i], lamW[i])) return HYDRO_ERR_ARG;
  }
  for (int i = 0; i < npatch; ++i) {
    void* o[5];
    for (int v = 0; v < 5; ++v) o[v] = lamW[i].U[v];
    c->launches += 1;
    cudaError_t e = c->ops->p2c_adjoint(make_io(W[i], lamW[i]), make_io(lamU[i], lamU[i]), o, c->prm, c->stream);
    if (e != cudaSuccess) return HYDRO_ERR_CUDA;
  }
  return HYDRO_OK;
}

int hydro_run(hydro_ctx* c, const hydro_patch* a, const hydro_patch* b, int nsteps, double* dt_hist_dev,
              int use_graph) {
  if (!c || !a || !b || nsteps < 1 || !dt_hist_dev) return HYDRO_ERR_ARG;
  if (!valid_patch(c, *a) || !valid_patch(c, *b) || a->ng != 0 || b->ng != 0) return HYDRO_ERR_ARG;
  if (!same_shape(*a, *b) || overlaps(c, *a, *b)) return HYDRO_ERR_ARG;
  auto enqueue = [&](cudaStream_t s) -> int {
    int rc = reset_slots(c, dt_hist_dev, 1, s);
    if (rc) return rc;
    cudaError_t e = c->ops->cfl(nullptr, make_io(*a, *a), 1, c->prm, dt_hist_dev, c->d_err, s);
    c->launches += 1;
    if (e != cudaSuccess) return HYDRO_ERR_CUDA;
    for (int n = 0; n < nsteps; ++n) {
      const hydro_patch& src = (n % 2 == 0) ? *a : *b;
      const hydro_patch& dst = (n % 2 == 0) ? *b : *a;
      rc = step_one_uniform(c, src, dst, dt_hist_dev + n, dt_hist_dev + n + 1, s);
      if (rc) return rc;
    }
    return HYDRO_OK;
  };
  if (!use_graph) return enqueue(c->stream);
  const bool hit = c->graph && c->g_a == a->U[0] && c->g_b == b->U[0] && c->g_n == nsteps && c->g_dt == dt_hist_dev &&
                   c->g_tile == c->tile_id && c->g_zc == c->zchunk;
  if (!hit) {
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    const long long before = c->launches;
    if (cudaStreamBeginCapture(c->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return HYDRO_ERR_CUDA;
    int rc = enqueue(c->capture);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->capture, &g);
    c->launches = before;  // capture launches nothing
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return HYDRO_ERR_CUDA;
    e = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      c->graph = nullptr;
      return HYDRO_ERR_CUDA;
    }
    c->g_a = a->U[0];
    c->g_b = b->U[0];
    c->g_n = nsteps;
    c->g_dt = dt_hist_dev;
    c->g_tile = c->tile_id;
    c->g_zc = c->zchunk;
  }
  c->launches += nsteps + 1;
  return cuda_status(cudaGraphLaunch(c->graph, c->stream));
}

int hydro_get_tuning(hydro_ctx* c, int* tile_id, int* zchunk) {
  if (!c) return HYDRO_ERR_ARG;
  if (tile_id) *tile_id = c->tile_id;
  if (zchunk) *zchunk = c->zchunk;
  return HYDRO_OK;
}

int hydro_set_tuning(hydro_ctx* c, int tile_id, int zchunk) {
  if (!c || tile_id < 0 || tile_id >= hydro::kNumTiles || zchunk < 1 || zchunk > 4096) return HYDRO_ERR_ARG;
  c->tile_id = tile_id;
  c->zchunk = zchunk;
  for (int k = 0; k < HYDRO_NUM_PATCH_CLASSES; ++k) c->cls_tile[k] = -1;
  return HYDRO_OK;
}

int hydro_get_class_tuning(hydro_ctx* c, int patch_class_id, int* tile_id, int* zchunk) {
  if (!c || patch_class_id < 0 || patch_class_id >= HYDRO_NUM_PATCH_CLASSES) return HYDRO_ERR_ARG;
  if (tile_id) *tile_id = class_tile(c, patch_class_id);
  if (zchunk) *zchunk = class_zc(c, patch_class_id);
  return HYDRO_OK;
}

int hydro_set_class_tuning(hydro_ctx* c, int patch_class_id, int tile_id, int zchunk) {
  if (!c || patch_class_id < 0 || patch_class_id >= HYDRO_NUM_PATCH_CLASSES) return HYDRO_ERR_ARG;
  if (tile_id == -1) {
    c->cls_tile[patch_class_id] = -1;
    return HYDRO_OK;
  }
  if (tile_id < 0 || tile_id >= hydro::kNumTiles || zchunk < 1 || zchunk > 4096) return HYDRO_ERR_ARG;
  c->cls_tile[patch_class_id] = tile_id;
  c->cls_zc[patch_class_id] = zchunk;
  return HYDRO_OK;
}

int hydro_autotune(hydro_ctx* c, const hydro_patch* in, const hydro_patch* out, int npatch, const double* dt_dev,
                   const char* cache_path) {
  if (!c || !in || !out || npatch < 1 || !dt_dev) return HYDRO_ERR_ARG;
  // signature of the patch set: count, precision and total cells
  long long cells = 0;
  for (int i = 0; i < npatch; ++i) cells += (long long)in[i].nx * in[i].ny * in[i].nz;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, c->device) != cudaSuccess) return HYDRO_ERR_CUDA;
  char key[512];
  std::snprintf(key, sizeof(key), "%s|sm%d|p%d|l%d|n%d|c%lld|g%d", prop.name, c->sm_count, c->cfg.precision,
                c->cfg.limiter, npatch, cells, in[0].ng);
  for (char* k = key; *k; ++k)
    if (*k == ' ') *k = '_';
  constexpr int NC = HYDRO_NUM_PATCH_CLASSES;
  if (cache_path) {
    // one line per tuning: key, tile, z chunk, then tile and z chunk of each patch-shape class (-1: none)
    if (FILE* f = std::fopen(cache_path, "r")) {
      char k2[512];
      int t, z, ct[NC], cz[NC];
      while (std::fscanf(f, "%511s %d %d %d %d %d %d %d %d", k2, &t, &z, &ct[0], &cz[0], &ct[1], &cz[1], &ct[2],
                         &cz[2]) == 3 + 2 * NC) {
        bool ok = std::strcmp(k2, key) == 0 && t >= 0 && t < hydro::kNumTiles && z >= 1;
        for (int k = 0; k < NC; ++k) ok = ok && ct[k] >= -1 && ct[k] < hydro::kNumTiles && (ct[k] < 0 || cz[k] >= 1);
        if (ok) {
          c->tile_id = t;
          c->zchunk = z;
          for (int k = 0; k < NC; ++k) {
            c->cls_tile[k] = ct[k];
            c->cls_zc[k] = cz[k];
          }
          std::fclose(f);
          return HYDRO_OK;
        }
      }
      std::fclose(f);
    }
  }
  for (int k = 0; k < NC; ++k) c->cls_tile[k] = -1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // time of 3 steps (after a warm-up that also builds the work-list) of a patch set at the current tuning
  auto time3 = [&](const hydro_patch* a, const hydro_patch* b, int n, const double* dt, float* ms) -> int {
    int rc = hydro_step(c, a, b, n, dt, nullptr);
    if (rc) return rc;
    cudaEventRecord(e0, c->stream);
    for (int r = 0; r < 3; ++r) hydro_step(c, a, b, n, dt, nullptr);
    cudaEventRecord(e1, c->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) return HYDRO_ERR_CUDA;
    cudaEventElapsedTime(ms, e0, e1);
    return HYDRO_OK;
  };
  // the fastest tile shape and z chunk for a patch set (uniform tuning)
  auto sweep = [&](const hydro_patch* a, const hydro_patch* b, int n, const double* dt, int* bt, int* bz,
                   float* best) -> int {
    long long cl = 0;
    int maxnz = 1;
    for (int i = 0; i < n; ++i) {
      cl += (long long)a[i].nx * a[i].ny * a[i].nz;
      maxnz = std::max(maxnz, a[i].nz);
    }
    // short z chunks only pay on small grids, where the longer ones leave SMs without a block
    const int zcs[] = {2, 4, 8, 16, 32, 64, 128};
    *best = 1e30f;
    for (int t = 0; t < (ppm(c) ? 1 : hydro::kNumTiles); ++t) {  // the PPM kernel has one tile shape
      for (int zc : zcs) {
        if (zc > std::max(8, maxnz)) continue;
        if (zc < 8 && cl > (1LL << 22)) continue;
        c->tile_id = t;
        c->zchunk = zc;
        float ms = 0;
        int rc = time3(a, b, n, dt, &ms);
        if (rc) return rc;
        if (ms < *best) {
          *best = ms;
          *bt = t;
          *bz = zc;
        }
      }
    }
    return HYDRO_OK;
  };
  int bt = c->tile_id, bz = c->zchunk;
  float best = 1e30f;
  int rc = sweep(in, out, npatch, dt_dev, &bt, &bz, &best);
  // a tile shape per patch-shape class, when the set holds patches of more than one class: each
  // class's best shape on its own patches, kept if the whole set then steps faster
  std::vector<int> cls((size_t)npatch);
  int present = 0, cnt[NC] = {};
  for (int i = 0; i < npatch; ++i) cnt[cls[i] = patch_class(in[i])]++;
  for (int k = 0; k < NC; ++k) present += cnt[k] > 0;
  int ct[NC] = {-1, -1, -1}, cz[NC] = {0, 0, 0};
  if (!rc && !ppm(c) && present > 1) {
    rc = ensure_device(&c->d_cls_dt, &c->cls_dt_cap, (size_t)npatch);
    for (int k = 0; k < NC && !rc; ++k) {
      if (!cnt[k]) continue;
      std::vector<hydro_patch> a, b;
      for (int i = 0; i < npatch; ++i)
        if (cls[i] == k) {
          a.push_back(in[i]);
          b.push_back(out[i]);
          // the class's time steps, gathered in order (one small device copy each)
          if (cudaMemcpyAsync(c->d_cls_dt + a.size() - 1, dt_dev + i, sizeof(double), cudaMemcpyDeviceToDevice,
                              c->stream) != cudaSuccess)
            rc = HYDRO_ERR_CUDA;
        }
      float bk = 0;
      if (!rc) rc = sweep(a.data(), b.data(), (int)a.size(), c->d_cls_dt, &ct[k], &cz[k], &bk);
    }
    if (!rc) {
      c->tile_id = bt;
      c->zchunk = bz;
      for (int k = 0; k < NC; ++k) {
        c->cls_tile[k] = cnt[k] ? ct[k] : -1;
        c->cls_zc[k] = cz[k];
      }
      float ms = 0;
      rc = time3(in, out, npatch, dt_dev, &ms);
      if (!rc && !(ms < 0.99f * best))
        for (int k = 0; k < NC; ++k) c->cls_tile[k] = -1;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) {
    for (int k = 0; k < NC; ++k) c->cls_tile[k] = -1;
    return rc;
  }
  c->tile_id = bt;
  c->zchunk = bz;
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "a")) {
      std::fprintf(f, "%s %d %d", key, bt, bz);
      for (int k = 0; k < NC; ++k) std::fprintf(f, " %d %d", c->cls_tile[k], c->cls_tile[k] >= 0 ? c->cls_zc[k] : 0);
      std::fprintf(f, "\n");
      std::fclose(f);
    }
  }
  return HYDRO_OK;
}

int hydro_get_error(hydro_ctx* c, unsigned* error_bits) {
  if (!c) return HYDRO_ERR_ARG;
  unsigned bits = 0;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return HYDRO_ERR_CUDA;
  if (cudaMemcpy(&bits, c->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return HYDRO_ERR_CUDA;
  if (error_bits) *error_bits = bits;
  return bits ? HYDRO_ERR_UNPHYSICAL : HYDRO_OK;
}

int hydro_clear_error(hydro_ctx* c) {
  if (!c) return HYDRO_ERR_ARG;
  return cuda_status(cudaMemsetAsync(c->d_err, 0, sizeof(unsigned), c->stream));
}

int hydro_launch_count(hydro_ctx* c, long long* count) {
  if (!c || !count) return HYDRO_ERR_ARG;
  *count = c->launches;
  return HYDRO_OK;
}

}  // extern "C"
