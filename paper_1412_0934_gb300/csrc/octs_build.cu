// Space-filling-curve order and neighbour table of one level's octs.  The paper's Ramses GPU
// procedure orders a level's cells along the space-filling curve before cutting them into chunks,
// and gathers each oct's neighbourhood for the hydro kernel (Sec. 3, Fig. 1).
//
// An oct sits at integer oct coordinates (X, Y, Z) of a periodic level with dims octs per axis.
// Its Morton key interleaves the bits of X, Y and Z, x lowest.  Distinct positions have distinct
// keys, so the order needs no comparison sort: each oct sets its key's bit in a bitmap over the
// key space, an exclusive prefix sum of the words' population counts is taken, and the rank of a
// present key is prefix[word] + popc(word & the bits below it).  The same O(1) lookup finds an
// oct's neighbours: the neighbour at an offset exists iff the bit of its (wrapped) key is set, and
// its index is order[rank].
//
// Launches: bitmap and order clear, keys into the bitmap, block-local word prefix sums, prefix sum
// of the block totals, ranks into order, neighbour table.  All integer arithmetic; the order and
// the table are unique, so every run gives the same result.
#include <cuda_runtime.h>

#include "internal.h"

namespace hydro {
namespace {

constexpr int kWordsPerBlock = 1024;  // words of one prefix-sum block (256 threads x 4)

// Bit b of v (b < 10) moved to bit 3b.
__device__ __forceinline__ unsigned spread3(unsigned v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

__device__ __forceinline__ unsigned morton(int X, int Y, int Z) {
  return spread3((unsigned)X) | (spread3((unsigned)Y) << 1) | (spread3((unsigned)Z) << 2);
}

__device__ __forceinline__ bool inside(int X, int Y, int Z, int3 d) {
  return X >= 0 && Y >= 0 && Z >= 0 && X < d.x && Y < d.y && Z < d.z;
}

// Rank of a key whose bit is set: the number of set bits below it.
__device__ __forceinline__ unsigned key_rank(unsigned key, const unsigned* bitmap, const unsigned* word_prefix,
                                             const unsigned* block_prefix) {
  const unsigned w = key >> 5;
  return block_prefix[w / kWordsPerBlock] + word_prefix[w] + __popc(bitmap[w] & ((1u << (key & 31)) - 1u));
}

// Each oct sets its key's bit; a position outside the level or already set flags the error word.
__global__ void k_oct_keys(const int* pos, int noct, int3 dims, unsigned* bitmap, unsigned* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= noct) return;
  const int X = pos[3 * i], Y = pos[3 * i + 1], Z = pos[3 * i + 2];
  if (!inside(X, Y, Z, dims)) {
    atomicOr(err, HYDRO_EBIT_BAD_TILE);
    return;
  }
  const unsigned key = morton(X, Y, Z);
  const unsigned bit = 1u << (key & 31);
  if (atomicOr(bitmap + (key >> 5), bit) & bit) atomicOr(err, HYDRO_EBIT_BAD_TILE);  // two octs at one position
}

// Inclusive prefix sum of v over the warp.
__device__ __forceinline__ unsigned warp_inclusive(unsigned v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Block b: exclusive prefix sums of the population counts of words b*1024 .. b*1024+1023 (four
// consecutive words per thread) and the block's total.
__global__ void __launch_bounds__(256) k_scan_words(const unsigned* bitmap, size_t nwords, unsigned* word_prefix,
                                                    unsigned* block_total) {
  __shared__ unsigned warp_total[8];
  const size_t base = (size_t)blockIdx.x * kWordsPerBlock + 4 * threadIdx.x;
  unsigned c[4], s = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    c[k] = base + k < nwords ? (unsigned)__popc(bitmap[base + k]) : 0u;
    s += c[k];
  }
  const unsigned inc = warp_inclusive(s);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 31) warp_total[w] = inc;
  __syncthreads();
  unsigned run = inc - s;
  for (int k = 0; k < w; ++k) run += warp_total[k];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (base + k < nwords) word_prefix[base + k] = run;
    run += c[k];
  }
  if (threadIdx.x == 255) block_total[blockIdx.x] = run;
}

// One block: the block totals become their exclusive prefix sums, 1024 at a time with a carry.
__global__ void __launch_bounds__(1024) k_scan_blocks(unsigned* block_prefix, int nblocks) {
  __shared__ unsigned warp_total[32];
  __shared__ unsigned carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int w = threadIdx.x >> 5;
  for (int base = 0; base < nblocks; base += 1024) {
    const int i = base + threadIdx.x;
    const unsigned v = i < nblocks ? block_prefix[i] : 0u;
    const unsigned inc = warp_inclusive(v);
    if ((threadIdx.x & 31) == 31) warp_total[w] = inc;
    __syncthreads();
    unsigned off = carry;
    for (int k = 0; k < w; ++k) off += warp_total[k];
    if (i < nblocks) block_prefix[i] = off + inc - v;
    __syncthreads();  // carry and warp_total read by all before they change
    if (threadIdx.x == 1023) carry = off + inc;
    __syncthreads();
  }
}

__global__ void k_oct_rank(const int* pos, int noct, int3 dims, const unsigned* bitmap, const unsigned* word_prefix,
                           const unsigned* block_prefix, int* order) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= noct) return;
  const int X = pos[3 * i], Y = pos[3 * i + 1], Z = pos[3 * i + 2];
  if (!inside(X, Y, Z, dims)) return;
  const unsigned r = key_rank(morton(X, Y, Z), bitmap, word_prefix, block_prefix);
  if (r < (unsigned)noct) order[r] = i;
}

// 32 octs x 27 neighbours per block: entry ((dz+1)*3 + dy+1)*3 + dx+1 of oct i is the oct at
// (X+dx, Y+dy, Z+dz) wrapped on the level, or -1; consecutive threads write consecutive entries.
__global__ void __launch_bounds__(864) k_oct_nbr(const int* pos, int noct, int3 dims, const unsigned* bitmap,
                                                 const unsigned* word_prefix, const unsigned* block_prefix,
                                                 const int* order, int* nbr) {
  const int t = threadIdx.x, lo = t / 27, n = t - 27 * lo;
  const int i = blockIdx.x * 32 + lo;
  if (i >= noct) return;
  int X = pos[3 * i], Y = pos[3 * i + 1], Z = pos[3 * i + 2];
  int out = -1;
  if (inside(X, Y, Z, dims)) {
    X += n % 3 - 1;
    Y += (n / 3) % 3 - 1;
    Z += n / 9 - 1;
    X += X < 0 ? dims.x : (X >= dims.x ? -dims.x : 0);
    Y += Y < 0 ? dims.y : (Y >= dims.y ? -dims.y : 0);
    Z += Z < 0 ? dims.z : (Z >= dims.z ? -dims.z : 0);
    const unsigned key = morton(X, Y, Z);
    if ((bitmap[key >> 5] >> (key & 31)) & 1u) {
      const unsigned r = key_rank(key, bitmap, word_prefix, block_prefix);
      if (r < (unsigned)noct) out = order[r];
    }
  }
  nbr[27LL * i + n] = out;
}

}  // namespace

cudaError_t launch_octs_build(const int* pos, int noct, const int dims[3], unsigned* bitmap, unsigned* word_prefix,
                              unsigned* block_prefix, size_t nwords, int* order, int* nbr, unsigned* err,
                              cudaStream_t s) {
  const int3 d = make_int3(dims[0], dims[1], dims[2]);
  const int nblocks = (int)((nwords + kWordsPerBlock - 1) / kWordsPerBlock);
  cudaError_t e = cudaMemsetAsync(bitmap, 0, nwords * sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(order, 0xff, (size_t)noct * sizeof(int), s);  // -1: no oct yet
  if (e != cudaSuccess) return e;
  const int g = (noct + 255) / 256;
  k_oct_keys<<<g, 256, 0, s>>>(pos, noct, d, bitmap, err);
  k_scan_words<<<nblocks, 256, 0, s>>>(bitmap, nwords, word_prefix, block_prefix);
  k_scan_blocks<<<1, 1024, 0, s>>>(block_prefix, nblocks);
  k_oct_rank<<<g, 256, 0, s>>>(pos, noct, d, bitmap, word_prefix, block_prefix, order);
  if (nbr) k_oct_nbr<<<(noct + 31) / 32, 864, 0, s>>>(pos, noct, d, bitmap, word_prefix, block_prefix, order, nbr);
  return cudaGetLastError();
}

}  // namespace hydro
