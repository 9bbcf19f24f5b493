// encode.cu -- App. C output records on the GPU.
//
// A record is the count -- one byte when below 255, else the byte 0xFF followed by the count as
// a big-endian 32-bit integer -- then the k-mer with four bases per byte (A=00 C=01 G=10 T=11,
// first base in the two high bits of the first byte; the unused low bits of the last byte are
// written as 0).  Every record is KB+1 or KB+5 bytes (KB = ceil(k/4)), so the byte offset of row
// i is i*(KB+1) + 4*(rows before i with count >= 255): the encoder counts long-count rows per
// tile, scans the tile sums, then writes every tile's records from its own offset.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace gerbil {

constexpr int ENC_THREADS = 256;
constexpr int ENC_ROWS = 8;  // consecutive rows per thread
constexpr int ENC_TILE = ENC_THREADS * ENC_ROWS;

__global__ void __launch_bounds__(ENC_THREADS) encode_count_kernel(const uint32_t* __restrict__ counts,
                                                                  unsigned long long n,
                                                                  unsigned long long* __restrict__ tile_long) {
  const unsigned long long t = blockIdx.x;
  const unsigned long long r0 = t * ENC_TILE + (unsigned long long)threadIdx.x * ENC_ROWS;
  uint32_t c = 0;
#pragma unroll
  for (int j = 0; j < ENC_ROWS; ++j)
    if (r0 + j < n) c += __ldg(counts + r0 + j) >= 255u ? 1u : 0u;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xFFFFFFFFu, c, o);
  __shared__ uint32_t s[ENC_THREADS / 32];
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long sum = 0;
    for (int w = 0; w < ENC_THREADS / 32; ++w) sum += s[w];
    tile_long[t] = sum;
  }
}

// In-place exclusive scan of the tile sums by one CTA; total[0] receives the sum.
__global__ void __launch_bounds__(1024) encode_scan_kernel(unsigned long long* __restrict__ v,
                                                          unsigned long long ntiles,
                                                          unsigned long long* __restrict__ total) {
  __shared__ unsigned long long warp_sum[32];
  __shared__ unsigned long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (unsigned long long base = 0; base < ntiles; base += blockDim.x) {
    const unsigned long long i = base + threadIdx.x;
    const unsigned long long x = i < ntiles ? v[i] : 0ull;
    unsigned long long incl = x;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const unsigned long long ws = lane < (int)(blockDim.x >> 5) ? warp_sum[lane] : 0ull;
      unsigned long long wi = ws;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
        if (lane >= o) wi += y;
      }
      if (lane < (int)(blockDim.x >> 5)) warp_sum[lane] = wi - ws;  // exclusive
    }
    __syncthreads();
    const unsigned long long c0 = carry;
    if (i < ntiles) v[i] = c0 + warp_sum[warp] + incl - x;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = c0 + warp_sum[warp] + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

// Eight bits of the 2k-bit key (W words, word 0 most significant) whose lowest bit sits at
// bit position t (t >= -6; bits below position 0 read as 0).
template <int W>
__device__ __forceinline__ uint32_t key_byte(const unsigned long long key[W], int t) {
  if (t < 0) return (uint32_t)(key[W - 1] << (-t)) & 0xFFu;
  const int wi = W - 1 - (t >> 6), off = t & 63;
  unsigned long long v = 0;
#pragma unroll
  for (int j = 0; j < W; ++j)
    if (j == wi) v = key[j] >> off;
  if (off > 56) {
#pragma unroll
    for (int j = 0; j < W; ++j)
      if (j == wi - 1) v |= key[j] << (64 - off);
  }
  return (uint32_t)v & 0xFFu;
}

template <int W>
__global__ void __launch_bounds__(ENC_THREADS) encode_write_kernel(EncodeParams P) {
  const unsigned long long t = blockIdx.x;
  const unsigned long long r0 = t * ENC_TILE + (unsigned long long)threadIdx.x * ENC_ROWS;
  const int KB = (P.k + 3) >> 2;
  uint32_t c[ENC_ROWS];
  uint32_t mine = 0;
#pragma unroll
  for (int j = 0; j < ENC_ROWS; ++j) {
    c[j] = (r0 + j < P.n) ? __ldg(P.counts + r0 + j) : 0u;
    mine += (r0 + j < P.n && c[j] >= 255u) ? 1u : 0u;
  }
  // long-count rows of this tile before this thread's rows
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = mine;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += y;
  }
  __shared__ uint32_t s[ENC_THREADS / 32];
  if (lane == 31) s[warp] = incl;
  __syncthreads();
  uint32_t before = incl - mine;
  for (int w = 0; w < warp; ++w) before += s[w];
  unsigned long long off = P.base + r0 * (unsigned long long)(KB + 1) +
                           4ull * (P.tile_long[t] + before);
#pragma unroll 1
  for (int j = 0; j < ENC_ROWS; ++j) {
    const unsigned long long r = r0 + j;
    if (r >= P.n) break;
    uint8_t* o = P.out + off;
    if (c[j] < 255u) {
      o[0] = (uint8_t)c[j];
      o += 1;
    } else {
      o[0] = 0xFFu;
      o[1] = (uint8_t)(c[j] >> 24);
      o[2] = (uint8_t)(c[j] >> 16);
      o[3] = (uint8_t)(c[j] >> 8);
      o[4] = (uint8_t)c[j];
      o += 5;
    }
    unsigned long long key[W];
#pragma unroll
    for (int q = 0; q < W; ++q) key[q] = __ldg(P.keys + r * W + q);
    // byte b holds bases 4b..4b+3: key bits 2k-8b-1 down to 2k-8b-8
    for (int b = 0; b < KB; ++b) o[b] = (uint8_t)key_byte<W>(key, 2 * P.k - 8 * b - 8);
    off += (c[j] < 255u ? 1u : 5u) + (unsigned)KB;
  }
}

cudaError_t launch_encode_count(const uint32_t* counts, unsigned long long n,
                                unsigned long long* tile_long, cudaStream_t st) {
  const unsigned long long tiles = (n + ENC_TILE - 1) / ENC_TILE;
  if (tiles == 0) return cudaSuccess;
  encode_count_kernel<<<(unsigned)tiles, ENC_THREADS, 0, st>>>(counts, n, tile_long);
  return cudaGetLastError();
}

cudaError_t launch_encode_scan(unsigned long long* tile_long, unsigned long long ntiles,
                               unsigned long long* total, cudaStream_t st) {
  encode_scan_kernel<<<1, 1024, 0, st>>>(tile_long, ntiles, total);
  return cudaGetLastError();
}

cudaError_t launch_encode_write(const EncodeParams& p, cudaStream_t st) {
  const unsigned long long tiles = (p.n + ENC_TILE - 1) / ENC_TILE;
  if (tiles == 0) return cudaSuccess;
  const int W = (2 * p.k + 63) / 64;
  switch (W) {
#define L_ENC(w) case w: encode_write_kernel<w><<<(unsigned)tiles, ENC_THREADS, 0, st>>>(p); break;
    L_ENC(1) L_ENC(2) L_ENC(3) L_ENC(4) L_ENC(5) L_ENC(6) L_ENC(7) L_ENC(8)
    L_ENC(9) L_ENC(10) L_ENC(11) L_ENC(12) L_ENC(13) L_ENC(14) L_ENC(15)
#undef L_ENC
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

unsigned long long encode_tiles(unsigned long long n) { return (n + ENC_TILE - 1) / ENC_TILE; }

}  // namespace gerbil
