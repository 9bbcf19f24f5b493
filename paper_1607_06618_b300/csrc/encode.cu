// encode.cu -- App. C output records on the GPU.
//
// A record is the count -- one byte when below 255, else the byte 0xFF followed by the count as
// a big-endian 32-bit integer -- then the k-mer with four bases per byte (A=00 C=01 G=10 T=11,
// first base in the two high bits of the first byte; the unused low bits of the last byte are
// written as 0).  Every record is KB+1 or KB+5 bytes (KB = ceil(k/4)), so the byte offset of row
// i is i*(KB+1) + 4*(rows before i with count >= 255): the encoder counts long-count rows per
// tile, scans the tile sums, then writes every tile's records from its own offset.
#include <algorithm>

#include "../../include/gerbil.h"
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

// Record writer.  A CTA takes one tile of ENC_TILE rows, a warp 32 consecutive rows (a chunk,
// one row per lane) at a time.  The lanes write their records into the warp's shared buffer,
// placed so that buffer and output agree modulo 16 bytes; the warp then copies the chunk's
// bytes out with 16-byte stores, and byte stores for the partial 16 bytes at either end (the
// neighbouring chunks own the other bytes there).  Chunk offsets within the tile come from a
// per-chunk count of long-count rows (ballot) and one scan over the tile's chunks.
constexpr int ENC_CHUNKS = ENC_TILE / 32;
constexpr int ENC_WARPS = ENC_THREADS / 32;
constexpr int ENC_MAX_REC = (GERBIL_MAX_K + 3) / 4 + 5;       // longest record
constexpr int ENC_BUF = (32 * ENC_MAX_REC + 16 + 15) / 16 * 16;  // per warp, 16-byte multiple

template <int W>
__global__ void __launch_bounds__(ENC_THREADS) encode_write_kernel(EncodeParams P) {
  __shared__ uint32_t s_long[ENC_CHUNKS];  // long-count rows per chunk, then their prefix
  __shared__ __align__(16) uint8_t s_buf[ENC_WARPS][ENC_BUF];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned long long t = blockIdx.x;
  const unsigned long long row0 = t * ENC_TILE;
  const int k = P.k;
  const int KB = (k + 3) >> 2;
  constexpr int CPW = ENC_CHUNKS / ENC_WARPS;  // chunks per warp: warp w takes w, w + 8, ...
  uint32_t cnt[CPW], lng[CPW];
#pragma unroll
  for (int i = 0; i < CPW; ++i) {
    const unsigned long long r = row0 + (unsigned long long)(warp + ENC_WARPS * i) * 32 + lane;
    cnt[i] = r < P.n ? __ldg(P.counts + r) : 0u;
    lng[i] = __ballot_sync(0xFFFFFFFFu, r < P.n && cnt[i] >= 255u);
    if (lane == 0) s_long[warp + ENC_WARPS * i] = __popc(lng[i]);
  }
  __syncthreads();
  if (warp == 0) {  // exclusive prefix over the tile's chunks, two per lane
    const uint32_t a = s_long[2 * lane], b = s_long[2 * lane + 1];
    uint32_t incl = a + b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += y;
    }
    const uint32_t ex = incl - a - b;
    __syncwarp();
    s_long[2 * lane] = ex;
    s_long[2 * lane + 1] = ex + a;
  }
  __syncthreads();
  const unsigned long long tile_off =
      P.base + row0 * (unsigned long long)(KB + 1) + 4ull * P.tile_long[t];
  const int s = 8 * KB - 2 * k;  // left shift that ends the key on a byte boundary (0..6)
  const int skip = 8 * W - KB;   // leading zero bytes of the shifted W-word key
  uint8_t* buf = s_buf[warp];
#pragma unroll
  for (int i = 0; i < CPW; ++i) {  // unrolled: cnt and lng stay in registers
    const int c = warp + ENC_WARPS * i;
    const unsigned long long r = row0 + (unsigned long long)c * 32 + lane;
    if (row0 + (unsigned long long)c * 32 >= P.n) break;  // the same for the whole warp
    const int nrows = (int)min(32ull, P.n - (row0 + (unsigned long long)c * 32));
    const unsigned long long g0 = tile_off + (unsigned long long)c * 32 * (KB + 1) + 4ull * s_long[c];
    const int a0 = (int)(((uintptr_t)P.out + g0) & 15);  // the buffer's byte a0 goes to out + g0
    const int bytes = nrows * (KB + 1) + 4 * __popc(lng[i]);
    if (lane < nrows) {
      uint8_t* o = buf + a0 + lane * (KB + 1) + 4 * __popc(lng[i] & ((1u << lane) - 1u));
      const uint32_t cv = cnt[i];
      if (cv < 255u) {
        *o++ = (uint8_t)cv;
      } else {
        o[0] = 0xFFu;
        o[1] = (uint8_t)(cv >> 24);
        o[2] = (uint8_t)(cv >> 16);
        o[3] = (uint8_t)(cv >> 8);
        o[4] = (uint8_t)cv;
        o += 5;
      }
      unsigned long long key[W];
#pragma unroll
      for (int q = 0; q < W; ++q) key[q] = __ldg(P.keys + r * W + q);
      if (s) {
#pragma unroll
        for (int q = 0; q < W; ++q)
          key[q] = (key[q] << s) | (q + 1 < W ? key[q + 1] >> (64 - s) : 0ull);
      }
      // big-endian bytes of the shifted key, the first `skip` (zero) bytes left out
#pragma unroll
      for (int q = 0; q < W; ++q)
#pragma unroll
        for (int y = 0; y < 8; ++y) {
          const int B = 8 * q + y - skip;
          if (B >= 0) o[B] = (uint8_t)(key[q] >> (56 - 8 * y));
        }
    }
    __syncwarp();
    // copy buf[a0, a0 + bytes) to out[g0, g0 + bytes)
    uint8_t* dst = P.out + (g0 - (unsigned long long)a0);  // 16-byte aligned
    const int e = a0 + bytes;
    const int h1 = min(16, e);  // head: bytes a0 .. 15 of the first 16
    if (lane >= a0 && lane < h1) dst[lane] = buf[lane];
    const int t0 = max(16, e & ~15);  // tail: the last partial 16, past the head
    if (lane < 16 && t0 + lane < e) dst[t0 + lane] = buf[t0 + lane];
    for (int x = 16 + 16 * lane; x + 16 <= e; x += 512)
      *reinterpret_cast<uint4*>(dst + x) = *reinterpret_cast<const uint4*>(buf + x);
    __syncwarp();
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
