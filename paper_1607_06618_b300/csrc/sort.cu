// sort.cu -- the rows of a result in ascending key order on the device (gerbil_opts.sorted_output).
//
// Keys are 2k-bit integers in W words, word 0 most significant, so ascending integer order is
// the lexicographic order of the k-mers (A < C < G < T; App. C's byte order).  The sort is a
// least-significant-digit radix sort with 8-bit digits over the 2k key bits: one stable
// counting pass per digit moves each row (key words and count) to its place.  A pass is three
// kernels: per-tile digit counts, per-digit prefix over the tiles (plus the digit bases), and a
// stable scatter in which every warp ranks its rows among equal digits with __match_any_sync.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace gerbil {

constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 8;                          // rows per lane of a tile
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;   // 2048 rows
constexpr int SORT_WARPS = SORT_THREADS / 32;

__device__ __forceinline__ uint32_t sort_digit(const unsigned long long* __restrict__ keys,
                                               unsigned long long i, int W, int pass) {
  const int bit = pass * 8;  // 8-bit digits never straddle a 64-bit word
  return (uint32_t)(keys[i * W + (W - 1 - (bit >> 6))] >> (bit & 63)) & 0xFFu;
}

// Row i of tile t, by warp w, item u, lane l: i = t*SORT_TILE + w*256 + u*32 + l, so a warp's
// items in (u, lane) order are its rows in input order (the ranking below is stable).
__device__ __forceinline__ unsigned long long sort_row(unsigned long long t, int w, int u, int lane) {
  return t * SORT_TILE + (unsigned long long)(w * (32 * SORT_ITEMS) + u * 32 + lane);
}

__global__ void __launch_bounds__(SORT_THREADS) sort_hist_kernel(const unsigned long long* __restrict__ keys,
                                                                unsigned long long n, int W, int pass,
                                                                uint32_t* __restrict__ hist,
                                                                unsigned long long ntiles) {
  __shared__ uint32_t c[256];
  c[threadIdx.x] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int u = 0; u < SORT_ITEMS; ++u) {
    const unsigned long long i = sort_row(blockIdx.x, w, u, lane);
    if (i < n) atomicAdd(&c[sort_digit(keys, i, W, pass)], 1u);
  }
  __syncthreads();
  hist[(unsigned long long)threadIdx.x * ntiles + blockIdx.x] = c[threadIdx.x];
}

// One CTA per digit: exclusive prefix of its counts over the tiles, in place; total[d] = sum.
__global__ void __launch_bounds__(1024) sort_colscan_kernel(uint32_t* __restrict__ hist,
                                                           unsigned long long ntiles,
                                                           uint32_t* __restrict__ total) {
  __shared__ uint32_t warp_sum[32];
  __shared__ uint32_t carry;
  uint32_t* v = hist + (unsigned long long)blockIdx.x * ntiles;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (unsigned long long base = 0; base < ntiles; base += blockDim.x) {
    const unsigned long long i = base + threadIdx.x;
    const uint32_t x = i < ntiles ? v[i] : 0u;
    uint32_t incl = x;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const uint32_t ws = lane < (int)(blockDim.x >> 5) ? warp_sum[lane] : 0u;
      uint32_t wi = ws;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
        if (lane >= o) wi += y;
      }
      if (lane < (int)(blockDim.x >> 5)) warp_sum[lane] = wi - ws;
    }
    __syncthreads();
    const uint32_t c0 = carry;
    if (i < ntiles) v[i] = c0 + warp_sum[warp] + incl - x;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = c0 + warp_sum[warp] + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) total[blockIdx.x] = carry;
}

// Exclusive prefix of the 256 digit totals (one CTA of 256 threads), in place.
__global__ void __launch_bounds__(256) sort_base_kernel(uint32_t* __restrict__ total) {
  __shared__ uint32_t s[256];
  s[threadIdx.x] = total[threadIdx.x];
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (int d = 0; d < 256; ++d) {
      const uint32_t t = s[d];
      s[d] = acc;
      acc += t;
    }
  }
  __syncthreads();
  total[threadIdx.x] = s[threadIdx.x];
}

__global__ void __launch_bounds__(SORT_THREADS) sort_scatter_kernel(
    const unsigned long long* __restrict__ kin, const uint32_t* __restrict__ cin,
    unsigned long long* __restrict__ kout, uint32_t* __restrict__ cout, unsigned long long n, int W,
    int pass, const uint32_t* __restrict__ hist, const uint32_t* __restrict__ base,
    unsigned long long ntiles) {
  __shared__ uint32_t wcnt[SORT_WARPS][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int d = lane; d < 256; d += 32) wcnt[w][d] = 0;
  __syncwarp();
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t dig[SORT_ITEMS], loc[SORT_ITEMS];
  // rank within the warp: rows of equal digit in input order
#pragma unroll
  for (int u = 0; u < SORT_ITEMS; ++u) {
    const unsigned long long i = sort_row(blockIdx.x, w, u, lane);
    const bool valid = i < n;
    const uint32_t vm = __ballot_sync(0xFFFFFFFFu, valid);
    dig[u] = valid ? sort_digit(kin, i, W, pass) : 0u;
    loc[u] = 0;
    if (valid) {
      const uint32_t peers = __match_any_sync(vm, dig[u]);
      loc[u] = wcnt[w][dig[u]] + __popc(peers & lt);
      __syncwarp(vm);
      if ((peers & lt) == 0) wcnt[w][dig[u]] += __popc(peers);  // the lowest lane of the group
    }
    __syncwarp();
  }
  __syncthreads();
  // thread d: the warps' exclusive prefix for digit d, plus the tile's and the digit's bases
  {
    const int d = threadIdx.x;
    uint32_t acc = base[d] + hist[(unsigned long long)d * ntiles + blockIdx.x];
#pragma unroll
    for (int q = 0; q < SORT_WARPS; ++q) {
      const uint32_t t = wcnt[q][d];
      wcnt[q][d] = acc;
      acc += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < SORT_ITEMS; ++u) {
    const unsigned long long i = sort_row(blockIdx.x, w, u, lane);
    if (i >= n) continue;
    const unsigned long long dst = (unsigned long long)wcnt[w][dig[u]] + loc[u];
    for (int j = 0; j < W; ++j) kout[dst * W + j] = kin[i * W + j];
    cout[dst] = cin[i];
  }
}

unsigned long long sort_tiles(unsigned long long n) { return (n + SORT_TILE - 1) / SORT_TILE; }

// One LSD pass of `pass` (digit bits 8*pass .. 8*pass+7) from (kin, cin) to (kout, cout).
// hist holds 256 * sort_tiles(n) entries, total 256.
cudaError_t launch_sort_pass(const unsigned long long* kin, const uint32_t* cin,
                             unsigned long long* kout, uint32_t* cout, unsigned long long n, int W,
                             int pass, uint32_t* hist, uint32_t* total, cudaStream_t st) {
  const unsigned long long ntiles = sort_tiles(n);
  if (ntiles == 0) return cudaSuccess;
  sort_hist_kernel<<<(unsigned)ntiles, SORT_THREADS, 0, st>>>(kin, n, W, pass, hist, ntiles);
  sort_colscan_kernel<<<256, 1024, 0, st>>>(hist, ntiles, total);
  sort_base_kernel<<<1, 256, 0, st>>>(total);
  sort_scatter_kernel<<<(unsigned)ntiles, SORT_THREADS, 0, st>>>(kin, cin, kout, cout, n, W, pass, hist,
                                                                  total, ntiles);
  return cudaGetLastError();
}

}  // namespace gerbil
