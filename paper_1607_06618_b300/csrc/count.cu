// count.cu -- phase two on the GPU: split super-mers into k-mers, canonicalise, count in
// open-addressing tables (Alg. 1), spill to overflow, recount the overflow, compact under the
// min-count filter (Sec. 2.2, Sec. 2.3 Phase Two, Sec. 2.4.2, Sec. 3.3-3.4, App. A -l).
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace gerbil {

// ---- table insert (Alg. 1) -------------------------------------------------------------------
// Probe sequence: slot0 = fastrange(hash), then linear steps, at most theta probes (Alg. 1's
// trial limit).  A slot is claimed by CAS on its meta word (empty -> CLAIMED|tag, count 1);
// the claimer writes the key words and publishes with a release OR.  A prober whose tag
// matches waits (bounded) for PUBLISHED, then compares the full key (acquire ordering makes
// the key words visible).  Returns 0 on success, 1 if theta probes found no room, 2 if a
// bounded wait gave up -- both of the latter send the k-mer to the overflow area, which is
// always correct because overflow counts are added to table counts before filtering.
template <int W>
__device__ __forceinline__ int table_insert(unsigned long long* __restrict__ tab, uint32_t cap,
                                            const unsigned long long key[W], unsigned long long h,
                                            uint32_t theta, uint32_t spin_limit) {
  uint32_t s = (uint32_t)(((h & 0xFFFFFFFFull) * (unsigned long long)cap) >> 32);
  const uint32_t tagw = META_CLAIMED | (uint32_t)((h >> 35) & META_TAG_MASK);
  const unsigned long long claim = ((unsigned long long)tagw << 32) | 1ull;
  for (uint32_t t = 0; t < theta; ++t) {
    unsigned long long* slot = tab + (unsigned long long)s * (W + 1);
    unsigned long long mt = ld_acquire(slot);
    if (mt == 0ull) {
      mt = cas_acquire(slot, 0ull, claim);
      if (mt == 0ull) {
#pragma unroll
        for (int j = 0; j < W; ++j) st_relaxed(slot + 1 + j, key[j]);
        red_or_release(slot, PUB64);
        return 0;
      }
    }
    if (((uint32_t)(mt >> 32) & ~(META_PUBLISHED | META_MERGED)) == tagw) {
      uint32_t spins = 0;
      while (!(mt & PUB64)) {
        if (++spins > spin_limit) return 2;
        __nanosleep(64);
        mt = ld_acquire(slot);
      }
      bool eq = true;
#pragma unroll
      for (int j = 0; j < W; ++j) eq &= (ld_relaxed(slot + 1 + j) == key[j]);
      if (eq) {
        red_add(slot, 1ull);
        return 0;
      }
    }
    s = (s + 1 == cap) ? 0u : s + 1;
  }
  return 1;
}

// Lookup in a complete table (no concurrent inserts); marks the slot MERGED and returns its
// count, or 0 if the key is absent.
template <int W>
__device__ __forceinline__ uint32_t table_take(unsigned long long* __restrict__ tab, uint32_t cap,
                                               const unsigned long long key[W],
                                               unsigned long long h) {
  uint32_t s = (uint32_t)(((h & 0xFFFFFFFFull) * (unsigned long long)cap) >> 32);
  const uint32_t tagw = META_CLAIMED | (uint32_t)((h >> 35) & META_TAG_MASK);
  for (uint32_t t = 0; t < cap; ++t) {
    unsigned long long* slot = tab + (unsigned long long)s * (W + 1);
    const unsigned long long mt = slot[0];
    if (mt == 0ull) return 0;
    if (((uint32_t)(mt >> 32) & ~(META_PUBLISHED | META_MERGED)) == tagw) {
      bool eq = true;
#pragma unroll
      for (int j = 0; j < W; ++j) eq &= (slot[1 + j] == key[j]);
      if (eq) {
        atom_or(slot, MERGED64);
        return (uint32_t)mt;
      }
    }
    s = (s + 1 == cap) ? 0u : s + 1;
  }
  return 0;
}

template <int W>
__device__ __forceinline__ void to_overflow(const CountParams& P, uint32_t widx,
                                            const unsigned long long key[W], int why) {
  if (why == 2) atomicAdd(&P.ctr->spin_demotions, 1ull);
  const unsigned long long idx = atomicAdd(&P.ctr->ovf_count, 1ull);
  if (idx < P.ovf_cap) {
#pragma unroll
    for (int j = 0; j < W; ++j) P.ovf[idx * W + j] = key[j];
  } else {
    set_err(P.ctr, ERR_OVF_FULL);
  }
  atomicAdd(P.bin_ovf + widx, 1u);
}

// ---- one tile of one bin: extract, canonicalise, insert ----------------------------------------
struct TileSmem {
  unsigned long long pos[COUNT_TILE];
  uint32_t koff[COUNT_TILE];
  uint32_t widx, tile, s_lo, ns;
};

// Last super-mer index s in [lo, hi) with koff[s] <= j (koff ascending within a bin).
__device__ __forceinline__ uint32_t last_le(const uint32_t* __restrict__ koff, uint32_t lo,
                                            uint32_t hi, uint32_t j) {
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(koff + mid) <= j) lo = mid; else hi = mid;
  }
  return lo;
}

template <int W>
__device__ __forceinline__ void count_tile(const CountParams& P, TileSmem& S) {
  // thread 0 located the bin (S.widx) and the tile within it (S.tile)
  const BinWork wk = P.work[S.widx];
  const uint32_t j0 = S.tile * COUNT_TILE;
  const uint32_t j1 = min(j0 + (uint32_t)COUNT_TILE, wk.n_kmers);
  const uint32_t* koff = P.sm_koff + wk.sm_begin;
  const unsigned long long* spos = P.sm_pos + wk.sm_begin;
  if (threadIdx.x == 0) {
    const uint32_t lo = last_le(koff, 0, wk.n_super, j0);
    const uint32_t hi = last_le(koff, lo, wk.n_super, j1 - 1);
    S.s_lo = lo;
    S.ns = hi - lo + 1;
    if (S.ns > (uint32_t)COUNT_TILE) {  // descriptors out of order: never expected
      set_err(P.ctr, ERR_STATE);
      S.ns = 0;
    }
  }
  __syncthreads();
  const uint32_t s_lo = S.s_lo, ns = S.ns;
  for (uint32_t i = threadIdx.x; i < ns; i += blockDim.x) {
    S.koff[i] = __ldg(koff + s_lo + i);
    S.pos[i] = __ldg(spos + s_lo + i);
  }
  __syncthreads();
  unsigned long long* tab = P.arena + wk.table_off * (W + 1);
#pragma unroll 1
  for (int r = 0; r < KMERS_PER_THREAD; ++r) {
    const uint32_t j = j0 + threadIdx.x + r * COUNT_THREADS;
    if (j >= j1 || ns == 0) break;
    uint32_t lo = 0, hi = ns;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (S.koff[mid] <= j) lo = mid; else hi = mid;
    }
    const unsigned long long pos = S.pos[lo] + (j - S.koff[lo]);
    unsigned long long key[W];
    load_kmer<W>(P.packed, pos, P.k, key);
    if (P.canonical) {
      unsigned long long rc[W];
      revcomp<W>(key, P.k, rc);
      if (key_less<W>(rc, key)) {
#pragma unroll
        for (int q = 0; q < W; ++q) key[q] = rc[q];
      }
    }
    const unsigned long long h = key_hash<W>(key);
    const int res = table_insert<W>(tab, wk.cap, key, h, P.theta, P.spin_limit);
    if (res) to_overflow<W>(P, S.widx, key, res);
  }
  __syncthreads();  // S is reused by the next tile
}

__device__ __forceinline__ void locate_tile(const CountParams& P, uint32_t gtile, TileSmem& S) {
  // last work entry whose tile_begin <= gtile
  uint32_t lo = 0, hi = P.nwork;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (P.work[mid].tile_begin <= gtile) lo = mid; else hi = mid;
  }
  S.widx = lo;
  S.tile = gtile - P.work[lo].tile_begin;
}

// Grid form: one CTA per tile.
template <int W>
__global__ void __launch_bounds__(COUNT_THREADS) insert_kernel(CountParams P) {
  __shared__ TileSmem S;
  if (threadIdx.x == 0) locate_tile(P, P.tile_base + blockIdx.x, S);
  __syncthreads();
  count_tile<W>(P, S);
}

// Persistent form: CTAs pop tile indices from a device work queue (tiles ordered by bin, so
// the bins in flight at any moment are few and their tables stay hot in L2).
template <int W>
__global__ void __launch_bounds__(COUNT_THREADS) insert_persistent_kernel(CountParams P) {
  __shared__ TileSmem S;
  __shared__ uint32_t next;
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned long long t = atomicAdd(&P.ctr->queue_head, 1ull);
      next = (t < P.ntiles) ? (uint32_t)t : 0xFFFFFFFFu;
      if (next != 0xFFFFFFFFu) locate_tile(P, next, S);
    }
    __syncthreads();
    if (next == 0xFFFFFFFFu) break;
    count_tile<W>(P, S);
  }
}

// ---- compaction under min_count (App. A -l) ----------------------------------------------------
__device__ __forceinline__ uint32_t work_of_slot(const BinWork* work, uint32_t nwork,
                                                 unsigned long long slot) {
  uint32_t lo = 0, hi = nwork;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (work[mid].table_off <= slot) lo = mid; else hi = mid;
  }
  return lo;
}

template <int W>
__device__ __forceinline__ void emit_rows(bool emit, const unsigned long long key[W], uint32_t c,
                                         unsigned long long* out_keys, uint32_t* out_counts,
                                         unsigned long long out_cap, Counters* ctr) {
  const unsigned int lane = threadIdx.x & 31;
  const unsigned int bal = __ballot_sync(0xFFFFFFFFu, emit);
  if (!bal) return;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(&ctr->out_count, (unsigned long long)__popc(bal));
  base = __shfl_sync(0xFFFFFFFFu, base, 0);
  if (emit) {
    const unsigned long long idx = base + __popc(bal & ((1u << lane) - 1u));
    if (idx < out_cap) {
#pragma unroll
      for (int j = 0; j < W; ++j) out_keys[idx * W + j] = key[j];
      out_counts[idx] = c;
    } else {
      set_err(ctr, ERR_OUT_FULL);
    }
  }
}

template <int W>
__global__ void __launch_bounds__(256) compact_kernel(CompactParams P) {
  const bool any_ovf = P.ctr->ovf_count != 0ull;
  const unsigned long long nthreads = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long warp0 = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) & ~31ull;
  const unsigned int lane = threadIdx.x & 31;
  unsigned long long ndist = 0;
  for (unsigned long long base = P.slot_lo + warp0; base < P.slot_hi; base += nthreads) {
    const unsigned long long slot = base + lane;
    bool emit = false;
    unsigned long long key[W];
    uint32_t c = 0;
    if (slot < P.slot_hi) {
      const unsigned long long* sp = P.arena + slot * (W + 1);
      const unsigned long long mt = sp[0];
      bool live = mt != 0ull;
      if (live && !(mt & PUB64)) {
        set_err(P.ctr, ERR_STATE);
        live = false;
      }
      bool take = live;
      if (live && any_ovf) {
        const uint32_t wi = work_of_slot(P.work, P.nwork, slot);
        const bool deferred = P.bin_ovf[wi] != 0u;
        take = (P.mode == 0) ? !deferred : deferred;
      } else if (P.mode == 1) {
        take = false;
      }
      if (take) {
        ++ndist;
#pragma unroll
        for (int j = 0; j < W; ++j) key[j] = sp[1 + j];
        c = (uint32_t)mt;
        if (P.mode == 1) {
          const uint32_t extra = table_take<W>(P.otab, P.ocap, key, key_hash<W>(key));
          if (extra) atomicAdd(&P.ctr->merged, 1ull);
          c += extra;
        }
        emit = c >= P.min_count;
      }
    }
    emit_rows<W>(emit, key, c, P.out_keys, P.out_counts, P.out_cap, P.ctr);
  }
  // distinct keys of the main tables (overflow-only keys are added by the overflow emit)
  for (int o = 16; o > 0; o >>= 1) ndist += __shfl_down_sync(0xFFFFFFFFu, ndist, o);
  if (lane == 0 && ndist) atomicAdd(&P.ctr->distinct, ndist);
}

// ---- overflow recount (Sec. 3.4 "Probing Strategy": the emergency area is counted after the
// file) -- a fresh table sized for all overflow k-mers, probed without a trial limit -----------
template <int W>
__global__ void __launch_bounds__(256) overflow_insert_kernel(OverflowParams P) {
  const unsigned long long n = min(P.ctr->ovf_count, P.ovf_cap);
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    unsigned long long key[W];
#pragma unroll
    for (int j = 0; j < W; ++j) key[j] = P.ovf[i * W + j];
    const int res = table_insert<W>(P.otab, P.ocap, key, key_hash<W>(key), P.ocap, P.spin_limit);
    if (res) set_err(P.ctr, ERR_SPIN);
  }
}

// Keys that exist only in the overflow table (not merged into a main-table key).
template <int W>
__global__ void __launch_bounds__(256) overflow_emit_kernel(OverflowParams P) {
  const unsigned long long nthreads = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long warp0 = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) & ~31ull;
  const unsigned int lane = threadIdx.x & 31;
  unsigned long long ndist = 0;
  for (unsigned long long base = warp0; base < P.ocap; base += nthreads) {
    const unsigned long long slot = base + lane;
    bool emit = false;
    unsigned long long key[W];
    uint32_t c = 0;
    if (slot < P.ocap) {
      const unsigned long long* sp = P.otab + slot * (W + 1);
      const unsigned long long mt = sp[0];
      if (mt != 0ull && !(mt & MERGED64)) {
        ++ndist;
#pragma unroll
        for (int j = 0; j < W; ++j) key[j] = sp[1 + j];
        c = (uint32_t)mt;
        emit = c >= P.min_count;
      }
    }
    emit_rows<W>(emit, key, c, P.out_keys, P.out_counts, P.out_cap, P.ctr);
  }
  for (int o = 16; o > 0; o >>= 1) ndist += __shfl_down_sync(0xFFFFFFFFu, ndist, o);
  if (lane == 0 && ndist) atomicAdd(&P.ctr->distinct, ndist);
}

// ---- launchers (W dispatch) ---------------------------------------------------------------------
#define GERBIL_W_SWITCH(W, CALL)          \
  switch (W) {                            \
    case 1: CALL(1); break;               \
    case 2: CALL(2); break;               \
    case 3: CALL(3); break;               \
    case 4: CALL(4); break;               \
    case 5: CALL(5); break;               \
    case 6: CALL(6); break;               \
    case 7: CALL(7); break;               \
    case 8: CALL(8); break;               \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t launch_insert(int W, const CountParams& p, unsigned grid, cudaStream_t st) {
  if (grid == 0) return cudaSuccess;
#define L_INSERT(w) insert_kernel<w><<<grid, COUNT_THREADS, 0, st>>>(p)
  GERBIL_W_SWITCH(W, L_INSERT)
#undef L_INSERT
  return cudaGetLastError();
}

cudaError_t launch_insert_persistent(int W, const CountParams& p, unsigned grid, cudaStream_t st) {
  if (grid == 0) return cudaSuccess;
#define L_PINSERT(w) insert_persistent_kernel<w><<<grid, COUNT_THREADS, 0, st>>>(p)
  GERBIL_W_SWITCH(W, L_PINSERT)
#undef L_PINSERT
  return cudaGetLastError();
}

cudaError_t launch_compact(int W, const CompactParams& p, int nsm, cudaStream_t st) {
  const unsigned long long n = p.slot_hi - p.slot_lo;
  if (n == 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::min<unsigned long long>((n + 255) / 256, (unsigned long long)nsm * 8);
#define L_COMPACT(w) compact_kernel<w><<<grid, 256, 0, st>>>(p)
  GERBIL_W_SWITCH(W, L_COMPACT)
#undef L_COMPACT
  return cudaGetLastError();
}

cudaError_t launch_overflow_insert(int W, const OverflowParams& p, int nsm, cudaStream_t st) {
  const unsigned grid = (unsigned)nsm * 4;
#define L_OINS(w) overflow_insert_kernel<w><<<grid, 256, 0, st>>>(p)
  GERBIL_W_SWITCH(W, L_OINS)
#undef L_OINS
  return cudaGetLastError();
}

cudaError_t launch_overflow_emit(int W, const OverflowParams& p, int nsm, cudaStream_t st) {
  const unsigned grid = (unsigned)std::min<unsigned long long>(((unsigned long long)p.ocap + 255) / 256,
                                                          (unsigned long long)nsm * 8);
#define L_OEMIT(w) overflow_emit_kernel<w><<<grid, 256, 0, st>>>(p)
  GERBIL_W_SWITCH(W, L_OEMIT)
#undef L_OEMIT
  return cudaGetLastError();
}

}  // namespace gerbil
