// count.cu -- phase two on the GPU: split super-mers into k-mers, canonicalise, count in
// open-addressing tables (Alg. 1), spill to overflow, recount the overflow, compact under the
// min-count filter (Sec. 2.2, Sec. 2.3 Phase Two, Sec. 2.4.2, Sec. 3.3-3.4, App. A -l).
#include <algorithm>

#include "common.cuh"
#include "insert.cuh"
#include "kernels.h"

namespace gerbil {

// ---- warp work items: extract, canonicalise, insert --------------------------------------------
// The k-mers of a bin are cut into items of wk.item_kmers (64, 128 or 256) consecutive k-mers
// (bin order).  Item i is done by one warp; imap[i] = (work index << 32 | first super-mer of
// the item), built by item_map_kernel, so a warp starts without searching.  The warp loads the
// item's super-mer descriptors into its own shared-memory slice; each lane then takes
// item_kmers/32 consecutive k-mers of the item, reads its bases through L1 and inserts.  No
// CTA-wide barrier is involved.

// One thread per work item: its work entry (the last with item_begin <= item) and, within the
// bin, the last super-mer whose first k-mer is at most the item's first k-mer (both binary
// searches), so that every thread does the same work whatever the bins' sizes.
__global__ void __launch_bounds__(256) item_map_kernel(const BinWork* __restrict__ work, uint32_t nwork,
                                                      const uint32_t* __restrict__ sm_koff,
                                                      unsigned long long* __restrict__ imap,
                                                      unsigned long long nitems) {
  for (unsigned long long it = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; it < nitems;
       it += (unsigned long long)gridDim.x * blockDim.x) {
    uint32_t lo = 0, hi = nwork;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (__ldg(&work[mid].item_begin) <= it) lo = mid; else hi = mid;
    }
    const unsigned long long j0 = (it - __ldg(&work[lo].item_begin)) * (unsigned long long)__ldg(&work[lo].item_kmers);
    const uint32_t* koff = sm_koff + __ldg(&work[lo].sm_begin);
    uint32_t a = 0, b = __ldg(&work[lo].n_super);
    while (b - a > 1) {
      const uint32_t mid = (a + b) >> 1;
      if (__ldg(koff + mid) <= j0) a = mid; else b = mid;
    }
    imap[it] = ((unsigned long long)lo << 32) | a;
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

// CTA-cooperative append: every thread contributes e rows; one atomic per CTA returns the base
// and an exclusive scan over the CTA gives every thread its first row.
__device__ __forceinline__ unsigned long long cta_append(uint32_t e, Counters* ctr,
                                                         uint32_t* wsum, unsigned long long* cbase) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  uint32_t incl = e;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (int i = 0; i < nwarp; ++i) {
      const uint32_t t = wsum[i];
      wsum[i] = acc;
      acc += t;
    }
    *cbase = acc ? atomicAdd(&ctr->out_count, (unsigned long long)acc) : 0ull;
  }
  __syncthreads();
  const unsigned long long first = *cbase + wsum[warp] + incl - e;
  __syncthreads();  // wsum / cbase are reused by the next call
  return first;
}

// Resident CTAs per SM the registers are held to: 4 while the slots held in flight fit without
// spills (slots of up to 64 bytes), else 3 (measured on k = 65: 3 -> 4 CTAs, 0.637 -> 0.605 ms;
// 6 or 8 slots in flight per thread were slower)
constexpr int compact_min_blocks(int SW) { return SW <= 8 ? 4 : 3; }
template <int W, int WS>
__global__ void __launch_bounds__(256, compact_min_blocks(slot_words(WS))) compact_kernel(CompactParams P) {
  constexpr int SW = slot_words(WS);
  constexpr int COMPACT_UNROLL = SW <= 4 ? 4 : 2;
  __shared__ uint32_t wsum[8];
  __shared__ unsigned long long cbase;
  const bool any_ovf = P.ctr->ovf_count != 0ull;
  unsigned long long ndist = 0;
  const unsigned long long chunk = (unsigned long long)blockDim.x * COMPACT_UNROLL;
  for (unsigned long long cb = P.slot_lo + blockIdx.x * chunk; cb < P.slot_hi;
       cb += (unsigned long long)gridDim.x * chunk) {
    unsigned long long v[COMPACT_UNROLL][SW];
#pragma unroll
    for (int u = 0; u < COMPACT_UNROLL; ++u) {
      const unsigned long long slot = cb + u * blockDim.x + threadIdx.x;
      if (slot < P.slot_hi) {
        load_slot<SW>(P.arena + slot * SW, v[u]);  // 32-byte loads where the slot allows
      } else {
#pragma unroll
        for (int i = 0; i < SW; ++i) v[u][i] = 0ull;
      }
    }
    uint32_t cnt[COMPACT_UNROLL];
    uint32_t e = 0;
#pragma unroll
    for (int u = 0; u < COMPACT_UNROLL; ++u) {
      const unsigned long long slot = cb + u * blockDim.x + threadIdx.x;
      const unsigned long long mt = v[u][0];
      bool live = mt != 0ull;
      if (live) {
        bool all = true;
#pragma unroll
        for (int j = 0; j < WS; ++j) all &= (v[u][1 + j] & MARK) != 0ull;
        if (!all) {  // a claimed slot whose key was never written: never expected
          set_err(P.ctr, ERR_STATE);
          live = false;
        }
      }
      // mode 0: bins without overflow; 1: bins with overflow, merged; 2: count rows only
      bool take = live && P.mode != 1;
      if (live && any_ovf && P.mode != 2) {
        const uint32_t wi = work_of_slot(P.work, P.nwork, slot);
        const bool deferred = P.bin_ovf[wi] != 0u;
        take = (P.mode == 0) ? !deferred : deferred;
      }
      uint32_t c = 0;
      if (take) {
        ++ndist;
        c = (uint32_t)mt;
        if (P.zero && P.mode != 2) {  // the slot is read (v) and done with: leave it empty
          ulonglong2* sp = reinterpret_cast<ulonglong2*>(P.arena + slot * SW);
#pragma unroll
          for (int i = 0; i < SW / 2; ++i) sp[i] = make_ulonglong2(0ull, 0ull);
        }
        if (P.mode == 1) {
          unsigned long long key[W];
          from_stored<W, WS>(&v[u][1], (uint32_t)(mt >> 32), key);
          const uint32_t extra = table_take<WS>(P.otab, P.ocap, &v[u][1], (uint32_t)(mt >> 32),
                                                key_hash<W>(key));
          if (extra) atomicAdd(&P.ctr->merged, 1ull);
          c += extra;
        }
        if (c < P.min_count) c = 0;
      }
      cnt[u] = c;
      e += c ? 1u : 0u;
    }
    unsigned long long row = cta_append(e, P.ctr, wsum, &cbase);
    if (P.mode == 2) continue;  // counting only
#pragma unroll
    for (int u = 0; u < COMPACT_UNROLL; ++u) {
      if (!cnt[u]) continue;
      if (row < P.out_cap) {
        unsigned long long key[W];
        from_stored<W, WS>(&v[u][1], (uint32_t)(v[u][0] >> 32), key);
#pragma unroll
        for (int j = 0; j < W; ++j) P.out_keys[row * W + j] = key[j];
        P.out_counts[row] = cnt[u];
      } else {
        set_err(P.ctr, ERR_OUT_FULL);
      }
      ++row;
    }
  }
  for (int o = 16; o > 0; o >>= 1) ndist += __shfl_down_sync(0xFFFFFFFFu, ndist, o);
  if ((threadIdx.x & 31) == 0 && ndist) atomicAdd(&P.ctr->distinct, ndist);
}

// Warp-cooperative append of the rows whose lane has emit set: one atomic per warp (used by the
// overflow-only emission, whose table is small).
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

// ---- fused persistent phase two --------------------------------------------------------------
// One queue holds, in bin order, the insert items of bin b followed by the compaction chunks of
// bin b-1.  Warps pop tasks; a compaction chunk waits (bounded) until every insert item of its
// bin is done, an insert item waits until the bin that used its table region before has been
// compacted.  Both waits are on tasks that were popped earlier by running warps, so they end.
// Tables of small bins live in a ring that fits in L2; compaction zeroes every slot it reads,
// so a region is clean when the next bin takes it, and the whole arena is zero after a call.

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Lane 0 waits with acquire loads until *ctr >= target (bounded by wait_ns; on timeout the
// error is recorded and the wait ends).
__device__ __forceinline__ void warp_wait_at_least(const uint32_t* ctr, uint32_t target,
                                                   unsigned long long wait_ns, Counters* c, int lane) {
  if (lane == 0 && ld_acquire_u32(ctr) < target) {  // (the acquire orders lane 0's loads)
    const unsigned long long t0 = globaltimer_ns();
    unsigned ns = 32;
    while (ld_acquire_u32(ctr) < target) {
      if (globaltimer_ns() - t0 > wait_ns) {
        set_err(c, ERR_QUEUE);
        break;
      }
      __nanosleep(ns);
      if (ns < 1024) ns *= 2;
    }
  }
  // the other lanes are ordered after lane 0's acquire by the warp barrier
  __syncwarp();
}

// Self-test of the bounded wait above: one warp waits for a flag that nothing sets, so the
// wait runs out after wait_ns, records ERR_QUEUE and the kernel returns.
__global__ void __launch_bounds__(32) wait_selftest_kernel(const uint32_t* flag,
                                                          unsigned long long wait_ns, Counters* c) {
  warp_wait_at_least(flag, 1u, wait_ns, c, (int)(threadIdx.x & 31));
}

cudaError_t launch_wait_selftest(const uint32_t* flag, unsigned long long wait_ns, Counters* c,
                                 cudaStream_t st) {
  wait_selftest_kernel<<<1, 32, 0, st>>>(flag, wait_ns, c);
  return cudaGetLastError();
}

// Every lane makes its writes visible, then lane 0 counts the task as done.
__device__ __forceinline__ void warp_signal(uint32_t* ctr, int lane) {
  __threadfence();
  __syncwarp();
  if (lane == 0) atomicAdd(ctr, 1u);
}

__device__ __forceinline__ uint32_t warp_excl_scan(uint32_t x, int lane, uint32_t* total) {
  uint32_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += y;
  }
  *total = __shfl_sync(0xFFFFFFFFu, incl, 31);
  return incl - x;
}

// One compaction chunk: count the rows (meta words only), take room for them with one atomic,
// then write them and zero the live slots.  Loads are issued in batches (all of a batch before
// any is used), since a warp issues in order and would otherwise wait once per slot.
constexpr int CB_META = 8;  // meta words per lane per batch (count pass)
constexpr int CB_SLOT = 4;  // slots per lane per batch (write pass)

template <int W, int WS>
__device__ __forceinline__ void compact_chunk(const FusedParams& F, const BinWork& wk, uint32_t c,
                                              int lane) {
  constexpr int SW = slot_words(WS);
  unsigned long long* tab = F.c.arena + wk.table_off * SW;
  const uint32_t lo = c * CHUNK_SLOTS, hi = min(lo + (uint32_t)CHUNK_SLOTS, wk.cap);
  uint32_t mine = 0, live = 0;
  for (uint32_t b0 = lo; b0 < hi; b0 += 32 * CB_META) {
    unsigned long long mt[CB_META];
#pragma unroll
    for (int u = 0; u < CB_META; ++u) {
      const uint32_t s = b0 + u * 32 + lane;
      mt[u] = s < hi ? ld_relaxed(tab + (unsigned long long)s * SW) : 0ull;
    }
#pragma unroll
    for (int u = 0; u < CB_META; ++u) {
      live += mt[u] != 0ull;
      mine += (mt[u] != 0ull && (uint32_t)mt[u] >= F.min_count);
    }
  }
  uint32_t total = 0, tlive = 0;
  const uint32_t excl = warp_excl_scan(mine, lane, &total);
  (void)warp_excl_scan(live, lane, &tlive);
  unsigned long long base = 0;
  if (lane == 0) {
    if (total) base = atomicAdd(&F.c.ctr->out_count, (unsigned long long)total);
    if (tlive) atomicAdd(&F.c.ctr->distinct, (unsigned long long)tlive);
  }
  unsigned long long row = __shfl_sync(0xFFFFFFFFu, base, 0) + excl;
  for (uint32_t b0 = lo; b0 < hi; b0 += 32 * CB_SLOT) {
    unsigned long long v[CB_SLOT][SW];
#pragma unroll
    for (int u = 0; u < CB_SLOT; ++u) {
      const uint32_t s = b0 + u * 32 + lane;
      if (s < hi) {
        load_slot<SW>(tab + (unsigned long long)s * SW, v[u]);
      } else {
#pragma unroll
        for (int i = 0; i < SW; ++i) v[u][i] = 0ull;
      }
    }
#pragma unroll
    for (int u = 0; u < CB_SLOT; ++u) {
      if (v[u][0] == 0ull) continue;
      unsigned long long* sp = tab + (unsigned long long)(b0 + u * 32 + lane) * SW;
      bool all = true;
#pragma unroll
      for (int j = 0; j < WS; ++j) all &= (v[u][1 + j] & MARK) != 0ull;
      if (!all) set_err(F.c.ctr, ERR_STATE);  // a claimed slot whose key was never written
      if ((uint32_t)v[u][0] >= F.min_count) {
        if (row < F.out_cap) {
          unsigned long long key[W];
          from_stored<W, WS>(&v[u][1], (uint32_t)(v[u][0] >> 32), key);
#pragma unroll
          for (int j = 0; j < W; ++j) F.out_keys[row * W + j] = key[j];
          F.out_counts[row] = (uint32_t)v[u][0];
        } else {
          set_err(F.c.ctr, ERR_OUT_FULL);
        }
        ++row;
      }
#pragma unroll
      for (int i = 0; i < SW; i += 2) st_relaxed_v2(sp + i, 0ull, 0ull);
    }
  }
}

template <int W, int WS>
__global__ void __launch_bounds__(256) fused_kernel(FusedParams F) {
  __shared__ WarpSmem S[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned long long* queue = F.queue;
  uint32_t checked = 0xFFFFFFFFu;  // bin whose dependencies this warp has seen complete
  unsigned long long t = 0;
  if (lane == 0) t = atomicAdd(queue, 1ull);
  t = __shfl_sync(0xFFFFFFFFu, t, 0);
  // a warp holds its current task and the next one, whose atomic is in flight meanwhile; a
  // task only ever waits on tasks queued before it, so holding a later one cannot block
  for (;;) {
    if (t >= F.ntasks) break;
    unsigned long long t_next = 0;
    if (lane == 0) t_next = atomicAdd(queue, 1ull);
    const unsigned long long e = __ldg(F.tasks + t);
    const uint32_t wi = (uint32_t)(e >> 32) & 0x7FFFFFFFu, pay = (uint32_t)e;
    const BinWork wk = F.c.work[wi];
    if (!(e >> 63)) {
      if (wi != checked) {  // completed dependencies stay complete
        for (uint32_t d = 0; d < wk.dep_count; ++d) {
          const uint32_t dw = __ldg(F.deps + wk.dep_begin + d);
          warp_wait_at_least(F.chunks_done + dw, F.c.work[dw].n_chunks, F.wait_ns, F.c.ctr, lane);
        }
        checked = wi;
      }
      insert_item<W, WS>(F.c, wi, wk, (uint32_t)(t - wk.task_insert), pay, S[warp], lane);
      warp_signal(F.items_done + wi, lane);
    } else {
      warp_wait_at_least(F.items_done + wi, wk.n_items, F.wait_ns, F.c.ctr, lane);
      compact_chunk<W, WS>(F, wk, pay, lane);
      warp_signal(F.chunks_done + wi, lane);
    }
    t = __shfl_sync(0xFFFFFFFFu, t_next, 0);
  }
}

// Queue entries: the insert items of every bin (first super-mer of each item) and its
// compaction chunks, at the positions the host gave each bin.
__global__ void __launch_bounds__(256) task_map_kernel(FusedParams F) {
  for (uint32_t wi = blockIdx.x; wi < F.c.nwork; wi += gridDim.x) {
    const BinWork wk = F.c.work[wi];
    const uint32_t* koff = F.c.sm_koff + wk.sm_begin;
    unsigned long long* tasks = const_cast<unsigned long long*>(F.tasks);
    for (uint32_t s = threadIdx.x; s < wk.n_super; s += blockDim.x) {
      const unsigned long long a = koff[s];
      const unsigned long long b = (s + 1 < wk.n_super) ? koff[s + 1] : wk.n_kmers;
      for (unsigned long long t = (a + ITEM_KMERS - 1) / ITEM_KMERS; t * ITEM_KMERS < b; ++t)
        tasks[wk.task_insert + t] = ((unsigned long long)wi << 32) | s;
    }
    for (uint32_t c = threadIdx.x; c < wk.n_chunks; c += blockDim.x)
      tasks[wk.task_compact + c] = (1ull << 63) | ((unsigned long long)wi << 32) | c;
  }
}

// ---- overflow recount (Sec. 3.4 "Probing Strategy": the emergency area is counted after the
// file) -- a fresh table sized for all overflow k-mers, probed without a trial limit -----------
template <int W, int WS>
__global__ void __launch_bounds__(256) overflow_insert_kernel(OverflowParams P) {
  const unsigned long long n = min(P.ctr->ovf_count, P.ovf_cap);
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    unsigned long long key[W];
#pragma unroll
    for (int j = 0; j < W; ++j) key[j] = P.ovf[i * W + j];
    unsigned long long st[WS];
    to_stored<W, WS>(key, st);
    const int res = table_insert<WS>(P.otab, P.ocap, st, key_tag<W>(key), key_hash<W>(key), P.ocap,
                                     P.spin_limit);
    if (res) set_err(P.ctr, ERR_SPIN);
  }
}

// Keys that exist only in the overflow table (not merged into a main-table key).
template <int W, int WS>
__global__ void __launch_bounds__(256) overflow_emit_kernel(OverflowParams P) {
  constexpr int SW = slot_words(WS);
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
      const unsigned long long* sp = P.otab + slot * SW;
      const unsigned long long mt = sp[0];
      if (mt != 0ull && !(mt & MERGED64)) {
        ++ndist;
        unsigned long long st[WS];
#pragma unroll
        for (int j = 0; j < WS; ++j) st[j] = sp[1 + j];
        from_stored<W, WS>(st, (uint32_t)(mt >> 32), key);
        c = (uint32_t)mt;
        emit = c >= P.min_count;
      }
    }
    emit_rows<W>(emit, key, c, P.out_keys, P.out_counts, P.out_cap, P.ctr);
  }
  for (int o = 16; o > 0; o >>= 1) ndist += __shfl_down_sync(0xFFFFFFFFu, ndist, o);
  if (lane == 0 && ndist) atomicAdd(&P.ctr->distinct, ndist);
}

// ---- launchers: dispatch on (W, WS) (GERBIL_KEY_SWITCH, insert.cuh) ---------------------------
int stored_words(int k) { return stored_words_of(k); }
int slot_words_for_k(int k) { return slot_words(stored_words(k)); }
uint32_t probe_window_for_k(int k) { return probe_window(slot_words_for_k(k)); }

cudaError_t launch_item_map(const CountParams& p, int nsm, cudaStream_t st) {
  if (p.nwork == 0 || p.nitems == 0) return cudaSuccess;
  const unsigned long long blocks = std::min<unsigned long long>((p.nitems + 255) / 256, (unsigned long long)nsm * 8);
  item_map_kernel<<<(unsigned)blocks, 256, 0, st>>>(p.work, p.nwork, p.sm_koff, p.imap, p.nitems);
  return cudaGetLastError();
}

cudaError_t launch_insert(int k, const CountParams& p, int persistent, int nsm, cudaStream_t st) {
  const unsigned long long need = (p.nitems - p.item_base + 7) / 8;
  if (need == 0) return cudaSuccess;
  const int W = (2 * k + 63) / 64, WS = stored_words(k);
  if (W <= 2) return launch_insert_w1_2(W, WS, p, need, persistent, nsm, st);
  if (W == 3) return launch_insert_w3(W, WS, p, need, persistent, nsm, st);
  if (W == 4) return launch_insert_w4(W, WS, p, need, persistent, nsm, st);
  if (W <= 7) return launch_insert_w5_7(W, WS, p, need, persistent, nsm, st);
  if (W <= 11) return launch_insert_w8_11(W, WS, p, need, persistent, nsm, st);
  return launch_insert_w12_15(W, WS, p, need, persistent, nsm, st);
}

cudaError_t launch_compact(int k, const CompactParams& p, int nsm, cudaStream_t st) {
  const unsigned long long n = p.slot_hi - p.slot_lo;
  if (n == 0) return cudaSuccess;
  const int W = (2 * k + 63) / 64, WS = stored_words(k);
  const unsigned long long per_cta = 256ull * 4;
  const unsigned grid = (unsigned)std::min<unsigned long long>((n + per_cta - 1) / per_cta,
                                                               (unsigned long long)nsm * 8);
#define L_COMPACT(w, ws) compact_kernel<w, ws><<<grid, 256, 0, st>>>(p)
  GERBIL_KEY_SWITCH(W, WS, L_COMPACT)
#undef L_COMPACT
  return cudaGetLastError();
}

cudaError_t launch_overflow_insert(int k, const OverflowParams& p, int nsm, cudaStream_t st) {
  const unsigned grid = (unsigned)nsm * 4;
  const int W = (2 * k + 63) / 64, WS = stored_words(k);
#define L_OINS(w, ws) overflow_insert_kernel<w, ws><<<grid, 256, 0, st>>>(p)
  GERBIL_KEY_SWITCH(W, WS, L_OINS)
#undef L_OINS
  return cudaGetLastError();
}

cudaError_t launch_overflow_emit(int k, const OverflowParams& p, int nsm, cudaStream_t st) {
  const unsigned grid = (unsigned)std::min<unsigned long long>(((unsigned long long)p.ocap + 255) / 256,
                                                               (unsigned long long)nsm * 8);
  const int W = (2 * k + 63) / 64, WS = stored_words(k);
#define L_OEMIT(w, ws) overflow_emit_kernel<w, ws><<<grid, 256, 0, st>>>(p)
  GERBIL_KEY_SWITCH(W, WS, L_OEMIT)
#undef L_OEMIT
  return cudaGetLastError();
}

cudaError_t launch_task_map(const FusedParams& p, cudaStream_t st) {
  if (p.c.nwork == 0) return cudaSuccess;
  task_map_kernel<<<std::min<unsigned>(p.c.nwork, 4096u), 256, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_fused(int k, const FusedParams& p, int nsm, cudaStream_t st) {
  if (p.ntasks == 0) return cudaSuccess;
  const int W = (2 * k + 63) / 64, WS = stored_words(k);
#define L_FUSED(w, ws)                                                                          \
  {                                                                                             \
    int per_sm = 0;                                                                             \
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused_kernel<w, ws>, \
                                                                  COUNT_THREADS, 0);            \
    if (e != cudaSuccess) return e;                                                             \
    const unsigned long long grid = std::min<unsigned long long>(                               \
        (p.ntasks + 7) / 8, (unsigned long long)nsm * std::max(1, per_sm));                     \
    fused_kernel<w, ws><<<(unsigned)grid, COUNT_THREADS, 0, st>>>(p);                           \
  }
  GERBIL_KEY_SWITCH(W, WS, L_FUSED)
#undef L_FUSED
  return cudaGetLastError();
}

}  // namespace gerbil

// ---- no-allocation entry point -----------------------------------------------------------------
// For callers that must not allocate device memory: the counting table lives in a file-scope
// device array of fixed size, held by every GPU that loads this library until the process
// exits.  Host code must not pass the array's name to a kernel (on the host it is only a
// stand-in); the device address comes from cudaGetSymbolAddress, once per device.

namespace gerbil {

constexpr unsigned long long NOALLOC_WORDS = 1ull << 22;  // 32 MiB
constexpr unsigned long long NOALLOC_HEAD = 16;           // counter words before the table
static __device__ __align__(256) unsigned long long g_noalloc_scratch[NOALLOC_WORDS];

// One warp per read, lanes over its windows; each k-mer is built straight from the ASCII bytes.
template <int W, int WS>
__global__ void __launch_bounds__(256) noalloc_insert_kernel(const uint8_t* __restrict__ seq,
                                                             const uint64_t* __restrict__ offsets,
                                                             uint64_t nreads, int k, int canonical,
                                                             unsigned long long* scratch, uint32_t cap) {
  unsigned long long* tab = scratch + NOALLOC_HEAD;
  const unsigned long long nw = (unsigned long long)gridDim.x * (blockDim.x >> 5);
  const int lane = threadIdx.x & 31;
  for (unsigned long long r = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
       r < nreads; r += nw) {
    const uint64_t a = offsets[r], b = offsets[r + 1];
    if (b < a + (uint64_t)k) continue;
    for (uint64_t p = a + lane; p + k <= b; p += 32) {
      unsigned long long key[W];
#pragma unroll
      for (int j = 0; j < W; ++j) key[j] = 0ull;
      bool ok = true;
      for (int i = 0; i < k && ok; ++i) {
        const uint32_t u = seq[p + i] & 0xDFu;
        ok = (u == 'A') | (u == 'C') | (u == 'G') | (u == 'T');
        uint32_t t = (u >> 1) & 3u;
        t ^= t >> 1;  // A0 C1 G2 T3
#pragma unroll
        for (int j = 0; j < W - 1; ++j) key[j] = (key[j] << 2) | (key[j + 1] >> 62);
        key[W - 1] = (key[W - 1] << 2) | t;
      }
      if (!ok) continue;
      if (canonical) {
        unsigned long long rc[W];
        revcomp<W>(key, k, rc);
        if (key_less<W>(rc, key)) {
#pragma unroll
          for (int q = 0; q < W; ++q) key[q] = rc[q];
        }
      }
      unsigned long long st[WS];
      to_stored<W, WS>(key, st);
      // flag bit 0: no free slot within cap probes; bit 1: a bounded wait for a peer's key
      // words gave up (reported apart, as a timeout)
      const int res = table_insert<WS>(tab, cap, st, key_tag<W>(key), key_hash<W>(key), cap, 1u << 20);
      if (res) atomicOr(reinterpret_cast<unsigned int*>(scratch + 1), res == 2 ? 2u : 1u);
    }
  }
}

template <int W, int WS>
__global__ void __launch_bounds__(256) noalloc_compact_kernel(unsigned long long* scratch, uint32_t cap,
                                                              uint32_t min_count,
                                                              unsigned long long* keys_out,
                                                              uint32_t* counts_out,
                                                              unsigned long long out_cap) {
  constexpr int SW = slot_words(WS);
  const unsigned long long* tab = scratch + NOALLOC_HEAD;
  for (unsigned long long s = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; s < cap;
       s += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long* sp = tab + s * SW;
    const unsigned long long mt = sp[0];
    if (mt == 0ull) continue;
    atomicAdd(scratch + 2, 1ull);
    if ((uint32_t)mt < min_count) continue;
    const unsigned long long row = atomicAdd(scratch + 0, 1ull);
    if (row >= out_cap) continue;  // the host reports the size that would have been needed
    unsigned long long st[WS], key[W];
#pragma unroll
    for (int j = 0; j < WS; ++j) st[j] = sp[1 + j];
    from_stored<W, WS>(st, (uint32_t)(mt >> 32), key);
#pragma unroll
    for (int j = 0; j < W; ++j) keys_out[row * W + j] = key[j];
    counts_out[row] = (uint32_t)mt;
  }
}

}  // namespace gerbil

#include <mutex>

#include "../../include/gerbil.h"

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[256];  // device address of the scratch array, per device
}  // namespace

extern "C" int gerbil_count_small_noalloc(const uint8_t* seq, const uint64_t* offsets,
                                          uint64_t nreads, uint64_t nbases, int k,
                                          uint32_t min_count, int canonical, uint64_t* keys_out,
                                          uint32_t* counts_out, uint64_t out_cap, uint64_t* n_out,
                                          void* cuda_stream) {
  using namespace gerbil;
  if (!n_out) return GERBIL_E_INVAL;
  *n_out = 0;
  if (k > GERBIL_MAX_K) return GERBIL_E_UNSUPPORTED;
  if (k < GERBIL_MIN_K || min_count < 1) return GERBIL_E_INVAL;
  if (nreads > 0 && (!seq || !offsets)) return GERBIL_E_INVAL;
  if (out_cap > 0 && (!keys_out || !counts_out)) return GERBIL_E_INVAL;
  const int W = (2 * k + 63) / 64, WS = stored_words(k), SW = slot_words(WS);
  const unsigned long long cap_max = (NOALLOC_WORDS - NOALLOC_HEAD) / (unsigned long long)SW;
  const uint64_t windows = nbases >= (uint64_t)k ? nbases - k + 1 : 0;
  if (windows > cap_max / 2) return GERBIL_E_INVAL;  // more k-mers than the scratch table holds
  const uint32_t cap = (uint32_t)std::min<unsigned long long>(cap_max, 2 * windows + 64);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return GERBIL_E_CUDA;
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GERBIL_E_CUDA;
      g_noalloc_ptr[dev] = p;
    }
    scratch = g_noalloc_ptr[dev];
  }
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GERBIL_E_CUDA;
  unsigned long long* sp = static_cast<unsigned long long*>(scratch);
  if (cudaMemsetAsync(sp, 0, (NOALLOC_HEAD + (unsigned long long)cap * SW) * 8, st) != cudaSuccess)
    return GERBIL_E_CUDA;
  const unsigned grid_i = (unsigned)std::max<unsigned long long>(
      1, std::min<unsigned long long>((nreads + 7) / 8, (unsigned long long)nsm * 8));
  const unsigned grid_c = (unsigned)std::min<unsigned long long>((cap + 255) / 256, (unsigned long long)nsm * 8);
  auto run = [&]() -> cudaError_t {
#define L_NOALLOC(w, ws)                                                                          \
  {                                                                                               \
    if (nreads) noalloc_insert_kernel<w, ws><<<grid_i, 256, 0, st>>>(seq, offsets, nreads, k,      \
                                                                     canonical ? 1 : 0, sp, cap); \
    noalloc_compact_kernel<w, ws><<<grid_c, 256, 0, st>>>(sp, cap, min_count,                     \
                                                          (unsigned long long*)keys_out,          \
                                                          counts_out, out_cap);                   \
  }
    GERBIL_KEY_SWITCH(W, WS, L_NOALLOC)
#undef L_NOALLOC
    return cudaGetLastError();
  };
  if (run() != cudaSuccess) return GERBIL_E_CUDA;
  unsigned long long head[3] = {0, 0, 0};
  if (cudaMemcpyAsync(head, sp, sizeof(head), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return GERBIL_E_CUDA;
  *n_out = head[0];
  if ((unsigned int)head[1] & 2u) return GERBIL_E_TIMEOUT;  // a bounded wait gave up
  if ((unsigned int)head[1] & 1u) return GERBIL_E_NOMEM;    // the scratch table ran full
  if (head[0] > out_cap) return GERBIL_E_INVAL;      // *n_out rows did not fit in out_cap
  return GERBIL_OK;
}
