// insert.cuh -- the phase-two insert kernel (extract, canonicalise, insert: Alg. 1, Sec. 2.3
// Phase Two, Sec. 2.4.2, Sec. 3.3-3.4) and the table helpers it shares with count.cu.  Its
// instantiations for every key width, probe scheme and work-item size are compiled in the
// insert_w*.cu files (one per group of key widths, so that they build in parallel).
#pragma once

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace gerbil {

// Calls f(std::integral_constant<int, i>) for i = B, B+S, ... below E (compile-time indices).
template <int B, int E, int S, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + S, E, S>(f);
  }
}

// Dispatch on the key width W = ceil(2k/64) and the stored chunks WS = stored_words_of(k)
// (W - 1 or W from two words on).
#define GERBIL_KEY_SWITCH(W, WS, CALL)                 \
  switch (W * 32 + WS) {                               \
    case 1 * 32 + 1: CALL(1, 1); break;                \
    case 2 * 32 + 1: CALL(2, 1); break;                \
    case 2 * 32 + 2: CALL(2, 2); break;                \
    case 3 * 32 + 2: CALL(3, 2); break;                \
    case 3 * 32 + 3: CALL(3, 3); break;                \
    case 4 * 32 + 3: CALL(4, 3); break;                \
    case 4 * 32 + 4: CALL(4, 4); break;                \
    case 5 * 32 + 4: CALL(5, 4); break;                \
    case 5 * 32 + 5: CALL(5, 5); break;                \
    case 6 * 32 + 5: CALL(6, 5); break;                \
    case 6 * 32 + 6: CALL(6, 6); break;                \
    case 7 * 32 + 6: CALL(7, 6); break;                \
    case 7 * 32 + 7: CALL(7, 7); break;                \
    case 8 * 32 + 7: CALL(8, 7); break;                \
    case 8 * 32 + 8: CALL(8, 8); break;                \
    case 9 * 32 + 8: CALL(9, 8); break;                \
    case 9 * 32 + 9: CALL(9, 9); break;                \
    case 10 * 32 + 9: CALL(10, 9); break;              \
    case 10 * 32 + 10: CALL(10, 10); break;            \
    case 11 * 32 + 10: CALL(11, 10); break;            \
    case 11 * 32 + 11: CALL(11, 11); break;            \
    case 12 * 32 + 11: CALL(12, 11); break;            \
    case 12 * 32 + 12: CALL(12, 12); break;            \
    case 13 * 32 + 12: CALL(13, 12); break;            \
    case 13 * 32 + 13: CALL(13, 13); break;            \
    case 14 * 32 + 13: CALL(14, 13); break;            \
    case 14 * 32 + 14: CALL(14, 14); break;            \
    case 15 * 32 + 14: CALL(15, 14); break;            \
    case 15 * 32 + 15: CALL(15, 15); break;            \
    default: return cudaErrorInvalidValue;             \
  }

// ---- table insert (Alg. 1) -------------------------------------------------------------------
// Probe sequence: slot0 = fastrange(hash), then linear steps, at most theta probes (Alg. 1's
// trial limit).  Each probe reads the whole slot with relaxed 16-byte loads.  An empty slot is
// claimed by CAS on its meta word (0 -> CLAIMED|tag, count 1; the tag is the key's low 30
// bits); the claimer then writes the marked key words.  A prober whose tag matches compares the
// rest of the key once every word carries its marker (bounded wait otherwise) and adds 1 to the
// count.  Returns 0 on success, 1 if theta
// probes found no room, 2 if a bounded wait gave up -- both send the k-mer to the overflow
// area, which is always correct because overflow counts are added to table counts before
// the min_count filter.
template <int WS>
__device__ __forceinline__ int table_insert_from(unsigned long long* __restrict__ tab, uint32_t cap,
                                                 const unsigned long long st[WS], uint32_t tag,
                                                 uint32_t theta, uint32_t spin_limit, uint32_t s,
                                                 unsigned long long v[slot_words(WS)]) {
  constexpr int SW = slot_words(WS);
  const uint32_t tagw = META_CLAIMED | (tag & META_TAG_MASK);
  const unsigned long long claim = ((unsigned long long)tagw << 32) | 1ull;
  for (uint32_t t = 0; t < theta; ++t) {
    unsigned long long* slot = tab + (unsigned long long)s * SW;
    if (t > 0) load_slot<SW>(slot, v);
    if (v[0] == 0ull) {
      const unsigned long long old = cas_relaxed(slot, 0ull, claim);
      if (old == 0ull) {
        // word 1 sits at byte 8 of the 16-byte aligned slot: store it alone, then aligned
        // pairs (slot + 2, slot + 4, ...)
        st_relaxed(slot + 1, st[0]);
#pragma unroll
        for (int j = 1; j < WS; j += 2) {
          if (j + 1 < WS) st_relaxed_v2(slot + 1 + j, st[j], st[j + 1]);
          else st_relaxed(slot + 1 + j, st[j]);
        }
        return 0;
      }
      v[0] = old;
#pragma unroll
      for (int j = 1; j < SW; ++j) v[j] = 0ull;  // re-read below
    }
    if (((uint32_t)(v[0] >> 32) & ~META_MERGED) == tagw) {
      for (uint32_t spins = 0;;) {
        bool all = true, eq = true;
#pragma unroll
        for (int j = 0; j < WS; ++j) {
          all &= (v[1 + j] & MARK) != 0ull;
          eq &= v[1 + j] == st[j];
        }
        if (all) {
          if (eq) {
            red_add(slot, 1ull);
            return 0;
          }
          break;  // another key with the same tag
        }
        if (++spins > spin_limit) return 2;
        if (spins > 1) __nanosleep(32);
        load_slot<SW>(slot, v);
      }
    }
    s = (s + 1 == cap) ? 0u : s + 1;
  }
  return 1;
}

__device__ __forceinline__ uint32_t slot_of(unsigned long long h, uint32_t cap) {
  return (uint32_t)(((h & 0xFFFFFFFFull) * (unsigned long long)cap) >> 32);
}

// st, tag: the key's stored chunks and its low 30 bits; h: its hash (the first slot)
template <int WS>
__device__ __forceinline__ int table_insert(unsigned long long* __restrict__ tab, uint32_t cap,
                                            const unsigned long long st[WS], uint32_t tag,
                                            unsigned long long h, uint32_t theta, uint32_t spin_limit) {
  constexpr int SW = slot_words(WS);
  const uint32_t s = slot_of(h, cap);
  unsigned long long v[SW];
  load_slot<SW>(tab + (unsigned long long)s * SW, v);
  return table_insert_from<WS>(tab, cap, st, tag, theta, spin_limit, s, v);
}

// Lookup in a complete table (no concurrent inserts); marks the slot MERGED and returns its
// count, or 0 if the key is absent.
template <int WS>
__device__ __forceinline__ uint32_t table_take(unsigned long long* __restrict__ tab, uint32_t cap,
                                               const unsigned long long st[WS], uint32_t tag,
                                               unsigned long long h) {
  constexpr int SW = slot_words(WS);
  uint32_t s = (uint32_t)(((h & 0xFFFFFFFFull) * (unsigned long long)cap) >> 32);
  const uint32_t tagw = META_CLAIMED | (tag & META_TAG_MASK);
  for (uint32_t t = 0; t < cap; ++t) {
    unsigned long long* slot = tab + (unsigned long long)s * SW;
    const unsigned long long mt = slot[0];
    if (mt == 0ull) return 0;
    if (((uint32_t)(mt >> 32) & ~META_MERGED) == tagw) {
      bool eq = true;
#pragma unroll
      for (int j = 0; j < WS; ++j) eq &= (slot[1 + j] == st[j]);
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

// Probe statistics of one placed k-mer (why = 0) or one sent to the overflow area (why != 0),
// placed at slot s after t steps.  Scheme 0: t slots were stepped over (first slot s - t,
// cyclic), and the lines count is the number of distinct 128-byte lines among the slots read.
// Scheme 1: t windows were passed (each scanned whole), then the window of s from its first
// slot; the lines count is the windows read (a window is the paper's unit of windowed probing,
// Sec. 3.3).
template <int SW>
__device__ __noinline__ void record_probe(const CountParams& P, const BinWork& wk, uint32_t s,
                                          uint32_t t, int why) {
  int b0, b1;
  if (why) {
    b0 = b1 = PROBE_BUCKETS - 1;
  } else {
    unsigned long long slots, lines;
    if (wk.scheme == 1) {
      constexpr uint32_t WIN = (128 / (8 * SW)) >= 1 ? (uint32_t)(128 / (8 * SW)) : 1u;
      slots = (unsigned long long)t * WIN + (s % WIN) + 1;
      lines = (unsigned long long)t + 1;
    } else {
      const unsigned long long s0 = (s >= t) ? s - t : s + wk.cap - t;
      const unsigned long long first = (wk.table_off + s0) * SW * 8 / 128;
      const unsigned long long last = (wk.table_off + s0 + t) * SW * 8 / 128;
      slots = (unsigned long long)t + 1;
      lines = last - first + 1;
    }
    b0 = (int)(slots < 33 ? slots : 33ull) - 1;
    b1 = (int)(lines < 33 ? lines : 33ull) - 1;
  }
  atomicAdd(P.probe_hist + b0, 1ull);
  atomicAdd(P.probe_hist + PROBE_BUCKETS + b1, 1ull);
}

struct WarpSmem {
  uint32_t koff[ITEM_KMERS];
  unsigned long long pos[ITEM_KMERS];
};

// A lane takes KPL = item_kmers/32 consecutive k-mers of the item.  Within a super-mer the next k-mer
// and its reverse complement follow from the previous ones by one base: shift the forward key
// left by two bits and append the new base; shift the reverse complement right by two bits and
// put the new base's complement on top.  Only the lane's first k-mer and the first k-mer of
// every new super-mer are cut from the packed words in full.

// Probe schemes (BinWork::scheme).  0: linear probing from a fastrange slot, one slot per step.
// 1: the paper's windowed double hashing (Sec. 3.3-3.4): the table is a sequence of windows of
// probe_window(SW) slots (one 128-byte line for slots of 16 or 32 bytes); the first window is
// fastrange(hash) over the windows, the next ones step by h2 = 1 + fastrange(bits 34..63 of the
// hash, windows - 1) windows (mod the window count), and every window is scanned from its first
// slot, one slot per step.  theta counts slots under scheme 0 and windows under scheme 1.
__host__ __device__ constexpr uint32_t probe_window(int SW) {
  return (128 / (8 * SW)) >= 1 ? (uint32_t)(128 / (8 * SW)) : 1u;
}
// Key widths whose reverse complement is taken afresh for every k-mer instead of rolled with
// it: where dropping it from the registers live during the probes buys one more CTA per SM
// (measured: 8 and 9 words run 3 CTAs instead of 2, k = 256 insert 8.34 -> 7.66 ms; 15 words
// run 2 instead of 1, k = 479 13.26 -> 10.72 ms; for 10-14 words it bought none and cost 3%).
__host__ __device__ constexpr bool rc_fresh(int W) { return W == 8 || W == 9 || W == 15; }

// CF: claim first (CountParams::cas_first), built for the default scheme and item size.
template <int W, int WS, bool STATS = false, int SCHEME = 0, int KPL = ITEM_KMERS / 32, bool CF = false>
__device__ __forceinline__ void insert_item(const CountParams& P, uint32_t wi, const BinWork& wk,
                                            uint32_t it, uint32_t s_lo, WarpSmem& S, int lane) {
  constexpr uint32_t ik = 32u * KPL;  // k-mers of the item, <= ITEM_KMERS
  const uint32_t j0 = it * ik;
  const uint32_t j1 = min(j0 + ik, wk.n_kmers);
  const uint32_t* koff = P.sm_koff + wk.sm_begin;
  const unsigned long long* spos = P.sm_pos + wk.sm_begin;
  // descriptors of the super-mers that hold k-mers [j0, j1): koff ascends, so they are the
  // ones from s_lo on whose first k-mer is below j1
  uint32_t ns = 0;
  for (uint32_t c = 0; c < ik; c += 32) {
    const uint32_t s = s_lo + c + lane;
    const bool have = s < wk.n_super;
    const uint32_t ko = have ? __ldg(koff + s) : wk.n_kmers;
    const unsigned long long po = have ? __ldg(spos + s) : 0ull;
    const bool in = have && (c + lane == 0 || ko < j1);
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, in);
    if (in) {
      S.koff[c + lane] = ko;
      S.pos[c + lane] = po;
    }
    const uint32_t cnt = __popc(bal);
    ns += cnt;
    if (cnt < 32) break;
  }
  __syncwarp();
  constexpr int SW = slot_words(WS);
  unsigned long long* tab = P.arena + wk.table_off * SW;
  const int k = P.k;
  const int nb0 = k - 32 * (W - 1);  // bases in key word 0
  const unsigned long long mask0 = (nb0 == 32) ? ~0ull : ((1ull << (2 * nb0)) - 1ull);
  constexpr bool ROLL_RC = !rc_fresh(W);
  const uint32_t ja = j0 + (uint32_t)lane * KPL;
  const uint32_t jb = min(ja + (uint32_t)KPL, j1);
  unsigned long long fwd[W], rc[W], pos = 0;
  uint32_t sidx = 0, send = 0;  // current super-mer and its first k-mer past the end
  constexpr uint32_t WIN = probe_window(SW);
  constexpr bool windowed = SCHEME == 1;
  const uint32_t nwin = wk.cap / WIN;  // scheme 1: the host makes cap a multiple of WIN
  // Each lane keeps one k-mer in flight and does one probe of it per step; a lane whose k-mer
  // is placed takes its next one at the start of the following step, while the other lanes go
  // on probing theirs.  A warp thus waits for the longest sum of probe chains over a lane's
  // k-mers, not for the longest chain of every k-mer in turn.
  // Keys of fourteen words do not keep their stored form in registers while they are probed:
  // each chunk is cut from fwd or rc when it is compared or written, which frees WS registers
  // (measured on the 10 Mbp long-read sweep: k = 448 insert 9.46 -> 8.38 ms, its 128-160 bytes
  // of spills gone; for 10-13 words, which do not spill at 2 CTAs per SM, it cost 1-4%)
  constexpr bool LAZY = ROLL_RC && W == 14;
  unsigned long long st[LAZY ? 1 : WS];
  bool urc = false;  // LAZY: the key is rc (else fwd)
  uint32_t tagw = 0, s = 0, t = 0, spins = 0;
  uint32_t wstep = 0;  // scheme 1: 30 hash bits that give the window step
  uint32_t j = ja;
  bool busy = false;
  // chunk u of the stored key in flight
  auto stored_u = [&](auto U) -> unsigned long long {
    constexpr int u = decltype(U)::value;
    if constexpr (LAZY) return stored_chunk<W, u>(fwd, rc, urc);
    else return st[u];
  };
#pragma unroll 1
  for (;;) {
    if (!busy) {
      if (j >= jb) break;
      if (j == ja || j >= send) {  // cut the k-mer in full
        if (j == ja) {
          uint32_t lo = 0, hi = ns;
          while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (S.koff[mid] <= j) lo = mid; else hi = mid;
          }
          sidx = lo;
        } else {
          ++sidx;
        }
        send = (sidx + 1 < ns) ? S.koff[sidx + 1] : 0xFFFFFFFFu;
        pos = S.pos[sidx] + (j - S.koff[sidx]);
        load_kmer<W>(P.packed, pos, k, fwd);
        if constexpr (ROLL_RC) revcomp<W>(fwd, k, rc);
      } else {  // roll by one base
        const unsigned long long q = pos + (unsigned long long)k;  // the new last base
        const unsigned long long b = (__ldg(P.packed + (q >> 5)) >> (62 - 2 * (int)(q & 31))) & 3ull;
#pragma unroll
        for (int u = 0; u < W - 1; ++u) fwd[u] = (fwd[u] << 2) | (fwd[u + 1] >> 62);
        fwd[W - 1] = (fwd[W - 1] << 2) | b;
        fwd[0] &= mask0;
        if constexpr (ROLL_RC) {
#pragma unroll
          for (int u = W - 1; u >= 1; --u) rc[u] = (rc[u] >> 2) | (rc[u - 1] << 62);
          rc[0] = (rc[0] >> 2) | ((3ull - b) << (2 * nb0 - 2));
        }
        ++pos;
      }
      // the widths of rc_fresh take the reverse complement afresh: it is then dead while the
      // k-mer is probed
      if constexpr (!ROLL_RC) revcomp<W>(fwd, k, rc);
      unsigned long long key[W];
      const bool use_rc = P.canonical && key_less<W>(rc, fwd);
#pragma unroll
      for (int u = 0; u < W; ++u) key[u] = use_rc ? rc[u] : fwd[u];
      const unsigned long long h = key_hash<W>(key);
      if constexpr (LAZY) urc = use_rc;
      else to_stored<W, WS>(key, st);
      tagw = META_CLAIMED | key_tag<W>(key);
      if constexpr (windowed) {
        s = slot_of(h, nwin) * WIN;
        wstep = (uint32_t)(h >> 34) & META_TAG_MASK;
      } else {
        s = slot_of(h, wk.cap);
      }
      t = 0;
      spins = 0;
      busy = true;
      ++j;
    }
    // one probe of slot s (Alg. 1)
    unsigned long long* slot = tab + (unsigned long long)s * SW;
    unsigned long long v[SW];
    const unsigned long long claim = ((unsigned long long)tagw << 32) | 1ull;
    bool claimed = false;
    if constexpr (CF) {
      // mostly new keys: claim first (one round trip when the slot is empty) and read the
      // key words only when the meta word's tag matches
      const unsigned long long old = cas_relaxed(slot, 0ull, claim);
      claimed = old == 0ull;
      if (!claimed) {
        if (((uint32_t)(old >> 32) & ~META_MERGED) == tagw) load_slot<SW>(slot, v);
        else v[0] = old;  // another key: its words are not looked at
      }
    } else {
      // mostly repeated keys: read the slot first (a found key costs one round trip)
      load_slot<SW>(slot, v);
      if (v[0] == 0ull) {
        claimed = cas_relaxed(slot, 0ull, claim) == 0ull;
        if (!claimed) continue;  // claimed by another lane meanwhile: look at the slot again
      }
    }
    if (claimed) {  // the slot is ours: its marked key words
      st_relaxed(slot + 1, stored_u(std::integral_constant<int, 0>{}));  // word 1 alone,
      static_for<1, WS, 2>([&](auto U) {                                // then aligned pairs
        constexpr int u = decltype(U)::value;
        if constexpr (u + 1 < WS)
          st_relaxed_v2(slot + 1 + u, stored_u(U), stored_u(std::integral_constant<int, u + 1>{}));
        else
          st_relaxed(slot + 1 + u, stored_u(U));
      });
      busy = false;
      if constexpr (STATS) record_probe<SW>(P, wk, s, t, 0);
      continue;
    }
    int why = 0;
    if (((uint32_t)(v[0] >> 32) & ~META_MERGED) == tagw) {
      // equal stored words carry their markers, so equality alone means the key is found;
      // the markers are looked at only when the words differ
      bool eq = true;
      static_for<0, WS, 1>([&](auto U) { eq &= v[1 + decltype(U)::value] == stored_u(U); });
      if (eq) {
        red_add(slot, 1ull);
        busy = false;
        if constexpr (STATS) record_probe<SW>(P, wk, s, t, 0);
        continue;
      }
      bool all = true;
#pragma unroll
      for (int u = 0; u < WS; ++u) all &= (v[1 + u] & MARK) != 0ull;
      if (!all) {  // the claimer has not written every key word yet: read the slot again
        if (++spins > P.spin_limit) {
          why = 2;
        } else {
          if (spins > 8) __nanosleep(32);
          continue;
        }
      }
    }
    if (!why) {  // the next slot of the probe sequence
      if constexpr (!windowed) {
        s = (s + 1 == wk.cap) ? 0u : s + 1;
        if (++t < P.theta) continue;
      } else {
        if ((s + 1) % WIN != 0u) {  // the next slot of the same window
          ++s;
          continue;
        }
        if (++t < P.theta) {  // the next window of the double-hashing sequence
          const uint32_t h2 = nwin > 1 ? 1u + (uint32_t)(((unsigned long long)wstep * (nwin - 1)) >> 30)
                                       : 0u;
          uint32_t w = s / WIN + h2;
          if (w >= nwin) w -= nwin;
          s = w * WIN;
          continue;
        }
      }
      why = 1;
    }
    unsigned long long key[W];
    if constexpr (LAZY) {
#pragma unroll
      for (int u = 0; u < W; ++u) key[u] = urc ? rc[u] : fwd[u];
    } else {
      from_stored<W, WS>(st, tagw, key);
    }
    to_overflow<W>(P, wi, key, why);
    if constexpr (STATS) record_probe<SW>(P, wk, s, t, why);
    busy = false;
  }
  __syncwarp();  // S is reused by the next item
}

template <int W, int WS, bool STATS, int SCHEME, int KPL, bool CF>
__device__ __forceinline__ void count_item(const CountParams& P, unsigned long long item,
                                           unsigned long long entry, WarpSmem& S, int lane) {
  const uint32_t wi = (uint32_t)(entry >> 32), s_lo = (uint32_t)entry;
  const BinWork wk = P.work[wi];
  insert_item<W, WS, STATS, SCHEME, KPL, CF>(P, wi, wk, (uint32_t)(item - wk.item_begin), s_lo, S, lane);
}

// Warps take items in bin order from a device counter (the next one is requested while the
// current one runs), so the bins in flight at any moment are few and their tables stay hot in
// L2; or (schedule 0) each warp strides over the items.  Launched with as many CTAs as fit on
// the GPU (persistent) or one warp per item.
// Resident CTAs per SM that the register allocation is held to, per key width (measured on
// k = 65, 99 and a 1000 bp read set at k = 150..479).  A cap pays while its spills stay small
// (about 64 bytes a thread): 5 for keys of up to three words, 4 for four or five, 3 for six to
// nine (eight and nine with the reverse complement taken afresh), 2 from ten words on (fifteen
// with it taken afresh: 128 registers, no spills).
#ifndef GERBIL_MINB_SMALL
#define GERBIL_MINB_SMALL 5
#endif
#ifndef GERBIL_MINB_MID
#define GERBIL_MINB_MID 4
#endif
#ifndef GERBIL_MINB_WIDE
#define GERBIL_MINB_WIDE 3
#endif
#ifndef GERBIL_MINB_XWIDE
#define GERBIL_MINB_XWIDE 2
#endif
constexpr int insert_min_blocks(int W) {
  return W <= 3 ? GERBIL_MINB_SMALL
                : W <= 5 ? GERBIL_MINB_MID
                : W <= 9 ? GERBIL_MINB_WIDE : GERBIL_MINB_XWIDE;
}

// STATS: the instantiation that records probe statistics (only launched while they are on).
template <int W, int WS, bool STATS, int SCHEME, int KPL, bool CF>
__device__ __forceinline__ void insert_items(const CountParams& P, WarpSmem* S) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (!P.schedule) {  // fixed: warp w takes items base + w, base + w + nw, ...
    const unsigned long long nw = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    for (unsigned long long item = P.item_base + blockIdx.x * (unsigned long long)(blockDim.x >> 5) + warp;
         item < P.nitems; item += nw)
      count_item<W, WS, STATS, SCHEME, KPL, CF>(P, item, __ldg(P.imap + item), S[warp], lane);
    return;
  }
  unsigned long long* queue = P.queue;
  unsigned long long item = 0;
  if (lane == 0) item = P.item_base + atomicAdd(queue, 1ull);
  item = __shfl_sync(0xFFFFFFFFu, item, 0);
  while (item < P.nitems) {
    unsigned long long next = 0;
    if (lane == 0) next = P.item_base + atomicAdd(queue, 1ull);
    const unsigned long long entry = __ldg(P.imap + item);
    count_item<W, WS, STATS, SCHEME, KPL, CF>(P, item, entry, S[warp], lane);
    item = __shfl_sync(0xFFFFFFFFu, next, 0);
  }
}

// CAP = false: the same kernel without the register cap, for keys of six or more words whose
// bins' tables average more than the L2 cache (CountParams::wide_tables).  Their probes go to
// HBM whatever the warps in flight, so the cap's spills cost time without hiding any more
// latency (measured: k = 200 with 126 GB of tables, 71.1 ms uncapped against 74.1 ms capped).
template <int W, int WS, bool STATS, bool CAP, int SCHEME, int KPL, bool CF>
__global__ void __launch_bounds__(256, CAP ? insert_min_blocks(W) : 1) insert_kernel(CountParams P) {
  __shared__ WarpSmem S[8];
  if constexpr (STATS) {
    // probe statistics: summed per CTA in shared memory, added to the global histogram once
    __shared__ unsigned long long hist[2 * PROBE_BUCKETS];
    for (int i = threadIdx.x; i < 2 * PROBE_BUCKETS; i += blockDim.x) hist[i] = 0ull;
    __syncthreads();
    unsigned long long* global_hist = P.probe_hist;
    CountParams Q = P;
    Q.probe_hist = hist;
    insert_items<W, WS, STATS, SCHEME, KPL, CF>(Q, S);
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * PROBE_BUCKETS; i += blockDim.x)
      if (hist[i]) atomicAdd(global_hist + i, hist[i]);
  } else {
    insert_items<W, WS, STATS, SCHEME, KPL, CF>(P, S);
  }
}


// Launch of one (key width, stored words, probe scheme, k-mers per lane) instantiation:
// persistent -- as many CTAs as are resident at once (occupancy query), each warp taking items
// -- or one warp per item.
template <int w, int ws, bool CAP, int SCHEME, int KPL, bool CF>
static cudaError_t launch_insert_as(const CountParams& p, unsigned long long need, int persistent,
                                    int nsm, cudaStream_t st) {
  unsigned long long grid = need;
  if (persistent) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, insert_kernel<w, ws, false, CAP, SCHEME, KPL, CF>, COUNT_THREADS, 0);
    if (e != cudaSuccess) return e;
    grid = std::min<unsigned long long>(need, (unsigned long long)nsm * std::max(1, per_sm));
  }
  // probe statistics always use the capped, read-first form (they time nothing; both probe
  // orders visit the same slots)
  if (p.probe_hist)
    insert_kernel<w, ws, true, true, SCHEME, KPL, false><<<(unsigned)grid, COUNT_THREADS, 0, st>>>(p);
  else
    insert_kernel<w, ws, false, CAP, SCHEME, KPL, CF><<<(unsigned)grid, COUNT_THREADS, 0, st>>>(p);
  return cudaGetLastError();
}

template <int w, int ws, int SCHEME, int KPL, bool CF = false>
static cudaError_t launch_insert_sk(const CountParams& p, unsigned long long need, int persistent,
                                    int nsm, cudaStream_t st) {
  if constexpr (w >= 6 && insert_min_blocks(w) > 1) {
    if (p.wide_tables && !p.probe_hist)
      return launch_insert_as<w, ws, false, SCHEME, KPL, CF>(p, need, persistent, nsm, st);
  }
  return launch_insert_as<w, ws, true, SCHEME, KPL, CF>(p, need, persistent, nsm, st);
}

// Work-item sizes other than 256 k-mers are compiled for keys of up to four words only; the
// claim-first probe order for the default scheme and item size only.
__host__ __device__ constexpr bool small_items_for(int w) { return w <= 4; }

template <int w, int ws>
static cudaError_t launch_insert_w(const CountParams& p, unsigned long long need, int persistent,
                                   int nsm, cudaStream_t st) {
  const int kpl = (int)(p.item_kmers / 32);
  if (p.scheme == 0 && kpl == 8) {
    if (p.cas_first && !p.probe_hist) return launch_insert_sk<w, ws, 0, 8, true>(p, need, persistent, nsm, st);
    return launch_insert_sk<w, ws, 0, 8>(p, need, persistent, nsm, st);
  }
  if (p.scheme == 1 && kpl == 8) return launch_insert_sk<w, ws, 1, 8>(p, need, persistent, nsm, st);
  if constexpr (small_items_for(w)) {
    if (p.scheme == 0 && kpl == 4) return launch_insert_sk<w, ws, 0, 4>(p, need, persistent, nsm, st);
    if (p.scheme == 1 && kpl == 4) return launch_insert_sk<w, ws, 1, 4>(p, need, persistent, nsm, st);
    if (p.scheme == 0 && kpl == 2) return launch_insert_sk<w, ws, 0, 2>(p, need, persistent, nsm, st);
    if (p.scheme == 1 && kpl == 2) return launch_insert_sk<w, ws, 1, 2>(p, need, persistent, nsm, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace gerbil
