// common.cuh -- device-side building blocks shared by the phase-one and phase-two kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gerbil {

// ---- device error word bits (host maps them to gerbil_status) ----------------------------
enum : uint32_t {
  ERR_OVF_FULL = 1u << 0,   // the overflow area was full: some k-mers were not recorded
  ERR_SPIN = 1u << 1,       // a bounded wait gave up where no fallback exists
  ERR_STATE = 1u << 2,      // a claimed slot was never published / descriptor mismatch
  ERR_OUT_FULL = 1u << 3,   // the result buffer was too small
  ERR_QUEUE = 1u << 4,      // a work-queue wait gave up
};

// Device counters block, one per context, cleared per call.
struct Counters {
  unsigned long long ovf_count;      // overflow-area cursor
  unsigned long long out_count;      // result cursor
  unsigned long long distinct;       // live slots seen by the compaction
  unsigned long long spin_demotions; // inserts demoted to overflow after a bounded wait
  unsigned long long queue_head;     // persistent-kernel work queue cursor
  unsigned long long merged;         // overflow keys merged into a main-table key
  unsigned long long pad[9];
  unsigned int err;                  // ERR_* bits
  unsigned int pad2;
};

// ---- table slot layout -------------------------------------------------------------------
// A slot is SW = even(WS+1) 64-bit words: word 0 = meta, words 1..WS = the rest of the key.
// meta's low 32 bits hold the count; the high 32 bits hold CLAIMED | MERGED | the key's low 30
// bits (its "tag": a reader whose tag differs has another key, without looking further); meta
// == 0 is an empty slot.  The key's bits from bit 30 up are cut into WS = max(1, ceil((2k -
// 30) / 63)) chunks of 63 bits, each with bit 63 set as a "written" marker.  A cleared word (0)
// can therefore never be mistaken for a written one: a reader that sees every marker set has
// read the final key, word by word, with relaxed loads and no ordering.
constexpr uint32_t META_CLAIMED = 1u << 31;
constexpr uint32_t META_MERGED = 1u << 30;
constexpr int KEY_TAG_BITS = 30;
constexpr uint32_t META_TAG_MASK = (1u << KEY_TAG_BITS) - 1;
constexpr unsigned long long MERGED64 = (unsigned long long)META_MERGED << 32;
constexpr unsigned long long MARK = 1ull << 63;
constexpr unsigned long long MASK63 = MARK - 1;

__host__ __device__ constexpr int slot_words(int WS) { return (WS + 2) & ~1; }
// chunks of the key beyond the tag: max(1, ceil((2k - 30) / 63))
__host__ __device__ constexpr int stored_words_of(int k) {
  return 2 * k <= KEY_TAG_BITS + 63 ? 1 : (2 * k - KEY_TAG_BITS + 62) / 63;
}

// the key's low 30 bits: its tag in the meta word
template <int W>
__device__ __forceinline__ uint32_t key_tag(const unsigned long long key[W]) {
  return (uint32_t)key[W - 1] & META_TAG_MASK;
}

// key (W words, word 0 most significant) -> WS marked 63-bit chunks of its bits from bit 30 up,
// chunk 0 least significant
template <int W, int WS>
__device__ __forceinline__ void to_stored(const unsigned long long key[W], unsigned long long st[WS]) {
#pragma unroll
  for (int c = 0; c < WS; ++c) {
    const int L = KEY_TAG_BITS + 63 * c, r = L >> 6, sh = L & 63;  // r counts words from the least significant
    unsigned long long v = 0;
    if (r < W) v = key[W - 1 - r] >> sh;
    if (sh >= 2 && r + 1 < W) v |= key[W - 2 - r] << (64 - sh);
    st[c] = MARK | (v & MASK63);
  }
}

// Chunk c of to_stored of the key that is b when use_b, else a (the chunks computed one at a
// time, for kernels that do not keep the stored form in registers).
template <int W, int C>
__device__ __forceinline__ unsigned long long stored_chunk(const unsigned long long a[W],
                                                           const unsigned long long b[W], bool use_b) {
  constexpr int L = KEY_TAG_BITS + 63 * C, r = L >> 6, sh = L & 63;
  unsigned long long v = 0;
  if constexpr (r < W) v = (use_b ? b[W - 1 - r] : a[W - 1 - r]) >> sh;
  if constexpr (sh >= 2 && r + 1 < W) v |= (use_b ? b[W - 2 - r] : a[W - 2 - r]) << (64 - sh);
  return MARK | (v & MASK63);
}

// the key from its tag (the low 30 bits of a meta word's high half, or the tag itself) and its
// stored chunks
template <int W, int WS>
__device__ __forceinline__ void from_stored(const unsigned long long st[WS], uint32_t tag,
                                            unsigned long long key[W]) {
#pragma unroll
  for (int j = 0; j < W; ++j) key[j] = 0;
  key[W - 1] = tag & META_TAG_MASK;
#pragma unroll
  for (int c = 0; c < WS; ++c) {
    const unsigned long long v = st[c] & MASK63;
    const int L = KEY_TAG_BITS + 63 * c, r = L >> 6, sh = L & 63;
    if (r < W) key[W - 1 - r] |= v << sh;
    if (sh >= 2 && r + 1 < W) key[W - 2 - r] |= v >> (64 - sh);
  }
}

__device__ __forceinline__ void ld_relaxed_v2(const unsigned long long* p, unsigned long long& a,
                                              unsigned long long& b) {
  asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}
__device__ __forceinline__ void st_relaxed_v2(unsigned long long* p, unsigned long long a,
                                              unsigned long long b) {
  asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}
__device__ __forceinline__ unsigned long long cas_relaxed(unsigned long long* p, unsigned long long cmp,
                                                          unsigned long long val) {
  unsigned long long old;
  asm volatile("atom.relaxed.gpu.global.cas.b64 %0, [%1], %2, %3;"
               : "=l"(old)
               : "l"(p), "l"(cmp), "l"(val)
               : "memory");
  return old;
}

__device__ __forceinline__ void ld_relaxed_v4(const unsigned long long* p, unsigned long long& a,
                                              unsigned long long& b, unsigned long long& c,
                                              unsigned long long& d) {
  asm volatile("ld.relaxed.gpu.global.v4.u64 {%0, %1, %2, %3}, [%4];"
               : "=l"(a), "=l"(b), "=l"(c), "=l"(d)
               : "l"(p)
               : "memory");
}

// All SW words of a slot with relaxed vector loads: 32-byte loads when the slot size is a
// multiple of 32 bytes (the slot is then 32-byte aligned in the 256-byte aligned arena), else
// 16-byte loads (every slot is 16-byte aligned).
template <int SW>
__device__ __forceinline__ void load_slot(const unsigned long long* slot, unsigned long long v[SW]) {
  if constexpr (SW % 4 == 0) {
#pragma unroll
    for (int i = 0; i < SW; i += 4) ld_relaxed_v4(slot + i, v[i], v[i + 1], v[i + 2], v[i + 3]);
  } else {
#pragma unroll
    for (int i = 0; i < SW; i += 2) ld_relaxed_v2(slot + i, v[i], v[i + 1]);
  }
}

// ---- memory-model helpers (PTX, gpu scope) -------------------------------------------------
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long cas_acquire(unsigned long long* p,
                                                          unsigned long long cmp,
                                                          unsigned long long val) {
  unsigned long long old;
  asm volatile("atom.acquire.gpu.global.cas.b64 %0, [%1], %2, %3;"
               : "=l"(old)
               : "l"(p), "l"(cmp), "l"(val)
               : "memory");
  return old;
}
__device__ __forceinline__ void red_add(unsigned long long* p, unsigned long long v) {
  asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void red_or_release(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.or.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long atom_or(unsigned long long* p, unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.relaxed.gpu.global.or.b64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
}

// ---- bases --------------------------------------------------------------------------------
// The packed stream holds base i of the input at word i/32, bits (63-2*(i%32), 62-2*(i%32)):
// first base in the high bits, A=0 C=1 G=2 T=3.  Masks hold base i at u32 word i/32, bit
// 31-(i%32).

// Reverse the order of the 32 two-bit groups of a word.
__device__ __forceinline__ unsigned long long rev2(unsigned long long x) {
  unsigned long long y = __brevll(x);
  return ((y >> 1) & 0x5555555555555555ull) | ((y & 0x5555555555555555ull) << 1);
}

// k-mer of k bases starting at base `pos`, as W words (word 0 most significant, right-aligned
// integer).  Reads W+1 words of the packed stream (the stream carries two words of padding).
template <int W>
__device__ __forceinline__ void load_kmer(const unsigned long long* __restrict__ packed,
                                          unsigned long long pos, int k,
                                          unsigned long long key[W]) {
  const unsigned long long* w = packed + (pos >> 5);
  const int o = 2 * int(pos & 31);
  unsigned long long v[W + 1];
#pragma unroll
  for (int j = 0; j <= W; ++j) v[j] = __ldg(w + j);
  unsigned long long L[W];
#pragma unroll
  for (int j = 0; j < W; ++j) L[j] = o ? ((v[j] << o) | (v[j + 1] >> (64 - o))) : v[j];
  const int s = 64 * W - 2 * k;  // 0 <= s < 64
#pragma unroll
  for (int j = W - 1; j >= 1; --j) key[j] = s ? ((L[j] >> s) | (L[j - 1] << (64 - s))) : L[j];
  key[0] = L[0] >> s;
}

// Reverse complement of a right-aligned k-mer (Sec. 2.4.2).
template <int W>
__device__ __forceinline__ void revcomp(const unsigned long long key[W], int k,
                                        unsigned long long rc[W]) {
  unsigned long long t[W];
#pragma unroll
  for (int j = 0; j < W; ++j) t[W - 1 - j] = rev2(~key[j]);
  const int s = 64 * W - 2 * k;
#pragma unroll
  for (int j = W - 1; j >= 1; --j) rc[j] = s ? ((t[j] >> s) | (t[j - 1] << (64 - s))) : t[j];
  rc[0] = t[0] >> s;
}

template <int W>
__device__ __forceinline__ bool key_less(const unsigned long long a[W],
                                         const unsigned long long b[W]) {
#pragma unroll
  for (int j = 0; j < W; ++j)
    if (a[j] != b[j]) return a[j] < b[j];
  return false;
}

// 64-bit hash of a key (the slot index uses the low 32 bits, the windowed scheme's window step
// bits 34..63): the words are folded into one by xor with distinct rotations, then mixed by two
// multiply/xorshift rounds -- two 64-bit multiplies whatever W.
template <int W>
__device__ __forceinline__ unsigned long long key_hash(const unsigned long long key[W]) {
  unsigned long long h = key[W - 1];
#pragma unroll
  for (int j = W - 2; j >= 0; --j) {
    const int r = (23 * (W - 1 - j)) & 63;
    h ^= r ? ((key[j] << r) | (key[j] >> (64 - r))) : key[j] * 0x94D049BB133111EBull;
  }
  h ^= h >> 31;
  h *= 0x9E3779B97F4A7C15ull;
  h ^= h >> 29;
  h *= 0xD6E8FEB86659FD93ull;
  h ^= h >> 32;
  return h;
}

// MurmurHash3 32-bit finalizer (Appleby): minimizer -> bin mixer.
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

__device__ __forceinline__ void set_err(Counters* c, uint32_t bits) { atomicOr(&c->err, bits); }

}  // namespace gerbil
