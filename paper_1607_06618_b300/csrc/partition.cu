// partition.cu -- phase one on the GPU: 2-bit encoding, rolling minimizers, super-mer split
// and bin scatter (Sec. 2.1, Fig. 1; Sec. 2.3 Phase One; Sec. 3.1-3.2).
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace gerbil {

// ---- N1: ASCII -> 2-bit codes + undetermined-base mask -------------------------------------
// One thread per 32 bases: packed word (A=0 C=1 G=2 T=3, first base high) and a 32-bit mask
// of undetermined bases (Sec. 2.4.1: anything but ACGTacgt).
__device__ __forceinline__ void encode_byte(uint32_t c, unsigned long long& word, uint32_t& mask,
                                            int j) {
  const uint32_t u = c & 0xDFu;  // upper case
  const bool ok = (u == 'A') | (u == 'C') | (u == 'G') | (u == 'T');
  uint32_t t = (u >> 1) & 3u;  // A->0 C->1 G->3 T->2
  t ^= t >> 1;                 // A->0 C->1 G->2 T->3
  word |= (unsigned long long)(ok ? t : 0u) << (62 - 2 * j);
  mask |= (ok ? 0u : 1u) << (31 - j);
}

// 0x80 in every byte of x that is not zero, 0 elsewhere (the low seven bits plus 0x7F carry
// into bit 7 when any is set; no byte carries into the next).
__device__ __forceinline__ uint32_t nonzero_bytes(uint32_t x) {
  return (((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x) & 0x80808080u;
}

// The same encoding for the four bases of one little-endian 32-bit word (first base in the low
// byte), all four bytes at once: codes = the four 2-bit codes, first base in bits 7..6; bad = the
// four undetermined flags, first base in bit 3.  Equal to encode_byte on each byte for every
// 32-bit input.
__device__ __forceinline__ void encode_word4(uint32_t v, uint32_t& codes, uint32_t& bad) {
  const uint32_t u = v & 0xDFDFDFDFu;
  const uint32_t none = nonzero_bytes(u ^ 0x41414141u) & nonzero_bytes(u ^ 0x43434343u) &
                        nonzero_bytes(u ^ 0x47474747u) & nonzero_bytes(u ^ 0x54545454u);
  uint32_t t = (u >> 1) & 0x03030303u;
  t ^= (t >> 1) & 0x01010101u;
  const uint32_t b = none >> 7;  // 1 in the low bit of every undetermined byte
  t &= (b ^ 0x01010101u) * 3u;   // undetermined bases encode as 0
  // Gather the byte fields with one multiply each: byte i's field lands at bit 30 - 2i (codes)
  // or 27 - i (flags), and no two partial products overlap.
  codes = (t * 0x40100401u) >> 24;
  bad = (b * 0x08040201u) >> 24;
}

__global__ void __launch_bounds__(256) encode_kernel(const uint8_t* __restrict__ seq, uint64_t n,
                                                     unsigned long long* __restrict__ packed,
                                                     uint32_t* __restrict__ nmask,
                                                     uint64_t nwords, int vec_ok) {
  for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < nwords;
       w += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t b0 = w * 32;
    unsigned long long word = 0;
    uint32_t mask = 0;
    if (vec_ok && b0 + 32 <= n) {
      const uint4* p = reinterpret_cast<const uint4*>(seq + b0);
      const uint4 a = __ldg(p), b = __ldg(p + 1);
      const uint32_t v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        uint32_t codes, bad;
        encode_word4(v[q], codes, bad);
        word |= (unsigned long long)codes << (56 - 8 * q);
        mask |= bad << (28 - 4 * q);
      }
    } else {
      for (int j = 0; j < 32; ++j) {
        if (b0 + j < n)
          encode_byte(seq[b0 + j], word, mask, j);
        else
          mask |= 1u << (31 - j);  // past the end: undetermined
      }
    }
    packed[w] = word;
    nmask[w] = mask;
  }
}

// Read boundaries: bit at every offsets[r] (read starts and the end of the last read).
// Offsets past the input or out of order are reported (err) and skipped.
__global__ void boundary_kernel(const uint64_t* __restrict__ offsets, uint64_t nreads, uint64_t n,
                                uint32_t* __restrict__ bmask, unsigned int* __restrict__ err) {
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r <= nreads;
       r += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = offsets[r];
    if (i > n || (r > 0 && offsets[r - 1] > i)) {
      atomicOr(err, ERR_STATE);
      continue;
    }
    atomicOr(bmask + (i >> 5), 1u << (31 - (i & 31)));
  }
}

// ---- N2/N3: minimizers, super-mers, bins ---------------------------------------------------
// One CTA owns the window starts [P0, P0+T) of the global base stream.  It stages the 2-bit
// bases and masks it needs in shared memory and gives every m-mer a key: 0 if the m-mer holds
// an undetermined base or straddles a read start, else 1 + its rank.  The sliding minimum of
// the keys over w = k-m+1 m-mers (van Herk / Gil-Werman: the m-mers are cut into blocks of w,
// each with its running minima from the left and from the right, and a window, which spans
// the end of one block and the start of the next, takes the minimum of one of each) is then 0
// exactly for the windows that are not counted (for m >= 2 every interior read start is
// straddled by one of the window's m-mers), and 1 + the minimizer's rank otherwise.  Super-mer
// starts and ends are two bit masks over the windows, one word of 32 windows per thread; a
// super-mer never runs past the next multiple of L_max, so the CTA looks at most
// L_max windows past its range.  Each super-mer becomes one record (start, k-mers, bin),
// appended with one atomic per warp, and counted into its bin.

constexpr int SEG = 8;  // consecutive m-mers per thread in the key pass
#ifndef GERBIL_SUPER_TILE
#define GERBIL_SUPER_TILE 3072
#endif
#ifndef GERBIL_SUPER_MINB
// resident CTAs per SM the registers are held to: 6 (39 registers, no spills); shared memory
// allows 7, at which the kernel spills 16 bytes and ran 0.5% slower on k = 65 and k = 99
#define GERBIL_SUPER_MINB 6
#endif
constexpr int SUPER_TILE = GERBIL_SUPER_TILE;  // window starts per CTA
constexpr int SUPER_WORDS = SUPER_TILE / 32 + 1;  // mask words holding a CTA's windows 0..tile

__device__ __forceinline__ unsigned long long bases64(const unsigned long long* sw, int lb) {
  const int w = lb >> 5, o = 2 * (lb & 31);
  return o ? ((sw[w] << o) | (sw[w + 1] >> (64 - o))) : sw[w];
}
__device__ __forceinline__ uint32_t bits32(const uint32_t* sm, int lb) {
  const int w = lb >> 5, o = lb & 31;
  return o ? ((sm[w] << o) | (sm[w + 1] >> (32 - o))) : sm[w];
}

// Bit 31-d of the result is set if any of bits 31-d .. 32-d-L of x is (L consecutive bases
// from base d, first base at bit 31): x OR-ed with itself shifted by 1 .. L-1, in doubling steps.
template <int L>
__device__ __forceinline__ uint32_t spread(uint32_t x) {
  if constexpr (L <= 1) {
    return x;
  } else {
    constexpr int H = L / 2;
    const uint32_t y = spread<H>(x);
    const uint32_t z = y | (y << H);          // covers 2H
    if constexpr (L % 2) return z | (x << (L - 1));
    else return z;
  }
}

// KMC2 reading (Sec. 3.1): demote m-mers that start with AAA or ACA or hold AA past
// position 0.  v holds m bases in its low 2m bits, first base most significant.
__device__ __forceinline__ uint32_t kmc2_demoted(uint32_t v, int m) {
  if (m < 3) return 0u;
  const uint32_t head = v >> (2 * m - 6);
  uint32_t d = (head == 0u) | (head == 4u);  // AAA = 000000, ACA = 000100
  const uint32_t lowbits = (1u << (2 * m)) - 1u;
  const uint32_t a = ~(v | (v >> 1)) & 0x55555555u & lowbits;  // low bit of group set iff A
  uint32_t pairs = a & (a >> 2);    // group g-1 flagged iff groups g and g-1 are A
  pairs &= ~(1u << (2 * (m - 2)));  // drop the pair at position 0
  return d | (pairs != 0u);
}

// The orderings of Sec. 3.1 on the 2-bit value c of an m-mer (A0 C1 G2 T3, first base high),
// as ranks (smaller = preferred); every one is a bijection of [0, 4^m) except KMC2, which adds
// a demotion bit above it.
//   CGAT: digits C0 G1 A2 T3 -- per base (h, l) -> (not (h xor l), h).
//   Roberts: bases at even positions counting the first base as position 1 (the 2nd, 4th, ...)
//     complemented, then digits C0 A1 T2 G3 -- complement is xor 3, the digit map is xor 1; so
//     CGCG... becomes CCCC..., the smallest, as the ordering intends.
//   Random: a fixed permutation of [0, 4^m): multiply by an odd constant and fold the high
//     half into the low half, twice, within 2m bits.
//   dfp(p): a table of ranks built on the host from sampled m-mer frequencies.
__device__ __forceinline__ uint32_t order_rank(uint32_t c, int m, int ordering,
                                               const uint32_t* __restrict__ table) {
  const uint32_t lowbits = (m >= 16) ? 0xFFFFFFFFu : ((1u << (2 * m)) - 1u);
  const uint32_t L = 0x55555555u & lowbits;  // low bit of every base
  switch (ordering) {
    case 0: return c | (kmc2_demoted(c, m) << 30);
    case 2: {
      const uint32_t h = (c >> 1) & L, l = c & L;
      return ((~(h ^ l) & L) << 1) | h;
    }
    case 3: {
      uint32_t even = 0;  // both bits of the 2nd, 4th, ... base
      for (int i = 1; i < m; i += 2) even |= 3u << (2 * (m - 1 - i));
      return c ^ even ^ L;
    }
    case 4: {
      unsigned long long x = c;
      x = (x * 0x9E3779B97F4A7C15ull) & lowbits;
      x ^= x >> m;
      x = (x * 0xBF58476D1CE4E5B9ull) & lowbits;
      x ^= x >> m;
      return (uint32_t)x;
    }
    case 5: return __ldg(table + c);
    default: return c;
  }
}

// MLEN: the minimizer length, so that every shift below is a constant; KMC2: the ordering is
// GERBIL_ORDER_KMC2 (the default), ranked inline instead of through order_rank's switch.
template <int MLEN, bool KMC2>
__global__ void __launch_bounds__(256, GERBIL_SUPER_MINB) supermer_kernel(SupermerParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const long long T = P.tile;
  const long long P0 = (long long)blockIdx.x * T;
  const long long nwin = (long long)P.nwin;
  if (P0 >= nwin) return;
  const long long P1 = min(P0 + T, nwin);
  const long long O = P0 - 1;  // global window / base of local index 0
  constexpr int m = MLEN;
  const int k = P.k, w = k - m + 1;
  const long long lmax = P.lmax;
  const int NW = (int)(min(P1 + lmax, nwin) - O);
  const int NQ = NW + (k - m);
  const int NB = NW + k - 1;
  const long long wlo = (O >= 0) ? (O >> 5) : -1;  // first staged word
  const int nsw = (int)(((O + NB - 1) >> 5) - wlo) + 2;

  // shared memory: staged words and masks | PRE (the keys, then their running minima from the
  // left within blocks of w) | SUF (the keys, then from the right) | SB | BB.  PRE and SUF are indexed through
  // pidx(q) = q + q/32, so that the eight stores of a thread's segment (stride 8 across the
  // warp) hit distinct banks.
  const int NSEG = (NQ + SEG - 1) / SEG;
  const int NQP = NQ + (NQ >> 5) + 1;
  unsigned long long* sw = reinterpret_cast<unsigned long long*>(smem);
  uint32_t* snm = reinterpret_cast<uint32_t*>(sw + nsw);
  uint32_t* sbm = snm + nsw;
  uint32_t* PRE = sbm + nsw;
  uint32_t* SUF = PRE + NQP;
  const int nbw = (NW + 31) >> 5;
  uint32_t* SB = SUF + NQP;
  uint32_t* BB = SB + nbw;

  const long long nwords = (long long)P.nwords;
  for (int i = threadIdx.x; i < nsw; i += blockDim.x) {
    const long long g = wlo + i;
    const bool in = g >= 0 && g < nwords;
    sw[i] = in ? __ldg(P.packed + g) : 0ull;
    snm[i] = in ? __ldg(P.nmask + g) : 0xFFFFFFFFu;
    sbm[i] = in ? __ldg(P.bmask + g) : 0xFFFFFFFFu;
  }
  __syncthreads();

  // keys of the m-mers, SEG consecutive ones per thread, all cut from one 32-base window and
  // its reverse complement, stored in PRE
  const int lbO = (int)(O - 32 * wlo);  // local base index of global base O
  const long long n = (long long)P.n;
  const uint32_t vmask = (1u << (2 * m)) - 1u;
  // local index ranges of m-mers inside the input (q >= 0, q + m <= n) and of windows
  // inside it (0 <= p < nwin), so that the loops below use 32-bit indices only
  const int q_lo = (O < 0) ? 1 : 0;
  const int q_hi = (int)min((long long)NQ, n - m - O + 1);
  const int p_hi = (int)min((long long)NW, nwin - O);
  const uint32_t Omod = (uint32_t)(((O % lmax) + lmax) % lmax);
  for (int seg = threadIdx.x; seg < NSEG; seg += blockDim.x) {
    const int q0 = seg * SEG;
    const int lb = lbO + q0;
    const unsigned long long win = bases64(sw, lb);
    const unsigned long long rcwin = rev2(~win);
    // bit 31-d of bad: m-mer q0+d holds an undetermined base, straddles a read start (one at
    // bases d+1 .. d+m-1), or lies outside [q_lo, q_hi)
    uint32_t bad = spread<m>(bits32(snm, lb));
    if constexpr (m >= 2) bad |= spread<m - 1>(bits32(sbm, lb) << 1);
    const int lo = q_lo - q0, hi = q_hi - q0;
    if (lo > 0) bad |= ~(0xFFFFFFFFu >> lo);
    if (hi < 32) bad |= hi <= 0 ? 0xFFFFFFFFu : (0xFFFFFFFFu >> hi);
    const int pq0 = q0 + (q0 >> 5);  // pidx(q0); a segment never crosses a 32-boundary
    auto key = [&](int d) -> uint32_t {
      if ((bad << d) & 0x80000000u) return 0u;
      const uint32_t v = (uint32_t)(win >> (64 - 2 * m - 2 * d)) & vmask;
      uint32_t c = v;
      if (P.canon_min) {
        const uint32_t rc = (uint32_t)(rcwin >> (2 * d)) & vmask;
        c = rc < v ? rc : v;
      }
      if constexpr (KMC2) return (c | (kmc2_demoted(c, m) << 30)) + 1u;
      else return order_rank(c, m, P.ordering, P.rank_table) + 1u;
    };
    if (q0 + SEG <= NQ) {
#pragma unroll
      for (int d = 0; d < SEG; ++d) PRE[pq0 + d] = SUF[pq0 + d] = key(d);
    } else {
      for (int d = 0; q0 + d < NQ; ++d) PRE[pq0 + d] = SUF[pq0 + d] = key(d);
    }
  }
  __syncthreads();
  // running minima within blocks of w m-mers, in place: one thread per block from the right
  // (SUF), and in the warps after those, one thread per block from the left (PRE); both arrays
  // start out holding the keys
  {
    const int nblk = (NQ + w - 1) / w;
    const int nblk32 = (nblk + 31) & ~31;  // the left-to-right threads start on a warp boundary
    for (int t = threadIdx.x; t < nblk32 + nblk; t += blockDim.x) {
      if (t < nblk32 && t >= nblk) continue;
      const bool right = t < nblk32;
      const int b0 = (right ? t : t - nblk32) * w;
      const int b1 = min(b0 + w, NQ);
      uint32_t run = 0xFFFFFFFFu;
      if (right) {
        for (int q = b1 - 1; q >= b0; --q) {
          run = min(run, SUF[q + (q >> 5)]);
          SUF[q + (q >> 5)] = run;
        }
      } else {
        for (int q = b0; q < b1; ++q) {
          run = min(run, PRE[q + (q >> 5)]);
          PRE[q + (q >> 5)] = run;
        }
      }
    }
  }
  __syncthreads();

  // window minimum: 0 = a window with an undetermined base or a read start inside, else
  // 1 + the minimizer's rank.  Window i covers m-mers i .. i+w-1: the end of i's block from i
  // (SUF) and the start of the next block up to i+w-1 (PRE), or all of i's block when i starts it
  auto wmin = [&](int i) -> uint32_t {
    const int bq = i + w - 1;
    return min(SUF[i + (i >> 5)], PRE[bq + (bq >> 5)]);
  };
  auto counted = [&](int i, uint32_t mk) -> bool {
    bool ok = i >= q_lo && i < p_hi && mk != 0u;
    if (m == 1 && ok) {  // m = 1: no m-mer straddles a read start, test the window itself
      const int lb = lbO + i;
      for (int c = 1; ok && c < k; c += 32) {
        const int l = min(32, k - c);
        ok = (bits32(sbm, lb + c) >> (32 - l)) == 0u;
      }
    }
    return ok;
  };

  // window minima and super-mer starts / boundaries as bit masks, one thread per mask word of
  // 32 consecutive windows, which it scans in order (no shuffles or votes): window i starts a
  // super-mer if it is counted and its predecessor is not, or has another minimizer, or i sits
  // on a multiple of L_max; a boundary is a start or an uncounted window (window 0, the
  // previous CTA's last, and the windows past NW are boundaries and never starts).
  {
    const uint32_t lm = (uint32_t)lmax;
    const bool pow2 = (lm & (lm - 1)) == 0;
    for (int wd = threadIdx.x; wd < nbw; wd += blockDim.x) {
      const int i0 = wd * 32;
      uint32_t pm = 0u, pv = 0u;  // minimum of window i0 - 1, and 1 if it is counted
      if (wd > 0) {
        pm = wmin(i0 - 1);
        pv = counted(i0 - 1, pm) ? 1u : 0u;
      }
      // PRE index of m-mer i0 + j + w - 1: base + j, plus one from the 32-boundary on
      const int c0 = i0 + w - 1;
      const int pbase = c0 + (c0 >> 5), jc = 32 - (c0 & 31);
      const int sbase = 33 * wd;  // SUF index of m-mer i0 + j: sbase + j
      uint32_t nz = 0u, df = 0u, ob = 0xFFFFFFFFu;
      auto scan = [&](auto FULL) {
        constexpr bool full = decltype(FULL)::value;
        uint32_t prev = pm;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          uint32_t mk = 0u;
          if (full || i0 + j < NW) mk = min(SUF[sbase + j], PRE[pbase + j + (j >= jc ? 1 : 0)]);
          nz |= (mk != 0u ? 1u : 0u) << j;
          df |= (mk != prev ? 1u : 0u) << j;
          prev = mk;
          if constexpr (m == 1) {  // no m-mer straddles a read start: test the window itself
            const int lb = lbO + i0 + j;
            bool ok = true;
            for (int c = 1; ok && c < k; c += 32) {
              const int l = min(32, k - c);
              ok = (bits32(sbm, lb + c) >> (32 - l)) == 0u;
            }
            if (!ok) ob &= ~(1u << j);
          }
        }
      };
      if (i0 + 32 <= NW) scan(std::true_type{});
      else scan(std::false_type{});
      // counted windows: q_lo <= i < p_hi, a minimum above 0 (and, for m = 1, no read start)
      uint32_t rb = 0xFFFFFFFFu;
      if (i0 < q_lo) rb &= 0xFFFFFFFFu << (q_lo - i0);
      const int hi = p_hi - i0;
      if (hi < 32) rb &= hi <= 0 ? 0u : ((1u << hi) - 1u);
      const uint32_t vb = nz & rb & ob;
      // windows on a multiple of L_max
      uint32_t cb = 0u;
      const uint32_t r0 = pow2 ? ((Omod + (uint32_t)i0) & (lm - 1u)) : ((Omod + (uint32_t)i0) % lm);
      for (unsigned long long c = r0 ? lm - r0 : 0u; c < 32ull; c += lm) cb |= 1u << c;
      uint32_t st = vb & (~((vb << 1) | pv) | df | cb);
      uint32_t bd = ~vb | st;
      if (wd == 0) {
        st &= ~1u;
        bd |= 1u;
      }
      SB[wd] = st;
      BB[wd] = bd;
    }
  }
  __syncthreads();

  // records: the starts among this CTA's windows 1..own, counted per mask word (an exclusive
  // prefix over the words by warp 0); room for all of the CTA's records is taken with one
  // atomic; then every thread takes starts r, r + 256, ... (records in window order): the word
  // holding start r, its bit, its end (the first boundary after it; a cut every L_max windows
  // bounds the search), its minimizer and bin
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int own = (int)(P1 - P0);
  const int ownw = (own >> 5) + 1;  // mask words holding windows 0..own (<= SUPER_WORDS)
  auto own_bits = [&](int wd) -> uint32_t {
    uint32_t b = SB[wd];
    if (wd == 0) b &= ~1u;                               // window 0 belongs to the previous CTA
    if (wd == (own >> 5)) b &= (2u << (own & 31)) - 1u;  // windows up to own
    return b;
  };
  __shared__ uint32_t s_wpre[SUPER_WORDS + 1];
  __shared__ unsigned long long s_rbase;
  if (warp == 0) {
    uint32_t carry = 0;
    for (int base = 0; base < ownw; base += 32) {
      const int wd = base + lane;
      const uint32_t c = wd < ownw ? __popc(own_bits(wd)) : 0u;
      uint32_t incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
      }
      if (wd < ownw) s_wpre[wd] = carry + incl - c;
      carry += __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
    if (lane == 0) {
      s_wpre[ownw] = carry;
      s_rbase = carry ? atomicAdd(P.rec_count, (unsigned long long)carry) : 0ull;
    }
  }
  __syncthreads();
  // one record per start i, the CTA's r-th: its end (the first boundary after it; a cut every
  // L_max windows bounds the search), its minimizer and bin
  auto emit = [&](int i, uint32_t r) {
    const int j = i + 1;
    int end = NW;
    for (int wj = j >> 5; wj < nbw; ++wj) {
      const uint32_t bb = BB[wj] & (wj == (j >> 5) ? (0xFFFFFFFFu << (j & 31)) : 0xFFFFFFFFu);
      if (bb) {
        end = min(NW, (wj << 5) + __ffs(bb) - 1);
        break;
      }
    }
    const uint32_t nk = (uint32_t)(end - i);
    const uint32_t h = fmix32((wmin(i) - 1u) & vmask);
    uint32_t bin;
    if (P.bounds) {
      uint32_t blo = 0, bhi = P.nbins - 1;  // number of split points <= h
      while (blo < bhi) {
        const uint32_t mid = (blo + bhi) >> 1;
        if (__ldg(P.bounds + mid) <= h) blo = mid + 1; else bhi = mid;
      }
      bin = blo;
    } else {
      bin = h % P.nbins;
    }
    atomicAdd(P.bin_nsuper + bin, 1ull);
    atomicAdd(P.bin_nkmers + bin, (unsigned long long)nk);
    const unsigned long long idx = s_rbase + r;
    if (idx < P.rec_cap)
      P.rec[idx] = make_ulonglong2((unsigned long long)(O + i), ((unsigned long long)bin << 32) | nk);
  };
  const uint32_t total = s_wpre[ownw];
  for (uint32_t r = threadIdx.x; r < total; r += blockDim.x) {
    int lo = 0, hi = ownw;  // s_wpre[lo] <= r < s_wpre[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (s_wpre[mid] <= r) lo = mid; else hi = mid;
    }
    uint32_t bits = own_bits(lo);
    for (uint32_t n = r - s_wpre[lo]; n > 0; --n) bits &= bits - 1u;  // drop the earlier starts
    emit(lo * 32 + __ffs(bits) - 1, r);
  }
}

// Scatter of the records into their bins.  A 64-bit atomic add of (1 << 32 | k-mers) takes
// both a super-mer's index and its first k-mer within the bin, so that within a bin super-mer
// order and k-mer order agree.  With few bins a CTA first sums its chunk of records per bin in
// shared memory (the same packed add, giving each record its place within the CTA's share)
// and then takes every bin's share with one global atomic.
constexpr int SCATTER_RPT = 8;       // records per thread per chunk
constexpr int SCATTER_MAX_BINS = 2048;

__global__ void __launch_bounds__(256) scatter_kernel(SupermerParams P, unsigned long long nrec) {
  extern __shared__ unsigned long long hist[];  // [nbins] local sums, then [nbins] global bases
  const uint32_t nb = P.nbins;
  const bool local = nb <= (uint32_t)SCATTER_MAX_BINS;
  const unsigned long long per = (unsigned long long)blockDim.x * SCATTER_RPT;
  for (unsigned long long c0 = blockIdx.x * per; c0 < nrec; c0 += (unsigned long long)gridDim.x * per) {
    ulonglong2 rec[SCATTER_RPT];
    unsigned long long mine[SCATTER_RPT];
    if (local) {
      for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = 0ull;
      __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < SCATTER_RPT; ++u) {
      const unsigned long long r = c0 + u * blockDim.x + threadIdx.x;
      if (r >= nrec) continue;
      rec[u] = P.rec[r];
      const uint32_t bin = (uint32_t)(rec[u].y >> 32), nk = (uint32_t)rec[u].y;
      mine[u] = atomicAdd(local ? hist + bin : P.bin_cursor + bin, (1ull << 32) | nk);
    }
    if (local) {
      __syncthreads();
      for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x)
        hist[nb + b] = hist[b] ? atomicAdd(P.bin_cursor + b, hist[b]) : 0ull;
      __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < SCATTER_RPT; ++u) {
      const unsigned long long r = c0 + u * blockDim.x + threadIdx.x;
      if (r >= nrec) continue;
      const uint32_t bin = (uint32_t)(rec[u].y >> 32);
      const unsigned long long g = local ? hist[nb + bin] : 0ull;
      const unsigned long long sidx = (g >> 32) + (mine[u] >> 32);
      const uint32_t koff = (uint32_t)g + (uint32_t)mine[u];
      if (sidx >= P.bin_nsuper[bin]) {  // never expected
        atomicOr(P.err, ERR_STATE);
        continue;
      }
      const unsigned long long idx = P.bin_sm_begin[bin] + sidx;
      P.sm_pos[idx] = rec[u].x;
      P.sm_koff[idx] = koff;
    }
    if (local) __syncthreads();  // hist is reused by the next chunk
  }
}

int supermer_tile() { return SUPER_TILE; }

size_t supermer_smem_bytes(int tile, int lmax, int k, int m) {
  (void)m;
  const long long NW = (long long)tile + 1 + lmax;
  const long long NQ = NW + k;  // upper bound (m >= 1)
  const long long NB = NW + k;
  const long long nsw = NB / 32 + 3;
  const long long NQP = NQ + NQ / 32 + 1;
  const long long nbw = (NW + 31) / 32;
  return nsw * 16 + 2 * NQP * 4 + 2 * nbw * 4 + 64;
}

cudaError_t launch_encode(const uint8_t* seq, uint64_t n, unsigned long long* packed,
                          uint32_t* nmask, uint64_t nwords, int vec_ok, int nsm,
                          cudaStream_t st) {
  if (nwords == 0) return cudaSuccess;
  const uint64_t blocks = std::min<uint64_t>((nwords + 255) / 256, (uint64_t)nsm * 16);
  encode_kernel<<<(unsigned)blocks, 256, 0, st>>>(seq, n, packed, nmask, nwords, vec_ok);
  return cudaGetLastError();
}

cudaError_t launch_boundary(const uint64_t* offsets, uint64_t nreads, uint64_t n, uint32_t* bmask,
                            unsigned int* err, cudaStream_t st) {
  const uint64_t blocks = std::min<uint64_t>((nreads + 1 + 255) / 256, 4096);
  boundary_kernel<<<(unsigned)blocks, 256, 0, st>>>(offsets, nreads, n, bmask, err);
  return cudaGetLastError();
}

// The dynamic shared memory limit is raised to one fixed ceiling (the same value from every
// host thread, so that concurrent contexts never lower it between another thread's setting
// and launch); the launch asks for what it needs.
constexpr int SUPER_SMEM_CEILING = 200 * 1024;

template <int M>
static cudaError_t launch_supermer_m(const SupermerParams& p, uint64_t blocks, size_t smem, cudaStream_t st) {
  if (smem > (size_t)SUPER_SMEM_CEILING) return cudaErrorInvalidValue;
  if (p.ordering == 0) {
    cudaError_t e = cudaFuncSetAttribute(supermer_kernel<M, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         SUPER_SMEM_CEILING);
    if (e != cudaSuccess) return e;
    supermer_kernel<M, true><<<(unsigned)blocks, 256, smem, st>>>(p);
  } else {
    cudaError_t e = cudaFuncSetAttribute(supermer_kernel<M, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         SUPER_SMEM_CEILING);
    if (e != cudaSuccess) return e;
    supermer_kernel<M, false><<<(unsigned)blocks, 256, smem, st>>>(p);
  }
  return cudaGetLastError();
}

cudaError_t launch_supermer(const SupermerParams& p, cudaStream_t st) {
  if (p.nwin == 0) return cudaSuccess;
  if (p.tile < 32 || p.tile > SUPER_TILE) return cudaErrorInvalidValue;  // record-word staging
  const uint64_t blocks = (p.nwin + p.tile - 1) / p.tile;
  const size_t smem = supermer_smem_bytes(p.tile, p.lmax, p.k, p.m);
  switch (p.m) {
    case 1: return launch_supermer_m<1>(p, blocks, smem, st);
    case 2: return launch_supermer_m<2>(p, blocks, smem, st);
    case 3: return launch_supermer_m<3>(p, blocks, smem, st);
    case 4: return launch_supermer_m<4>(p, blocks, smem, st);
    case 5: return launch_supermer_m<5>(p, blocks, smem, st);
    case 6: return launch_supermer_m<6>(p, blocks, smem, st);
    case 7: return launch_supermer_m<7>(p, blocks, smem, st);
    case 8: return launch_supermer_m<8>(p, blocks, smem, st);
    case 9: return launch_supermer_m<9>(p, blocks, smem, st);
    case 10: return launch_supermer_m<10>(p, blocks, smem, st);
    case 11: return launch_supermer_m<11>(p, blocks, smem, st);
    case 12: return launch_supermer_m<12>(p, blocks, smem, st);
    case 13: return launch_supermer_m<13>(p, blocks, smem, st);
    case 14: return launch_supermer_m<14>(p, blocks, smem, st);
    case 15: return launch_supermer_m<15>(p, blocks, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

// One warp per sampled read (reads 0, every, 2 * every, ...), lanes over its m-mer starts; an
// m-mer with an undetermined base is skipped.
__global__ void __launch_bounds__(256) mmer_freq_kernel(const unsigned long long* __restrict__ packed,
                                                       const uint32_t* __restrict__ nmask,
                                                       const uint64_t* __restrict__ offsets,
                                                       uint64_t nreads, uint32_t every, int m,
                                                       int canon_min, uint32_t* __restrict__ freq) {
  const int lane = threadIdx.x & 31;
  const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const uint64_t w0 = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  for (uint64_t r = w0 * every; r < nreads; r += nwarps * every) {
    const uint64_t start = offsets[r], end = offsets[r + 1];
    for (uint64_t q = start + lane; q + m <= end; q += 32) {
      const uint64_t wq = q >> 5;
      const int o = (int)(q & 31);
      const uint32_t nm = o ? ((nmask[wq] << o) | (nmask[wq + 1] >> (32 - o))) : nmask[wq];
      if (nm >> (32 - m)) continue;
      const unsigned long long win = o ? ((packed[wq] << (2 * o)) | (packed[wq + 1] >> (64 - 2 * o)))
                                       : packed[wq];
      const uint32_t v = (uint32_t)(win >> (64 - 2 * m));
      uint32_t c = v;
      if (canon_min) {
        const uint32_t rc = (uint32_t)(rev2(~(unsigned long long)v) >> (64 - 2 * m));
        c = rc < v ? rc : v;
      }
      atomicAdd(freq + c, 1u);
    }
  }
}

cudaError_t launch_mmer_freq(const unsigned long long* packed, const uint32_t* nmask,
                             const uint64_t* offsets, uint64_t nreads, uint32_t every, int m,
                             int canon_min, uint32_t* freq, int nsm, cudaStream_t st) {
  if (nreads == 0) return cudaSuccess;
  const uint64_t sampled = (nreads + every - 1) / every;
  const unsigned blocks = (unsigned)std::min<uint64_t>((sampled + 7) / 8, (uint64_t)nsm * 16);
  mmer_freq_kernel<<<blocks, 256, 0, st>>>(packed, nmask, offsets, nreads, every, m, canon_min, freq);
  return cudaGetLastError();
}

cudaError_t launch_scatter(const SupermerParams& p, unsigned long long nrec, int nsm, cudaStream_t st) {
  if (nrec == 0) return cudaSuccess;
  const unsigned long long per = 256ull * SCATTER_RPT;
  const unsigned blocks = (unsigned)std::min<unsigned long long>((nrec + per - 1) / per, (unsigned long long)nsm * 8);
  const size_t smem = p.nbins <= (uint32_t)SCATTER_MAX_BINS ? (size_t)p.nbins * 16 : 0;
  // at most SCATTER_MAX_BINS * 16 = 32 KB: within the default limit, no attribute needed
  scatter_kernel<<<blocks, 256, smem, st>>>(p, nrec);
  return cudaGetLastError();
}

}  // namespace gerbil
