// kmer_oracle.cpp -- plain, slow, obviously correct CPU oracle for Gerbil's counting path.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or call this
// file; only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline legs (cpu_baseline
// and its sample check, the reference arm, each config's oracle rate and sample check, the k
// sweep's oracle rate and sample check) use it.  It shares no code, header, table or constant
// generator with the CUDA library.
//
// Every function works on ASCII strings, exactly as the paper states the problem:
//   * the k-mer counting problem (Abstract; Sec. 1): a histogram of all length-k substrings;
//   * undetermined bases (Sec. 2.4.1): every k-mer containing a non-ACGT symbol is ignored;
//   * reverse complement / canonical form (Sec. 2.4.2): reverse the k-mer, swap A<->T and
//     C<->G; the canonical k-mer is the lexicographically smaller of the two;
//   * minimal occurrence (App. A, flag -l): only k-mers with count >= min_count are output;
//   * minimizers and super-mers (Sec. 2.1, Fig. 1): a super-mer is a maximal substring whose
//     k-mers share one minimizer; the KMC2 ordering (Sec. 3.1) ranks the m-mers;
//   * output record encoding (App. C).
// Readings of points the paper leaves open are stated where they are used.
//
// Parity status: every function here is pinned by tests/test_oracle_pins.py (worked examples
// of Fig. 1, Sec. 2.4.2 and App. C, brute force on tiny inputs, closed forms, invariants).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <string>
#include <vector>

namespace {

// ---- plain string helpers --------------------------------------------------------------

// Sec. 2.4.1 reading: A, C, G, T in either case are determined bases; every other byte is "N".
bool is_base(uint8_t c) {
    return c == 'A' || c == 'C' || c == 'G' || c == 'T' || c == 'a' || c == 'c' || c == 'g' ||
           c == 't';
}

char upper(uint8_t c) { return (c >= 'a' && c <= 'z') ? char(c - 'a' + 'A') : char(c); }

// Sec. 2.4.2: reverse the string and replace A<->T, C<->G (written into r).
char complement_base(char c) {
    if (c == 'A') return 'T';
    if (c == 'C') return 'G';
    if (c == 'G') return 'C';
    if (c == 'T') return 'A';
    return '?';
}

void reverse_complement_into(const std::string& s, std::string& r) {
    r.resize(s.size());
    for (size_t i = 0; i < s.size(); ++i) {
        char c = s[s.size() - 1 - i];
        char d = '?';
        if (c == 'A') d = 'T';
        if (c == 'C') d = 'G';
        if (c == 'G') d = 'C';
        if (c == 'T') d = 'A';
        r[i] = d;
    }
}

std::string reverse_complement(const std::string& s) {
    std::string r;
    reverse_complement_into(s, r);
    return r;
}

// App. C base code: A=0, C=1, G=2, T=3.
uint64_t base_code(char c) {
    if (c == 'A') return 0;
    if (c == 'C') return 1;
    if (c == 'G') return 2;
    return 3;
}

// A k-mer as a big integer in base 4, first base most significant, spread over W 64-bit
// words, word 0 most significant.  Because ASCII orders 'A'<'C'<'G'<'T', this numeric order
// equals the lexicographic order of the strings.
std::vector<uint64_t> pack_words(const std::string& s, int W) {
    std::vector<uint64_t> w(W, 0);
    for (char c : s) {
        // shift the whole W-word integer left by two bits
        for (int j = 0; j < W; ++j) {
            uint64_t carry = (j + 1 < W) ? (w[j + 1] >> 62) : 0;
            w[j] = (w[j] << 2) | carry;
        }
        w[W - 1] |= base_code(c);
    }
    return w;
}

// FNV-1a 64-bit over the bytes of a string (Fowler, Noll, Vo).  Used only to split the
// oracle's work into G disjoint passes; unrelated to any hashing of the counting method.
uint64_t fnv1a64(const std::string& s) {
    uint64_t h = 0xcbf29ce484222325ull;
    for (char c : s) {
        h ^= uint64_t(uint8_t(c));
        h *= 0x100000001b3ull;
    }
    return h;
}

// The window [p, p+k) of read r is counted iff it lies inside the read and holds only
// determined bases.  The caller supplies the read's bytes.
bool window_ok(const uint8_t* read, uint64_t p, int k) {
    for (int i = 0; i < k; ++i)
        if (!is_base(read[p + i])) return false;
    return true;
}

std::string window_string(const uint8_t* read, uint64_t p, int len) {
    std::string s(len, '?');
    for (int i = 0; i < len; ++i) s[i] = upper(read[p + i]);
    return s;
}

// The same window copied into a reused string (no allocation per window).
void window_into(const uint8_t* read, uint64_t p, int len, std::string& s) {
    s.resize(len);
    for (int i = 0; i < len; ++i) s[i] = upper(read[p + i]);
}

struct CountResult {
    int W = 1;
    std::vector<uint64_t> keys;    // n * W words
    std::vector<uint64_t> counts;  // n
};

struct PartitionResult {
    // one row per super-mer: global start position, number of k-mers, bin, minimizer value
    std::vector<uint64_t> pos;
    std::vector<uint32_t> nkmers;
    std::vector<uint32_t> bin;
    std::vector<uint64_t> minimizer;
};

// ---- minimizer ordering (Sec. 3.1) --------------------------------------------------------

// KMC2 ordering, our reading of "lexicographic A<C<G<T with built-in exceptions for m-mers
// that start with AAA or ACA": an m-mer is demoted (ranked after every other m-mer) if it
// starts with AAA, starts with ACA, or contains AA at any position other than the very
// beginning.  Within each class the order is lexicographic.
bool kmc2_demoted(const std::string& s) {
    if (s.size() >= 3 && (s.compare(0, 3, "AAA") == 0 || s.compare(0, 3, "ACA") == 0))
        return true;
    return s.find("AA", 1) != std::string::npos;
}

uint64_t mmer_value(const std::string& s) {
    uint64_t v = 0;
    for (char c : s) v = v * 4 + base_code(c);
    return v;
}

enum { ORDER_KMC2 = 0, ORDER_LEX = 1, ORDER_CGAT = 2, ORDER_ROBERTS = 3, ORDER_RANDOM = 4,
       ORDER_DFP = 5 };

// Base-4 number of the string under an alphabet order given as the rank of A, C, G, T.
uint64_t alphabet_value(const std::string& s, const int rank_of[4]) {
    uint64_t v = 0;
    for (char c : s) v = v * 4 + uint64_t(rank_of[base_code(c)]);
    return v;
}

// Rank of an m-mer string under the ordering (Sec. 3.1): smaller rank = preferred minimizer.
uint64_t mmer_rank(const std::string& s, int ordering) {
    uint64_t v = mmer_value(s);
    uint64_t four_m = 1;
    for (size_t i = 0; i < s.size(); ++i) four_m *= 4;
    switch (ordering) {
        case ORDER_LEX:
            return v;
        case ORDER_CGAT: {  // lexicographic with C < G < A < T
            static const int r[4] = {2, 0, 1, 3};  // A C G T
            return alphabet_value(s, r);
        }
        case ORDER_ROBERTS: {  // the 2nd, 4th, ... base complemented, then C < A < T < G
            std::string t = s;
            for (size_t i = 1; i < t.size(); i += 2) t[i] = complement_base(t[i]);
            static const int r[4] = {1, 0, 3, 2};  // A C G T
            return alphabet_value(t, r);
        }
        case ORDER_RANDOM: {  // a fixed permutation of the 4^m values
            const uint64_t mask = four_m - 1;
            const int m = int(s.size());
            uint64_t x = (v * 0x9E3779B97F4A7C15ull) & mask;
            x ^= x >> m;
            x = (x * 0xBF58476D1CE4E5B9ull) & mask;
            x ^= x >> m;
            return x;
        }
        default:  // KMC2
            return kmc2_demoted(s) ? v + four_m : v;
    }
}

// MurmurHash3's 32-bit finalizer (Appleby), used as the minimizer -> bin mixer.  The paper
// leaves the map from minimizers to temporary files open; our reading: bin = fmix32(value)
// mod nbins, or, given nbins-1 ascending split points, the number of split points <= fmix32.
uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

uint32_t bin_of(uint64_t minimizer, uint32_t nbins, const uint32_t* bounds) {
    uint32_t h = fmix32(uint32_t(minimizer));
    if (!bounds) return h % nbins;
    uint32_t b = 0;
    for (uint32_t i = 0; i + 1 < nbins; ++i)
        if (bounds[i] <= h) b = i + 1;
    return b;
}

}  // namespace

extern "C" {

// Number of N-free k-windows (closed-form total of all counts at min_count = 1).
// Written as its own loop so that it does not share a code path with oracle_count.
uint64_t oracle_windows(const uint8_t* seq, const uint64_t* offsets, uint64_t nreads, int k) {
    uint64_t total = 0;
    for (uint64_t r = 0; r < nreads; ++r) {
        uint64_t len = offsets[r + 1] - offsets[r];
        uint64_t run = 0;  // length of the current run of determined bases
        for (uint64_t i = 0; i < len; ++i) {
            if (is_base(seq[offsets[r] + i])) {
                ++run;
                if (run >= uint64_t(k)) ++total;
            } else {
                run = 0;
            }
        }
    }
    return total;
}

// The k-mer counting problem, by its definition.  For every read and every window of k
// determined bases, the k-mer x (or, with canonical != 0, the smaller of x and its reverse
// complement) is counted in a std::map keyed by the k-mer string.  With npass > 1, only keys
// whose FNV-1a hash is = pass (mod npass) are kept: the same definition restricted to a
// disjoint slice of the keys, so that large inputs fit in host memory.
// Returns 0 and a handle on success; 1 on invalid arguments.
int oracle_count(const uint8_t* seq, const uint64_t* offsets, uint64_t nreads, int k,
                 int canonical, uint64_t min_count, uint32_t npass, uint32_t pass, void** out) {
    if (k < 1 || npass < 1 || pass >= npass) return 1;
    std::map<std::string, uint64_t> hist;
    std::string x, rc;
    for (uint64_t r = 0; r < nreads; ++r) {
        const uint8_t* read = seq + offsets[r];
        uint64_t len = offsets[r + 1] - offsets[r];
        if (len < uint64_t(k)) continue;
        for (uint64_t p = 0; p + k <= len; ++p) {
            if (!window_ok(read, p, k)) continue;
            window_into(read, p, k, x);
            const std::string* key = &x;
            if (canonical) {
                reverse_complement_into(x, rc);
                if (rc < x) key = &rc;
            }
            if (npass > 1 && fnv1a64(*key) % npass != pass) continue;
            hist[*key] += 1;
        }
    }
    CountResult* res = new CountResult;
    res->W = (2 * k + 63) / 64;
    for (const auto& kv : hist) {
        if (kv.second < min_count) continue;
        std::vector<uint64_t> w = pack_words(kv.first, res->W);
        res->keys.insert(res->keys.end(), w.begin(), w.end());
        res->counts.push_back(kv.second);
    }
    *out = res;
    return 0;
}

uint64_t oracle_count_size(void* h) { return static_cast<CountResult*>(h)->counts.size(); }

void oracle_count_copy(void* h, uint64_t* keys, uint64_t* counts) {
    CountResult* r = static_cast<CountResult*>(h);
    std::copy(r->keys.begin(), r->keys.end(), keys);
    std::copy(r->counts.begin(), r->counts.end(), counts);
}

void oracle_count_free(void* h) { delete static_cast<CountResult*>(h); }

// Phase one by its definition (Sec. 2.1, Fig. 1, Sec. 3.1).  For every window of k
// determined bases: its minimizer is the m-mer of smallest rank among its k-m+1 m-mers; with
// canonical_min != 0 each m-mer is first replaced by the smaller of itself and its reverse
// complement (our reading: this puts a k-mer and its reverse complement in the same bin).
// A super-mer is a maximal run of consecutive counted windows of one read that share the
// minimizer value.  Readings: a run is also cut before every window whose global start
// position is a multiple of lmax, which bounds a super-mer at lmax k-mers; the bin of a
// super-mer is bin_of(minimizer).  Rows are emitted in input order.
// Distance from pivot, dfp(p) (Sec. 3.1).  Frequencies of the m-mers are taken from a sample of
// the input -- our reading: every `every`-th read (reads 0, every, 2*every, ...), every m-mer
// of it without an undetermined base, canonical when minimizers are -- then the m-mers are
// sorted by ascending frequency (equal frequencies: by value), and re-sorted by the distance
// of that position to the pivot floor(4^m * p) (equal distances: the smaller position first).
// The rank of an m-mer is its place in the second order.
std::vector<uint32_t> dfp_ranks(const uint8_t* seq, const uint64_t* offsets, uint64_t nreads,
                                int m, int canonical_min, float p, uint32_t every) {
    const uint64_t n4 = uint64_t(1) << (2 * m);
    std::vector<uint64_t> freq(n4, 0);
    for (uint64_t r = 0; r < nreads; r += every) {
        const uint8_t* read = seq + offsets[r];
        const uint64_t len = offsets[r + 1] - offsets[r];
        for (uint64_t q = 0; q + m <= len; ++q) {
            if (!window_ok(read, q, m)) continue;
            std::string s = window_string(read, q, m);
            if (canonical_min) {
                std::string t = reverse_complement(s);
                if (t < s) s = t;
            }
            freq[mmer_value(s)] += 1;
        }
    }
    std::vector<uint64_t> by_freq(n4);
    for (uint64_t v = 0; v < n4; ++v) by_freq[v] = v;
    std::sort(by_freq.begin(), by_freq.end(), [&](uint64_t a, uint64_t b) {
        return freq[a] != freq[b] ? freq[a] < freq[b] : a < b;
    });
    // p is the 32-bit value of the library's option: the pivot is floor(4^m * p) in doubles
    double pd = p < 0 ? 0.0 : (p > 1 ? 1.0 : double(p));
    const uint64_t pivot = std::min<uint64_t>(n4 - 1, uint64_t(std::floor(double(n4) * pd)));
    std::vector<uint64_t> order(n4);  // positions in the frequency order
    for (uint64_t i = 0; i < n4; ++i) order[i] = i;
    auto dist = [&](uint64_t i) { return i > pivot ? i - pivot : pivot - i; };
    std::sort(order.begin(), order.end(), [&](uint64_t a, uint64_t b) {
        return dist(a) != dist(b) ? dist(a) < dist(b) : a < b;
    });
    std::vector<uint32_t> rank(n4);
    for (uint64_t r2 = 0; r2 < n4; ++r2) rank[by_freq[order[r2]]] = uint32_t(r2);
    return rank;
}

int oracle_partition_dfp(const uint8_t* seq, const uint64_t* offsets, uint64_t nreads, int k,
                         int m, uint32_t nbins, const uint32_t* bounds, int ordering,
                         int canonical_min, uint32_t lmax, float dfp_p, uint32_t dfp_every,
                         void** out) {
    if (m < 1 || m >= k || m > 15 || nbins < 1 || lmax < 1) return 1;
    if (ordering == ORDER_DFP && (m > 12 || dfp_every < 1)) return 1;
    std::vector<uint32_t> table;
    if (ordering == ORDER_DFP) table = dfp_ranks(seq, offsets, nreads, m, canonical_min, dfp_p, dfp_every);
    auto rank_of = [&](const std::string& s) -> uint64_t {
        return ordering == ORDER_DFP ? table[mmer_value(s)] : mmer_rank(s, ordering);
    };
    PartitionResult* res = new PartitionResult;
    for (uint64_t r = 0; r < nreads; ++r) {
        const uint8_t* read = seq + offsets[r];
        uint64_t len = offsets[r + 1] - offsets[r];
        if (len < uint64_t(k)) continue;
        bool prev_ok = false;
        uint64_t prev_min = 0;
        for (uint64_t p = 0; p + k <= len; ++p) {
            if (!window_ok(read, p, k)) {
                prev_ok = false;
                continue;
            }
            uint64_t best_rank = ~0ull, best_value = 0;
            for (int q = 0; q + m <= k; ++q) {
                std::string s = window_string(read, p + q, m);
                if (canonical_min) {
                    std::string t = reverse_complement(s);
                    if (t < s) s = t;
                }
                uint64_t rk = rank_of(s);
                if (rk < best_rank) {
                    best_rank = rk;
                    best_value = mmer_value(s);
                }
            }
            uint64_t gpos = offsets[r] + p;
            bool starts = !prev_ok || best_value != prev_min || gpos % lmax == 0;
            if (starts) {
                res->pos.push_back(gpos);
                res->nkmers.push_back(1);
                // the bin is a function of the minimizer: of its rank (a bijection of the
                // m-mer for every ordering; equal to the m-mer's value for KMC2 and LEX)
                res->bin.push_back(bin_of(best_rank & ((1ull << (2 * m)) - 1), nbins, bounds));
                res->minimizer.push_back(best_value);
            } else {
                res->nkmers.back() += 1;
            }
            prev_ok = true;
            prev_min = best_value;
        }
    }
    *out = res;
    return 0;
}

int oracle_partition(const uint8_t* seq, const uint64_t* offsets, uint64_t nreads, int k, int m,
                     uint32_t nbins, const uint32_t* bounds, int ordering, int canonical_min,
                     uint32_t lmax, void** out) {
    return oracle_partition_dfp(seq, offsets, nreads, k, m, nbins, bounds, ordering, canonical_min,
                                lmax, 0.5f, 16, out);
}

// dfp ranks of every m-mer value (exposed for pinning the ordering).
int oracle_dfp_ranks(const uint8_t* seq, const uint64_t* offsets, uint64_t nreads, int m,
                     int canonical_min, float p, uint32_t every, uint32_t* out) {
    if (m < 1 || m > 12 || every < 1) return 1;
    std::vector<uint32_t> t = dfp_ranks(seq, offsets, nreads, m, canonical_min, p, every);
    std::copy(t.begin(), t.end(), out);
    return 0;
}

uint64_t oracle_partition_size(void* h) { return static_cast<PartitionResult*>(h)->pos.size(); }

void oracle_partition_copy(void* h, uint64_t* pos, uint32_t* nkmers, uint32_t* bin,
                           uint64_t* minimizer) {
    PartitionResult* r = static_cast<PartitionResult*>(h);
    std::copy(r->pos.begin(), r->pos.end(), pos);
    std::copy(r->nkmers.begin(), r->nkmers.end(), nkmers);
    std::copy(r->bin.begin(), r->bin.end(), bin);
    std::copy(r->minimizer.begin(), r->minimizer.end(), minimizer);
}

void oracle_partition_free(void* h) { delete static_cast<PartitionResult*>(h); }

// Rank of one m-mer string under an ordering (exposed for pinning the KMC2 reading).
uint64_t oracle_mmer_rank(const char* s, int ordering) { return mmer_rank(std::string(s), ordering); }

uint32_t oracle_bin_of(uint64_t minimizer, uint32_t nbins, const uint32_t* bounds) {
    return bin_of(minimizer, nbins, bounds);
}

// App. C: one output record.  The counter takes one byte if it is below 255, else the byte
// 0xFF followed by the counter as a 32-bit unsigned integer, most significant byte first
// (the worked example 345 -> FF 00 00 01 59).  Then the k-mer, four bases per byte, A=00
// C=01 G=10 T=11, first base in the high bits; undefined trailing bits are written as 0.
// Returns the record length, or -1 if cap is too small or the k-mer holds a non-ACGT byte.
int oracle_encode_record(const char* kmer, uint32_t count, uint8_t* out, int cap) {
    int k = int(strlen(kmer));
    int need = (count < 255 ? 1 : 5) + (k + 3) / 4;
    if (need > cap) return -1;
    int o = 0;
    if (count < 255) {
        out[o++] = uint8_t(count);
    } else {
        out[o++] = 0xFF;
        out[o++] = uint8_t(count >> 24);
        out[o++] = uint8_t(count >> 16);
        out[o++] = uint8_t(count >> 8);
        out[o++] = uint8_t(count);
    }
    for (int i = 0; i < k; i += 4) {
        uint8_t b = 0;
        for (int j = 0; j < 4; ++j) {
            b <<= 2;
            if (i + j < k) {
                char c = upper(uint8_t(kmer[i + j]));
                if (!is_base(uint8_t(c))) return -1;
                b |= uint8_t(base_code(c));
            }
        }
        out[o++] = b;
    }
    return o;
}

}  // extern "C"
