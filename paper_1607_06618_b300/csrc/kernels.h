// kernels.h -- launch interface between the host runtime (runtime.cu) and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace gerbil {

struct Counters;

// ---- phase one ------------------------------------------------------------------------------
struct SupermerParams {
  const unsigned long long* packed;  // 2-bit bases, nwords + 2 padding words
  const uint32_t* nmask;             // undetermined-base mask, nwords + 2 words
  const uint32_t* bmask;             // read-start mask, nwords + 2 words
  uint64_t n;                        // bases in the input
  uint64_t nwords;                   // ceil((n + 1) / 32)
  uint64_t nwin;                     // window starts: n - k + 1 (0 if n < k)
  int k, m;
  int ordering, canon_min;
  uint32_t lmax;                     // super-mer cap L_max
  uint32_t nbins;
  const uint32_t* bounds;            // device, nbins-1 split points, or NULL
  const uint32_t* rank_table;        // dfp ordering: rank of every m-mer value (4^m entries)
  int tile;                          // window starts per CTA
  // supermer_kernel: per-bin counts and one record per super-mer
  unsigned long long* bin_nsuper;
  unsigned long long* bin_nkmers;
  ulonglong2* rec;                   // (start, bin << 32 | k-mers)
  unsigned long long rec_cap;
  unsigned long long* rec_count;     // records produced (may exceed rec_cap: then rerun)
  // scatter_kernel
  const unsigned long long* bin_sm_begin;
  unsigned long long* bin_cursor;    // (super-mers << 32) | k-mers, cleared before pass 1
  unsigned long long* sm_pos;        // global start of each super-mer
  uint32_t* sm_koff;                 // first k-mer of each super-mer within its bin
  unsigned int* err;                 // ERR_* bits
};

cudaError_t launch_encode(const uint8_t* seq, uint64_t n, unsigned long long* packed,
                          uint32_t* nmask, uint64_t nwords, int vec_ok, int nsm, cudaStream_t st);
cudaError_t launch_boundary(const uint64_t* offsets, uint64_t nreads, uint64_t n, uint32_t* bmask,
                            unsigned int* err, cudaStream_t st);
cudaError_t launch_supermer(const SupermerParams& p, cudaStream_t st);
// Frequencies of the (canonical) m-mers of every `every`-th read, for the dfp ordering.
cudaError_t launch_mmer_freq(const unsigned long long* packed, const uint32_t* nmask,
                             const uint64_t* offsets, uint64_t nreads, uint32_t every, int m,
                             int canon_min, uint32_t* freq, int nsm, cudaStream_t st);
cudaError_t launch_scatter(const SupermerParams& p, unsigned long long nrec, int nsm, cudaStream_t st);
size_t supermer_smem_bytes(int tile, int lmax, int k, int m);
int supermer_tile();  // window starts per CTA of the super-mer kernel

// ---- phase two ------------------------------------------------------------------------------
// One entry per bin being counted.
struct BinWork {
  unsigned long long sm_begin;   // first super-mer of the bin in sm_pos / sm_koff
  unsigned long long table_off;  // first slot of the bin's table in the arena
  uint32_t n_super;
  uint32_t n_kmers;
  uint32_t cap;                  // table slots
  uint32_t item_begin;           // first global work item of the bin
  // fused (persistent) form only
  uint32_t task_insert;          // queue position of the bin's first insert item
  uint32_t task_compact;         // queue position of the bin's first compaction chunk
  uint32_t n_items;
  uint32_t n_chunks;
  uint32_t dep_begin;            // this bin's entries in FusedParams::deps: the earlier bins
  uint32_t dep_count;            // whose table regions it reuses (their compaction comes first)
  uint32_t item_kmers;           // k-mers per insert work item of this bin: 64, 128 or 256
  uint32_t scheme;               // probe scheme: 0 linear, 1 windowed double hashing (count.cu)
};

constexpr int COUNT_THREADS = 256;
constexpr int ITEM_KMERS = 256;  // the largest work item: k-mers of an item staged per warp



struct CountParams {
  const unsigned long long* packed;
  const unsigned long long* sm_pos;
  const uint32_t* sm_koff;
  const BinWork* work;
  uint32_t nwork;
  unsigned long long nitems;     // end of the items of this launch
  unsigned long long item_base;  // first item of this launch
  unsigned long long* queue;     // item counter (schedule 1), zero before the launch
  unsigned long long* imap;      // item -> (work index << 32 | first super-mer of the item)
  int k;
  int canonical;
  uint32_t theta;                // max probes (Alg. 1)
  uint32_t spin_limit;           // bounded wait on a slot whose key is being written
  int schedule;                  // 1: items from a device counter in order; 0: fixed striding
  unsigned long long* arena;     // all tables, slot_words_for_k(k) words per slot
  unsigned long long* ovf;       // overflow area, W words per k-mer
  unsigned long long ovf_cap;
  uint32_t* bin_ovf;             // overflow k-mers per work entry
  Counters* ctr;
  // probe statistics (NULL: off): per placed k-mer, slots read and 128-byte lines touched
  unsigned long long* probe_hist;  // [2][PROBE_BUCKETS]
  // 1: the bins' tables average more than the L2 cache (keys of six or more words then run the
  // insert kernel without its register cap)
  int wide_tables;
  int scheme;                    // probe scheme of every bin of the launch (BinWork::scheme)
  int cas_first;                 // 1: every probe claims with a CAS before reading the key
                                 // words (mostly new keys); 0: reads the slot first
  uint32_t item_kmers;           // k-mers per work item of every bin of the launch: 64, 128
                                 // or 256 (64 and 128 for keys of up to four words only)
};

// Probe histogram buckets: [0, 32) = 1..32 probes, 32 = more, 33 = sent to the overflow area.
constexpr int PROBE_BUCKETS = 34;

constexpr int CHUNK_SLOTS = 2048;  // slots per compaction task of the fused kernel

// Persistent phase-two kernel: one queue of insert items and compaction chunks in bin order.
struct FusedParams {
  CountParams c;                 // insert side (c.imap unused)
  const unsigned long long* tasks;  // (compact << 63 | work index << 32 | s_lo or chunk)
  const uint32_t* deps;          // work indices, see BinWork::dep_begin
  unsigned long long ntasks;
  uint32_t* items_done;          // per work entry
  uint32_t* chunks_done;         // per work entry
  uint32_t min_count;
  unsigned long long* out_keys;
  uint32_t* out_counts;
  unsigned long long out_cap;
  unsigned long long wait_ns;    // bound of every dependency wait
  unsigned long long* queue;     // queue head (own 256-byte line)
};

struct CompactParams {
  const BinWork* work;
  uint32_t nwork;
  unsigned long long slot_lo, slot_hi;  // slots of the arena to scan
  unsigned long long* arena;
  const uint32_t* bin_ovf;
  int mode;                      // 0: skip bins with overflow; 1: only those, merged with O;
                                 // 2: count rows only (out_count), write nothing
  unsigned long long* otab;      // overflow recount table
  uint32_t ocap;
  uint32_t min_count;
  unsigned long long* out_keys;
  uint32_t* out_counts;
  unsigned long long out_cap;
  Counters* ctr;
  int zero;                      // modes 0 and 1: zero every slot taken (the arena stays clean)
};

struct OverflowParams {
  const unsigned long long* ovf;
  unsigned long long ovf_cap;
  unsigned long long* otab;
  uint32_t ocap;
  uint32_t spin_limit;
  uint32_t min_count;
  unsigned long long* out_keys;
  uint32_t* out_counts;
  unsigned long long out_cap;
  Counters* ctr;
};

// Table slots hold the key's low 30 bits in the meta word and the rest cut into
// stored_words(k) = max(1, ceil((2k - 30) / 63)) marked words (see common.cuh); a slot is
// slot_words_for_k(k) 64-bit words.  Launchers dispatch on k.
int stored_words(int k);
int slot_words_for_k(int k);
// slots per probe window of scheme 1 for keys of length k (a table's cap and first slot are
// multiples of it when it uses scheme 1)
uint32_t probe_window_for_k(int k);
// imap of items [0, p.nitems): one thread per item (p.work, p.nwork, p.sm_koff)
cudaError_t launch_item_map(const CountParams& p, int nsm, cudaStream_t st);
cudaError_t launch_task_map(const FusedParams& p, cudaStream_t st);
cudaError_t launch_fused(int k, const FusedParams& p, int nsm, cudaStream_t st);
cudaError_t launch_insert(int k, const CountParams& p, int persistent, int nsm, cudaStream_t st);
// the insert launches of each group of key widths (insert_w*.cu)
cudaError_t launch_insert_w1_2(int W, int WS, const CountParams& p, unsigned long long need,
                            int persistent, int nsm, cudaStream_t st);
cudaError_t launch_insert_w3(int W, int WS, const CountParams& p, unsigned long long need,
                            int persistent, int nsm, cudaStream_t st);
cudaError_t launch_insert_w4(int W, int WS, const CountParams& p, unsigned long long need,
                            int persistent, int nsm, cudaStream_t st);
cudaError_t launch_insert_w5_7(int W, int WS, const CountParams& p, unsigned long long need,
                            int persistent, int nsm, cudaStream_t st);
cudaError_t launch_insert_w8_11(int W, int WS, const CountParams& p, unsigned long long need,
                            int persistent, int nsm, cudaStream_t st);
cudaError_t launch_insert_w12_15(int W, int WS, const CountParams& p, unsigned long long need,
                            int persistent, int nsm, cudaStream_t st);
// one warp waits (bounded by wait_ns) for *flag >= 1, which nothing sets: records ERR_QUEUE
cudaError_t launch_wait_selftest(const uint32_t* flag, unsigned long long wait_ns, Counters* c,
                                 cudaStream_t st);
cudaError_t launch_compact(int k, const CompactParams& p, int nsm, cudaStream_t st);
cudaError_t launch_overflow_insert(int k, const OverflowParams& p, int nsm, cudaStream_t st);
cudaError_t launch_overflow_emit(int k, const OverflowParams& p, int nsm, cudaStream_t st);

// ---- ascending key order of a result (sort.cu) ----
unsigned long long sort_tiles(unsigned long long n);
cudaError_t launch_sort_pass(const unsigned long long* kin, const uint32_t* cin,
                             unsigned long long* kout, uint32_t* cout, unsigned long long n, int W,
                             int pass, uint32_t* hist, uint32_t* total, cudaStream_t st);

// ---- App. C output records (encode.cu) ----
struct EncodeParams {
  const unsigned long long* keys;  // [n][W]
  const uint32_t* counts;          // [n]
  unsigned long long n;
  int k;
  const unsigned long long* tile_long;  // exclusive prefix of long-count rows per tile
  uint8_t* out;
  unsigned long long base;  // byte offset of row 0's record in out
};
cudaError_t launch_encode_count(const uint32_t* counts, unsigned long long n,
                                unsigned long long* tile_long, cudaStream_t st);
cudaError_t launch_encode_scan(unsigned long long* tile_long, unsigned long long ntiles,
                               unsigned long long* total, cudaStream_t st);
cudaError_t launch_encode_write(const EncodeParams& p, cudaStream_t st);
unsigned long long encode_tiles(unsigned long long n);

}  // namespace gerbil
