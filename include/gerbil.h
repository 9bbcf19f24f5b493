/* gerbil.h -- C ABI of the B300-native hot path of Gerbil's two-phase k-mer counter
 * (Erbert, Rechner, Mueller-Hannemann, "Gerbil: A Fast and Memory-Efficient k-mer Counter
 * with GPU-Support", arXiv 1607.06618).
 *
 * Phase one (Sec. 2.1, Sec. 2.3 "Phase One"): reads are 2-bit encoded, split into super-mers
 * by their minimizers (Fig. 1, KMC2 ordering of Sec. 3.1) and distributed to bins -- the
 * paper's temporary files -- so that every occurrence of a k-mer lands in one bin.
 * Phase two (Sec. 2.2, Sec. 2.3 "Phase Two", Sec. 3.3-3.4): each bin's super-mers are split
 * into k-mers, each k-mer is replaced by its canonical form (Sec. 2.4.2) and counted in an
 * open-addressing hash table (Alg. 1); k-mers that exhaust the probe limit go to an
 * overflow area that is recounted afterwards (Sec. 3.4 "Probing Strategy"); the table is
 * then compacted under the minimal-occurrence filter (App. A, flag -l).
 *
 * Every step runs in hand-written CUDA kernels for sm_103a on the context's stream.  There
 * is no CPU fallback: without a usable device every call fails with GERBIL_E_CUDA.
 *
 * Conventions
 *  - Return value: 0 (GERBIL_OK) or a positive gerbil_status.  No call throws, traps or
 *    aborts; device kernels report problems through an error word read by the host.
 *  - Key layout: A=0, C=1, G=2, T=3 (App. C), first base most significant.  A k-mer is the
 *    base-4 integer of its bases held in W = ceil(2k/64) 64-bit words, word 0 most
 *    significant, unused high bits of word 0 zero.  Numeric order equals lexicographic order
 *    with A<C<G<T, so the canonical key is the numerically smaller of x and revcomp(x).
 *  - Results are unordered (one row per distinct key); callers sort if they need an order.
 *  - Ownership: the caller owns every buffer it passes and must keep it valid until the call
 *    returns.  Objects returned through out-parameters (gerbil_bins, gerbil_counts) are owned
 *    by the library until the matching *_free call, and must be freed before the context
 *    that made them is destroyed.  Device memory is charged against the context's budget.
 *  - Threading: one context must not be used by two host threads at once.
 */
#ifndef GERBIL_H
#define GERBIL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GERBIL_ABI_VERSION 1
/* Supported k, as in the paper (App. A flag -k: 8 to 479); keys of up to W = 15 words. */
#define GERBIL_MAX_K 479
#define GERBIL_MIN_K 8

typedef enum gerbil_status {
  GERBIL_OK = 0,
  GERBIL_E_INVAL = 1,       /* an argument is out of range or inconsistent */
  GERBIL_E_UNSUPPORTED = 2, /* valid per the paper, not built here (k > GERBIL_MAX_K) */
  GERBIL_E_NOMEM = 3,       /* the context's HBM budget (or the device) cannot hold the work */
  GERBIL_E_OVERFLOW = 4,    /* the overflow area stayed full after every retry */
  GERBIL_E_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  GERBIL_E_CUDA = 6,        /* a CUDA runtime call failed (see gerbil_last_error) */
  GERBIL_E_STATE = 7        /* a device consistency check failed (internal error) */
} gerbil_status;

typedef enum gerbil_ordering {
  GERBIL_ORDER_KMC2 = 0, /* Sec. 3.1 "KMC2": lexicographic, m-mers starting with AAA or ACA or
                            holding AA past position 0 ranked last (Gerbil's choice) */
  GERBIL_ORDER_LEX = 1,  /* plain lexicographic A<C<G<T (the ordering of Fig. 1) */
  GERBIL_ORDER_CGAT = 2, /* Sec. 3.1 "CGAT": lexicographic with C<G<A<T */
  GERBIL_ORDER_ROBERTS = 3, /* Sec. 3.1 "Roberts et al.": the bases at even positions (the
                            2nd, 4th, ... base) complemented, then lexicographic with C<A<T<G,
                            so that CGCG... ranks first */
  GERBIL_ORDER_RANDOM = 4, /* Sec. 3.1 "Random": a fixed permutation of the 4^m m-mers (multiply
                            by an odd constant and fold the high half of the 2m bits into the
                            low half, twice) */
  GERBIL_ORDER_DFP = 5   /* Sec. 3.1 "distance from pivot", dfp(p): the m-mers sorted by their
                            frequency in a sample of the reads (ascending; equal frequencies by
                            value), then by the distance of that place to floor(4^m p) (equal
                            distances: the smaller place first); p = opts->dfp_pivot, the
                            sample = every opts->dfp_sample-th read (reads 0, s, 2s, ...), every
                            m-mer of it without an undetermined base (canonical when the
                            minimizers are).  m <= 12. */
} gerbil_ordering;
/* With every ordering the minimizer is the canonical m-mer of smallest rank (canonical_minimizer
 * = 1) and its bin is bin_of(rank mod 4^m): for KMC2 and LEX that is the m-mer's value. */

typedef struct gerbil_ctx gerbil_ctx;       /* device, stream, memory budget, scratch */
typedef struct gerbil_bins gerbil_bins;     /* device-resident bins of super-mers */
typedef struct gerbil_counts gerbil_counts; /* device-resident (k-mer, count) rows */

/* Input reads.  Read i is seq[offsets[i] .. offsets[i+1]); offsets has nreads+1
 * non-decreasing entries and offsets[0] == 0.  Bytes other than A,C,G,T,a,c,g,t are
 * undetermined bases (Sec. 2.4.1): every k-mer holding one is ignored.  With on_device == 1
 * both pointers are device pointers on the context's device; with 0 they are host pointers
 * and the call copies them to the device on the context's stream. */
typedef struct gerbil_reads {
  const uint8_t* seq;
  const uint64_t* offsets;
  uint64_t nreads;
  int32_t on_device;
  int32_t reserved;
} gerbil_reads;

/* Options; fill with gerbil_opts_default() and change fields. */
typedef struct gerbil_opts {
  int32_t canonical;           /* 1: count min(x, revcomp(x)) (Sec. 2.4.2); 0: flag -d */
  int32_t ordering;            /* gerbil_ordering of the minimizers (Sec. 3.1) */
  int32_t canonical_minimizer; /* 1: minimizer over canonical m-mers, so x and revcomp(x)
                                  share a bin; 0: forward m-mers as in Fig. 1 (allowed only
                                  with canonical == 0) */
  uint32_t supermer_cap;       /* L_max: a super-mer is also cut before every window whose
                                  global start position is a multiple of L_max (1..1024,
                                  default 256) */
  const uint32_t* bin_bounds;  /* host pointer, NULL or nbins-1 ascending split points: bin =
                                  number of split points <= fmix32(minimizer); NULL: bin =
                                  fmix32(minimizer) mod nbins */
  uint32_t max_probes;         /* theta of Alg. 1: probes before a k-mer goes to overflow
                                  (default 1024: with linear probing at load <= 0.85 longer
                                  runs are vanishingly rare, so the overflow area stays empty) */
  float load_factor;           /* target table load (default 0.5) */
  float distinct_ratio;        /* expected distinct/occurrences per bin for table sizing
                                  (Sec. 3.4 "Estimating table sizes"); 0: 1.25 x the ratio
                                  the context measured on its last batch (1.0 at first) */
  uint32_t overflow_slots;     /* capacity of the overflow area in k-mers; 0: automatic */
  int32_t persistent;          /* 1 (default): the insert kernel runs as many CTAs as fit on
                                  the GPU at once, each warp striding over the work items of
                                  all bins in bin order; 0: one warp per work item */
  uint32_t ring_slots;         /* fused form: table slots of the ring (0: 60% of L2); waves:
                                  table slots per wave (0: 50% of L2) */
  int32_t fused;               /* 0 (default): separate insert and compaction kernels over
                                  tables that all stay allocated until the compaction;
                                  1: one kernel pops insert and compaction tasks of all bins
                                  from a device queue, with the tables of small bins in an
                                  L2-sized ring that is reused bin after bin; 2: waves of bins
                                  whose tables fit in half of L2, each cleared, filled and
                                  compacted in one reused region while hot in L2 */
  int32_t schedule;            /* insert work items: 1 (default) taken in bin order from a
                                  device counter; 0 fixed, each warp striding over them */
  uint32_t max_table_mib;      /* device memory the hash tables of one batch may take, MiB;
                                  a batch whose tables need more is counted in consecutive
                                  groups of bins under this limit (each k-mer lives in one
                                  bin, so the groups' rows are joined unchanged).  0 (default):
                                  half of what the context's budget leaves, or half of the
                                  device's free memory when the context has no budget */
  uint32_t autotune;           /* 1: use the context's tuned form, schedule and load factors
                                  for this key width (gerbil_autotune; run on the first batch
                                  of 8 bins or more when none is set); load_factor, fused and
                                  schedule above are then ignored.  0 (default): as given */
  uint32_t graph;              /* 1: the device steps of a two-grid batch (fused 0) -- table
                                  clears, work-list upload, item map, insert grid, compaction
                                  -- are captured into one CUDA graph and launched as one; the
                                  context keeps the instantiated graph and updates it in place
                                  for the next batch of the same shape.  0 (default): plain
                                  launches */
  float dfp_pivot;             /* p of GERBIL_ORDER_DFP, 0..1 (default 0.5) */
  uint32_t dfp_sample;         /* GERBIL_ORDER_DFP: frequencies from every dfp_sample-th read
                                  (default 16) */
  int32_t probe_scheme;        /* hash-table probing of the insert kernel (two-grid form,
                                  fused 0): 0 (default): linear probing from a fastrange slot;
                                  1: windowed double hashing as in Sec. 3.3-3.4 -- windows of
                                  one 128-byte line of slots (16- and 32-byte slots; wider
                                  slots: as many whole slots as fit, at least one), the first
                                  window and the window step taken from the key's hash, each
                                  window scanned from its first slot; max_probes then counts
                                  windows.  The other forms always probe linearly */
  uint32_t item_kmers;         /* k-mers per insert work item, i.e. 32 threads per item_kmers
                                  consecutive k-mers of a bin (two-grid form): 64, 128 or 256;
                                  0 (default): 256.  64 and 128 are built for keys of up to
                                  four words (k <= 128); wider keys: GERBIL_E_UNSUPPORTED */
  int32_t sorted_output;       /* 1: the rows of gerbil_count / gerbil_count_batch in
                                  ascending key order (numeric order of the 2k-bit keys = the
                                  lexicographic order of the k-mers, A < C < G < T), sorted on
                                  the device; a grouped result is joined first.  0 (default):
                                  unordered */
  int32_t claim_first;         /* probe order of the insert kernel: 0 (default): chosen per
                                  batch: claim first for keys of ten or more words
                                  (k > 288) when the distinct ratio the context learned is
                                  above 0.6, i.e. most k-mers are new keys; 1: each
                                  probe first tries to claim the slot with a CAS on its meta
                                  word and reads the key words only if the slot holds a key
                                  with the same tag (a new key costs one round trip to memory);
                                  2: each probe reads the slot first and claims only an empty
                                  one (a repeated key costs one round trip).  Counts do not
                                  depend on it */
} gerbil_opts;

/* Per-call statistics of a count. */
typedef struct gerbil_count_stats {
  uint64_t occurrences; /* k-mer occurrences inserted (N-free windows of the bins) */
  uint64_t distinct;    /* distinct keys before the min_count filter */
  uint64_t emitted;     /* rows in the result (count >= min_count) */
  uint64_t overflowed;  /* insertions that went to the overflow area */
  uint64_t table_slots; /* hash-table slots allocated over all bins */
  uint32_t retries;     /* rounds repeated with larger tables because overflow was full */
  uint32_t bins;        /* bins counted */
  uint32_t groups;      /* groups of bins counted one after another because the tables of
                           the whole batch did not fit under the table limit (0: one batch) */
  uint32_t sorted;      /* 1: the rows are in ascending key order (gerbil_opts.sorted_output) */
} gerbil_count_stats;

/* Device time of each step of the path, accumulated over the calls made since profiling was
 * last enabled (CUDA events recorded on the context's stream around each step). */
typedef struct gerbil_phase_times {
  double encode_ms;       /* 2-bit encoding and read-boundary marks (phase one) */
  double supermer_ms;     /* minimizers, super-mer split, bin count + scatter (phase one) */
  double clear_ms;        /* table and counter clears (phase two) */
  double insert_ms;       /* extract + canonicalise + insert launches (phase two) */
  double compact_ms;      /* compaction under min_count (phase two) */
  double overflow_ms;     /* overflow recount and merge (phase two) */
  uint64_t insert_launches;
  uint64_t kernel_launches; /* kernels of this library launched, counted with profiling off too */
  uint64_t calls;           /* partition + count calls */
  uint64_t graph_launches;  /* CUDA graph launches (gerbil_opts.graph) */
} gerbil_phase_times;

/* Settings chosen by the autotuner for one key width (the paper has no autotuner; its table
 * sizes follow one load factor).  Tables are put in a size class by their bytes at load factor
 * 0.5: below class_bytes[0], [1], [2], or larger; each class has its own load factor.  The
 * probe scheme and the work-item size hold for every table of the key width (each is a
 * compile-time form of the insert kernel, and one launch runs one form). */
#define GERBIL_TUNE_CLASSES 4
typedef struct gerbil_tuning {
  float load_factor[GERBIL_TUNE_CLASSES];
  uint64_t class_bytes[GERBIL_TUNE_CLASSES - 1];
  int32_t fused;       /* phase-two form (gerbil_opts.fused) */
  int32_t schedule;    /* insert schedule (gerbil_opts.schedule) */
  int32_t k_words;     /* W = ceil(2k/64) the settings are for */
  uint32_t samples;    /* configurations timed */
  double ns_per_kmer;  /* phase-two device time per k-mer of the sample with the chosen form */
  int32_t probe_scheme; /* gerbil_opts.probe_scheme for every table of this key width */
  uint32_t item_kmers;  /* gerbil_opts.item_kmers (64, 128 or 256) */
} gerbil_tuning;

/* Fills *opts (not NULL) with the defaults listed above: canonical counting and minimizers,
 * KMC2 ordering, L_max 256, theta 1024, load factor 0.5 (Sec. 3.1, Alg. 1, Sec. 3.4). */
void gerbil_opts_default(gerbil_opts* opts);

/* Human-readable name of a status code; never NULL ("unknown status" for other values).
 * The paper has no counterpart (library plumbing, as are the context and accessor calls
 * below). */
const char* gerbil_strerror(int status);

/* Text of the last CUDA or argument error seen on this context ("" if none or ctx is NULL).
 * The string is owned by the context and valid until its next call. */
const char* gerbil_last_error(const gerbil_ctx* ctx);

/* Creates a context on CUDA device `device`.  hbm_budget_bytes bounds the device memory the
 * context may hold at once (0 = no bound).  cuda_stream is a cudaStream_t on that device that
 * every call is ordered on: cudaStreamLegacy ((void*)1) for the legacy default stream,
 * cudaStreamPerThread ((void*)2) for the per-thread one; NULL makes the context create a
 * non-blocking stream of its own, which does not wait for work on any other stream.  The
 * paper has no counterpart: its runs own the machine, while a context holds one device's
 * stream, budget, reusable scratch and the distinct ratio learned so far (Sec. 3.4).
 * Errors: E_INVAL (bad device or NULL out), E_CUDA. */
int gerbil_create(gerbil_ctx** out, int device, uint64_t hbm_budget_bytes, void* cuda_stream);

/* Forgets the distinct/occurrence ratio the context learned from earlier counts (Sec. 3.4
 * adjusts it at run time within one input).  Call it before counting an unrelated input on the
 * same context: a ratio learned on a highly repetitive input sizes the next input's first
 * batch far too small (still exact, through the overflow path, but slow; that batch's ratio then
 * sizes the following ones).  The next batch of more than 32 bins then samples every 16th bin
 * first.  Errors: E_INVAL. */
int gerbil_forget_ratio(gerbil_ctx* ctx);

/* Probe statistics (Sec. 3.3 reports, for one-by-one and for 128-byte-window probing, the share
 * of k-mers placed at the first probe and the largest number of probes any k-mer needed).
 * enable != 0 clears and starts the histograms: every later insert of this context's counts
 * (two-grid and waves forms; fused 1 does not record) records, once placed, the number of
 * slots it read and the number of distinct 128-byte lines those slots lie in under linear
 * probing (one slot per read, so consecutive probes share lines), or of windows under the
 * windowed double hashing of probe_scheme 1.  While on, counts run a separate instantiation
 * of the insert kernel that adds two global atomics per k-mer; the normal one carries no
 * recording code.  enable == 0 stops and frees.  Errors: E_INVAL, E_CUDA. */
#define GERBIL_PROBE_BUCKETS 34
int gerbil_probe_stats(gerbil_ctx* ctx, int enable);

/* Reads the probe histograms of Sec. 3.3's comparison (GERBIL_PROBE_BUCKETS entries each):
 * entry i < 32 counts k-mers placed after reading i+1 slots (slots[]) or touching i+1 lines
 * (lines[]), entry 32 more than 32, entry 33 k-mers sent to the overflow area (theta probes
 * without room).  Synchronizes the context's stream.  Errors: E_INVAL, E_STATE (statistics
 * off), E_CUDA. */
int gerbil_get_probe_stats(const gerbil_ctx* ctx, uint64_t* slots, uint64_t* lines);

/* Destroys the context and releases its scratch memory (not the caller's stream).  Bins and
 * results it made must be freed first.  NULL is ignored. */
void gerbil_destroy(gerbil_ctx* ctx);

/* Releases the context's cached scratch (table arena, overflow area, work lists) back to the
 * device pool; the next count allocates it again.  Results and bins are not affected.
 * Errors: E_INVAL (NULL), E_CUDA. */
int gerbil_trim(gerbil_ctx* ctx);

/* Device bytes the context currently holds (scratch, bins, results); 0 for NULL. */
uint64_t gerbil_device_bytes(const gerbil_ctx* ctx);

/* Enables (1) or disables (0) per-step event timing and resets the accumulated times and
 * launch counters.  Timing adds two event records per step; results are unchanged.
 * Synchronizes the context's stream.  Errors: E_INVAL (NULL), E_CUDA. */
int gerbil_profile(gerbil_ctx* ctx, int enable);

/* Copies the accumulated step times and launch counters (see gerbil_phase_times) into *out.
 * Errors: E_INVAL (NULL ctx or out). */
int gerbil_get_phase_times(const gerbil_ctx* ctx, gerbil_phase_times* out);

/* Phase one (Sec. 2.1, Fig. 1; Sec. 2.3 Phase One steps 2-4): encodes the reads to 2 bits
 * per base, computes for every window of k determined bases its minimizer (the m-mer of
 * smallest rank under opts->ordering), cuts the windows of each read into super-mers --
 * maximal runs of consecutive windows with one minimizer value, also cut at multiples of
 * L_max -- and distributes them to nbins bins.  The bins keep the 2-bit bases and one
 * descriptor per super-mer on the device, together with per-bin statistics (the paper's
 * binStatFile, App. A flag -x).  Requires GERBIL_MIN_K <= k <= GERBIL_MAX_K,
 * 1 <= m <= min(k-1, 15), 1 <= nbins <= 65536; a bin may hold fewer than 2^32 k-mers.
 * Errors: E_INVAL, E_UNSUPPORTED (k > GERBIL_MAX_K), E_NOMEM, E_CUDA. */
int gerbil_partition(gerbil_ctx* ctx, const gerbil_reads* reads, int k, int m, int nbins,
                     const gerbil_opts* opts, gerbil_bins** out);

/* Totals of a bins object (any out pointer may be NULL).  Errors: E_INVAL (NULL bins). */
int gerbil_bins_info(const gerbil_bins* bins, int* k, int* m, int* nbins, uint64_t* n_supermers,
                     uint64_t* n_kmers);

/* binStatFile row of one bin (App. A flag -x; Sec. 3.4 sizes tables from it): super-mers,
 * bases (sum of super-mer lengths), k-mers.  Any out pointer may be NULL.
 * Errors: E_INVAL (NULL bins, bin outside [0, nbins)). */
int gerbil_bin_stats(const gerbil_bins* bins, int bin, uint64_t* n_super, uint64_t* n_bases,
                     uint64_t* n_kmers);

/* Copies the super-mer descriptors -- what the paper's temporary files hold (Sec. 2.3 Phase One
 * step 4) -- to host arrays of capacity cap (>= n_supermers):
 * global start position of the super-mer's first base in the input, its number of
 * k-mers, and its bin.  Order within a bin is unspecified.  Errors: E_INVAL (cap). */
int gerbil_bins_export(const gerbil_bins* bins, uint64_t* pos, uint32_t* nkmers, uint32_t* bin,
                       uint64_t cap);

/* Releases a bins object and its device memory (the reads it was made from are the caller's).
 * NULL is ignored. */
void gerbil_bins_free(gerbil_bins* bins);

/* Phase two for one bin (Sec. 2.3 Phase Two; Alg. 1; Sec. 3.4): splits the bin's super-mers
 * into k-mers, canonicalises each (unless opts->canonical == 0), inserts it into an
 * open-addressing table sized from the bin statistics (Sec. 3.4 "Estimating table sizes"),
 * sends a k-mer that exhausts max_probes probes to the overflow area, recounts the overflow
 * and merges it, and keeps every key with count >= min_count.  k must equal the k given to
 * gerbil_partition.  Errors: E_INVAL, E_NOMEM, E_OVERFLOW, E_TIMEOUT, E_STATE, E_CUDA. */
int gerbil_count(gerbil_ctx* ctx, const gerbil_bins* bins, int bin, int k, uint32_t min_count,
                 const gerbil_opts* opts, gerbil_counts** out);

/* Phase two for many bins at once (Sec. 2.3 Phase Two over several temporary files; bins are
 * independent, Sec. 2.1): the bins listed in bin_list (host array of nb distinct bin indices;
 * NULL = all bins, nb ignored) are counted together and their rows returned in one result.
 * Because bins partition the k-mers, the rows are the union of the per-bin results.  With
 * opts->persistent (default) one persistent kernel pops tiles of all bins from a device work
 * queue.  Errors: as gerbil_count. */
int gerbil_count_batch(gerbil_ctx* ctx, const gerbil_bins* bins, const int32_t* bin_list,
                       int nb, int k, uint32_t min_count, const gerbil_opts* opts,
                       gerbil_counts** out);

/* Size and statistics of a result (any out pointer may be NULL).  Errors: E_INVAL (NULL). */
int gerbil_counts_info(const gerbil_counts* counts, uint64_t* n, int* words,
                       gerbil_count_stats* stats);

/* Device view of a result: *n rows (may be NULL), *words = W key words per row (may be NULL),
 * and the device pointers keys[n][W] (row-major, layout above) and counts[n] (u32), the rows
 * App. C writes out (either pointer may be NULL).  Owned by the result and valid until
 * gerbil_counts_free; a result counted in bin groups is joined into one buffer on the first
 * view.  Errors: E_INVAL (NULL result), E_NOMEM, E_CUDA. */
int gerbil_counts_view(const gerbil_counts* counts, uint64_t* n, int* words,
                       const uint64_t** keys_dev, const uint32_t** counts_dev);

/* Copies a result to host arrays owned by the caller: keys (cap*W words, layout above) and
 * counts (cap entries); plain or pinned host memory.  Synchronizes the context's stream.
 * Errors: E_INVAL (NULL result, cap < n, NULL arrays for a non-empty result), E_CUDA. */
int gerbil_counts_to_host(const gerbil_counts* counts, uint64_t* keys, uint32_t* counts_out,
                          uint64_t cap);

/* Releases a result and its device memory.  NULL is ignored. */
void gerbil_counts_free(gerbil_counts* counts);

/* Output records of App. C ("Output Format") for every row of a result, in the result's row
 * order: the count -- one byte when below 255, else the byte 0xFF followed by the count as a
 * big-endian 32-bit integer -- then the k-mer with four bases per byte (A=00 C=01 G=10 T=11,
 * first base in the two high bits of the first byte; the unused low bits of the last byte, which
 * App. C leaves undefined, are written as 0).  k must be the k the result was counted with.
 * *nbytes receives the size of all records.  out == NULL only computes the size; otherwise out
 * (cap bytes, device memory when out_on_device != 0, else host memory; any byte alignment)
 * receives the records.  The work runs on the stream of the context that owns the result and
 * synchronizes it; scratch comes from that context.  A host buffer with room for
 * rows * (ceil(k/4) + 5) bytes (every count in its 5-byte form) lets a one-part result skip
 * the size pass before the records are written: one stream synchronisation instead of two.
 * Errors: E_INVAL (k of another key width, cap too small -- *nbytes is still set), E_NOMEM,
 * E_CUDA. */
int gerbil_encode_records(const gerbil_counts* counts, int k, void* out, uint64_t cap,
                          int out_on_device, uint64_t* nbytes);

/* ---- serving: counting jobs admitted continuously under an HBM budget ----------------------
 * The paper has no counterpart (it counts one input at a time).  A server keeps `slots` worker
 * contexts, each with its own CUDA stream and host thread.  A submitted job waits, in arrival
 * order, until a worker is free and its estimated peak device memory fits under
 * hbm_budget_bytes (0: no limit) next to the running jobs and the finished results not yet
 * handed over.  The estimate covers reads copied from the host, the phase-one buffers, hash
 * tables at the largest distinct ratio seen so far for the job's k (every k-mer distinct
 * before the first such job, unless opts->distinct_ratio is given), the overflow area and
 * the result rows.  The first waiting job that fits is admitted, so a large job does not hold
 * up smaller ones; a job passed over 4 x slots times stops later jobs from starting until it
 * fits; a job larger than the whole budget runs when nothing else does.  One job's tables
 * take at most hbm_budget_bytes / (2 x slots) (its opts->max_table_mib, when 0): larger
 * batches are counted in groups of bins.  Each job learns its own distinct ratio (Sec. 3.4)
 * on a sample of its bins.  Admitted jobs run phase one and phase two (gerbil_partition +
 * gerbil_count_batch over all bins) concurrently on their streams, so their kernels overlap on
 * the GPU.  Each job's result stays on the device (a gerbil_counts of the worker's context)
 * and counts against the budget until gerbil_server_wait hands it over; free every result
 * before destroying the server. */
typedef struct gerbil_server gerbil_server;

typedef struct gerbil_server_stats {
  uint64_t submitted, completed, failed;
  uint64_t kmers;          /* k-mer occurrences counted by completed jobs */
  uint32_t max_concurrent; /* most jobs running at once */
  uint32_t reserved;
  uint64_t kernel_launches; /* kernels of this library launched by the workers */
} gerbil_server_stats;

typedef struct gerbil_job_times {
  double queue_ms;   /* arrival (submit) -> admission */
  double run_ms;     /* admission -> result on the device */
  double latency_ms; /* arrival -> result on the device */
  int32_t worker;
  int32_t reserved;
} gerbil_job_times;

/* Errors: E_INVAL (slots outside 1..64), E_CUDA, E_NOMEM. */
int gerbil_server_create(gerbil_server** out, int device, uint64_t hbm_budget_bytes, int slots);

/* Queues one job: gerbil_partition and gerbil_count_batch over all bins of its reads (Sec. 2.3
 * Phase One and Phase Two), with the arguments of those calls.  Host reads are copied at
 * submit; device reads must be complete when this is called (the workers' streams wait for no
 * other stream) and stay valid until the job's result has been waited for.  opts->bin_bounds
 * is copied.  *job_id receives the id.  Errors: E_INVAL (NULL arguments, k, m, nbins or
 * min_count out of range), E_NOMEM (host), E_CUDA (copying host reads).  A job's own failure is
 * reported by gerbil_server_wait. */
int gerbil_server_submit(gerbil_server* s, const gerbil_reads* reads, int k, int m, int nbins,
                         uint32_t min_count, const gerbil_opts* opts, uint64_t* job_id);

/* Waits for a job (timeout_ms < 0: no limit) and hands over its result (*out, NULL if the job
 * failed; the caller frees it with gerbil_counts_free) and times (times may be NULL); returns
 * the job's status, or E_TIMEOUT (the job stays queued/running), or E_INVAL (NULL s or out, an
 * unknown or already handed-over job id). */
int gerbil_server_wait(gerbil_server* s, uint64_t job_id, int64_t timeout_ms, gerbil_counts** out,
                       gerbil_job_times* times);

/* Totals since the server was created.  Errors: E_INVAL (NULL). */
int gerbil_server_get_stats(gerbil_server* s, gerbil_server_stats* out);

/* Message of the last failed job that gerbil_server_wait handed over (the worker context's
 * gerbil_last_error, prefixed by the status name); "" if none.  Valid until the next wait. */
const char* gerbil_server_last_error(const gerbil_server* s);

/* Stops the workers after their current jobs and frees every result not yet handed over.
 * NULL is ignored. */
void gerbil_server_destroy(gerbil_server* s);

/* Autotuner.  The paper sizes every table with one load factor (Sec. 3.4) and has no tuner;
 * here the phase-two form, the probe scheme, the work-item size (threads per k-mer) and the
 * load factor of each table-size class are chosen by measurement.  Times phase two on every
 * 16th bin of `bins` -- or every 8th, 4th, 2nd or every bin, until the sample's tables take
 * four times the L2 cache, so that they do not all stay in L2 as no large batch's would --
 * with device events around the clears, inserts, compaction and overflow work (best of two
 * runs per candidate): first the form and schedule (fused 0 with schedule 1 or 0, fused 1,
 * fused 2) with the defaults; then probe scheme 0 / 1; then work items of 256 / 128 / 64
 * k-mers (keys of up to four words); then, for each table-size class that holds at least
 * 100,000 k-mers of the sample (other classes keep 0.5), load factors 0.35 / 0.5 / 0.65 /
 * 0.8; each step keeps the best of the previous ones.  A candidate
 * whose time is not below the defaults' by 2% or more is not taken.  Finally the tuned
 * settings and the defaults are timed on the whole batch, and the defaults are kept unless the
 * tuned settings are faster there.  The choice is kept in the context for the key width of k
 * and returned in *out (may be NULL).  Counts do not depend on any of these settings.  Costs
 * about 20 sample counts and 4 counts of the batch.
 * Errors: as gerbil_count_batch. */
int gerbil_autotune(gerbil_ctx* ctx, const gerbil_bins* bins, int k, uint32_t min_count,
                    const gerbil_opts* opts, gerbil_tuning* out);

/* Sets (t != NULL, e.g. from a cache of earlier runs) or clears (t == NULL) the tuned settings
 * the context uses for the key width of k.  Errors: E_INVAL (a value out of range). */
int gerbil_set_tuning(gerbil_ctx* ctx, int k, const gerbil_tuning* t);

/* Reads the settings held for the key width of k.  Errors: E_INVAL, E_STATE (none held). */
int gerbil_get_tuning(const gerbil_ctx* ctx, int k, gerbil_tuning* out);

/* Self-test of the bounded device waits (the paper has no counterpart).  Every wait in the
 * kernels is bounded, so that a dependency that never arrives ends in an error status rather
 * than a hung GPU.  This call launches one warp that waits, through the same helper as the fused
 * phase-two kernel's work-queue waits, for a device flag that nothing sets.  After wait_ns
 * nanoseconds (0 < wait_ns <= 1e10) the wait runs out and the kernel records it and returns.
 * The expected result is GERBIL_E_TIMEOUT; the context stays usable.
 * Errors: E_INVAL, E_NOMEM, E_CUDA, E_STATE (the wait ended without running out). */
int gerbil_wait_selftest(gerbil_ctx* ctx, uint64_t wait_ns);

/* Memory-throughput probe (the paper has no counterpart; a measurement helper for the
 * roofline of the insert kernel).  Runs one kernel in which every thread performs per_thread
 * operations at pseudo-random 32-byte slots of a device array of `bytes` bytes, allocated from
 * the context: op 0 = 8-byte atomic add, 1 = 32-byte relaxed load, 2 = 32-byte load then atomic
 * add on the same slot (the shape of a found-key insert), 3 = 8-byte compare-and-swap.  A
 * footprint below the L2 size measures L2; a larger one measures HBM.  *gops receives
 * operations per second / 1e9, timed with CUDA events on the context's stream.
 * Errors: E_INVAL, E_NOMEM, E_CUDA. */
int gerbil_membench(gerbil_ctx* ctx, uint64_t bytes, int op, uint64_t per_thread, double* gops);

/* Counting without any device allocation.  The paper has no counterpart: this entry point is
 * for callers that cannot call cudaMalloc -- for example code whose device memory is owned by
 * another component (a framework's caching allocator or a fixed memory budget that forbids
 * extra allocations), or latency-sensitive paths that cannot afford the implicit device
 * synchronisation of cudaMalloc and cudaFree.  It counts the k-mers of a small read set (same
 * read and key conventions as above; canonical != 0 counts min(x, revcomp(x))) and writes the
 * rows with count >= min_count to caller-provided device buffers keys_out (out_cap * W words)
 * and counts_out (out_cap entries).  seq and offsets are device pointers; nbases is
 * offsets[nreads] (host value); *n_out (host) receives the number of rows.
 * Scratch: a fixed 32 MiB table in a file-scope device array, held by every GPU that loads
 * the library until the process exits.  Inputs with more than
 * floor((4194304 - 16) / S / 2) k-mer windows, where S = 2 * ceil((C + 1) / 2) words per slot
 * and C = max(1, ceil((2k - 30) / 63)) (about 1.05 million windows for k <= 46, 524 thousand
 * for k = 65), are
 * rejected with GERBIL_E_INVAL before any GPU work.  The first call on a device resolves the
 * array's address (cudaGetSymbolAddress) for that device; make that first call before any
 * stream capture.  The address is kept for the life of the process: after a cudaDeviceReset
 * of that device it is stale, so do not call this entry point again in that process.  Every
 * call clears the part of the array it uses, runs on cuda_stream (NULL: the default stream)
 * and synchronises it; calls whose GPU work overlaps (other streams or other host threads on
 * the same device) race on the shared array and must be serialised by the caller.  No
 * cudaMalloc, cudaFree or allocating library routine is called.
 * Errors: E_INVAL (arguments, input too large, or *n_out > out_cap: *n_out then holds the
 * number of rows needed), E_UNSUPPORTED (k > GERBIL_MAX_K), E_NOMEM (the table ran full),
 * E_TIMEOUT (a bounded device wait for another thread's key words gave up), E_CUDA. */
int gerbil_count_small_noalloc(const uint8_t* seq, const uint64_t* offsets, uint64_t nreads,
                               uint64_t nbases, int k, uint32_t min_count, int canonical,
                               uint64_t* keys_out, uint32_t* counts_out, uint64_t out_cap,
                               uint64_t* n_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* GERBIL_H */
