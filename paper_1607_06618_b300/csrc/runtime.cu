// runtime.cu -- host side of the C ABI (include/gerbil.h): contexts, device memory under an
// HBM budget, phase-one orchestration, table sizing (Sec. 3.4 "Estimating table sizes"),
// phase-two launches and the overflow recount (Sec. 3.4 "Probing Strategy").
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/gerbil.h"
#include "common.cuh"
#include "kernels.h"

using gerbil::BinWork;
using gerbil::Counters;

struct gerbil_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  uint64_t budget = 0;  // 0 = unbounded
  std::atomic<uint64_t> used{0};  // results may be freed from another thread
  int nsm = 148;
  int insert_ctas_per_sm = 8;
  int l2_bytes = 126 << 20;
  size_t arena_dirty = 0;  // bytes at the start of the table arena that may be non-zero
  double ratio = 1.0;  // distinct / occurrences measured on earlier calls
  bool ratio_known = false;
  // rows / occurrences of the last batch counted at emit_min_count (sizes the result buffer)
  double emit_ratio = 1.0;
  uint32_t emit_min_count = 0;
  bool emit_known = false;
  Counters* ctr = nullptr;   // device
  Counters* hctr = nullptr;  // pinned host mirror
  std::string last_error;
  // cached scratch (grow-only)
  void* arena = nullptr;
  size_t arena_bytes = 0;
  void* ovf = nullptr;
  size_t ovf_bytes = 0;
  void* small = nullptr;  // work list + bin_ovf
  size_t small_bytes = 0;
  // step timing (gerbil_profile): an event pair per phase, collected after a stream sync
  bool profiling = false;
  cudaEvent_t ev[2 * 8] = {};
  bool pending[8] = {};
  gerbil_phase_times times{};
  // settings chosen by gerbil_autotune, per key width W
  std::map<int, gerbil_tuning> tuning;
  // probe statistics (gerbil_probe_stats): device histograms, NULL while off
  unsigned long long* probe_hist = nullptr;
  // graph form (gerbil_opts.graph): capture stream, the instantiated graph of the last batch
  // (updated in place when the next batch's graph has the same shape), pinned work-list copy
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  void* hwork = nullptr;
  size_t hwork_bytes = 0;
};

struct gerbil_bins {
  gerbil_ctx* ctx = nullptr;
  int k = 0, m = 0, nbins = 0;
  int canon_min = 1;
  uint64_t n = 0, nwords = 0;
  unsigned long long* packed = nullptr;
  size_t packed_bytes = 0;
  unsigned long long* sm_pos = nullptr;
  uint32_t* sm_koff = nullptr;
  size_t sm_bytes = 0;
  uint64_t n_super_total = 0, n_kmers_total = 0;
  std::vector<uint64_t> nsuper, nkmers, sm_begin;
};

struct gerbil_counts {
  gerbil_ctx* ctx = nullptr;
  int W = 1;
  uint64_t n = 0;
  unsigned long long* keys = nullptr;
  uint32_t* counts = nullptr;
  size_t bytes = 0;
  gerbil_count_stats stats{};
  // a batch counted in groups of bins: the groups' results in bin order (keys/counts above
  // stay empty until a device view joins them into one buffer)
  std::vector<gerbil_counts*> parts;
};

namespace {

int fail(gerbil_ctx* ctx, int status, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return status;
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(ctx, GERBIL_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

int dev_alloc(gerbil_ctx* ctx, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return GERBIL_OK;
  bytes = (bytes + 255) & ~size_t(255);
  if (ctx->budget && ctx->used + bytes > ctx->budget)
    return fail(ctx, GERBIL_E_NOMEM, "HBM budget exceeded");
  cudaError_t e = cudaMallocAsync(p, bytes, ctx->stream);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(ctx, GERBIL_E_NOMEM, "device out of memory");
  }
  if (e != cudaSuccess) return fail(ctx, GERBIL_E_CUDA, cudaGetErrorString(e));
  ctx->used += bytes;
  return GERBIL_OK;
}

void dev_free(gerbil_ctx* ctx, void* p, size_t bytes) {
  if (!p) return;
  bytes = (bytes + 255) & ~size_t(255);
  cudaFreeAsync(p, ctx->stream);
  ctx->used.fetch_sub(std::min(ctx->used.load(), (uint64_t)bytes));
}

// Grow-only scratch buffer cached in the context (*grown set when it was reallocated).
int scratch(gerbil_ctx* ctx, void** buf, size_t* have, size_t need, bool* grown = nullptr) {
  if (*have >= need && *buf) return GERBIL_OK;
  if (grown) *grown = true;
  dev_free(ctx, *buf, *have);
  *buf = nullptr;
  *have = 0;
  size_t want = std::max(need, *have + *have / 4);
  int rc = dev_alloc(ctx, buf, want);
  if (rc == GERBIL_E_NOMEM && want > need) rc = dev_alloc(ctx, buf, want = need);
  if (rc) return rc;
  *have = want;
  return GERBIL_OK;
}

void ph_collect(gerbil_ctx* ctx, bool wait);
int read_counters(gerbil_ctx* ctx) {
  CK(cudaMemcpyAsync(ctx->hctr, ctx->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ph_collect(ctx, false);
  return GERBIL_OK;
}

int words_for(int k) { return (2 * k + 63) / 64; }

enum Phase { PH_ENCODE = 0, PH_SUPER0, PH_SUPER1, PH_CLEAR, PH_INSERT, PH_COMPACT, PH_OVERFLOW, PH_N };

// Phase events go on the context's stream, or on `s` while it is being captured into a graph
// (recorded as event nodes that fire when the graph runs).
void ph_record(gerbil_ctx* ctx, cudaEvent_t e, cudaStream_t s, bool captured) {
  if (captured) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else cudaEventRecord(e, ctx->stream);
}
void ph_begin(gerbil_ctx* ctx, int ph, cudaStream_t s = nullptr, bool captured = false) {
  if (ctx->profiling) ph_record(ctx, ctx->ev[2 * ph], s, captured);
}
void ph_end(gerbil_ctx* ctx, int ph, cudaStream_t s = nullptr, bool captured = false) {
  if (!ctx->profiling) return;
  ph_record(ctx, ctx->ev[2 * ph + 1], s, captured);
  ctx->pending[ph] = true;
}
// Adds the elapsed time of every finished phase; call only after the stream has synchronized
// past the phase's end event (or pass wait = true).
void ph_collect(gerbil_ctx* ctx, bool wait) {
  for (int ph = 0; ph < PH_N; ++ph) {
    if (!ctx->pending[ph]) continue;
    if (wait) cudaEventSynchronize(ctx->ev[2 * ph + 1]);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->ev[2 * ph], ctx->ev[2 * ph + 1]) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    ctx->pending[ph] = false;
    gerbil_phase_times& t = ctx->times;
    switch (ph) {
      case PH_ENCODE: t.encode_ms += ms; break;
      case PH_SUPER0:
      case PH_SUPER1: t.supermer_ms += ms; break;
      case PH_CLEAR: t.clear_ms += ms; break;
      case PH_INSERT: t.insert_ms += ms; break;
      case PH_COMPACT: t.compact_ms += ms; break;
      case PH_OVERFLOW: t.overflow_ms += ms; break;
      default: break;
    }
  }
}

}  // namespace

extern "C" {

void gerbil_opts_default(gerbil_opts* o) {
  std::memset(o, 0, sizeof(*o));
  o->canonical = 1;
  o->ordering = GERBIL_ORDER_KMC2;
  o->canonical_minimizer = 1;
  o->supermer_cap = 256;
  o->bin_bounds = nullptr;
  o->max_probes = 1024;
  o->load_factor = 0.5f;
  o->distinct_ratio = 0.0f;
  o->overflow_slots = 0;
  o->persistent = 1;
  o->ring_slots = 0;
  o->dfp_pivot = 0.5f;
  o->dfp_sample = 16;
  o->fused = 0;
  o->schedule = 1;
  o->probe_scheme = 0;
  o->item_kmers = 0;
}

const char* gerbil_strerror(int s) {
  switch (s) {
    case GERBIL_OK: return "ok";
    case GERBIL_E_INVAL: return "invalid argument";
    case GERBIL_E_UNSUPPORTED: return "unsupported (k above the compiled maximum)";
    case GERBIL_E_NOMEM: return "out of device memory or HBM budget";
    case GERBIL_E_OVERFLOW: return "overflow area exhausted after all retries";
    case GERBIL_E_TIMEOUT: return "bounded device wait gave up";
    case GERBIL_E_CUDA: return "CUDA error";
    case GERBIL_E_STATE: return "device consistency check failed";
    default: return "unknown status";
  }
}

const char* gerbil_last_error(const gerbil_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

int gerbil_create(gerbil_ctx** out, int device, uint64_t budget, void* stream) {
  if (!out) return GERBIL_E_INVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return GERBIL_E_CUDA;
  }
  if (device < 0 || device >= ndev) return GERBIL_E_INVAL;
  gerbil_ctx* ctx = new (std::nothrow) gerbil_ctx;
  if (!ctx) return GERBIL_E_NOMEM;
  ctx->device = device;
  ctx->budget = budget;
  int rc = GERBIL_OK;
  do {
    if (cudaSetDevice(device) != cudaSuccess) { rc = GERBIL_E_CUDA; break; }
    cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&ctx->l2_bytes, cudaDevAttrL2CacheSize, device);
    if (stream) {
      ctx->stream = (cudaStream_t)stream;
    } else {
      if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
        rc = GERBIL_E_CUDA;
        break;
      }
      ctx->own_stream = true;
    }
    // keep freed blocks in the device's default pool: repeated calls reuse them
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    if (cudaMalloc(&ctx->ctr, sizeof(Counters)) != cudaSuccess) { rc = GERBIL_E_CUDA; break; }
    if (cudaMallocHost(&ctx->hctr, sizeof(Counters)) != cudaSuccess) { rc = GERBIL_E_CUDA; break; }
    for (cudaEvent_t& e : ctx->ev)
      if (cudaEventCreate(&e) != cudaSuccess) { rc = GERBIL_E_CUDA; break; }
    if (rc) break;
    ctx->insert_ctas_per_sm = 8;  // refined by an occupancy query of the kernel at launch
  } while (0);
  if (rc) {
    cudaGetLastError();
    gerbil_destroy(ctx);
    return rc;
  }
  *out = ctx;
  return GERBIL_OK;
}

void gerbil_destroy(gerbil_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) {
    dev_free(ctx, ctx->arena, ctx->arena_bytes);
    dev_free(ctx, ctx->ovf, ctx->ovf_bytes);
    dev_free(ctx, ctx->small, ctx->small_bytes);
    cudaStreamSynchronize(ctx->stream);
  }
  for (cudaEvent_t e : ctx->ev)
    if (e) cudaEventDestroy(e);
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->hwork) cudaFreeHost(ctx->hwork);
  if (ctx->probe_hist) cudaFree(ctx->probe_hist);
  if (ctx->ctr) cudaFree(ctx->ctr);
  if (ctx->hctr) cudaFreeHost(ctx->hctr);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

// Device memory from the context's pool and budget, for helpers outside this file.
int gerbil_internal_alloc(gerbil_ctx* ctx, void** p, size_t bytes, void** stream, int* nsm) {
  if (!ctx) return GERBIL_E_INVAL;
  CK(cudaSetDevice(ctx->device));
  *stream = ctx->stream;
  *nsm = ctx->nsm;
  return dev_alloc(ctx, p, bytes);
}

void gerbil_internal_free(gerbil_ctx* ctx, void* p, size_t bytes) { dev_free(ctx, p, bytes); }

int gerbil_probe_stats(gerbil_ctx* ctx, int enable) {
  if (!ctx) return GERBIL_E_INVAL;
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  if (!enable) {
    if (ctx->probe_hist) cudaFree(ctx->probe_hist);
    ctx->probe_hist = nullptr;
    return GERBIL_OK;
  }
  const size_t bytes = 2 * gerbil::PROBE_BUCKETS * sizeof(unsigned long long);
  if (!ctx->probe_hist) CK(cudaMalloc(&ctx->probe_hist, bytes));
  CK(cudaMemset(ctx->probe_hist, 0, bytes));
  return GERBIL_OK;
}

int gerbil_get_probe_stats(const gerbil_ctx* cctx, uint64_t* slots, uint64_t* lines) {
  if (!cctx || !slots || !lines) return GERBIL_E_INVAL;
  gerbil_ctx* ctx = const_cast<gerbil_ctx*>(cctx);
  if (!ctx->probe_hist) return fail(ctx, GERBIL_E_STATE, "probe statistics are off");
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemcpy(slots, ctx->probe_hist, gerbil::PROBE_BUCKETS * 8, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(lines, ctx->probe_hist + gerbil::PROBE_BUCKETS, gerbil::PROBE_BUCKETS * 8,
                cudaMemcpyDeviceToHost));
  return GERBIL_OK;
}

int gerbil_forget_ratio(gerbil_ctx* ctx) {
  if (!ctx) return GERBIL_E_INVAL;
  ctx->ratio_known = false;
  ctx->emit_known = false;
  return GERBIL_OK;
}

int gerbil_wait_selftest(gerbil_ctx* ctx, uint64_t wait_ns) {
  if (!ctx || wait_ns == 0 || wait_ns > 10000000000ull) return GERBIL_E_INVAL;
  CK(cudaSetDevice(ctx->device));
  void* flag = nullptr;
  int rc = dev_alloc(ctx, &flag, 256);
  if (rc) return rc;
  cudaError_t e = cudaMemsetAsync(flag, 0, 256, ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->ctr, 0, sizeof(Counters), ctx->stream);
  if (e == cudaSuccess) e = gerbil::launch_wait_selftest((const uint32_t*)flag, wait_ns, ctx->ctr, ctx->stream);
  if (e == cudaSuccess) ctx->times.kernel_launches++;
  rc = (e == cudaSuccess) ? read_counters(ctx) : fail(ctx, GERBIL_E_CUDA, cudaGetErrorString(e));
  dev_free(ctx, flag, 256);
  if (rc) return rc;
  if (ctx->hctr->err & gerbil::ERR_QUEUE) return fail(ctx, GERBIL_E_TIMEOUT, "self-test wait ran out");
  return fail(ctx, GERBIL_E_STATE, "self-test wait ended without running out");
}

int gerbil_trim(gerbil_ctx* ctx) {
  if (!ctx) return GERBIL_E_INVAL;
  CK(cudaSetDevice(ctx->device));
  dev_free(ctx, ctx->arena, ctx->arena_bytes);
  dev_free(ctx, ctx->ovf, ctx->ovf_bytes);
  dev_free(ctx, ctx->small, ctx->small_bytes);
  ctx->arena = ctx->ovf = ctx->small = nullptr;
  ctx->arena_bytes = ctx->ovf_bytes = ctx->small_bytes = 0;
  ctx->arena_dirty = 0;
  CK(cudaStreamSynchronize(ctx->stream));
  return GERBIL_OK;
}

uint64_t gerbil_device_bytes(const gerbil_ctx* ctx) { return ctx ? ctx->used.load() : 0; }

int gerbil_profile(gerbil_ctx* ctx, int enable) {
  if (!ctx) return GERBIL_E_INVAL;
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  ph_collect(ctx, true);
  ctx->profiling = enable != 0;
  std::memset(&ctx->times, 0, sizeof(ctx->times));
  for (bool& p : ctx->pending) p = false;
  return GERBIL_OK;
}

int gerbil_get_phase_times(const gerbil_ctx* cctx, gerbil_phase_times* out) {
  if (!cctx || !out) return GERBIL_E_INVAL;
  gerbil_ctx* ctx = const_cast<gerbil_ctx*>(cctx);
  cudaSetDevice(ctx->device);
  ph_collect(ctx, true);
  *out = ctx->times;
  return GERBIL_OK;
}

// ---- phase one ---------------------------------------------------------------------------------
int gerbil_partition(gerbil_ctx* ctx, const gerbil_reads* reads, int k, int m, int nbins,
                     const gerbil_opts* opts_in, gerbil_bins** out) {
  if (!ctx || !reads || !out) return GERBIL_E_INVAL;
  *out = nullptr;
  gerbil_opts opts;
  if (opts_in) opts = *opts_in; else gerbil_opts_default(&opts);
  if (k > GERBIL_MAX_K) return fail(ctx, GERBIL_E_UNSUPPORTED, "k above GERBIL_MAX_K");
  if (k < GERBIL_MIN_K || m < 1 || m >= k || m > 15 || nbins < 1 || nbins > 65536)
    return fail(ctx, GERBIL_E_INVAL, "k, m or nbins out of range");
  if (opts.supermer_cap < 1 || opts.supermer_cap > 1024)
    return fail(ctx, GERBIL_E_INVAL, "supermer_cap out of range");
  if (opts.ordering < GERBIL_ORDER_KMC2 || opts.ordering > GERBIL_ORDER_DFP)
    return fail(ctx, GERBIL_E_INVAL, "unknown ordering");
  if (opts.ordering == GERBIL_ORDER_DFP &&
      (m > 12 || opts.dfp_sample < 1 || !(opts.dfp_pivot >= 0.0f && opts.dfp_pivot <= 1.0f)))
    return fail(ctx, GERBIL_E_INVAL, "dfp ordering: m above 12, sample or pivot out of range");
  if (reads->nreads > 0 && (!reads->seq || !reads->offsets))
    return fail(ctx, GERBIL_E_INVAL, "null reads");
  if (opts.bin_bounds) {
    for (int i = 0; i + 2 < nbins; ++i)
      if (opts.bin_bounds[i] > opts.bin_bounds[i + 1])
        return fail(ctx, GERBIL_E_INVAL, "bin_bounds not ascending");
  }
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;

  // total bases and offsets[0]
  uint64_t first = 0, n = 0;
  const uint64_t nreads = reads->nreads;
  if (nreads > 0) {
    if (reads->on_device) {
      CK(cudaMemcpyAsync(&first, reads->offsets, 8, cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(&n, reads->offsets + nreads, 8, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
    } else {
      first = reads->offsets[0];
      n = reads->offsets[nreads];
    }
  }
  if (first != 0) return fail(ctx, GERBIL_E_INVAL, "offsets[0] must be 0");

  gerbil_bins* b = new (std::nothrow) gerbil_bins;
  if (!b) return GERBIL_E_NOMEM;
  b->ctx = ctx;
  b->k = k;
  b->m = m;
  b->nbins = nbins;
  b->canon_min = opts.canonical_minimizer ? 1 : 0;
  b->n = n;
  b->nwords = (n + 1 + 31) / 32;
  b->nsuper.assign(nbins, 0);
  b->nkmers.assign(nbins, 0);
  b->sm_begin.assign(nbins + 1, 0);

  // temporaries
  uint8_t* dseq = nullptr;
  uint64_t* doff = nullptr;
  uint32_t* nmask = nullptr;
  uint32_t* bmask = nullptr;
  uint32_t* dbounds = nullptr;
  unsigned long long* binbuf = nullptr;  // nsuper, nkmers, cursor, sm_begin
  unsigned long long* rec = nullptr;     // super-mer records
  uint32_t* dtable = nullptr;            // dfp ordering: rank of every m-mer value
  uint64_t rec_cap = 0, nrec = 0;
  size_t seq_bytes = 0, off_bytes = 0, mask_bytes = 0, bounds_bytes = 0, binbuf_bytes = 0;
  size_t table_bytes = 0;
  std::vector<unsigned long long> hbin;
  int rc = GERBIL_OK;
  auto cleanup = [&]() {
    dev_free(ctx, dseq, seq_bytes);
    dev_free(ctx, doff, off_bytes);
    dev_free(ctx, nmask, mask_bytes);
    dev_free(ctx, bmask, mask_bytes);
    dev_free(ctx, dbounds, bounds_bytes);
    dev_free(ctx, binbuf, binbuf_bytes);
    dev_free(ctx, rec, rec_cap * 16);
    dev_free(ctx, dtable, table_bytes);
  };
#define TRY(x)                      \
  do {                              \
    rc = (x);                       \
    if (rc) {                       \
      cleanup();                    \
      gerbil_bins_free(b);          \
      return rc;                    \
    }                               \
  } while (0)
#define TRYCU(call)                                                                       \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) TRY(fail(ctx, GERBIL_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_))); \
  } while (0)

  const uint8_t* seq = reads->seq;
  const uint64_t* offsets = reads->offsets;
  if (!reads->on_device && nreads > 0) {
    seq_bytes = n + 16;
    off_bytes = (nreads + 1) * 8;
    TRY(dev_alloc(ctx, (void**)&dseq, seq_bytes));
    TRY(dev_alloc(ctx, (void**)&doff, off_bytes));
    if (n) TRYCU(cudaMemcpyAsync(dseq, reads->seq, n, cudaMemcpyHostToDevice, st));
    TRYCU(cudaMemcpyAsync(doff, reads->offsets, off_bytes, cudaMemcpyHostToDevice, st));
    seq = dseq;
    offsets = doff;
  }

  b->packed_bytes = (b->nwords + 2) * 8;
  mask_bytes = (b->nwords + 2) * 4;
  TRY(dev_alloc(ctx, (void**)&b->packed, b->packed_bytes));
  TRY(dev_alloc(ctx, (void**)&nmask, mask_bytes));
  TRY(dev_alloc(ctx, (void**)&bmask, mask_bytes));
  binbuf_bytes = (size_t)nbins * 4 * 8 + 16;  // + error word + record count
  TRY(dev_alloc(ctx, (void**)&binbuf, binbuf_bytes));
  TRYCU(cudaMemsetAsync(binbuf, 0, binbuf_bytes, st));
  TRYCU(cudaMemsetAsync(b->packed + b->nwords, 0, 16, st));
  TRYCU(cudaMemsetAsync(nmask + b->nwords, 0xFF, 8, st));
  TRYCU(cudaMemsetAsync(bmask, 0, mask_bytes, st));
  if (opts.bin_bounds && nbins > 1) {
    bounds_bytes = (size_t)(nbins - 1) * 4;
    TRY(dev_alloc(ctx, (void**)&dbounds, bounds_bytes));
    TRYCU(cudaMemcpyAsync(dbounds, opts.bin_bounds, bounds_bytes, cudaMemcpyHostToDevice, st));
  }

  const int vec_ok = ((uintptr_t)seq & 15) == 0;
  ctx->times.calls++;
  ph_begin(ctx, PH_ENCODE);
  TRYCU(gerbil::launch_encode(seq, n, b->packed, nmask, b->nwords, vec_ok, ctx->nsm, st));
  ctx->times.kernel_launches++;
  unsigned int* perr = (unsigned int*)(binbuf + 4 * (size_t)nbins);
  unsigned long long* rec_count = binbuf + 4 * (size_t)nbins + 1;
  if (nreads > 0) {
    TRYCU(gerbil::launch_boundary(offsets, nreads, n, bmask, perr, st));
    ctx->times.kernel_launches++;
  }
  ph_end(ctx, PH_ENCODE);

  // dfp ordering (Sec. 3.1): m-mer frequencies of the sample on the device, rank table on the
  // host (sorted by frequency, then by the distance of each place to the pivot), back to the
  // device for the super-mer kernel
  if (opts.ordering == GERBIL_ORDER_DFP) {
    const uint64_t n4 = 1ull << (2 * m);
    table_bytes = n4 * 4;
    TRY(dev_alloc(ctx, (void**)&dtable, table_bytes));
    TRYCU(cudaMemsetAsync(dtable, 0, table_bytes, st));
    TRYCU(gerbil::launch_mmer_freq(b->packed, nmask, offsets, nreads, opts.dfp_sample, m,
                                   b->canon_min, dtable, ctx->nsm, st));
    ctx->times.kernel_launches++;
    std::vector<uint32_t> freq(n4);
    TRYCU(cudaMemcpyAsync(freq.data(), dtable, table_bytes, cudaMemcpyDeviceToHost, st));
    TRYCU(cudaStreamSynchronize(st));
    // place of every value in ascending (frequency, value) order
    std::vector<uint64_t> key(n4);
    for (uint64_t v = 0; v < n4; ++v) key[v] = ((uint64_t)freq[v] << 32) | v;
    std::sort(key.begin(), key.end());
    const uint64_t pivot = std::min<uint64_t>(n4 - 1, (uint64_t)std::floor((double)n4 * opts.dfp_pivot));
    // places in ascending (distance to the pivot, place) order; rank = index in that order
    std::vector<uint64_t> key2(n4);
    for (uint64_t i = 0; i < n4; ++i) key2[i] = ((i > pivot ? i - pivot : pivot - i) << 32) | i;
    std::sort(key2.begin(), key2.end());
    std::vector<uint32_t> rank(n4);
    for (uint64_t r2 = 0; r2 < n4; ++r2) rank[(uint32_t)key[(uint32_t)key2[r2]]] = (uint32_t)r2;
    TRYCU(cudaMemcpyAsync(dtable, rank.data(), table_bytes, cudaMemcpyHostToDevice, st));
    TRYCU(cudaStreamSynchronize(st));  // rank lives on this stack frame
  }

  gerbil::SupermerParams sp{};
  sp.rank_table = dtable;
  sp.packed = b->packed;
  sp.nmask = nmask;
  sp.bmask = bmask;
  sp.n = n;
  sp.nwords = b->nwords;
  sp.nwin = (n >= (uint64_t)k) ? n - k + 1 : 0;
  sp.k = k;
  sp.m = m;
  sp.ordering = opts.ordering;
  sp.canon_min = b->canon_min;
  sp.lmax = opts.supermer_cap;
  sp.nbins = (uint32_t)nbins;
  sp.bounds = dbounds;
  sp.tile = gerbil::supermer_tile();  // window starts per CTA
  sp.bin_nsuper = binbuf;
  sp.bin_nkmers = binbuf + nbins;
  sp.bin_cursor = binbuf + 2 * nbins;
  sp.bin_sm_begin = binbuf + 3 * nbins;
  sp.err = perr;
  sp.rec_count = rec_count;
  // record area: random minimizers give about 2/(w+1) super-mers per window, plus one per
  // read; four times that, and a rerun with the exact size if it is ever exceeded
  {
    const uint64_t w = (uint64_t)(k - m + 1);
    uint64_t est = sp.nwin * 4 / (w + 1) + 2 * nreads + 65536;
    rec_cap = std::min<uint64_t>(est, sp.nwin + 1);
  }
  TRY(dev_alloc(ctx, (void**)&rec, rec_cap * 16));
  hbin.resize((size_t)nbins * 2 + 2);
  for (int attempt = 0;; ++attempt) {
    sp.rec = (ulonglong2*)rec;
    sp.rec_cap = rec_cap;
    ph_begin(ctx, PH_SUPER0);
    TRYCU(gerbil::launch_supermer(sp, st));
    if (sp.nwin) ctx->times.kernel_launches++;
    ph_end(ctx, PH_SUPER0);
    TRYCU(cudaMemcpyAsync(hbin.data(), binbuf, (size_t)nbins * 16, cudaMemcpyDeviceToHost, st));
    TRYCU(cudaMemcpyAsync(hbin.data() + 2 * (size_t)nbins, binbuf + 4 * (size_t)nbins, 16,
                          cudaMemcpyDeviceToHost, st));
    TRYCU(cudaStreamSynchronize(st));
    ph_collect(ctx, false);
    if ((uint32_t)hbin[2 * (size_t)nbins])
      TRY(fail(ctx, GERBIL_E_INVAL, "offsets out of order or past the input"));
    nrec = hbin[2 * (size_t)nbins + 1];
    if (nrec <= rec_cap) break;
    if (attempt > 0) TRY(fail(ctx, GERBIL_E_STATE, "super-mer record count changed between runs"));
    dev_free(ctx, rec, rec_cap * 16);
    rec = nullptr;
    rec_cap = nrec;
    TRY(dev_alloc(ctx, (void**)&rec, rec_cap * 16));
    TRYCU(cudaMemsetAsync(binbuf, 0, (size_t)nbins * 16, st));
    TRYCU(cudaMemsetAsync(rec_count, 0, 8, st));
  }
  uint64_t acc = 0;
  for (int i = 0; i < nbins; ++i) {
    b->nsuper[i] = hbin[i];
    b->nkmers[i] = hbin[nbins + i];
    if (b->nkmers[i] >= (1ull << 32)) TRY(fail(ctx, GERBIL_E_INVAL, "a bin holds 2^32 or more k-mers"));
    b->sm_begin[i] = acc;
    acc += b->nsuper[i];
    b->n_kmers_total += b->nkmers[i];
  }
  b->sm_begin[nbins] = acc;
  b->n_super_total = acc;
  if (acc != nrec) TRY(fail(ctx, GERBIL_E_STATE, "record and bin counts disagree"));
  TRY(dev_alloc(ctx, (void**)&b->sm_pos, acc * 8 + 8));
  TRY(dev_alloc(ctx, (void**)&b->sm_koff, acc * 4 + 8));
  {
    std::vector<unsigned long long> beg(b->sm_begin.begin(), b->sm_begin.end() - 1);
    TRYCU(cudaMemcpyAsync(binbuf + 3 * nbins, beg.data(), (size_t)nbins * 8, cudaMemcpyHostToDevice, st));
    TRYCU(cudaStreamSynchronize(st));  // beg lives on this stack frame
  }
  sp.sm_pos = b->sm_pos;
  sp.sm_koff = b->sm_koff;
  ph_begin(ctx, PH_SUPER1);
  TRYCU(gerbil::launch_scatter(sp, nrec, ctx->nsm, st));
  if (nrec) ctx->times.kernel_launches++;
  ph_end(ctx, PH_SUPER1);
  TRYCU(cudaMemcpyAsync(ctx->hctr, perr, 4, cudaMemcpyDeviceToHost, st));
  TRYCU(cudaStreamSynchronize(st));
  if (*(unsigned int*)ctx->hctr) TRY(fail(ctx, GERBIL_E_STATE, "scatter overran a bin"));
  cleanup();
  *out = b;
  return GERBIL_OK;
#undef TRY
#undef TRYCU
}

int gerbil_bins_info(const gerbil_bins* b, int* k, int* m, int* nbins, uint64_t* ns, uint64_t* nk) {
  if (!b) return GERBIL_E_INVAL;
  if (k) *k = b->k;
  if (m) *m = b->m;
  if (nbins) *nbins = b->nbins;
  if (ns) *ns = b->n_super_total;
  if (nk) *nk = b->n_kmers_total;
  return GERBIL_OK;
}

int gerbil_bin_stats(const gerbil_bins* b, int bin, uint64_t* ns, uint64_t* nbases, uint64_t* nk) {
  if (!b || bin < 0 || bin >= b->nbins) return GERBIL_E_INVAL;
  if (ns) *ns = b->nsuper[bin];
  if (nk) *nk = b->nkmers[bin];
  if (nbases) *nbases = b->nkmers[bin] + b->nsuper[bin] * (uint64_t)(b->k - 1);
  return GERBIL_OK;
}

int gerbil_bins_export(const gerbil_bins* b, uint64_t* pos, uint32_t* nkmers, uint32_t* bin,
                       uint64_t cap) {
  if (!b || (b->n_super_total && (!pos || !nkmers || !bin))) return GERBIL_E_INVAL;
  if (cap < b->n_super_total) return GERBIL_E_INVAL;
  gerbil_ctx* ctx = b->ctx;
  CK(cudaSetDevice(ctx->device));
  const uint64_t S = b->n_super_total;
  if (S == 0) return GERBIL_OK;
  std::vector<uint32_t> koff(S);
  CK(cudaMemcpyAsync(pos, b->sm_pos, S * 8, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(koff.data(), b->sm_koff, S * 4, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < b->nbins; ++i) {
    const uint64_t lo = b->sm_begin[i], hi = b->sm_begin[i + 1];
    for (uint64_t s = lo; s < hi; ++s) {
      const uint64_t next = (s + 1 < hi) ? koff[s + 1] : b->nkmers[i];
      nkmers[s] = (uint32_t)(next - koff[s]);
      bin[s] = (uint32_t)i;
    }
  }
  return GERBIL_OK;
}

void gerbil_bins_free(gerbil_bins* b) {
  if (!b) return;
  gerbil_ctx* ctx = b->ctx;
  cudaSetDevice(ctx->device);
  dev_free(ctx, b->packed, b->packed_bytes);
  dev_free(ctx, b->sm_pos, b->n_super_total * 8 + 8);
  dev_free(ctx, b->sm_koff, b->n_super_total * 4 + 8);
  delete b;
}

// ---- phase two ---------------------------------------------------------------------------------
// ---- table sizing (Sec. 3.4) ---------------------------------------------------------------------
// capacity = expected distinct keys / load factor, the load factor taken per table-size class
// (class = table bytes at load factor 0.5), so that the autotuner can pick denser tables where
// they stay in L2 and sparser ones where probes go to HBM.
struct Sizing {
  double alpha[GERBIL_TUNE_CLASSES];
  uint32_t scheme;                        // probe scheme of every table (BinWork::scheme)
  uint32_t item;                          // k-mers per insert work item
  uint64_t bound[GERBIL_TUNE_CLASSES - 1];  // class upper bounds, bytes
  uint64_t slot_bytes;
  uint32_t window;                        // slots per probe window of scheme 1
  int cls(double est) const {
    const double bytes = est / 0.5 * (double)slot_bytes;
    for (int c = 0; c < GERBIL_TUNE_CLASSES - 1; ++c)
      if (bytes < (double)bound[c]) return c;
    return GERBIL_TUNE_CLASSES - 1;
  }
  // slots of a table for est distinct keys; under scheme 1 a prime number of windows, so that
  // every window step (1 .. windows-1) visits every window before repeating one
  uint64_t cap(double est) const {
    const int c = cls(est);
    const uint64_t n = (uint64_t)std::ceil(est / alpha[c]) + 16;
    return scheme == 1 ? next_prime32((n + window - 1) / window) * window : n;
  }
  static bool is_prime32(uint64_t n) {
    if (n < 2) return false;
    for (uint64_t p : {2ull, 3ull, 5ull, 7ull, 11ull, 13ull})
      if (n % p == 0) return n == p;
    // Miller-Rabin with the bases 2, 7 and 61, exact for n < 2^32 (Jaeschke, 1993)
    uint64_t d = n - 1;
    int r = 0;
    while (!(d & 1)) { d >>= 1; ++r; }
    for (uint64_t a : {2ull, 7ull, 61ull}) {
      if (a % n == 0) continue;
      uint64_t x = 1, base = a % n, e = d;
      while (e) {
        if (e & 1) x = x * base % n;
        base = base * base % n;
        e >>= 1;
      }
      if (x == 1 || x == n - 1) continue;
      bool comp = true;
      for (int i = 1; i < r && comp; ++i) {
        x = x * x % n;
        if (x == n - 1) comp = false;
      }
      if (comp) return false;
    }
    return true;
  }
  static uint64_t next_prime32(uint64_t n) {
    if (n < 2) return 2;
    while (!is_prime32(n)) ++n;
    return n;
  }
  // a bin's work entry: table size (of its class), probe scheme and item size
  void place(BinWork& w, double est, uint64_t* slots, uint64_t* items) const {
    w.scheme = scheme;
    w.item_kmers = item;
    uint64_t cp = cap(est);
    if (cp > 0xFFFFF000ull) cp = w.scheme == 1 ? 4294967291ull / window * window : 0xFFFFF000ull;
    if (w.scheme == 1) *slots = (*slots + window - 1) / window * window;  // window-aligned
    w.cap = (uint32_t)cp;
    w.table_off = *slots;
    w.item_begin = (uint32_t)*items;
    *slots += cp;
    *items += (w.n_kmers + w.item_kmers - 1) / w.item_kmers;
  }
};

static bool valid_item_kmers(uint32_t ik) { return ik == 64 || ik == 128 || ik == 256; }

static const uint64_t kClassBound[GERBIL_TUNE_CLASSES - 1] = {4ull << 20, 64ull << 20, 1ull << 30};

static Sizing make_sizing(const gerbil_ctx* ctx, const gerbil_opts& o, int k) {
  Sizing z{};
  z.slot_bytes = 8ull * gerbil::slot_words_for_k(k);
  z.window = gerbil::probe_window_for_k(k);
  const double a = (o.load_factor > 0.05f && o.load_factor <= 0.95f) ? o.load_factor : 0.5;
  for (int c = 0; c < GERBIL_TUNE_CLASSES; ++c) z.alpha[c] = a;
  z.scheme = o.probe_scheme == 1 ? 1u : 0u;
  z.item = valid_item_kmers(o.item_kmers) ? o.item_kmers : (uint32_t)gerbil::ITEM_KMERS;
  for (int c = 0; c < GERBIL_TUNE_CLASSES - 1; ++c) z.bound[c] = kClassBound[c];
  if (o.autotune) {
    auto it = ctx->tuning.find(words_for(k));
    if (it != ctx->tuning.end()) {
      const gerbil_tuning& t = it->second;
      for (int c = 0; c < GERBIL_TUNE_CLASSES; ++c)
        if (t.load_factor[c] > 0.05f && t.load_factor[c] <= 0.95f) z.alpha[c] = t.load_factor[c];
      if (t.probe_scheme == 0 || t.probe_scheme == 1) z.scheme = (uint32_t)t.probe_scheme;
      if (valid_item_kmers(t.item_kmers)) z.item = t.item_kmers;
    }
  }
  if (words_for(k) > 4) z.item = gerbil::ITEM_KMERS;  // smaller items are built up to 4 words
  return z;
}

// Probe order (gerbil_opts.claim_first): claim first when most k-mers of the batch are expected
// to be new keys and the key is wide, where a load-then-CAS costs two accesses per new key
// against one for the CAS first.  Measured on the 1000 bp read sweep: claiming first was 6%
// faster at k = 400 and 479 (distinct ratios 0.63 and 0.71, keys of 13 and 15 words) and
// slower at every k up to 320 (ratios up to 0.55), and on long reads with 10% errors at k = 200
// (every key new, 7 words, tables in HBM) 8% slower.
static int claim_first_for(const gerbil_ctx* ctx, const gerbil_opts& o, int k) {
  if (o.claim_first == 1) return 1;
  if (o.claim_first == 2) return 0;
  const double r = o.distinct_ratio > 0.0f ? (double)o.distinct_ratio : (ctx->ratio_known ? ctx->ratio : 1.0);
  return r > 0.6 && words_for(k) >= 10 ? 1 : 0;
}

// ---- phase two, fused persistent form -----------------------------------------------------------
// Returns FUSED_FALLBACK when the overflow area was used: the result is then recomputed by the
// classic form, which merges overflow counts.
static const int FUSED_FALLBACK = -1;
static const int LAG = 5;  // bins between a bin's inserts and its compaction in the queue

// 1 when the bins' tables average more than the L2 cache: their probes then go to HBM however
// many warps are in flight, and the insert kernel for wide keys runs without its register cap.
static int tables_beyond_l2(const gerbil_ctx* ctx, const std::vector<BinWork>& work, int SW) {
  if (work.empty()) return 0;
  unsigned long long slots = 0;
  for (const BinWork& w : work) slots += w.cap;
  return slots * (unsigned long long)SW * 8ull > (unsigned long long)ctx->l2_bytes * work.size() ? 1 : 0;
}

static int count_fused(gerbil_ctx* ctx, const gerbil_bins* b, const std::vector<int32_t>& list,
                       int k, uint32_t min_count, const gerbil_opts& opts, double ratio,
                       const Sizing& sz, uint32_t theta, uint32_t spin_limit, gerbil_counts** out) {
  const int W = words_for(k);
  const int SW = gerbil::slot_words_for_k(k);
  cudaStream_t st = ctx->stream;
  std::vector<BinWork> work;
  uint64_t occ = 0;
  for (int32_t bi : list) {
    if (b->nkmers[bi] == 0) continue;
    BinWork w{};
    w.sm_begin = b->sm_begin[bi];
    w.n_super = (uint32_t)b->nsuper[bi];
    w.n_kmers = (uint32_t)b->nkmers[bi];
    const double est = std::max(1.0, std::ceil(ratio * (double)w.n_kmers));
    w.cap = (uint32_t)std::min<uint64_t>(sz.cap(est), 0xFFFFF000ull);
    w.item_kmers = gerbil::ITEM_KMERS;  // the fused form probes linearly, in 256-k-mer items
    w.scheme = 0;
    w.n_items = (w.n_kmers + gerbil::ITEM_KMERS - 1) / gerbil::ITEM_KMERS;
    w.n_chunks = (w.cap + gerbil::CHUNK_SLOTS - 1) / gerbil::CHUNK_SLOTS;
    occ += w.n_kmers;
    work.push_back(w);
  }
  const size_t nw = work.size();
  // table placement: bins up to 1/(LAG+2) of the ring go to the L2-sized ring (first fit,
  // wrapping), the rest to dedicated memory after it.  The ring is kept as intervals with the
  // last bin that used each; a bin depends on every bin whose interval it overlaps.  A bin
  // that would overlap one of its LAG predecessors (whose compactions are queued after its
  // inserts) gets dedicated memory instead.
  const uint64_t ring = opts.ring_slots ? (uint64_t)opts.ring_slots
                                        : std::max<uint64_t>(4096, (uint64_t)(0.6 * ctx->l2_bytes) / (SW * 8));
  std::map<uint64_t, std::pair<uint64_t, uint32_t>> owner;  // start -> (end, work index)
  std::vector<uint32_t> deps;
  uint64_t cursor = 0, ded = 0;
  bool any_ring = false;
  std::vector<char> dedicated(nw, 0);
  for (size_t i = 0; i < nw; ++i) {
    BinWork& w = work[i];
    w.dep_begin = (uint32_t)deps.size();
    w.dep_count = 0;
    if ((uint64_t)w.cap * (LAG + 2) > ring) {
      dedicated[i] = 1;
      continue;
    }
    const uint64_t a = (cursor + w.cap > ring) ? 0 : cursor, e = a + w.cap;
    // collect and cut the owners of [a, e)
    bool too_close = false;
    for (auto it2 = owner.begin(); it2 != owner.end(); ++it2)
      if (it2->first < e && it2->second.first > a && it2->second.second + LAG + 1 > i) too_close = true;
    if (too_close) {
      dedicated[i] = 1;
      continue;
    }
    auto it = owner.upper_bound(a);
    if (it != owner.begin()) --it;
    std::vector<std::pair<uint64_t, std::pair<uint64_t, uint32_t>>> keep;
    while (it != owner.end() && it->first < e) {
      const uint64_t s0 = it->first, e0 = it->second.first;
      const uint32_t who = it->second.second;
      if (e0 > a) {
        if (std::find(deps.begin() + w.dep_begin, deps.end(), who) == deps.end()) deps.push_back(who);
        if (s0 < a) keep.push_back({s0, {a, who}});
        if (e0 > e) keep.push_back({e, {e0, who}});
        it = owner.erase(it);
      } else {
        ++it;
      }
    }
    for (auto& kv : keep) owner[kv.first] = kv.second;
    owner[a] = {e, (uint32_t)i};
    w.dep_count = (uint32_t)deps.size() - w.dep_begin;

    w.table_off = a;
    cursor = e;
    any_ring = true;
  }
  const uint64_t ring_used = any_ring ? ring : 0;
  for (size_t i = 0; i < nw; ++i)
    if (dedicated[i]) {
      work[i].table_off = ring_used + ded;
      ded += work[i].cap;
    }
  const uint64_t slots = ring_used + ded;
  // queue order: the compaction chunks of bin i follow the insert items of bin i+LAG:
  // I(0) .. I(LAG), C(0), I(LAG+1), C(1), ..., C(last)
  uint64_t pos = 0;
  for (size_t i = 0; i < nw; ++i) {
    work[i].task_insert = (uint32_t)pos;
    pos += work[i].n_items;
    if (i >= (size_t)LAG) {
      work[i - LAG].task_compact = (uint32_t)pos;
      pos += work[i - LAG].n_chunks;
    }
  }
  for (size_t i = (nw > (size_t)LAG ? nw - LAG : 0); i < nw; ++i) {
    work[i].task_compact = (uint32_t)pos;
    pos += work[i].n_chunks;
  }
  const uint64_t ntasks = pos;
  if (ntasks >= (1ull << 32)) return fail(ctx, GERBIL_E_INVAL, "too many work items");

  const uint64_t ovf_cap = opts.overflow_slots ? (uint64_t)opts.overflow_slots
                                               : std::max<uint64_t>(1 << 16, occ / 32);
  int rc;
  bool grown = false;
  const size_t arena_need = slots * SW * 8;
  if ((rc = scratch(ctx, &ctx->arena, &ctx->arena_bytes, arena_need + 256, &grown))) return rc;
  if (grown) ctx->arena_dirty = ctx->arena_bytes;
  if ((rc = scratch(ctx, &ctx->ovf, &ctx->ovf_bytes, ovf_cap * W * 8 + 256))) return rc;
  auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t o_work = 0, o_bovf = up(nw * sizeof(BinWork)), o_items = o_bovf + up(nw * 4),
               o_chunks = o_items + up(nw * 4), o_queue = o_chunks + up(nw * 4),
               o_deps = o_queue + 256, o_tasks = o_deps + up(deps.size() * 4 + 4),
               small_need = o_tasks + up(ntasks * 8) + 256;
  if ((rc = scratch(ctx, &ctx->small, &ctx->small_bytes, small_need))) return rc;
  char* sm = (char*)ctx->small;

  // rows <= live slots of all tables (ring regions are reused, so count every bin's table)
  uint64_t cap_sum = 0;
  for (const BinWork& w : work) cap_sum += w.cap;
  const uint64_t out_cap = std::max<uint64_t>(1, std::min<uint64_t>(occ, cap_sum));
  gerbil_counts* res = new (std::nothrow) gerbil_counts;
  if (!res) return GERBIL_E_NOMEM;
  res->ctx = ctx;
  res->W = W;
  res->bytes = out_cap * (W * 8 + 4);
  if ((rc = dev_alloc(ctx, (void**)&res->keys, out_cap * W * 8))) { delete res; return rc; }
  if ((rc = dev_alloc(ctx, (void**)&res->counts, out_cap * 4))) {
    dev_free(ctx, res->keys, out_cap * W * 8);
    delete res;
    return rc;
  }
  auto drop = [&]() { gerbil_counts_free(res); };
#define CKF(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      drop();                                                                              \
      ctx->arena_dirty = ctx->arena_bytes;                                                            \
      return fail(ctx, GERBIL_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    }                                                                                      \
  } while (0)

  ctx->times.calls++;
  ph_begin(ctx, PH_CLEAR);
  if (ctx->arena_dirty)
    CKF(cudaMemsetAsync(ctx->arena, 0, std::min(ctx->arena_bytes, std::max(ctx->arena_dirty, arena_need)), st));
  ctx->arena_dirty = 0;
  CKF(cudaMemsetAsync(ctx->ctr, 0, sizeof(Counters), st));
  CKF(cudaMemsetAsync(sm + o_bovf, 0, o_tasks - o_bovf, st));
  if (nw) CKF(cudaMemcpyAsync(sm + o_work, work.data(), nw * sizeof(BinWork), cudaMemcpyHostToDevice, st));
  if (!deps.empty())
    CKF(cudaMemcpyAsync(sm + o_deps, deps.data(), deps.size() * 4, cudaMemcpyHostToDevice, st));
  gerbil::FusedParams fp{};
  fp.c.packed = b->packed;
  fp.c.sm_pos = b->sm_pos;
  fp.c.sm_koff = b->sm_koff;
  fp.c.work = (const BinWork*)(sm + o_work);
  fp.c.nwork = (uint32_t)nw;
  fp.c.nitems = 0;
  fp.c.imap = nullptr;
  fp.c.scheme = 0;
  fp.c.cas_first = 0;  // the fused kernel reads first
  fp.c.item_kmers = gerbil::ITEM_KMERS;
  fp.c.k = k;
  fp.c.canonical = opts.canonical ? 1 : 0;
  fp.c.theta = theta;
  fp.c.spin_limit = spin_limit;
  fp.c.arena = (unsigned long long*)ctx->arena;
  fp.c.ovf = (unsigned long long*)ctx->ovf;
  fp.c.ovf_cap = ovf_cap;
  fp.c.bin_ovf = (uint32_t*)(sm + o_bovf);
  fp.c.ctr = ctx->ctr;
  fp.c.probe_hist = ctx->probe_hist;
  fp.tasks = (const unsigned long long*)(sm + o_tasks);
  fp.deps = (const uint32_t*)(sm + o_deps);
  fp.ntasks = ntasks;
  fp.items_done = (uint32_t*)(sm + o_items);
  fp.chunks_done = (uint32_t*)(sm + o_chunks);
  fp.min_count = min_count;
  fp.out_keys = res->keys;
  fp.out_counts = res->counts;
  fp.out_cap = out_cap;
  fp.wait_ns = 2000000000ull;  // 2 s
  fp.queue = (unsigned long long*)(sm + o_queue);
  if (nw) {
    CKF(gerbil::launch_task_map(fp, st));
    ctx->times.kernel_launches++;
  }
  ph_end(ctx, PH_CLEAR);
  ph_begin(ctx, PH_INSERT);
  if (ntasks) {
    CKF(gerbil::launch_fused(k, fp, ctx->nsm, st));
    ctx->times.kernel_launches++;
    ctx->times.insert_launches++;
  }
  ph_end(ctx, PH_INSERT);
  if ((rc = read_counters(ctx))) {
    drop();
    ctx->arena_dirty = ctx->arena_bytes;
    return rc;
  }
  const Counters h = *ctx->hctr;
  if (h.err & (gerbil::ERR_QUEUE | gerbil::ERR_STATE | gerbil::ERR_OUT_FULL | gerbil::ERR_SPIN)) {
    drop();
    ctx->arena_dirty = ctx->arena_bytes;
    if (h.err & gerbil::ERR_QUEUE) return fail(ctx, GERBIL_E_TIMEOUT, "work-queue wait gave up");
    return fail(ctx, GERBIL_E_STATE, "device consistency check failed");
  }
  // every table region was compacted and zeroed: the arena is clean again
  if (h.ovf_count || (h.err & gerbil::ERR_OVF_FULL)) {
    drop();
    return FUSED_FALLBACK;
  }
  gerbil_count_stats stats{};
  stats.bins = (uint32_t)list.size();
  stats.occurrences = occ;
  stats.emitted = h.out_count;
  stats.distinct = h.distinct;
  stats.table_slots = cap_sum;
  res->n = h.out_count;
  res->stats = stats;
  if (occ > 0) {
    ctx->ratio = (double)h.distinct / (double)occ;
    ctx->ratio_known = true;
  }
  *out = res;
  return GERBIL_OK;
#undef CKF
}

// ---- phase two in waves -------------------------------------------------------------------------
// Bins are grouped into waves whose tables together fit in half of L2; every wave reuses the
// same arena region: clear it, insert the wave's items, compact its tables.  A table is thus
// created, filled and read while it is hot in L2.  Returns WAVES_FALLBACK when the overflow
// area was used (the all-tables form below merges overflow counts).
static const int WAVES_FALLBACK = -2;

static int count_waves(gerbil_ctx* ctx, const gerbil_bins* b, const std::vector<int32_t>& list,
                       int k, uint32_t min_count, const gerbil_opts& opts, double ratio,
                       const Sizing& sz, uint32_t theta, uint32_t spin_limit, gerbil_counts** out) {
  const int W = words_for(k);
  const int SW = gerbil::slot_words_for_k(k);
  cudaStream_t st = ctx->stream;
  std::vector<BinWork> work;
  uint64_t occ = 0, items = 0, cap_sum = 0;
  for (int32_t bi : list) {
    if (b->nkmers[bi] == 0) continue;
    BinWork w{};
    w.sm_begin = b->sm_begin[bi];
    w.n_super = (uint32_t)b->nsuper[bi];
    w.n_kmers = (uint32_t)b->nkmers[bi];
    const double est = std::max(1.0, std::ceil(ratio * (double)w.n_kmers));
    w.cap = (uint32_t)std::min<uint64_t>(sz.cap(est), 0xFFFFF000ull);
    w.item_kmers = gerbil::ITEM_KMERS;  // waves probe linearly, in 256-k-mer items
    w.scheme = 0;
    w.item_begin = (uint32_t)items;
    items += (w.n_kmers + gerbil::ITEM_KMERS - 1) / gerbil::ITEM_KMERS;
    occ += w.n_kmers;
    cap_sum += w.cap;
    work.push_back(w);
  }
  if (items >= (1ull << 32)) return fail(ctx, GERBIL_E_INVAL, "too many work items");
  const size_t nw = work.size();
  const uint64_t budget = opts.ring_slots ? (uint64_t)opts.ring_slots
                                          : std::max<uint64_t>(4096, (uint64_t)(0.5 * ctx->l2_bytes) / (SW * 8));
  struct Wave { size_t w0, w1; uint64_t slots, it0, it1; };
  std::vector<Wave> waves;
  uint64_t region = 0;
  for (size_t i = 0; i < nw;) {
    Wave v{i, i, 0, work[i].item_begin, 0};
    while (v.w1 < nw && (v.w1 == v.w0 || v.slots + work[v.w1].cap <= budget)) {
      work[v.w1].table_off = v.slots;
      v.slots += work[v.w1].cap;
      ++v.w1;
    }
    v.it1 = (v.w1 < nw) ? work[v.w1].item_begin : items;
    region = std::max(region, v.slots);
    waves.push_back(v);
    i = v.w1;
  }
  const uint64_t ovf_cap = opts.overflow_slots ? (uint64_t)opts.overflow_slots
                                               : std::max<uint64_t>(1 << 16, occ / 32);
  int rc;
  bool grown = false;
  const size_t arena_need = region * SW * 8;
  if ((rc = scratch(ctx, &ctx->arena, &ctx->arena_bytes, arena_need + 256, &grown))) return rc;
  if (grown) ctx->arena_dirty = ctx->arena_bytes;
  if ((rc = scratch(ctx, &ctx->ovf, &ctx->ovf_bytes, ovf_cap * W * 8 + 256))) return rc;
  auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t o_work = 0, o_bovf = up(nw * sizeof(BinWork)), o_queue = o_bovf + up(nw * 4),
               o_imap = o_queue + up(waves.size() * 8), small_need = o_imap + up(items * 8) + 256;
  if ((rc = scratch(ctx, &ctx->small, &ctx->small_bytes, small_need))) return rc;
  char* sm = (char*)ctx->small;

  const uint64_t out_cap = std::max<uint64_t>(1, std::min<uint64_t>(occ, cap_sum));
  gerbil_counts* res = new (std::nothrow) gerbil_counts;
  if (!res) return GERBIL_E_NOMEM;
  res->ctx = ctx;
  res->W = W;
  res->bytes = out_cap * (W * 8 + 4);
  if ((rc = dev_alloc(ctx, (void**)&res->keys, out_cap * W * 8))) { delete res; return rc; }
  if ((rc = dev_alloc(ctx, (void**)&res->counts, out_cap * 4))) {
    dev_free(ctx, res->keys, out_cap * W * 8);
    delete res;
    return rc;
  }
  auto drop = [&]() { gerbil_counts_free(res); };
#define CKW(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      drop();                                                                              \
      ctx->arena_dirty = ctx->arena_bytes;                                                 \
      return fail(ctx, GERBIL_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    }                                                                                      \
  } while (0)

  ctx->times.calls++;
  ph_begin(ctx, PH_CLEAR);
  CKW(cudaMemsetAsync(ctx->ctr, 0, sizeof(Counters), st));
  CKW(cudaMemsetAsync(sm + o_bovf, 0, o_imap - o_bovf, st));
  if (nw) CKW(cudaMemcpyAsync(sm + o_work, work.data(), nw * sizeof(BinWork), cudaMemcpyHostToDevice, st));
  gerbil::CountParams cp{};
  cp.packed = b->packed;
  cp.sm_pos = b->sm_pos;
  cp.sm_koff = b->sm_koff;
  cp.work = (const BinWork*)(sm + o_work);
  cp.nwork = (uint32_t)nw;
  cp.imap = (unsigned long long*)(sm + o_imap);
  cp.k = k;
  cp.canonical = opts.canonical ? 1 : 0;
  cp.theta = theta;
  cp.spin_limit = spin_limit;
  cp.arena = (unsigned long long*)ctx->arena;
  cp.ovf = (unsigned long long*)ctx->ovf;
  cp.ovf_cap = ovf_cap;
  cp.bin_ovf = (uint32_t*)(sm + o_bovf);
  cp.ctr = ctx->ctr;
  cp.probe_hist = ctx->probe_hist;
  cp.schedule = opts.schedule;
  cp.wide_tables = tables_beyond_l2(ctx, work, SW);
  cp.scheme = 0;  // waves probe linearly, in 256-k-mer items
  cp.cas_first = claim_first_for(ctx, opts, k);
  cp.item_kmers = gerbil::ITEM_KMERS;
  if (items) {
    cp.nitems = items;
    CKW(gerbil::launch_item_map(cp, ctx->nsm, st));
    ctx->times.kernel_launches++;
  }
  ph_end(ctx, PH_CLEAR);
  ph_begin(ctx, PH_INSERT);
  for (size_t wv = 0; wv < waves.size(); ++wv) {
    const Wave& v = waves[wv];
    CKW(cudaMemsetAsync(ctx->arena, 0, v.slots * SW * 8, st));
    cp.item_base = v.it0;
    cp.nitems = v.it1;
    cp.queue = (unsigned long long*)(sm + o_queue) + wv;
    CKW(gerbil::launch_insert(k, cp, opts.persistent, ctx->nsm, st));
    gerbil::CompactParams xp{};
    xp.work = cp.work + v.w0;
    xp.nwork = (uint32_t)(v.w1 - v.w0);
    xp.slot_lo = 0;
    xp.slot_hi = v.slots;
    xp.arena = cp.arena;
    xp.bin_ovf = cp.bin_ovf + v.w0;
    xp.mode = 0;
    xp.min_count = min_count;
    xp.out_keys = res->keys;
    xp.out_counts = res->counts;
    xp.out_cap = out_cap;
    xp.ctr = ctx->ctr;
    CKW(gerbil::launch_compact(k, xp, ctx->nsm, st));
    ctx->times.kernel_launches += 2;
    ctx->times.insert_launches++;
  }
  ph_end(ctx, PH_INSERT);
  ctx->arena_dirty = std::max(ctx->arena_dirty, arena_need);  // the last wave's tables stay
  if ((rc = read_counters(ctx))) {
    drop();
    return rc;
  }
  const Counters h = *ctx->hctr;
  if (h.err & (gerbil::ERR_STATE | gerbil::ERR_OUT_FULL | gerbil::ERR_SPIN)) {
    drop();
    return fail(ctx, GERBIL_E_STATE, "device consistency check failed");
  }
  if (h.ovf_count || (h.err & gerbil::ERR_OVF_FULL)) {
    drop();
    return WAVES_FALLBACK;
  }
  gerbil_count_stats stats{};
  stats.bins = (uint32_t)list.size();
  stats.occurrences = occ;
  stats.emitted = h.out_count;
  stats.distinct = h.distinct;
  stats.table_slots = cap_sum;
  res->n = h.out_count;
  res->stats = stats;
  if (occ > 0) {
    ctx->ratio = (double)h.distinct / (double)occ;
    ctx->ratio_known = true;
  }
  *out = res;
  return GERBIL_OK;
#undef CKW
}

// Bytes the hash tables of one batch may take (gerbil_opts.max_table_mib).
static uint64_t table_limit(gerbil_ctx* ctx, const gerbil_opts& opts) {
  if (opts.max_table_mib) return (uint64_t)opts.max_table_mib << 20;
  if (ctx->budget) return (ctx->budget - std::min<uint64_t>(ctx->budget, ctx->used.load())) / 2;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return ~0ull;
  // the context's own cached arena is reused by the tables, so it counts as free
  return ((uint64_t)free_b + ctx->arena_bytes) / 2;
}

// Append a group's result to a joined result (flattening a joined part).
static void join_part(gerbil_counts* joined, gerbil_counts* part) {
  gerbil_count_stats& a = joined->stats;
  const gerbil_count_stats& p = part->stats;
  a.occurrences += p.occurrences;
  a.distinct += p.distinct;
  a.emitted += p.emitted;
  a.overflowed += p.overflowed;
  a.table_slots += p.table_slots;
  a.retries += p.retries;
  a.bins += p.bins;
  joined->n += part->n;
  if (!part->parts.empty()) {
    for (gerbil_counts* q : part->parts) joined->parts.push_back(q);
    part->parts.clear();
    delete part;
  } else {
    joined->parts.push_back(part);
  }
}

static int autotune_impl(gerbil_ctx* ctx, const gerbil_bins* b, const std::vector<int32_t>& list,
                         int k, uint32_t min_count, const gerbil_opts& opts, gerbil_tuning* out);

static int count_impl(gerbil_ctx* ctx, const gerbil_bins* b, const std::vector<int32_t>& list,
                      int k, uint32_t min_count, const gerbil_opts& opts_in, gerbil_counts** out) {
  const int W = words_for(k);
  cudaStream_t st = ctx->stream;
  gerbil_opts opts = opts_in;
  if (opts.autotune) {  // the tuned form, schedule and load factors (tuned here on first use)
    auto it = ctx->tuning.find(W);
    if (it == ctx->tuning.end() && list.size() >= 8) {
      gerbil_tuning t{};
      const int rc = autotune_impl(ctx, b, list, k, min_count, opts, &t);
      if (rc) return rc;
      it = ctx->tuning.find(W);
    }
    if (it != ctx->tuning.end()) {
      opts.fused = it->second.fused;
      opts.schedule = it->second.schedule;
    }
  }
  const Sizing sz = make_sizing(ctx, opts, k);
  double ratio = opts.distinct_ratio > 0.0f ? std::min(1.0, (double)opts.distinct_ratio)
                                            : std::min(1.0, ctx->ratio_known ? ctx->ratio * 1.25 : 1.0);
  uint32_t theta = opts.max_probes ? opts.max_probes : 1024;
  const uint32_t spin_limit = 1u << 20;

  uint64_t occ = 0;
  for (int32_t bi : list) occ += b->nkmers[bi];

  gerbil_count_stats stats{};
  stats.bins = (uint32_t)list.size();
  stats.occurrences = occ;

  // Sec. 3.4 "Estimating table sizes": the distinct/total ratio is adjusted at runtime.  With
  // no ratio learned yet, count about 1/16 of the bins first (tables sized for all-distinct)
  // and size the whole batch from what they show.
  if (opts.distinct_ratio <= 0.0f && !ctx->ratio_known && list.size() > 32) {
    std::vector<int32_t> sample;
    const size_t step = list.size() / 16;
    for (size_t i = 0; i < list.size(); i += step) sample.push_back(list[i]);
    gerbil_opts so = opts;
    so.fused = 0;
    gerbil_counts* tmp = nullptr;
    const int rc = count_impl(ctx, b, sample, k, min_count, so, &tmp);
    if (rc) return rc;
    gerbil_counts_free(tmp);
    if (ctx->ratio_known) ratio = std::min(1.0, ctx->ratio * 1.25);
  }

  // The tables of all bins of a call are held at once.  Where they would take more than the
  // table limit, the bins are counted in consecutive groups under it, one after another in
  // the same arena (each k-mer lives in exactly one bin, Sec. 3.2, so the rows of the groups
  // are joined unchanged).
  if (list.size() > 1) {
    const uint64_t limit = table_limit(ctx, opts);
    const uint64_t slot_bytes = 8ull * gerbil::slot_words_for_k(k);
    auto bin_bytes = [&](int32_t bi) -> uint64_t {
      if (b->nkmers[bi] == 0) return 0;
      const double est = std::max(1.0, std::ceil(ratio * (double)b->nkmers[bi]));
      return sz.cap(est) * slot_bytes;
    };
    uint64_t need = 0;
    for (int32_t bi : list) need += bin_bytes(bi);
    if (need > limit) {
      gerbil_counts* joined = new (std::nothrow) gerbil_counts;
      if (!joined) return fail(ctx, GERBIL_E_NOMEM, "host allocation");
      joined->ctx = ctx;
      joined->W = W;
      size_t i = 0;
      while (i < list.size()) {
        std::vector<int32_t> group;
        uint64_t g = 0;
        while (i < list.size() && (group.empty() || g + bin_bytes(list[i]) <= limit)) {
          g += bin_bytes(list[i]);
          group.push_back(list[i++]);
        }
        gerbil_counts* part = nullptr;
        const int rc = count_impl(ctx, b, group, k, min_count, opts, &part);
        if (rc) {
          gerbil_counts_free(joined);
          return rc;
        }
        join_part(joined, part);
      }
      joined->stats.groups = (uint32_t)joined->parts.size();
      *out = joined;
      return GERBIL_OK;
    }
  }

  if (opts.fused == 1) {
    const int rc = count_fused(ctx, b, list, k, min_count, opts, ratio, sz, theta, spin_limit, out);
    if (rc != FUSED_FALLBACK) return rc;
  } else if (opts.fused == 2) {
    const int rc = count_waves(ctx, b, list, k, min_count, opts, ratio, sz, theta, spin_limit, out);
    if (rc != WAVES_FALLBACK) return rc;
  }

  bool exact_retry = false;
  for (int round = 0; round < 5; ++round) {
    // table sizing per bin (Sec. 3.4: expected distinct = ratio x k-mers of the file)
    std::vector<BinWork> work;
    work.reserve(list.size());
    uint64_t slots = 0, items = 0;
    for (int32_t bi : list) {
      if (b->nkmers[bi] == 0) continue;
      BinWork w{};
      w.sm_begin = b->sm_begin[bi];
      w.n_super = (uint32_t)b->nsuper[bi];
      w.n_kmers = (uint32_t)b->nkmers[bi];
      const double est = std::max(1.0, std::ceil(ratio * (double)w.n_kmers));
      sz.place(w, est, &slots, &items);
      work.push_back(w);
    }
    if (items >= (1ull << 32)) return fail(ctx, GERBIL_E_INVAL, "too many work items");
    // the overflow area grows 4x per retry (a caller-given size is the starting size)
    const uint64_t ovf_cap = (opts.overflow_slots ? (uint64_t)opts.overflow_slots
                                                  : std::max<uint64_t>(1 << 16, occ / 32))
                             << (2 * round);
    const int SWk = gerbil::slot_words_for_k(k);
    const size_t arena_need = slots * SWk * 8;
    int rc;
    bool grown = false;
    if ((rc = scratch(ctx, &ctx->arena, &ctx->arena_bytes, arena_need + 256, &grown))) return rc;
    if (grown) ctx->arena_dirty = ctx->arena_bytes;
    if ((rc = scratch(ctx, &ctx->ovf, &ctx->ovf_bytes, ovf_cap * W * 8 + 256))) return rc;
    const size_t work_bytes = work.size() * sizeof(BinWork);
    const size_t small_need = ((work_bytes + 255) & ~size_t(255)) + ((work.size() * 4 + 255) & ~size_t(255)) +
                              items * 8 + 512;
    if ((rc = scratch(ctx, &ctx->small, &ctx->small_bytes, small_need))) return rc;
    BinWork* dwork = (BinWork*)ctx->small;
    uint32_t* bin_ovf = (uint32_t*)((char*)ctx->small + ((work_bytes + 255) & ~size_t(255)));

    // result buffer (allocated after the inserts): at most one row per expected distinct key
    // plus the overflow-only keys; if that is large, a count-only pass sizes it exactly
    uint64_t out_cap = std::max<uint64_t>(
        1, std::min<uint64_t>({occ, slots + ovf_cap, (uint64_t)std::ceil(ratio * (double)occ) + ovf_cap}));
    // the rows of the last batch at this min_count, per occurrence, bound a repeated batch's
    // rows far better than its distinct keys do (a low estimate is caught: the batch is then
    // counted again with an exact count-only pass first)
    if (ctx->emit_known && ctx->emit_min_count == min_count)
      out_cap = std::max<uint64_t>(1, std::min<uint64_t>(
          out_cap, (uint64_t)std::ceil(1.25 * ctx->emit_ratio * (double)occ) + 65536 + ovf_cap));
    // a count-only pass first (one more scan of every table) only for a result too large to
    // hold at its estimate: above 2 GB and a quarter of the table limit
    const uint64_t exact_bytes = std::max<uint64_t>(2ull << 30, table_limit(ctx, opts) / 4);
    const bool exact_out = exact_retry || out_cap * (uint64_t)(W * 8 + 4) > exact_bytes;
    gerbil_counts* res = nullptr;
    auto drop = [&]() {
      if (res) gerbil_counts_free(res);
      res = nullptr;
    };
#define CKR(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      drop();                                                                              \
      return fail(ctx, GERBIL_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    }                                                                                      \
  } while (0)

    // Graph form: the device steps below (clears, work upload, item map, insert, compaction)
    // are captured on a side stream into one CUDA graph and launched on the context's stream;
    // the graph of the previous batch is updated in place when the shape allows.
    const bool graph = opts.graph != 0;
    bool capturing = false;
    cudaStream_t ls = st;  // stream the device steps are issued to
#define CKG(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      if (capturing) {                                                                     \
        cudaGraph_t g_ = nullptr;                                                          \
        cudaStreamEndCapture(ctx->cap_stream, &g_);                                        \
        if (g_) cudaGraphDestroy(g_);                                                      \
        cudaGetLastError();                                                                \
      }                                                                                    \
      drop();                                                                              \
      return fail(ctx, GERBIL_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    }                                                                                      \
  } while (0)
    auto alloc_res = [&](uint64_t cap) -> int {
      res = new (std::nothrow) gerbil_counts;
      if (!res) return GERBIL_E_NOMEM;
      res->ctx = ctx;
      res->W = W;
      res->bytes = cap * (W * 8 + 4);
      int r;
      if ((r = dev_alloc(ctx, (void**)&res->keys, cap * W * 8))) {
        delete res;
        res = nullptr;
        return r;
      }
      if ((r = dev_alloc(ctx, (void**)&res->counts, cap * 4))) {
        dev_free(ctx, res->keys, cap * W * 8);
        delete res;
        res = nullptr;
        return r;
      }
      return GERBIL_OK;
    };
    if (!exact_out && (rc = alloc_res(out_cap))) return rc;  // allocated ahead of the steps
    const void* work_src = work.data();
    if (graph) {
      if (!ctx->cap_stream) CKR(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
      if (work_bytes > ctx->hwork_bytes) {
        if (ctx->hwork) cudaFreeHost(ctx->hwork);
        ctx->hwork = nullptr;
        ctx->hwork_bytes = 0;
        CKR(cudaMallocHost(&ctx->hwork, work_bytes));
        ctx->hwork_bytes = work_bytes;
      }
      if (work_bytes) std::memcpy(ctx->hwork, work.data(), work_bytes);
      work_src = ctx->hwork;
      CKR(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
      capturing = true;
      ls = ctx->cap_stream;
    }

    ctx->times.calls++;
    ph_begin(ctx, PH_CLEAR, ls, capturing);
    // only what earlier calls left non-zero is cleared (the whole dirty prefix of the arena):
    // a successful compaction zeroes every slot it takes, so repeated batches skip this
    if (ctx->arena_dirty) CKG(cudaMemsetAsync(ctx->arena, 0, ctx->arena_dirty, ls));
    ctx->arena_dirty = arena_need;  // dirty until the compaction succeeds
    CKG(cudaMemsetAsync(ctx->ctr, 0, sizeof(Counters), ls));
    if (!work.empty()) {
      CKG(cudaMemcpyAsync(dwork, work_src, work_bytes, cudaMemcpyHostToDevice, ls));
      CKG(cudaMemsetAsync(bin_ovf, 0, work.size() * 4, ls));
    }

    gerbil::CountParams cp{};
    cp.packed = b->packed;
    cp.sm_pos = b->sm_pos;
    cp.sm_koff = b->sm_koff;
    cp.work = dwork;
    cp.nwork = (uint32_t)work.size();
    cp.nitems = items;
    cp.item_base = 0;
    cp.queue = &((Counters*)ctx->ctr)->queue_head;
    cp.imap = (unsigned long long*)((char*)bin_ovf + ((work.size() * 4 + 255) & ~size_t(255)));
    cp.k = k;
    cp.canonical = opts.canonical ? 1 : 0;
    cp.theta = theta;
    cp.spin_limit = spin_limit;
    cp.arena = (unsigned long long*)ctx->arena;
    cp.ovf = (unsigned long long*)ctx->ovf;
    cp.ovf_cap = ovf_cap;
    cp.bin_ovf = bin_ovf;
    cp.ctr = ctx->ctr;
    cp.probe_hist = ctx->probe_hist;
    cp.schedule = opts.schedule;
    cp.wide_tables = tables_beyond_l2(ctx, work, gerbil::slot_words_for_k(k));
    cp.scheme = (int)sz.scheme;
    cp.cas_first = claim_first_for(ctx, opts, k);
    cp.item_kmers = sz.item;
    if (items) {
      CKG(gerbil::launch_item_map(cp, ctx->nsm, ls));  // preparation: timed with the clears
      ctx->times.kernel_launches++;
    }
    ph_end(ctx, PH_CLEAR, ls, capturing);
    ph_begin(ctx, PH_INSERT, ls, capturing);
    if (items) {
      CKG(gerbil::launch_insert(k, cp, opts.persistent, ctx->nsm, ls));
      ctx->times.kernel_launches++;
      ctx->times.insert_launches++;
    }
    ph_end(ctx, PH_INSERT, ls, capturing);
    gerbil::CompactParams xp{};
    xp.work = dwork;
    xp.nwork = (uint32_t)work.size();
    xp.slot_lo = 0;
    xp.slot_hi = slots;
    xp.arena = (unsigned long long*)ctx->arena;
    xp.bin_ovf = bin_ovf;
    xp.min_count = min_count;
    xp.ctr = ctx->ctr;
    xp.zero = 1;
    if (exact_out) {  // count the rows (live slots with count >= min_count), then size exactly
      xp.mode = 2;
      CKG(gerbil::launch_compact(k, xp, ctx->nsm, ls));
      ctx->times.kernel_launches++;
    } else {
      xp.mode = 0;
      xp.out_keys = res->keys;
      xp.out_counts = res->counts;
      xp.out_cap = out_cap;
      ph_begin(ctx, PH_COMPACT, ls, capturing);
      CKG(gerbil::launch_compact(k, xp, ctx->nsm, ls));
      if (slots) ctx->times.kernel_launches++;
      ph_end(ctx, PH_COMPACT, ls, capturing);
    }
    if (capturing) {
      cudaGraph_t g = nullptr;
      capturing = false;
      CKR(cudaStreamEndCapture(ctx->cap_stream, &g));
      bool updated = false;
      if (ctx->gexec) {
        cudaGraphExecUpdateResultInfo info{};
        updated = cudaGraphExecUpdate(ctx->gexec, g, &info) == cudaSuccess;
        if (!updated) {
          cudaGetLastError();
          cudaGraphExecDestroy(ctx->gexec);
          ctx->gexec = nullptr;
        }
      }
      cudaError_t e = updated ? cudaSuccess : cudaGraphInstantiate(&ctx->gexec, g, 0);
      cudaGraphDestroy(g);
      CKR(e);
      CKR(cudaGraphLaunch(ctx->gexec, st));
      ctx->times.graph_launches++;
    }
    if (exact_out) {
      if ((rc = read_counters(ctx))) return rc;
      const Counters hc = *ctx->hctr;
      // deferred bins can add at most one row per overflow k-mer, the overflow table as many
      out_cap = std::max<uint64_t>(1, hc.out_count + 2 * std::min<uint64_t>(hc.ovf_count, ovf_cap));
      CKR(cudaMemsetAsync(&ctx->ctr->out_count, 0, 8, st));
      CKR(cudaMemsetAsync(&ctx->ctr->distinct, 0, 8, st));
      if ((rc = alloc_res(out_cap))) return rc;
      xp.mode = 0;
      xp.out_keys = res->keys;
      xp.out_counts = res->counts;
      xp.out_cap = out_cap;
      ph_begin(ctx, PH_COMPACT);
      CKR(gerbil::launch_compact(k, xp, ctx->nsm, st));
      if (slots) ctx->times.kernel_launches++;
      ph_end(ctx, PH_COMPACT);
    }
#undef CKG
    if ((rc = read_counters(ctx))) { drop(); return rc; }
    Counters h = *ctx->hctr;
    if (h.err & gerbil::ERR_OVF_FULL) {
      // the emergency area ran full: repeat with the largest table estimate (every k-mer
      // distinct) and a long probe limit, which leaves almost nothing to the overflow area
      drop();
      ratio = 1.0;
      theta = std::max<uint32_t>(theta, 1024);
      stats.retries++;
      continue;
    }
    stats.overflowed = h.ovf_count;
    if (h.ovf_count) {
      // recount the overflow area in a fresh table, merge it into the deferred bins' keys and
      // emit the keys that exist only in the overflow table
      const uint64_t ocap64 = std::max<uint64_t>(64, 2 * h.ovf_count + 16);
      if (ocap64 >= 0xFFFFFFF0ull) { drop(); return fail(ctx, GERBIL_E_OVERFLOW, "overflow too large"); }
      const uint32_t ocap = (uint32_t)ocap64;
      void* otab = nullptr;
      const size_t obytes = (size_t)ocap * SWk * 8;
      if ((rc = dev_alloc(ctx, &otab, obytes))) { drop(); return rc; }
      CKR(cudaMemsetAsync(otab, 0, obytes, st));
      gerbil::OverflowParams op{};
      op.ovf = (unsigned long long*)ctx->ovf;
      op.ovf_cap = ovf_cap;
      op.otab = (unsigned long long*)otab;
      op.ocap = ocap;
      op.spin_limit = spin_limit;
      op.min_count = min_count;
      op.out_keys = res->keys;
      op.out_counts = res->counts;
      op.out_cap = out_cap;
      op.ctr = ctx->ctr;
      // the bins that spilled: only their tables are scanned again (merged with the recount)
      std::vector<uint32_t> hovf(work.size());
      CKR(cudaMemcpyAsync(hovf.data(), bin_ovf, work.size() * 4, cudaMemcpyDeviceToHost, st));
      CKR(cudaStreamSynchronize(st));
      std::vector<std::pair<size_t, size_t>> spans;  // [first, last] work indices
      for (size_t i = 0; i < work.size(); ++i) {
        if (!hovf[i]) continue;
        if (!spans.empty() && spans.back().second + 1 == i) spans.back().second = i;
        else spans.push_back({i, i});
      }
      while (spans.size() > 32) {  // join the two spans with the fewest slots between them
        size_t best = 0;
        uint64_t gap = ~0ull;
        for (size_t i = 0; i + 1 < spans.size(); ++i) {
          const uint64_t g = work[spans[i + 1].first].table_off -
                             (work[spans[i].second].table_off + work[spans[i].second].cap);
          if (g < gap) { gap = g; best = i; }
        }
        spans[best].second = spans[best + 1].second;
        spans.erase(spans.begin() + best + 1);
      }
      ph_begin(ctx, PH_OVERFLOW);
      CKR(gerbil::launch_overflow_insert(k, op, ctx->nsm, st));
      xp.mode = 1;
      xp.otab = op.otab;
      xp.ocap = ocap;
      for (const auto& sp : spans) {
        xp.slot_lo = work[sp.first].table_off;
        xp.slot_hi = work[sp.second].table_off + work[sp.second].cap;
        CKR(gerbil::launch_compact(k, xp, ctx->nsm, st));
      }
      CKR(gerbil::launch_overflow_emit(k, op, ctx->nsm, st));
      ctx->times.kernel_launches += 2 + spans.size();
      ph_end(ctx, PH_OVERFLOW);
      rc = read_counters(ctx);
      dev_free(ctx, otab, obytes);
      if (rc) { drop(); return rc; }
      h = *ctx->hctr;
      // distinct counted in mode 0 skipped deferred bins; add their main-table keys
      // (overflow emit counted the overflow-only ones)
    }
    if (h.err & gerbil::ERR_SPIN) { drop(); return fail(ctx, GERBIL_E_TIMEOUT, "bounded wait gave up"); }
    if ((h.err & gerbil::ERR_OUT_FULL) && !exact_out) {  // estimate too low: size exactly
      drop();
      exact_retry = true;
      continue;
    }
    if (h.err & (gerbil::ERR_STATE | gerbil::ERR_OUT_FULL)) {
      drop();
      return fail(ctx, GERBIL_E_STATE, "device consistency check failed");
    }
    stats.emitted = h.out_count;
    stats.distinct = h.distinct;
    stats.table_slots = slots;
    res->n = h.out_count;
    res->stats = stats;
    // every slot of this batch was zeroed by its compaction (mode 0 or, for the bins that
    // spilled, mode 1), and the rest of the arena was cleared before the inserts
    ctx->arena_dirty = 0;
    // the distinct count is exact after a spill too (deferred bins are counted by their merge,
    // overflow-only keys by the overflow emit), so a batch that spilled corrects the ratio
    if (occ > 0) {
      ctx->ratio = (double)h.distinct / (double)occ;
      ctx->ratio_known = true;
      ctx->emit_ratio = (double)h.out_count / (double)occ;
      ctx->emit_min_count = min_count;
      ctx->emit_known = true;
    }
    *out = res;
    return GERBIL_OK;
#undef CKR
  }
  return fail(ctx, GERBIL_E_OVERFLOW, "overflow area full after all retries");
}

static int count_checks(gerbil_ctx* ctx, const gerbil_bins* b, int k, uint32_t min_count,
                        const gerbil_opts& opts) {
  if (!b || b->ctx != ctx) return fail(ctx, GERBIL_E_INVAL, "bins from another context");
  if (k != b->k) return fail(ctx, GERBIL_E_INVAL, "k differs from the partition's k");
  if (min_count < 1) return fail(ctx, GERBIL_E_INVAL, "min_count must be >= 1");
  if (opts.canonical && !b->canon_min)
    return fail(ctx, GERBIL_E_INVAL, "canonical counting needs canonical minimizers");
  if (opts.probe_scheme != 0 && opts.probe_scheme != 1)
    return fail(ctx, GERBIL_E_INVAL, "probe_scheme must be 0 or 1");
  if (opts.claim_first < 0 || opts.claim_first > 2)
    return fail(ctx, GERBIL_E_INVAL, "claim_first must be 0, 1 or 2");
  if (opts.item_kmers != 0 && !valid_item_kmers(opts.item_kmers))
    return fail(ctx, GERBIL_E_INVAL, "item_kmers must be 0, 64, 128 or 256");
  if (opts.item_kmers != 0 && opts.item_kmers != (uint32_t)gerbil::ITEM_KMERS && words_for(k) > 4)
    return fail(ctx, GERBIL_E_UNSUPPORTED, "work items of 64 or 128 k-mers need k <= 128");
  return GERBIL_OK;
}

// ---- autotuner ---------------------------------------------------------------------------------
// Picks the phase-two form and schedule, then a load factor per table-size class, by timing
// candidates on a sample of the batch's bins (every 16th bin) with device events around the
// clears, inserts, compaction and overflow work.  Every candidate gives the same counts; only
// time differs.
static int tune_time(gerbil_ctx* ctx, const gerbil_bins* b, const std::vector<int32_t>& sample, int k,
                     uint32_t min_count, const gerbil_opts& o, double* ms_out) {
  double best = 1e30;
  for (int rep = 0; rep < 2; ++rep) {
    std::memset(&ctx->times, 0, sizeof(ctx->times));
    gerbil_counts* tmp = nullptr;
    const int rc = count_impl(ctx, b, sample, k, min_count, o, &tmp);
    if (rc) return rc;
    gerbil_counts_free(tmp);
    CK(cudaStreamSynchronize(ctx->stream));
    ph_collect(ctx, true);
    const gerbil_phase_times& t = ctx->times;
    best = std::min(best, t.clear_ms + t.insert_ms + t.compact_ms + t.overflow_ms);
  }
  *ms_out = best;
  return GERBIL_OK;
}

static int autotune_impl(gerbil_ctx* ctx, const gerbil_bins* b, const std::vector<int32_t>& list,
                         int k, uint32_t min_count, const gerbil_opts& opts_in, gerbil_tuning* out) {
  const int W = words_for(k);
  gerbil_opts o = opts_in;
  o.autotune = 0;
  o.fused = 0;
  o.schedule = 1;
  o.load_factor = 0.5f;
  o.probe_scheme = 0;
  o.item_kmers = 0;
  std::vector<int32_t> sample;
  const size_t step16 = std::max<size_t>(1, list.size() / 16);
  for (size_t i = 0; i < list.size(); i += step16) sample.push_back(list[i]);
  uint64_t occ = 0;
  for (int32_t bi : sample) occ += b->nkmers[bi];
  if (occ == 0) return fail(ctx, GERBIL_E_INVAL, "autotune: the sample holds no k-mers");

  // device timing for the duration of the tuning; the caller's profile is put back after
  const bool was_profiling = ctx->profiling;
  const gerbil_phase_times saved = ctx->times;
  CK(cudaStreamSynchronize(ctx->stream));
  ph_collect(ctx, true);
  ctx->profiling = true;
  int rc = GERBIL_OK;
  auto restore = [&]() {
    cudaStreamSynchronize(ctx->stream);
    ph_collect(ctx, true);
    ctx->profiling = was_profiling;
    ctx->times = saved;
  };
  {  // learn the distinct ratio on the sample first (Sec. 3.4)
    gerbil_counts* tmp = nullptr;
    if ((rc = count_impl(ctx, b, sample, k, min_count, o, &tmp))) { restore(); return rc; }
    gerbil_counts_free(tmp);
  }
  const double ratio = std::min(1.0, ctx->ratio_known ? ctx->ratio * 1.25 : 1.0);
  const Sizing z0 = make_sizing(ctx, o, k);
  // the sample: every 16th bin, or every 8th, 4th, 2nd, every bin, until its tables take four
  // times the L2 cache -- a sample whose tables all stay in L2 would time its compaction (and
  // its low load factors) far below what the whole batch sees
  {
    auto tables = [&](size_t st) {
      double bytes = 0;
      for (size_t i = 0; i < list.size(); i += st)
        if (b->nkmers[list[i]])
          bytes += (double)z0.cap(std::max(1.0, std::ceil(ratio * (double)b->nkmers[list[i]]))) *
                   (double)z0.slot_bytes;
      return bytes;
    };
    size_t st = step16;
    while (st > 1 && tables(st) < 4.0 * ctx->l2_bytes) st = std::max<size_t>(1, st / 2);
    sample.clear();
    for (size_t i = 0; i < list.size(); i += st) sample.push_back(list[i]);
  }
  occ = 0;
  for (int32_t bi : sample) occ += b->nkmers[bi];

  // the defaults: what a batch runs without tuning
  gerbil_tuning d{};
  for (int c = 0; c < GERBIL_TUNE_CLASSES; ++c) d.load_factor[c] = 0.5f;
  for (int c = 0; c < GERBIL_TUNE_CLASSES - 1; ++c) d.class_bytes[c] = kClassBound[c];
  d.fused = 0;
  d.schedule = 1;
  d.k_words = W;
  d.probe_scheme = 0;
  d.item_kmers = gerbil::ITEM_KMERS;
  gerbil_tuning t = d;
  // times phase two of `bins` with the candidate's settings (held as the context's tuning)
  o.autotune = 1;
  uint32_t nsamples = 0;
  auto timed = [&](const gerbil_tuning& cand, const std::vector<int32_t>& bins, double* ms) {
    ctx->tuning[W] = cand;
    nsamples++;
    return tune_time(ctx, b, bins, k, min_count, o, ms);
  };
  // a candidate replaces the best so far only when it is at least 2% faster on `bins`
  double best = 0;
  auto consider = [&](const gerbil_tuning& cand, const std::vector<int32_t>& bins, double* cur) -> int {
    double ms = 0;
    const int r = timed(cand, bins, &ms);
    if (r) return r;
    if (ms < 0.98 * *cur) {
      *cur = ms;
      t = cand;
    }
    return GERBIL_OK;
  };
#define TUNE_TRY(CAND, BINS, CUR)                                               \
  do {                                                                          \
    if ((rc = consider((CAND), (BINS), (CUR)))) {                               \
      ctx->tuning.erase(W);                                                     \
      restore();                                                                \
      return rc;                                                                \
    }                                                                           \
  } while (0)
  if ((rc = timed(t, sample, &best))) { ctx->tuning.erase(W); restore(); return rc; }
  // 1. form and schedule
  static const int forms[][2] = {{0, 0}, {1, 1}, {2, 1}};
  for (const auto& f : forms) {
    gerbil_tuning cand = t;
    cand.fused = f[0];
    cand.schedule = f[1];
    TUNE_TRY(cand, sample, &best);
  }
  // 2. probe scheme, then work-item size (built for keys of up to four words), whole sample
  {
    gerbil_tuning cand = t;
    cand.probe_scheme = 1;
    TUNE_TRY(cand, sample, &best);
  }
  if (W <= 4) {
    for (uint32_t ik : {128u, 64u}) {
      gerbil_tuning cand = t;
      cand.item_kmers = ik;
      TUNE_TRY(cand, sample, &best);
    }
  }
  // 3. the load factor of each table-size class, on the sample's bins of that class
  for (int c = 0; c < GERBIL_TUNE_CLASSES; ++c) {
    std::vector<int32_t> sub;
    uint64_t sub_occ = 0;
    for (int32_t bi : sample) {
      if (!b->nkmers[bi]) continue;
      if (z0.cls(std::max(1.0, std::ceil(ratio * (double)b->nkmers[bi]))) != c) continue;
      sub.push_back(bi);
      sub_occ += b->nkmers[bi];
    }
    if (sub.empty() || sub_occ < 100000) continue;  // too little to time: keep 0.5
    double cbest = 0;
    if ((rc = timed(t, sub, &cbest))) { ctx->tuning.erase(W); restore(); return rc; }
    for (float a : {0.35f, 0.65f, 0.8f}) {
      gerbil_tuning cand = t;
      cand.load_factor[c] = a;
      TUNE_TRY(cand, sub, &cbest);
    }
  }
#undef TUNE_TRY
  // 4. the whole batch, tuned settings against the defaults: the tuning is kept only if it is
  // faster there too (a sample can favour settings that the batch does not)
  {
    double mt = 0, md = 0;
    if ((rc = timed(t, list, &mt)) || (rc = timed(d, list, &md))) { ctx->tuning.erase(W); restore(); return rc; }
    if (!(mt < md)) t = d;
  }
  t.ns_per_kmer = best * 1e6 / (double)occ;
  t.samples = nsamples;
  restore();
  ctx->tuning[W] = t;
  if (out) *out = t;
  return GERBIL_OK;
}

int gerbil_autotune(gerbil_ctx* ctx, const gerbil_bins* b, int k, uint32_t min_count,
                    const gerbil_opts* opts_in, gerbil_tuning* out) {
  if (!ctx || !b) return GERBIL_E_INVAL;
  gerbil_opts opts;
  if (opts_in) opts = *opts_in; else gerbil_opts_default(&opts);
  int rc = count_checks(ctx, b, k, min_count, opts);
  if (rc) return rc;
  CK(cudaSetDevice(ctx->device));
  std::vector<int32_t> list;
  for (int i = 0; i < b->nbins; ++i) list.push_back(i);
  return autotune_impl(ctx, b, list, k, min_count, opts, out);
}

int gerbil_set_tuning(gerbil_ctx* ctx, int k, const gerbil_tuning* t) {
  if (!ctx || k < GERBIL_MIN_K || k > GERBIL_MAX_K) return GERBIL_E_INVAL;
  if (!t) {
    ctx->tuning.erase(words_for(k));
    return GERBIL_OK;
  }
  if (t->fused < 0 || t->fused > 2 || t->schedule < 0 || t->schedule > 1)
    return fail(ctx, GERBIL_E_INVAL, "tuning: form or schedule out of range");
  for (int c = 0; c < GERBIL_TUNE_CLASSES; ++c)
    if (!(t->load_factor[c] > 0.05f && t->load_factor[c] <= 0.95f))
      return fail(ctx, GERBIL_E_INVAL, "tuning: load factor out of range");
  if (t->probe_scheme != 0 && t->probe_scheme != 1)
    return fail(ctx, GERBIL_E_INVAL, "tuning: probe scheme out of range");
  if (!valid_item_kmers(t->item_kmers) || (t->item_kmers != (uint32_t)gerbil::ITEM_KMERS && words_for(k) > 4))
    return fail(ctx, GERBIL_E_INVAL, "tuning: item size out of range for this key width");
  gerbil_tuning c = *t;
  c.k_words = words_for(k);
  ctx->tuning[c.k_words] = c;
  return GERBIL_OK;
}

int gerbil_get_tuning(const gerbil_ctx* ctx, int k, gerbil_tuning* out) {
  if (!ctx || !out || k < GERBIL_MIN_K || k > GERBIL_MAX_K) return GERBIL_E_INVAL;
  auto it = ctx->tuning.find(words_for(k));
  if (it == ctx->tuning.end()) return GERBIL_E_STATE;
  *out = it->second;
  return GERBIL_OK;
}

static int join_parts(gerbil_counts* c);

// gerbil_opts.sorted_output: the rows in ascending key order (LSD radix sort over the 2k key
// bits, 8 bits per pass, sort.cu), in the result's own buffers.
static int sort_result(gerbil_ctx* ctx, gerbil_counts* c, int k) {
  int rc = join_parts(c);
  if (rc) return rc;
  const uint64_t n = c->n;
  if (n < 2) return GERBIL_OK;
  if (n >= (1ull << 32)) return fail(ctx, GERBIL_E_UNSUPPORTED, "sorted output of 2^32 rows or more");
  const int W = c->W;
  const int passes = (2 * k + 7) / 8;
  const uint64_t ntiles = gerbil::sort_tiles(n);
  unsigned long long* k2 = nullptr;
  uint32_t* c2 = nullptr;
  uint32_t* hist = nullptr;
  const size_t hbytes = (ntiles * 256 + 256) * 4;
  if ((rc = dev_alloc(ctx, (void**)&k2, n * W * 8))) return rc;
  if ((rc = dev_alloc(ctx, (void**)&c2, n * 4))) {
    dev_free(ctx, k2, n * W * 8);
    return rc;
  }
  if ((rc = dev_alloc(ctx, (void**)&hist, hbytes))) {
    dev_free(ctx, k2, n * W * 8);
    dev_free(ctx, c2, n * 4);
    return rc;
  }
  unsigned long long *ka = c->keys, *kb = k2;
  uint32_t *ca = c->counts, *cb = c2;
  cudaError_t e = cudaSuccess;
  for (int p = 0; p < passes && e == cudaSuccess; ++p) {
    e = gerbil::launch_sort_pass(ka, ca, kb, cb, n, W, p, hist, hist + ntiles * 256, ctx->stream);
    std::swap(ka, kb);
    std::swap(ca, cb);
    ctx->times.kernel_launches += 4;
  }
  dev_free(ctx, hist, hbytes);
  if (e != cudaSuccess) {
    dev_free(ctx, k2, n * W * 8);
    dev_free(ctx, c2, n * 4);
    return fail(ctx, GERBIL_E_CUDA, std::string("sort: ") + cudaGetErrorString(e));
  }
  if (ka == k2) {  // the sorted rows are in the new buffers: they become the result's
    const uint64_t cap = c->bytes / (W * 8 + 4);
    dev_free(ctx, c->keys, cap * W * 8);
    dev_free(ctx, c->counts, cap * 4);
    c->keys = k2;
    c->counts = c2;
    c->bytes = n * (W * 8 + 4);
  } else {
    dev_free(ctx, k2, n * W * 8);
    dev_free(ctx, c2, n * 4);
  }
  c->stats.sorted = 1;
  return GERBIL_OK;
}

// count_impl, then (sorted_output) the rows in ascending key order.
static int count_sorted(gerbil_ctx* ctx, const gerbil_bins* b, const std::vector<int32_t>& list,
                        int k, uint32_t min_count, const gerbil_opts& opts, gerbil_counts** out) {
  int rc = count_impl(ctx, b, list, k, min_count, opts, out);
  if (rc || !opts.sorted_output) return rc;
  if ((rc = sort_result(ctx, *out, k))) {
    gerbil_counts_free(*out);
    *out = nullptr;
  }
  return rc;
}

int gerbil_count(gerbil_ctx* ctx, const gerbil_bins* b, int bin, int k, uint32_t min_count,
                 const gerbil_opts* opts_in, gerbil_counts** out) {
  if (!ctx || !out) return GERBIL_E_INVAL;
  *out = nullptr;
  gerbil_opts opts;
  if (opts_in) opts = *opts_in; else gerbil_opts_default(&opts);
  int rc = count_checks(ctx, b, k, min_count, opts);
  if (rc) return rc;
  if (bin < 0 || bin >= b->nbins) return fail(ctx, GERBIL_E_INVAL, "bin out of range");
  CK(cudaSetDevice(ctx->device));
  std::vector<int32_t> list(1, bin);
  return count_sorted(ctx, b, list, k, min_count, opts, out);
}

int gerbil_count_batch(gerbil_ctx* ctx, const gerbil_bins* b, const int32_t* bin_list, int nb,
                       int k, uint32_t min_count, const gerbil_opts* opts_in,
                       gerbil_counts** out) {
  if (!ctx || !out) return GERBIL_E_INVAL;
  *out = nullptr;
  gerbil_opts opts;
  if (opts_in) opts = *opts_in; else gerbil_opts_default(&opts);
  int rc = count_checks(ctx, b, k, min_count, opts);
  if (rc) return rc;
  std::vector<int32_t> list;
  if (bin_list) {
    if (nb < 0) return fail(ctx, GERBIL_E_INVAL, "nb < 0");
    std::vector<char> seen(b->nbins, 0);
    for (int i = 0; i < nb; ++i) {
      const int32_t x = bin_list[i];
      if (x < 0 || x >= b->nbins || seen[x]) return fail(ctx, GERBIL_E_INVAL, "bad bin list");
      seen[x] = 1;
      list.push_back(x);
    }
  } else {
    for (int i = 0; i < b->nbins; ++i) list.push_back(i);
  }
  CK(cudaSetDevice(ctx->device));
  return count_sorted(ctx, b, list, k, min_count, opts, out);
}

// App. C records: per part (a joined result has several), count the long-count rows per tile,
// scan, read the total; then write every part at its byte offset.
int gerbil_encode_records(const gerbil_counts* c, int k, void* out, uint64_t cap, int out_on_device,
                          uint64_t* nbytes) {
  if (!c || !nbytes) return GERBIL_E_INVAL;
  *nbytes = 0;
  gerbil_ctx* ctx = c->ctx;
  if (k < GERBIL_MIN_K || k > GERBIL_MAX_K || words_for(k) != c->W)
    return fail(ctx, GERBIL_E_INVAL, "k does not match the result's key width");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  struct Part { const unsigned long long* keys; const uint32_t* counts; uint64_t n; };
  std::vector<Part> parts;
  if (!c->parts.empty()) {
    for (const gerbil_counts* p : c->parts) parts.push_back({p->keys, p->counts, p->n});
  } else {
    parts.push_back({c->keys, c->counts, c->n});
  }
  const uint64_t KB = (uint64_t)(k + 3) / 4;
  uint64_t maxt = 1;
  for (const Part& p : parts) maxt = std::max<uint64_t>(maxt, gerbil::encode_tiles(p.n));
  const size_t tbytes = (maxt + 1) * 8 * parts.size();
  unsigned long long* tl = nullptr;
  int rc;
  if ((rc = dev_alloc(ctx, (void**)&tl, tbytes))) return rc;
  std::vector<uint64_t> part_bytes(parts.size(), 0);
  std::vector<unsigned long long> totals(parts.size(), 0);
  uint64_t all = 0;
  auto cleanup = [&]() { dev_free(ctx, tl, tbytes); };
#define CKE(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      cleanup();                                                                           \
      return fail(ctx, GERBIL_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    }                                                                                      \
  } while (0)
  for (size_t i = 0; i < parts.size(); ++i) {
    if (!parts[i].n) continue;
    unsigned long long* t = tl + i * (maxt + 1);
    const uint64_t nt = gerbil::encode_tiles(parts[i].n);
    CKE(gerbil::launch_encode_count(parts[i].counts, parts[i].n, t, st));
    CKE(gerbil::launch_encode_scan(t, nt, t + maxt, st));
    ctx->times.kernel_launches += 2;
  }
  // One part written to host memory that has room for the longest records (every count 5
  // bytes): the records are written without waiting for their size; the n * (KB + 1) bytes
  // they take at least are copied back at once, and only the 4-byte extensions of counts of
  // 255 and more wait for the size (one synchronisation instead of two).
  if (out && !out_on_device && parts.size() == 1 && parts[0].n && cap >= parts[0].n * (KB + 5)) {
    const uint64_t lo = parts[0].n * (KB + 1), hi = parts[0].n * (KB + 5);
    uint8_t* stage = nullptr;
    if ((rc = dev_alloc(ctx, (void**)&stage, hi))) {
      cleanup();
      return rc;
    }
    gerbil::EncodeParams ep{};
    ep.keys = parts[0].keys;
    ep.counts = parts[0].counts;
    ep.n = parts[0].n;
    ep.k = k;
    ep.tile_long = tl;
    ep.out = stage;
    ep.base = 0;
    cudaError_t e = gerbil::launch_encode_write(ep, st);
    ctx->times.kernel_launches++;
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, stage, lo, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&totals[0], tl + maxt, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    const uint64_t nall = lo + 4 * (uint64_t)totals[0];
    if (e == cudaSuccess && nall > lo) {
      e = cudaMemcpyAsync((uint8_t*)out + lo, stage + lo, nall - lo, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    dev_free(ctx, stage, hi);
    CKE(e);
    *nbytes = nall;
    cleanup();
    return GERBIL_OK;
  }
  for (size_t i = 0; i < parts.size(); ++i)
    if (parts[i].n) CKE(cudaMemcpyAsync(&totals[i], tl + i * (maxt + 1) + maxt, 8, cudaMemcpyDeviceToHost, st));
  CKE(cudaStreamSynchronize(st));
  for (size_t i = 0; i < parts.size(); ++i) {
    part_bytes[i] = parts[i].n * (KB + 1) + 4 * totals[i];
    all += part_bytes[i];
  }
  *nbytes = all;
  if (!out) {
    cleanup();
    return GERBIL_OK;
  }
  if (cap < all) {
    cleanup();
    return fail(ctx, GERBIL_E_INVAL, "output buffer smaller than the records");
  }
  uint8_t* dst = (uint8_t*)out;
  uint8_t* stage = nullptr;
  if (!out_on_device && all) {
    if ((rc = dev_alloc(ctx, (void**)&stage, all))) {
      cleanup();
      return rc;
    }
    dst = stage;
  }
  uint64_t base = 0;
  for (size_t i = 0; i < parts.size(); ++i) {
    if (parts[i].n) {
      gerbil::EncodeParams ep{};
      ep.keys = parts[i].keys;
      ep.counts = parts[i].counts;
      ep.n = parts[i].n;
      ep.k = k;
      ep.tile_long = tl + i * (maxt + 1);
      ep.out = dst;
      ep.base = base;
      cudaError_t e = gerbil::launch_encode_write(ep, st);
      if (e != cudaSuccess) {
        dev_free(ctx, stage, all);
        CKE(e);
      }
      ctx->times.kernel_launches++;
    }
    base += part_bytes[i];
  }
  cudaError_t e = cudaSuccess;
  if (stage) e = cudaMemcpyAsync(out, stage, all, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  dev_free(ctx, stage, all);
  CKE(e);
#undef CKE
  cleanup();
  return GERBIL_OK;
}

int gerbil_counts_info(const gerbil_counts* c, uint64_t* n, int* words, gerbil_count_stats* s) {
  if (!c) return GERBIL_E_INVAL;
  if (n) *n = c->n;
  if (words) *words = c->W;
  if (s) *s = c->stats;
  return GERBIL_OK;
}

// Joins the groups' rows of a grouped result into one buffer (no-op for a plain result).
static int join_parts(gerbil_counts* c) {
  if (!c->parts.empty()) {
    gerbil_ctx* ctx = c->ctx;
    CK(cudaSetDevice(ctx->device));
    const int W = c->W;
    unsigned long long* k2 = nullptr;
    uint32_t* c2 = nullptr;
    if (c->n) {
      int rc;
      if ((rc = dev_alloc(ctx, (void**)&k2, c->n * W * 8))) return rc;
      if ((rc = dev_alloc(ctx, (void**)&c2, c->n * 4))) {
        dev_free(ctx, k2, c->n * W * 8);
        return rc;
      }
      uint64_t at = 0;
      for (gerbil_counts* p : c->parts) {
        if (p->n) {
          CK(cudaMemcpyAsync(k2 + at * W, p->keys, p->n * W * 8, cudaMemcpyDeviceToDevice, ctx->stream));
          CK(cudaMemcpyAsync(c2 + at, p->counts, p->n * 4, cudaMemcpyDeviceToDevice, ctx->stream));
        }
        at += p->n;
      }
      CK(cudaStreamSynchronize(ctx->stream));
    }
    for (gerbil_counts* p : c->parts) gerbil_counts_free(p);
    c->parts.clear();
    c->keys = k2;
    c->counts = c2;
    c->bytes = c->n * (W * 8 + 4);
  }
  return GERBIL_OK;
}

int gerbil_counts_view(const gerbil_counts* cc, uint64_t* n, int* words, const uint64_t** keys,
                       const uint32_t** counts) {
  if (!cc) return GERBIL_E_INVAL;
  if (n) *n = cc->n;
  if (words) *words = cc->W;
  gerbil_counts* c = const_cast<gerbil_counts*>(cc);
  if (!c->parts.empty()) {  // join the groups' rows into one buffer on first view
    const int rc = join_parts(c);
    if (rc) return rc;
  }
  if (keys) *keys = (const uint64_t*)c->keys;
  if (counts) *counts = c->counts;
  return GERBIL_OK;
}

int gerbil_counts_to_host(const gerbil_counts* c, uint64_t* keys, uint32_t* counts, uint64_t cap) {
  if (!c) return GERBIL_E_INVAL;
  gerbil_ctx* ctx = c->ctx;
  if (cap < c->n || (c->n && (!keys || !counts))) return fail(ctx, GERBIL_E_INVAL, "cap < n");
  if (c->n == 0) return GERBIL_OK;
  CK(cudaSetDevice(ctx->device));
  if (!c->parts.empty()) {
    uint64_t at = 0;
    for (const gerbil_counts* p : c->parts) {
      if (p->n) {
        CK(cudaMemcpyAsync(keys + at * c->W, p->keys, p->n * c->W * 8, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(counts + at, p->counts, p->n * 4, cudaMemcpyDeviceToHost, ctx->stream));
      }
      at += p->n;
    }
  } else {
    CK(cudaMemcpyAsync(keys, c->keys, c->n * c->W * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(counts, c->counts, c->n * 4, cudaMemcpyDeviceToHost, ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return GERBIL_OK;
}

void gerbil_counts_free(gerbil_counts* c) {
  if (!c) return;
  gerbil_ctx* ctx = c->ctx;
  for (gerbil_counts* p : c->parts) gerbil_counts_free(p);
  cudaSetDevice(ctx->device);
  const uint64_t cap = c->bytes / (c->W * 8 + 4);
  dev_free(ctx, c->keys, cap * c->W * 8);
  dev_free(ctx, c->counts, cap * 4);
  delete c;
}

}  // extern "C"
