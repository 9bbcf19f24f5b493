// server.cu -- counting jobs served continuously under an HBM budget (host runtime).
//
// The paper runs one job (one input) at a time.  A server here keeps `slots` worker contexts,
// each with its own CUDA stream and host thread; a submitted job waits in arrival order until
// a worker is free and its estimated device memory fits under the budget next to the jobs
// already running and the results not yet handed over (the first waiting job that fits is
// taken, so small jobs are not held up by a large one; a job passed over 4 x slots times
// blocks the admission of later ones until it fits).  Admitted jobs run concurrently on their
// own streams, so their kernels overlap on the GPU; each job's result stays on the device
// until the caller takes it.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/gerbil.h"
#include "kernels.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  uint64_t id = 0;
  std::vector<uint8_t> seq;       // host copy of the reads (when submitted from host memory)
  std::vector<uint64_t> offsets;
  const uint8_t* dseq = nullptr;  // or device pointers owned by the caller
  const uint64_t* doff = nullptr;
  uint64_t nreads = 0, nbases = 0;
  int k = 0, m = 0, nbins = 0;
  uint32_t min_count = 1;
  gerbil_opts opts{};
  std::vector<uint32_t> bounds;
  uint64_t est_bytes = 0;
  Clock::time_point arrival, start, done;
  int status = -1;  // -1 pending, -2 running, else gerbil_status
  gerbil_counts* result = nullptr;
  uint64_t result_bytes = 0;
  int worker = -1;
  int passed_over = 0;  // later jobs admitted while this one waited
  std::string error;    // the worker context's message when the job failed
};

}  // namespace

struct gerbil_server {
  int device = 0;
  uint64_t budget = 0;
  std::vector<gerbil_ctx*> ctx;
  std::vector<std::thread> threads;
  std::mutex mu;
  std::condition_variable cv;       // workers wait for admissible jobs
  std::condition_variable done_cv;  // callers wait for results
  std::deque<Job*> pending;
  std::map<uint64_t, Job*> jobs;
  uint64_t next_id = 1;
  uint64_t reserved = 0;  // estimated bytes of the running jobs
  uint64_t held = 0;      // bytes of finished results not yet handed over
  uint64_t table_cap = 0; // hash-table bytes one job may hold at once (0: no limit)
  std::map<int, double> ratio_of_k;  // largest distinct/occurrence ratio seen per k
  bool stop = false;
  gerbil_server_stats stats{};
  std::vector<uint64_t> running_per_worker;
  std::vector<uint64_t> launches_per_worker;  // kernel launches of each worker's context
  std::string last_error;  // message of the last failed job handed over by gerbil_server_wait
};


namespace {

// Device bytes a job needs at its peak: phase one (reads copied from the host, the 2-bit
// stream and masks, the super-mer record area, the bins' record arrays) or phase two (the
// 2-bit stream and record arrays, hash tables at the distinct ratio seen for this k -- every
// k-mer distinct when none was -- up to the server's table cap, the overflow area and the
// result rows), whichever is larger.
uint64_t estimate_bytes(const gerbil_server* s, const Job& j) {
  const int k = j.k, m = j.m;
  const double W = (2 * k + 63) / 64;
  const double slot = 8.0 * (double)gerbil::slot_words_for_k(k);
  const gerbil_opts& o = j.opts;
  const double alpha = (o.load_factor > 0.05f && o.load_factor <= 0.95f) ? o.load_factor : 0.5;
  double ratio = 1.0;
  if (o.distinct_ratio > 0.0f) {
    ratio = std::min(1.0, (double)o.distinct_ratio);
  } else {
    auto it = s->ratio_of_k.find(k);
    if (it != s->ratio_of_k.end()) ratio = std::min(1.0, it->second * 1.25);
  }
  const double n = (double)j.nbases, nr = (double)j.nreads;
  const double nwin = std::max(0.0, n - nr * (k - 1));
  const double w = (double)(k - m + 1);
  const double reads = j.dseq ? 0.0 : n + 8.0 * (nr + 1);
  const double stream = n / 4 + n / 4;  // 2-bit words and the two masks
  const double recs = (nwin * 4 / (w + 1) + 2 * nr + 65536) * 16;
  const double nsuper = nwin * 2 / (w + 1) + nr;
  const double arrays = nsuper * 12;
  double tables = nwin * ratio / alpha * slot + (double)j.nbins * 16 * slot;
  if (s->table_cap) tables = std::min(tables, (double)s->table_cap);
  const double ovf = std::max(65536.0, nwin / 32) * W * 8;
  const double rows = nwin * ratio * (8 * W + 4);
  const double phase1 = reads + stream + recs + arrays;
  const double phase2 = n / 4 + arrays + tables + ovf + rows;
  return (uint64_t)std::max(phase1, phase2) + (64ull << 20);
}

void run_job(gerbil_server* s, int w, Job* j) {
  gerbil_ctx* ctx = s->ctx[w];
  gerbil_reads r{};
  r.nreads = j->nreads;
  if (j->dseq) {
    r.seq = j->dseq;
    r.offsets = j->doff;
    r.on_device = 1;
  } else {
    r.seq = j->seq.data();
    r.offsets = j->offsets.data();
    r.on_device = 0;
  }
  gerbil_opts o = j->opts;
  if (!j->bounds.empty()) o.bin_bounds = j->bounds.data();
  if (!o.max_table_mib && s->table_cap) o.max_table_mib = (uint32_t)std::max<uint64_t>(1, s->table_cap >> 20);
  gerbil_forget_ratio(ctx);  // each job learns its own distinct ratio (Sec. 3.4)
  gerbil_bins* bins = nullptr;
  gerbil_counts* res = nullptr;
  int rc = gerbil_partition(ctx, &r, j->k, j->m, j->nbins, &o, &bins);
  if (rc == GERBIL_OK) rc = gerbil_count_batch(ctx, bins, nullptr, 0, j->k, j->min_count, &o, &res);
  if (bins) gerbil_bins_free(bins);
  gerbil_trim(ctx);  // give the context's cached scratch back to the pool for other jobs
  gerbil_phase_times pt{};
  gerbil_get_phase_times(ctx, &pt);  // this worker's context, read by its own thread
  const std::string err = rc != GERBIL_OK ? std::string(gerbil_strerror(rc)) + ": " + gerbil_last_error(ctx) : "";
  std::lock_guard<std::mutex> lock(s->mu);
  j->error = err;
  s->launches_per_worker[w] = pt.kernel_launches;
  j->status = rc;
  j->result = res;
  j->done = Clock::now();
  s->reserved -= std::min(s->reserved, j->est_bytes);
  s->running_per_worker[w] = 0;
  if (rc == GERBIL_OK) {
    gerbil_count_stats st{};
    uint64_t n = 0;
    int W = 1;
    gerbil_counts_info(res, &n, &W, &st);
    j->result_bytes = n * (8ull * W + 4);
    s->held += j->result_bytes;
    s->stats.completed++;
    s->stats.kmers += st.occurrences;
    if (st.occurrences) {
      double& r = s->ratio_of_k[j->k];
      r = std::max(r, (double)st.distinct / (double)st.occurrences);
    }
  } else {
    s->stats.failed++;
  }
  j->seq.clear();
  j->seq.shrink_to_fit();
  s->done_cv.notify_all();
  s->cv.notify_all();
}

void worker_loop(gerbil_server* s, int w) {
  cudaSetDevice(s->device);
  for (;;) {
    Job* j = nullptr;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      for (;;) {
        if (s->stop) return;
        // the first waiting job, in arrival order, that fits next to the running ones and
        // the held results; a job larger than the whole budget runs when nothing else does;
        // once the oldest job has been passed over 4 x slots times, only it may start
        const int max_pass = 4 * (int)s->ctx.size();
        for (auto it = s->pending.begin(); it != s->pending.end(); ++it) {
          const uint64_t busy = s->reserved + s->held;
          if (s->budget == 0 || (*it)->est_bytes + busy <= s->budget ||
              (s->reserved == 0 && (*it)->est_bytes > s->budget)) {
            j = *it;
            for (auto jt = s->pending.begin(); jt != it; ++jt) (*jt)->passed_over++;
            s->pending.erase(it);
            break;
          }
          if ((*it)->passed_over >= max_pass) break;
        }
        if (j) break;
        s->cv.wait(lock);
      }
      j->status = -2;
      j->worker = w;
      j->start = Clock::now();
      s->reserved += j->est_bytes;
      s->running_per_worker[w] = 1;
      uint32_t running = 0;
      for (uint64_t x : s->running_per_worker) running += (uint32_t)x;
      s->stats.max_concurrent = std::max(s->stats.max_concurrent, running);
    }
    run_job(s, w, j);
  }
}

}  // namespace

extern "C" {

int gerbil_server_create(gerbil_server** out, int device, uint64_t hbm_budget_bytes, int slots) {
  if (!out || slots < 1 || slots > 64) return GERBIL_E_INVAL;
  *out = nullptr;
  gerbil_server* s = new (std::nothrow) gerbil_server;
  if (!s) return GERBIL_E_NOMEM;
  s->device = device;
  s->budget = hbm_budget_bytes;
  // one job's hash tables take at most half of an equal share of the budget; a job whose
  // tables need more counts its bins in groups under that cap
  s->table_cap = hbm_budget_bytes ? hbm_budget_bytes / (2 * (uint64_t)slots) : 0;
  s->running_per_worker.assign(slots, 0);
  s->launches_per_worker.assign(slots, 0);
  for (int w = 0; w < slots; ++w) {
    gerbil_ctx* c = nullptr;
    const int rc = gerbil_create(&c, device, 0, nullptr);
    if (rc) {
      for (gerbil_ctx* x : s->ctx) gerbil_destroy(x);
      delete s;
      return rc;
    }
    s->ctx.push_back(c);
  }
  for (int w = 0; w < slots; ++w) s->threads.emplace_back(worker_loop, s, w);
  *out = s;
  return GERBIL_OK;
}

int gerbil_server_submit(gerbil_server* s, const gerbil_reads* reads, int k, int m, int nbins,
                         uint32_t min_count, const gerbil_opts* opts, uint64_t* job_id) {
  if (!s || !reads || !job_id) return GERBIL_E_INVAL;
  if (k < GERBIL_MIN_K || k > GERBIL_MAX_K || m < 1 || m >= k || m > 15 || nbins < 1 ||
      nbins > 65536 || min_count < 1)
    return GERBIL_E_INVAL;
  Job* j = new (std::nothrow) Job;
  if (!j) return GERBIL_E_NOMEM;
  j->arrival = Clock::now();
  j->nreads = reads->nreads;
  j->k = k;
  j->m = m;
  j->nbins = nbins;
  j->min_count = min_count;
  if (opts) j->opts = *opts; else gerbil_opts_default(&j->opts);
  if (j->opts.bin_bounds && nbins > 1) j->bounds.assign(j->opts.bin_bounds, j->opts.bin_bounds + nbins - 1);
  j->opts.bin_bounds = nullptr;
  if (reads->nreads > 0) {
    if (reads->on_device) {
      uint64_t last = 0;
      cudaSetDevice(s->device);
      if (cudaMemcpy(&last, reads->offsets + reads->nreads, 8, cudaMemcpyDeviceToHost) != cudaSuccess) {
        delete j;
        return GERBIL_E_CUDA;
      }
      j->nbases = last;
      j->dseq = reads->seq;
      j->doff = reads->offsets;
    } else {
      j->nbases = reads->offsets[reads->nreads];
      j->seq.assign(reads->seq, reads->seq + j->nbases);
      j->offsets.assign(reads->offsets, reads->offsets + reads->nreads + 1);
    }
  } else {
    j->offsets.assign(1, 0);
  }
  std::lock_guard<std::mutex> lock(s->mu);
  j->est_bytes = estimate_bytes(s, *j);
  j->id = s->next_id++;
  s->jobs[j->id] = j;
  s->pending.push_back(j);
  s->stats.submitted++;
  *job_id = j->id;
  s->cv.notify_all();
  return GERBIL_OK;
}

int gerbil_server_wait(gerbil_server* s, uint64_t job_id, int64_t timeout_ms, gerbil_counts** out,
                       gerbil_job_times* times) {
  if (!s || !out) return GERBIL_E_INVAL;
  *out = nullptr;
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return GERBIL_E_INVAL;
  Job* j = it->second;
  auto ready = [&] { return j->status >= 0; };
  if (timeout_ms < 0) {
    s->done_cv.wait(lock, ready);
  } else if (!s->done_cv.wait_for(lock, std::chrono::milliseconds(timeout_ms), ready)) {
    return GERBIL_E_TIMEOUT;
  }
  const int rc = j->status;
  *out = j->result;
  if (rc != GERBIL_OK) s->last_error = j->error;
  s->held -= std::min(s->held, j->result_bytes);  // the caller owns the result from here
  s->cv.notify_all();
  if (times) {
    auto ms = [](Clock::duration d) { return std::chrono::duration<double, std::milli>(d).count(); };
    times->queue_ms = ms(j->start - j->arrival);
    times->run_ms = ms(j->done - j->start);
    times->latency_ms = ms(j->done - j->arrival);
    times->worker = j->worker;
  }
  s->jobs.erase(it);
  delete j;
  return rc;
}

const char* gerbil_server_last_error(const gerbil_server* s) {
  return s ? s->last_error.c_str() : "";
}

int gerbil_server_get_stats(gerbil_server* s, gerbil_server_stats* out) {
  if (!s || !out) return GERBIL_E_INVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  *out = s->stats;
  out->kernel_launches = 0;
  for (uint64_t x : s->launches_per_worker) out->kernel_launches += x;
  return GERBIL_OK;
}

void gerbil_server_destroy(gerbil_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  for (std::thread& t : s->threads) t.join();
  for (auto& kv : s->jobs) {
    if (kv.second->result) gerbil_counts_free(kv.second->result);
    delete kv.second;
  }
  for (gerbil_ctx* c : s->ctx) gerbil_destroy(c);
  delete s;
}

}  // extern "C"
