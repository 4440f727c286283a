// serve.cu -- a minimizer server with continuous batching (host code).
//
// Requests (one packed sequence each) are queued by sws_server_submit.  A dispatcher thread forms
// batches from the queue and runs each on a free slot: a slot owns a batch graph (batch.cu), a
// CUDA stream and pinned staging buffers, so several batches are on the device at once and a
// request that arrives while others run joins the next batch as soon as a slot is free.  Requests
// are admitted in arrival order while the device memory they need (their share of the slot's
// buffers) fits the server's HBM budget next to the requests already in flight.
//
// Layout of a batch: request i occupies bases [s_i, s_i + L_i) of the slot's packed stream, s_i a
// multiple of 4 so that its bytes can be copied as they are; the 0..3 bases up to the next
// request's start form a padding "read" too short to hold a window.  Positions are read-local,
// so every request gets exactly the picks it would get alone.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/sws.h"
#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id = 0;
  std::vector<uint8_t> seq;  // packed bases
  uint64_t nbases = 0;
  Clock::time_point t_submit, t_done;
  std::vector<uint32_t> hash, pos;
  bool done = false;
  int status = SWS_OK;
};

struct Slot {
  sws_batch *bt = nullptr;
  sws_batch_io io{};
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  uint8_t *h_seq = nullptr;       // pinned
  int64_t *h_offs = nullptr;      // pinned
  uint32_t *h_hash = nullptr;     // pinned
  uint32_t *h_pos = nullptr;      // pinned
  uint64_t *h_po = nullptr;       // pinned
  uint64_t *h_count = nullptr;    // pinned
  uint64_t copied = 0;            // picks copied back by the first read-back
  std::vector<Request *> members;
  uint64_t bytes = 0;             // device bytes charged to the admitted requests
  bool busy = false;
};

}  // namespace

struct sws_server {
  sws_ctx *ctx = nullptr;
  sws_server_config cfg{};
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request *> pending;
  std::unordered_map<uint64_t, Request *> reqs;
  uint64_t next_id = 1;
  uint64_t inflight_bytes = 0;
  bool stop = false;
  std::thread worker;
  // result buffers of retrieved requests, reused (already faulted in) for later results
  std::vector<std::vector<uint32_t>> free_bufs;
  // statistics
  std::vector<double> latencies;
  uint64_t bases_done = 0, batches = 0;
  Clock::time_point t_first, t_last;
  bool any = false;
};

namespace {

uint64_t rup(uint64_t v, uint64_t a) { return (v + a - 1) / a * a; }

// Device bytes a request of n bases occupies in a slot (input, staging and output shares).
uint64_t request_bytes(uint64_t n) { return n / 4 + 24 * n + 64; }

// Run f(0 .. m-1) on up to 8 threads (this one included) when the batch moves enough data
// (`work` elements) for the threads to pay off; the host copies are what bounds a server.
template <class F>
void parallel_for(size_t m, uint64_t work, F f) {
  unsigned nt = std::thread::hardware_concurrency() / 2;
  nt = nt < 1 ? 1 : (nt > 8 ? 8 : nt);
  if (work < (1u << 18) || m < 2 || nt < 2) {
    for (size_t i = 0; i < m; ++i) f(i);
    return;
  }
  if (nt > m) nt = (unsigned)m;
  std::vector<std::thread> th;
  for (unsigned t = 1; t < nt; ++t)
    th.emplace_back([&, t] {
      for (size_t i = t; i < m; i += nt) f(i);
    });
  for (size_t i = 0; i < m; i += nt) f(i);
  for (auto &x : th) x.join();
}

void finish_slot(sws_server *s, Slot &sl) {
  // picks of every member: [po[2i], po[2i+1]) -- the odd entries are padding reads
  const uint64_t count = *sl.h_count;
  if (count > sl.copied) {  // the first read-back was short: fetch the rest
    cudaMemcpyAsync(sl.h_hash + sl.copied, static_cast<uint32_t *>(sl.io.hash) + sl.copied,
                    (count - sl.copied) * 4, cudaMemcpyDeviceToHost, sl.stream);
    cudaMemcpyAsync(sl.h_pos + sl.copied, sl.io.pos + sl.copied, (count - sl.copied) * 4, cudaMemcpyDeviceToHost,
                    sl.stream);
    cudaStreamSynchronize(sl.stream);
  }
  const int st = sws_batch_sync(sl.bt);
  const Clock::time_point now = Clock::now();
  const size_t m = sl.members.size();
  // result buffers: reused ones from the pool (short lock), filled without the lock so that
  // submissions and retrievals proceed meanwhile, then handed to the requests
  std::vector<std::vector<uint32_t>> bufs(2 * m);
  {
    std::lock_guard<std::mutex> lock(s->mu);
    for (size_t j = 0; j < 2 * m && !s->free_bufs.empty(); ++j) {
      bufs[j].swap(s->free_bufs.back());
      s->free_bufs.pop_back();
    }
  }
  parallel_for(m, sl.h_po[2 * m], [&](size_t i) {
    const uint64_t a = sl.h_po[2 * i], b = sl.h_po[2 * i + 1];
    bufs[2 * i].assign(sl.h_hash + a, sl.h_hash + b);
    bufs[2 * i + 1].assign(sl.h_pos + a, sl.h_pos + b);
  });
  std::lock_guard<std::mutex> lock(s->mu);
  for (size_t i = 0; i < m; ++i) {
    Request *r = sl.members[i];
    r->hash.swap(bufs[2 * i]);
    r->pos.swap(bufs[2 * i + 1]);
    r->status = st;
    r->done = true;
    r->t_done = now;
    r->seq.clear();
    r->seq.shrink_to_fit();
    s->latencies.push_back(std::chrono::duration<double>(r->t_done - r->t_submit).count());
    s->bases_done += r->nbases;
  }
  s->inflight_bytes -= sl.bytes;
  s->t_last = now;
  sl.members.clear();
  sl.bytes = 0;
  sl.busy = false;
  s->cv_done.notify_all();
}

// Copy the members' bases into the slot, launch the batch and the read-back.
void launch_slot(sws_server *s, Slot &sl) {
  uint64_t base = 0;
  const size_t m = sl.members.size();
  for (size_t i = 0; i < m; ++i) {
    Request *r = sl.members[i];
    sl.h_offs[2 * i] = (int64_t)base;
    sl.h_offs[2 * i + 1] = (int64_t)(base + r->nbases);
    base = rup(base + r->nbases, 4);
  }
  sl.h_offs[2 * m] = (int64_t)base;
  parallel_for(m, base / 4, [&](size_t i) {
    const Request *r = sl.members[i];
    memcpy(sl.h_seq + sl.h_offs[2 * i] / 4, r->seq.data(), r->seq.size());
  });
  const uint64_t nreads = 2 * m;
  cudaMemcpyAsync(sl.io.seq, sl.h_seq, base / 4, cudaMemcpyHostToDevice, sl.stream);
  cudaMemcpyAsync(sl.io.offsets, sl.h_offs, (nreads + 1) * 8, cudaMemcpyHostToDevice, sl.stream);
  sws_batch_run(sl.bt, nreads, base, sl.stream);
  // read back the counts and a generous first share of the picks (about 2/(w+1) per base)
  sl.copied = std::min<uint64_t>(sl.io.capacity, 3 * base / (uint64_t)(s->cfg.w + 1) + 4096);
  cudaMemcpyAsync(sl.h_count, sl.io.count, 8, cudaMemcpyDeviceToHost, sl.stream);
  cudaMemcpyAsync(sl.h_po, sl.io.pick_offsets, (nreads + 1) * 8, cudaMemcpyDeviceToHost, sl.stream);
  cudaMemcpyAsync(sl.h_hash, sl.io.hash, sl.copied * 4, cudaMemcpyDeviceToHost, sl.stream);
  cudaMemcpyAsync(sl.h_pos, sl.io.pos, sl.copied * 4, cudaMemcpyDeviceToHost, sl.stream);
  cudaEventRecord(sl.ev, sl.stream);
}

void worker_loop(sws_server *s) {
  cudaSetDevice(s->ctx->device);
  while (true) {
    bool progress = false;
    // completions
    for (Slot &sl : s->slots) {
      if (sl.busy && cudaEventQuery(sl.ev) == cudaSuccess) {
        finish_slot(s, sl);
        progress = true;
      }
    }
    // admissions: fill every free slot from the queue
    for (Slot &sl : s->slots) {
      if (sl.busy) continue;
      {
        std::lock_guard<std::mutex> lock(s->mu);
        uint64_t bases = 0;
        while (!s->pending.empty()) {
          Request *r = s->pending.front();
          const uint64_t need = rup(bases, 4) + r->nbases;
          const uint64_t bytes = request_bytes(r->nbases);
          if (sl.members.size() + 1 > s->cfg.max_requests_per_batch || need > s->cfg.max_bases_per_batch) break;
          if (s->inflight_bytes + bytes > s->cfg.hbm_budget_bytes && s->inflight_bytes > 0) break;
          s->pending.pop_front();
          sl.members.push_back(r);
          sl.bytes += bytes;
          s->inflight_bytes += bytes;
          bases = need;
        }
      }
      if (!sl.members.empty()) {
        launch_slot(s, sl);
        sl.busy = true;
        progress = true;
        std::lock_guard<std::mutex> lock(s->mu);
        ++s->batches;
      }
    }
    std::unique_lock<std::mutex> lock(s->mu);
    bool any_busy = false;
    for (const Slot &sl : s->slots) any_busy |= sl.busy;
    if (s->stop && !any_busy && s->pending.empty()) break;
    if (!progress) {
      if (any_busy) {
        lock.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
      } else {
        s->cv_work.wait_for(lock, std::chrono::milliseconds(5));
      }
    }
  }
}

sws_status cuda_err(cudaError_t e, const char *what) {
  char msg[256];
  snprintf(msg, sizeof(msg), "%s: %s", what, cudaGetErrorString(e));
  return sws::report_error(SWS_ERR_CUDA, msg);
}

void free_slots(sws_server *s) {
  for (Slot &sl : s->slots) {
    if (sl.bt) sws_batch_destroy(sl.bt);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.ev) cudaEventDestroy(sl.ev);
    for (void *p : {(void *)sl.h_seq, (void *)sl.h_offs, (void *)sl.h_hash, (void *)sl.h_pos, (void *)sl.h_po,
                    (void *)sl.h_count})
      if (p) cudaFreeHost(p);
  }
  s->slots.clear();
}

}  // namespace

extern "C" {

sws_status sws_server_create(sws_ctx *ctx, const sws_server_config *cfg, sws_server **out) {
  if (!out || !cfg || !ctx) return sws::report_error(SWS_ERR_INVALID, "NULL argument");
  *out = nullptr;
  sws_status st = sws::check_minimizer_args(cfg->k, cfg->w, cfg->mode);
  if (st) return st;
  if (2 * cfg->k > 32) return sws::report_error(SWS_ERR_UNSUPPORTED, "the server returns 32-bit keys: k <= 16");
  if (cfg->slots < 1 || cfg->max_requests_per_batch < 1 || cfg->max_bases_per_batch < 64)
    return sws::report_error(SWS_ERR_INVALID, "slots, max_requests_per_batch >= 1 and max_bases_per_batch >= 64");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return sws::report_error(SWS_ERR_CUDA, "cudaSetDevice");
  sws_server *s = new sws_server();
  s->ctx = ctx;
  s->cfg = *cfg;
  if (s->cfg.hbm_budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    s->cfg.hbm_budget_bytes = fr / 2;
  }
  const uint64_t maxb = cfg->max_bases_per_batch, maxr = 2 * cfg->max_requests_per_batch;
  s->slots.resize(cfg->slots);
  for (Slot &sl : s->slots) {
    st = sws_batch_create(ctx, maxr, maxb, cfg->k, cfg->w, cfg->mode, SWS_BATCH_DEFAULT, &sl.bt);
    if (st) break;
    sws_batch_io_get(sl.bt, &sl.io);
    cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.h_seq, maxb / 4 + 64);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.h_offs, (maxr + 1) * 8);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.h_hash, sl.io.capacity * 4);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.h_pos, sl.io.capacity * 4);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.h_po, (maxr + 1) * 8);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.h_count, 8);
    if (e != cudaSuccess) {
      st = cuda_err(e, "server slot");
      break;
    }
  }
  if (st) {
    free_slots(s);
    delete s;
    return st;
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return SWS_OK;
}

sws_status sws_server_submit(sws_server *s, const uint8_t *packed, uint64_t nbases, uint64_t *request_id) {
  if (!s || !request_id || (nbases && !packed)) return sws::report_error(SWS_ERR_INVALID, "NULL argument");
  if (nbases > s->cfg.max_bases_per_batch)
    return sws::report_error(SWS_ERR_CAPACITY, "request longer than max_bases_per_batch");
  Request *r = new Request();
  r->seq.assign(packed, packed + (nbases + 3) / 4);
  if (nbases % 4) r->seq.back() &= (uint8_t)((1u << (2 * (nbases % 4))) - 1u);  // pad bits zero
  r->nbases = nbases;
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    r->id = s->next_id++;
    if (!s->any) {
      s->t_first = r->t_submit;
      s->any = true;
    }
    s->reqs[r->id] = r;
    s->pending.push_back(r);
    *request_id = r->id;
  }
  s->cv_work.notify_one();
  return SWS_OK;
}

sws_status sws_server_submit_batch(sws_server *s, const uint8_t *const *packed, const uint64_t *nbases, uint64_t count,
                                   uint64_t *request_ids) {
  if (!s || (count && (!packed || !nbases || !request_ids))) return sws::report_error(SWS_ERR_INVALID, "NULL argument");
  for (uint64_t i = 0; i < count; ++i) {
    if (nbases[i] && !packed[i]) return sws::report_error(SWS_ERR_INVALID, "NULL sequence");
    if (nbases[i] > s->cfg.max_bases_per_batch)
      return sws::report_error(SWS_ERR_CAPACITY, "request longer than max_bases_per_batch");
  }
  std::vector<Request *> rs(count);
  for (uint64_t i = 0; i < count; ++i) {  // copies outside the lock
    Request *r = new Request();
    r->seq.assign(packed[i], packed[i] + (nbases[i] + 3) / 4);
    if (nbases[i] % 4) r->seq.back() &= (uint8_t)((1u << (2 * (nbases[i] % 4))) - 1u);
    r->nbases = nbases[i];
    rs[i] = r;
  }
  const Clock::time_point now = Clock::now();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (!s->any && count) {
      s->t_first = now;
      s->any = true;
    }
    for (uint64_t i = 0; i < count; ++i) {
      Request *r = rs[i];
      r->t_submit = now;
      r->id = s->next_id++;
      s->reqs[r->id] = r;
      s->pending.push_back(r);
      request_ids[i] = r->id;
    }
  }
  s->cv_work.notify_one();
  return SWS_OK;
}

sws_status sws_server_wait(sws_server *s, uint64_t request_id, double timeout_s, int *done) {
  if (!s || !done) return sws::report_error(SWS_ERR_INVALID, "NULL argument");
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end()) return sws::report_error(SWS_ERR_INVALID, "unknown request id");
  Request *r = it->second;
  if (!r->done && timeout_s > 0)
    s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), [&] { return r->done; });
  *done = r->done ? 1 : 0;
  return SWS_OK;
}

sws_status sws_server_result(sws_server *s, uint64_t request_id, uint32_t *hash, uint32_t *pos, uint64_t capacity,
                             uint64_t *count, double *latency_s) {
  if (!s || !count) return sws::report_error(SWS_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end()) return sws::report_error(SWS_ERR_INVALID, "unknown request id");
  Request *r = it->second;
  if (!r->done) return sws::report_error(SWS_ERR_INVALID, "request not finished");
  *count = r->hash.size();
  if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
  if (r->hash.size() > capacity) return sws::report_error(SWS_ERR_CAPACITY, "result larger than capacity");
  if (!r->hash.empty()) {
    if (!hash || !pos) return sws::report_error(SWS_ERR_INVALID, "NULL output");
    memcpy(hash, r->hash.data(), r->hash.size() * 4);
    memcpy(pos, r->pos.data(), r->pos.size() * 4);
  }
  const int st = r->status;
  s->reqs.erase(it);
  if (s->free_bufs.size() < 8192) {  // keep the buffers for later results
    r->hash.clear();
    r->pos.clear();
    s->free_bufs.push_back(std::move(r->hash));
    s->free_bufs.push_back(std::move(r->pos));
  }
  delete r;
  return st == SWS_OK ? SWS_OK : sws::report_error(st, "a device-side wait ran out while serving this request");
}

sws_status sws_server_stats(sws_server *s, sws_server_statistics *out) {
  if (!s || !out) return sws::report_error(SWS_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  memset(out, 0, sizeof(*out));
  std::vector<double> l = s->latencies;
  std::sort(l.begin(), l.end());
  out->completed = l.size();
  out->batches = s->batches;
  out->bases = s->bases_done;
  out->pending = s->pending.size();
  if (!l.empty()) {
    out->p50_s = l[(size_t)(0.50 * (l.size() - 1))];
    out->p99_s = l[(size_t)(0.99 * (l.size() - 1))];
    out->max_s = l.back();
    double sum = 0;
    for (double v : l) sum += v;
    out->mean_s = sum / l.size();
  }
  if (s->any) out->span_s = std::chrono::duration<double>(s->t_last - s->t_first).count();
  return SWS_OK;
}

sws_status sws_server_reset_stats(sws_server *s) {
  if (!s) return sws::report_error(SWS_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  s->latencies.clear();
  s->bases_done = 0;
  s->batches = 0;
  s->any = false;
  return SWS_OK;
}

sws_status sws_server_destroy(sws_server *s) {
  if (!s) return SWS_OK;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->ctx->device);
  free_slots(s);
  for (auto &kv : s->reqs) delete kv.second;
  delete s;
  return SWS_OK;
}

}  // extern "C"
