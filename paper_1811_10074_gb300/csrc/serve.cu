// serve.cu -- a minimizer server with continuous batching (host code).
//
// Requests (one packed sequence each) are queued by sws_server_submit.  A dispatcher thread forms
// batches from the queue and runs each on a free slot: a slot owns a batch graph (batch.cu), a
// CUDA stream and pinned buffers, so several batches are on the device at once and a request that
// arrives while others run joins the next batch as soon as a slot is free.  Requests are admitted
// in arrival order while the device memory they need (their share of the slot's buffers) fits
// the server's HBM budget next to the requests already in flight.
//
// Host copies are what bounds a server, so each byte is copied once on the host:
// * a submitted sequence is copied straight into a pinned input arena (a ring); the requests of a
//   batch normally sit back to back there and go to the device in one copy;
// * a batch's picks come back from the device into a pinned result block, and the requests'
//   answers stay there: sws_server_collect hands out pointers into the block (many answers per
//   call) and sws_server_release gives the memory back; sws_server_result copies one answer out.
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
constexpr uint64_t NO_ARENA = ~0ull;

struct Request {
  uint64_t id = 0;
  uint64_t nbases = 0, nbytes = 0;
  uint64_t arena_off = NO_ARENA;  // its packed bases in the input arena ...
  std::vector<uint8_t> seq;       // ... or here, when the arena had no room
  Clock::time_point t_submit, t_done;
  int block = -1;                 // result block holding its picks
  uint64_t first = 0, count = 0;  // picks [first, first + count) of the block
  bool done = false, collected = false;
  int status = SWS_OK;
};

// Pinned memory of one batch's picks; free once every request that points into it is released.
struct Block {
  uint32_t *hash = nullptr, *pos = nullptr;
  uint64_t refs = 0;
  bool in_use = false;
};

struct Slot {
  sws_batch *bt = nullptr;
  sws_batch_io io{};
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  uint8_t *h_seq = nullptr;    // pinned staging for requests outside the arena
  int64_t *h_offs = nullptr;   // pinned
  uint64_t *h_po = nullptr;    // pinned
  uint64_t *h_count = nullptr; // pinned
  int block = -1;
  uint64_t copied = 0;         // picks copied back by the first read-back
  std::vector<Request *> members;
  uint64_t bytes = 0;          // device bytes charged to the admitted requests
  bool busy = false;
};

// A ring of pinned bytes handed out in FIFO order; a region can be freed in any order, and the
// ring's tail advances over the freed prefix.
struct Arena {
  uint8_t *base = nullptr;
  uint64_t size = 0, head = 0, used = 0;
  std::deque<std::pair<uint64_t, uint64_t>> live;  // (offset, bytes) in allocation order
  std::deque<bool> freed;
  // Offset of n contiguous bytes, or NO_ARENA.
  uint64_t alloc(uint64_t n) {
    if (n == 0 || n > size) return NO_ARENA;
    const uint64_t tail = live.empty() ? head : live.front().first;
    uint64_t off = NO_ARENA;
    if (live.empty()) {
      head = 0;
      off = 0;
    } else if (head >= tail) {  // free: [head, size) and [0, tail)
      if (size - head >= n) off = head;
      else if (tail >= n) off = 0;
    } else if (tail - head >= n) {  // free: [head, tail)
      off = head;
    }
    if (off == NO_ARENA) return NO_ARENA;
    live.emplace_back(off, n);
    freed.push_back(false);
    head = off + n;
    used += n;
    return off;
  }
  void release(uint64_t off) {
    for (size_t i = 0; i < live.size(); ++i)
      if (live[i].first == off && !freed[i]) {
        freed[i] = true;
        used -= live[i].second;
        break;
      }
    while (!live.empty() && freed.front()) {
      live.pop_front();
      freed.pop_front();
    }
  }
};

}  // namespace

struct sws_server {
  sws_ctx *ctx = nullptr;
  sws_server_config cfg{};
  std::vector<Slot> slots;
  std::vector<Block> blocks;
  Arena arena;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request *> pending;
  std::deque<Request *> completed;  // answered and not yet collected, in completion order
  std::unordered_map<uint64_t, Request *> reqs;
  uint64_t next_id = 1;
  uint64_t inflight_bytes = 0;
  bool stop = false;
  std::thread worker;
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

// Run f(0 .. m-1) on up to 8 threads (this one included) when there are at least `work` bytes to
// move, so that large submissions copy at memory speed.
template <class F>
void parallel_for(size_t m, uint64_t work, F f) {
  unsigned nt = std::thread::hardware_concurrency() / 2;
  nt = nt < 1 ? 1 : (nt > 8 ? 8 : nt);
  if (work < (1u << 20) || m < 2 || nt < 2) {
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

// A result block no batch or request uses (called with the lock held), or -1.
int free_block(sws_server *s) {
  for (size_t i = 0; i < s->blocks.size(); ++i)
    if (!s->blocks[i].in_use) return (int)i;
  return -1;
}

// Drop one request's hold on its result block (lock held).
void unref_block(sws_server *s, Request *r) {
  if (r->block < 0) return;
  Block &b = s->blocks[r->block];
  if (--b.refs == 0) {
    b.in_use = false;
    s->cv_work.notify_one();  // a slot may have been waiting for a block
  }
  r->block = -1;
}

void finish_slot(sws_server *s, Slot &sl) {
  // picks of every member: [po[2i], po[2i+1]) -- the odd entries are padding reads
  const uint64_t count = *sl.h_count;
  Block &blk = s->blocks[sl.block];
  if (count > sl.copied) {  // the first read-back was short: fetch the rest
    cudaMemcpyAsync(blk.hash + sl.copied, static_cast<uint32_t *>(sl.io.hash) + sl.copied,
                    (count - sl.copied) * 4, cudaMemcpyDeviceToHost, sl.stream);
    cudaMemcpyAsync(blk.pos + sl.copied, sl.io.pos + sl.copied, (count - sl.copied) * 4, cudaMemcpyDeviceToHost,
                    sl.stream);
    cudaStreamSynchronize(sl.stream);
  }
  const int st = sws_batch_sync(sl.bt);
  const Clock::time_point now = Clock::now();
  std::lock_guard<std::mutex> lock(s->mu);
  const size_t m = sl.members.size();
  blk.refs = m;
  for (size_t i = 0; i < m; ++i) {
    Request *r = sl.members[i];
    r->block = sl.block;
    r->first = sl.h_po[2 * i];
    r->count = sl.h_po[2 * i + 1] - sl.h_po[2 * i];
    r->status = st;
    r->done = true;
    r->t_done = now;
    if (r->arena_off != NO_ARENA) s->arena.release(r->arena_off);
    r->arena_off = NO_ARENA;
    r->seq.clear();
    r->seq.shrink_to_fit();
    s->completed.push_back(r);
    s->latencies.push_back(std::chrono::duration<double>(r->t_done - r->t_submit).count());
    s->bases_done += r->nbases;
  }
  if (m == 0) blk.in_use = false;
  s->inflight_bytes -= sl.bytes;
  s->t_last = now;
  sl.members.clear();
  sl.bytes = 0;
  sl.block = -1;
  sl.busy = false;
  s->cv_done.notify_all();
}

// Copy the members' bases to the device (runs of requests adjacent in the arena in one copy),
// launch the batch and the read-back into the slot's result block.
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
  for (size_t i = 0; i < m;) {
    Request *r = sl.members[i];
    const uint64_t dst = (uint64_t)sl.h_offs[2 * i] / 4;
    if (r->arena_off == NO_ARENA) {  // a request the arena had no room for: through the staging
      memcpy(sl.h_seq + dst, r->seq.data(), r->nbytes);
      cudaMemcpyAsync(sl.io.seq + dst, sl.h_seq + dst, r->nbytes, cudaMemcpyHostToDevice, sl.stream);
      ++i;
      continue;
    }
    uint64_t run = r->nbytes;
    size_t j = i + 1;
    while (j < m && sl.members[j]->arena_off != NO_ARENA && sl.members[j]->arena_off == r->arena_off + run) {
      run += sl.members[j]->nbytes;
      ++j;
    }
    cudaMemcpyAsync(sl.io.seq + dst, s->arena.base + r->arena_off, run, cudaMemcpyHostToDevice, sl.stream);
    i = j;
  }
  const uint64_t nreads = 2 * m;
  cudaMemcpyAsync(sl.io.offsets, sl.h_offs, (nreads + 1) * 8, cudaMemcpyHostToDevice, sl.stream);
  sws_batch_run(sl.bt, nreads, base, sl.stream);
  // read back the counts and a generous first share of the picks (about 2/(w+1) per base)
  Block &blk = s->blocks[sl.block];
  sl.copied = std::min<uint64_t>(sl.io.capacity, 3 * base / (uint64_t)(s->cfg.w + 1) + 4096);
  cudaMemcpyAsync(sl.h_count, sl.io.count, 8, cudaMemcpyDeviceToHost, sl.stream);
  cudaMemcpyAsync(sl.h_po, sl.io.pick_offsets, (nreads + 1) * 8, cudaMemcpyDeviceToHost, sl.stream);
  cudaMemcpyAsync(blk.hash, sl.io.hash, sl.copied * 4, cudaMemcpyDeviceToHost, sl.stream);
  cudaMemcpyAsync(blk.pos, sl.io.pos, sl.copied * 4, cudaMemcpyDeviceToHost, sl.stream);
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
    // admissions: fill every free slot that can get a result block from the queue
    for (Slot &sl : s->slots) {
      if (sl.busy) continue;
      {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->pending.empty()) break;
        const int b = free_block(s);
        if (b < 0) break;  // every block holds answers not yet released
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
        if (sl.members.empty()) break;
        sl.block = b;
        s->blocks[b].in_use = true;
        ++s->batches;
      }
      launch_slot(s, sl);
      sl.busy = true;
      progress = true;
    }
    std::unique_lock<std::mutex> lock(s->mu);
    bool any_busy = false;
    for (const Slot &sl : s->slots) any_busy |= sl.busy;
    // stop once nothing runs and nothing queued can start (every result block is held by answers
    // nobody released)
    if (s->stop && !any_busy && (s->pending.empty() || free_block(s) < 0)) break;
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

void free_all(sws_server *s) {
  for (Slot &sl : s->slots) {
    if (sl.bt) sws_batch_destroy(sl.bt);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.ev) cudaEventDestroy(sl.ev);
    for (void *p : {(void *)sl.h_seq, (void *)sl.h_offs, (void *)sl.h_po, (void *)sl.h_count})
      if (p) cudaFreeHost(p);
  }
  s->slots.clear();
  for (Block &b : s->blocks) {
    if (b.hash) cudaFreeHost(b.hash);
    if (b.pos) cudaFreeHost(b.pos);
  }
  s->blocks.clear();
  if (s->arena.base) cudaFreeHost(s->arena.base);
  s->arena.base = nullptr;
}

// Make a request for n bases (lock NOT held): its bytes go to the arena when `off` is valid, else
// to its own vector.
Request *make_request(sws_server *s, const uint8_t *packed, uint64_t nbases, uint64_t off) {
  Request *r = new Request();
  r->nbases = nbases;
  r->nbytes = (nbases + 3) / 4;
  r->arena_off = off;
  uint8_t *dst;
  if (off != NO_ARENA) {
    dst = s->arena.base + off;
  } else {
    r->seq.resize(r->nbytes);
    dst = r->seq.data();
  }
  if (r->nbytes) {
    memcpy(dst, packed, r->nbytes);
    if (nbases % 4) dst[r->nbytes - 1] &= (uint8_t)((1u << (2 * (nbases % 4))) - 1u);  // pad bits zero
  }
  return r;
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
  cudaError_t e = cudaSuccess;
  for (Slot &sl : s->slots) {
    st = sws_batch_create(ctx, maxr, maxb, cfg->k, cfg->w, cfg->mode, SWS_BATCH_DEFAULT, &sl.bt);
    if (st) break;
    sws_batch_io_get(sl.bt, &sl.io);
    e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.h_seq, maxb / 4 + 64);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.h_offs, (maxr + 1) * 8);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.h_po, (maxr + 1) * 8);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.h_count, 8);
    if (e != cudaSuccess) break;
  }
  // result blocks: one per slot in flight plus as many again for answers not yet released
  if (!st && e == cudaSuccess) {
    s->blocks.resize(2 * (size_t)cfg->slots + 2);
    const uint64_t cap = s->slots[0].io.capacity;
    for (Block &b : s->blocks) {
      e = cudaMallocHost((void **)&b.hash, cap * 4);
      if (e == cudaSuccess) e = cudaMallocHost((void **)&b.pos, cap * 4);
      if (e != cudaSuccess) break;
    }
  }
  // the input arena: room for every slot's batch eight times over (at least 64 MB), so that a
  // burst of submissions normally goes straight to pinned memory
  if (!st && e == cudaSuccess) {
    s->arena.size = std::max<uint64_t>(8 * (uint64_t)cfg->slots * (maxb / 4 + 64), 64ull << 20);
    e = cudaMallocHost((void **)&s->arena.base, s->arena.size);
  }
  if (!st && e != cudaSuccess) st = cuda_err(e, "server buffers");
  if (st) {
    free_all(s);
    delete s;
    return st;
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return SWS_OK;
}

sws_status sws_server_submit(sws_server *s, const uint8_t *packed, uint64_t nbases, uint64_t *request_id) {
  if (!s || !request_id) return sws::report_error(SWS_ERR_INVALID, "NULL argument");
  return sws_server_submit_batch(s, &packed, &nbases, 1, request_id);
}

sws_status sws_server_submit_batch(sws_server *s, const uint8_t *const *packed, const uint64_t *nbases, uint64_t count,
                                   uint64_t *request_ids) {
  if (!s || (count && (!packed || !nbases || !request_ids))) return sws::report_error(SWS_ERR_INVALID, "NULL argument");
  for (uint64_t i = 0; i < count; ++i) {
    if (nbases[i] && !packed[i]) return sws::report_error(SWS_ERR_INVALID, "NULL sequence");
    if (nbases[i] > s->cfg.max_bases_per_batch)
      return sws::report_error(SWS_ERR_CAPACITY, "request longer than max_bases_per_batch");
  }
  // room in the arena for each request (in order), then the copies outside the lock
  std::vector<uint64_t> off(count);
  uint64_t total = 0;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    for (uint64_t i = 0; i < count; ++i) {
      off[i] = s->arena.alloc((nbases[i] + 3) / 4);
      total += (nbases[i] + 3) / 4;
    }
  }
  std::vector<Request *> rs(count);
  parallel_for(count, total, [&](size_t i) { rs[i] = make_request(s, packed[i], nbases[i], off[i]); });
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
  Request *r = nullptr;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end()) return sws::report_error(SWS_ERR_INVALID, "unknown request id");
    r = it->second;
    if (!r->done) return sws::report_error(SWS_ERR_INVALID, "request not finished");
    *count = r->count;
    if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    if (r->count > capacity) return sws::report_error(SWS_ERR_CAPACITY, "result larger than capacity");
    if (r->count && (!hash || !pos)) return sws::report_error(SWS_ERR_INVALID, "NULL output");
    s->reqs.erase(it);  // this call owns the request now; its block stays held until the copy
    if (!r->collected) {
      auto c = std::find(s->completed.begin(), s->completed.end(), r);
      if (c != s->completed.end()) s->completed.erase(c);
      r->collected = true;
    }
  }
  if (r->count) {
    const Block &b = s->blocks[r->block];
    memcpy(hash, b.hash + r->first, r->count * 4);
    memcpy(pos, b.pos + r->first, r->count * 4);
  }
  const int st = r->status;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    unref_block(s, r);
  }
  delete r;
  return st == SWS_OK ? SWS_OK : sws::report_error(st, "a device-side wait ran out while serving this request");
}

sws_status sws_server_collect(sws_server *s, uint64_t max_n, double timeout_s, uint64_t *ids, uint64_t *counts,
                              const uint32_t **hash, const uint32_t **pos, double *latency_s, uint64_t *n_out) {
  if (!s || !n_out || (max_n && (!ids || !counts || !hash || !pos)))
    return sws::report_error(SWS_ERR_INVALID, "NULL argument");
  *n_out = 0;
  std::unique_lock<std::mutex> lock(s->mu);
  auto ready = [&] { return !s->completed.empty(); };
  if (!ready() && timeout_s > 0) s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), ready);
  uint64_t n = 0;
  int status = SWS_OK;
  while (n < max_n && ready()) {
    Request *r = s->completed.front();
    s->completed.pop_front();
    r->collected = true;
    const Block &b = s->blocks[r->block];
    ids[n] = r->id;
    counts[n] = r->count;
    hash[n] = b.hash + r->first;
    pos[n] = b.pos + r->first;
    if (latency_s) latency_s[n] = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    if (r->status != SWS_OK) status = r->status;
    ++n;
  }
  *n_out = n;
  return status == SWS_OK ? SWS_OK
                          : sws::report_error(status, "a device-side wait ran out while serving a collected request");
}

sws_status sws_server_release(sws_server *s, const uint64_t *ids, uint64_t n) {
  if (!s || (n && !ids)) return sws::report_error(SWS_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  sws_status st = SWS_OK;
  for (uint64_t i = 0; i < n; ++i) {
    auto it = s->reqs.find(ids[i]);
    if (it == s->reqs.end() || !it->second->done) {
      st = sws::report_error(SWS_ERR_INVALID, "release of an unknown or unfinished request");
      continue;
    }
    Request *r = it->second;
    s->reqs.erase(it);
    if (!r->collected) {  // released without being collected
      auto c = std::find(s->completed.begin(), s->completed.end(), r);
      if (c != s->completed.end()) s->completed.erase(c);
    }
    unref_block(s, r);
    delete r;
  }
  return st;
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
  free_all(s);
  for (auto &kv : s->reqs) delete kv.second;
  delete s;
  return SWS_OK;
}

}  // extern "C"
