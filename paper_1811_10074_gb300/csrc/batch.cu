// batch.cu -- batched minimizers: many reads of uneven length, stored back to back, processed by
// one persistent launch (Sec. 2.4 applied to every read), with the whole pipeline -- descriptor
// upload, memsets, the tile-barrier pre-pass, the minimizer kernel(s), the scan, the gather and
// the pick-offset fix-up -- captured once in a CUDA graph and replayed for every batch.
//
// A graph's launch arguments are fixed, so the kernels are launched for the largest batch the
// object was created for and read the actual sizes (reads, bases, windows, tiles) from a small
// device descriptor that the graph's first node copies from pinned host memory.  The algorithm is
// the single-pass kernel (hashed k-mers, k <= 16, 4 <= w <= 17), else the staged kernel
// specialized on w; on request every applicable graph, the single-kernel look-back path included,
// is timed on a synthetic batch of the largest size when the object is made and the fastest kept.
#include <cstdio>
#include <cstring>

#include "../../include/sws.h"
#include "internal.h"

struct sws_batch {
  sws_ctx *ctx = nullptr;
  int device = 0;
  uint64_t max_reads = 0, max_bases = 0, capacity = 0;
  int k = 0, w = 0, mode = 0;
  int hash_bytes = 4;
  // caller-visible device buffers
  uint8_t *seq = nullptr;
  int64_t *offsets = nullptr;
  void *hash = nullptr;
  uint32_t *pos = nullptr;
  uint64_t *pick_offsets = nullptr;
  uint64_t *count = nullptr;
  // private device state
  unsigned long long *d_desc = nullptr;
  unsigned long long *h_desc = nullptr;  // pinned
  void *ws = nullptr;
  uint64_t ws_bytes = 0;
  int *d_err = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec[3] = {nullptr, nullptr, nullptr};  // per path
  int path = -1;                                  // sws::BatchPath
  float tuned_ms[3] = {-1.f, -1.f, -1.f};
  cudaEvent_t done = nullptr;
  bool launched = false;
};

namespace {

enum BatchPath { PATH_STAGED = 0, PATH_LOOKBACK = 1, PATH_SINGLE = 2 };

uint64_t rup(uint64_t v, uint64_t a) { return (v + a - 1) / a * a; }

sws_status err_cuda(cudaError_t e, const char *what) {
  char msg[256];
  snprintf(msg, sizeof(msg), "%s: %s", what, cudaGetErrorString(e));
  return sws::report_error(SWS_ERR_CUDA, msg);
}

#define BT_CUDA(expr)                                 \
  do {                                                \
    cudaError_t e_ = (expr);                          \
    if (e_ != cudaSuccess) return err_cuda(e_, #expr); \
  } while (0)

// Workspace layouts of both paths for the largest batch, overlaid in one buffer.
struct Layout {
  uint64_t tiles, bytes;
  // staged
  uint64_t counts, scan, tilebar, shash, spos, sfirst, fix;
  // look-back
  uint64_t status, counter, ltilebar, lfix;
  // single pass
  uint64_t sfix;
};

Layout layout_for(const sws_batch *b, int path) {
  Layout L{};
  const uint64_t span = (uint64_t)(b->w + b->k - 1);
  const uint64_t nwin = b->max_bases >= span ? b->max_bases - span + 1 : 0;
  const uint64_t fixb = ((b->max_reads + 1023) / 1024 + 1) * 8;
  if (path == PATH_SINGLE) {
    const uint64_t tw = (uint64_t)sws::dna_min_tile_windows();
    L.tiles = (nwin + tw - 1) / tw;
    L.sfix = rup(sws::dna_min_ws_bytes(b->max_bases, b->k, b->w), 256);
    L.bytes = L.sfix + rup(fixb, 256);
  } else if (path == PATH_STAGED) {
    const uint64_t tw = (uint64_t)sws::mini_staged_tile_windows(sws::SRC_DNA, b->k, b->w);
    L.tiles = (nwin + tw - 1) / tw;
    const uint64_t slots = L.tiles * tw;
    L.counts = 0;
    L.scan = rup((L.tiles + 1) * 4, 256);
    L.tilebar = L.scan + rup(sws::scan_u32_scratch_words(L.tiles + 1) * 4, 256);
    L.shash = L.tilebar + rup(L.tiles * 8, 256);
    L.spos = L.shash + rup(slots * (uint64_t)sws::mini_fast_hash_bytes(sws::SRC_DNA, b->k), 256);
    L.sfirst = L.spos + rup(slots * 4, 256);
    L.fix = L.sfirst + rup(slots * 4, 256);
    L.bytes = L.fix + rup(fixb, 256);
  } else {
    const uint64_t tw = (uint64_t)sws::mini_tile_windows(b->w);
    L.tiles = (nwin + tw - 1) / tw;
    L.status = 0;
    L.counter = rup(L.tiles * 8, 256);
    L.ltilebar = L.counter + 256;
    L.lfix = L.ltilebar + rup(L.tiles * 8, 256);
    L.bytes = L.lfix + rup(fixb, 256);
  }
  return L;
}

// Queue the whole pipeline of one path on stream `st` (captured into a graph by the caller).
sws_status enqueue(sws_batch *b, int path, cudaStream_t st) {
  const Layout L = layout_for(b, path);
  char *ws = static_cast<char *>(b->ws);
  BT_CUDA(cudaMemcpyAsync(b->d_desc, b->h_desc, sws::BD_WORDS * 8, cudaMemcpyHostToDevice, st));
  BT_CUDA(cudaMemsetAsync(b->pick_offsets, 0xff, (b->max_reads + 1) * 8, st));
  BT_CUDA(cudaMemsetAsync(b->count, 0, 8, st));
  sws::MiniArgs a{};
  a.seq = b->seq;
  a.n = b->max_bases;
  a.k = b->k;
  a.w = b->w;
  a.mode = b->mode;
  a.bar = b->offsets;
  a.nbar = b->max_reads;
  a.hash_out = b->hash;
  a.pos_out = b->pos;
  a.capacity = b->capacity;
  a.count_out = b->count;
  a.pick_offsets = b->pick_offsets;
  a.err = b->d_err;
  a.desc = b->d_desc;
  uint64_t *fix;
  cudaError_t e;
  if (path == PATH_SINGLE) {
    sws::DnaMinArgs d{};
    d.seq = b->seq;
    d.n = b->max_bases;
    d.k = b->k;
    d.w = b->w;
    d.barrier = sws::BAR_READS;
    d.bar = b->offsets;
    d.nbar = b->max_reads;
    d.pick_offsets = b->pick_offsets;
    d.desc = b->d_desc;
    d.key_out = static_cast<uint32_t *>(b->hash);
    d.key_out64 = static_cast<unsigned long long *>(b->hash);
    d.pos_out = b->pos;
    d.capacity = b->capacity;
    d.count_out = b->count;
    fix = reinterpret_cast<uint64_t *>(ws + L.sfix);
    e = sws::launch_dna_min(d, ws, b->d_err, b->ctx->num_sms, st);
  } else if (path == PATH_STAGED) {
    a.tile_counts = reinterpret_cast<uint32_t *>(ws + L.counts);
    a.scan_tmp = reinterpret_cast<uint32_t *>(ws + L.scan);
    a.tile_bar = reinterpret_cast<uint2 *>(ws + L.tilebar);
    a.stg_hash = ws + L.shash;
    a.stg_pos = reinterpret_cast<uint32_t *>(ws + L.spos);
    a.stg_first = reinterpret_cast<uint32_t *>(ws + L.sfirst);
    fix = reinterpret_cast<uint64_t *>(ws + L.fix);
    e = sws::launch_minimizers_staged(a, sws::SRC_DNA, sws::BAR_READS, L.tiles, st);
  } else {
    BT_CUDA(cudaMemsetAsync(ws, 0, L.ltilebar, st));
    a.status = reinterpret_cast<unsigned long long *>(ws + L.status);
    a.tile_counter = reinterpret_cast<unsigned int *>(ws + L.counter);
    a.tile_bar = reinterpret_cast<uint2 *>(ws + L.ltilebar);
    fix = reinterpret_cast<uint64_t *>(ws + L.lfix);
    e = sws::launch_minimizers_lookback(a, sws::SRC_DNA, sws::BAR_READS, L.tiles, st);
  }
  if (e != cudaSuccess) return err_cuda(e, "batch kernels");
  e = sws::launch_pick_offsets_fixup(b->pick_offsets, b->max_reads, b->count, fix, st, b->d_desc);
  if (e != cudaSuccess) return err_cuda(e, "batch fix-up");
  return SWS_OK;
}

void set_desc(sws_batch *b, int path, uint64_t nreads, uint64_t total) {
  const uint64_t span = (uint64_t)(b->w + b->k - 1);
  const uint64_t nwin = (nreads > 0 && total >= span) ? total - span + 1 : 0;
  const uint64_t tw = (uint64_t)(path == PATH_SINGLE   ? sws::dna_min_tile_windows()
                                 : path == PATH_STAGED ? sws::mini_staged_tile_windows(sws::SRC_DNA, b->k, b->w)
                                                       : sws::mini_tile_windows(b->w));
  const uint64_t tiles = (nwin + tw - 1) / tw;
  memset(b->h_desc, 0, sws::BD_WORDS * 8);
  b->h_desc[sws::BD_NREADS] = nreads;
  b->h_desc[sws::BD_TOTAL] = total;
  b->h_desc[sws::BD_NWIN] = nwin;
  b->h_desc[sws::BD_TILES] = tiles;
  b->h_desc[sws::BD_SCAN_LEN] = tiles + 1;
}

sws_status capture(sws_batch *b, int path) {
  // run once outside capture (sets kernel attributes, sizes the grids), then capture
  set_desc(b, path, 0, 0);
  sws_status s = enqueue(b, path, b->cap);
  if (s) return s;
  BT_CUDA(cudaStreamSynchronize(b->cap));
  cudaGraph_t g = nullptr;
  BT_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  s = enqueue(b, path, b->cap);
  cudaError_t e = cudaStreamEndCapture(b->cap, &g);
  if (s) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return err_cuda(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&b->exec[path], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return err_cuda(e, "cudaGraphInstantiate");
  return SWS_OK;
}

// Synthetic batch for tuning: equal-length reads of pseudo-random bases (xorshift per byte).
__global__ void k_fill_tune_batch(uint8_t *seq, uint64_t nbytes, int64_t *offs, uint64_t nreads, uint64_t total) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = i; j < nbytes; j += stride) {
    uint32_t x = (uint32_t)(j * 2654435761u) ^ 0x9E3779B9u;
    x ^= x << 13;
    x ^= x >> 17;
    x ^= x << 5;
    seq[j] = (uint8_t)x;
  }
  for (uint64_t r = i; r <= nreads; r += stride) offs[r] = (int64_t)(total * r / (nreads ? nreads : 1));
}

sws_status time_path(sws_batch *b, int path, float *ms) {
  cudaEvent_t e0, e1;
  BT_CUDA(cudaEventCreate(&e0));
  BT_CUDA(cudaEventCreate(&e1));
  set_desc(b, path, b->max_reads, b->max_bases);
  BT_CUDA(cudaGraphLaunch(b->exec[path], b->cap));
  BT_CUDA(cudaEventRecord(e0, b->cap));
  const int reps = 3;
  for (int i = 0; i < reps; ++i) BT_CUDA(cudaGraphLaunch(b->exec[path], b->cap));
  BT_CUDA(cudaEventRecord(e1, b->cap));
  BT_CUDA(cudaEventSynchronize(e1));
  float t = 0;
  BT_CUDA(cudaEventElapsedTime(&t, e0, e1));
  *ms = t / reps;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return SWS_OK;
}

void free_batch(sws_batch *b) {
  if (!b) return;
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  for (auto &x : b->exec)
    if (x) cudaGraphExecDestroy(x);
  if (b->done) cudaEventDestroy(b->done);
  if (b->cap) cudaStreamDestroy(b->cap);
  cudaFree(b->seq);
  cudaFree(b->offsets);
  cudaFree(b->hash);
  cudaFree(b->pos);
  cudaFree(b->pick_offsets);
  cudaFree(b->count);
  cudaFree(b->d_desc);
  cudaFree(b->ws);
  cudaFree(b->d_err);
  if (b->h_desc) cudaFreeHost(b->h_desc);
  delete b;
}

}  // namespace

extern "C" {

sws_status sws_batch_create(sws_ctx *ctx, uint64_t max_reads, uint64_t max_bases, int k, int w, int mode,
                            int options, sws_batch **out) {
  if (!out) return sws::report_error(SWS_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!ctx) return sws::report_error(SWS_ERR_INVALID, "context is NULL");
  sws_status s = sws::check_minimizer_args(k, w, mode);
  if (s) return s;
  if (max_reads == 0 || max_bases == 0) return sws::report_error(SWS_ERR_INVALID, "max_reads and max_bases must be > 0");
  if (max_bases >= (1ull << 32)) return sws::report_error(SWS_ERR_INVALID, "a batch must hold fewer than 2^32 bases");
  if (options < SWS_BATCH_DEFAULT || options > SWS_BATCH_LOOKBACK) return sws::report_error(SWS_ERR_INVALID, "unknown options");
  BT_CUDA(cudaSetDevice(ctx->device));
  sws_batch *b = new sws_batch();
  b->ctx = ctx;
  b->device = ctx->device;
  b->max_reads = max_reads;
  b->max_bases = max_bases;
  b->k = k;
  b->w = w;
  b->mode = mode;
  b->hash_bytes = 2 * k <= 32 ? 4 : 8;
  b->capacity = max_bases;
  const bool staged_ok = sws::mini_staged_tile_windows(sws::SRC_DNA, k, w) > 0;  // any w: generic kernel staged
  const bool single_ok = sws::dna_min_fits(max_bases, k, w, mode);  // hashed k-mers, k <= 16, 4 <= w <= 17
  uint64_t ws_bytes = layout_for(b, PATH_LOOKBACK).bytes;
  if (staged_ok && layout_for(b, PATH_STAGED).bytes > ws_bytes) ws_bytes = layout_for(b, PATH_STAGED).bytes;
  if (single_ok && layout_for(b, PATH_SINGLE).bytes > ws_bytes) ws_bytes = layout_for(b, PATH_SINGLE).bytes;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void **p, uint64_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes ? bytes : 16);
  };
  alloc((void **)&b->seq, rup((max_bases + 3) / 4, 16) + 16);
  alloc((void **)&b->offsets, (max_reads + 1) * 8);
  alloc(&b->hash, b->capacity * b->hash_bytes);
  alloc((void **)&b->pos, b->capacity * 4);
  alloc((void **)&b->pick_offsets, (max_reads + 1) * 8);
  alloc((void **)&b->count, 8);
  alloc((void **)&b->d_desc, sws::BD_WORDS * 8);
  alloc(&b->ws, ws_bytes);
  alloc((void **)&b->d_err, 256);
  if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, 256);
  if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_desc, sws::BD_WORDS * 8);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_batch(b);
    return sws::report_error(SWS_ERR_OOM, "cannot allocate the batch buffers");
  }
  b->ws_bytes = ws_bytes;
  const bool force_lookback = options == SWS_BATCH_LOOKBACK || (!staged_ok && !single_ok);
  const bool tune = options == SWS_BATCH_TUNE && (staged_ok || single_ok);
  // the default: the single pass where it applies, else the staged path
  const int first = force_lookback ? PATH_LOOKBACK : single_ok ? PATH_SINGLE : PATH_STAGED;
  s = capture(b, first);
  if (!s && tune) {
    if (staged_ok && first != PATH_STAGED) s = capture(b, PATH_STAGED);
    if (!s) s = capture(b, PATH_LOOKBACK);
  }
  if (s) {
    free_batch(b);
    return s;
  }
  b->path = first;
  if (tune) {
    // autotune: time every captured graph on a synthetic batch of the largest size
    const uint64_t len = max_bases / max_reads;
    k_fill_tune_batch<<<1024, 256, 0, b->cap>>>(b->seq, (max_bases + 3) / 4, b->offsets, max_reads,
                                                len * max_reads);
    if ((e = cudaGetLastError()) != cudaSuccess) {
      free_batch(b);
      return err_cuda(e, "tuning batch");
    }
    for (int p = 0; p < 3 && !s; ++p)
      if (b->exec[p]) s = time_path(b, p, &b->tuned_ms[p]);
    if (s) {
      free_batch(b);
      return s;
    }
    for (int p = 0; p < 3; ++p)
      if (b->exec[p] && b->tuned_ms[p] < b->tuned_ms[b->path]) b->path = p;
  }
  e = cudaStreamSynchronize(b->cap);
  if (e != cudaSuccess) {
    free_batch(b);
    return err_cuda(e, "batch set-up");
  }
  *out = b;
  return SWS_OK;
}

sws_status sws_batch_destroy(sws_batch *b) {
  free_batch(b);
  return SWS_OK;
}

sws_status sws_batch_io_get(sws_batch *b, sws_batch_io *io) {
  if (!b || !io) return sws::report_error(SWS_ERR_INVALID, "NULL argument");
  io->seq = b->seq;
  io->offsets = b->offsets;
  io->hash = b->hash;
  io->pos = b->pos;
  io->pick_offsets = b->pick_offsets;
  io->count = b->count;
  io->capacity = b->capacity;
  io->max_reads = b->max_reads;
  io->max_bases = b->max_bases;
  io->path = b->path;
  for (int p = 0; p < 3; ++p) io->tuned_ms[p] = b->tuned_ms[p];
  return SWS_OK;
}

sws_status sws_batch_run(sws_batch *b, uint64_t nreads, uint64_t total_bases, void *stream) {
  if (!b) return sws::report_error(SWS_ERR_INVALID, "batch is NULL");
  if (nreads > b->max_reads || total_bases > b->max_bases)
    return sws::report_error(SWS_ERR_INVALID, "batch larger than the sizes it was created for");
  BT_CUDA(cudaSetDevice(b->device));
  // the pinned descriptor is read by the previous run's first node: let that run start first
  if (b->launched) BT_CUDA(cudaEventSynchronize(b->done));
  set_desc(b, b->path, nreads, total_bases);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  BT_CUDA(cudaGraphLaunch(b->exec[b->path], st));
  BT_CUDA(cudaEventRecord(b->done, st));
  b->launched = true;
  return SWS_OK;
}

sws_status sws_batch_sync(sws_batch *b) {
  if (!b) return sws::report_error(SWS_ERR_INVALID, "batch is NULL");
  BT_CUDA(cudaSetDevice(b->device));
  if (b->launched) BT_CUDA(cudaEventSynchronize(b->done));
  int err = 0;
  BT_CUDA(cudaMemcpy(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    BT_CUDA(cudaMemset(b->d_err, 0, sizeof(int)));
    return sws::report_error(SWS_ERR_TIMEOUT, "a bounded device-side wait ran out in a batch run");
  }
  return SWS_OK;
}

}  // extern "C"
