// api.cu -- the C ABI declared in include/sws.h: argument checks, the context and its device
// workspace, and dispatch to the kernels.  Host code only.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/sws.h"
#include "internal.h"

namespace {

thread_local std::string g_err = "no error";

sws_status fail(sws_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

sws_status cuda_fail(cudaError_t e, const char *what) {
  return fail(SWS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define SWS_CUDA(expr)                                 \
  do {                                                 \
    cudaError_t e_ = (expr);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #expr); \
  } while (0)

sws_status enter(sws_ctx *ctx) {
  if (!ctx) return fail(SWS_ERR_INVALID, "context is NULL");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  return SWS_OK;
}

uint64_t round_up(uint64_t v, uint64_t a) { return (v + a - 1) / a * a; }

// Make the workspace at least `bytes` long.  Growing waits for the device (the old buffer may
// still be in use by queued work) and is refused while `stream` is being captured.
sws_status ensure_ws(sws_ctx *ctx, uint64_t bytes, cudaStream_t stream) {
  if (bytes <= ctx->ws_size) return SWS_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
    return fail(SWS_ERR_OOM, "workspace must grow to %llu bytes during stream capture; call sws_reserve first",
                (unsigned long long)bytes);
  const uint64_t want = round_up(bytes + bytes / 4, 1 << 20);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
  if (ctx->ws) cudaFree(ctx->ws);
  ctx->ws = nullptr;
  ctx->ws_size = 0;
  e = cudaMalloc(&ctx->ws, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->ws = nullptr;
    return fail(SWS_ERR_OOM, "cannot allocate %llu bytes of workspace", (unsigned long long)want);
  }
  ctx->ws_size = want;
  return SWS_OK;
}

int op_esize(int op) { return op == SWS_OP_AFFINE_U32 ? 8 : 4; }

bool aligned_to(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Workspace of a minimizer launch: status words, a 256-byte slot for the tile counter, one
// tile-barrier word per tile, then `extra` bytes.
struct MiniWs {
  uint64_t status_bytes, counter_off, tilebar_off, extra_off, total;
};
MiniWs mini_ws_layout(uint64_t num_tiles, uint64_t extra) {
  MiniWs L;
  L.status_bytes = round_up(num_tiles * 8, 256);
  L.counter_off = L.status_bytes;
  L.tilebar_off = L.counter_off + 256;
  L.extra_off = L.tilebar_off + round_up(num_tiles * 8, 256);
  L.total = L.extra_off + round_up(extra, 256);
  return L;
}

sws_status check_mini_args(int k, int w, int mode) {
  if (k < 1 || k > 32) return fail(SWS_ERR_INVALID, "k must be in [1, 32] (got %d)", k);
  if (w < 1) return fail(SWS_ERR_INVALID, "w must be >= 1 (got %d)", w);
  if (sws::mini_tile_windows(w) == 0) return fail(SWS_ERR_UNSUPPORTED, "w = %d exceeds the supported maximum", w);
  if (mode < SWS_MINI_HASH || mode > SWS_MINI_FWD) return fail(SWS_ERR_INVALID, "unknown key mode %d", mode);
  return SWS_OK;
}

}  // namespace

namespace sws {
// For other translation units: record an error message for sws_last_error().
sws_status report_error(sws_status s, const char *msg) { return fail(s, "%s", msg); }
// For other translation units: the argument checks of the minimizer entry points.
sws_status check_minimizer_args(int k, int w, int mode) { return check_mini_args(k, w, mode); }
}  // namespace sws

extern "C" {

const char *sws_last_error(void) { return g_err.c_str(); }

sws_status sws_create(sws_ctx **out, int device) {
  if (!out) return fail(SWS_ERR_INVALID, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  SWS_CUDA(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(SWS_ERR_INVALID, "device %d out of range (%d devices)", device, ndev);
  SWS_CUDA(cudaSetDevice(device));
  sws_ctx *c = new sws_ctx();
  c->device = device;
  cudaError_t e = cudaMalloc(&c->d_err, 256);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "cudaMalloc(error word)");
  }
  e = cudaMemset(c->d_err, 0, 256);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) {
    cudaFree(c->d_err);
    delete c;
    return cuda_fail(e, "context setup");
  }
  *out = c;
  return SWS_OK;
}

sws_status sws_destroy(sws_ctx *ctx) {
  if (!ctx) return SWS_OK;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->d_err) cudaFree(ctx->d_err);
  delete ctx;
  return SWS_OK;
}

sws_status sws_reserve(sws_ctx *ctx, uint64_t bytes) {
  sws_status s = enter(ctx);
  if (s) return s;
  return ensure_ws(ctx, bytes, nullptr);
}

sws_status sws_sync(sws_ctx *ctx, void *stream) {
  sws_status s = enter(ctx);
  if (s) return s;
  SWS_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  int err = 0;
  SWS_CUDA(cudaMemcpy(&err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    SWS_CUDA(cudaMemset(ctx->d_err, 0, sizeof(int)));
    return fail(SWS_ERR_TIMEOUT, "a bounded device-side wait ran out (bits 0x%x); results of the affected calls are invalid",
                err);
  }
  return SWS_OK;
}

sws_status sws_selftest_wait_timeout(sws_ctx *ctx, int which, void *stream) {
  sws_status s = enter(ctx);
  if (s) return s;
  if (which != 0 && which != 1) return fail(SWS_ERR_INVALID, "which must be 0 (look-back) or 1 (mbarrier)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // two status words after the error word in the context's error block (zero = never written)
  unsigned long long *status = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(ctx->d_err) + 64);
  SWS_CUDA(cudaMemsetAsync(status, 0, 2 * sizeof(unsigned long long), st));
  cudaError_t e = sws::launch_selftest_wait(which, status, ctx->d_err, st);
  if (e != cudaSuccess) return cuda_fail(e, "self-test launch");
  return SWS_OK;
}

sws_status sws_selftest_minimizer_timeout(sws_ctx *ctx, uint64_t *count_out, void *stream) {
  sws_status s = enter(ctx);
  if (s) return s;
  if (!count_out) return fail(SWS_ERR_INVALID, "count_out is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // three tiles of k = 15, w = 10 windows over a zeroed scratch sequence in the workspace
  const int k = 15, w = 10;
  const uint64_t tiles = 3;
  const uint64_t nwin = tiles * (uint64_t)sws::mini_tile_windows(w);
  const uint64_t n = nwin + (uint64_t)(w + k - 1) - 1;
  const uint64_t seq_bytes = round_up((n + 3) / 4, 256);
  const MiniWs L = mini_ws_layout(tiles, seq_bytes);
  s = ensure_ws(ctx, L.total, st);
  if (s) return s;
  char *ws = static_cast<char *>(ctx->ws);
  SWS_CUDA(cudaMemsetAsync(ws, 0, L.tilebar_off, st));
  SWS_CUDA(cudaMemsetAsync(ws + L.extra_off, 0, seq_bytes, st));
  SWS_CUDA(cudaMemsetAsync(count_out, 0xff, sizeof(uint64_t), st));
  sws::MiniArgs a{};
  a.seq = reinterpret_cast<const uint8_t *>(ws + L.extra_off);
  a.n = n;
  a.k = k;
  a.w = w;
  a.mode = SWS_MINI_HASH;
  a.count_out = count_out;
  a.status = reinterpret_cast<unsigned long long *>(ws);
  a.tile_counter = reinterpret_cast<unsigned int *>(ws + L.counter_off);
  a.tile_bar = reinterpret_cast<uint2 *>(ws + L.tilebar_off);
  a.err = ctx->d_err;
  a.withhold_copy = 1;
  cudaError_t e = sws::launch_minimizers_lookback(a, sws::SRC_DNA, sws::BAR_NBLOCK, tiles, st);
  if (e != cudaSuccess) return cuda_fail(e, "self-test launch");
  return SWS_OK;
}

sws_status sws_sliding_sum(sws_ctx *ctx, int op, int w, const void *in, void *out, uint64_t n, int variant,
                           void *stream) {
  sws_status s = enter(ctx);
  if (s) return s;
  if (op < SWS_OP_ADD_I32 || op > SWS_OP_ADD_F32) return fail(SWS_ERR_INVALID, "unknown operator %d", op);
  if (w < 1) return fail(SWS_ERR_INVALID, "w must be >= 1 (got %d)", w);
  if (variant < SWS_VARIANT_AUTO || variant > SWS_VARIANT_BLOCK_COMBINE_WARP)
    return fail(SWS_ERR_INVALID, "unknown variant %d", variant);
  if (n < (uint64_t)w) return SWS_OK;
  if (!in || !out) return fail(SWS_ERR_INVALID, "in/out is NULL");
  const int es = op_esize(op);
  if (!aligned_to(in, es) || !aligned_to(out, es))
    return fail(SWS_ERR_INVALID, "in/out must be aligned to the element size (%d bytes)", es);
  {
    const uintptr_t a = reinterpret_cast<uintptr_t>(in), b = reinterpret_cast<uintptr_t>(out);
    const uintptr_t ae = a + n * (uint64_t)es, be = b + (n - w + 1) * (uint64_t)es;
    if (a < be && b < ae) return fail(SWS_ERR_INVALID, "in and out overlap");
  }
  if (variant == SWS_VARIANT_PREFIX_DIFF && op != SWS_OP_ADD_I32 && op != SWS_OP_XOR_I32)
    return fail(SWS_ERR_INVALID, "prefix-difference needs an invertible operator (ADD_I32 or XOR_I32)");
  sws::SlideLaunch L;
  L.op = op;
  L.variant = variant;
  L.num_sms = ctx->num_sms;
  L.err = ctx->d_err;
  if (variant == SWS_VARIANT_AUTO) {  // a variant sws_tune_sliding_sum chose for this (op, w)
    std::lock_guard<std::mutex> g(ctx->tune_mu);
    auto it = ctx->tuned.find({op, w});
    if (it != ctx->tuned.end() && n >= it->second.n / 8) {
      L.variant = it->second.variant;
      L.shape = it->second.shape;
    }
  }
  // the smaller tile when it keeps the halo re-read under an eighth of the tile
  const int small_len = sws::slide_tile_len(sws::CFG_SMALL, es);
  L.cfg = (w - 1) * 8 <= small_len ? sws::CFG_SMALL : sws::CFG_LARGE;
  if (sws::slide_tile_outputs(L.cfg, es, w) == 0)
    return fail(SWS_ERR_UNSUPPORTED, "w = %d is larger than the tile of this build", w);
  cudaError_t e = sws::launch_sliding_sum(L, in, out, n, w, static_cast<cudaStream_t>(stream));
  if (e == cudaErrorNotSupported &&
      (variant == SWS_VARIANT_BLOCK_COMBINE_STREAM || variant == SWS_VARIANT_BLOCK_COMBINE_WARP))
    return fail(SWS_ERR_UNSUPPORTED, "the streamed block combine does not apply to w = %d, n = %llu at this alignment",
                w, (unsigned long long)n);
  if (e != cudaSuccess) return cuda_fail(e, "sliding-sum launch");
  return SWS_OK;
}

sws_status sws_tune_sliding_sum(sws_ctx *ctx, int op, int w, uint64_t n, int *variant_out, float *ms_out,
                                void *stream) {
  sws_status s = enter(ctx);
  if (s) return s;
  if (op < SWS_OP_ADD_I32 || op > SWS_OP_ADD_F32) return fail(SWS_ERR_INVALID, "unknown operator %d", op);
  if (w < 1) return fail(SWS_ERR_INVALID, "w must be >= 1 (got %d)", w);
  if (n < (uint64_t)w) return fail(SWS_ERR_INVALID, "n must be >= w");
  const int es = op_esize(op);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint64_t in_bytes = round_up(n * (uint64_t)es, 256);
  s = ensure_ws(ctx, 2 * in_bytes, st);
  if (s) return s;
  char *in = static_cast<char *>(ctx->ws);
  char *out = in + in_bytes;
  cudaError_t e = sws::launch_fill_pattern(in, n * (uint64_t)es, st);
  if (e != cudaSuccess) return cuda_fail(e, "tuning input");
  sws::SlideLaunch L;
  L.op = op;
  L.num_sms = ctx->num_sms;
  L.err = ctx->d_err;
  const int small_len = sws::slide_tile_len(sws::CFG_SMALL, es);
  L.cfg = (w - 1) * 8 <= small_len ? sws::CFG_SMALL : sws::CFG_LARGE;
  if (sws::slide_tile_outputs(L.cfg, es, w) == 0)
    return fail(SWS_ERR_UNSUPPORTED, "w = %d is larger than the tile of this build", w);
  cudaEvent_t e0, e1;
  SWS_CUDA(cudaEventCreate(&e0));
  SWS_CUDA(cudaEventCreate(&e1));
  // best of five launches of the current L, after one untimed launch; e carries errors
  auto time_it = [&](float &t) {
    t = 1e30f;
    for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) {
      e = cudaEventRecord(e0, st);
      if (e == cudaSuccess) e = sws::launch_sliding_sum(L, in, out, n, w, st);
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float x = 0;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&x, e0, e1);
      if (e == cudaSuccess && x < t) t = x;
    }
  };
  // the library's fixed rule (AUTO without a tuned entry) first, after warming the GPU up with
  // at least 10 ms of it (clocks ramp from idle), so that every variant is timed at speed
  float ms[SWS_VARIANT_COUNT];
  L.variant = SWS_VARIANT_AUTO;
  L.shape = 0;
  float warm = 0.0f;
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  for (int i = 0; i < 400 && e == cudaSuccess && warm < 10.0f; ++i) {
    e = sws::launch_sliding_sum(L, in, out, n, w, st);
    if (e == cudaSuccess && (i & 7) == 7) {
      e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&warm, e0, e1);
    }
  }
  float rule_t = 0.0f;
  time_it(rule_t);
  ms[SWS_VARIANT_AUTO] = rule_t;
  int best = -1, best_shape = 0;
  float best_t = 0.0f;
  for (int v = 0; v < SWS_VARIANT_COUNT && e == cudaSuccess; ++v) {
    if (v == SWS_VARIANT_AUTO) continue;
    ms[v] = -1.0f;
    if (v == SWS_VARIANT_PREFIX_DIFF && op != SWS_OP_ADD_I32 && op != SWS_OP_XOR_I32) continue;
    // the warp-private variant is timed in each of its run shapes; the others once
    const int nshapes = v == SWS_VARIANT_BLOCK_COMBINE_WARP ? sws::kWarpShapes : 1;
    for (int sh = 1; sh <= nshapes; ++sh) {
      L.variant = v;
      L.shape = v == SWS_VARIANT_BLOCK_COMBINE_WARP ? sh : 0;
      e = sws::launch_sliding_sum(L, in, out, n, w, st);  // warm-up; also tells whether v applies
      if (e == cudaErrorNotSupported || e == cudaErrorInvalidValue) {  // v does not apply to (op, w, n)
        cudaGetLastError();
        e = cudaSuccess;
        break;
      }
      if (e != cudaSuccess) break;
      float t = 0.0f;
      time_it(t);
      if (e != cudaSuccess) break;
      if (ms[v] < 0 || t < ms[v]) ms[v] = t;  // per variant: its best shape
      if (best < 0 || t < best_t) {
        best = v;
        best_shape = L.shape;
        best_t = t;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e, "tuning run");
  if (best < 0) return fail(SWS_ERR_UNSUPPORTED, "no variant applies to w = %d", w);
  if (best_t > 0.98f * rule_t) {  // not clearly faster than the fixed rule: keep the rule
    best = SWS_VARIANT_AUTO;
    best_shape = 0;
  }
  {
    std::lock_guard<std::mutex> g(ctx->tune_mu);
    ctx->tuned[{op, w}] = {best, best_shape, n};
  }
  if (variant_out) *variant_out = best;
  if (ms_out) memcpy(ms_out, ms, sizeof(ms));
  return SWS_OK;
}

sws_status sws_kmers(sws_ctx *ctx, const uint8_t *seq, uint64_t n, int k, int kind, void *out, void *stream) {
  sws_status s = enter(ctx);
  if (s) return s;
  if (k < 1 || k > 32) return fail(SWS_ERR_INVALID, "k must be in [1, 32] (got %d)", k);
  if (kind < SWS_KMER_FWD || kind > SWS_KMER_HASH) return fail(SWS_ERR_INVALID, "unknown k-mer kind %d", kind);
  if (n < (uint64_t)k) return SWS_OK;
  if (!seq || !out) return fail(SWS_ERR_INVALID, "seq/out is NULL");
  if (!aligned_to(out, 2 * k <= 32 ? 4 : 8)) return fail(SWS_ERR_INVALID, "out is not aligned to its element size");
  cudaError_t e = sws::launch_kmers(seq, n, k, kind, out, ctx->d_err, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "k-mer launch");
  return SWS_OK;
}

// Workspace of the staged minimizer path: per-tile counts (+1 for the total), scan scratch, one
// barrier summary per tile, then the staging slots (hash, position, and for read batches the read
// index of a read's first pick), then `extra` bytes.
struct StagedWs {
  uint64_t counts_off, scan_off, tilebar_off, hash_off, pos_off, first_off, extra_off, total;
};
StagedWs staged_ws_layout(uint64_t tiles, int tile_windows, int hash_bytes, bool reads, uint64_t extra) {
  StagedWs L;
  const uint64_t slots = tiles * (uint64_t)tile_windows;
  L.counts_off = 0;
  L.scan_off = round_up((tiles + 1) * 4, 256);
  L.tilebar_off = L.scan_off + round_up(sws::scan_u32_scratch_words(tiles + 1) * 4, 256);
  L.hash_off = L.tilebar_off + round_up(tiles * 8, 256);
  L.pos_off = L.hash_off + round_up(slots * (uint64_t)hash_bytes, 256);
  L.first_off = L.pos_off + round_up(slots * 4, 256);
  L.extra_off = L.first_off + (reads ? round_up(slots * 4, 256) : 0);
  L.total = L.extra_off + round_up(extra, 256);
  return L;
}

// Fill the workspace pointers of `a` and queue the minimizer kernels (staged path when it
// applies, look-back path otherwise).  `extra` bytes of workspace are returned in *extra_ptr.
sws_status run_minimizers(sws_ctx *ctx, sws::MiniArgs &a, int source, int barrier, uint64_t nwin, uint64_t extra,
                          void **extra_ptr, cudaStream_t st) {
  // The staged path (five launches) pays off once the input fills the GPU; below that the
  // single-kernel look-back path has the lower latency.
  const uint64_t tw = (uint64_t)sws::mini_staged_tile_windows(source, a.k, a.w);
  const bool staged = tw > 0 && nwin >= 4 * tw * (uint64_t)ctx->num_sms;
  if (staged) {
    const uint64_t tiles = (nwin + tw - 1) / tw;
    if (tiles >= 0xffffffffull) return fail(SWS_ERR_INVALID, "input too long");
    // a count-only run needs no staging slots
    const StagedWs L = staged_ws_layout(tiles, a.count_only ? 0 : (int)tw, sws::mini_fast_hash_bytes(source, a.k),
                                        barrier == sws::BAR_READS, extra);
    sws_status s = ensure_ws(ctx, L.total, st);
    if (s) return s;
    char *w = static_cast<char *>(ctx->ws);
    a.tile_counts = reinterpret_cast<uint32_t *>(w + L.counts_off);
    a.scan_tmp = reinterpret_cast<uint32_t *>(w + L.scan_off);
    a.tile_bar = reinterpret_cast<uint2 *>(w + L.tilebar_off);
    a.stg_hash = w + L.hash_off;
    a.stg_pos = reinterpret_cast<uint32_t *>(w + L.pos_off);
    a.stg_first = reinterpret_cast<uint32_t *>(w + L.first_off);
    a.err = ctx->d_err;
    if (extra_ptr) *extra_ptr = w + L.extra_off;
    cudaError_t e = sws::launch_minimizers_staged(a, source, barrier, tiles, st);
    if (e != cudaSuccess) return cuda_fail(e, "staged minimizer launch");
    return SWS_OK;
  }
  const uint64_t tiles = sws::mini_lookback_tiles(nwin, a.w);
  const MiniWs L = mini_ws_layout(tiles, extra);
  sws_status s = ensure_ws(ctx, L.total, st);
  if (s) return s;
  char *w = static_cast<char *>(ctx->ws);
  SWS_CUDA(cudaMemsetAsync(w, 0, L.tilebar_off, st));
  a.status = reinterpret_cast<unsigned long long *>(w);
  a.tile_counter = reinterpret_cast<unsigned int *>(w + L.counter_off);
  a.tile_bar = reinterpret_cast<uint2 *>(w + L.tilebar_off);
  a.err = ctx->d_err;
  if (extra_ptr) *extra_ptr = w + L.extra_off;
  cudaError_t e = sws::launch_minimizers_lookback(a, source, barrier, tiles, st);
  if (e != cudaSuccess) return cuda_fail(e, "minimizer launch");
  return SWS_OK;
}

static sws_status minimizers_common(sws_ctx *ctx, int source, const uint8_t *seq, const uint32_t *keys, uint64_t n,
                                    int k, int w, int mode, const int64_t *nblocks, uint64_t n_nblocks,
                                    void *hash_out, uint32_t *pos_out, uint64_t capacity, uint64_t *count_out,
                                    void *stream, bool count_only = false) {
  sws_status s = enter(ctx);
  if (s) return s;
  s = check_mini_args(k, w, mode);
  if (s) return s;
  if (!count_out) return fail(SWS_ERR_INVALID, "count_out is NULL");
  if (capacity > 0 && (!hash_out || !pos_out)) return fail(SWS_ERR_INVALID, "hash_out/pos_out is NULL");
  if (n >= (1ull << 32)) return fail(SWS_ERR_INVALID, "sequences must be shorter than 2^32");
  if (n_nblocks > 0 && !nblocks) return fail(SWS_ERR_INVALID, "nblocks is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint64_t span = source == sws::SRC_DNA ? (uint64_t)(w + k - 1) : (uint64_t)w;
  const uint64_t nwin = n >= span ? n - span + 1 : 0;
  if (nwin == 0) {
    SWS_CUDA(cudaMemsetAsync(count_out, 0, sizeof(uint64_t), st));
    return SWS_OK;
  }
  if (source == sws::SRC_DNA && !seq) return fail(SWS_ERR_INVALID, "seq is NULL");
  if (source == sws::SRC_KEYS && !keys) return fail(SWS_ERR_INVALID, "keys is NULL");
  if (source == sws::SRC_KEYS && !count_only && sws::keys_min_applies(keys, n, w)) {
    // w <= 17: the single-pass kernel of keys_min.cu
    s = ensure_ws(ctx, sws::keys_min_ws_bytes(n, w), st);
    if (s) return s;
    cudaError_t e = sws::launch_keys_min(keys, n, w, static_cast<uint32_t *>(hash_out), pos_out, capacity, count_out,
                                         ctx->ws, ctx->d_err, ctx->num_sms, st);
    if (e != cudaSuccess) return cuda_fail(e, "key minimizer launch");
    return SWS_OK;
  }
  if (source == sws::SRC_DNA && !count_only && sws::dna_min_applies(seq, n, k, w, mode)) {
    // hashed k-mers, k <= 16, 4 <= w <= 17: the single-pass kernel of keys_min.cu
    s = ensure_ws(ctx, sws::dna_min_ws_bytes(n, k, w), st);
    if (s) return s;
    sws::DnaMinArgs d{};
    d.seq = seq;
    d.n = n;
    d.k = k;
    d.w = w;
    d.barrier = n_nblocks > 0 ? sws::BAR_NBLOCK : -1;
    d.bar = nblocks;
    d.nbar = n_nblocks;
    d.key_out = static_cast<uint32_t *>(hash_out);
    d.key_out64 = static_cast<unsigned long long *>(hash_out);
    d.pos_out = pos_out;
    d.capacity = capacity;
    d.count_out = count_out;
    cudaError_t e = sws::launch_dna_min(d, ctx->ws, ctx->d_err, ctx->num_sms, st);
    if (e != cudaSuccess) return cuda_fail(e, "DNA minimizer launch");
    return SWS_OK;
  }
  sws::MiniArgs a{};
  a.seq = seq;
  a.keys = keys;
  a.n = n;
  a.k = source == sws::SRC_DNA ? k : 1;
  a.w = w;
  a.mode = mode;
  a.bar = nblocks;
  a.nbar = n_nblocks;
  a.hash_out = hash_out;
  a.pos_out = pos_out;
  a.capacity = capacity;
  a.count_out = count_out;
  a.count_only = count_only ? 1 : 0;
  return run_minimizers(ctx, a, source, sws::BAR_NBLOCK, nwin, 0, nullptr, st);
}

sws_status sws_minimizers(sws_ctx *ctx, const uint8_t *seq, uint64_t n, int k, int w, int mode,
                          const int64_t *nblocks, uint64_t n_nblocks, void *hash_out, uint32_t *pos_out,
                          uint64_t capacity, uint64_t *count_out, void *stream) {
  return minimizers_common(ctx, sws::SRC_DNA, seq, nullptr, n, k, w, mode, nblocks, n_nblocks, hash_out, pos_out,
                           capacity, count_out, stream);
}

sws_status sws_minimizers_count(sws_ctx *ctx, const uint8_t *seq, uint64_t n, int k, int w, int mode,
                                const int64_t *nblocks, uint64_t n_nblocks, uint64_t *count_out, void *stream) {
  return minimizers_common(ctx, sws::SRC_DNA, seq, nullptr, n, k, w, mode, nblocks, n_nblocks, nullptr, nullptr, 0,
                           count_out, stream, /*count_only=*/true);
}

sws_status sws_build_table(sws_ctx *ctx, const uint8_t *seq, uint64_t n, int k, int w, int mode,
                           const int64_t *nblocks, uint64_t n_nblocks, int bucket_bits, void *sorted_hash,
                           uint32_t *sorted_pos, uint64_t capacity, uint64_t *bucket_offsets, uint64_t *count,
                           void *stream) {
  sws_status s = enter(ctx);
  if (s) return s;
  s = check_mini_args(k, w, mode);
  if (s) return s;
  const int hash_bits = 2 * k;
  if (bucket_bits < 0 || bucket_bits > hash_bits || bucket_bits > 32)
    return fail(SWS_ERR_INVALID, "bucket_bits must be in [0, min(2k, 32)] (got %d)", bucket_bits);
  if (!count || !bucket_offsets) return fail(SWS_ERR_INVALID, "count/bucket_offsets is NULL");
  if (capacity > 0 && (!sorted_hash || !sorted_pos)) return fail(SWS_ERR_INVALID, "sorted_hash/sorted_pos is NULL");
  *count = 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // 1. the minimizers, written straight into the caller's output arrays (the sort's first pass
  //    reads them and its last pass overwrites them; a one-pass sort, 2k <= 8, stages them in the
  //    workspace first); the count goes to a word of the context's error block
  uint64_t *d_count = reinterpret_cast<uint64_t *>(reinterpret_cast<char *>(ctx->d_err) + 128);
  s = minimizers_common(ctx, sws::SRC_DNA, seq, nullptr, n, k, w, mode, nblocks, n_nblocks, sorted_hash, sorted_pos,
                        capacity, d_count, stream);
  if (s) return s;
  uint64_t m = 0;
  SWS_CUDA(cudaMemcpyAsync(&m, d_count, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
  SWS_CUDA(cudaStreamSynchronize(st));
  {
    int err = 0;
    SWS_CUDA(cudaMemcpy(&err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
      SWS_CUDA(cudaMemset(ctx->d_err, 0, sizeof(int)));
      return fail(SWS_ERR_TIMEOUT, "a bounded device-side wait ran out while finding the minimizers (bits 0x%x)", err);
    }
  }
  *count = m;
  if (m > capacity)
    return fail(SWS_ERR_CAPACITY, "%llu minimizers exceed the capacity %llu", (unsigned long long)m,
                (unsigned long long)capacity);
  // 2. the seed table over the m hits, in place
  const bool wide = hash_bits > 32;
  const uint64_t hs = wide ? 8 : 4;
  const bool one_pass = hash_bits <= 8;
  const uint64_t kbytes = round_up(m * 8, 256), vbytes = wide ? round_up(m * 4, 256) : 0;
  const uint64_t hbytes = round_up(sws::table_hist_words(m) * 4, 256);
  const uint64_t bbytes = round_up(sws::table_bsum_words(m) * 4, 256);
  const uint64_t gbytes = round_up(sws::table_gap_bytes(bucket_bits), 256);
  const uint64_t mbytes = round_up(sws::table_msd_bytes(m), 256);
  const uint64_t copy_bytes = one_pass ? round_up(m * hs, 256) + round_up(m * 4, 256) : 0;
  const uint64_t total = 2 * kbytes + 2 * vbytes + hbytes + bbytes + gbytes + 256 + mbytes + copy_bytes;
  s = ensure_ws(ctx, total, st);
  if (s) return s;
  char *ws = static_cast<char *>(ctx->ws);
  const void *in_hash = sorted_hash;
  const uint32_t *in_pos = sorted_pos;
  if (one_pass && m > 0) {
    char *c = ws + total - copy_bytes;
    SWS_CUDA(cudaMemcpyAsync(c, sorted_hash, m * hs, cudaMemcpyDeviceToDevice, st));
    SWS_CUDA(cudaMemcpyAsync(c + round_up(m * hs, 256), sorted_pos, m * 4, cudaMemcpyDeviceToDevice, st));
    in_hash = c;
    in_pos = reinterpret_cast<const uint32_t *>(c + round_up(m * hs, 256));
  }
  sws::TableArgs a{};
  a.hash = in_hash;
  a.pos = in_pos;
  a.m = m;
  a.hash_bits = hash_bits;
  a.bucket_bits = bucket_bits;
  a.sorted_hash = sorted_hash;
  a.sorted_pos = sorted_pos;
  a.offsets = bucket_offsets;
  a.ws_keys[0] = reinterpret_cast<unsigned long long *>(ws);
  a.ws_keys[1] = reinterpret_cast<unsigned long long *>(ws + kbytes);
  a.ws_vals[0] = wide ? reinterpret_cast<uint32_t *>(ws + 2 * kbytes) : nullptr;
  a.ws_vals[1] = wide ? reinterpret_cast<uint32_t *>(ws + 2 * kbytes + vbytes) : nullptr;
  a.ws_hist = reinterpret_cast<uint32_t *>(ws + 2 * kbytes + 2 * vbytes);
  a.ws_bsum = reinterpret_cast<uint32_t *>(ws + 2 * kbytes + 2 * vbytes + hbytes);
  a.ws_gaps = ws + 2 * kbytes + 2 * vbytes + hbytes + bbytes;
  a.ws_ngaps = reinterpret_cast<unsigned long long *>(ws + 2 * kbytes + 2 * vbytes + hbytes + bbytes + gbytes);
  a.gap_cap = sws::table_gap_capacity(bucket_bits);
  a.ws_msd = ws + 2 * kbytes + 2 * vbytes + hbytes + bbytes + gbytes + 256;
  cudaError_t e = sws::launch_table(a, st);
  if (e != cudaSuccess) return cuda_fail(e, "seed-table launch");
  return SWS_OK;
}

sws_status sws_minimizers_from_keys(sws_ctx *ctx, const uint32_t *keys, uint64_t m, int w, uint32_t *key_out,
                                    uint32_t *pos_out, uint64_t capacity, uint64_t *count_out, void *stream) {
  return minimizers_common(ctx, sws::SRC_KEYS, nullptr, keys, m, 1, w, SWS_MINI_HASH, nullptr, 0, key_out, pos_out,
                           capacity, count_out, stream);
}

sws_status sws_minimizers_batch(sws_ctx *ctx, const uint8_t *seq, const int64_t *base_offsets, uint64_t nreads,
                                uint64_t total_bases, int k, int w, int mode, void *hash_out, uint32_t *pos_out,
                                uint64_t capacity, uint64_t *pick_offsets, uint64_t *count_out, void *stream) {
  sws_status s = enter(ctx);
  if (s) return s;
  s = check_mini_args(k, w, mode);
  if (s) return s;
  if (!count_out || !pick_offsets) return fail(SWS_ERR_INVALID, "count_out/pick_offsets is NULL");
  if (capacity > 0 && (!hash_out || !pos_out)) return fail(SWS_ERR_INVALID, "hash_out/pos_out is NULL");
  if (nreads > 0 && !base_offsets) return fail(SWS_ERR_INVALID, "base_offsets is NULL");
  if (total_bases >= (1ull << 32)) return fail(SWS_ERR_INVALID, "a batch must hold fewer than 2^32 bases");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint64_t span = (uint64_t)(w + k - 1);
  const uint64_t nwin = total_bases >= span ? total_bases - span + 1 : 0;
  if (nreads == 0 || nwin == 0) {
    SWS_CUDA(cudaMemsetAsync(count_out, 0, sizeof(uint64_t), st));
    SWS_CUDA(cudaMemsetAsync(pick_offsets, 0, (nreads + 1) * sizeof(uint64_t), st));
    return SWS_OK;
  }
  if (!seq) return fail(SWS_ERR_INVALID, "seq is NULL");
  SWS_CUDA(cudaMemsetAsync(pick_offsets, 0xff, (nreads + 1) * sizeof(uint64_t), st));
  const uint64_t fix_blocks = (nreads + 1023) / 1024 + 1;
  if (sws::dna_min_applies(seq, total_bases, k, w, mode)) {
    // hashed k-mers, k <= 16, 4 <= w <= 17: the single-pass kernel with read starts as barriers
    const uint64_t dws = (sws::dna_min_ws_bytes(total_bases, k, w) + 255) / 256 * 256;
    s = ensure_ws(ctx, dws + fix_blocks * 8, st);
    if (s) return s;
    sws::DnaMinArgs d{};
    d.seq = seq;
    d.n = total_bases;
    d.k = k;
    d.w = w;
    d.barrier = sws::BAR_READS;
    d.bar = base_offsets;
    d.nbar = nreads;
    d.pick_offsets = pick_offsets;
    d.key_out = static_cast<uint32_t *>(hash_out);
    d.key_out64 = static_cast<unsigned long long *>(hash_out);
    d.pos_out = pos_out;
    d.capacity = capacity;
    d.count_out = count_out;
    cudaError_t e = sws::launch_dna_min(d, ctx->ws, ctx->d_err, ctx->num_sms, st);
    if (e != cudaSuccess) return cuda_fail(e, "DNA minimizer launch");
    e = sws::launch_pick_offsets_fixup(pick_offsets, nreads, count_out,
                                       reinterpret_cast<uint64_t *>(static_cast<char *>(ctx->ws) + dws), st);
    if (e != cudaSuccess) return cuda_fail(e, "pick-offset fix-up launch");
    return SWS_OK;
  }
  sws::MiniArgs a{};
  a.seq = seq;
  a.n = total_bases;
  a.k = k;
  a.w = w;
  a.mode = mode;
  a.bar = base_offsets;
  a.nbar = nreads;
  a.hash_out = hash_out;
  a.pos_out = pos_out;
  a.capacity = capacity;
  a.count_out = count_out;
  a.pick_offsets = pick_offsets;
  void *fix = nullptr;
  s = run_minimizers(ctx, a, sws::SRC_DNA, sws::BAR_READS, nwin, fix_blocks * 8, &fix, st);
  if (s) return s;
  cudaError_t e = sws::launch_pick_offsets_fixup(pick_offsets, nreads, count_out, static_cast<uint64_t *>(fix), st);
  if (e != cudaSuccess) return cuda_fail(e, "pick-offset fix-up launch");
  return SWS_OK;
}

sws_status sws_kmer_table(sws_ctx *ctx, const void *hash, const uint32_t *pos, uint64_t m, int hash_bits,
                          int bucket_bits, void *sorted_hash, uint32_t *sorted_pos, uint64_t *bucket_offsets,
                          void *stream) {
  sws_status s = enter(ctx);
  if (s) return s;
  if (hash_bits < 1 || hash_bits > 64) return fail(SWS_ERR_INVALID, "hash_bits must be in [1, 64] (got %d)", hash_bits);
  if (bucket_bits < 0 || bucket_bits > hash_bits || bucket_bits > 32)
    return fail(SWS_ERR_INVALID, "bucket_bits must be in [0, min(hash_bits, 32)] (got %d)", bucket_bits);
  if (m >= (1ull << 32)) return fail(SWS_ERR_INVALID, "at most 2^32 - 1 hits");
  if (!bucket_offsets) return fail(SWS_ERR_INVALID, "bucket_offsets is NULL");
  if (m > 0 && (!hash || !pos || !sorted_hash || !sorted_pos)) return fail(SWS_ERR_INVALID, "NULL array");
  const uint64_t hs = hash_bits > 32 ? 8 : 4;
  if (m > 0) {
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(hash), a1 = a0 + m * hs;
    const uintptr_t b0 = reinterpret_cast<uintptr_t>(sorted_hash), b1 = b0 + m * hs;
    const uintptr_t c0 = reinterpret_cast<uintptr_t>(pos), c1 = c0 + m * 4;
    const uintptr_t d0 = reinterpret_cast<uintptr_t>(sorted_pos), d1 = d0 + m * 4;
    if ((a0 < b1 && b0 < a1) || (c0 < d1 && d0 < c1)) return fail(SWS_ERR_INVALID, "inputs and outputs overlap");
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool wide = hash_bits > 32;
  const uint64_t kbytes = round_up(m * 8, 256), vbytes = wide ? round_up(m * 4, 256) : 0;
  const uint64_t hbytes = round_up(sws::table_hist_words(m) * 4, 256);
  const uint64_t bbytes = round_up(sws::table_bsum_words(m) * 4, 256);
  const uint64_t gbytes = round_up(sws::table_gap_bytes(bucket_bits), 256);
  const uint64_t mbytes = round_up(sws::table_msd_bytes(m), 256);
  const uint64_t total = 2 * kbytes + 2 * vbytes + hbytes + bbytes + gbytes + 256 + mbytes;
  s = ensure_ws(ctx, total, st);
  if (s) return s;
  char *w = static_cast<char *>(ctx->ws);
  sws::TableArgs a{};
  a.hash = hash;
  a.pos = pos;
  a.m = m;
  a.hash_bits = hash_bits;
  a.bucket_bits = bucket_bits;
  a.sorted_hash = sorted_hash;
  a.sorted_pos = sorted_pos;
  a.offsets = bucket_offsets;
  a.ws_keys[0] = reinterpret_cast<unsigned long long *>(w);
  a.ws_keys[1] = reinterpret_cast<unsigned long long *>(w + kbytes);
  a.ws_vals[0] = wide ? reinterpret_cast<uint32_t *>(w + 2 * kbytes) : nullptr;
  a.ws_vals[1] = wide ? reinterpret_cast<uint32_t *>(w + 2 * kbytes + vbytes) : nullptr;
  a.ws_hist = reinterpret_cast<uint32_t *>(w + 2 * kbytes + 2 * vbytes);
  a.ws_bsum = reinterpret_cast<uint32_t *>(w + 2 * kbytes + 2 * vbytes + hbytes);
  a.ws_gaps = w + 2 * kbytes + 2 * vbytes + hbytes + bbytes;
  a.ws_ngaps = reinterpret_cast<unsigned long long *>(w + 2 * kbytes + 2 * vbytes + hbytes + bbytes + gbytes);
  a.gap_cap = sws::table_gap_capacity(bucket_bits);
  a.ws_msd = w + 2 * kbytes + 2 * vbytes + hbytes + bbytes + gbytes + 256;
  cudaError_t e = sws::launch_table(a, st);
  if (e != cudaSuccess) return cuda_fail(e, "seed-table launch");
  return SWS_OK;
}

sws_status sws_minimizer_strands(sws_ctx *ctx, const uint8_t *seq, uint64_t n, int k, const int64_t *base_offsets,
                                 const uint64_t *pick_offsets, uint64_t nreads, const uint32_t *pos, uint64_t m,
                                 uint8_t *strand_out, void *stream) {
  sws_status s = enter(ctx);
  if (s) return s;
  if (k < 1 || k > 32) return fail(SWS_ERR_INVALID, "k must be in [1, 32] (got %d)", k);
  if (m == 0) return SWS_OK;
  if (!seq || !pos || !strand_out) return fail(SWS_ERR_INVALID, "NULL array");
  if ((base_offsets == nullptr) != (pick_offsets == nullptr))
    return fail(SWS_ERR_INVALID, "base_offsets and pick_offsets go together");
  if (base_offsets && nreads == 0) return fail(SWS_ERR_INVALID, "a batch needs nreads >= 1");
  cudaError_t e = sws::launch_strands(seq, n, k, base_offsets, pick_offsets, base_offsets ? nreads : 0, pos, m,
                                      strand_out, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "strand launch");
  return SWS_OK;
}

sws_status sws_seed_lookup(sws_ctx *ctx, const void *sorted_hash, uint64_t m, int hash_bits, int bucket_bits,
                           const uint64_t *bucket_offsets, const void *query_hash, uint64_t nq, uint64_t *first,
                           uint32_t *count, void *stream) {
  sws_status s = enter(ctx);
  if (s) return s;
  if (hash_bits < 1 || hash_bits > 64) return fail(SWS_ERR_INVALID, "hash_bits must be in [1, 64] (got %d)", hash_bits);
  if (bucket_bits < 0 || bucket_bits > hash_bits || bucket_bits > 32)
    return fail(SWS_ERR_INVALID, "bucket_bits must be in [0, min(hash_bits, 32)] (got %d)", bucket_bits);
  if (m >= (1ull << 32)) return fail(SWS_ERR_INVALID, "at most 2^32 - 1 table entries");
  if (nq == 0) return SWS_OK;
  if (!bucket_offsets || !query_hash || !first || !count || (m > 0 && !sorted_hash))
    return fail(SWS_ERR_INVALID, "NULL array");
  cudaError_t e = sws::launch_seed_lookup(sorted_hash, hash_bits, bucket_bits, bucket_offsets, query_hash, nq, first,
                                          count, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "seed-lookup launch");
  return SWS_OK;
}

sws_status sws_seed_hits(sws_ctx *ctx, const uint64_t *first, const uint32_t *count, uint64_t nq, uint32_t max_occ,
                         const uint32_t *sorted_pos, uint32_t *hit_query, uint32_t *hit_pos, uint64_t capacity,
                         uint64_t *hit_count, void *stream) {
  sws_status s = enter(ctx);
  if (s) return s;
  if (nq >= (1ull << 32)) return fail(SWS_ERR_INVALID, "at most 2^32 - 1 queries");
  if (!hit_count) return fail(SWS_ERR_INVALID, "hit_count is NULL");
  if (nq > 0 && (!first || !count || !sorted_pos)) return fail(SWS_ERR_INVALID, "NULL array");
  if (capacity > 0 && (!hit_query || !hit_pos)) return fail(SWS_ERR_INVALID, "hit_query/hit_pos is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint64_t bytes = round_up(sws::seed_hit_tiles(nq) * 8, 256) + 256;
  s = ensure_ws(ctx, bytes, st);
  if (s) return s;
  cudaError_t e = sws::launch_seed_hits(first, count, nq, max_occ, sorted_pos, hit_query, hit_pos, capacity, hit_count,
                                        static_cast<unsigned long long *>(ctx->ws), st);
  if (e != cudaSuccess) return cuda_fail(e, "seed-hits launch");
  return SWS_OK;
}

}  // extern "C"
