// noalloc.cu -- minimizers for callers that cannot allocate device memory.
//
// sws_minimizers keeps the scratch of its ordered output (one status word per tile, a tile
// counter, one barrier summary per tile) in a context workspace that grows with cudaMalloc.
// Some callers cannot allocate: code running inside a device-memory allocator's own hooks (an
// allocation there would re-enter the allocator), programs whose device memory is fully handed
// out in advance by a framework that owns every byte, and latency-critical paths that must not
// pay for, or risk the failure of, an allocation.  For them, sws_minimizers_noalloc runs the
// single-kernel (look-back) minimizer path with its scratch in a fixed array that this file
// declares in device global memory; a call allocates nothing and needs no context.
//
// The array lives as long as the library is loaded, on every device that loads it (4 MiB each).
// Its device address is looked up (cudaGetSymbolAddress, with that device current) on the first
// call made in each CUDA context of a device and kept for that context: a device reset or a new
// primary context reloads the module at another address, so the cached address is keyed on the
// context handle, never reused across contexts.  Host code never passes the symbol itself.
#include <cstdio>
#include <mutex>

#include <cuda.h>

#include "../../include/sws.h"
#include "internal.h"

// Scratch of sws_minimizers_noalloc: [0, 256) error word and tile counter, then one 8-byte status
// word per tile, then one 8-byte barrier summary per tile.
static constexpr unsigned long long kNoallocScratchBytes = 4ull << 20;
static constexpr unsigned long long kNoallocHeader = 256;
static constexpr unsigned long long kNoallocMaxTiles = (kNoallocScratchBytes - kNoallocHeader) / 16;
static __device__ __align__(256) unsigned char sws_noalloc_scratch[kNoallocScratchBytes];

namespace {

constexpr int kMaxDevices = 128;
std::mutex g_mu;
struct Cached {
  CUcontext ctx;       // the context the address belongs to
  unsigned char *addr;
};
Cached g_addr[kMaxDevices] = {};

using CtxGetCurrent = CUresult (*)(CUcontext *);

// cuCtxGetCurrent from the driver, looked up once through the runtime (no -lcuda).
CtxGetCurrent ctx_get_current() {
  static CtxGetCurrent fn = []() -> CtxGetCurrent {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<CtxGetCurrent>(p);
    return nullptr;
  }();
  return fn;
}

// Device address of the scratch array in the current context of the current device (set up on
// the first call in that context).
int scratch_address(unsigned char **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return sws::report_error(SWS_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return sws::report_error(SWS_ERR_UNSUPPORTED, "device index too large");
  CtxGetCurrent get = ctx_get_current();
  if (!get) return sws::report_error(SWS_ERR_CUDA, "cuCtxGetCurrent is not available");
  auto lookup = [](unsigned char **addr) -> int {
    void *p = nullptr;
    const cudaError_t le = cudaGetSymbolAddress(&p, sws_noalloc_scratch);
    if (le != cudaSuccess || !p) {
      char msg[256];
      snprintf(msg, sizeof(msg), "cudaGetSymbolAddress of the fixed scratch failed: %s", cudaGetErrorString(le));
      return sws::report_error(SWS_ERR_CUDA, msg);
    }
    *addr = static_cast<unsigned char *>(p);
    return SWS_OK;
  };
  std::lock_guard<std::mutex> lock(g_mu);
  CUcontext cur = nullptr;
  if (get(&cur) != CUDA_SUCCESS) return sws::report_error(SWS_ERR_CUDA, "cuCtxGetCurrent failed");
  if (cur != nullptr && g_addr[dev].ctx == cur && g_addr[dev].addr) {
    *out = g_addr[dev].addr;
    return SWS_OK;
  }
  // first call in this context (the lookup also makes the runtime set the context up)
  unsigned char *addr = nullptr;
  const int s = lookup(&addr);
  if (s) return s;
  if (get(&cur) != CUDA_SUCCESS || !cur) return sws::report_error(SWS_ERR_CUDA, "no current CUDA context");
  g_addr[dev] = Cached{cur, addr};
  *out = addr;
  return SWS_OK;
}

}  // namespace

extern "C" sws_status sws_minimizers_noalloc(const uint8_t *seq, uint64_t n, int k, int w, int mode,
                                             const int64_t *nblocks, uint64_t n_nblocks, void *hash_out,
                                             uint32_t *pos_out, uint64_t capacity, uint64_t *count_out,
                                             void *stream) {
  sws_status s = sws::check_minimizer_args(k, w, mode);
  if (s) return s;
  if (!count_out) return sws::report_error(SWS_ERR_INVALID, "count_out is NULL");
  if (capacity > 0 && (!hash_out || !pos_out)) return sws::report_error(SWS_ERR_INVALID, "hash_out/pos_out is NULL");
  if (n >= (1ull << 32)) return sws::report_error(SWS_ERR_INVALID, "sequences must be shorter than 2^32");
  if (n_nblocks > 0 && !nblocks) return sws::report_error(SWS_ERR_INVALID, "nblocks is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint64_t span = (uint64_t)(w + k - 1);
  const uint64_t nwin = n >= span ? n - span + 1 : 0;
  const uint64_t tiles = sws::mini_lookback_tiles(nwin, w);
  if (tiles == 0) {
    cudaError_t e = cudaMemsetAsync(count_out, 0, sizeof(uint64_t), st);
    return e == cudaSuccess ? SWS_OK : sws::report_error(SWS_ERR_CUDA, cudaGetErrorString(e));
  }
  if (tiles > kNoallocMaxTiles) {
    char msg[256];
    snprintf(msg, sizeof(msg),
             "sws_minimizers_noalloc: %llu bases need %llu tiles, but its fixed scratch holds %llu "
             "(about %llu windows at w = %d); use sws_minimizers",
             (unsigned long long)n, (unsigned long long)tiles, kNoallocMaxTiles,
             (unsigned long long)(kNoallocMaxTiles * (uint64_t)sws::mini_tile_windows(w)), w);
    return sws::report_error(SWS_ERR_INVALID, msg);
  }
  if (!seq) return sws::report_error(SWS_ERR_INVALID, "seq is NULL");
  unsigned char *base = nullptr;
  s = scratch_address(&base);
  if (s) return s;
  // The array keeps the previous call's contents: clear the error word, the tile counter and
  // the status words (barrier summaries are rewritten by every call that uses them); all-ones in
  // count_out marks a call whose ordered output could not be completed.
  cudaError_t e = cudaMemsetAsync(base, 0, kNoallocHeader + tiles * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(count_out, 0xff, sizeof(uint64_t), st);
  if (e != cudaSuccess) return sws::report_error(SWS_ERR_CUDA, cudaGetErrorString(e));
  sws::MiniArgs a{};
  a.seq = seq;
  a.n = n;
  a.k = k;
  a.w = w;
  a.mode = mode;
  a.bar = nblocks;
  a.nbar = n_nblocks;
  a.hash_out = hash_out;
  a.pos_out = pos_out;
  a.capacity = capacity;
  a.count_out = count_out;
  a.err = reinterpret_cast<int *>(base);
  a.tile_counter = reinterpret_cast<unsigned int *>(base + 128);
  a.status = reinterpret_cast<unsigned long long *>(base + kNoallocHeader);
  a.tile_bar = reinterpret_cast<uint2 *>(base + kNoallocHeader + kNoallocMaxTiles * 8);
  e = sws::launch_minimizers_lookback(a, sws::SRC_DNA, sws::BAR_NBLOCK, tiles, st);
  if (e != cudaSuccess) return sws::report_error(SWS_ERR_CUDA, cudaGetErrorString(e));
  return SWS_OK;
}
