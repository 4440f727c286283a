// keys_min.cu -- the paper's timed task (Sec. 4) on the GPU: the deduplicated sliding minimum of
// a precomputed key array (Eq. 2 with (+) = min over keys ordered by (value, position), picks of
// consecutive windows stored once, Sec. 2.4), for windows of w = 1..17 keys, in ONE pass over the
// keys with the picks written in position order.
//
// Tiles.  A tile is 4096 consecutive windows; thread t of the 256-thread CTA owns windows
// 16t .. 16t+15 of the tile and reads keys 16t .. 16t+w+14 of it (its own 16 and the first w-1 of
// the next thread's).  A tile's keys arrive in shared memory by one 2-D TMA copy of 130 rows of
// 128 bytes (the key array viewed as rows of 32 keys): the row before the tile (its last key
// decides whether the tile's first window stores a pick), the tile's 128 rows, and the row after
// (the halo of the last windows).  The 128-byte swizzle puts 16-byte unit u of shared row r at
// unit u ^ (r & 7), so each quarter-warp's 16-byte reads fall in distinct bank groups.  Keys of
// a final partial row are not in the tensor map; the threads that need them load them directly.
//
// Window minima.  Blocks of w keys aligned at the thread's first key: window j is the suffix of
// block j/w from j combined with the prefix of the next block up to j+w-1 (the block combine of
// Eq. 2 with blocks of exactly w, van Herk / Gil-Werman), about three compares per window, all in
// registers.  Keys compare by value and carry their position (a compile-time constant): a suffix
// step takes an equal key (the left one), a prefix step does not, and the suffix part wins ties
// against the prefix part, so every window knows its leftmost least key.  A window stores a pick
// when its pick differs from the previous window's pick, which the values decide: its least key
// differs from the previous window's, or equals it while the previous pick was the previous
// window's first key (which has left).
//
// Order.  CTA b of G takes tiles b, b + G and b + 2G first (so that an input of a few tiles per CTA
// is spread evenly), then tiles 3G, 3G + 1, ... by an atomic ticket, so each CTA takes its tiles in
// increasing order.  A tile's pick count goes to its status word as soon as it is known; the
// tile's picks wait in one of three shared-memory slots while the CTA computes its next two
// tiles, and then the CTA finds their output offset as the end of its own previous tile's picks
// plus the counts of all tiles between the two -- published by then, since each is published
// right after it is computed and every ticket below this one is held by a running CTA (the two
// tiles of slack absorb CTAs that run behind).  That costs each thread one or two reads of hot
// status words per tile, issued before the tile's work; there is no staging area, no second
// pass, no inclusive-prefix chain, and one CTA barrier per tile.  A tile with more picks than a
// slot holds is placed at once, after the deferred ones.  Every wait is bounded: a wait that runs out records the fault, the CTA publishes a
// failure mark instead of its later counts, and every tile after it then fails as well (its
// offset would include a missing count), so the final count is never written.
#include <cstdint>
#include <cstdio>
#include <mutex>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "keys_min.cuh"

namespace sws {

using namespace keysmin;

namespace {

using EncodeTiledK = PFN_cuTensorMapEncodeTiled_v12000;

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime (no -lcuda).
EncodeTiledK encode_tiled_k() {
  static EncodeTiledK fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledK>(p);
  });
  return fn;
}

}  // namespace


bool dna_min_fits(uint64_t n, int k, int w, int mode) {
  if (mode != SWS_MINI_HASH || k < 1 || k > 29 || w < 4 || w > KMAXW || n < (uint64_t)k + 32) return false;
  const uint64_t m = n - (uint64_t)k + 1;
  return m <= (1ull << 32) - (1ull << 14) && (uint64_t)w <= m;
}

bool dna_min_applies(const uint8_t *seq, uint64_t n, int k, int w, int mode) {
  return (reinterpret_cast<uintptr_t>(seq) & 3u) == 0 && dna_min_fits(n, k, w, mode);
}

int dna_min_tile_windows() { return KTILE; }

static uint64_t dna_tiles(uint64_t n, int k, int w) {
  const uint64_t m = n - (uint64_t)k + 1;
  return (m - (uint64_t)w + KTILE) / KTILE;  // ceil(nwin / KTILE), nwin = m - w + 1
}

uint64_t dna_min_ws_bytes(uint64_t n, int k, int w) {
  const uint64_t m = n - (uint64_t)k + 1;
  return (keys_min_ws_bytes(m, w) + 255) / 256 * 256 + dna_tiles(n, k, w) * sizeof(uint2);
}

cudaError_t launch_dna_min(const DnaMinArgs &d, void *ws, int *err, int num_sms, cudaStream_t st) {
  if (!dna_min_applies(d.seq, d.n, d.k, d.w, SWS_MINI_HASH)) return cudaErrorInvalidValue;
  const uint64_t m = d.n - (uint64_t)d.k + 1;  // k-mers: the keys
  const uint64_t nwin = m - (uint64_t)d.w + 1;
  const uint64_t tiles = dna_tiles(d.n, d.k, d.w);
  cudaError_t e = cudaMemsetAsync(ws, 0, keys_min_ws_bytes(m, d.w), st);
  if (e != cudaSuccess) return e;
  KeysArgs a{};
  a.seq = d.seq;
  a.nbytes = (d.n + 3) / 4;
  a.k = (uint32_t)d.k;
  a.kmask = d.k <= 16 ? 0xFFFFFFFFu >> (32 - 2 * d.k) : 0u;
  a.m = (uint32_t)m;
  a.n_full = (uint32_t)m;
  a.nwin = (uint32_t)nwin;
  a.num_tiles = (uint32_t)tiles;
  a.hdr = static_cast<KeysHeader *>(ws);
  a.status = reinterpret_cast<uint32_t *>(static_cast<char *>(ws) + 256);
  a.key_out = d.key_out;
  a.key_out64 = d.key_out64;
  a.pos_out = d.pos_out;
  a.capacity = d.capacity;
  a.count_out = d.count_out;
  a.err = err;
  a.bar = d.bar;
  a.nbar = d.nbar;
  a.pick_offsets = d.pick_offsets;
  a.desc = d.desc;
  int kb = KB_NONE;
  if (d.barrier == BAR_NBLOCK && d.nbar > 0) kb = KB_NBLOCK;
  if (d.barrier == BAR_READS) kb = KB_READS;
  if (kb != KB_NONE) {
    // per tile the barriers that can touch its windows (tiles of KTILE windows)
    uint2 *tile_bar = reinterpret_cast<uint2 *>(static_cast<char *>(ws) + (keys_min_ws_bytes(m, d.w) + 255) / 256 * 256);
    MiniArgs ma{};
    ma.bar = d.bar;
    ma.nbar = d.nbar;
    ma.tile_bar = tile_bar;
    ma.desc = d.desc;
    if (tile_barriers_needed(ma, SRC_DNA, d.barrier))
      e = launch_tile_barriers(ma, SRC_DNA, d.barrier, tiles, KTILE, d.w + d.k - 1, st);
    else  // one read: no barrier between its windows
      e = cudaMemsetAsync(tile_bar, 0, tiles * sizeof(uint2), st);
    if (e != cudaSuccess) return e;
    a.tile_bar = tile_bar;
  }
  if (d.k > 16) {  // 64-bit keys
    if (kb == KB_NBLOCK) return launch_dna64_nblock(a, d.w, num_sms, st);
    if (kb == KB_READS) return launch_dna64_reads(a, d.w, num_sms, st);
    return launch_dna64_none(a, d.w, num_sms, st);
  }
  if (kb == KB_NBLOCK) return launch_dna_nblock(a, d.w, num_sms, st);
  if (kb == KB_READS) return launch_dna_reads(a, d.w, num_sms, st);
  return launch_dna_none(a, d.w, num_sms, st);
}

bool keys_min_applies(const uint32_t *keys, uint64_t m, int w) {
  return w >= 1 && w <= KMAXW && m >= 32 && m <= (1ull << 32) - (1ull << 14) && (uint64_t)w <= m &&
         (reinterpret_cast<uintptr_t>(keys) & 15u) == 0 && encode_tiled_k() != nullptr;
}

uint64_t keys_min_ws_bytes(uint64_t m, int w) {
  const uint64_t nwin = m - (uint64_t)w + 1;
  return 256 + (nwin + KTILE - 1) / KTILE * 4;
}

cudaError_t launch_keys_min(const uint32_t *keys, uint64_t m, int w, uint32_t *key_out, uint32_t *pos_out,
                            uint64_t capacity, uint64_t *count_out, void *ws, int *err, int num_sms,
                            cudaStream_t st) {
  if (!keys_min_applies(keys, m, w)) return cudaErrorInvalidValue;
  const uint64_t nwin = m - (uint64_t)w + 1;
  const uint64_t tiles = (nwin + KTILE - 1) / KTILE;
  const uint64_t rows = m / 32;
  CUtensorMap map;
  const cuuint64_t gdim[2] = {32, rows};
  const cuuint64_t gstride[1] = {128};
  const cuuint32_t box[2] = {32, (cuuint32_t)KROWS};
  const cuuint32_t estr[2] = {1, 1};
  if (encode_tiled_k()(&map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<uint32_t *>(keys), gdim, gstride, box,
                       estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(ws, 0, keys_min_ws_bytes(m, w), st);
  if (e != cudaSuccess) return e;
  KeysArgs a{};
  a.keys = keys;
  a.m = (uint32_t)m;
  a.n_full = (uint32_t)(rows * 32);
  a.nwin = (uint32_t)nwin;
  a.num_tiles = (uint32_t)tiles;
  a.hdr = static_cast<KeysHeader *>(ws);
  a.status = reinterpret_cast<uint32_t *>(static_cast<char *>(ws) + 256);
  a.key_out = key_out;
  a.pos_out = pos_out;
  a.capacity = capacity;
  a.count_out = count_out;
  a.err = err;
  switch (w) {
    case 1: return launch_w_keys<1, false, KB_NONE>(map, a, num_sms, st);
    case 2: return launch_w_keys<2, false, KB_NONE>(map, a, num_sms, st);
    case 3: return launch_w_keys<3, false, KB_NONE>(map, a, num_sms, st);
    case 4: return launch_w_keys<4, false, KB_NONE>(map, a, num_sms, st);
    case 5: return launch_w_keys<5, false, KB_NONE>(map, a, num_sms, st);
    case 6: return launch_w_keys<6, false, KB_NONE>(map, a, num_sms, st);
    case 7: return launch_w_keys<7, false, KB_NONE>(map, a, num_sms, st);
    case 8: return launch_w_keys<8, false, KB_NONE>(map, a, num_sms, st);
    case 9: return launch_w_keys<9, false, KB_NONE>(map, a, num_sms, st);
    case 10: return launch_w_keys<10, false, KB_NONE>(map, a, num_sms, st);
    case 11: return launch_w_keys<11, false, KB_NONE>(map, a, num_sms, st);
    case 12: return launch_w_keys<12, false, KB_NONE>(map, a, num_sms, st);
    case 13: return launch_w_keys<13, false, KB_NONE>(map, a, num_sms, st);
    case 14: return launch_w_keys<14, false, KB_NONE>(map, a, num_sms, st);
    case 15: return launch_w_keys<15, false, KB_NONE>(map, a, num_sms, st);
    case 16: return launch_w_keys<16, false, KB_NONE>(map, a, num_sms, st);
    case 17: return launch_w_keys<17, false, KB_NONE>(map, a, num_sms, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sws
