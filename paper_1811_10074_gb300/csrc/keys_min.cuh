// keys_min.cuh -- the single-pass sliding-minimum kernel of keys_min.cu (precomputed keys, or
// hashed k-mers of packed bases with optional N-block or read-start barriers), shared by the
// translation units that instantiate its forms.
#pragma once

#include <cstdint>
#include <type_traits>

#include <cuda.h>

#include "../../include/sws.h"
#include "common.cuh"
#include "internal.h"
#include "mini_common.cuh"
#include "tma.cuh"

namespace sws {
namespace keysmin {


constexpr int KNT = 256;                  // threads per CTA
constexpr int KWPT = 16;                  // windows per thread
constexpr int KTILE = KNT * KWPT;         // windows per tile
constexpr int KMAXW = 17;                 // the largest w: a thread's keys fit in 32 registers
constexpr int KROWS = KTILE / 32 + 2;     // rows per stage: the row before, 128, the row after
constexpr int KSTAGE_BYTES = KROWS * 128; // bytes one copy brings
constexpr int KSTAGE_STRIDE = (KSTAGE_BYTES + 1023) / 1024 * 1024;  // 1024-aligned for the swizzle
constexpr int KSTAGES = 3;
constexpr int KSLOTS = 3;                 // pick slots: a tile is placed two tiles after it is counted
constexpr int KCAP = 2560;                // picks a slot holds (more: the tile is placed at once)
constexpr int KSLOT_BYTES = KCAP * 8;     // (key, tile-relative position) per pick
constexpr size_t KSMEM = 1024 + (size_t)KSTAGES * KSTAGE_STRIDE + (size_t)KSLOTS * KSLOT_BYTES;  // 2 CTAs/SM
constexpr size_t KSMEM_DNA = 1024 + (size_t)KSLOTS * KSLOT_BYTES;  // the DNA form: pick slots only
// Barriers of the DNA form: none, N-blocks (windows touching one are dropped), or read starts of
// a batch (windows crossing one are dropped; positions read-local; each read's first pick noted).
constexpr int KB_NONE = 0, KB_NBLOCK = 1, KB_READS = 2;
constexpr int KBMAX = 128;  // barriers of a tile kept in shared memory (more: read from global)
// read batches: a slot also keeps, per pick, the read it is the first pick of (or 0xFFFFFFFF)
constexpr int KSLOT_BYTES_R = KCAP * 12;
constexpr size_t KSMEM_DNA_R = 1024 + (size_t)KSLOTS * KSLOT_BYTES_R;
// 64-bit keys (hashed k-mers with 16 < k <= 29): a key is (hash << cb) | code, the code being the
// k-mer's position + 1 in the tile (cb = 13, k <= 25) or in the thread's frame (cb = 6), so that
// position -1 of the frame has the least code and the plain 64-bit minimum of a window is its
// leftmost least key.  A slot holds KCAP64 picks: the packed keys themselves (cb = 13, outside
// read batches), else hashes and positions, and for read batches the first-pick reads.
constexpr int KCAP64 = 2048;
__host__ __device__ constexpr int slot_bytes(bool k64, int kb) {
  return k64 ? KCAP64 * (12 + (kb == KB_READS ? 4 : 0)) : (kb == KB_READS ? KSLOT_BYTES_R : KSLOT_BYTES);
}
constexpr uint32_t ST_DONE = 0x80000000u;  // status: count published (low bits)
constexpr uint32_t ST_FAIL = 0xC0000000u;  // status: the tile failed
constexpr uint32_t ST_COUNT = 0x3FFFFFFFu;

// Workspace header of one launch (zeroed with the status words).
struct KeysHeader {
  unsigned int ticket;  // next tile
  unsigned int done;    // CTAs that have finished
  unsigned int fail;    // nonzero: some CTA failed
  unsigned int pad;
  unsigned long long total;  // picks of all tiles (written when the last tile is placed)
};

struct KeysArgs {
  const uint32_t *keys;
  // DNA form: the 2-bit packed sequence (4-byte aligned, nbytes bytes) whose hashed canonical
  // k-mers (k <= 16) are the keys
  const uint8_t *seq;
  uint64_t nbytes;
  uint32_t k, kmask;
  // barriers (DNA form): N-blocks int64 [nbar][2], or read offsets int64 [nbar + 1]; per tile the
  // first barrier that can touch it and how many (k_tile_barriers); each read's first pick index
  const int64_t *bar;
  uint64_t nbar;
  const uint2 *tile_bar;
  uint64_t *pick_offsets;
  const unsigned long long *desc;  // a batch graph: sizes of this run (read batches)
  uint32_t m;          // keys (at most 2^32 - 2^14, so that every index below fits 32 bits)
  uint32_t n_full;     // keys in whole 32-key rows (the tensor map's extent)
  uint32_t nwin;       // windows = m - w + 1
  uint32_t num_tiles;
  uint32_t *status;    // one word per tile, zeroed before the launch
  KeysHeader *hdr;     // zeroed before the launch
  uint32_t *key_out;
  unsigned long long *key_out64;  // 64-bit keys
  uint32_t *pos_out;
  uint64_t capacity;
  uint64_t *count_out;
  int *err;
};

__device__ __forceinline__ void st_relaxed_u32(uint32_t *p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Byte offset in a stage of tile-local key q (q = -32 .. KTILE + 31): shared row 1 + q/32 (row 0
// holds the keys before the tile), 16-byte unit swizzled by the row.
__device__ __forceinline__ int stage_offset(int q) {
  const int s = q + 32, row = s >> 5, col = s & 31;
  return row * 128 + ((((col >> 2) ^ (row & 7))) << 4) + ((col & 3) << 2);
}

// DNA form.  Packed word wi (bases 16 wi .. 16 wi + 15) of the sequence; bytes past its end read
// as zero (the k-mers they would touch are past the last one and never used).
__device__ __forceinline__ uint32_t seq_word(const KeysArgs &a, uint32_t wi) {
  const uint64_t b = 4ull * wi;
  if (b + 4 <= a.nbytes) return __ldg(reinterpret_cast<const uint32_t *>(a.seq) + wi);
  uint32_t v = 0;
  for (int i = 0; i < 4; ++i)
    if (b + i < a.nbytes) v |= (uint32_t)a.seq[b + i] << (8 * i);
  return v;
}
// Key of the k-mer at position p: its hashed canonical value (0xFFFFFFFF past the last k-mer).
__device__ __forceinline__ uint32_t dna_key(const KeysArgs &a, uint32_t p) {
  if (p >= a.m) return 0xFFFFFFFFu;
  const uint32_t wi = p >> 4;
  const uint32_t v = __funnelshift_r(seq_word(a, wi), seq_word(a, wi + 1), 2 * (p & 15));  // bases p .. p+15
  return mini::key_value32(mini::kmer32(v, (int)a.k, a.kmask), SWS_MINI_HASH, a.kmask);
}

// Hash of the k-mer at position p for 16 < k <= 29 (~0 past the last k-mer), unpacked.
__device__ __forceinline__ unsigned long long dna_key64(const KeysArgs &a, uint32_t p) {
  if (p >= a.m) return ~0ull;
  const uint32_t wi = p >> 4, sh = 2 * (p & 15);
  const uint32_t w0 = seq_word(a, wi), w1 = seq_word(a, wi + 1), w2 = seq_word(a, wi + 2);
  const unsigned long long x = ((unsigned long long)__funnelshift_r(w1, w2, sh) << 32) | __funnelshift_r(w0, w1, sh);
  const unsigned long long kmask = (1ull << (2 * a.k)) - 1ull;
  return mini::key_value64_wide(mini::kmer64(x, (int)a.k, kmask), SWS_MINI_HASH, (uint32_t)(kmask >> 32));
}

// Minimum of every window j = 0..15 of a thread over distinct 64-bit keys (position in the low
// bits), by the same blocks of W: no tie to break.
template <int W>
__device__ __forceinline__ void window_minima64(const unsigned long long (&X)[32], unsigned long long (&mv)[KWPT]) {
  constexpr int NK = KWPT + W - 1;
  unsigned long long S[KWPT], P[NK];
#pragma unroll
  for (int b = 0; b * W < KWPT; ++b) {
    const int lo = b * W, hi = b * W + W - 1;
    unsigned long long v = X[hi];
    if (hi < KWPT) S[hi] = v;
#pragma unroll
    for (int i = hi - 1; i >= lo; --i) {
      v = X[i] < v ? X[i] : v;
      if (i < KWPT) S[i] = v;
    }
  }
#pragma unroll
  for (int b = 1; b * W <= KWPT + W - 2; ++b) {
    const int lo = b * W;
    const int hi = lo + W - 2 < NK - 1 ? lo + W - 2 : NK - 1;
    unsigned long long v = X[lo];
    P[lo] = v;
#pragma unroll
    for (int i = lo + 1; i <= hi; ++i) {
      v = X[i] < v ? X[i] : v;
      P[i] = v;
    }
  }
#pragma unroll
  for (int j = 0; j < KWPT; ++j) {
    if (j % W == 0) mv[j] = S[j];
    else mv[j] = S[j] < P[j + W - 1] ? S[j] : P[j + W - 1];
  }
}

// Minimum of every window j = 0..15 of a thread (keys X[j .. j+W-1]) and the thread-relative
// position of its leftmost least key, by blocks of W aligned at X[0].
template <int W>
__device__ __forceinline__ void window_minima(const uint32_t (&X)[32], uint32_t (&mv)[KWPT], int (&mp)[KWPT]) {
  constexpr int NK = KWPT + W - 1;
  // suffix minima of the blocks that hold a window start (equal keys: the left one)
  uint32_t Sv[KWPT];
  int Sp[KWPT];
#pragma unroll
  for (int b = 0; b * W < KWPT; ++b) {
    const int lo = b * W, hi = b * W + W - 1;  // hi <= NK - 1
    uint32_t v = X[hi];
    int p = hi;
    if (hi < KWPT) {
      Sv[hi] = v;
      Sp[hi] = p;
    }
#pragma unroll
    for (int i = hi - 1; i >= lo; --i) {
      if (X[i] <= v) {
        v = X[i];
        p = i;
      }
      if (i < KWPT) {
        Sv[i] = v;
        Sp[i] = p;
      }
    }
  }
  // prefix minima of the blocks that hold a window end j + W - 1 of a window j that is not a
  // block start (equal keys: the earlier one stays)
  uint32_t Pv[NK];
  int Pp[NK];
#pragma unroll
  for (int b = 1; b * W <= KWPT + W - 2; ++b) {
    const int lo = b * W;
    const int hi = lo + W - 2 < NK - 1 ? lo + W - 2 : NK - 1;
    uint32_t v = X[lo];
    int p = lo;
    Pv[lo] = v;
    Pp[lo] = p;
#pragma unroll
    for (int i = lo + 1; i <= hi; ++i) {
      if (X[i] < v) {
        v = X[i];
        p = i;
      }
      Pv[i] = v;
      Pp[i] = p;
    }
  }
  // window = suffix part (left) + prefix part (right); the left part wins ties
#pragma unroll
  for (int j = 0; j < KWPT; ++j) {
    if (j % W == 0) {
      mv[j] = Sv[j];
      mp[j] = Sp[j];
    } else {
      const int e = j + W - 1;
      const bool c = Sv[j] <= Pv[e];
      mv[j] = c ? Sv[j] : Pv[e];
      mp[j] = c ? Sp[j] : Pp[e];
    }
  }
}



// This thread's share of the counts of tiles lo .. hi-1, polling (bounded) any not yet published.
// bad: bit 0 = a tile failed, bit 1 = a count was not published within the wait bound.
__device__ __forceinline__ unsigned long long partial_counts(const uint32_t *status, long long lo, long long hi,
                                                             int &bad) {
  unsigned long long sum = 0;
  for (long long j = lo + threadIdx.x; j < hi; j += KNT) {
    uint32_t v = ld_relaxed_u32(&status[j]);
    if (!(v & ST_DONE)) {
      const unsigned long long t0 = tma::now_ns();
      while (!(v & ST_DONE)) {
        if (tma::now_ns() - t0 > tma::kWaitNs) {
          bad |= 2;
          break;
        }
        __nanosleep(100);
        v = ld_relaxed_u32(&status[j]);
      }
    }
    if ((v & ST_FAIL) == ST_FAIL) bad |= 1;
    sum += v & ST_COUNT;
  }
  return sum;
}

// Wait (bounded) until status word *p, last read as v, is published; returns it.
__device__ __forceinline__ uint32_t await_status(const uint32_t *p, uint32_t v, int &bad) {
  if (!(v & ST_DONE)) {
    v = ld_relaxed_u32(p);
    const unsigned long long t0 = tma::now_ns();
    while (!(v & ST_DONE)) {
      if (tma::now_ns() - t0 > tma::kWaitNs) {
        bad |= 2;
        break;
      }
      __nanosleep(100);
      v = ld_relaxed_u32(p);
    }
  }
  if ((v & ST_FAIL) == ST_FAIL) bad |= 1;
  return v;
}

// The same summed over the CTA (barriers inside; every thread gets the total and the bad bits).
__device__ __forceinline__ unsigned long long cta_counts(const uint32_t *status, long long lo, long long hi, int &bad,
                                                         unsigned long long *red, int *flag) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int b = 0;
  unsigned long long sum = partial_counts(status, lo, hi, b);
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) sum += __shfl_xor_sync(kFull, sum, d);
  b = (int)__reduce_or_sync(kFull, (unsigned)b);
  __syncthreads();  // the scratch may still be read from its last use
  if (lane == 0) {
    red[warp] = sum;
    flag[warp] = b;
  }
  __syncthreads();
  sum = 0;
  b = 0;
#pragma unroll
  for (int i = 0; i < KNT / 32; ++i) {
    sum += red[i];
    b |= flag[i];
  }
  bad |= b;
  return sum;
}

// Copy a placed tile's picks from its slot to the output (keys, positions): one pick per thread
// and round, so every warp store covers 128 consecutive bytes.  A slot holds tile-relative
// positions, or read-local ones (read batches) with, after the KCAP picks, the read each pick is
// the first pick of; that read's pick offset is the pick's output index.  The marker array is kept
// all-empty between tiles: set only for first picks, and cleared here once read.
template <int KB, bool K64>
__device__ __forceinline__ void write_slot(unsigned char *slot, uint32_t cnt, uint32_t tile,
                                           unsigned long long base, const KeysArgs &a, bool packed = false,
                                           int vshift = 0) {
  constexpr int CAP = K64 ? KCAP64 : KCAP;
  const uint2 *sl = reinterpret_cast<const uint2 *>(slot);                     // 32-bit keys
  const unsigned long long *sv = reinterpret_cast<const unsigned long long *>(slot);  // 64-bit keys
  const uint32_t *sp = reinterpret_cast<const uint32_t *>(slot + CAP * 8);          // their positions
  uint32_t *first = reinterpret_cast<uint32_t *>(slot + CAP * (K64 ? 12 : 8));
  const uint32_t pos0 = KB == KB_READS ? 0u : tile * (uint32_t)KTILE;
  if (KB == KB_READS)
    for (uint32_t x = threadIdx.x; x < cnt; x += KNT) {
      const uint32_t r = first[x];
      if (r != 0xFFFFFFFFu) {
        a.pick_offsets[r] = base + x;
        first[x] = 0xFFFFFFFFu;
      }
    }
  const bool all = base + cnt <= a.capacity;
  for (uint32_t x = threadIdx.x; x < cnt; x += KNT) {
    const unsigned long long gi = base + x;
    if (all || gi < a.capacity) {
      if constexpr (K64) {
        const unsigned long long v = sv[x];
        if (packed) {  // (hash << 13) | (tile position + 1)
          a.key_out64[gi] = v >> 13;
          a.pos_out[gi] = pos0 + ((uint32_t)v & 8191u) - 1u;
        } else {
          a.key_out64[gi] = v;
          a.pos_out[gi] = pos0 + sp[x];
        }
      } else {
        const uint2 pk = sl[x];
        a.key_out[gi] = pk.x >> vshift;  // 32-bit DNA keys are held shifted left
        a.pos_out[gi] = pos0 + pk.y;
      }
    }
  }
}

template <int W, bool DNA, int KB, bool K64 = false>
__global__ void __launch_bounds__(KNT, 2) k_keys_min(const __grid_constant__ CUtensorMap tmap, KeysArgs a) {
  static_assert(KB == KB_NONE || DNA, "barriers belong to the DNA form");
  static_assert(!K64 || DNA, "64-bit keys belong to the DNA form");
  using V = std::conditional_t<K64, unsigned long long, uint32_t>;
  constexpr int SLOTB = slot_bytes(K64, KB);
  constexpr int CAP = K64 ? KCAP64 : KCAP;  // picks a slot holds
  extern __shared__ __align__(16) unsigned char ksm_raw[];
  // barriers of the tile of stage s in buffer s: (start, end) pairs and the index of the first and
  // their number.  Loaded one tile ahead, read before and after the tile's barrier, rewritten two
  // tiles later (after the next barrier).
  __shared__ long long s_bv[KB != KB_NONE ? KSTAGES : 1][KB != KB_NONE ? 2 * KBMAX : 1];
  __shared__ uint2 s_bt[KSTAGES];
  __shared__ long long s_rs0[KSTAGES];  // read batches: start of the tile's first read (read g_lo)
  __shared__ __align__(8) unsigned long long s_bar[KSTAGES];
  __shared__ uint32_t s_tk[KSTAGES];
  __shared__ int s_issued[KSTAGES];  // a copy was issued into the stage and not yet waited for
  // per iteration parity, per warp: its pick count, failure bits, and its share of the counts
  // before the tile being placed (every sum of pick counts is below 2^32: picks <= keys < 2^32)
  __shared__ uint4 s_sum[2][KNT / 32];
  __shared__ unsigned long long s_red_sync[KNT / 32];
  __shared__ int s_flag_sync[KNT / 32];
  unsigned char *stages = ksm_raw + ((1024u - (tma::smem_u32(ksm_raw) & 1023u)) & 1023u);
  unsigned char *slots = stages + (DNA ? 0 : KSTAGES * KSTAGE_STRIDE);  // the DNA form stages nothing
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (KB == KB_READS && a.desc) {  // a batch graph: this run's sizes
    const uint64_t n = a.desc[BD_TOTAL];
    const uint64_t m = n >= a.k ? n - a.k + 1 : 0;
    a.m = (uint32_t)m;
    a.nwin = (uint32_t)a.desc[BD_NWIN];
    a.num_tiles = (uint32_t)a.desc[BD_TILES];
    a.nbytes = (n + 3) / 4;
    a.nbar = a.desc[BD_NREADS];
  }
  const uint32_t T = a.num_tiles;
  constexpr uint32_t NONE = 0xFFFFFFFFu;
  // 64-bit keys: code bits, and whether a slot keeps the packed keys themselves
  const int cb = K64 && a.k <= 25 ? 13 : 6;
  const bool pk = K64 && KB != KB_READS && cb == 13;
  // 32-bit DNA keys are hashes shifted left by 32 - 2k (the same order), shifted back on output
  const int ks = DNA && !K64 ? 32 - 2 * (int)a.k : 0;
  // barrier i of the list: an N-block [start, end), or a read start (start = end), read i + 1
  auto gstart = [&](uint64_t i) -> long long { return KB == KB_NBLOCK ? a.bar[2 * i] : a.bar[i + 1]; };
  auto gend = [&](uint64_t i) -> long long { return KB == KB_NBLOCK ? a.bar[2 * i + 1] : a.bar[i + 1]; };
  // all threads: tile `tile`'s barriers into buffer `buf` (a tile with more than KBMAX keeps its
  // list in global memory)
  auto load_bars = [&](uint32_t tile, int buf) {
    if (KB == KB_NONE || tile >= T) return;
    const uint2 tbr = a.tile_bar[tile];
    if (t == 0) {
      s_bt[buf] = tbr;
      if (KB == KB_READS) s_rs0[buf] = a.bar[tbr.x];
    }
    if (tbr.y <= (uint32_t)KBMAX)
      for (uint32_t i = t; i < tbr.y; i += KNT) {
        s_bv[buf][2 * i] = gstart(tbr.x + i);
        s_bv[buf][2 * i + 1] = gend(tbr.x + i);
      }
  };

  auto issue = [&](int s, uint32_t tile) {  // thread 0: rows 128 tile - 1 .. 128 tile + 128
    tma::mbar_arrive_expect_tx(&s_bar[s], KSTAGE_BYTES);
    tma::tensor_g2s_2d(stages + s * KSTAGE_STRIDE, &tmap, 0, (int)(tile * (KTILE / 32)) - 1, &s_bar[s]);
  };
  auto set_failed = [&](bool &failed, int why) {  // uniform; thread 0 records the cause
    if (!failed && t == 0) {
      if (why) atomicOr(a.err, why);
      atomicOr(&a.hdr->fail, 1u);
    }
    failed = true;
  };
  if (t == 0) {
    if (!DNA) {
      tma::prefetch_tensormap(&tmap);
#pragma unroll
      for (int s = 0; s < KSTAGES; ++s) tma::mbar_init(&s_bar[s], 1);
      tma::fence_mbar_init();
    }
#pragma unroll
    for (int s = 0; s < KSTAGES; ++s) {
      const uint32_t tk = blockIdx.x + (uint32_t)s * gridDim.x;
      s_tk[s] = tk;
      s_issued[s] = !DNA && tk < T;
      if (!DNA && tk < T) issue(s, tk);
    }
  }
  // thread 0 holds one ticket beyond the stages, taken a tile early so that the atomic's round
  // trip is not on the path of a refill
  const uint32_t first_dyn = (uint32_t)KSTAGES * gridDim.x;  // the first ticket handed out dynamically
  uint32_t spare = t == 0 ? first_dyn + atomicAdd(&a.hdr->ticket, 1u) : 0u;
  if constexpr (KB == KB_READS)  // first-pick markers: empty
    for (int i = t; i < KSLOTS * CAP; i += KNT)
      reinterpret_cast<uint32_t *>(slots + (i / CAP) * SLOTB + CAP * (K64 ? 12 : 8))[i % CAP] = NONE;
  __syncthreads();
  if (KB != KB_NONE) {
    load_bars(s_tk[0], 0);
    __syncthreads();
  }

  uint32_t phases = 0;             // bit s: parity of stage s's next completion
  int run_tile = -1;               // the last tile whose picks were placed ...
  unsigned long long run_end = 0;  // ... and the end of its picks in the output
  // tiles counted but not yet placed (at most KSLOTS - 1), oldest first, with their slots
  int L = 0;
  uint32_t pt0 = NONE, pt1 = NONE, pc0 = 0, pc1 = 0;
  int ps0 = 0, ps1 = 0;
  uint32_t pushes = 0;  // tiles deferred so far: the next one goes to slot pushes % KSLOTS
  bool failed = false;  // uniform across the CTA
  // this thread's 16-byte units in a stage, the same for every tile: its own keys q0 .. q0+15 in
  // shared row 1 + t/2, units 4 (t&1) .. +3, and the next thread's first keys in the same row
  // (t even, units 4..7) or the next row (units 0..3); a unit u of row r sits at u ^ (r & 7)
  const int q0 = t * KWPT;
  const int row_a = 1 + (t >> 1), row_b = row_a + (t & 1);
  const int base_a = row_a * 128 + ((((t & 1) * 4) ^ (row_a & 4)) << 4), r3a = row_a & 3;
  const int base_b = row_b * 128 + (((t & 1 ? 0 : 4) ^ (row_b & 4)) << 4), r3b = row_b & 3;
  for (int it = 0;; ++it) {
    const int s = it % KSTAGES, par = it & 1;
    const uint32_t tile = s_tk[s];
    if (tile >= T) break;
    // the next tile's barriers, visible after this tile's barrier (its ticket was written at least
    // one barrier ago; its buffer was last read two tiles ago, before the previous tile's barrier)
    if (KB != KB_NONE) load_bars(s_tk[(it + 1) % KSTAGES], (it + 1) % KSTAGES);
    // ---- this tile's keys (each thread waits for the copy itself) ---------------------------------
    const bool issued = !DNA && s_issued[s] != 0 && !failed;  // a failed CTA waits for its copies at exit
    // the counts before the oldest deferred tile (placed after this tile's barrier): two status
    // words per thread read now, so that the round trip overlaps this tile's work
    const bool pop = L == KSLOTS - 1 && !failed;
    const int j0 = run_tile + 1 + t;
    uint32_t sv0 = 0, sv1 = 0;
    if (pop && j0 < (int)pt0) sv0 = ld_relaxed_u32(&a.status[j0]);
    if (pop && j0 + KNT < (int)pt0) sv1 = ld_relaxed_u32(&a.status[j0 + KNT]);
    const bool ok = DNA || (issued && tma::mbar_wait_bounded(&s_bar[s], (phases >> s) & 1u));
    const bool wok = __all_sync(kFull, ok);
    const uint32_t tb = tile * (uint32_t)KTILE;  // first window (and key) of the tile
    const uint32_t g0 = tb + (uint32_t)q0;      // this thread's first window
    V mv[KWPT];
    int mp[KWPT];
    unsigned mask = 0;      // windows that store a pick
    unsigned firstm = 0;    // barriers: stored picks that open an N-free stretch or a read
    uint32_t qstart = 0;    // barriers: the first one (in the tile's list) ending after g0 - 1
    // read batches: window g0 + j lies in read g_lo + qstart + (j >= d1) + (j >= d2), which starts
    // at r0, c1 or c2 (unless more than two reads start among the windows: many)
    int d1 = KWPT, d2 = KWPT;
    uint32_t r0 = 0, c1 = 0, c2 = 0;
    bool many = false;
    if (wok) {
      V X[32];
      V xm1;
      if constexpr (K64) {
        // 64-bit keys, (hash << cb) | code: k-mers g0 .. g0+15 from packed words g0/16 .. g0/16 + 2,
        // reversed once; the halo and the k-mer before the warp as in the 32-bit form
        const uint32_t coff = cb == 13 ? (uint32_t)q0 : 0u;  // code of frame position p: coff + p + 1
        const uint32_t wbase = g0 - (uint32_t)lane * KWPT;
        uint32_t pe = 0xFFFFFFFFu;
        if (lane < W - 1) pe = wbase + (uint32_t)(32 * KWPT + lane);
        else if (lane == 31 && wbase > 0) pe = wbase - 1;
        const unsigned long long extra = pe != 0xFFFFFFFFu ? dna_key64(a, pe) : ~0ull;  // unpacked
        const unsigned long long kmask = (1ull << (2 * a.k)) - 1ull;
        const uint32_t khi = (uint32_t)(kmask >> 32);
        if (g0 + KWPT <= a.m && 4ull * ((g0 >> 4) + 3) <= a.nbytes) {
          const uint32_t *sw = reinterpret_cast<const uint32_t *>(a.seq) + (g0 >> 4);
          const uint32_t v0 = __ldg(sw), v1 = __ldg(sw + 1), v2 = __ldg(sw + 2);
          const uint32_t r2 = mini::rev_pairs32(v0), r1 = mini::rev_pairs32(v1), r0w = mini::rev_pairs32(v2);
          const int fsh = 64 - 2 * (int)a.k;  // 6 .. 30 for 16 < k <= 29
          // the hash state stays below 2^(2k): HB bounds its high word's bits (2k - 32); CB = cb
          auto keys16 = [&](auto hb, auto cbc) {
            constexpr int HB = decltype(hb)::value, CB = decltype(cbc)::value;
#pragma unroll
            for (int j = 0; j < KWPT; ++j) {
              const uint32_t lo = j == 0 ? r1 : __funnelshift_r(r0w, r1, 32 - 2 * j);  // bases j+31 .. j+16
              const uint32_t hi = j == 0 ? r2 : __funnelshift_r(r1, r2, 32 - 2 * j);   // bases j+15 .. j
              const unsigned long long fw = ((unsigned long long)(hi >> fsh) << 32) | __funnelshift_r(lo, hi, fsh);
              const unsigned long long w64 =
                  ((unsigned long long)__funnelshift_r(v1, v2, 2 * j) << 32) | __funnelshift_r(v0, v1, 2 * j);
              const unsigned long long rc = ~w64 & kmask;
              X[j] = (mini::wang_mix64_hb<HB>(fw < rc ? fw : rc, khi) << CB) | (unsigned long long)(coff + j + 1);
            }
          };
          if (a.k <= 23) keys16(std::integral_constant<int, 14>{}, std::integral_constant<int, 13>{});
          else if (a.k <= 25) keys16(std::integral_constant<int, 26>{}, std::integral_constant<int, 13>{});
          else keys16(std::integral_constant<int, 26>{}, std::integral_constant<int, 6>{});
        } else {
#pragma unroll
          for (int j = 0; j < KWPT; ++j) {
            const unsigned long long h = dna_key64(a, g0 + (uint32_t)j);
            X[j] = h == ~0ull ? ~0ull : (h << cb) | (unsigned long long)(coff + j + 1);
          }
        }
        // each lane's extra k-mer packed once, with the code it has where it is used: lanes 0 .. W-2
        // hold lane 31's halo (frame positions KWPT + lane), lane 31 the k-mer before the warp
        // (lane 0's frame position -1)
        uint32_t ecode;
        if (cb == 13) ecode = (wbase - tb) + (lane == 31 ? 0u : (uint32_t)(32 * KWPT + lane + 1));
        else ecode = lane == 31 ? 0u : (uint32_t)(KWPT + lane + 1);
        const unsigned long long extra_p = extra == ~0ull ? ~0ull : (extra << cb) | (unsigned long long)ecode;
        xm1 = __shfl_sync(kFull, extra_p, 31);
        // the next lane's keys carry its frame's codes: the same in the tile (cb = 13), 16 less in
        // a thread's frame (cb = 6: a valid key's low word is never all ones, the sentinel's is)
        auto halo = [&](auto cbc) {
          constexpr int CB = decltype(cbc)::value;
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            if (i < W - 1) {
              const unsigned long long dn = __shfl_down_sync(kFull, X[i], 1);
              const unsigned long long ex = __shfl_sync(kFull, extra_p, i);
              unsigned long long nb = dn;
              if (CB == 6) {
                const uint32_t dlo = (uint32_t)dn;
                nb = ((dn >> 32) << 32) | (unsigned long long)(dlo == 0xFFFFFFFFu ? dlo : dlo + (uint32_t)KWPT);
              }
              X[KWPT + i] = lane == 31 ? ex : nb;
            } else {
              X[KWPT + i] = ~0ull;
            }
          }
        };
        if (cb == 13) halo(std::integral_constant<int, 13>{});
        else halo(std::integral_constant<int, 6>{});
      } else if constexpr (DNA) {
        // keys of k-mers g0 .. g0+15 from packed words g0/16 and g0/16 + 1 (g0 is a multiple of 16);
        // the next thread's first W-1 keys by shuffle, lane 31's from the extra k-mers of lanes
        // 0 .. W-2 (the next warp's first W-1); lane 31's own extra k-mer is the one before the
        // warp's first, which lane 0 needs (xm1).  Each lane hashes at most one extra k-mer.
        const uint32_t wbase = g0 - (uint32_t)lane * KWPT;  // the warp's first k-mer
        uint32_t pe = 0xFFFFFFFFu;
        if (lane < W - 1) pe = wbase + (uint32_t)(32 * KWPT + lane);
        else if (lane == 31 && wbase > 0) pe = wbase - 1;
        const uint32_t ex0 = pe != 0xFFFFFFFFu ? dna_key(a, pe) : 0xFFFFFFFFu;
        const uint32_t extra = ex0 == 0xFFFFFFFFu ? ex0 : ex0 << ks;
        if (g0 + KWPT <= a.m && 4ull * ((g0 >> 4) + 2) <= a.nbytes) {
          const uint32_t *sw = reinterpret_cast<const uint32_t *>(a.seq) + (g0 >> 4);
          const uint32_t v0 = __ldg(sw), v1 = __ldg(sw + 1);
          // the 32 bases reversed once (base i at bits 62 - 2i of rhi:rlo): the forward k-mer at j
          // is then one funnel shift and one shift, with no per-k-mer reversal
          const uint32_t rhi = mini::rev_pairs32(v0), rlo = mini::rev_pairs32(v1);
          const int fsh = 32 - 2 * (int)a.k;  // = ks
          const uint32_t hm = 0xFFFFFFFFu << fsh;
#pragma unroll
          for (int j = 0; j < KWPT; ++j) {
            const uint32_t rc = ~__funnelshift_r(v0, v1, 2 * j) & a.kmask;
            const uint32_t fw = (j == 0 ? rhi : __funnelshift_r(rlo, rhi, 32 - 2 * j)) >> fsh;
            X[j] = mini::wang_mix32_hi((fw < rc ? fw : rc) << fsh, hm);
          }
        } else {
#pragma unroll
          for (int j = 0; j < KWPT; ++j) {
            const uint32_t h = dna_key(a, g0 + (uint32_t)j);
            X[j] = h == 0xFFFFFFFFu ? h : h << ks;
          }
        }
        xm1 = __shfl_sync(kFull, extra, 31);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          if (i < W - 1) {
            const uint32_t dn = __shfl_down_sync(kFull, X[i], 1);
            const uint32_t ex = __shfl_sync(kFull, extra, i);
            X[KWPT + i] = lane == 31 ? ex : dn;
          } else {
            X[KWPT + i] = 0xFFFFFFFFu;
          }
        }
      } else {
        const unsigned char *st = stages + s * KSTAGE_STRIDE;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const uint4 u = *reinterpret_cast<const uint4 *>(st + base_a + ((c ^ r3a) << 4));
          X[4 * c] = u.x;
          X[4 * c + 1] = u.y;
          X[4 * c + 2] = u.z;
          X[4 * c + 3] = u.w;
        }
        constexpr int NU = (W - 1 + 3) / 4;  // 16-byte units of the next thread's keys needed
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if (c < NU) {
            const uint4 u = *reinterpret_cast<const uint4 *>(st + base_b + ((c ^ r3b) << 4));
            X[16 + 4 * c] = u.x;
            X[16 + 4 * c + 1] = u.y;
            X[16 + 4 * c + 2] = u.z;
            X[16 + 4 * c + 3] = u.w;
          } else {
            X[16 + 4 * c] = X[16 + 4 * c + 1] = X[16 + 4 * c + 2] = X[16 + 4 * c + 3] = 0xFFFFFFFFu;
          }
        }
        xm1 = lane == 0 ? *reinterpret_cast<const uint32_t *>(st + stage_offset(q0 - 1)) : 0u;
        if (g0 + KWPT + W - 1 > a.n_full) {  // keys of the final partial row (or past the end)
#pragma unroll
          for (int i = 0; i < KWPT + W - 1; ++i) {
            const uint32_t gi = g0 + (uint32_t)i;
            if (gi >= a.n_full) X[i] = gi < a.m ? a.keys[gi] : 0xFFFFFFFFu;
          }
          if (lane == 0 && g0 >= 1 && g0 - 1 >= a.n_full && g0 - 1 < a.m) xm1 = a.keys[g0 - 1];
        }
      }
      if constexpr (K64) {
        window_minima64<W>(X, mv);
#pragma unroll
        for (int j = 0; j < KWPT; ++j)
          mp[j] = (int)(((uint32_t)mv[j] & ((1u << cb) - 1u)) - (cb == 13 ? (uint32_t)q0 : 0u)) - 1;
      } else {
        window_minima<W>(X, mv, mp);
      }
      // A window stores a pick when its pick (the position of its leftmost least key) differs
      // from the previous window's.  The window before this thread's first is the previous lane's
      // last (its position shifted to this thread's frame).  For lane 0 of a warp it is the key
      // before the warp (position -1) with keys 0 .. w-2, and window 0 (keys 0 .. w-1) is one
      // block of the combine: if its leftmost least key is key w-1 the two picks differ, else that
      // key is also the leftmost least of keys 0 .. w-2 and the picks agree unless the key before
      // is not larger.
      const int pp = __shfl_up_sync(kFull, mp[KWPT - 1], 1) - KWPT;
      const bool same0 = lane == 0 ? (mp[0] <= W - 2 && xm1 > mv[0]) : mp[0] == pp;
      mask = (!same0 || g0 == 0) ? 1u : 0u;
#pragma unroll
      for (int j = 1; j < KWPT; ++j) mask |= (unsigned)(mp[j] != mp[j - 1]) << j;
      const int left = (int)(a.nwin - g0);  // windows of this thread inside the sequence (if > 0)
      if (g0 >= a.nwin) mask = 0;
      else if (left < KWPT) mask &= (1u << left) - 1u;
      if constexpr (KB != KB_NONE) {
        // a window touching a barrier is dropped; the first window after a dropped one always
        // stores its pick (a new N-free stretch, or a new read)
        const uint2 tbr = s_bt[s];
        const uint32_t nb = tbr.y;
        const long long span = (long long)W + a.k - 1;
        const long long pf = (long long)g0 - 1;
        // the list from shared memory, or (more than KBMAX barriers) from global memory: one
        // uniform choice per tile, each accessor inlined into its own copy of the walk
        auto walk = [&](auto bst, auto ben) -> unsigned {
          uint32_t q = 0, hi = nb;
          while (q < hi) {
            const uint32_t mid = (q + hi) >> 1;
            if (ben(mid) > pf) hi = mid;
            else q = mid + 1;
          }
          qstart = q;
          if constexpr (KB == KB_READS) {
            r0 = (uint32_t)(q == 0 ? s_rs0[s] : bst(q - 1));
            if (q < nb) {
              c1 = (uint32_t)bst(q);
              d1 = c1 - g0 < (uint32_t)KWPT ? (int)(c1 - g0) : KWPT;
            }
            if (q + 1 < nb) {
              c2 = (uint32_t)bst(q + 1);
              d2 = c2 - g0 < (uint32_t)KWPT ? (int)(c2 - g0) : KWPT;
            }
            many = q + 2 < nb && bst(q + 2) - (long long)g0 < KWPT;
          }
          // windows g0 - 1 .. g0 + 15 as bits 0 .. 16: barrier [bs, be) drops the windows
          // [bs - span + 1, be - 1]; the barriers from q on, while they reach this thread's windows
          unsigned v = (2u << KWPT) - 1u;
          for (uint32_t qq = q; qq < nb; ++qq) {
            const long long bs = bst(qq);
            if (bs - span + 1 > (long long)g0 + KWPT - 1) break;  // it and every later one start beyond
            const long long lo = bs - span + 1 - pf, hi2 = ben(qq) - 1 - pf;
            if (hi2 >= 0) {
              const int l = lo < 0 ? 0 : (int)lo, h = hi2 > KWPT ? KWPT : (int)hi2;
              v &= ~(((2u << h) - 1u) & ~((1u << l) - 1u));
            }
          }
          return v;
        };
        unsigned v17 =
            nb <= (uint32_t)KBMAX
                ? walk([&](uint32_t i) -> long long { return s_bv[s][2 * i]; },
                       [&](uint32_t i) -> long long { return s_bv[s][2 * i + 1]; })
                : walk([&](uint32_t i) -> long long { return gstart(tbr.x + i); },
                       [&](uint32_t i) -> long long { return gend(tbr.x + i); });
        const long long lim = (long long)a.nwin - pf;  // bits of windows past the last are dropped
        if (lim <= 0) v17 = 0;
        else if (lim <= KWPT) v17 &= (1u << lim) - 1u;
        if (g0 == 0) v17 &= ~1u;  // no window before the first
        const unsigned vmask = v17 >> 1;
        const bool pvalid = v17 & 1u;
        const unsigned prevv = ((vmask << 1) | (pvalid ? 1u : 0u)) & ((1u << KWPT) - 1u);
        firstm = vmask & ~prevv;
        mask = (mask | firstm) & vmask;
      }
    }
    const uint32_t cnt = __popc(mask);
    uint32_t inc = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t u = __shfl_up_sync(kFull, inc, d);
      if (lane >= d) inc += u;
    }
    // the counts before the oldest deferred tile, placed below once the barrier has summed them
    int bad = 0;
    uint32_t part = 0;
    if (pop) {
      if (j0 < (int)pt0) part += await_status(&a.status[j0], sv0, bad) & ST_COUNT;
      if (j0 + KNT < (int)pt0) part += await_status(&a.status[j0 + KNT], sv1, bad) & ST_COUNT;
      if (run_tile + 1 + 2 * KNT < (int)pt0)  // a long gap (rare): the rest
        part += (uint32_t)partial_counts(a.status, run_tile + 1 + 2 * KNT, pt0, bad);
    }
    part = __reduce_add_sync(kFull, part);
    bad = (int)__reduce_or_sync(kFull, (unsigned)(bad | (issued && !wok ? 4 : 0)));
    if (lane == 31) s_sum[par][warp] = make_uint4(inc, (uint32_t)bad, part, 0u);
    __syncthreads();  // the one barrier of a tile
    // lane i reads warp i's summary; sums and this warp's offset by shuffles
    const uint4 v = lane < KNT / 32 ? s_sum[par][lane] : make_uint4(0u, 0u, 0u, 0u);
    const uint32_t tot = __reduce_add_sync(kFull, v.x);
    const int flags = (int)__reduce_or_sync(kFull, v.y);
    const unsigned long long between = __reduce_add_sync(kFull, v.z);
    uint32_t wi = v.x;
#pragma unroll
    for (int d = 1; d < KNT / 32; d <<= 1) {
      const uint32_t u = __shfl_up_sync(kFull, wi, d);
      if (lane >= d) wi += u;
    }
    const uint32_t woff = __shfl_sync(kFull, wi - v.x, warp);
    if (issued) {
      if (flags & 4) {
        set_failed(failed, DEVERR_COPY_TIMEOUT);  // the copy did not land in time
      } else {
        phases ^= 1u << s;
        if (t == 0) s_issued[s] = 0;
      }
    }
    if (flags & 3) set_failed(failed, (flags & 2) ? DEVERR_LOOKBACK_TIMEOUT : 0);
    // ---- publish this tile's count and refill the stage with the next ticket's tile ---------------
    if (t == 0) {
      st_relaxed_u32(&a.status[tile], failed ? ST_FAIL : (ST_DONE | tot));
      const uint32_t nt = spare;
      spare = first_dyn + atomicAdd(&a.hdr->ticket, 1u);
      s_tk[s] = nt;
      if (!DNA && nt < T && !failed && !s_issued[s]) {
        s_issued[s] = 1;
        tma::fence_proxy_async_smem();
        issue(s, nt);
      }
    }
    if (failed) continue;
    // ---- place the oldest deferred tile: the end of this CTA's tile before it plus the counts of
    //      every tile in between (published two tiles ago or earlier) ----------------------------------
    if (pop) {
      const unsigned long long base = run_end + between;
      write_slot<KB, K64>(slots + ps0 * SLOTB, pc0, pt0, base, a, pk, ks);
      if (t == 0 && pt0 == T - 1) a.hdr->total = base + pc0;
      run_tile = pt0;
      run_end = base + pc0;
      pt0 = pt1;
      pc0 = pc1;
      ps0 = ps1;
      --L;
    }
    if (tot <= (uint32_t)CAP) {
      // ---- defer this tile: its picks wait in the next slot -----------------------------------------
      const int sl = (int)(pushes % KSLOTS);
      ++pushes;
      unsigned char *slotp = slots + sl * SLOTB;
      uint32_t idx = woff + inc - cnt;  // this thread's first place in the slot
      auto put = [&](uint32_t i, V v, uint32_t posf) {
        if constexpr (K64) {
          reinterpret_cast<unsigned long long *>(slotp)[i] = v >> cb;
          reinterpret_cast<uint32_t *>(slotp + CAP * 8)[i] = posf;
        } else {
          reinterpret_cast<uint2 *>(slotp)[i] = make_uint2(v, posf);
        }
      };
      if constexpr (KB == KB_READS) {
        // read-local positions; a first pick of a read also marks that read in the slot's marker
        // array (empty elsewhere)
        uint32_t *fst = reinterpret_cast<uint32_t *>(slotp + CAP * (K64 ? 12 : 8));
        const uint2 tbr = s_bt[s];
        if (!many) {
          // at most two reads start among the windows: window j's read starts at r0, c1 or c2
          const uint32_t pbq = tb + (uint32_t)q0;
          const uint32_t pb0 = pbq - r0, pb1 = pbq - c1, pb2 = pbq - c2;
          const uint32_t idx0 = idx;
#pragma unroll
          for (int j = 0; j < KWPT; ++j) {
            if ((mask >> j) & 1u) {
              const uint32_t pb = j >= d2 ? pb2 : (j >= d1 ? pb1 : pb0);
              put(idx, mv[j], pb + (uint32_t)mp[j]);
              ++idx;
            }
          }
          for (unsigned f = firstm; f; f &= f - 1u) {
            const int j = __ffs(f) - 1;
            fst[idx0 + __popc(mask & ((1u << j) - 1u))] = tbr.x + qstart + (uint32_t)((j >= d1) + (j >= d2));
          }
        } else {
          const bool in_smem = tbr.y <= (uint32_t)KBMAX;
          uint32_t qq = qstart;
          for (int j = 0; j < KWPT; ++j) {
            if ((mask >> j) & 1u) {
              while (qq < tbr.y && (in_smem ? s_bv[s][2 * qq + 1] : gend(tbr.x + qq)) <= (long long)g0 + j) ++qq;
              // read g_lo + qq starts where barrier qq - 1 is
              const uint32_t rs = (uint32_t)(qq == 0 ? s_rs0[s] : (in_smem ? s_bv[s][2 * qq - 2] : gstart(tbr.x + qq - 1)));
              put(idx, mv[j], tb + (uint32_t)(q0 + mp[j]) - rs);
              if ((firstm >> j) & 1u) fst[idx] = tbr.x + qq;
              ++idx;
            }
          }
        }
      } else if (K64 && pk) {
        // the packed keys carry their tile positions
#pragma unroll
        for (int j = 0; j < KWPT; ++j) {
          if ((mask >> j) & 1u) {
            reinterpret_cast<unsigned long long *>(slotp)[idx] = mv[j];
            ++idx;
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < KWPT; ++j) {
          if ((mask >> j) & 1u) {
            put(idx, mv[j], (uint32_t)(q0 + mp[j]));
            ++idx;
          }
        }
      }
      if (L == 0) {
        pt0 = tile;
        pc0 = tot;
        ps0 = sl;
      } else {
        pt1 = tile;
        pc1 = tot;
        ps1 = sl;
      }
      ++L;
    } else {
      // ---- a tile with more picks than a slot holds: place every deferred tile, then this one,
      //      now (the threads write this tile's picks straight from their registers) -----------------
      while (L > 0 && !failed) {
        int b2 = 0;
        const unsigned long long btw = cta_counts(a.status, run_tile + 1, pt0, b2, s_red_sync, s_flag_sync);
        if (b2) {
          set_failed(failed, (b2 & 2) ? DEVERR_LOOKBACK_TIMEOUT : 0);
          break;
        }
        const unsigned long long base = run_end + btw;
        write_slot<KB, K64>(slots + ps0 * SLOTB, pc0, pt0, base, a, pk, ks);
        if (t == 0 && pt0 == T - 1) a.hdr->total = base + pc0;
        run_tile = pt0;
        run_end = base + pc0;
        pt0 = pt1;
        pc0 = pc1;
        ps0 = ps1;
        --L;
      }
      if (!failed) {
        int b2 = 0;
        const unsigned long long btw = cta_counts(a.status, run_tile + 1, tile, b2, s_red_sync, s_flag_sync);
        if (b2) {
          set_failed(failed, (b2 & 2) ? DEVERR_LOOKBACK_TIMEOUT : 0);
        } else {
          const unsigned long long base = run_end + btw;
          unsigned long long r = base + woff + inc - cnt;
          const uint2 tbr = KB == KB_READS ? s_bt[s] : make_uint2(0u, 0u);
          uint32_t qq = qstart;
#pragma unroll
          for (int j = 0; j < KWPT; ++j) {
            if ((mask >> j) & 1u) {
              uint32_t pos = tb + (uint32_t)(q0 + mp[j]);
              if (KB == KB_READS) {
                const bool in_smem = tbr.y <= (uint32_t)KBMAX;
                uint32_t rd;
                if (!many) {
                  const int i = (j >= d1) + (j >= d2);
                  rd = tbr.x + qstart + (uint32_t)i;
                  pos -= i == 0 ? r0 : i == 1 ? c1 : c2;
                } else {
                  while (qq < tbr.y && (in_smem ? s_bv[s][2 * qq + 1] : gend(tbr.x + qq)) <= (long long)g0 + j) ++qq;
                  rd = tbr.x + qq;
                  pos -= (uint32_t)(qq == 0 ? s_rs0[s] : (in_smem ? s_bv[s][2 * qq - 2] : gstart(tbr.x + qq - 1)));
                }
                if ((firstm >> j) & 1u) a.pick_offsets[rd] = r;
              }
              if (r < a.capacity) {
                if constexpr (K64) a.key_out64[r] = mv[j] >> cb;
                else a.key_out[r] = mv[j] >> ks;
                a.pos_out[r] = pos;
              }
              ++r;
            }
          }
          if (t == 0 && tile == T - 1) a.hdr->total = base + tot;
          run_tile = tile;
          run_end = base + tot;
        }
      }
    }
  }
  // ---- the deferred tiles left at the end ---------------------------------------------------------
  while (L > 0 && !failed) {
    int b2 = 0;
    const unsigned long long btw = cta_counts(a.status, run_tile + 1, pt0, b2, s_red_sync, s_flag_sync);
    if (b2) {
      set_failed(failed, (b2 & 2) ? DEVERR_LOOKBACK_TIMEOUT : 0);
      break;
    }
    const unsigned long long base = run_end + btw;
    write_slot<KB, K64>(slots + ps0 * SLOTB, pc0, pt0, base, a, pk, ks);
    if (t == 0 && pt0 == T - 1) a.hdr->total = base + pc0;
    run_tile = pt0;
    run_end = base + pc0;
    pt0 = pt1;
    pc0 = pc1;
    ps0 = ps1;
    --L;
  }
  if (t == 0) {
    // copies still in flight after a time-out: give them a bounded chance to land
    if (failed)
      for (int s = 0; s < KSTAGES; ++s)
        if (s_issued[s]) tma::mbar_wait_bounded(&s_bar[s], (phases >> s) & 1u);
    // the last CTA to finish publishes the count, unless some CTA failed
    __threadfence();
    const unsigned done = atomicAdd(&a.hdr->done, 1u);
    if (done == gridDim.x - 1) {
      __threadfence();
      const unsigned fail = atomicAdd(&a.hdr->fail, 0u);
      if (fail == 0) *a.count_out = *reinterpret_cast<volatile unsigned long long *>(&a.hdr->total);
    }
  }
}

template <int W, bool DNA, int KB, bool K64 = false>
cudaError_t launch_w_keys(const CUtensorMap &map, const KeysArgs &a, int num_sms, cudaStream_t st) {
  auto kern = k_keys_min<W, DNA, KB, K64>;
  constexpr size_t smem = !DNA ? KSMEM : 1024 + (size_t)KSLOTS * slot_bytes(K64, KB);
  static int per_sm[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int nb = (dev >= 0 && dev < 64) ? per_sm[dev] : 0;
  if (nb == 0) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, KNT, smem);
    if (e != cudaSuccess) return e;
    if (nb < 1) return cudaErrorInvalidConfiguration;
    if (dev >= 0 && dev < 64) per_sm[dev] = nb;
  }
  uint64_t grid = (uint64_t)num_sms * (uint64_t)nb;
  if (grid > a.num_tiles) grid = a.num_tiles;
  kern<<<(unsigned)grid, KNT, smem, st>>>(map, a);
  return cudaGetLastError();
}


// The DNA form for window lengths 4..17, one barrier kind each (keys_min_dna*.cu).
cudaError_t launch_dna_none(const KeysArgs &a, int w, int num_sms, cudaStream_t st);
cudaError_t launch_dna_nblock(const KeysArgs &a, int w, int num_sms, cudaStream_t st);
cudaError_t launch_dna_reads(const KeysArgs &a, int w, int num_sms, cudaStream_t st);
// The same with 64-bit keys (16 < k <= 29; keys_min_dna64*.cu).
cudaError_t launch_dna64_none(const KeysArgs &a, int w, int num_sms, cudaStream_t st);
cudaError_t launch_dna64_nblock(const KeysArgs &a, int w, int num_sms, cudaStream_t st);
cudaError_t launch_dna64_reads(const KeysArgs &a, int w, int num_sms, cudaStream_t st);

}  // namespace keysmin
}  // namespace sws
