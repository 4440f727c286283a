// minimizer.cu -- k-mers, canonical hashed k-mers and (w,k)-minimizers (Sec. 2.4), fused into
// one pass per CTA tile.
//
// A k-mer is the sliding sum of k bases under concatenation (Sec. 2.4).  With the packed layout
// (base i at bits 2i.. of the little-endian bit stream) a 32- or 64-bit funnel shift at bit 2i
// yields bases i, i+1, ... in ascending bit pairs, which is already the reverse complement after
// a bitwise NOT; the forward k-mer is the same word with its 2-bit groups reversed.  So each
// k-mer costs O(1) no matter what k is -- the "recurrent" form of a sliding sum (Sec. 5).
//
// Minimizers: for each window p the least key among k-mers p .. p+w-1, keys ordered by (value,
// position), is the sliding minimum of Eq. 2 with (+) = min; it is computed with the
// block-combine routine (common.cuh), O(1) per window.  Consecutive windows with the same pick
// store it once (Sec. 2.4, Fig. 2).  Output order is the order of positions, so tiles place
// their picks with a decoupled look-back over per-tile counts: a tile takes its index from an
// atomic counter (so every predecessor is already running), publishes its count, and sums its
// predecessors' counts, waiting at most a bounded time.
#include <cstdio>
#include <type_traits>

#include "../../include/sws.h"
#include "common.cuh"
#include "internal.h"
#include "mini_common.cuh"

namespace sws {

using namespace mini;

namespace {

constexpr int MNT = 256;  // threads per CTA
constexpr int MVPT = 16;  // k-mers per thread
constexpr int ML = MNT * MVPT;
constexpr int MAXB = 128;                 // barriers kept in shared memory per tile
constexpr int STAGE_BYTES_MINI = ((MNT + 6) * 4 + 15) / 16 * 16;
constexpr int STAGE_BYTES_KMER = ((MNT + 3) * 4 + 15) / 16 * 16;
// ---- the fused minimizer kernel --------------------------------------------------------------
template <class KOp, int SRC, int BAR, bool STAGED>
struct MiniSmem {
  using BC = BlockCombine<KOp, MNT, MVPT>;
  static constexpr int OFF_BASES = 0;
  static constexpr int OFF_BC = STAGE_BYTES_MINI;
  // the block-combine buffer, reused for the tile's picks: hash (4 or 8 bytes), position, and in
  // a staged read batch the read index of a read's first pick
  static constexpr int PICKS =
      ML * ((sizeof(typename KeyTraits<KOp>::T) == 8 ? 4 : 8) + 4 + (STAGED && BAR == BAR_READS ? 4 : 0));
  static constexpr int BC_BYTES = (int)sizeof(typename BC::Shared) > PICKS ? (int)sizeof(typename BC::Shared) : PICKS;
  static constexpr int OFF_BAR = OFF_BC + (BC_BYTES + 15) / 16 * 16;
  static constexpr int BYTES = OFF_BAR + MAXB * 16;
};

// STAGED: instead of ordering its picks by the look-back, a tile writes them to its fixed slot
// of the staging area with its count (ordered afterwards by a scan and a gather, as the staged
// kernel of minimizer_fast.cu does); tiles then never wait for one another.
template <class KOp, int SRC, int BAR, bool STAGED>
__global__ void __launch_bounds__(MNT) k_minimizers(MiniArgs a, int TW, int span, uint64_t nwin,
                                                    const uint2 *__restrict__ tile_bar) {
  using BC = BlockCombine<KOp, MNT, MVPT>;
  using KT = KeyTraits<KOp>;
  using Key = typename KT::T;
  using SM = MiniSmem<KOp, SRC, BAR, STAGED>;
  extern __shared__ __align__(16) unsigned char smem[];
  uint8_t *sbases = smem + SM::OFF_BASES;
  typename BC::Shared &sbc = *reinterpret_cast<typename BC::Shared *>(smem + SM::OFF_BC);
  long long *sbar = reinterpret_cast<long long *>(smem + SM::OFF_BAR);
  __shared__ unsigned long long s_mbar;
  __shared__ uint32_t s_tile;
  __shared__ int s_phase;
  __shared__ uint32_t s_last_pos[MNT];
  __shared__ unsigned char s_last_valid[MNT];
  __shared__ uint32_t s_wcount[MNT / 32];
  __shared__ unsigned long long s_excl;
  __shared__ int s_failed;

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (!STAGED) {
    if (t == 0) s_tile = atomicAdd(a.tile_counter, 1u);
    __syncthreads();
  }
  const uint32_t tile = STAGED ? blockIdx.x : s_tile;
  uint64_t n = a.n;  // bases (or keys)
  uint32_t num_tiles = gridDim.x;
  if (a.desc) {  // a batch graph launched for the largest batch: sizes of this run
    n = a.desc[BD_TOTAL];
    nwin = a.desc[BD_NWIN];
    num_tiles = (uint32_t)a.desc[BD_TILES];
    if (tile >= num_tiles) return;
  }
  if (STAGED && t == 0 && tile == 0) a.tile_counts[num_tiles] = 0;  // the scan's last entry becomes the total
  const long long p0 = (long long)tile * TW;  // first emitted window of the tile
  const long long ifirst = p0 - 1;             // k-mer / window of local index 0

  // Barriers (N-blocks or read starts) that can touch this tile's windows.
  uint32_t g_lo = 0, nb = 0;
  if (tile_bar != nullptr) {
    const uint2 tb = tile_bar[tile];
    g_lo = tb.x;
    nb = tb.y;
  }
  const bool bar_in_smem = nb <= (uint32_t)MAXB;
  if (bar_in_smem) {
    for (uint32_t i = t; i < nb; i += MNT) {
      if (BAR == BAR_NBLOCK) {
        sbar[2 * i] = a.bar[2 * (g_lo + i)];
        sbar[2 * i + 1] = a.bar[2 * (g_lo + i) + 1];
      } else {
        const long long s = a.bar[g_lo + i + 1];
        sbar[2 * i] = s;
        sbar[2 * i + 1] = s;
      }
    }
  }
  auto bar_start = [&](uint32_t i) -> long long {
    if (bar_in_smem) return sbar[2 * i];
    return BAR == BAR_NBLOCK ? a.bar[2 * (g_lo + i)] : a.bar[g_lo + i + 1];
  };
  auto bar_end = [&](uint32_t i) -> long long {
    if (bar_in_smem) return sbar[2 * i + 1];
    return BAR == BAR_NBLOCK ? a.bar[2 * (g_lo + i) + 1] : a.bar[g_lo + i + 1];
  };

  // Keys of this thread's MVPT k-mers.
  Key x[MVPT];
  bool ok = true;
  if (SRC == SRC_DNA) {
    if (t == 0) s_phase = (int)((unsigned long long)(ifirst + a.w) % (unsigned long long)a.w);
    ok = stage_bytes(sbases, a.seq, (n + 3) / 4, p0 / 4 - 16, STAGE_BYTES_MINI, &s_mbar, a.err, !a.withhold_copy);
    const uint32_t *W = reinterpret_cast<const uint32_t *>(sbases);
    const int k = a.k;
    if (2 * k <= 32) {
      const uint32_t kmask = 0xFFFFFFFFu >> (32 - 2 * k);
      const uint32_t w0 = W[3 + t], w1 = W[4 + t], w2 = W[5 + t];
#pragma unroll
      for (int j = 0; j < MVPT; ++j) {
        // k-mer j of this thread starts at bit 126 + 32 t + 2 j of the staged bytes
        const uint32_t bits = j == 0 ? __funnelshift_r(w0, w1, 30) : __funnelshift_r(w1, w2, 2 * (j - 1));
        const long long i = ifirst + t * MVPT + j;
        const Kmer32 q = kmer32(bits, k, kmask);
        const uint32_t v = key_value32(q, a.mode, kmask);
        x[j] = (i >= 0 && (unsigned long long)i + k <= n) ? KT::make(v, (uint32_t)i) : KT::none();
      }
    } else {
      const unsigned long long kmask = 0xFFFFFFFFFFFFFFFFull >> (64 - 2 * k);
      const uint32_t w0 = W[3 + t], w1 = W[4 + t], w2 = W[5 + t], w3 = W[6 + t];
#pragma unroll
      for (int j = 0; j < MVPT; ++j) {
        uint32_t lo32, hi32;
        if (j == 0) {
          lo32 = __funnelshift_r(w0, w1, 30);
          hi32 = __funnelshift_r(w1, w2, 30);
        } else {
          lo32 = __funnelshift_r(w1, w2, 2 * (j - 1));
          hi32 = __funnelshift_r(w2, w3, 2 * (j - 1));
        }
        const unsigned long long bits = ((unsigned long long)hi32 << 32) | lo32;
        const long long i = ifirst + t * MVPT + j;
        const Kmer64 q = kmer64(bits, k, kmask);
        const unsigned long long v = key_value64(q, a.mode, kmask);
        x[j] = (i >= 0 && (unsigned long long)i + k <= n) ? KT::make(v, (uint32_t)i) : KT::none();
      }
    }
  } else {
    if (t == 0) s_phase = (int)((unsigned long long)(ifirst + a.w) % (unsigned long long)a.w);
#pragma unroll
    for (int j = 0; j < MVPT; ++j) {
      const long long i = ifirst + t * MVPT + j;
      x[j] = (i >= 0 && (unsigned long long)i < n) ? KT::make(__ldg(a.keys + i), (uint32_t)i) : KT::none();
    }
    __syncthreads();
  }

  // Sliding minimum over w keys (block-combine).
  const int r0 = (int)(((unsigned)s_phase + (unsigned)(t * MVPT)) % (unsigned)a.w);
  Key m[MVPT];
  BC::run(sbc, x, r0, a.w, m);

  // Window validity: inside [0, nwin) and touching no barrier.
  const long long pf = ifirst + t * MVPT;  // this thread's first window
  unsigned vmask = 0;
  uint32_t q = 0;
  {
    // first barrier with end > pf (binary search over the tile's list)
    uint32_t lo = 0, hi = nb;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (bar_end(mid) > pf) hi = mid;
      else lo = mid + 1;
    }
    q = lo;
  }
  uint32_t read_of_first = 0;
  if (BAR == BAR_READS) read_of_first = g_lo + q;
  uint32_t qj[MVPT];
#pragma unroll
  for (int j = 0; j < MVPT; ++j) {
    const long long p = pf + j;
    while (q < nb && bar_end(q) <= p) ++q;
    qj[j] = q;
    const bool in_range = p >= 0 && (unsigned long long)p < nwin;
    const bool clear = (q == nb) || (bar_start(q) > p + span - 1);
    vmask |= (unsigned)(in_range && clear && ok) << j;
  }
  (void)read_of_first;

  // Deduplicate: window o emits iff valid and (previous invalid or a different pick).
  s_last_pos[t] = KT::pos(m[MVPT - 1]);
  s_last_valid[t] = (unsigned char)((vmask >> (MVPT - 1)) & 1u);
  __syncthreads();
  uint32_t prev_pos = t > 0 ? s_last_pos[t - 1] : 0u;
  bool prev_valid = t > 0 ? (s_last_valid[t - 1] != 0) : false;
  unsigned emask = 0, firstmask = 0;
#pragma unroll
  for (int j = 0; j < MVPT; ++j) {
    const int o = t * MVPT + j;
    const bool v = (vmask >> j) & 1u;
    const uint32_t pp = KT::pos(m[j]);
    const bool e = v && o >= 1 && o <= TW && (!prev_valid || pp != prev_pos);
    emask |= (unsigned)e << j;
    firstmask |= (unsigned)(e && !prev_valid) << j;
    prev_pos = pp;
    prev_valid = v;
  }

  // CTA exclusive scan of pick counts.
  const uint32_t cnt = __popc(emask);
  uint32_t inc = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t u = __shfl_up_sync(kFull, inc, d);
    if (lane >= d) inc += u;
  }
  if (lane == 31) s_wcount[warp] = inc;
  __syncthreads();
  uint32_t woff = 0, total = 0;
#pragma unroll
  for (int i = 0; i < MNT / 32; ++i) {
    const uint32_t c = s_wcount[i];
    if (i < warp) woff += c;
    total += c;
  }
  const uint32_t toff = woff + inc - cnt;  // picks of this tile before this thread

  using HashT = typename std::conditional<sizeof(Key) == 8, uint32_t, unsigned long long>::type;
  HashT *sh_hash = reinterpret_cast<HashT *>(&sbc);
  uint32_t *sh_pos = reinterpret_cast<uint32_t *>(sh_hash + ML);
  uint32_t *sh_first = sh_pos + ML;  // staged read batches: read index of a read's first pick
  if (STAGED && a.count_only) {
    if (t == 0) a.tile_counts[tile] = total;
    return;
  }
  if (STAGED) {
    // stage the tile's picks in order in shared memory, then copy them to the tile's slot
    __syncthreads();  // the block-combine buffer is reused
    uint32_t r = toff;
#pragma unroll
    for (int j = 0; j < MVPT; ++j) {
      if ((emask >> j) & 1u) {
        uint32_t pos = KT::pos(m[j]);
        if (BAR == BAR_READS) {
          const uint32_t rd = g_lo + qj[j];
          pos = (uint32_t)((long long)pos - a.bar[rd]);
          sh_first[r] = ((firstmask >> j) & 1u) ? rd : 0xFFFFFFFFu;
        }
        sh_hash[r] = (HashT)KT::hash(m[j]);
        sh_pos[r] = pos;
        ++r;
      }
    }
    __syncthreads();
    const uint64_t slot = (uint64_t)tile * TW;
    HashT *gh = static_cast<HashT *>(a.stg_hash);
    for (uint32_t i = t; i < total; i += MNT) {
      gh[slot + i] = sh_hash[i];
      a.stg_pos[slot + i] = sh_pos[i];
      if (BAR == BAR_READS) a.stg_first[slot + i] = sh_first[i];
    }
    if (t == 0) a.tile_counts[tile] = total;
    return;
  }

  // a tile whose input copy timed out fails the ordered output (the count is never written)
  const bool copy_failed = __syncthreads_or(!ok);
  if (warp == 0) {
    bool failed = false;
    const unsigned long long ex = lookback_warp(a.status, tile, total, a.err, failed, copy_failed);
    if (lane == 0) {
      s_excl = ex;
      s_failed = failed ? 1 : 0;
    }
  }
  __syncthreads();
  if (s_failed) return;
  const unsigned long long base = s_excl;

  // Stage picks in shared memory (reusing the block-combine buffer), then store coalesced.
  uint32_t r = toff;
#pragma unroll
  for (int j = 0; j < MVPT; ++j) {
    if ((emask >> j) & 1u) {
      uint32_t pos = KT::pos(m[j]);
      if (BAR == BAR_READS) {
        const uint32_t rd = g_lo + qj[j];  // read index of window p
        pos = (uint32_t)((long long)pos - a.bar[rd]);
        if ((firstmask >> j) & 1u) a.pick_offsets[rd] = base + r;
      }
      sh_hash[r] = (HashT)KT::hash(m[j]);
      sh_pos[r] = pos;
      ++r;
    }
  }
  __syncthreads();
  HashT *gh = static_cast<HashT *>(a.hash_out);
  for (uint32_t i = t; i < total; i += MNT) {
    const unsigned long long gi = base + i;
    if (gi < a.capacity) {
      gh[gi] = sh_hash[i];
      a.pos_out[gi] = sh_pos[i];
    }
  }
  if (t == 0 && (unsigned long long)tile * TW + TW >= nwin) {
    // the tile holding the last window knows the final count
    *a.count_out = base + total;
  }
}

// Per tile: the first barrier that can touch its windows and how many can.
template <int BAR>
__global__ void k_tile_barriers(const int64_t *__restrict__ bar, uint64_t nbar, uint64_t ntiles, int TW, int span,
                                uint2 *__restrict__ out, const unsigned long long *__restrict__ desc) {
  if (desc) {
    nbar = desc[BD_NREADS];
    ntiles = desc[BD_TILES];
  }
  const uint64_t tile = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tile >= ntiles) return;
  const long long lo_lim = (long long)tile * TW - 1;            // first window of the tile
  const long long hi_lim = (long long)tile * TW + TW - 1 + span - 1;  // last base any window touches
  const uint64_t cnt = BAR == BAR_NBLOCK ? nbar : (nbar > 0 ? nbar - 1 : 0);
  auto start = [&](uint64_t i) -> long long { return BAR == BAR_NBLOCK ? bar[2 * i] : bar[i + 1]; };
  auto end = [&](uint64_t i) -> long long { return BAR == BAR_NBLOCK ? bar[2 * i + 1] : bar[i + 1]; };
  uint64_t lo = 0, hi = cnt;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (end(mid) > lo_lim) hi = mid;
    else lo = mid + 1;
  }
  const uint64_t g = lo;
  lo = g;
  hi = cnt;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (start(mid) > hi_lim) hi = mid;
    else lo = mid + 1;
  }
  out[tile] = make_uint2((uint32_t)g, (uint32_t)(lo - g));
}

// ---- k-mer values -----------------------------------------------------------------------------
template <bool WIDE>
__global__ void __launch_bounds__(MNT) k_kmers(const uint8_t *__restrict__ seq, uint64_t n, int k, int kind,
                                               void *__restrict__ out, int *err) {
  __shared__ __align__(16) uint8_t sb[STAGE_BYTES_KMER];
  __shared__ unsigned long long s_mbar;
  const int t = threadIdx.x;
  const unsigned long long i0 = (unsigned long long)blockIdx.x * ML;
  stage_bytes(sb, seq, (n + 3) / 4, (long long)(i0 / 4), STAGE_BYTES_KMER, &s_mbar, err);
  const uint32_t *W = reinterpret_cast<const uint32_t *>(sb);
  const unsigned long long m = n - (unsigned long long)k + 1;
  const unsigned long long g = i0 + (unsigned long long)t * MVPT;
  if (!WIDE) {
    const uint32_t kmask = 0xFFFFFFFFu >> (32 - 2 * k);
    const uint32_t w0 = W[t], w1 = W[t + 1];
    uint32_t v[MVPT];
#pragma unroll
    for (int j = 0; j < MVPT; ++j) {
      const Kmer32 q = kmer32(__funnelshift_r(w0, w1, 2 * j), k, kmask);
      const uint32_t c = q.fwd < q.rc ? q.fwd : q.rc;
      v[j] = kind == SWS_KMER_FWD ? q.fwd : kind == SWS_KMER_RC ? q.rc : kind == SWS_KMER_CANONICAL ? c : wang_mix32(c, kmask);
    }
    uint32_t *o = static_cast<uint32_t *>(out);
    if (g + MVPT <= m && (reinterpret_cast<uintptr_t>(o) & 15u) == 0) {
      store_vec<uint32_t, MVPT>(o + g, v);
    } else {
#pragma unroll
      for (int j = 0; j < MVPT; ++j)
        if (g + j < m) o[g + j] = v[j];
    }
  } else {
    const unsigned long long kmask = 0xFFFFFFFFFFFFFFFFull >> (64 - 2 * k);
    const uint32_t w0 = W[t], w1 = W[t + 1], w2 = W[t + 2];
    unsigned long long v[MVPT];
#pragma unroll
    for (int j = 0; j < MVPT; ++j) {
      const uint32_t lo32 = __funnelshift_r(w0, w1, 2 * j), hi32 = __funnelshift_r(w1, w2, 2 * j);
      const Kmer64 q = kmer64(((unsigned long long)hi32 << 32) | lo32, k, kmask);
      const unsigned long long c = q.fwd < q.rc ? q.fwd : q.rc;
      v[j] = kind == SWS_KMER_FWD ? q.fwd : kind == SWS_KMER_RC ? q.rc : kind == SWS_KMER_CANONICAL ? c : wang_mix64(c, kmask);
    }
    unsigned long long *o = static_cast<unsigned long long *>(out);
    if (g + MVPT <= m && (reinterpret_cast<uintptr_t>(o) & 15u) == 0) {
      store_vec<unsigned long long, MVPT>(o + g, v);
    } else {
#pragma unroll
      for (int j = 0; j < MVPT; ++j)
        if (g + j < m) o[g + j] = v[j];
    }
  }
}

// ---- batch pick offsets: suffix minimum ------------------------------------------------------
constexpr int FIX_NT = 256, FIX_PER = 4, FIX_BLOCK = FIX_NT * FIX_PER;

__global__ void k_fix_block_min(const uint64_t *__restrict__ po, uint64_t nreads, uint64_t *__restrict__ bmin,
                                const unsigned long long *__restrict__ desc) {
  __shared__ uint64_t s[FIX_NT];
  if (desc) nreads = desc[BD_NREADS];
  const uint64_t b0 = (uint64_t)blockIdx.x * FIX_BLOCK;
  uint64_t v = ~0ull;
  for (int j = 0; j < FIX_PER; ++j) {
    const uint64_t i = b0 + (uint64_t)j * FIX_NT + threadIdx.x;
    if (i < nreads) v = min(v, po[i]);
  }
  s[threadIdx.x] = v;
  __syncthreads();
  for (int d = FIX_NT / 2; d > 0; d >>= 1) {
    if ((int)threadIdx.x < d) s[threadIdx.x] = min(s[threadIdx.x], s[threadIdx.x + d]);
    __syncthreads();
  }
  if (threadIdx.x == 0) bmin[blockIdx.x] = s[0];
}

// Within a block of FIX_NT threads: the minimum of x over the threads after this one, and of
// `carry`; tot (every thread) gets the minimum over all threads and carry.
__device__ __forceinline__ uint64_t fix_suffix_after(uint64_t x, uint64_t carry, uint64_t *wsuf, uint64_t &tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {  // inclusive suffix minimum within the warp
    const uint64_t u = __shfl_down_sync(0xFFFFFFFFu, x, d);
    if (lane + d < 32) x = min(x, u);
  }
  if (lane == 0) wsuf[warp] = x;
  __syncthreads();
  uint64_t after = carry;
  tot = carry;
  for (int w2 = 0; w2 < FIX_NT / 32; ++w2) {
    const uint64_t v = wsuf[w2];
    tot = min(tot, v);
    if (w2 > warp) after = min(after, v);
  }
  const uint64_t nxt = __shfl_down_sync(0xFFFFFFFFu, x, 1);
  __syncthreads();  // wsuf may be rewritten by the caller's next round
  return lane == 31 ? after : min(after, nxt);
}

// Exclusive suffix minimum over the block minima, seeded with the total count (one block; rounds
// of FIX_NT block minima from the last).
__global__ void __launch_bounds__(FIX_NT) k_fix_scan(uint64_t *__restrict__ bmin, uint64_t nblocks,
                                                    const uint64_t *__restrict__ count,
                                                    const unsigned long long *__restrict__ desc) {
  __shared__ uint64_t wsuf[FIX_NT / 32];
  if (desc) nblocks = (desc[BD_NREADS] + FIX_BLOCK - 1) / FIX_BLOCK;
  uint64_t carry = *count;
  for (uint64_t hi = nblocks; hi > 0;) {
    const uint64_t lo = hi > (uint64_t)FIX_NT ? hi - FIX_NT : 0;
    const uint64_t b = lo + threadIdx.x;
    const uint64_t v = b < hi ? bmin[b] : ~0ull;
    uint64_t tot;
    const uint64_t out = fix_suffix_after(v, carry, wsuf, tot);
    if (b < hi) bmin[b] = out;
    carry = tot;
    hi = lo;
  }
}

__global__ void k_fix_apply(uint64_t *__restrict__ po, uint64_t nreads, const uint64_t *__restrict__ bcarry,
                            const uint64_t *__restrict__ count, const unsigned long long *__restrict__ desc) {
  __shared__ uint64_t s[FIX_BLOCK];
  if (desc) nreads = desc[BD_NREADS];
  if ((uint64_t)blockIdx.x * FIX_BLOCK >= nreads && blockIdx.x > 0) return;
  const uint64_t *carry_src = nreads == 0 ? count : bcarry;
  const uint64_t b0 = (uint64_t)blockIdx.x * FIX_BLOCK;
  for (int j = threadIdx.x; j < FIX_BLOCK; j += FIX_NT) {
    const uint64_t i = b0 + j;
    s[j] = i < nreads ? po[i] : ~0ull;
  }
  __syncthreads();
  {
    // inclusive suffix minimum of s, seeded with the carry from the blocks after this one: each
    // thread its FIX_PER consecutive entries, then across threads
    const uint64_t carry = nreads == 0 ? *count : carry_src[blockIdx.x];
    uint64_t e[FIX_PER];
#pragma unroll
    for (int j = 0; j < FIX_PER; ++j) e[j] = s[threadIdx.x * FIX_PER + j];
#pragma unroll
    for (int j = FIX_PER - 2; j >= 0; --j) e[j] = min(e[j], e[j + 1]);
    __shared__ uint64_t wsuf[FIX_NT / 32];
    uint64_t tot;
    const uint64_t ex = fix_suffix_after(e[0], carry, wsuf, tot);
#pragma unroll
    for (int j = 0; j < FIX_PER; ++j) s[threadIdx.x * FIX_PER + j] = min(e[j], ex);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < FIX_BLOCK; j += FIX_NT) {
    const uint64_t i = b0 + j;
    if (i < nreads) po[i] = s[j];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) po[nreads] = *count;
}

template <class KOp, int SRC, int BAR, bool STAGED = false>
cudaError_t launch_mini_t(const MiniArgs &a, uint64_t num_tiles, const uint2 *tile_bar, cudaStream_t st) {
  using SM = MiniSmem<KOp, SRC, BAR, STAGED>;
  auto kern = k_minimizers<KOp, SRC, BAR, STAGED>;
  const size_t sm = SM::BYTES;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  const int TW = mini_tile_windows(a.w);
  const int span = SRC == SRC_DNA ? a.w + a.k - 1 : a.w;
  const uint64_t nwin = SRC == SRC_DNA ? (a.n >= (uint64_t)span ? a.n - span + 1 : 0) : (a.n >= (uint64_t)a.w ? a.n - a.w + 1 : 0);
  kern<<<(unsigned)num_tiles, MNT, sm, st>>>(a, TW, span, nwin, tile_bar);
  return cudaGetLastError();
}

}  // namespace

int mini_tile_windows(int w) {
  const int tw = (ML - w) / 64 * 64;
  return tw >= 64 ? tw : 0;
}

bool tile_barriers_needed(const MiniArgs &a, int source, int barrier) {
  if (a.desc) return source == SRC_DNA && barrier == BAR_READS;  // batch graphs: decided at run time
  return source == SRC_DNA && ((barrier == BAR_NBLOCK && a.nbar > 0) || (barrier == BAR_READS && a.nbar > 1));
}

cudaError_t launch_tile_barriers(const MiniArgs &a, int source, int barrier, uint64_t num_tiles, int TW, int span,
                                 cudaStream_t st) {
  if (!tile_barriers_needed(a, source, barrier) || num_tiles == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((num_tiles + 255) / 256);
  if (barrier == BAR_NBLOCK)
    k_tile_barriers<BAR_NBLOCK><<<blocks, 256, 0, st>>>(a.bar, a.nbar, num_tiles, TW, span, a.tile_bar, a.desc);
  else
    k_tile_barriers<BAR_READS><<<blocks, 256, 0, st>>>(a.bar, a.nbar, num_tiles, TW, span, a.tile_bar, a.desc);
  return cudaGetLastError();
}

uint64_t mini_lookback_tiles(uint64_t nwin, int w) {
  const int tw = mini_tile_windows(w);
  if (tw == 0 || nwin == 0) return 0;
  return (nwin + tw - 1) / tw;
}

cudaError_t launch_minimizers_lookback(const MiniArgs &a, int source, int barrier, uint64_t num_tiles,
                                       cudaStream_t st) {
  if (num_tiles == 0) return cudaSuccess;
  if (num_tiles > 0xffffffffull) return cudaErrorInvalidValue;
  const uint2 *tile_bar = nullptr;
  const int TW = mini_tile_windows(a.w);
  const int span = source == SRC_DNA ? a.w + a.k - 1 : a.w;
  cudaError_t e = launch_tile_barriers(a, source, barrier, num_tiles, TW, span, st);
  if (e != cudaSuccess) return e;
  if (tile_barriers_needed(a, source, barrier)) tile_bar = a.tile_bar;
  const bool wide = source == SRC_DNA && 2 * a.k > 32;
  if (source == SRC_KEYS) return launch_mini_t<OpMinKey64, SRC_KEYS, BAR_NBLOCK>(a, num_tiles, nullptr, st);
  if (barrier == BAR_READS) {
    if (wide) return launch_mini_t<OpMinKey96, SRC_DNA, BAR_READS>(a, num_tiles, tile_bar, st);
    return launch_mini_t<OpMinKey64, SRC_DNA, BAR_READS>(a, num_tiles, tile_bar, st);
  }
  if (wide) return launch_mini_t<OpMinKey96, SRC_DNA, BAR_NBLOCK>(a, num_tiles, tile_bar, st);
  return launch_mini_t<OpMinKey64, SRC_DNA, BAR_NBLOCK>(a, num_tiles, tile_bar, st);
}

// The generic kernel in staged mode (any w, any k): one CTA per tile of mini_tile_windows(w)
// windows, picks and counts to the staging area (tile barriers already computed by the caller).
cudaError_t launch_minimizers_generic_staged(const MiniArgs &a, int source, int barrier, uint64_t num_tiles,
                                             const uint2 *tile_bar, cudaStream_t st) {
  if (num_tiles == 0) return cudaSuccess;
  if (num_tiles > 0xffffffffull) return cudaErrorInvalidValue;
  const bool wide = source == SRC_DNA && 2 * a.k > 32;
  if (source == SRC_KEYS) return launch_mini_t<OpMinKey64, SRC_KEYS, BAR_NBLOCK, true>(a, num_tiles, nullptr, st);
  if (barrier == BAR_READS) {
    if (wide) return launch_mini_t<OpMinKey96, SRC_DNA, BAR_READS, true>(a, num_tiles, tile_bar, st);
    return launch_mini_t<OpMinKey64, SRC_DNA, BAR_READS, true>(a, num_tiles, tile_bar, st);
  }
  if (wide) return launch_mini_t<OpMinKey96, SRC_DNA, BAR_NBLOCK, true>(a, num_tiles, tile_bar, st);
  return launch_mini_t<OpMinKey64, SRC_DNA, BAR_NBLOCK, true>(a, num_tiles, tile_bar, st);
}

cudaError_t launch_pick_offsets_fixup(uint64_t *po, uint64_t nreads, const uint64_t *count, uint64_t *scratch,
                                      cudaStream_t st, const unsigned long long *desc) {
  const uint64_t nblocks = (nreads + FIX_BLOCK - 1) / FIX_BLOCK;
  if (nblocks == 0) {
    k_fix_apply<<<1, FIX_NT, 0, st>>>(po, 0, count, count, desc);
    return cudaGetLastError();
  }
  k_fix_block_min<<<(unsigned)nblocks, FIX_NT, 0, st>>>(po, nreads, scratch, desc);
  k_fix_scan<<<1, FIX_NT, 0, st>>>(scratch, nblocks, count, desc);
  k_fix_apply<<<(unsigned)nblocks, FIX_NT, 0, st>>>(po, nreads, scratch, count, desc);
  return cudaGetLastError();
}

cudaError_t launch_kmers(const uint8_t *seq, uint64_t n, int k, int kind, void *out, int *err, cudaStream_t st) {
  const uint64_t m = n - (uint64_t)k + 1;
  const uint64_t blocks = (m + ML - 1) / ML;
  if (blocks > 0x7fffffffull) return cudaErrorInvalidValue;
  if (2 * k <= 32) k_kmers<false><<<(unsigned)blocks, MNT, 0, st>>>(seq, n, k, kind, out, err);
  else k_kmers<true><<<(unsigned)blocks, MNT, 0, st>>>(seq, n, k, kind, out, err);
  return cudaGetLastError();
}

}  // namespace sws
