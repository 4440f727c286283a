// minimizer_fast.cu -- minimizers for window lengths w = 4..256 (any k <= 32, or precomputed
// 32-bit keys), in three steps that never wait on one another inside a kernel:
//
//   1. k_mini_stage (persistent, one CTA per resident slot, tiles assigned statically): keys of a
//      tile's k-mers, the least key of every window (Sec. 2.4) by block-combine, which windows
//      store a new pick, and where; the tile's picks go to a fixed slot of a staging area and the
//      count to a per-tile word.  The next tile's packed bases are fetched by TMA (cp.async.bulk
//      into the other of two shared buffers, completed on an mbarrier) while this one computes.
//   2. an exclusive scan of the per-tile counts (scan_u32 in table.cu);
//   3. k_mini_gather: each CTA copies one tile's picks to their final, position-ordered place.
//
// The staging costs about 16 bytes of traffic per pick; in exchange no CTA ever waits for another
// (the single-kernel path in minimizer.cu orders its output with a look-back instead).
//
// Details of step 1:
// * w <= 16: a tile starts at a multiple of w and a thread owns VPT = w * floor(16 / w) consecutive
//   k-mers, so the blocks of w are whole, compile-time groups of registers: the block-combine
//   (in-block suffix minimum with the next block's prefix minimum) needs no segment bookkeeping and
//   runs on the key values themselves (32-bit for 2k <= 32 and precomputed keys, 64-bit otherwise).
// * 16 < w <= 256 (w known at run time): a thread's 16 k-mers are a chunk; with chunk prefix and
//   suffix minima and chunk minima in shared memory, window o is the suffix minimum at o, the
//   minima of the whole chunks it covers, and the prefix minimum at o + w - 1 (Eq. 2 combined over
//   blocks shorter than w): still O(1) per window for a fixed w, with no segmented scan.
// * Ties.  Keys are ordered by (value, position).  Instead of 64-bit keys, the scans carry a 32-bit
//   value and the position of its leftmost occurrence: a prefix step takes the new element only
//   when strictly smaller, a suffix step when smaller or equal, and a window's suffix part (left)
//   wins ties against its prefix part (right).  Every window then knows its pick's position, and a
//   window stores a pick when its position differs from the previous window's.
#include <cstdio>
#include <type_traits>

#include "../../include/sws.h"
#include "common.cuh"
#include "internal.h"
#include "mini_common.cuh"

namespace sws {

using namespace mini;

namespace {

constexpr int FNT = 256;
constexpr int FNW = FNT / 32;
constexpr int FMAXB = 128;

// W = 4..16: blocks of w whole in each thread's registers.  W = 0 (CHUNK): any w in 17..CHUNK_MAXW
// given at run time; each thread's 16 k-mers form a chunk, and a window is the suffix of its first
// chunk, whole chunks, and a prefix of its last chunk.
constexpr int CHUNK = 0;
constexpr int CHUNK_VPT = 16;
constexpr int CHUNK_MAXW = 256;
__host__ __device__ constexpr int chunk_tile_windows(int w) {  // TW <= L - 2w + 1, a multiple of 16
  return (FNT * CHUNK_VPT - 2 * w + 1) / 16 * 16;
}

template <int W, int SRC, int BAR, class V>
struct Geo {
  static constexpr bool CH = W == CHUNK;
  static constexpr int NB = CH ? 1 : 16 / W;              // blocks of w per thread
  static constexpr int VPT = CH ? CHUNK_VPT : W * NB;     // k-mers per thread
  static constexpr int L = FNT * VPT;                     // k-mers per tile
  static constexpr int TW = CH ? L : (FNT * NB - 2) * W;  // windows per tile (CH: an upper bound)
  static constexpr int STAGE = SRC == SRC_DNA ? ((63 + L + 16) / 4 + 16 + 15) / 16 * 16 : (L + 8) * 4;
  // picks: value (V), position, and for read batches the read index of a read's first pick
  static constexpr int PICK_BYTES = TW * ((int)sizeof(V) + (BAR == BAR_READS ? 8 : 4));
  // CH: chunk prefix minima (value, position) at padded index o + o/16, then per chunk its minimum
  // (value, position) and last key; they are dead once the windows are known, and the picks reuse
  // the space.  Otherwise, DNA: keys of the tile, sx[o + 1] (keys: read from the stage).
  static constexpr int LP = L + L / 16;
  static constexpr int CH_BYTES = LP * ((int)sizeof(V) + 4) + FNT * (2 * (int)sizeof(V) + 4);
  static constexpr int SX_BYTES = CH ? (CH_BYTES > PICK_BYTES ? CH_BYTES : PICK_BYTES)
                                     : (SRC == SRC_DNA ? (L + 2) * (int)sizeof(V) : 0);
  static constexpr int OFF_SX = 2 * STAGE;
  static constexpr int OFF_BAR = OFF_SX + (SX_BYTES + 15) / 16 * 16;
  static constexpr int OFF_PICKS = CH ? OFF_SX : OFF_BAR + FMAXB * 16;
  static constexpr int BYTES = CH ? OFF_BAR + FMAXB * 16 : OFF_PICKS + PICK_BYTES;
};

__device__ __forceinline__ long long floor_div(long long a, long long b) {
  return a >= 0 ? a / b : -((-a + b - 1) / b);
}

struct Staging {
  long long gb0;   // global byte of staged byte 0
  long long lo;    // first byte of the bulk copy
  long long bulk;  // bytes of the bulk copy (0: none)
};

template <int W, int BAR, int SRC, class V>
__global__ void __launch_bounds__(FNT) k_mini_stage(MiniArgs a, uint64_t nwin, int span,
                                                    const uint2 *__restrict__ tile_bar, uint32_t num_tiles) {
  using G = Geo<W, SRC, BAR, V>;
  constexpr V NONE = ~(V)0;
  constexpr int VPT = G::VPT, NB = G::NB, WM1 = W > 1 ? W - 1 : 1;
  const int w = G::CH ? a.w : W;                              // window length
  const int TW = G::CH ? chunk_tile_windows(a.w) : G::TW;     // windows per tile
  extern __shared__ __align__(16) unsigned char smem[];
  V *sx = reinterpret_cast<V *>(smem + G::OFF_SX);
  long long *sbar = reinterpret_cast<long long *>(smem + G::OFF_BAR);
  V *sh_hash = reinterpret_cast<V *>(smem + G::OFF_PICKS);
  uint32_t *sh_pos = reinterpret_cast<uint32_t *>(sh_hash + G::TW);
  uint32_t *sh_first = sh_pos + G::TW;  // read batches only
  __shared__ unsigned long long s_mbar[2];
  __shared__ Staging s_st[2];
  __shared__ uint32_t s_wcount[FNW];

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  uint64_t n = a.n;
  if (a.desc) {  // a batch graph: sizes of this run
    n = a.desc[BD_TOTAL];
    nwin = a.desc[BD_NWIN];
    num_tiles = (uint32_t)a.desc[BD_TILES];
  }
  const uint8_t *src = SRC == SRC_DNA ? a.seq : reinterpret_cast<const uint8_t *>(a.keys);
  const uint64_t nbytes = SRC == SRC_DNA ? (n + 3) / 4 : n * 4;
  const bool src_aligned = (reinterpret_cast<uintptr_t>(src) & 15u) == 0;

  // Thread 0: start the bulk copy of tile `tile`'s bases (or keys) into buffer b.
  auto issue = [&](int b, uint32_t tile) {
    const long long i0 = (long long)tile * TW - w;
    const long long gb0 = SRC == SRC_DNA ? floor_div(i0, 64) * 16 : floor_div(i0, 4) * 16;
    const long long lo = gb0 > 0 ? gb0 : 0;
    long long hi = gb0 + G::STAGE;
    if (hi > (long long)nbytes) hi = (long long)nbytes;
    const long long bulk = (src_aligned && hi > lo) ? ((hi - lo) & ~15ll) : 0;
    s_st[b] = Staging{gb0, lo, bulk};
    if (bulk > 0) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&s_mbar[b], (uint32_t)bulk);
      bulk_g2s(smem + b * G::STAGE + (lo - gb0), src + lo, (uint32_t)bulk, &s_mbar[b]);
    }
  };

  if (t == 0) {
    mbar_init(&s_mbar[0], 1);
    mbar_init(&s_mbar[1], 1);
    fence_mbar_init();
    if (blockIdx.x < num_tiles) issue(0, blockIdx.x);
    if (blockIdx.x == 0) a.tile_counts[num_tiles] = 0;  // the scan's last entry becomes the total
  }
  __syncthreads();
  unsigned phases = 0u;  // bit b: parity of the next completion of buffer b's mbarrier

  int it = 0;
  for (uint32_t tile = blockIdx.x; tile < num_tiles; tile += gridDim.x, ++it) {
    const int b = it & 1;
    if (t == 0 && tile + gridDim.x < num_tiles) issue(b ^ 1, tile + gridDim.x);
    const long long p0 = (long long)tile * TW;  // first window of the tile
    const long long i0 = p0 - w;                // k-mer (and window) of local index 0
    uint8_t *stage = smem + b * G::STAGE;

    // ---- bases (or keys) of this tile in shared memory; barriers that can touch it ------------
    const Staging stg = s_st[b];
    bool ok = true;
    if (stg.bulk > 0) {
      const uint32_t ph = (phases >> b) & 1u;
      ok = tma::mbar_wait_bounded(&s_mbar[b], ph);
      if (!ok) {
        if (t == 0) atomicOr(a.err, DEVERR_COPY_TIMEOUT);
        tma::mbar_wait_bounded(&s_mbar[b], ph);  // one more bounded chance for the copy to land
      }
      phases ^= 1u << b;
    }
    {
      // bytes the bulk copy did not bring: [0, head) and [tail, STAGE) of the stage
      const int head = (int)(stg.lo - stg.gb0), tail = (int)(stg.lo + stg.bulk - stg.gb0);
      const int nhead = stg.bulk > 0 ? head : G::STAGE;
      for (int i = t; i < nhead; i += FNT) {
        const long long g = stg.gb0 + i;
        stage[i] = (g >= 0 && g < (long long)nbytes) ? src[g] : (uint8_t)0;
      }
      if (stg.bulk > 0) {
        for (int i = tail + t; i < G::STAGE; i += FNT) {
          const long long g = stg.gb0 + i;
          stage[i] = (g < (long long)nbytes) ? src[g] : (uint8_t)0;
        }
      }
    }
    uint32_t g_lo = 0, nb = 0;
    if (tile_bar != nullptr) {
      const uint2 tb = tile_bar[tile];
      g_lo = tb.x;
      nb = tb.y;
    }
    const bool bar_in_smem = nb <= (uint32_t)FMAXB;
    if (bar_in_smem) {
      for (uint32_t i = t; i < nb; i += FNT) {
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
    __syncthreads();
    auto bar_start = [&](uint32_t i) -> long long {
      if (bar_in_smem) return sbar[2 * i];
      return BAR == BAR_NBLOCK ? a.bar[2 * (g_lo + i)] : a.bar[g_lo + i + 1];
    };
    auto bar_end = [&](uint32_t i) -> long long {
      if (bar_in_smem) return sbar[2 * i + 1];
      return BAR == BAR_NBLOCK ? a.bar[2 * (g_lo + i) + 1] : a.bar[g_lo + i + 1];
    };

    // ---- keys (32-bit values) ------------------------------------------------------------------
    const long long ifirst = i0 + (long long)t * VPT;
    const long long tlo = p0 - 1, thi = p0 + TW - 1;  // windows this tile looks at
    const bool interior = nb == 0 && tlo >= 0 && (unsigned long long)thi < nwin;
    const long long lastv = (long long)n - (SRC == SRC_DNA ? a.k : 1);  // last valid k-mer
    const int jlo = interior ? 0 : (ifirst < 0 ? (int)(-ifirst < VPT ? -ifirst : VPT) : 0);
    const int jhi = interior ? VPT : (lastv < ifirst ? 0 : (int)(lastv - ifirst + 1 < VPT ? lastv - ifirst + 1 : VPT));
    V x[VPT];
    if (SRC == SRC_DNA) {
      const uint32_t *sw = reinterpret_cast<const uint32_t *>(stage);
      const int r = (int)(i0 - 4 * stg.gb0) + t * VPT;  // staged base of this thread's first k-mer
      const int q = r >> 4, s = (r & 15) * 2;
      const uint32_t v0 = __funnelshift_r(sw[q], sw[q + 1], s);  // bases r .. r+15
      const uint32_t v1 = __funnelshift_r(sw[q + 1], sw[q + 2], s);
      const int k = a.k;
      // one loop per key mode, so the mode test is not repeated for every k-mer
      auto keys = [&](auto mode_c) {
        constexpr int MODE = decltype(mode_c)::value;
        // The thread's bases are reversed once (2-bit groups, words swapped): the forward k-mer at
        // offset j is then a funnel shift of the reversed words by a constant and one shift by a
        // k-dependent amount, with no per-k-mer reversal; the reverse complement is the
        // complemented window itself.
        if (sizeof(V) == 4) {
          const uint32_t kmask = 0xFFFFFFFFu >> (32 - 2 * k);
          const uint32_t rhi = rev_pairs32(v0), rlo = rev_pairs32(v1);  // base i at bit 62 - 2i
          const int fsh = 32 - 2 * k;
#pragma unroll
          for (int j = 0; j < VPT; ++j) {
            const uint32_t fw = (j == 0 ? rhi : __funnelshift_r(rlo, rhi, 32 - 2 * j)) >> fsh;
            if (MODE == SWS_MINI_FWD) {
              x[j] = (V)fw;
            } else {
              const uint32_t rc = ~__funnelshift_r(v0, v1, 2 * j) & kmask;
              const uint32_t c = fw < rc ? fw : rc;
              x[j] = (V)(MODE == SWS_MINI_CANONICAL ? c : wang_mix32(c, kmask));
            }
          }
        } else {
          const uint32_t v2 = __funnelshift_r(sw[q + 2], sw[q + 3], s);
          const unsigned long long kmask = 2 * k == 64 ? ~0ull : ((1ull << (2 * k)) - 1ull);
          const uint32_t r2 = rev_pairs32(v0), r1 = rev_pairs32(v1), r0 = rev_pairs32(v2);  // base i at bit 94 - 2i
          const int fsh = 64 - 2 * k;  // 0 .. 30: 2k > 32 here
#pragma unroll
          for (int j = 0; j < VPT; ++j) {
            const uint32_t lo = j == 0 ? r1 : __funnelshift_r(r0, r1, 32 - 2 * j);  // bases j+31 .. j+16
            const uint32_t hi = j == 0 ? r2 : __funnelshift_r(r1, r2, 32 - 2 * j);  // bases j+15 .. j
            const unsigned long long fw =
                ((unsigned long long)(hi >> fsh) << 32) | __funnelshift_r(lo, hi, fsh);
            if (MODE == SWS_MINI_FWD) {
              x[j] = (V)fw;
            } else {
              const unsigned long long w64 = ((unsigned long long)__funnelshift_r(v1, v2, 2 * j) << 32) |
                                             __funnelshift_r(v0, v1, 2 * j);
              const unsigned long long rc = ~w64 & kmask;
              const unsigned long long c = fw < rc ? fw : rc;
              x[j] = (V)(MODE == SWS_MINI_CANONICAL ? c : wang_mix64_wide(c, (uint32_t)(kmask >> 32)));
            }
          }
        }
      };
      if (a.mode == SWS_MINI_HASH) keys(std::integral_constant<int, SWS_MINI_HASH>{});
      else if (a.mode == SWS_MINI_CANONICAL) keys(std::integral_constant<int, SWS_MINI_CANONICAL>{});
      else keys(std::integral_constant<int, SWS_MINI_FWD>{});
    } else {
      const uint32_t *sk = reinterpret_cast<const uint32_t *>(stage);
      const int r = (int)(i0 - stg.gb0 / 4) + t * VPT;
#pragma unroll
      for (int j = 0; j < VPT; ++j) x[j] = (V)sk[r + j];
    }
    if (!interior) {  // k-mers outside the sequence never win a window
#pragma unroll
      for (int j = 0; j < VPT; ++j)
        if (j < jlo || j >= jhi) x[j] = NONE;
    }
    const int o0 = t * VPT;
    V y[VPT];
    uint32_t yp[VPT];
    uint32_t ypprev;  // pick of the window just before this thread's first
    // positions in y/yp/ypprev are tile-local (chunked form) or offsets from o0 (register form)
    const uint32_t pos_base = (uint32_t)i0 + (G::CH ? 0u : (uint32_t)o0);
    if constexpr (!G::CH) {
      // DNA: every thread needs the next thread's first w-1 keys and the key before its own, so the
      // tile's keys go through shared memory; precomputed keys are read from the stage directly.
      const V *kx;  // kx[o]: key of tile-local k-mer o
      if (SRC == SRC_DNA) {
#pragma unroll
        for (int j = 0; j < VPT; ++j) sx[1 + t * VPT + j] = x[j];
        __syncthreads();
        kx = sx + 1;
      } else {
        kx = reinterpret_cast<const V *>(stage) + (i0 - stg.gb0 / 4);  // V is 32-bit for precomputed keys
      }

      // ---- window minima and their leftmost positions, by block-combine on registers -----------
      // Positions are offsets from the thread's first k-mer o0 (constants in the scans; -1 is the
      // k-mer before it).  In-block prefix minima keep the earliest position
      // on ties (strict <), suffix minima the earliest too (<=); a window's suffix part lies left of
      // its prefix part, so ties between the two go to the suffix.
      V xn[WM1];  // the next thread's first w-1 keys
#pragma unroll
      for (int i = 0; i < W - 1; ++i) xn[i] = kx[(t + 1 < FNT ? t + 1 : t) * VPT + i];
      const V xprev = t > 0 ? kx[t * VPT - 1] : NONE;  // key of k-mer ifirst - 1 (unused for thread 0)
      V P[VPT], S[VPT], Pn[WM1];
      uint32_t Pp[VPT], Sp[VPT], Pnp[WM1];
#pragma unroll
      for (int b2 = 0; b2 < NB; ++b2) {
        P[b2 * W] = x[b2 * W];
        Pp[b2 * W] = b2 * W;
#pragma unroll
        for (int i = 1; i < W; ++i) {
          const int j = b2 * W + i;
          const bool c = x[j] < P[j - 1];
          P[j] = c ? x[j] : P[j - 1];
          Pp[j] = c ? (uint32_t)j : Pp[j - 1];
        }
        S[b2 * W + W - 1] = x[b2 * W + W - 1];
        Sp[b2 * W + W - 1] = b2 * W + W - 1;
#pragma unroll
        for (int i = W - 2; i >= 0; --i) {
          const int j = b2 * W + i;
          const bool c = x[j] <= S[j + 1];
          S[j] = c ? x[j] : S[j + 1];
          Sp[j] = c ? (uint32_t)j : Sp[j + 1];
        }
      }
      if (W > 1) {
        Pn[0] = xn[0];
        Pnp[0] = VPT;
#pragma unroll
        for (int i = 1; i < W - 1; ++i) {
          const bool c = xn[i] < Pn[i - 1];
          Pn[i] = c ? xn[i] : Pn[i - 1];
          Pnp[i] = c ? (uint32_t)(VPT + i) : Pnp[i - 1];
        }
      }
#pragma unroll
      for (int b2 = 0; b2 < NB; ++b2) {
        y[b2 * W] = S[b2 * W];
        yp[b2 * W] = Sp[b2 * W];
#pragma unroll
        for (int i = 1; i < W; ++i) {
          const int j = b2 * W + i;
          const V pr = (b2 + 1 < NB) ? P[(b2 + 1) * W + i - 1] : Pn[i - 1];
          const uint32_t prp = (b2 + 1 < NB) ? Pp[(b2 + 1) * W + i - 1] : Pnp[i - 1];
          const bool c = S[j] <= pr;
          y[j] = c ? S[j] : pr;
          yp[j] = c ? Sp[j] : prp;
        }
      }
      // pick of the window just before this thread's first: k-mer ifirst-1 and this block's first w-1
      ypprev = W > 1 ? (xprev <= P[W > 1 ? W - 2 : 0] ? 0xFFFFFFFFu : Pp[W > 1 ? W - 2 : 0])
                                    : 0xFFFFFFFFu;
    } else {
      // ---- chunks of 16 k-mers: window [o, o + w - 1] = suffix of o's chunk, the whole chunks
      // between, and a prefix of the chunk holding o + w - 1 (Eq. 2 with blocks shorter than w).
      // Ties: prefix minima keep the earliest position (strict <), suffix minima too (<=), and each
      // later piece replaces the running minimum only when strictly smaller.
      V *cPv = reinterpret_cast<V *>(smem + G::OFF_SX);        // [LP] chunk prefix minima
      uint32_t *cPp = reinterpret_cast<uint32_t *>(cPv + G::LP);  // [LP] their positions
      V *cTv = reinterpret_cast<V *>(cPp + G::LP);              // [FNT] chunk minima
      V *cLast = cTv + FNT;                                      // [FNT] each chunk's last key
      uint32_t *cTp = reinterpret_cast<uint32_t *>(cLast + FNT);  // [FNT] chunk minima positions
      auto pad = [](int o) { return o + (o >> 4); };              // conflict-free strided access
      V P[VPT], S[VPT];
      uint32_t Pp[VPT], Sp[VPT];
      P[0] = x[0];
      Pp[0] = o0;
#pragma unroll
      for (int j = 1; j < VPT; ++j) {
        const bool c = x[j] < P[j - 1];
        P[j] = c ? x[j] : P[j - 1];
        Pp[j] = c ? (uint32_t)(o0 + j) : Pp[j - 1];
      }
      S[VPT - 1] = x[VPT - 1];
      Sp[VPT - 1] = o0 + VPT - 1;
#pragma unroll
      for (int j = VPT - 2; j >= 0; --j) {
        const bool c = x[j] <= S[j + 1];
        S[j] = c ? x[j] : S[j + 1];
        Sp[j] = c ? (uint32_t)(o0 + j) : Sp[j + 1];
      }
#pragma unroll
      for (int j = 0; j < VPT; ++j) {
        cPv[pad(o0 + j)] = P[j];
        cPp[pad(o0 + j)] = Pp[j];
      }
      cTv[t] = S[0];
      cTp[t] = Sp[0];
      cLast[t] = x[VPT - 1];
      __syncthreads();
      // w - 1 = 16 A + c: window o0 + j ends in chunk t + A (j + c < 16) or t + A + 1; the window
      // [o0, o0 + w - 2] before it ends in chunk t + B, B = (w - 2) / 16.
      const int A = (w - 1) >> 4, c = (w - 1) & 15, B = (w - 2) >> 4;
      V M0 = NONE, Mb = NONE;  // minima of chunks t+1 .. t+A-1 and t+1 .. t+B-1
      uint32_t M0p = 0, Mbp = 0;
      for (int i = 1; i < A; ++i) {
        if (i == B) {
          Mb = M0;
          Mbp = M0p;
        }
        const int u = t + i < FNT ? t + i : FNT - 1;  // past the tile: windows this tile does not emit
        const V v = cTv[u];
        if (v < M0) {
          M0 = v;
          M0p = cTp[u];
        }
      }
      if (B == A) {
        Mb = M0;
        Mbp = M0p;
      }
      V M1 = M0;  // chunks t+1 .. t+A
      uint32_t M1p = M0p;
      {
        const int u = t + A < FNT ? t + A : FNT - 1;
        const V v = cTv[u];
        if (v < M1) {
          M1 = v;
          M1p = cTp[u];
        }
      }
#pragma unroll
      for (int j = 0; j < VPT; ++j) {
        const int q = o0 + j + w - 1 < G::L ? o0 + j + w - 1 : G::L - 1;
        const bool far = j + c >= 16;
        V acc = S[j];
        uint32_t accp = Sp[j];
        const V m = far ? M1 : M0;
        if (m < acc) {
          acc = m;
          accp = far ? M1p : M0p;
        }
        const V pv = cPv[pad(q)];
        if (pv < acc) {
          acc = pv;
          accp = cPp[pad(q)];
        }
        y[j] = acc;
        yp[j] = accp;
      }
      // the window before: k-mer o0 - 1, then [o0, o0 + w - 2] (the whole chunk when w = 17)
      V part = S[0];
      uint32_t partp = Sp[0];
      if (B > 0) {
        if (Mb < part) {
          part = Mb;
          partp = Mbp;
        }
        const int q = o0 + w - 2 < G::L ? o0 + w - 2 : G::L - 1;
        const V pv = cPv[pad(q)];
        if (pv < part) {
          part = pv;
          partp = cPp[pad(q)];
        }
      }
      const V xprev = t > 0 ? cLast[t - 1] : NONE;
      ypprev = xprev <= part ? (uint32_t)(o0 - 1) : partp;
    }

    // ---- window validity -------------------------------------------------------------------------
    unsigned vmask;
    bool pvalid;
    uint32_t qj[BAR == BAR_READS ? VPT : 1];  // barrier index of each window (read batches)
    if (interior) {
      vmask = (1u << VPT) - 1u;
      pvalid = true;
#pragma unroll
      for (int j = 0; j < (BAR == BAR_READS ? VPT : 1); ++j) qj[j] = 0;
    } else {
      uint32_t q = 0, hi = nb;
      const long long pf = ifirst - 1;
      while (q < hi) {
        const uint32_t mid = (q + hi) >> 1;
        if (bar_end(mid) > pf) hi = mid;
        else q = mid + 1;
      }
      auto valid_at = [&](long long p, uint32_t qq) {
        const bool in_range = p >= 0 && (unsigned long long)p < nwin;
        const bool clear = (qq == nb) || (bar_start(qq) > p + span - 1);
        return in_range && clear;
      };
      pvalid = valid_at(pf, q);
      vmask = 0;
      if (q == nb || bar_end(q) > ifirst + VPT - 1) {
        // No barrier ends among this thread's windows (the common case, also in read batches), so
        // barrier q bounds them all: the valid ones are p in [0, nwin) with p + span - 1 below its
        // start, a run of consecutive j.
        long long jlo = -ifirst, jhi = (long long)nwin - ifirst;
        if (q < nb) {
          const long long lim = bar_start(q) - span + 1 - ifirst;
          if (lim < jhi) jhi = lim;
        }
        if (jlo < 0) jlo = 0;
        if (jhi > VPT) jhi = VPT;
        if (jhi > jlo) vmask = ((1u << jhi) - 1u) & ~((1u << jlo) - 1u);
        if (BAR == BAR_READS) {
#pragma unroll
          for (int j = 0; j < (BAR == BAR_READS ? VPT : 1); ++j) qj[j] = q;
        }
      } else {
#pragma unroll
        for (int j = 0; j < VPT; ++j) {
          const long long p = ifirst + j;
          while (q < nb && bar_end(q) <= p) ++q;
          if (BAR == BAR_READS) qj[BAR == BAR_READS ? j : 0] = q;
          vmask |= (unsigned)valid_at(p, q) << j;
        }
      }
    }
    if (!ok) {
      vmask = 0;
      pvalid = false;
    }

    // ---- windows that store a pick: valid, and the previous window invalid or picked elsewhere ---
    // windows this tile emits are o in [w, w + TW): all but those of the first and last threads
    unsigned rmask = (1u << VPT) - 1u;
    if (o0 < w) rmask &= ~((1u << (w - o0 < VPT ? w - o0 : VPT)) - 1u);
    if (o0 + VPT > w + TW) rmask &= (1u << (w + TW - o0 > 0 ? w + TW - o0 : 0)) - 1u;
    unsigned emask = 0, firstmask = 0;
    if (pvalid && vmask == (1u << VPT) - 1u) {  // every window valid (the common case)
      uint32_t pp = ypprev;
#pragma unroll
      for (int j = 0; j < VPT; ++j) {
        emask |= (unsigned)(yp[j] != pp) << j;
        pp = yp[j];
      }
    } else {
      bool pv = pvalid;  // validity of the window before (not limited to this tile's range)
      uint32_t pp = ypprev;
#pragma unroll
      for (int j = 0; j < VPT; ++j) {
        const bool v = (vmask >> j) & 1u;
        const bool e = v && (!pv || yp[j] != pp);
        emask |= (unsigned)e << j;
        firstmask |= (unsigned)(e && !pv) << j;
        pv = v;
        pp = yp[j];
      }
    }
    emask &= rmask;
    firstmask &= rmask;
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
    for (int i = 0; i < FNW; ++i) {
      const uint32_t c = s_wcount[i];
      if (i < warp) woff += c;
      total += c;
    }
    if (!a.count_only) {
      uint32_t r = woff + inc - cnt;
#pragma unroll
      for (int j = 0; j < VPT; ++j) {
        if ((emask >> j) & 1u) {
          uint32_t pos = pos_base + yp[j];
          if (BAR == BAR_READS) {
            const uint32_t rd = g_lo + qj[BAR == BAR_READS ? j : 0];
            pos = (uint32_t)((long long)pos - a.bar[rd]);
            sh_first[r] = ((firstmask >> j) & 1u) ? rd : 0xFFFFFFFFu;
          }
          sh_hash[r] = y[j];
          sh_pos[r] = pos;
          ++r;
        }
      }
    }
    __syncthreads();
    const uint64_t slot = (uint64_t)tile * TW;
    for (uint32_t i = t; i < (a.count_only ? 0u : total); i += FNT) {
      static_cast<V *>(a.stg_hash)[slot + i] = sh_hash[i];
      a.stg_pos[slot + i] = sh_pos[i];
      if (BAR == BAR_READS) a.stg_first[slot + i] = sh_first[i];
    }
    if (t == 0) a.tile_counts[tile] = total;
    __syncthreads();
  }
}

// Step 3: one CTA per tile copies its staged picks to their place (offsets = scanned counts).
// Each thread loads up to four picks before it stores any, so a CTA keeps many independent
// requests in flight (the copy is latency bound otherwise).
constexpr int GNT = 256, GUNROLL = 4;

template <int BAR, class V>
__global__ void __launch_bounds__(GNT) k_mini_gather(MiniArgs a, uint32_t num_tiles, int TW) {
  if (a.desc) num_tiles = (uint32_t)a.desc[BD_TILES];
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.count_out = a.tile_counts[num_tiles];
  V *gh = static_cast<V *>(a.hash_out);
  const V *sh = static_cast<const V *>(a.stg_hash);
  for (uint32_t tile = blockIdx.x; tile < num_tiles; tile += gridDim.x) {
    const uint32_t o = a.tile_counts[tile], c = a.tile_counts[tile + 1] - o;
    const uint64_t slot = tile * (uint64_t)TW;
    for (uint32_t b = 0; b < c; b += GNT * GUNROLL) {
      V h[GUNROLL];
      uint32_t p[GUNROLL], f[GUNROLL];
#pragma unroll
      for (int u = 0; u < GUNROLL; ++u) {
        const uint32_t i = b + u * GNT + threadIdx.x;
        if (i < c) {
          h[u] = sh[slot + i];
          p[u] = a.stg_pos[slot + i];
          f[u] = BAR == BAR_READS ? a.stg_first[slot + i] : 0xFFFFFFFFu;
        }
      }
#pragma unroll
      for (int u = 0; u < GUNROLL; ++u) {
        const uint32_t i = b + u * GNT + threadIdx.x;
        if (i < c) {
          const uint64_t gi = (uint64_t)o + i;
          if (gi < a.capacity) {
            gh[gi] = h[u];
            a.pos_out[gi] = p[u];
          }
          if (BAR == BAR_READS && f[u] != 0xFFFFFFFFu) a.pick_offsets[f[u]] = gi;
        }
      }
    }
  }
}

// Count-only runs: the total from the scanned per-tile counts.
__global__ void k_mini_total(MiniArgs a, uint32_t num_tiles) {
  if (a.desc) num_tiles = (uint32_t)a.desc[BD_TILES];
  if (threadIdx.x == 0) *a.count_out = a.tile_counts[num_tiles];
}

template <int W, int BAR, int SRC, class V>
cudaError_t launch_w(const MiniArgs &a, uint64_t num_tiles, const uint2 *tile_bar, uint64_t nwin, int span,
                     int num_sms, cudaStream_t st) {
  auto kern = k_mini_stage<W, BAR, SRC, V>;
  const size_t sm = Geo<W, SRC, BAR, V>::BYTES;
  static int per_sm = 0;  // resident CTAs per SM for this instantiation
  if (per_sm == 0) {
    if (sm > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    int b = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, FNT, sm);
    if (e != cudaSuccess) return e;
    per_sm = b > 0 ? b : 1;
  }
  uint64_t grid = (uint64_t)per_sm * (uint64_t)num_sms;
  if (grid > num_tiles) grid = num_tiles;
  kern<<<(unsigned)grid, FNT, sm, st>>>(a, nwin, span, tile_bar, (uint32_t)num_tiles);
  return cudaGetLastError();
}

template <int BAR, int SRC, class V>
cudaError_t launch_bar(const MiniArgs &a, uint64_t num_tiles, const uint2 *tile_bar, uint64_t nwin, int span,
                       int num_sms, cudaStream_t st) {
  switch (a.w) {
    case 4: return launch_w<4, BAR, SRC, V>(a, num_tiles, tile_bar, nwin, span, num_sms, st);
    case 5: return launch_w<5, BAR, SRC, V>(a, num_tiles, tile_bar, nwin, span, num_sms, st);
    case 6: return launch_w<6, BAR, SRC, V>(a, num_tiles, tile_bar, nwin, span, num_sms, st);
    case 7: return launch_w<7, BAR, SRC, V>(a, num_tiles, tile_bar, nwin, span, num_sms, st);
    case 8: return launch_w<8, BAR, SRC, V>(a, num_tiles, tile_bar, nwin, span, num_sms, st);
    case 9: return launch_w<9, BAR, SRC, V>(a, num_tiles, tile_bar, nwin, span, num_sms, st);
    case 10: return launch_w<10, BAR, SRC, V>(a, num_tiles, tile_bar, nwin, span, num_sms, st);
    case 11: return launch_w<11, BAR, SRC, V>(a, num_tiles, tile_bar, nwin, span, num_sms, st);
    case 12: return launch_w<12, BAR, SRC, V>(a, num_tiles, tile_bar, nwin, span, num_sms, st);
    case 13: return launch_w<13, BAR, SRC, V>(a, num_tiles, tile_bar, nwin, span, num_sms, st);
    case 14: return launch_w<14, BAR, SRC, V>(a, num_tiles, tile_bar, nwin, span, num_sms, st);
    case 15: return launch_w<15, BAR, SRC, V>(a, num_tiles, tile_bar, nwin, span, num_sms, st);
    case 16: return launch_w<16, BAR, SRC, V>(a, num_tiles, tile_bar, nwin, span, num_sms, st);
    default:
      if (a.w > 16 && a.w <= CHUNK_MAXW) return launch_w<CHUNK, BAR, SRC, V>(a, num_tiles, tile_bar, nwin, span, num_sms, st);
      return cudaErrorNotSupported;
  }
}

}  // namespace

bool mini_fast_applies(int source, int k, int w) {
  return w >= 4 && w <= CHUNK_MAXW && (source == SRC_KEYS || (k >= 1 && k <= 32));
}

int mini_fast_hash_bytes(int source, int k) { return source == SRC_DNA && 2 * k > 32 ? 8 : 4; }

int mini_fast_tile_windows(int w) {
  if (w >= 4 && w <= 16) return (FNT * (16 / w) - 2) * w;
  return w > 16 && w <= CHUNK_MAXW ? chunk_tile_windows(w) : 0;
}

int mini_staged_tile_windows(int source, int k, int w) {
  return mini_fast_applies(source, k, w) ? mini_fast_tile_windows(w) : mini_tile_windows(w);
}

cudaError_t launch_minimizers_staged(const MiniArgs &a, int source, int barrier, uint64_t num_tiles, cudaStream_t st) {
  if (num_tiles == 0) return cudaSuccess;
  if (num_tiles >= 0xffffffffull) return cudaErrorInvalidValue;
  const bool specialised = mini_fast_applies(source, a.k, a.w);
  const int TW = mini_staged_tile_windows(source, a.k, a.w);
  const int span = source == SRC_DNA ? a.w + a.k - 1 : a.w;
  const uint64_t nwin = a.n >= (uint64_t)span ? a.n - span + 1 : 0;
  cudaError_t e = launch_tile_barriers(a, source, barrier, num_tiles, TW, span, st);
  if (e != cudaSuccess) return e;
  const uint2 *tile_bar = tile_barriers_needed(a, source, barrier) ? a.tile_bar : nullptr;
  int dev = 0, num_sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const bool k64 = mini_fast_hash_bytes(source, a.k) == 8;
  using U64 = unsigned long long;
  if (!specialised) e = launch_minimizers_generic_staged(a, source, barrier, num_tiles, tile_bar, st);
  else if (source == SRC_KEYS) e = launch_bar<BAR_NBLOCK, SRC_KEYS, uint32_t>(a, num_tiles, nullptr, nwin, span, num_sms, st);
  else if (barrier == BAR_READS)
    e = k64 ? launch_bar<BAR_READS, SRC_DNA, U64>(a, num_tiles, tile_bar, nwin, span, num_sms, st)
            : launch_bar<BAR_READS, SRC_DNA, uint32_t>(a, num_tiles, tile_bar, nwin, span, num_sms, st);
  else
    e = k64 ? launch_bar<BAR_NBLOCK, SRC_DNA, U64>(a, num_tiles, tile_bar, nwin, span, num_sms, st)
            : launch_bar<BAR_NBLOCK, SRC_DNA, uint32_t>(a, num_tiles, tile_bar, nwin, span, num_sms, st);
  if (e != cudaSuccess) return e;
  if (a.desc) e = scan_u32_dev(a.tile_counts, num_tiles + 1, a.desc + BD_SCAN_LEN, a.scan_tmp, st);
  else e = scan_u32(a.tile_counts, num_tiles + 1, a.scan_tmp, st);
  if (e != cudaSuccess) return e;
  if (a.count_only) {
    k_mini_total<<<1, 32, 0, st>>>(a, (uint32_t)num_tiles);
    return cudaGetLastError();
  }
  const unsigned blocks = (unsigned)(num_tiles < (1u << 20) ? num_tiles : (1u << 20));
  if (barrier == BAR_READS) {
    if (k64) k_mini_gather<BAR_READS, U64><<<blocks, GNT, 0, st>>>(a, (uint32_t)num_tiles, TW);
    else k_mini_gather<BAR_READS, uint32_t><<<blocks, GNT, 0, st>>>(a, (uint32_t)num_tiles, TW);
  } else {
    if (k64) k_mini_gather<BAR_NBLOCK, U64><<<blocks, GNT, 0, st>>>(a, (uint32_t)num_tiles, TW);
    else k_mini_gather<BAR_NBLOCK, uint32_t><<<blocks, GNT, 0, st>>>(a, (uint32_t)num_tiles, TW);
  }
  return cudaGetLastError();
}

}  // namespace sws
