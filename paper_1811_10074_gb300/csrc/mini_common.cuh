// mini_common.cuh -- device pieces shared by the minimizer kernels: TMA bulk staging of packed
// bases (cp.async.bulk completed on an mbarrier, bounded waits), k-mer arithmetic on the packed
// bit stream, Wang's mix, minimizer keys, and the decoupled look-back over per-tile counts.
#pragma once

#include <cstdint>
#include <type_traits>

#include "../../include/sws.h"
#include "common.cuh"
#include "internal.h"
#include "tma.cuh"

namespace sws {
namespace mini {

constexpr unsigned long long FLAG_AGG = 1ull << 62;
constexpr unsigned long long FLAG_INC = 2ull << 62;
constexpr unsigned long long FLAG_ERR = 3ull << 62;
constexpr unsigned long long VALUE_MASK = (1ull << 62) - 1;

// ---- PTX helpers ----------------------------------------------------------------------------
using tma::bulk_g2s;
using tma::fence_mbar_init;
using tma::fence_proxy_async_smem;
using tma::mbar_arrive_expect_tx;
using tma::mbar_init;
using tma::mbar_try_wait;
using tma::smem_u32;

__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
  return v;
}

// Stage bytes [gb0, gb0 + sbytes) of the packed sequence into shared memory (zeros outside
// [0, nbytes)).  The 16-byte-aligned interior goes by one TMA bulk copy completed on an
// mbarrier; the ragged edge bytes are loaded by the threads.  Returns false (and records the
// fault) if the copy did not complete within the spin limit.  With issue = false the copy is
// announced on the mbarrier but never started (the failure self-test: the wait then runs out).
__device__ inline bool stage_bytes(uint8_t *sdst, const uint8_t *__restrict__ seq, uint64_t nbytes, long long gb0,
                            int sbytes, unsigned long long *bar, int *err, bool issue = true) {
  const long long lo = gb0 > 0 ? gb0 : 0;
  long long hi = gb0 + sbytes;
  if (hi > (long long)nbytes) hi = (long long)nbytes;
  const bool aligned = ((reinterpret_cast<uintptr_t>(seq) & 15u) == 0);
  const long long bulk = (aligned && hi > lo) ? ((hi - lo) & ~15ll) : 0;
  if (threadIdx.x == 0 && bulk > 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(bar, (uint32_t)bulk);
    if (issue) bulk_g2s(sdst + (lo - gb0), seq + lo, (uint32_t)bulk, bar);
  }
  for (int b = threadIdx.x; b < sbytes; b += blockDim.x) {
    const long long g = gb0 + b;
    if (g >= lo && g < lo + bulk) continue;
    sdst[b] = (g >= 0 && g < (long long)nbytes) ? seq[g] : (uint8_t)0;
  }
  __syncthreads();
  bool ok = true;
  if (bulk > 0) {
    ok = tma::mbar_wait_bounded(bar, 0);
    if (!ok) {
      atomicOr(err, DEVERR_COPY_TIMEOUT);
      // give an issued copy one more bounded chance to land before the CTA can exit
      if (issue) tma::mbar_wait_bounded(bar, 0);
    }
  }
  return ok;
}

// ---- k-mer arithmetic -----------------------------------------------------------------------
// Wang's 64-bit integer mix, written in its multiplicative form, truncated to the mask m after
// every step (a bijection on [0, m]).
__device__ __forceinline__ uint32_t wang_mix32(uint32_t x, uint32_t m) {
  x = (x * 0x1FFFFFu + 0xFFFFFFFFu) & m;  // (x << 21) - x - 1
  x ^= x >> 24;
  x = (x * 265u) & m;
  x ^= x >> 14;
  x = (x * 21u) & m;
  x ^= x >> 28;
  x = (x * 0x80000001u) & m;
  return x;
}
// wang_mix32 of x, computed on X = x << s (s = 32 - 2k, hm = 0xFFFFFFFF << s) and returned as
// wang_mix32(x, 2^(2k) - 1) << s: arithmetic modulo 2^(2k) in the high 2k bits is plain 32-bit
// arithmetic, so no multiply needs a mask; a right shift clears the low s bits it brings in.  The
// additive constant -1 modulo 2^(2k), shifted, is hm itself.
__device__ __forceinline__ uint32_t wang_mix32_hi(uint32_t X, uint32_t hm) {
  X = X * 0x1FFFFFu + hm;
  X ^= (X >> 24) & hm;
  X *= 265u;
  X ^= (X >> 14) & hm;
  X *= 21u;
  X ^= (X >> 28) & hm;
  X *= 0x80000001u;
  return X;
}
__device__ __forceinline__ unsigned long long wang_mix64(unsigned long long x, unsigned long long m) {
  x = (x * 0x1FFFFFull + 0xFFFFFFFFFFFFFFFFull) & m;
  x ^= x >> 24;
  x = (x * 265ull) & m;
  x ^= x >> 14;
  x = (x * 21ull) & m;
  x ^= x >> 28;
  x = (x * 0x80000001ull) & m;
  return x;
}
// The same mix for a mask m = 2^b - 1 with 32 < b <= 64, given as its high word: the low word
// of m is all ones, so only the high word is ever masked.
__device__ __forceinline__ unsigned long long wang_mix64_wide(unsigned long long x, uint32_t mhi) {
  auto mask = [mhi](unsigned long long v) {
    return ((unsigned long long)((uint32_t)(v >> 32) & mhi) << 32) | (uint32_t)v;
  };
  x = mask(x * 0x1FFFFFull + 0xFFFFFFFFFFFFFFFFull);
  x ^= x >> 24;
  x = mask(x * 265ull);
  x ^= x >> 14;
  x = mask(x * 21ull);
  x ^= x >> 28;
  x = mask(x * 0x80000001ull);
  return x;
}
// wang_mix64_wide when every value it forms stays below 2^(32 + HB) (2k = 32 + HB bits): a right
// shift by s >= HB leaves nothing in the high word, so that xor-shift only changes the low word.
template <int HB>
__device__ __forceinline__ unsigned long long wang_mix64_hb(unsigned long long x, uint32_t mhi) {
  auto mask = [mhi](unsigned long long v) {
    return ((unsigned long long)((uint32_t)(v >> 32) & mhi) << 32) | (uint32_t)v;
  };
  auto xs = [](unsigned long long v, int s) {
    const uint32_t lo = (uint32_t)v, hi = (uint32_t)(v >> 32);
    if (HB <= s) return ((unsigned long long)hi << 32) | (lo ^ __funnelshift_r(lo, hi, s));
    return v ^ (v >> s);
  };
  x = mask(x * 0x1FFFFFull + 0xFFFFFFFFFFFFFFFFull);
  x = xs(x, 24);
  x = mask(x * 265ull);
  x = xs(x, 14);
  x = mask(x * 21ull);
  x = xs(x, 28);
  x = mask(x * 0x80000001ull);
  return x;
}
// Reverse the order of the 2-bit groups of a word.
__device__ __forceinline__ uint32_t rev_pairs32(uint32_t x) {
  x = __brev(x);
  return ((x >> 1) & 0x55555555u) | ((x & 0x55555555u) << 1);
}
__device__ __forceinline__ unsigned long long rev_pairs64(unsigned long long x) {
  x = __brevll(x);
  return ((x >> 1) & 0x5555555555555555ull) | ((x & 0x5555555555555555ull) << 1);
}

// (fwd, rc, canonical, hash, key-value) of one k-mer from the bases in the low bits of x.
struct Kmer32 {
  uint32_t fwd, rc;
};
__device__ __forceinline__ Kmer32 kmer32(uint32_t x, int k, uint32_t kmask) {
  Kmer32 r;
  r.rc = ~x & kmask;
  r.fwd = rev_pairs32(x) >> (32 - 2 * k);
  return r;
}
struct Kmer64 {
  unsigned long long fwd, rc;
};
__device__ __forceinline__ Kmer64 kmer64(unsigned long long x, int k, unsigned long long kmask) {
  Kmer64 r;
  r.rc = ~x & kmask;
  r.fwd = rev_pairs64(x) >> (64 - 2 * k);
  return r;
}
__device__ __forceinline__ uint32_t key_value32(const Kmer32 &q, int mode, uint32_t kmask) {
  if (mode == SWS_MINI_FWD) return q.fwd;
  const uint32_t c = q.fwd < q.rc ? q.fwd : q.rc;
  return mode == SWS_MINI_CANONICAL ? c : wang_mix32(c, kmask);
}
__device__ __forceinline__ unsigned long long key_value64(const Kmer64 &q, int mode, unsigned long long kmask) {
  if (mode == SWS_MINI_FWD) return q.fwd;
  const unsigned long long c = q.fwd < q.rc ? q.fwd : q.rc;
  return mode == SWS_MINI_CANONICAL ? c : wang_mix64(c, kmask);
}
// key_value64 for k > 16 (2k > 32 bits), the mask given by its high word.
__device__ __forceinline__ unsigned long long key_value64_wide(const Kmer64 &q, int mode, uint32_t kmask_hi) {
  if (mode == SWS_MINI_FWD) return q.fwd;
  const unsigned long long c = q.fwd < q.rc ? q.fwd : q.rc;
  return mode == SWS_MINI_CANONICAL ? c : wang_mix64_wide(c, kmask_hi);
}

// ---- keys -----------------------------------------------------------------------------------
template <class KOp>
struct KeyTraits;
template <>
struct KeyTraits<OpMinKey64> {
  using T = unsigned long long;
  static __device__ __forceinline__ T make(unsigned long long h, uint32_t pos) { return (h << 32) | pos; }
  static __device__ __forceinline__ uint32_t pos(T k) { return (uint32_t)k; }
  static __device__ __forceinline__ unsigned long long hash(T k) { return k >> 32; }
  static __device__ __forceinline__ T none() { return ~0ull; }
};
template <>
struct KeyTraits<OpMinKey96> {
  using T = Key96;
  static __device__ __forceinline__ T make(unsigned long long h, uint32_t pos) {
    return Key96{(uint32_t)h, (uint32_t)(h >> 32), pos};
  }
  static __device__ __forceinline__ uint32_t pos(T k) { return k.pos; }
  static __device__ __forceinline__ unsigned long long hash(T k) { return OpMinKey96::h(k); }
  static __device__ __forceinline__ T none() { return OpMinKey96::identity(); }
};

// Warp-level look-back (warp 0 of a CTA): 32 predecessors per poll.  Returns the number of picks
// of all earlier tiles; sets `failed` if a wait ran out or an earlier tile failed.  A tile that
// failed itself (self_failed: its input never arrived) publishes the failure at once instead of a
// count, so every later tile fails too and the final count is never written.
__device__ inline unsigned long long lookback_warp(unsigned long long *status, uint32_t tile, unsigned long long agg,
                                                   int *err, bool &failed, bool self_failed = false) {
  const int lane = threadIdx.x & 31;
  failed = false;
  if (self_failed) {
    if (lane == 0) st_relaxed(&status[tile], FLAG_ERR);
    failed = true;
    return 0;
  }
  if (tile == 0) {
    if (lane == 0) st_relaxed(&status[0], FLAG_INC | agg);
    return 0;
  }
  if (lane == 0) st_relaxed(&status[tile], FLAG_AGG | agg);
  unsigned long long excl = 0;
  long long base = (long long)tile - 1;
  while (true) {
    const long long idx = base - lane;
    unsigned long long s = FLAG_INC;
    unsigned long long t0 = 0;
    while (true) {
      s = idx >= 0 ? ld_relaxed(&status[idx]) : FLAG_INC;
      if (__all_sync(kFull, (s >> 62) != 0ull)) break;
      const unsigned long long now = tma::now_ns();
      if (t0 == 0) t0 = now;
      if (now - t0 > tma::kWaitNs) {
        failed = true;
        break;
      }
      __nanosleep(64);
    }
    if (failed) break;
    if (__ballot_sync(kFull, (s >> 62) == 3ull)) {
      failed = true;
      break;
    }
    const unsigned inc = __ballot_sync(kFull, (s >> 62) == 2ull);
    unsigned long long v = s & VALUE_MASK;
    if (inc) {
      if (lane > __ffs(inc) - 1) v = 0;
      excl += warp_sum_u64(v);
      break;
    }
    excl += warp_sum_u64(v);
    base -= 32;
  }
  if (lane == 0) {
    if (failed) {
      st_relaxed(&status[tile], FLAG_ERR);
      atomicOr(err, DEVERR_LOOKBACK_TIMEOUT);
    } else {
      st_relaxed(&status[tile], FLAG_INC | (excl + agg));
    }
  }
  return excl;
}

}  // namespace mini
}  // namespace sws
