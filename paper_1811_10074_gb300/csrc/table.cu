// table.cu -- the seed table of Sec. 2.4 (Fig. 1): a position table listing every (seed, position)
// hit sorted by seed, and a pointer table giving, for each bucket of seed values, where its hits
// begin.  Here seeds are the minimizer hashes; bucket(h) = h >> (hash_bits - bucket_bits).
//
// The position table is a stable LSD radix sort over the hash bits, 8 bits per pass.  When the
// hash has at most 32 bits, hash and position travel as one 64-bit key (hash << 32 | pos), so a
// pass moves 8 bytes per hit in and out; otherwise the hash is a 64-bit key and the position a
// 32-bit value.  A pass is three kernels: per-tile digit histograms (digit-major), an exclusive
// scan of them, and a scatter in which each CTA ranks its tile's digits stably (warp-striped
// tiles, __match_any_sync peer groups, per-warp running counters), stages the tile in digit order
// in shared memory, and writes runs of equal digits to consecutive addresses.  Stability keeps the
// input order (positions ascending, as minimizers come out) within equal hashes.
//
// The pointer table: offsets[b] = index of the first hit whose bucket is >= b, filled by one pass
// over the sorted hashes; each hit fills the gap of buckets since its predecessor (long gaps are
// deferred to a second, grid-wide fill).
#include <cstdint>

#include "../../include/sws.h"
#include "common.cuh"
#include "internal.h"

namespace sws {

namespace {

constexpr int RNT = 256;        // threads per CTA
constexpr int RKPT = 16;        // keys per thread
constexpr int RTILE = RNT * RKPT;
constexpr int RBINS = 256;
constexpr int RWARPS = RNT / 32;
constexpr int SCAN_NT = 256, SCAN_PER = 16, SCAN_BLOCK = SCAN_NT * SCAN_PER;
constexpr uint32_t GAP_DIRECT = 256;  // gaps up to this many buckets are filled by their thread

// ---- pass input / output ------------------------------------------------------------------
// Pass input: either the caller's (hash, pos) arrays or the previous pass's keys.
struct PassIn {
  const unsigned long long *keys;  // previous pass (or nullptr: read the caller's arrays)
  const uint32_t *vals;            // previous pass values (WIDE only)
  const uint32_t *hash32;          // caller input, hash_bits <= 32
  const unsigned long long *hash64;
  const uint32_t *pos;
};
struct PassOut {
  unsigned long long *keys;  // next pass (or nullptr: write the caller's arrays)
  uint32_t *vals;
  uint32_t *hash32;
  unsigned long long *hash64;
  uint32_t *pos;
};

template <bool WIDE>
__device__ __forceinline__ void fetch(const PassIn &in, uint64_t i, unsigned long long &key, uint32_t &val) {
  if (in.keys) {
    key = in.keys[i];
    if (WIDE) val = in.vals[i];
  } else if (!WIDE) {
    key = ((unsigned long long)in.hash32[i] << 32) | in.pos[i];
  } else {
    key = in.hash64[i];
    val = in.pos[i];
  }
}

template <bool WIDE>
__device__ __forceinline__ void emit(const PassOut &out, uint64_t i, unsigned long long key, uint32_t val) {
  if (out.keys) {
    out.keys[i] = key;
    if (WIDE) out.vals[i] = val;
  } else if (!WIDE) {
    out.hash32[i] = (uint32_t)(key >> 32);
    out.pos[i] = (uint32_t)key;
  } else {
    out.hash64[i] = key;
    out.pos[i] = val;
  }
}

__device__ __forceinline__ int digit_of(unsigned long long key, int shift) { return (int)((key >> shift) & 0xFFull); }

// Lanes of the warp holding the same digit as this lane (valid lanes only match valid lanes):
// one ballot per digit bit.  Ballots issue on the ordinary pipes; __match_any_sync, which computes
// the same mask, occupies the address-divergence unit for many cycles per call and bounded the
// scatter kernel.
__device__ __forceinline__ unsigned digit_peers(int d, bool valid) {
  const unsigned vb = __ballot_sync(kFull, valid);
  unsigned peers = valid ? vb : ~vb;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const bool bit = (d >> b) & 1;
    const unsigned m = __ballot_sync(kFull, bit);
    peers &= bit ? m : ~m;
  }
  return peers;
}

// ---- per-tile digit histograms --------------------------------------------------------------
template <bool WIDE>
__global__ void __launch_bounds__(RNT) k_radix_hist(PassIn in, uint64_t m, int shift, uint32_t *__restrict__ hist,
                                                    uint32_t ntiles) {
  __shared__ uint32_t h[RBINS];
  const int t = threadIdx.x;
  h[t] = 0;
  __syncthreads();
  const uint64_t base = (uint64_t)blockIdx.x * RTILE;
  // all loads first (the digit needs the key only, not the position of a wide key), then the counts
  unsigned long long key[RKPT];
#pragma unroll
  for (int j = 0; j < RKPT; ++j) {
    const uint64_t i = base + (uint64_t)j * RNT + t;
    key[j] = 0;
    if (i < m)
      key[j] = in.keys ? in.keys[i] : WIDE ? in.hash64[i] : (unsigned long long)in.hash32[i] << 32;
  }
#pragma unroll
  for (int j = 0; j < RKPT; ++j)
    if (base + (uint64_t)j * RNT + t < m) atomicAdd(&h[digit_of(key[j], shift)], 1u);
  __syncthreads();
  hist[(uint64_t)t * ntiles + blockIdx.x] = h[t];
}

// ---- exclusive scan of uint32 counts (three kernels) ------------------------------------------
__global__ void __launch_bounds__(SCAN_NT) k_scan_reduce(const uint32_t *__restrict__ a, uint64_t len,
                                                         uint32_t *__restrict__ bsum,
                                                         const unsigned long long *__restrict__ dlen) {
  __shared__ uint32_t s[SCAN_NT / 32];
  if (dlen) len = *dlen;
  const uint64_t b0 = (uint64_t)blockIdx.x * SCAN_BLOCK;
  if (b0 >= len && b0 > 0) return;
  uint32_t v = 0;
  for (int j = 0; j < SCAN_PER; ++j) {
    const uint64_t i = b0 + (uint64_t)j * SCAN_NT + threadIdx.x;
    if (i < len) v += a[i];
  }
  v = __reduce_add_sync(kFull, v);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int i = 0; i < SCAN_NT / 32; ++i) t += s[i];
    bsum[blockIdx.x] = t;
  }
}

// Exclusive scan of the block sums by one CTA (sequential over chunks of SCAN_NT).
__global__ void __launch_bounds__(SCAN_NT) k_scan_blocks(uint32_t *__restrict__ bsum, uint64_t nb,
                                                         const unsigned long long *__restrict__ dlen) {
  __shared__ uint32_t s[SCAN_NT / 32];
  __shared__ uint32_t carry;
  if (dlen) nb = (*dlen + SCAN_BLOCK - 1) / SCAN_BLOCK;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint64_t c = 0; c < nb; c += SCAN_NT) {
    const uint64_t i = c + threadIdx.x;
    const uint32_t v = i < nb ? bsum[i] : 0u;
    uint32_t inc = v;
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t u = __shfl_up_sync(kFull, inc, d);
      if (lane >= d) inc += u;
    }
    if (lane == 31) s[warp] = inc;
    __syncthreads();
    uint32_t off = carry;
    uint32_t tot = 0;
    for (int k = 0; k < SCAN_NT / 32; ++k) {
      if (k < warp) off += s[k];
      tot += s[k];
    }
    if (i < nb) bsum[i] = off + inc - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(SCAN_NT) k_scan_apply(uint32_t *__restrict__ a, uint64_t len,
                                                        const uint32_t *__restrict__ bsum,
                                                        const unsigned long long *__restrict__ dlen) {
  __shared__ uint32_t s[SCAN_NT / 32];
  if (dlen) len = *dlen;
  if ((uint64_t)blockIdx.x * SCAN_BLOCK >= len) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t b0 = (uint64_t)blockIdx.x * SCAN_BLOCK + (uint64_t)threadIdx.x * SCAN_PER;
  uint32_t v[SCAN_PER];
  uint32_t tot = 0;
#pragma unroll
  for (int j = 0; j < SCAN_PER; ++j) {
    v[j] = (b0 + j < len) ? a[b0 + j] : 0u;
    tot += v[j];
  }
  uint32_t inc = tot;
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t u = __shfl_up_sync(kFull, inc, d);
    if (lane >= d) inc += u;
  }
  if (lane == 31) s[warp] = inc;
  __syncthreads();
  uint32_t off = bsum[blockIdx.x];
  for (int k = 0; k < warp; ++k) off += s[k];
  off += inc - tot;
#pragma unroll
  for (int j = 0; j < SCAN_PER; ++j) {
    if (b0 + j < len) a[b0 + j] = off;
    off += v[j];
  }
}

// ---- stable scatter ---------------------------------------------------------------------------
// One CTA per tile.  A wide key's value (the position) is parked in shared memory in input order
// as soon as it is loaded, so it holds no register while the keys are ranked; the digit and the
// key's rank within its warp share one register.  (A persistent form that loads the next tile while
// writing this one out measured slower, and so did 4-byte cp.async copies of the values.)
template <bool WIDE>
__global__ void __launch_bounds__(RNT, 3) k_radix_scatter(PassIn in, PassOut out, uint64_t m, int shift,
                                                          const uint32_t *__restrict__ hist, uint32_t ntiles) {
  extern __shared__ __align__(16) unsigned char rsm[];
  unsigned long long *s_keys = reinterpret_cast<unsigned long long *>(rsm);          // RTILE
  uint32_t *s_vals = reinterpret_cast<uint32_t *>(s_keys + RTILE);                  // RTILE if WIDE
  uint32_t *s_vraw = s_vals + (WIDE ? RTILE : 0);                                   // RTILE if WIDE
  uint32_t(*s_wcnt)[RBINS] = reinterpret_cast<uint32_t(*)[RBINS]>(s_vraw + (WIDE ? RTILE : 0));
  __shared__ uint32_t s_tstart[RBINS];  // tile-local start of each digit
  __shared__ uint32_t s_delta[RBINS];   // global start of each digit for this tile - s_tstart
  __shared__ uint32_t s_wsum[RWARPS];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const uint64_t base = (uint64_t)blockIdx.x * RTILE;
  const uint64_t wbase = base + (uint64_t)warp * (RKPT * 32);
  const int wslot = warp * (RKPT * 32) + lane;  // s_vraw slot of key j: wslot + 32 j

  for (int i = t; i < RWARPS * RBINS; i += RNT) (&s_wcnt[0][0])[i] = 0;
  __syncthreads();

  unsigned long long key[RKPT];
  uint32_t rd[RKPT];  // digit << 16 | rank within the warp (ranks < 512; digit RBINS past the end)
#pragma unroll
  for (int j = 0; j < RKPT; ++j) {
    const uint64_t i = wbase + (uint64_t)j * 32 + lane;
    key[j] = 0;
    rd[j] = (uint32_t)RBINS << 16;  // out of range: its own peer group, never written
    if (i < m) {
      if (WIDE) {
        key[j] = in.keys ? in.keys[i] : in.hash64[i];
        s_vraw[wslot + 32 * j] = in.keys ? in.vals[i] : in.pos[i];
      } else {
        key[j] = in.keys ? in.keys[i] : ((unsigned long long)in.hash32[i] << 32) | in.pos[i];
      }
      rd[j] = (uint32_t)digit_of(key[j], shift) << 16;
    }
  }
  // stable ranks within the warp's 512 keys, in index order (j, then lane)
#pragma unroll
  for (int j = 0; j < RKPT; ++j) {
    const int d = (int)(rd[j] >> 16);
    const unsigned peers = digit_peers(d, d < RBINS);
    const int leader = __ffs(peers) - 1;
    const uint32_t before = __popc(peers & lanemask_lt(lane));
    uint32_t b = 0;
    if (lane == leader && d < RBINS) {
      b = s_wcnt[warp][d];
      s_wcnt[warp][d] = b + (uint32_t)__popc(peers);
    }
    b = __shfl_sync(kFull, b, leader);
    rd[j] |= b + before;
    __syncwarp();
  }
  __syncthreads();
  // digit t: offsets of each warp, tile total, tile-local start (exclusive scan over digits)
  {
    uint32_t run = 0;
    for (int wq = 0; wq < RWARPS; ++wq) {
      const uint32_t c = s_wcnt[wq][t];
      s_wcnt[wq][t] = run;
      run += c;
    }
    uint32_t inc = run;
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t u = __shfl_up_sync(kFull, inc, d);
      if (lane >= d) inc += u;
    }
    if (lane == 31) s_wsum[warp] = inc;
    s_delta[t] = hist[(uint64_t)t * ntiles + blockIdx.x];  // the digit's global start, for now
    __syncthreads();
    uint32_t off = 0;
    for (int k = 0; k < warp; ++k) off += s_wsum[k];
    const uint32_t tstart = off + inc - run;
    s_tstart[t] = tstart;
    s_delta[t] -= tstart;  // >= 0: the tile's keys of smaller digits all precede the global start
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < RKPT; ++j) {
    const int d = (int)(rd[j] >> 16);
    if (d < RBINS) {
      const uint32_t idx = s_tstart[d] + s_wcnt[warp][d] + (rd[j] & 0xFFFFu);
      s_keys[idx] = key[j];
      if (WIDE) s_vals[idx] = s_vraw[wslot + 32 * j];
    }
  }
  __syncthreads();
  const uint64_t left = m - base;
  const uint32_t cnt = left < (uint64_t)RTILE ? (uint32_t)left : (uint32_t)RTILE;
  for (uint32_t i = t; i < cnt; i += RNT) {
    const unsigned long long k = s_keys[i];
    const uint64_t dst = (uint64_t)s_delta[digit_of(k, shift)] + i;
    emit<WIDE>(out, dst, k, s_vals[WIDE ? i : 0]);
  }
}

// ---- pointer table ----------------------------------------------------------------------------
struct Gap {
  uint64_t lo, hi;  // buckets [lo, hi] receive `val`
  uint64_t val;
};

template <bool WIDE>
__device__ __forceinline__ uint64_t bucket_at(const void *sorted_hash, uint64_t i, int shift) {
  if (WIDE) return static_cast<const unsigned long long *>(sorted_hash)[i] >> shift;
  return (uint64_t)(static_cast<const uint32_t *>(sorted_hash)[i] >> shift);
}

template <bool WIDE>
__global__ void k_offsets_fill(const void *__restrict__ sorted_hash, uint64_t m, int shift, uint64_t nbuckets,
                               uint64_t *__restrict__ offsets, Gap *__restrict__ gaps,
                               unsigned long long *__restrict__ ngaps, uint64_t gap_cap) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > m) return;
  // hit i (or the end sentinel) starts every bucket after its predecessor's, up to its own
  const uint64_t lo = i == 0 ? 0 : bucket_at<WIDE>(sorted_hash, i - 1, shift) + 1;
  const uint64_t hi = i == m ? nbuckets : bucket_at<WIDE>(sorted_hash, i, shift);
  if (hi < lo) return;
  if (hi - lo < GAP_DIRECT) {
    for (uint64_t b = lo; b <= hi; ++b) offsets[b] = i;
  } else {
    const unsigned long long slot = atomicAdd(ngaps, 1ull);
    if (slot < gap_cap) gaps[slot] = Gap{lo, hi, i};
  }
}

__global__ void k_offsets_gaps(uint64_t *__restrict__ offsets, const Gap *__restrict__ gaps,
                               const unsigned long long *__restrict__ ngaps, uint64_t gap_cap) {
  uint64_t n = *ngaps;
  if (n > gap_cap) n = gap_cap;
  for (uint64_t gidx = blockIdx.x; gidx < n; gidx += gridDim.x) {
    const Gap g = gaps[gidx];
    for (uint64_t b = g.lo + threadIdx.x; b <= g.hi; b += blockDim.x) offsets[b] = g.val;
  }
}

template <bool WIDE>
cudaError_t sort_t(const TableArgs &a, cudaStream_t st) {
  const uint64_t m = a.m;
  const uint32_t ntiles = (uint32_t)((m + RTILE - 1) / RTILE);
  const int passes = (a.hash_bits + 7) / 8;
  const int key_shift0 = WIDE ? 0 : 32;
  unsigned long long *buf[2] = {a.ws_keys[0], a.ws_keys[1]};
  uint32_t *vbuf[2] = {a.ws_vals[0], a.ws_vals[1]};
  for (int p = 0; p < passes; ++p) {
    PassIn in{};
    PassOut out{};
    if (p == 0) {
      in.hash32 = static_cast<const uint32_t *>(a.hash);
      in.hash64 = static_cast<const unsigned long long *>(a.hash);
      in.pos = a.pos;
    } else {
      in.keys = buf[(p - 1) & 1];
      in.vals = vbuf[(p - 1) & 1];
    }
    if (p == passes - 1) {
      out.hash32 = static_cast<uint32_t *>(a.sorted_hash);
      out.hash64 = static_cast<unsigned long long *>(a.sorted_hash);
      out.pos = a.sorted_pos;
    } else {
      out.keys = buf[p & 1];
      out.vals = vbuf[p & 1];
    }
    const int shift = key_shift0 + 8 * p;
    k_radix_hist<WIDE><<<ntiles, RNT, 0, st>>>(in, m, shift, a.ws_hist, ntiles);
    cudaError_t e = scan_u32(a.ws_hist, (uint64_t)RBINS * ntiles, a.ws_bsum, st);
    if (e != cudaSuccess) return e;
    const size_t sm = (size_t)RTILE * (8 + (WIDE ? 8 : 0)) + (size_t)RWARPS * RBINS * 4;
    if (p == 0 && sm > 48 * 1024) {
      e = cudaFuncSetAttribute(k_radix_scatter<WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    k_radix_scatter<WIDE><<<ntiles, RNT, sm, st>>>(in, out, m, shift, a.ws_hist, ntiles);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <bool WIDE>
cudaError_t offsets_t(const TableArgs &a, cudaStream_t st) {
  const int shift = a.hash_bits - a.bucket_bits;
  const uint64_t nbuckets = 1ull << a.bucket_bits;
  cudaError_t e = cudaMemsetAsync(a.ws_ngaps, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const uint64_t threads = a.m + 1;
  k_offsets_fill<WIDE><<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
      a.sorted_hash, a.m, shift, nbuckets, a.offsets, reinterpret_cast<Gap *>(a.ws_gaps), a.ws_ngaps, a.gap_cap);
  k_offsets_gaps<<<1024, 256, 0, st>>>(a.offsets, reinterpret_cast<const Gap *>(a.ws_gaps), a.ws_ngaps, a.gap_cap);
  return cudaGetLastError();
}

}  // namespace

uint64_t scan_u32_scratch_words(uint64_t len) { return (len + SCAN_BLOCK - 1) / SCAN_BLOCK + 1; }

cudaError_t scan_u32(uint32_t *a, uint64_t len, uint32_t *bsum, cudaStream_t st) {
  const uint64_t nb = (len + SCAN_BLOCK - 1) / SCAN_BLOCK;
  if (nb == 0) return cudaSuccess;
  k_scan_reduce<<<(unsigned)nb, SCAN_NT, 0, st>>>(a, len, bsum, nullptr);
  k_scan_blocks<<<1, SCAN_NT, 0, st>>>(bsum, nb, nullptr);
  k_scan_apply<<<(unsigned)nb, SCAN_NT, 0, st>>>(a, len, bsum, nullptr);
  return cudaGetLastError();
}

cudaError_t scan_u32_dev(uint32_t *a, uint64_t max_len, const unsigned long long *dlen, uint32_t *bsum,
                         cudaStream_t st) {
  const uint64_t nb = (max_len + SCAN_BLOCK - 1) / SCAN_BLOCK;
  if (nb == 0) return cudaSuccess;
  k_scan_reduce<<<(unsigned)nb, SCAN_NT, 0, st>>>(a, max_len, bsum, dlen);
  k_scan_blocks<<<1, SCAN_NT, 0, st>>>(bsum, nb, dlen);
  k_scan_apply<<<(unsigned)nb, SCAN_NT, 0, st>>>(a, max_len, bsum, dlen);
  return cudaGetLastError();
}

uint64_t table_gap_capacity(int bucket_bits) { return ((1ull << bucket_bits) + 1) / (GAP_DIRECT + 1) + 2; }
uint64_t table_hist_words(uint64_t m) { return (uint64_t)RBINS * ((m + RTILE - 1) / RTILE); }
uint64_t table_bsum_words(uint64_t m) { return (table_hist_words(m) + SCAN_BLOCK - 1) / SCAN_BLOCK + 1; }
uint64_t table_gap_bytes(int bucket_bits) { return table_gap_capacity(bucket_bits) * sizeof(Gap); }

cudaError_t launch_table(const TableArgs &a, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (a.m > 0) {
    e = a.hash_bits > 32 ? sort_t<true>(a, st) : sort_t<false>(a, st);
    if (e != cudaSuccess) return e;
  }
  return a.hash_bits > 32 ? offsets_t<true>(a, st) : offsets_t<false>(a, st);
}

}  // namespace sws
