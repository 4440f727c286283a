// seed.cu -- the seeding stage of seed-filter-extend (Sec. 2.3) through the seed table of
// Sec. 2.4 (Fig. 1): for each query seed, the seed pointer table (bucket offsets) and the sorted
// position table give the run of reference hits with the same seed hash.
//
//   k_seed_lookup  one thread per query: bucket range from the pointer table, a binary search in
//                  the bucket for the first equal hash, and a galloping search for the end of
//                  the run of equal hashes -> (first, count).
//   k_hits_count   per tile of queries, the number of hits kept by the repeat filter (a seed with
//                  more than max_occ hits is dropped);
//   k_hits_scan    exclusive scan of the tile totals (one CTA, 64-bit);
//   k_hits_write   per tile again: each query's kept hits as (query, position) pairs at its
//                  offset, in query order and, per query, in position order (the position table
//                  keeps positions ascending within a hash).
#include <cstdint>

#include "../../include/sws.h"
#include "common.cuh"
#include "internal.h"

namespace sws {
namespace {

constexpr int QNT = 256;           // threads per CTA
constexpr int QPT = 4;             // queries per thread in the hit kernels
constexpr int QTILE = QNT * QPT;   // queries per tile

template <bool WIDE>
__device__ __forceinline__ unsigned long long hash_at(const void *h, uint64_t i) {
  if (WIDE) return static_cast<const unsigned long long *>(h)[i];
  return static_cast<const uint32_t *>(h)[i];
}

template <bool WIDE>
__global__ void __launch_bounds__(QNT) k_seed_lookup(const void *__restrict__ sorted_hash, int shift,
                                                     uint64_t nbuckets, const uint64_t *__restrict__ offsets,
                                                     const void *__restrict__ query, uint64_t nq,
                                                     uint64_t *__restrict__ first, uint32_t *__restrict__ count) {
  const uint64_t i = (uint64_t)blockIdx.x * QNT + threadIdx.x;
  if (i >= nq) return;
  const unsigned long long q = hash_at<WIDE>(query, i);
  const uint64_t b = shift >= 64 ? 0 : (uint64_t)(q >> shift);
  if (b >= nbuckets) {  // a hash outside [0, 2^hash_bits): no hits
    first[i] = 0;
    count[i] = 0;
    return;
  }
  uint64_t lo = offsets[b], hi = offsets[b + 1];
  const uint64_t end = hi;
  while (lo < hi) {  // first index of the bucket with hash >= q
    const uint64_t mid = lo + (hi - lo) / 2;
    if (hash_at<WIDE>(sorted_hash, mid) < q) lo = mid + 1;
    else hi = mid;
  }
  const uint64_t a = lo;
  uint64_t c = 0;
  if (a < end && hash_at<WIDE>(sorted_hash, a) == q) {
    // the end of the run by galloping from its start: a seed usually has one or a few hits, so the
    // first probe (next to a, in the same cache line) mostly settles it
    uint64_t known = a + 1, step = 1, probe = a + 1;  // [a, known) all hold q
    while (probe < end && hash_at<WIDE>(sorted_hash, probe) == q) {
      known = probe + 1;
      step <<= 1;
      probe = a + step;
    }
    uint64_t top = probe < end ? probe : end;  // hash at top differs from q, or top = end
    while (known < top) {
      const uint64_t mid = known + (top - known) / 2;
      if (hash_at<WIDE>(sorted_hash, mid) == q) known = mid + 1;
      else top = mid;
    }
    c = known - a;
  }
  first[i] = a;
  count[i] = (uint32_t)c;
}

__device__ __forceinline__ uint32_t kept(uint32_t c, uint32_t max_occ) { return (max_occ == 0 || c <= max_occ) ? c : 0u; }

// Block-wide exclusive scan of per-thread 64-bit values; returns the thread's offset and the total.
__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long v, unsigned long long &total,
                                                             unsigned long long *s_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned long long u = __shfl_up_sync(kFull, inc, d);
    if (lane >= d) inc += u;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  unsigned long long off = 0;
  total = 0;
#pragma unroll
  for (int k = 0; k < QNT / 32; ++k) {
    const unsigned long long c = s_warp[k];
    if (k < warp) off += c;
    total += c;
  }
  return off + inc - v;
}

__global__ void __launch_bounds__(QNT) k_hits_count(const uint32_t *__restrict__ count, uint64_t nq, uint32_t max_occ,
                                                    unsigned long long *__restrict__ tile_sum) {
  __shared__ unsigned long long s_warp[QNT / 32];
  const uint64_t q0 = (uint64_t)blockIdx.x * QTILE + (uint64_t)threadIdx.x * QPT;
  unsigned long long v = 0;
#pragma unroll
  for (int j = 0; j < QPT; ++j)
    if (q0 + j < nq) v += kept(count[q0 + j], max_occ);
  unsigned long long total;
  (void)block_excl_scan(v, total, s_warp);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

// Exclusive scan of the tile totals in place; the grand total goes to *hit_count.
__global__ void __launch_bounds__(QNT) k_hits_scan(unsigned long long *__restrict__ tile_sum, uint64_t ntiles,
                                                   uint64_t *__restrict__ hit_count) {
  __shared__ unsigned long long s_warp[QNT / 32];
  __shared__ unsigned long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint64_t c = 0; c < ntiles; c += QNT) {
    const uint64_t i = c + threadIdx.x;
    const unsigned long long v = i < ntiles ? tile_sum[i] : 0ull;
    unsigned long long total;
    const unsigned long long off = block_excl_scan(v, total, s_warp);
    if (i < ntiles) tile_sum[i] = carry + off;
    __syncthreads();
    if (threadIdx.x == 0) carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) *hit_count = carry;
}

__global__ void __launch_bounds__(QNT) k_hits_write(const uint64_t *__restrict__ first, const uint32_t *__restrict__ count,
                                                    uint64_t nq, uint32_t max_occ,
                                                    const uint32_t *__restrict__ sorted_pos,
                                                    const unsigned long long *__restrict__ tile_off,
                                                    uint32_t *__restrict__ hit_query, uint32_t *__restrict__ hit_pos,
                                                    uint64_t capacity) {
  __shared__ unsigned long long s_warp[QNT / 32];
  const uint64_t q0 = (uint64_t)blockIdx.x * QTILE + (uint64_t)threadIdx.x * QPT;
  uint32_t c[QPT];
  unsigned long long v = 0;
#pragma unroll
  for (int j = 0; j < QPT; ++j) {
    c[j] = q0 + j < nq ? kept(count[q0 + j], max_occ) : 0u;
    v += c[j];
  }
  unsigned long long total;
  unsigned long long o = tile_off[blockIdx.x] + block_excl_scan(v, total, s_warp);
#pragma unroll
  for (int j = 0; j < QPT; ++j) {
    if (c[j] == 0) continue;
    const uint64_t f = first[q0 + j];
    for (uint32_t t = 0; t < c[j]; ++t, ++o) {
      if (o < capacity) {
        hit_query[o] = (uint32_t)(q0 + j);
        hit_pos[o] = sorted_pos[f + t];
      }
    }
  }
}

}  // namespace

uint64_t seed_hit_tiles(uint64_t nq) { return (nq + QTILE - 1) / QTILE; }

cudaError_t launch_seed_lookup(const void *sorted_hash, int hash_bits, int bucket_bits, const uint64_t *offsets,
                               const void *query, uint64_t nq, uint64_t *first, uint32_t *count, cudaStream_t st) {
  if (nq == 0) return cudaSuccess;
  const uint64_t blocks = (nq + QNT - 1) / QNT;
  if (blocks > 0x7fffffffull) return cudaErrorInvalidValue;
  const int shift = hash_bits - bucket_bits;
  const uint64_t nbuckets = 1ull << bucket_bits;
  if (hash_bits > 32)
    k_seed_lookup<true><<<(unsigned)blocks, QNT, 0, st>>>(sorted_hash, shift, nbuckets, offsets, query, nq, first, count);
  else
    k_seed_lookup<false><<<(unsigned)blocks, QNT, 0, st>>>(sorted_hash, shift, nbuckets, offsets, query, nq, first, count);
  return cudaGetLastError();
}

cudaError_t launch_seed_hits(const uint64_t *first, const uint32_t *count, uint64_t nq, uint32_t max_occ,
                             const uint32_t *sorted_pos, uint32_t *hit_query, uint32_t *hit_pos, uint64_t capacity,
                             uint64_t *hit_count, unsigned long long *tile_ws, cudaStream_t st) {
  const uint64_t ntiles = seed_hit_tiles(nq);
  if (ntiles > 0x7fffffffull) return cudaErrorInvalidValue;
  if (ntiles > 0) k_hits_count<<<(unsigned)ntiles, QNT, 0, st>>>(count, nq, max_occ, tile_ws);
  k_hits_scan<<<1, QNT, 0, st>>>(tile_ws, ntiles, hit_count);
  if (ntiles > 0)
    k_hits_write<<<(unsigned)ntiles, QNT, 0, st>>>(first, count, nq, max_occ, sorted_pos, tile_ws, hit_query, hit_pos,
                                                   capacity);
  return cudaGetLastError();
}

}  // namespace sws
