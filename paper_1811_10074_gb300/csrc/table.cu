// table.cu -- the seed table of Sec. 2.4 (Fig. 1): a position table listing every (seed, position)
// hit sorted by seed, and a pointer table giving, for each bucket of seed values, where its hits
// begin.  Here seeds are the minimizer hashes; bucket(h) = h >> (hash_bits - bucket_bits).
//
// The position table is a stable sort by hash.  For 16 < hash_bits <= 40 and at least 2^16 hits
// it is the segmented sort below (two 8-bit MSD passes, then each of the 65,536 buckets sorted on
// its own, in shared memory where it fits).  Otherwise it is a stable LSD radix sort over the hash
// bits, 8 bits per pass: when the hash has at most 32 bits, hash and position travel as one 64-bit
// key (hash << 32 | pos), so a pass moves 8 bytes per hit in and out; otherwise the hash is a
// 64-bit key and the position a 32-bit value.  A pass (of either sort) is three kernels: per-tile
// digit histograms (digit-major), an exclusive scan of them, and a scatter in which each CTA ranks
// its tile's digits stably (warp-striped tiles, ballot peer groups, per-warp running counters),
// stages the tile in digit order in shared memory, and writes runs of equal digits to consecutive
// addresses.  Stability keeps the
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
  // packing pass of the segmented sort: keys receive one 64-bit record per hit,
  // (hash & pack_mask) << 32 | position, and vals is unused
  int pack;
  unsigned long long pack_mask;
};

// A tile of a segmented pass: `count` keys from `start`, column `col` of its segment's block of
// the digit histograms (which holds seg_tiles columns per digit from hist_base on).  A null
// descriptor array means uniform tiles of RTILE keys over [0, m) with one block of ntiles columns.
struct TileDesc {
  unsigned long long start;
  unsigned long long hist_base;
  uint32_t count, seg_tiles, col, pad;
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
  if (out.pack) {
    out.keys[i] = WIDE ? ((key & out.pack_mask) << 32) | val : (key & ((out.pack_mask << 32) | 0xFFFFFFFFull));
  } else if (out.keys) {
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
// Tile `b` of a pass: first key, end, and the index of digit 0 of its histogram column.
struct TileAt {
  uint64_t base, end, h0, hstride;
};
__device__ __forceinline__ TileAt tile_at(const TileDesc *tiles, uint32_t b, uint64_t m, uint32_t ntiles) {
  TileAt r;
  if (tiles) {
    const TileDesc d = tiles[b];
    r.base = d.start;
    r.end = d.start + d.count;
    r.h0 = d.hist_base + d.col;
    r.hstride = d.seg_tiles;
  } else {
    r.base = (uint64_t)b * RTILE;
    r.end = r.base + RTILE < m ? r.base + RTILE : m;
    r.h0 = b;
    r.hstride = ntiles;
  }
  return r;
}

template <bool WIDE>
__global__ void __launch_bounds__(RNT) k_radix_hist(PassIn in, uint64_t m, int shift, uint32_t *__restrict__ hist,
                                                    uint32_t ntiles, const TileDesc *__restrict__ tiles) {
  __shared__ uint32_t h[RBINS];
  const int t = threadIdx.x;
  const TileAt ta = tile_at(tiles, blockIdx.x, m, ntiles);
  if (tiles && ta.end == ta.base) return;  // a descriptor past the last tile of the pass
  m = ta.end;
  h[t] = 0;
  __syncthreads();
  const uint64_t base = ta.base;
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
  hist[ta.h0 + (uint64_t)t * ta.hstride] = h[t];
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
                                                          const uint32_t *__restrict__ hist, uint32_t ntiles,
                                                          const TileDesc *__restrict__ tiles) {
  extern __shared__ __align__(16) unsigned char rsm[];
  unsigned long long *s_keys = reinterpret_cast<unsigned long long *>(rsm);          // RTILE
  uint32_t *s_vals = reinterpret_cast<uint32_t *>(s_keys + RTILE);                  // RTILE if WIDE
  uint32_t *s_vraw = s_vals + (WIDE ? RTILE : 0);                                   // RTILE if WIDE
  uint32_t(*s_wcnt)[RBINS] = reinterpret_cast<uint32_t(*)[RBINS]>(s_vraw + (WIDE ? RTILE : 0));
  __shared__ uint32_t s_tstart[RBINS];  // tile-local start of each digit
  __shared__ uint32_t s_delta[RBINS];   // global start of each digit for this tile - s_tstart
  __shared__ uint32_t s_wsum[RWARPS];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const TileAt ta = tile_at(tiles, blockIdx.x, m, ntiles);
  if (tiles && ta.end == ta.base) return;  // a descriptor past the last tile of the pass
  m = ta.end;
  const uint64_t base = ta.base;
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
    s_delta[t] = hist[ta.h0 + (uint64_t)t * ta.hstride];  // the digit's global start, for now
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
    k_radix_hist<WIDE><<<ntiles, RNT, 0, st>>>(in, m, shift, a.ws_hist, ntiles, nullptr);
    cudaError_t e = scan_u32(a.ws_hist, (uint64_t)RBINS * ntiles, a.ws_bsum, st);
    if (e != cudaSuccess) return e;
    const size_t sm = (size_t)RTILE * (8 + (WIDE ? 8 : 0)) + (size_t)RWARPS * RBINS * 4;
    if (p == 0 && sm > 48 * 1024) {
      e = cudaFuncSetAttribute(k_radix_scatter<WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    k_radix_scatter<WIDE><<<ntiles, RNT, sm, st>>>(in, out, m, shift, a.ws_hist, ntiles, nullptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ---- segmented sort for 16 < hash_bits <= 40 ---------------------------------------------------
// A: one stable pass on the top 8 hash bits (digit g) that packs each hit into a 64-bit record,
//    (low hash_bits - 8 bits) << 32 | position;
// B: one stable pass on the next 8 bits (digit d) within each segment g, tiles never crossing a
//    segment (descriptors built on the device from A's histogram);
// C: every bucket (g, d) -- about m / 65536 hits -- sorted on its own in shared memory, each
//    record's position replaced by its index within the bucket (its input order, which A and B
//    kept), so that sorting by value orders by (hash, input order): the stable order; then the
//    hash is rebuilt from g and the record, and the position read back from the bucket's input.
// 28 bytes per hit in A (8 of histogram, 12 in, 8 out), 24 in B, 20 in C, against 32 per pass in
// the LSD sort.
constexpr int SEG = 256;                   // segments (digit g) and buckets per segment (digit d)
constexpr int BNT = 512;                   // threads of a bucket-sort CTA
constexpr int BSUB_BITS = 12;              // sub-bins of the in-memory counting sort (at most)
constexpr uint32_t BNSUB = 1u << BSUB_BITS;
constexpr int BSUB_BITS2 = 13;             // the same for the big-bucket CTA
constexpr uint32_t BNSUB2 = 1u << BSUB_BITS2;
constexpr uint32_t BCAP = 12288;           // items a CTA sorts in shared memory
constexpr uint32_t BCROWD = 64;            // a fuller sub-bin sends its bucket to the LSD path
constexpr int BKPT = 4;                    // records per thread per chunk of the LSD path
constexpr int BBATCH = 8;                  // loads in flight per thread in the shared-memory sort
constexpr size_t BSMEM = (size_t)BNSUB * 4 + (size_t)BCAP * 4;  // 64 KB: 2 CTAs per SM (registers)
constexpr int BNT2 = 1024;                 // threads of the big-bucket CTA
constexpr uint32_t BCAP2 = 49152;          // items of the big-bucket CTA (one per SM); < 2^16
constexpr size_t BSMEM2 = (size_t)BNSUB2 * 4 + (size_t)BCAP2 * 4;  // 224 KB
constexpr int UNT = 1024;                  // threads of the one CTA that lists the big buckets

// Buckets the shared-memory sort leaves to the LSD path, and the work counter of the kernel that
// takes them.  Zeroed before pass C.
struct BucketLists {
  uint32_t n;
  uint32_t next;
  uint32_t list[SEG * SEG];
};

struct SegInfo {
  unsigned long long start;  // first hit of segment g
  unsigned long long size;
  uint32_t tiles;            // tiles of pass B in the segment
  uint32_t tile0;            // index of its first tile
};

// One CTA: segment bounds from A's scanned histogram (digit-major: digit g, tile 0 at g * ntiles),
// tiles per segment and their prefix.
__global__ void __launch_bounds__(SEG) k_seg_info(const uint32_t *__restrict__ histA, uint32_t ntilesA, uint64_t m,
                                                  SegInfo *__restrict__ seg, uint32_t *__restrict__ total_tiles) {
  __shared__ uint32_t s[SEG / 32];
  const int g = threadIdx.x, lane = g & 31, warp = g >> 5;
  const uint64_t start = histA[(uint64_t)g * ntilesA];
  const uint64_t next = g + 1 < SEG ? histA[(uint64_t)(g + 1) * ntilesA] : m;
  const uint64_t size = next - start;
  const uint32_t nt = (uint32_t)((size + RTILE - 1) / RTILE);
  uint32_t inc = nt;
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t u = __shfl_up_sync(kFull, inc, d);
    if (lane >= d) inc += u;
  }
  if (lane == 31) s[warp] = inc;
  __syncthreads();
  uint32_t off = 0;
  for (int i = 0; i < warp; ++i) off += s[i];
  seg[g] = SegInfo{start, size, nt, off + inc - nt};
  if (g == SEG - 1) *total_tiles = off + inc;
}

// Pass B's tile descriptors: tile i lies in the segment whose tiles cover it.  Descriptors past
// the last tile get count 0 (their CTAs return at once).
__global__ void k_tile_desc(const SegInfo *__restrict__ seg, const uint32_t *__restrict__ total_tiles,
                            uint32_t max_tiles, TileDesc *__restrict__ tiles) {
  __shared__ uint32_t s_t0[SEG];
  for (int g = threadIdx.x; g < SEG; g += blockDim.x) s_t0[g] = seg[g].tile0;
  __syncthreads();
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= max_tiles) return;
  TileDesc d{};
  if (i < *total_tiles) {
    int lo = 0, hi = SEG - 1;  // the last segment with tile0 <= i (segments without tiles share tile0)
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s_t0[mid] <= i) lo = mid;
      else hi = mid - 1;
    }
    while (seg[lo].tiles == 0) --lo;  // an empty segment shares its tile0 with the next one
    const SegInfo sg = seg[lo];
    const uint32_t col = i - sg.tile0;
    const uint64_t st = sg.start + (uint64_t)col * RTILE;
    const uint64_t left = sg.size - (uint64_t)col * RTILE;
    d.start = st;
    d.count = (uint32_t)(left < (uint64_t)RTILE ? left : (uint64_t)RTILE);
    d.seg_tiles = sg.tiles;
    d.col = col;
    d.hist_base = (unsigned long long)SEG * sg.tile0;
  }
  tiles[i] = d;
}

// Bucket (g, d) starts: digit d's entry in column 0 of segment g's block of B's scanned histogram
// (an empty segment: its start).  bstart[SEG * SEG] = m.
__global__ void k_bucket_starts(const SegInfo *__restrict__ seg, const uint32_t *__restrict__ histB, uint64_t m,
                                unsigned long long *__restrict__ bstart) {
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b > SEG * SEG) return;
  if (b == SEG * SEG) {
    bstart[b] = m;
    return;
  }
  const SegInfo sg = seg[b / SEG];
  const uint32_t d = b % SEG;
  bstart[b] = sg.tiles ? histB[(uint64_t)SEG * sg.tile0 + (uint64_t)d * sg.tiles] : sg.start;
}

// Pass C.  Bucket (g, d) -- records of X in input order -- is sorted in shared memory as 4-byte
// items, (hash bits below the sub-bin) << 16 | index of the record within the bucket: a counting
// sort into sub-bins on the top remaining hash bits (shared-memory atomics, in any order); then the
// item at each place of a sub-bin, its record read again from X (by then in L2), goes to the
// sub-bin's start plus its rank among the sub-bin's items, which orders equal hashes by index,
// i.e. stably: the full hash (g << (hash_bits - 8) | record >> 32) and the position (low word).
// A bucket of more than BCAP records is sorted the same way by a CTA that has an SM to itself
// (k_bucket_big).  Buckets of more than BCAP2 records, or with a sub-bin of more than BCROWD (many
// hits of a few hashes), take the LSD path.
__device__ __forceinline__ void bucket_write(unsigned long long rec, uint64_t i, uint32_t g, int hash_bits,
                                             void *sorted_hash, uint32_t *sorted_pos) {
  const unsigned long long h = ((unsigned long long)g << (hash_bits - 8)) | (rec >> 32);
  if (hash_bits > 32) static_cast<unsigned long long *>(sorted_hash)[i] = h;
  else static_cast<uint32_t *>(sorted_hash)[i] = (uint32_t)h;
  sorted_pos[i] = (uint32_t)rec;
}

// The pointer table filled by pass C: with bucket_bits = 16 + e (4 <= e <= 10), sort bucket s holds
// the table buckets [s << e, (s + 1) << e), and their entries depend on its own hits only: entry
// (s << e) + l is the index of its first hit whose table bucket is >= that one (start + n if none).
struct PtrTable {
  uint64_t *offsets;
  int e;  // bucket_bits - 16, or -1: the table is filled elsewhere
};

// The same entries from the bucket's sorted output (the LSD path), once it is visible to the CTA.
__device__ void bucket_offsets(uint32_t s, uint64_t start, uint32_t n, const void *sorted_hash, int hash_bits,
                               PtrTable pt) {
  const int tshift = hash_bits - 16 - pt.e;
  const uint32_t nb = 1u << pt.e, lmask = nb - 1;
  uint64_t *o = pt.offsets + ((uint64_t)s << pt.e);
  auto local = [&](uint32_t j) -> uint32_t {
    const unsigned long long h = hash_bits > 32 ? static_cast<const unsigned long long *>(sorted_hash)[start + j]
                                                : static_cast<const uint32_t *>(sorted_hash)[start + j];
    return (uint32_t)(h >> tshift) & lmask;
  };
  for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) {
    const uint32_t hi = local(j), lo = j ? local(j - 1) + 1 : 0u;  // hit j starts the buckets lo .. hi
    for (uint32_t l = lo; l <= hi; ++l) o[l] = start + j;
  }
  const uint32_t lo = n ? local(n - 1) + 1 : 0u;  // buckets after the last hit
  for (uint32_t l = lo + threadIdx.x; l < nb; l += blockDim.x) o[l] = start + n;
}

// Sub-bins of a bucket: the top sb of the rbits = hash_bits - 16 remaining hash bits; lbits below
// them go into the items; 2^align sub-bins make one table bucket when pass C fills the table.
struct SubBins {
  int sb, sshift, align;
  uint32_t nsub, smask, lmask;
};
__device__ __forceinline__ SubBins sub_bins(int hash_bits, PtrTable pt, int max_bits) {
  SubBins S;
  const int rbits = hash_bits - 16;
  S.sb = rbits < max_bits ? rbits : max_bits;
  S.sshift = 32 + rbits - S.sb;
  S.nsub = 1u << S.sb;
  S.smask = S.nsub - 1;
  S.lmask = (1u << (rbits - S.sb)) - 1u;
  S.align = pt.e >= 0 ? S.sb - pt.e : 0;
  return S;
}

// Sub-bin counters: a 32-bit word each, or (PACK) a 16-bit half each, sub-bin c in half c & 1 of
// word c >> 1 (the values stay below 2^16: a CTA that packs holds at most BCAP2 records).
template <bool PACK>
struct SubCnt {
  uint32_t *w;
  __device__ __forceinline__ uint32_t get(uint32_t c) const {
    return PACK ? (w[c >> 1] >> ((c & 1u) << 4)) & 0xFFFFu : w[c];
  }
  __device__ __forceinline__ uint32_t bump(uint32_t c) const {  // the value before the increment
    if (!PACK) return atomicAdd(&w[c], 1u);
    const uint32_t sh = (c & 1u) << 4;
    return (atomicAdd(&w[c >> 1], 1u << sh) >> sh) & 0xFFFFu;
  }
};

// Counts src[0, n) into the sub-bins and scans the counts into starts.  Returns, in every thread,
// whether a sub-bin holds more than BCROWD records.
template <int NT, uint32_t NSUB, bool PACK>
__device__ bool count_scan(const unsigned long long *__restrict__ src, uint32_t n, const SubBins &S,
                           SubCnt<PACK> cnt, uint32_t *s_w) {
  const uint32_t nr = S.nsub, nwords = PACK ? nr / 2 : nr;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (uint32_t i = t; i < nwords; i += NT) cnt.w[i] = 0;
  __syncthreads();
  // every loop over records issues BBATCH loads per thread before it uses them
  for (uint32_t i0 = t; i0 < n; i0 += NT * BBATCH) {
    unsigned long long r[BBATCH];
#pragma unroll
    for (int q = 0; q < BBATCH; ++q) r[q] = i0 + q * NT < n ? src[i0 + q * NT] : 0ull;
#pragma unroll
    for (int q = 0; q < BBATCH; ++q)
      if (i0 + q * NT < n) cnt.bump((uint32_t)(r[q] >> S.sshift) & S.smask);
  }
  __syncthreads();
  // each thread a run of `per` counts (an even number of whole words when packed)
  constexpr int LOC = (int)(NSUB / NT) > 2 ? (int)(NSUB / NT) : 2;
  uint32_t per = (nr + NT - 1) / NT;
  if (PACK && per < 2) per = 2;
  uint32_t loc[LOC];
  uint32_t tot = 0;
  bool crowd = false;
#pragma unroll
  for (int q = 0; q < LOC; ++q) {
    const uint32_t i = t * per + q;
    loc[q] = (q < (int)per && i < nr) ? cnt.get(i) : 0u;
    crowd |= loc[q] > BCROWD;
    tot += loc[q];
  }
  uint32_t inc = tot;
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t u = __shfl_up_sync(kFull, inc, d);
    if (lane >= d) inc += u;
  }
  if (lane == 31) s_w[warp] = inc;
  __syncthreads();
  uint32_t off = 0;
  for (int i = 0; i < warp; ++i) off += s_w[i];
  off += inc - tot;
  if constexpr (PACK) {  // whole words: sub-bins i (even) and i + 1
#pragma unroll
    for (int q = 0; q < LOC; q += 2) {
      const uint32_t i = t * per + q;
      if (q < (int)per && i < nr) cnt.w[i >> 1] = off | ((off + loc[q]) << 16);
      off += loc[q] + loc[q + 1];
    }
  } else {
#pragma unroll
    for (int q = 0; q < LOC; ++q) {
      const uint32_t i = t * per + q;
      if (q < (int)per && i < nr) cnt.w[i] = off;
      off += loc[q];
    }
  }
  return __syncthreads_or(crowd);
}

// Places src's n records (the bucket's records in input order; starts of the sub-bins in cnt)
// as items by sub-bin, fills the table entries of the sub-bins, and writes the output range
// [start + out0, start + out0 + n): the item at place j of sub-bin c goes to c's start + its rank
// there (the number of smaller items: lower hash bits, or equal bits and a smaller index), so each
// sub-bin comes out ordered by (hash, index) without being sorted in place.  The record an item
// names is read again (from L2), for the output and for its sub-bin.
template <int NT, bool PACK>
__device__ void place_rank_write(const unsigned long long *__restrict__ src, uint32_t n, const SubBins &S,
                                 SubCnt<PACK> cnt, uint32_t *items, uint64_t start, uint32_t out0, uint32_t b,
                                 int hash_bits, void *sorted_hash, uint32_t *sorted_pos, PtrTable pt) {
  const int t = threadIdx.x;
  const uint32_t nr = S.nsub;
  for (uint32_t i0 = t; i0 < n; i0 += NT * BBATCH) {
    unsigned long long r[BBATCH];
#pragma unroll
    for (int q = 0; q < BBATCH; ++q) r[q] = i0 + q * NT < n ? src[i0 + q * NT] : 0ull;
#pragma unroll
    for (int q = 0; q < BBATCH; ++q) {
      const uint32_t i = i0 + q * NT, c = (uint32_t)(r[q] >> S.sshift) & S.smask;
      if (i < n) items[cnt.bump(c)] = (((uint32_t)(r[q] >> 32) & S.lmask) << 16) | i;
    }
  }
  __syncthreads();
  // each counter now holds the end of its sub-bin, i.e. the start of the next
  if (pt.e >= 0) {  // each table bucket starts where its first sub-bin does
    uint64_t *o = pt.offsets + ((uint64_t)b << pt.e);
    for (uint32_t l = t; l < (nr >> S.align); l += NT) {
      const uint32_t f = l << S.align;
      o[l] = start + out0 + (f ? cnt.get(f - 1) : 0u);
    }
  }
  // the output from here, indexed by 32-bit places; the hash's top bits are the segment's
  const unsigned long long hg = (unsigned long long)(b / SEG) << (hash_bits - 8);
  const uint64_t o0 = start + out0;
  unsigned long long *oh64 = static_cast<unsigned long long *>(sorted_hash) + o0;
  uint32_t *oh32 = static_cast<uint32_t *>(sorted_hash) + o0, *op = sorted_pos + o0;
  const bool wide = hash_bits > 32;
  for (uint32_t j0 = t; j0 < n; j0 += NT * BBATCH) {
    uint32_t it[BBATCH];
    unsigned long long r[BBATCH];
#pragma unroll
    for (int q = 0; q < BBATCH; ++q) {
      it[q] = j0 + q * NT < n ? items[j0 + q * NT] : 0u;
      r[q] = j0 + q * NT < n ? src[it[q] & 0xFFFFu] : 0ull;
    }
#pragma unroll
    for (int q = 0; q < BBATCH; ++q) {
      if (j0 + q * NT < n) {
        const uint32_t c = (uint32_t)(r[q] >> S.sshift) & S.smask;
        const uint32_t a0 = c ? cnt.get(c - 1) : 0u, e = cnt.get(c);
        uint32_t p = a0;
        for (uint32_t k = a0; k < e; ++k) p += items[k] < it[q] ? 1u : 0u;
        const unsigned long long h = hg | (r[q] >> 32);
        if (wide) oh64[p] = h;
        else oh32[p] = (uint32_t)h;
        op[p] = (uint32_t)r[q];
      }
    }
  }
}

__device__ __forceinline__ bool is_big(uint64_t n) { return n > BCAP; }

// One CTA of UNT threads: the list of big buckets (more than BCAP records), in
// bucket order, and its length.
__global__ void __launch_bounds__(UNT) k_big_list(const unsigned long long *__restrict__ bstart,
                                                  uint32_t *__restrict__ big, uint32_t *__restrict__ nbig) {
  constexpr int PER = SEG * SEG / UNT;
  __shared__ uint32_t s_w[UNT / 32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  uint64_t mask = 0;  // bit q: bucket t * PER + q is big
  uint32_t tot = 0;
#pragma unroll 8
  for (int q = 0; q < PER; ++q) {
    const uint32_t b = t * PER + q;
    if (is_big(bstart[b + 1] - bstart[b])) {
      mask |= 1ull << q;
      ++tot;
    }
  }
  uint32_t inc = tot;
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t u = __shfl_up_sync(kFull, inc, d);
    if (lane >= d) inc += u;
  }
  if (lane == 31) s_w[warp] = inc;
  __syncthreads();
  uint32_t off = 0, all = 0;
  for (int i = 0; i < UNT / 32; ++i) {
    if (i < warp) off += s_w[i];
    all += s_w[i];
  }
  off += inc - tot;
  for (; mask; mask &= mask - 1) big[off++] = t * PER + (uint32_t)__ffsll((long long)mask) - 1;
  if (t == 0) *nbig = all;
}

// One CTA per bucket: a bucket of at most BCAP records sorted, or listed for the LSD path when a
// sub-bin is crowded; big buckets are left to k_bucket_big.
__global__ void __launch_bounds__(BNT, 2) k_bucket_sort(const unsigned long long *__restrict__ bstart,
                                                        const unsigned long long *__restrict__ X, int hash_bits,
                                                        void *sorted_hash, uint32_t *sorted_pos,
                                                        BucketLists *__restrict__ lists, PtrTable pt) {
  extern __shared__ __align__(16) uint32_t bsm[];
  uint32_t *cnt = bsm, *items = bsm + BNSUB;
  __shared__ uint32_t s_w[BNT / 32];
  const uint32_t b = blockIdx.x;
  const int t = threadIdx.x;
  const uint64_t start = bstart[b], n64 = bstart[b + 1] - start;
  if (is_big(n64)) return;
  if (n64 == 0) {  // the table entries only
    if (pt.e >= 0)
      for (uint32_t l = t; l < (1u << pt.e); l += BNT) pt.offsets[((uint64_t)b << pt.e) + l] = start;
    return;
  }
  const uint32_t n = (uint32_t)n64;
  const unsigned long long *xb = X + start;
  const SubBins S = sub_bins(hash_bits, pt, BSUB_BITS);
  if (count_scan<BNT, BNSUB, false>(xb, n, S, SubCnt<false>{cnt}, s_w)) {
    if (t == 0) lists->list[atomicAdd(&lists->n, 1u)] = b;
    return;
  }
  place_rank_write<BNT, false>(xb, n, S, SubCnt<false>{cnt}, items, start, 0, b, hash_bits, sorted_hash, sorted_pos, pt);
}

// A big bucket (more than BCAP records) by one CTA of BNT2 threads with the SM's shared memory to
// itself: the same sort with 2^BSUB_BITS2 sub-bins (a few items each), up to BCAP2 items; a larger
// one is listed for the LSD path.
__global__ void __launch_bounds__(BNT2, 1) k_bucket_big(const uint32_t *__restrict__ big,
                                                        const uint32_t *__restrict__ nbig,
                                                        const unsigned long long *__restrict__ bstart,
                                                        const unsigned long long *__restrict__ X, int hash_bits,
                                                        void *sorted_hash, uint32_t *sorted_pos,
                                                        BucketLists *__restrict__ lists, PtrTable pt) {
  extern __shared__ __align__(16) uint32_t bsm[];
  uint32_t *cnt = bsm, *items = bsm + BNSUB2;
  __shared__ uint32_t s_w[BNT2 / 32];
  if (blockIdx.x >= *nbig) return;
  const uint32_t b = big[blockIdx.x];
  const uint64_t start = bstart[b];
  const uint32_t n = (uint32_t)(bstart[b + 1] - start);
  const unsigned long long *xb = X + start;
  const SubBins S = sub_bins(hash_bits, pt, BSUB_BITS2);
  if (n > BCAP2 || count_scan<BNT2, BNSUB2, false>(xb, n, S, SubCnt<false>{cnt}, s_w)) {
    if (threadIdx.x == 0) lists->list[atomicAdd(&lists->n, 1u)] = b;
    return;
  }
  place_rank_write<BNT2, false>(xb, n, S, SubCnt<false>{cnt}, items, start, 0, b, hash_bits, sorted_hash, sorted_pos, pt);
}

// Takes the next listed bucket (0xFFFFFFFF when none is left), the same for all threads.
__device__ uint32_t next_listed(BucketLists *lists, uint32_t *s_b) {
  if (threadIdx.x == 0) {
    const uint32_t i = atomicAdd(&lists->next, 1u);
    *s_b = i < lists->n ? lists->list[i] : 0xFFFFFFFFu;
  }
  __syncthreads();
  const uint32_t b = *s_b;
  __syncthreads();
  return b;
}

// Persistent: the listed buckets (more than BCAP2 records, or crowded sub-bins: many hits of a few
// hashes), each by one CTA as a stable LSD on the remaining hash bits in global memory, 8 per
// pass, between the bucket's range of X and the same range of Y.  A pass counts the digits, then
// walks the bucket in chunks of BNT * BKPT records: each warp ranks its 32 * BKPT consecutive
// records (peer ballots, per-warp digit counters), the counters are scanned across warps, and each
// record goes to its digit's running base + the warps before + its rank.  The last pass writes
// the output.
__global__ void __launch_bounds__(BNT) k_bucket_lsd(const unsigned long long *__restrict__ bstart,
                                                    unsigned long long *X, unsigned long long *Y, int hash_bits,
                                                    void *sorted_hash, uint32_t *sorted_pos,
                                                    BucketLists *__restrict__ lists, PtrTable pt) {
  __shared__ uint32_t s_base[RBINS];           // running output base of each digit
  __shared__ uint32_t s_wc[BNT / 32][RBINS];   // per-warp counts of the chunk, then their prefixes
  __shared__ uint32_t s_b;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int rbits = hash_bits - 16;
  const int passes = (rbits + 7) / 8;
  for (;;) {
    const uint32_t b = next_listed(lists, &s_b);
    if (b == 0xFFFFFFFFu) return;
    const uint64_t start = bstart[b], n = bstart[b + 1] - start;
    const uint32_t g = b / SEG;
    const unsigned long long *src = X + start;
    unsigned long long *dst = Y + start;
    for (int p = 0; p < passes; ++p) {
      const int shift = 32 + 8 * p;
      const uint32_t dmask = (8 * (p + 1) <= rbits) ? 0xFFu : ((1u << (rbits - 8 * p)) - 1u);
      const bool last = p == passes - 1;
      for (int i = t; i < RBINS; i += BNT) s_base[i] = 0;
      __syncthreads();
      for (uint64_t i = t; i < n; i += BNT) atomicAdd(&s_base[(uint32_t)(src[i] >> shift) & dmask], 1u);
      __syncthreads();
      if (warp == 0) {  // exclusive scan of the 256 counts, 8 per lane
        uint32_t c[RBINS / 32], tot = 0;
#pragma unroll
        for (int q = 0; q < RBINS / 32; ++q) {
          c[q] = s_base[lane * (RBINS / 32) + q];
          tot += c[q];
        }
        uint32_t inc = tot;
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t u = __shfl_up_sync(kFull, inc, d);
          if (lane >= d) inc += u;
        }
        uint32_t run = inc - tot;
#pragma unroll
        for (int q = 0; q < RBINS / 32; ++q) {
          s_base[lane * (RBINS / 32) + q] = run;
          run += c[q];
        }
      }
      __syncthreads();
      for (uint64_t c0 = 0; c0 < n; c0 += (uint64_t)BNT * BKPT) {
        for (int i = t; i < (BNT / 32) * RBINS; i += BNT) (&s_wc[0][0])[i] = 0;
        __syncthreads();
        unsigned long long r[BKPT];
        uint32_t rd[BKPT];  // digit << 16 | rank within the warp's chunk (digit RBINS: no record)
#pragma unroll
        for (int j = 0; j < BKPT; ++j) {
          const uint64_t i = c0 + (uint64_t)warp * (32 * BKPT) + (uint64_t)j * 32 + lane;
          r[j] = i < n ? src[i] : 0ull;
          rd[j] = i < n ? (((uint32_t)(r[j] >> shift) & dmask) << 16) : ((uint32_t)RBINS << 16);
        }
#pragma unroll
        for (int j = 0; j < BKPT; ++j) {
          const int d = (int)(rd[j] >> 16);
          const unsigned peers = digit_peers(d, d < RBINS);
          const int leader = __ffs(peers) - 1;
          uint32_t o = 0;
          if (lane == leader && d < RBINS) {
            o = s_wc[warp][d];
            s_wc[warp][d] = o + (uint32_t)__popc(peers);
          }
          rd[j] |= __shfl_sync(kFull, o, leader) + (uint32_t)__popc(peers & lanemask_lt(lane));
          __syncwarp();
        }
        __syncthreads();
        uint32_t chunk_tot = 0;
        if (t < RBINS) {  // digit t: the warps' counts become their offsets within the chunk
          for (int wq = 0; wq < BNT / 32; ++wq) {
            const uint32_t c = s_wc[wq][t];
            s_wc[wq][t] = chunk_tot;
            chunk_tot += c;
          }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < BKPT; ++j) {
          const int d = (int)(rd[j] >> 16);
          if (d < RBINS) {
            const uint32_t o = s_base[d] + s_wc[warp][d] + (rd[j] & 0xFFFFu);
            if (last) bucket_write(r[j], start + o, g, hash_bits, sorted_hash, sorted_pos);
            else dst[o] = r[j];
          }
        }
        __syncthreads();
        if (t < RBINS) s_base[t] += chunk_tot;
        __syncthreads();
      }
      const unsigned long long *nsrc = dst;
      dst = const_cast<unsigned long long *>(src);
      src = nsrc;
    }
    __syncthreads();
    if (pt.e >= 0) bucket_offsets(b, start, (uint32_t)n, sorted_hash, hash_bits, pt);
  }
}

// The pointer table from the bucket starts when bucket_bits <= 16 (table bucket b begins where sort
// bucket b << (16 - bucket_bits) does), or only its last entry when pass C fills the rest.
__global__ void k_offsets_from_starts(const unsigned long long *__restrict__ bstart, int bucket_bits, int fused,
                                      uint64_t *__restrict__ offsets) {
  const uint64_t nb = 1ull << bucket_bits;
  const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (fused) {
    if (b == 0) offsets[nb] = bstart[SEG * SEG];
    return;
  }
  if (b <= nb) offsets[b] = b < nb ? bstart[b << (16 - bucket_bits)] : bstart[SEG * SEG];
}

// Workspace of the segmented sort, after the histograms: segment info, the tile count and the
// piece count, the listed buckets, pass B's tile descriptors, bucket starts, the pieces.
struct MsdWs {
  SegInfo *seg;
  uint32_t *total;
  uint32_t *nbig;
  BucketLists *lists;
  TileDesc *tiles;
  unsigned long long *bstart;
  uint32_t *big;
};
uint64_t msd_max_tiles(uint64_t m) { return (m + RTILE - 1) / RTILE + SEG; }
uint64_t msd_max_big(uint64_t m) { return m / BCAP < (uint64_t)SEG * SEG ? m / BCAP + 1 : (uint64_t)SEG * SEG; }
constexpr uint64_t kListsBytes = (sizeof(BucketLists) + 255) / 256 * 256;
constexpr uint64_t kStartsBytes = ((uint64_t)SEG * SEG + 1) * 8 + 248;
MsdWs msd_layout(void *base, uint64_t m) {
  char *p = static_cast<char *>(base);
  MsdWs w;
  w.seg = reinterpret_cast<SegInfo *>(p);
  p += SEG * sizeof(SegInfo);
  w.total = reinterpret_cast<uint32_t *>(p);
  w.nbig = w.total + 1;
  p += 256;
  w.lists = reinterpret_cast<BucketLists *>(p);
  p += kListsBytes;
  w.tiles = reinterpret_cast<TileDesc *>(p);
  p += msd_max_tiles(m) * sizeof(TileDesc);
  w.bstart = reinterpret_cast<unsigned long long *>(p);
  p += kStartsBytes;
  w.big = reinterpret_cast<uint32_t *>(p);
  return w;
}

bool msd_applies(uint64_t m, int hash_bits) {
  // 16 < hash_bits <= 40 (a record holds hash_bits - 8 hash bits), and inputs large enough to
  // fill the buckets; m < 2^32 holds for every table
  return hash_bits > 16 && hash_bits <= 40 && m >= (1u << 16);
}

// Pass C fills the pointer table itself for 20 <= bucket_bits <= 26 (16 to 1024 entries a sort
// bucket, so that pieces can begin at table-bucket boundaries); bucket_bits <= 16 takes it from the
// bucket starts; the other sizes take the general fill.
bool msd_fills_offsets(int bucket_bits) { return bucket_bits >= 20 && bucket_bits <= 26; }
bool msd_done_offsets(int bucket_bits) { return bucket_bits <= 16 || msd_fills_offsets(bucket_bits); }

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

template <bool WIDE>
cudaError_t msd_sort_t(const TableArgs &a, cudaStream_t st) {
  const uint64_t m = a.m;
  const int H = a.hash_bits;
  const uint32_t ntA = (uint32_t)((m + RTILE - 1) / RTILE);
  const uint32_t maxB = (uint32_t)msd_max_tiles(m);
  const MsdWs w = msd_layout(a.ws_msd, m);
  const size_t smW = (size_t)RTILE * (8 + (WIDE ? 8 : 0)) + (size_t)RWARPS * RBINS * 4;
  const size_t smN = (size_t)RTILE * 8 + (size_t)RWARPS * RBINS * 4;
  cudaError_t e = cudaSuccess;
  static bool attr = false;
  if (!attr) {
    for (auto f : {(const void *)k_radix_scatter<true>, (const void *)k_radix_scatter<false>})
      if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smW);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_bucket_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BSMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_bucket_big, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BSMEM2);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  // A: top 8 hash bits, hits packed into records
  PassIn inA{};
  inA.hash32 = static_cast<const uint32_t *>(a.hash);
  inA.hash64 = static_cast<const unsigned long long *>(a.hash);
  inA.pos = a.pos;
  PassOut outA{};
  outA.keys = a.ws_keys[0];
  outA.pack = 1;
  outA.pack_mask = (1ull << (H - 8)) - 1ull;
  const int shiftA = WIDE ? H - 8 : 32 + H - 8;
  k_radix_hist<WIDE><<<ntA, RNT, 0, st>>>(inA, m, shiftA, a.ws_hist, ntA, nullptr);
  e = scan_u32(a.ws_hist, (uint64_t)RBINS * ntA, a.ws_bsum, st);
  if (e != cudaSuccess) return e;
  k_radix_scatter<WIDE><<<ntA, RNT, smW, st>>>(inA, outA, m, shiftA, a.ws_hist, ntA, nullptr);
  // B: the next 8 bits within each segment
  k_seg_info<<<1, SEG, 0, st>>>(a.ws_hist, ntA, m, w.seg, w.total);
  k_tile_desc<<<(maxB + 255) / 256, 256, 0, st>>>(w.seg, w.total, maxB, w.tiles);
  PassIn inB{};
  inB.keys = a.ws_keys[0];
  PassOut outB{};
  outB.keys = a.ws_keys[1];
  const int shiftB = 32 + H - 16;
  k_radix_hist<false><<<maxB, RNT, 0, st>>>(inB, m, shiftB, a.ws_hist, 0, w.tiles);
  e = scan_u32(a.ws_hist, (uint64_t)RBINS * maxB, a.ws_bsum, st);
  if (e != cudaSuccess) return e;
  k_radix_scatter<false><<<maxB, RNT, smN, st>>>(inB, outB, m, shiftB, a.ws_hist, 0, w.tiles);
  // C: every bucket on its own, large ones in pieces; the rest by the LSD path
  k_bucket_starts<<<(SEG * SEG + 1 + 255) / 256, 256, 0, st>>>(w.seg, a.ws_hist, m, w.bstart);
  k_big_list<<<1, UNT, 0, st>>>(w.bstart, w.big, w.nbig);
  e = cudaMemsetAsync(w.lists, 0, 2 * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  const PtrTable pt{a.offsets, msd_fills_offsets(a.bucket_bits) ? a.bucket_bits - 16 : -1};
  k_bucket_sort<<<SEG * SEG, BNT, BSMEM, st>>>(w.bstart, a.ws_keys[1], H, a.sorted_hash, a.sorted_pos, w.lists,
                                               pt);
  k_bucket_big<<<(unsigned)msd_max_big(m), BNT2, BSMEM2, st>>>(w.big, w.nbig, w.bstart, a.ws_keys[1], H,
                                                               a.sorted_hash, a.sorted_pos, w.lists, pt);
  k_bucket_lsd<<<2 * sm_count(), BNT, 0, st>>>(w.bstart, a.ws_keys[1], a.ws_keys[0], H, a.sorted_hash,
                                               a.sorted_pos, w.lists, pt);
  if (msd_done_offsets(a.bucket_bits)) {
    const uint64_t nb = a.bucket_bits <= 16 ? (1ull << a.bucket_bits) + 1 : 1;
    k_offsets_from_starts<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(w.bstart, a.bucket_bits, pt.e >= 0,
                                                                         a.offsets);
  }
  return cudaGetLastError();
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
uint64_t table_hist_words(uint64_t m) { return (uint64_t)RBINS * ((m + RTILE - 1) / RTILE + SEG); }
uint64_t table_msd_bytes(uint64_t m) {
  return SEG * sizeof(SegInfo) + 256 + kListsBytes + msd_max_tiles(m) * sizeof(TileDesc) + kStartsBytes +
         (uint64_t)SEG * SEG * 4;
}
uint64_t table_bsum_words(uint64_t m) { return (table_hist_words(m) + SCAN_BLOCK - 1) / SCAN_BLOCK + 1; }
uint64_t table_gap_bytes(int bucket_bits) { return table_gap_capacity(bucket_bits) * sizeof(Gap); }

cudaError_t launch_table(const TableArgs &a, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (a.m > 0) {
    if (a.ws_msd && msd_applies(a.m, a.hash_bits)) {
      e = a.hash_bits > 32 ? msd_sort_t<true>(a, st) : msd_sort_t<false>(a, st);
      if (e != cudaSuccess || msd_done_offsets(a.bucket_bits)) return e;
    } else {
      e = a.hash_bits > 32 ? sort_t<true>(a, st) : sort_t<false>(a, st);
    }
    if (e != cudaSuccess) return e;
  }
  return a.hash_bits > 32 ? offsets_t<true>(a, st) : offsets_t<false>(a, st);
}

}  // namespace sws
