// strand.cu -- the strand of each minimizer pick (Sec. 2.4 over canonical k-mers, which pick
// min(forward, reverse complement)): 0 when the forward k-mer at the pick is the smaller or the
// two are equal (a palindrome), 1 when the reverse complement is the smaller.  One thread per
// pick reads the pick's k bases from the 2-bit packed stream (at most nine bytes), rebuilds the
// forward and reverse-complement values and compares them.  Picks of a read batch carry
// read-local positions: the thread finds its read by a binary search in the pick offsets.
#include <cstdint>

#include "../../include/sws.h"
#include "common.cuh"
#include "internal.h"
#include "mini_common.cuh"

namespace sws {
namespace {

__global__ void __launch_bounds__(256) k_strands(const uint8_t *__restrict__ seq, uint64_t n, int k,
                                                 const int64_t *__restrict__ base_offsets,
                                                 const uint64_t *__restrict__ pick_offsets, uint64_t nreads,
                                                 const uint32_t *__restrict__ pos, uint64_t m,
                                                 uint8_t *__restrict__ strand) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  uint64_t base = pos[i];
  if (base_offsets) {
    uint64_t lo = 0, hi = nreads;  // the read r with pick_offsets[r] <= i < pick_offsets[r+1]
    while (hi - lo > 1) {
      const uint64_t mid = (lo + hi) / 2;
      if (pick_offsets[mid] <= i) lo = mid;
      else hi = mid;
    }
    base += (uint64_t)base_offsets[lo];
  }
  if (base + (uint64_t)k > n) {
    strand[i] = 255;
    return;
  }
  // bases base .. base+k-1, base j of the window at bits 2j (the packing's order)
  const uint64_t b0 = base >> 2;
  const uint64_t last = (base + (uint64_t)k - 1) >> 2;
  unsigned long long lo64 = 0, hi64 = 0;  // up to 9 bytes: 72 bits
  for (uint64_t b = b0; b <= last; ++b) {
    const unsigned long long v = seq[b];
    const int sh = (int)(b - b0) * 8;
    if (sh < 64) lo64 |= v << sh;
    else hi64 |= v << (sh - 64);
  }
  const int off = (int)(base & 3) * 2;
  const unsigned long long x = off ? ((lo64 >> off) | (hi64 << (64 - off))) : lo64;
  const unsigned long long kmask = 2 * k == 64 ? ~0ull : ((1ull << (2 * k)) - 1ull);
  const mini::Kmer64 q = mini::kmer64(x, k, kmask);
  strand[i] = q.rc < q.fwd ? 1 : 0;
}

}  // namespace

cudaError_t launch_strands(const uint8_t *seq, uint64_t n, int k, const int64_t *base_offsets,
                           const uint64_t *pick_offsets, uint64_t nreads, const uint32_t *pos, uint64_t m,
                           uint8_t *strand, cudaStream_t st) {
  if (m == 0) return cudaSuccess;
  const uint64_t blocks = (m + 255) / 256;
  if (blocks > 0x7fffffffull) return cudaErrorInvalidValue;
  k_strands<<<(unsigned)blocks, 256, 0, st>>>(seq, n, k, base_offsets, pick_offsets, nreads, pos, m, strand);
  return cudaGetLastError();
}

}  // namespace sws
