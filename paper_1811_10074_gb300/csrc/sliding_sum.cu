// sliding_sum.cu -- streaming kernels for the sliding window sum of Eq. 2 (Sec. 2.2):
//     y_p = x_p (+) x_{p+1} (+) ... (+) x_{p+w-1},  p = 0 .. n-w.
//
// Every kernel works on independent CTA tiles: a tile owns TO consecutive outputs and reads
// the TO + w - 1 inputs they need (the w-1 halo is re-read by the next tile, normally from L2).
// Inputs go straight from HBM into registers with 16-byte loads, outputs leave with 16-byte
// streaming stores, so HBM sees ~4+4 bytes per int32 element.  Three schemes:
//
//   block-combine  in-block suffix (+) next-block prefix (common.cuh), O(1) (+) per output, any
//                  associative operator.  The restatement of Alg. 2 (Sec. 3.1) for a CTA.
//   doubling       windows of 2^s built in ceil(log2 w) levels in shared memory, O(log w) per
//                  output (Sec. 2.2 / Sec. 3.1: prefix scans inside each window).  Idempotent
//                  operators finish with two overlapping 2^t windows; the others combine the
//                  binary digits of w in order, which needs associativity only.
//   block-combine, streamed   the same arithmetic for w a multiple of the thread chunk, in a
//                  persistent kernel whose tiles arrive in shared memory by 2-D TMA copies
//                  issued ahead of the compute (k_slide_tma).
//   prefix-diff    for invertible operators (add mod 2^32, xor): y_p = T_{p+w-1} (-) T_{p-1},
//                  with T the running sum from the tile start (the "recurrent" sliding sums of
//                  Sec. 5), O(1) per output and independent of w.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <mutex>

#include "../../include/sws.h"
#include "common.cuh"
#include "internal.h"
#include "tma.cuh"

namespace sws {

namespace {

template <int NT_, int VPT4_, int VPT8_>
struct CfgShape {
  static constexpr int NT = NT_;
  static constexpr int VPT4 = VPT4_;
  static constexpr int VPT8 = VPT8_;
};
using CfgSmall = CfgShape<256, 16, 8>;
using CfgLarge = CfgShape<512, 16, 8>;

template <class T>
__device__ __forceinline__ bool aligned16(const T *p) {
  return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

// Load this thread's VPT elements of the tile starting at global index g (identity past n).
template <class Op, int VPT>
__device__ __forceinline__ void load_tile(const typename Op::T *__restrict__ in, uint64_t n, uint64_t g, bool vec,
                                          typename Op::T (&x)[VPT]) {
  if (vec && g + VPT <= n) {
    load_vec<typename Op::T, VPT>(in + g, x);
  } else {
#pragma unroll
    for (int j = 0; j < VPT; ++j) x[j] = (g + j < n) ? in[g + j] : Op::identity();
  }
}

template <class Op, int VPT>
__device__ __forceinline__ void store_tile(typename Op::T *__restrict__ out, uint64_t nout, uint64_t g, int o, int TO,
                                           bool vec, const typename Op::T (&y)[VPT]) {
  if (vec && o + VPT <= TO && g + VPT <= nout) {
    store_vec<typename Op::T, VPT>(out + g, y);
  } else {
#pragma unroll
    for (int j = 0; j < VPT; ++j)
      if (o + j < TO && g + j < nout) out[g + j] = y[j];
  }
}

// ------------------------------------------------------------------------------------------
// Block-combine
// ------------------------------------------------------------------------------------------
template <class Op, int NT, int VPT>
__global__ void __launch_bounds__(NT) k_slide_bc(const typename Op::T *__restrict__ in, typename Op::T *__restrict__ out,
                                                 uint64_t n, int w, int TO) {
  using BC = BlockCombine<Op, NT, VPT>;
  using T = typename Op::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  typename BC::Shared &sh = *reinterpret_cast<typename BC::Shared *>(smem_raw);
  __shared__ int s_r0;

  const uint64_t t0 = (uint64_t)blockIdx.x * (uint64_t)TO;
  const int o = threadIdx.x * VPT;
  const uint64_t g = t0 + (uint64_t)o;
  const bool vec = aligned16(in) && aligned16(out);
  T x[VPT];
  load_tile<Op, VPT>(in, n, g, vec, x);
  if (threadIdx.x == 0) s_r0 = (int)(t0 % (uint64_t)w);
  __syncthreads();
  const int r0 = (int)(((unsigned)s_r0 + (unsigned)o) % (unsigned)w);
  T y[VPT];
  BC::run(sh, x, r0, w, y);
  store_tile<Op, VPT>(out, n - (uint64_t)w + 1, g, o, TO, vec, y);
}

// ------------------------------------------------------------------------------------------
// Block-combine, w a multiple of VPT: blocks are whole thread chunks
// ------------------------------------------------------------------------------------------
// A tile starts at a multiple of w, so block b of the tile is exactly the G = w / VPT threads
// bG .. bG+G-1.  In-thread prefix and suffix sums then need no segmentation, the carries are
// scans over groups of G lanes (lane-aligned when G divides 32; whole warps when G is a
// multiple of 32), and the shifted read P_{p+w-1} is row t+G of the prefix array, element j-1
// -- a 16-byte-vector read from a padded row layout that is bank-conflict free.
template <class Op, int NT, int VPT>
__global__ void __launch_bounds__(NT) k_slide_al(const typename Op::T *__restrict__ in,
                                                 typename Op::T *__restrict__ out, uint64_t n, int w, int TO) {
  using T = typename Op::T;
  constexpr int NW = NT / 32;
  constexpr int EPV = 16 / (int)sizeof(T);  // elements per 16-byte unit
  constexpr int UPR = VPT / EPV;            // 16-byte units per thread row
  constexpr int ROW = UPR + 1;              // padded row (units)
  static_assert(VPT % EPV == 0, "rows must be whole 16-byte units");
  extern __shared__ __align__(16) uint4 sm4[];
  __shared__ T s_wf[NW], s_wb[NW];

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int G = w / VPT;
  const uint64_t t0 = (uint64_t)blockIdx.x * (uint64_t)TO;
  const uint64_t g = t0 + (uint64_t)t * VPT;
  const bool vec = aligned16(in) && aligned16(out);
  T x[VPT];
  load_tile<Op, VPT>(in, n, g, vec, x);
  T P[VPT], S[VPT];
  P[0] = x[0];
#pragma unroll
  for (int j = 1; j < VPT; ++j) P[j] = Op::op(P[j - 1], x[j]);
  S[VPT - 1] = x[VPT - 1];
#pragma unroll
  for (int j = VPT - 2; j >= 0; --j) S[j] = Op::op(x[j], S[j + 1]);

  const int pos = t % G;  // position of this thread inside its block
  const bool head = pos == 0, tail = pos == G - 1;
  T cP = P[VPT - 1], cS = S[0];
  if (G <= 32) {
    // segments of G lanes, aligned to lane multiples of G
    const int base = lane - pos;
    T vf = P[VPT - 1], vb = S[0];
    for (int d = 1; d < G; d <<= 1) {
      const T u = shfl_up_t(vf, d);
      const T v = shfl_down_t(vb, d);
      if (pos >= d) vf = Op::op(u, vf);
      if (pos + d < G) vb = Op::op(vb, v);
    }
    const T ef = shfl_up_t(vf, 1);
    const T eb = shfl_down_t(vb, 1);
    (void)base;
    cP = ef;
    cS = eb;
  } else {
    // blocks are m = G/32 whole warps: plain warp scans plus carries across the block's warps
    const int m = G >> 5, wp = warp % m;
    T vf = warp_seg_scan_fwd<Op>(P[VPT - 1], 0u, lane);
    T vb = warp_seg_scan_bwd<Op>(S[0], 0u, lane);
    if (lane == 31) s_wf[warp] = vf;
    if (lane == 0) s_wb[warp] = vb;
    __syncthreads();
    const T ef = shfl_up_t(vf, 1);
    const T eb = shfl_down_t(vb, 1);
    T cwf = Op::identity(), cwb = Op::identity();
    for (int i = warp - wp; i < warp; ++i) cwf = (i == warp - wp) ? s_wf[i] : Op::op(cwf, s_wf[i]);
    for (int i = warp - wp + m - 1; i > warp; --i) cwb = (i == warp - wp + m - 1) ? s_wb[i] : Op::op(s_wb[i], cwb);
    if (lane == 0) cP = cwf;
    else cP = wp > 0 ? Op::op(cwf, ef) : ef;
    if (lane == 31) cS = cwb;
    else cS = wp < m - 1 ? Op::op(eb, cwb) : eb;
  }
  if (!head) {
#pragma unroll
    for (int j = 0; j < VPT; ++j) P[j] = Op::op(cP, P[j]);
  }
  if (!tail) {
#pragma unroll
    for (int j = 0; j < VPT; ++j) S[j] = Op::op(S[j], cS);
  }
  {
    uint4 u[UPR];
    memcpy(u, P, sizeof(u));
#pragma unroll
    for (int c = 0; c < UPR; ++c) sm4[t * ROW + c] = u[c];
  }
  __syncthreads();
  T y[VPT];
  int tn = t + G;
  if (tn > NT - 1) tn = NT - 1;  // only threads whose outputs lie past TO get here
  {
    uint4 u[UPR];
#pragma unroll
    for (int c = 0; c < UPR; ++c) u[c] = sm4[tn * ROW + c];
    T Pn[VPT];
    memcpy(Pn, u, sizeof(u));
    const T *prow = reinterpret_cast<const T *>(sm4 + (tn - 1) * ROW);
    const T plast = prow[VPT - 1];
    y[0] = head ? S[0] : Op::op(S[0], plast);
#pragma unroll
    for (int j = 1; j < VPT; ++j) y[j] = Op::op(S[j], Pn[j - 1]);
  }
  store_tile<Op, VPT>(out, n - (uint64_t)w + 1, g, t * VPT, TO, vec, y);
}

// ------------------------------------------------------------------------------------------
// Block-combine, w a multiple of VPT, persistent, input staged by TMA
// ------------------------------------------------------------------------------------------
// The arithmetic of k_slide_al, fed differently.  A grid of a few CTAs per SM walks the tiles
// round-robin; tile i's L inputs arrive in shared memory by one 2-D TMA copy (the array viewed
// as rows of 128 bytes) issued STAGES tiles ahead on an mbarrier, so HBM sees a steady stream of
// bulk reads while the threads scan.  The copy uses the 128-byte swizzle: 16-byte unit u of row
// r lands at unit u ^ (r & 7), so the four units of thread t's 64-byte chunk (row t/2, units
// 4(t&1) .. 4(t&1)+3) fall in eight distinct bank groups across every quarter-warp and the
// reads are conflict free.  Tiles start at multiples of lcm(w, 128 bytes): whole blocks and
// whole rows.  Elements of a final partial row are not in the tensor map (the copy fills them
// with zeros); the threads that own them load them directly.  Every wait is bounded; on a
// time-out the CTA flags DEVERR_COPY_TIMEOUT, lets its own copies land (bounded) and returns.
constexpr int kStreamRowBytes = 128;

__device__ __forceinline__ bool stream_wait(unsigned long long *bar, uint32_t parity) {
  return tma::mbar_wait_bounded(bar, parity);
}

template <class Op, int NT, int VPT, int STAGES, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_slide_tma(const __grid_constant__ CUtensorMap tmap, const typename Op::T *__restrict__ in,
                typename Op::T *__restrict__ out, uint64_t n, uint64_t n_full, int w, int TO, uint64_t tiles,
                int *err) {
  using T = typename Op::T;
  constexpr int NW = NT / 32;
  constexpr int EPV = 16 / (int)sizeof(T);
  constexpr int UPR = VPT / EPV;  // 16-byte units per thread chunk
  constexpr int ROW = UPR + 1;    // padded row of the shared prefix array
  constexpr int TILE_BYTES = NT * VPT * (int)sizeof(T);
  static_assert(VPT * (int)sizeof(T) * 2 == kStreamRowBytes, "a thread chunk is half a 128-byte row");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long full[STAGES];
  __shared__ T s_wf[NW], s_wb[NW];

  unsigned char *stage0 = smem_raw + ((1024u - (tma::smem_u32(smem_raw) & 1023u)) & 1023u);
  uint4 *sm4 = reinterpret_cast<uint4 *>(stage0 + STAGES * TILE_BYTES);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int G = w / VPT;
  const uint64_t rows_per_tile = (uint64_t)TO * sizeof(T) / kStreamRowBytes;
  const uint64_t stride = gridDim.x;

  if (t == 0) {
    tma::prefetch_tensormap(&tmap);
#pragma unroll
    for (int s = 0; s < STAGES; ++s) tma::mbar_init(&full[s], 1);
    tma::fence_mbar_init();
  }
  __syncthreads();
  if (t == 0) {
#pragma unroll
    for (int s = 0; s < STAGES; ++s) {
      const uint64_t tile = blockIdx.x + (uint64_t)s * stride;
      if (tile < tiles) {
        tma::mbar_arrive_expect_tx(&full[s], TILE_BYTES);
        tma::tensor_g2s_2d(stage0 + s * TILE_BYTES, &tmap, 0, (int)(tile * rows_per_tile), &full[s]);
      }
    }
  }
  const bool vec = aligned16(out);
  const uint64_t nout = n - (uint64_t)w + 1;
  int it = 0;
  for (uint64_t tile = blockIdx.x; tile < tiles; tile += stride, ++it) {
    const int s = it % STAGES;
    const bool ok = stream_wait(&full[s], (uint32_t)(it / STAGES) & 1u);
    T x[VPT];
    if (ok) {
      const unsigned char *src = stage0 + s * TILE_BYTES + (t >> 1) * kStreamRowBytes;
      const int sw = (t >> 1) & 7;
      uint4 u[UPR];
#pragma unroll
      for (int c = 0; c < UPR; ++c) u[c] = *reinterpret_cast<const uint4 *>(src + ((((t & 1) * UPR + c) ^ sw) << 4));
      memcpy(x, u, sizeof(u));
    }
    if (!__syncthreads_and(ok)) {
      if (t == 0) {
        atomicOr(err, DEVERR_COPY_TIMEOUT);
        // let every copy this CTA still has in flight land before it exits (bounded)
        for (int j = 0; j < STAGES; ++j) {
          const uint64_t tj = tile + (uint64_t)j * stride;
          if (tj < tiles) stream_wait(&full[(it + j) % STAGES], (uint32_t)((it + j) / STAGES) & 1u);
        }
      }
      return;
    }
    if (t == 0) {
      const uint64_t nt = tile + (uint64_t)STAGES * stride;
      if (nt < tiles) {
        tma::fence_proxy_async_smem();
        tma::mbar_arrive_expect_tx(&full[s], TILE_BYTES);
        tma::tensor_g2s_2d(stage0 + s * TILE_BYTES, &tmap, 0, (int)(nt * rows_per_tile), &full[s]);
      }
    }
    const uint64_t g = tile * (uint64_t)TO + (uint64_t)t * VPT;
    if (g + VPT > n_full) {
#pragma unroll
      for (int j = 0; j < VPT; ++j)
        if (g + j >= n_full) x[j] = (g + j < n) ? in[g + j] : Op::identity();
    }

    T P[VPT], S[VPT];
    P[0] = x[0];
#pragma unroll
    for (int j = 1; j < VPT; ++j) P[j] = Op::op(P[j - 1], x[j]);
    S[VPT - 1] = x[VPT - 1];
#pragma unroll
    for (int j = VPT - 2; j >= 0; --j) S[j] = Op::op(x[j], S[j + 1]);

    const int pos = t % G;
    const bool head = pos == 0, tail = pos == G - 1;
    T cP, cS;
    if (G <= 32) {
      T vf = P[VPT - 1], vb = S[0];
      for (int d = 1; d < G; d <<= 1) {
        const T a = shfl_up_t(vf, d);
        const T b = shfl_down_t(vb, d);
        if (pos >= d) vf = Op::op(a, vf);
        if (pos + d < G) vb = Op::op(vb, b);
      }
      cP = shfl_up_t(vf, 1);
      cS = shfl_down_t(vb, 1);
    } else {
      const int m = G >> 5, wp = warp % m;
      const T vf = warp_seg_scan_fwd<Op>(P[VPT - 1], 0u, lane);
      const T vb = warp_seg_scan_bwd<Op>(S[0], 0u, lane);
      if (lane == 31) s_wf[warp] = vf;
      if (lane == 0) s_wb[warp] = vb;
      __syncthreads();
      const T ef = shfl_up_t(vf, 1);
      const T eb = shfl_down_t(vb, 1);
      T cwf = Op::identity(), cwb = Op::identity();
      for (int i = warp - wp; i < warp; ++i) cwf = (i == warp - wp) ? s_wf[i] : Op::op(cwf, s_wf[i]);
      for (int i = warp - wp + m - 1; i > warp; --i) cwb = (i == warp - wp + m - 1) ? s_wb[i] : Op::op(s_wb[i], cwb);
      cP = lane == 0 ? cwf : (wp > 0 ? Op::op(cwf, ef) : ef);
      cS = lane == 31 ? cwb : (wp < m - 1 ? Op::op(eb, cwb) : eb);
    }
    if (!head) {
#pragma unroll
      for (int j = 0; j < VPT; ++j) P[j] = Op::op(cP, P[j]);
    }
    if (!tail) {
#pragma unroll
      for (int j = 0; j < VPT; ++j) S[j] = Op::op(S[j], cS);
    }
    {
      uint4 u[UPR];
      memcpy(u, P, sizeof(u));
#pragma unroll
      for (int c = 0; c < UPR; ++c) sm4[t * ROW + c] = u[c];
    }
    __syncthreads();
    T y[VPT];
    {
      const int tn = t + G < NT ? t + G : NT - 1;  // past the tile only for outputs beyond TO
      uint4 u[UPR];
#pragma unroll
      for (int c = 0; c < UPR; ++c) u[c] = sm4[tn * ROW + c];
      T Pn[VPT];
      memcpy(Pn, u, sizeof(u));
      const T plast = reinterpret_cast<const T *>(sm4 + (tn - 1) * ROW)[VPT - 1];
      y[0] = head ? S[0] : Op::op(S[0], plast);
#pragma unroll
      for (int j = 1; j < VPT; ++j) y[j] = Op::op(S[j], Pn[j - 1]);
    }
    store_tile<Op, VPT>(out, nout, g, t * VPT, TO, vec, y);
  }
}

// ------------------------------------------------------------------------------------------
// Block-combine, w = VPT * G with G a power of two <= 32: warp-private streaming (no barriers)
// ------------------------------------------------------------------------------------------
// Each warp owns a contiguous run of warp-tiles (32 lanes x VPT elements, 2 KB) and walks it in
// order; its own ring of shared-memory stages is filled by 2-D TMA copies (128-byte swizzle, so
// the lane reads are conflict free) that one lane issues ahead, on the warp's own mbarriers.
// Blocks of w are G lanes, aligned in the warp.  Lane l needs the prefix sums of the lane G
// later: one shuffle per element.  For lanes l < 32 - G that lane is in the same warp-tile; for
// the others it wraps to the first block of the next warp-tile, so those lanes keep their suffix
// sums for one iteration and emit the previous warp-tile's outputs with the next one's prefixes.
// No CTA barrier, no shared-memory exchange, and no halo: each input is read once (plus one
// warp-tile at the end of each warp's run).  Bounded waits as in k_slide_tma.
template <class Op, int VPT, int NWARP, int SW, int NSTAGE>
__global__ void __launch_bounds__(NWARP * 32)
    k_slide_warp(const __grid_constant__ CUtensorMap tmap, const typename Op::T *__restrict__ in,
                 typename Op::T *__restrict__ out, uint64_t n, uint64_t n_full, int w, uint64_t nwt,
                 uint64_t per_warp, int *err) {
  using T = typename Op::T;
  constexpr int EPV = 16 / (int)sizeof(T);
  constexpr int UPR = VPT / EPV;                     // 16-byte units per lane chunk
  constexpr int WT = 32 * VPT;                       // elements per warp-tile
  constexpr int WT_BYTES = WT * (int)sizeof(T);      // 2 KB
  constexpr int STAGE_BYTES = SW * WT_BYTES;
  static_assert(VPT * (int)sizeof(T) * 2 == kStreamRowBytes, "a lane chunk is half a 128-byte row");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bars[NWARP][NSTAGE];

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char *ring = smem_raw + ((1024u - (tma::smem_u32(smem_raw) & 1023u)) & 1023u) +
                        (size_t)warp * NSTAGE * STAGE_BYTES;
  const int G = w / VPT;
  const int pos = lane & (G - 1);
  const bool head = pos == 0, tail = pos == G - 1, late = lane >= 32 - G;
  const uint64_t gw = (uint64_t)blockIdx.x * NWARP + warp;
  const uint64_t k0 = gw * per_warp;
  if (lane == 0) {
    for (int s = 0; s < NSTAGE; ++s) tma::mbar_init(&bars[warp][s], 1);
    tma::fence_mbar_init();
  }
  __syncwarp();
  if (k0 >= nwt) return;
  const uint64_t k1 = k0 + per_warp < nwt ? k0 + per_warp : nwt;  // this warp's outputs: warp-tiles [k0, k1)
  const uint64_t kend = k1 < nwt ? k1 + 1 : k1;                    // plus the next one's prefixes
  const uint64_t nstages = (kend - k0 + SW - 1) / SW;
  auto issue = [&](uint64_t st) {  // lane 0: stage st of this warp's run into its ring slot
    unsigned long long *bar = &bars[warp][st % NSTAGE];
    tma::mbar_arrive_expect_tx(bar, STAGE_BYTES);
    tma::tensor_g2s_2d(ring + (st % NSTAGE) * STAGE_BYTES, &tmap, 0, (int)((k0 + st * SW) * (WT_BYTES / kStreamRowBytes)),
                       bar);
  };
  if (lane == 0) {
    tma::prefetch_tensormap(&tmap);
    for (uint64_t st = 0; st < (uint64_t)NSTAGE && st < nstages; ++st) issue(st);
  }
  const bool vec = aligned16(out);
  const uint64_t nout = n - (uint64_t)w + 1;
  T Sprev[VPT];
#pragma unroll
  for (int j = 0; j < VPT; ++j) Sprev[j] = Op::identity();
  for (uint64_t kk = k0; kk < kend; ++kk) {
    const uint64_t st = (kk - k0) / SW;
    const int sub = (int)((kk - k0) % SW);
    const int slot = (int)(st % NSTAGE);
    if (sub == 0) {
      const bool ok = stream_wait(&bars[warp][slot], (uint32_t)(st / NSTAGE) & 1u);
      if (!__all_sync(kFull, ok)) {
        if (lane == 0) {
          atomicOr(err, DEVERR_COPY_TIMEOUT);
          for (uint64_t s2 = st; s2 < st + NSTAGE && s2 < nstages; ++s2)
            stream_wait(&bars[warp][s2 % NSTAGE], (uint32_t)(s2 / NSTAGE) & 1u);
        }
        return;
      }
    }
    // this lane's VPT elements: row sub*16 + lane/2 of the stage, units 4(lane&1) .. +3, swizzled
    T x[VPT];
    {
      const int row = sub * (WT_BYTES / kStreamRowBytes) + (lane >> 1);
      const unsigned char *src = ring + slot * STAGE_BYTES + row * kStreamRowBytes;
      uint4 u[UPR];
#pragma unroll
      for (int c = 0; c < UPR; ++c) u[c] = *reinterpret_cast<const uint4 *>(src + ((((lane & 1) * UPR + c) ^ (row & 7)) << 4));
      memcpy(x, u, sizeof(u));
    }
    const uint64_t g = kk * (uint64_t)WT + (uint64_t)lane * VPT;
    if (g + VPT > n_full) {
#pragma unroll
      for (int j = 0; j < VPT; ++j)
        if (g + j >= n_full) x[j] = (g + j < n) ? in[g + j] : Op::identity();
    }
    if (sub == SW - 1 || kk + 1 == kend) {  // the stage is consumed: refill its slot
      __syncwarp();
      if (lane == 0 && st + NSTAGE < nstages) {
        tma::fence_proxy_async_smem();
        issue(st + NSTAGE);
      }
    }
    T P[VPT], S[VPT];
    P[0] = x[0];
#pragma unroll
    for (int j = 1; j < VPT; ++j) P[j] = Op::op(P[j - 1], x[j]);
    S[VPT - 1] = x[VPT - 1];
#pragma unroll
    for (int j = VPT - 2; j >= 0; --j) S[j] = Op::op(x[j], S[j + 1]);
    {
      T vf = P[VPT - 1], vb = S[0];
      for (int d = 1; d < G; d <<= 1) {
        const T a = shfl_up_t(vf, d);
        const T b = shfl_down_t(vb, d);
        if (pos >= d) vf = Op::op(a, vf);
        if (pos + d < G) vb = Op::op(vb, b);
      }
      const T cP = shfl_up_t(vf, 1);
      const T cS = shfl_down_t(vb, 1);
      if (!head) {
#pragma unroll
        for (int j = 0; j < VPT; ++j) P[j] = Op::op(cP, P[j]);
      }
      if (!tail) {
#pragma unroll
        for (int j = 0; j < VPT; ++j) S[j] = Op::op(S[j], cS);
      }
    }
    // outputs: this warp-tile's (early lanes) or the previous one's (late lanes)
    const int src_lane = (lane + G) & 31;
    const T plast = shfl_idx_t(P[VPT - 1], (lane + G - 1) & 31);
    T y[VPT];
    y[0] = head ? (late ? Sprev[0] : S[0]) : Op::op(late ? Sprev[0] : S[0], plast);
#pragma unroll
    for (int j = 1; j < VPT; ++j) y[j] = Op::op(late ? Sprev[j] : S[j], shfl_idx_t(P[j - 1], src_lane));
    const bool mine = late ? (kk > k0) : (kk < k1);
    if (mine) {
      const uint64_t go = late ? g - (uint64_t)WT : g;
      store_tile<Op, VPT>(out, nout, go, 0, 0x7fffffff, vec, y);
    }
#pragma unroll
    for (int j = 0; j < VPT; ++j) Sprev[j] = S[j];
  }
}

// ------------------------------------------------------------------------------------------
// Block-combine, w = 32 * M * VPT (blocks of M whole warp-tiles): warp-private streaming
// ------------------------------------------------------------------------------------------
// Each warp walks its run of blocks with each block one stage of its shared-memory ring (2-D TMA,
// 128-byte swizzle).  Outputs of block b need block b's suffix sums and block b+1's prefix sums
// at the same offset, which belong to the same lane: the warp keeps blocks b and b+1 resident and,
// warp-tile by warp-tile, scans b+1 forward (carrying the running total of its earlier warp-
// tiles) and b backward (carrying the totals of its later warp-tiles, known from when b was the
// next block), combining as it goes.  No CTA barrier, no halo: each input is read from HBM once.
template <class Op, int VPT, int M, int NWARP, int NSTAGE>
__global__ void __launch_bounds__(NWARP * 32)
    k_slide_wblk(const __grid_constant__ CUtensorMap tmap, const typename Op::T *__restrict__ in,
                 typename Op::T *__restrict__ out, uint64_t n, uint64_t n_full, uint64_t nob, uint64_t per_warp,
                 int *err) {
  using T = typename Op::T;
  constexpr int EPV = 16 / (int)sizeof(T);
  constexpr int UPR = VPT / EPV;
  constexpr int WT = 32 * VPT;
  constexpr int WT_BYTES = WT * (int)sizeof(T);
  constexpr int BLK = M * WT;                  // w
  constexpr int STAGE_BYTES = M * WT_BYTES;    // one block
  static_assert(VPT * (int)sizeof(T) * 2 == kStreamRowBytes, "a lane chunk is half a 128-byte row");
  static_assert(NSTAGE >= 3, "blocks b and b+1 stay resident while b+2 loads");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bars[NWARP][NSTAGE];

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char *ring = smem_raw + ((1024u - (tma::smem_u32(smem_raw) & 1023u)) & 1023u) +
                        (size_t)warp * NSTAGE * STAGE_BYTES;
  const uint64_t gw = (uint64_t)blockIdx.x * NWARP + warp;
  const uint64_t b0 = gw * per_warp;
  if (lane == 0) {
    for (int s = 0; s < NSTAGE; ++s) tma::mbar_init(&bars[warp][s], 1);
    tma::fence_mbar_init();
  }
  __syncwarp();
  if (b0 >= nob) return;
  const uint64_t b1 = b0 + per_warp < nob ? b0 + per_warp : nob;  // output blocks [b0, b1)
  const uint64_t nst = b1 - b0 + 1;                                  // input blocks b0 .. b1
  auto issue = [&](uint64_t s) {
    unsigned long long *bar = &bars[warp][s % NSTAGE];
    tma::mbar_arrive_expect_tx(bar, STAGE_BYTES);
    tma::tensor_g2s_2d(ring + (s % NSTAGE) * STAGE_BYTES, &tmap, 0, (int)((b0 + s) * (STAGE_BYTES / kStreamRowBytes)),
                       bar);
  };
  if (lane == 0) {
    tma::prefetch_tensormap(&tmap);
    for (uint64_t s = 0; s < (uint64_t)NSTAGE && s < nst; ++s) issue(s);
  }
  // lane chunk j of the block in stage s (global block b), patched past the tensor's full rows
  auto load_chunk = [&](uint64_t s, uint64_t b, int j, T (&x)[VPT]) {
    const int row = j * (WT_BYTES / kStreamRowBytes) + (lane >> 1);
    const unsigned char *src = ring + (s % NSTAGE) * STAGE_BYTES + row * kStreamRowBytes;
    uint4 u[UPR];
#pragma unroll
    for (int c = 0; c < UPR; ++c) u[c] = *reinterpret_cast<const uint4 *>(src + ((((lane & 1) * UPR + c) ^ (row & 7)) << 4));
    memcpy(x, u, sizeof(u));
    const uint64_t g = b * (uint64_t)BLK + (uint64_t)j * WT + (uint64_t)lane * VPT;
    if (g + VPT > n_full) {
#pragma unroll
      for (int i = 0; i < VPT; ++i)
        if (g + i >= n_full) x[i] = (g + i < n) ? in[g + i] : Op::identity();
    }
  };
  const bool vec = aligned16(out);
  const uint64_t nout = n - (uint64_t)BLK + 1;
  T tot[M];  // warp-tile totals of the block that is "next" (becomes "current" one step later)
  for (uint64_t s = 0; s < nst; ++s) {
    const uint64_t b = b0 + s;  // the block in stage s: "next"; block b-1 is "current"
    const bool ok = stream_wait(&bars[warp][s % NSTAGE], (uint32_t)(s / NSTAGE) & 1u);
    if (!__all_sync(kFull, ok)) {
      if (lane == 0) {
        atomicOr(err, DEVERR_COPY_TIMEOUT);
        for (uint64_t s2 = s; s2 < s + NSTAGE && s2 < nst; ++s2)
          stream_wait(&bars[warp][s2 % NSTAGE], (uint32_t)(s2 / NSTAGE) & 1u);
      }
      return;
    }
    // suffix carries of the current block: sufT[j] = tot[j] (+) ... (+) tot[M-1]
    T sufT[M + 1];
    sufT[M] = Op::identity();
#pragma unroll
    for (int j = M - 1; j >= 0; --j) sufT[j] = (s > 0) ? Op::op(tot[j], sufT[j + 1]) : Op::identity();
    T carryP = Op::identity();  // prefix of the next block up to the end of the previous warp-tile
#pragma unroll
    for (int j = 0; j < M; ++j) {
      // next block, warp-tile j: prefix sums from the block start
      T P[VPT];
      load_chunk(s, b, j, P);
#pragma unroll
      for (int i = 1; i < VPT; ++i) P[i] = Op::op(P[i - 1], P[i]);
      T v = P[VPT - 1];
      for (int d = 1; d < 32; d <<= 1) {
        const T a = shfl_up_t(v, d);
        if (lane >= d) v = Op::op(a, v);
      }
      const T wtot = shfl_idx_t(v, 31);
      T ex = shfl_up_t(v, 1);
      ex = lane == 0 ? carryP : Op::op(carryP, ex);
#pragma unroll
      for (int i = 0; i < VPT; ++i) P[i] = Op::op(ex, P[i]);
      if (s > 0) {
        // current block, warp-tile j: suffix sums to the block end
        T S[VPT];
        load_chunk(s - 1, b - 1, j, S);
#pragma unroll
        for (int i = VPT - 2; i >= 0; --i) S[i] = Op::op(S[i], S[i + 1]);
        T u = S[0];
        for (int d = 1; d < 32; d <<= 1) {
          const T a = shfl_down_t(u, d);
          if (lane + d < 32) u = Op::op(u, a);
        }
        T es = shfl_down_t(u, 1);
        es = lane == 31 ? sufT[j + 1] : Op::op(es, sufT[j + 1]);
#pragma unroll
        for (int i = 0; i < VPT; ++i) S[i] = Op::op(S[i], es);
        // y = S (current) (+) P (next) at the previous element
        const T pprev = shfl_up_t(P[VPT - 1], 1);
        T y[VPT];
        y[0] = (lane == 0 && j == 0) ? S[0] : Op::op(S[0], lane == 0 ? carryP : pprev);
#pragma unroll
        for (int i = 1; i < VPT; ++i) y[i] = Op::op(S[i], P[i - 1]);
        const uint64_t go = (b - 1) * (uint64_t)BLK + (uint64_t)j * WT + (uint64_t)lane * VPT;
        store_tile<Op, VPT>(out, nout, go, 0, 0x7fffffff, vec, y);
      }
      carryP = Op::op(carryP, wtot);
      tot[j] = wtot;
    }
    // stage s-1 (the current block) is consumed: refill its slot
    __syncwarp();
    if (lane == 0 && s >= 1 && s - 1 + NSTAGE < nst) {
      tma::fence_proxy_async_smem();
      issue(s - 1 + NSTAGE);
    }
  }
}

// ------------------------------------------------------------------------------------------
// Block-combine for w in {1, 2, 4, 8} dividing VPT: everything in registers
// ------------------------------------------------------------------------------------------
// Each thread owns VPT consecutive outputs starting at a multiple of VPT (hence of W) and loads
// the VPT + W - 1 inputs they need (the W - 1 extra ones come from the next thread's chunk, out
// of L1).  Blocks of W are compile-time: S within block b, P within block b+1, one (+) per output.
template <class Op, int W, int VPT>
__global__ void __launch_bounds__(256) k_slide_small(const typename Op::T *__restrict__ in,
                                                     typename Op::T *__restrict__ out, uint64_t n) {
  using T = typename Op::T;
  constexpr int EPV = 16 / (int)sizeof(T);
  constexpr int EXT = W > 1 ? ((W - 1 + EPV - 1) / EPV) * EPV : 0;
  static_assert(VPT % W == 0, "W must divide VPT");
  const uint64_t nout = n - (uint64_t)W + 1;
  const uint64_t g = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * (uint64_t)VPT;
  if (g >= nout) return;
  const bool vec = aligned16(in) && aligned16(out);
  T x[VPT + EXT];
  if (vec && g + VPT + EXT <= n) {
    T a[VPT];
    load_vec<T, VPT>(in + g, a);
#pragma unroll
    for (int j = 0; j < VPT; ++j) x[j] = a[j];
    if (EXT > 0) {
      T b[EXT > 0 ? EXT : EPV];
      load_vec<T, (EXT > 0 ? EXT : EPV)>(in + g + VPT, b);
#pragma unroll
      for (int j = 0; j < EXT; ++j) x[VPT + j] = b[j];
    }
  } else {
#pragma unroll
    for (int j = 0; j < VPT + EXT; ++j) x[j] = (g + j < n) ? in[g + j] : Op::identity();
  }
  T y[VPT];
#pragma unroll
  for (int b = 0; b < VPT / W; ++b) {
    T S[W], Pn[W > 1 ? W - 1 : 1];
    S[W - 1] = x[b * W + W - 1];
#pragma unroll
    for (int i = W - 2; i >= 0; --i) S[i] = Op::op(x[b * W + i], S[i + 1]);
    if (W > 1) {
      Pn[0] = x[(b + 1) * W];
#pragma unroll
      for (int i = 1; i < W - 1; ++i) Pn[i] = Op::op(Pn[i - 1], x[(b + 1) * W + i]);
    }
    y[b * W] = S[0];
#pragma unroll
    for (int i = 1; i < W; ++i) y[b * W + i] = Op::op(S[i], Pn[i - 1]);
  }
  store_tile<Op, VPT>(out, nout, g, 0, VPT, vec, y);
}

// ------------------------------------------------------------------------------------------
// Doubling
// ------------------------------------------------------------------------------------------
template <class Op>
struct IsIdempotent {
  static constexpr bool value = false;
};
template <>
struct IsIdempotent<OpMinI32> {
  static constexpr bool value = true;
};
template <>
struct IsIdempotent<OpMaxI32> {
  static constexpr bool value = true;
};

template <class Op, int NT, int VPT>
__global__ void __launch_bounds__(NT) k_slide_dbl(const typename Op::T *__restrict__ in,
                                                  typename Op::T *__restrict__ out, uint64_t n, int w, int TO) {
  using T = typename Op::T;
  constexpr int L = NT * VPT;
  constexpr int PADL = L + NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *buf0 = reinterpret_cast<T *>(smem_raw);
  T *buf1 = buf0 + PADL;
  auto pad = [](int i) { return i + i / VPT; };
  auto rd = [&](const T *b, int i) { return b[pad(i < L ? i : L - 1)]; };

  const uint64_t t0 = (uint64_t)blockIdx.x * (uint64_t)TO;
  const int o = threadIdx.x * VPT;
  const uint64_t g = t0 + (uint64_t)o;
  const bool vec = aligned16(in) && aligned16(out);
  T cur[VPT];
  load_tile<Op, VPT>(in, n, g, vec, cur);
#pragma unroll
  for (int j = 0; j < VPT; ++j) buf0[pad(o + j)] = cur[j];
  __syncthreads();

  const int top = 31 - __clz(w);  // 2^top <= w < 2^(top+1)
  T y[VPT];
  if (IsIdempotent<Op>::value) {
    for (int s = 0; s < top; ++s) {
      const T *src = (s & 1) ? buf1 : buf0;
      T *dst = (s & 1) ? buf0 : buf1;
#pragma unroll
      for (int j = 0; j < VPT; ++j) cur[j] = Op::op(cur[j], rd(src, o + j + (1 << s)));
#pragma unroll
      for (int j = 0; j < VPT; ++j) dst[pad(o + j)] = cur[j];
      __syncthreads();
    }
    const T *fin = (top & 1) ? buf1 : buf0;
    const int off = w - (1 << top);
#pragma unroll
    for (int j = 0; j < VPT; ++j) y[j] = Op::op(cur[j], rd(fin, o + j + off));
  } else {
    bool have = false;
    int lo = 0;
    for (int s = 0; s <= top; ++s) {
      const T *src = (s & 1) ? buf1 : buf0;  // windows of 2^s
      if ((w >> s) & 1) {
        const int off = w - lo - (1 << s);
#pragma unroll
        for (int j = 0; j < VPT; ++j) {
          const T v = rd(src, o + j + off);
          y[j] = have ? Op::op(v, y[j]) : v;
        }
        have = true;
        lo += 1 << s;
      }
      if (s < top) {
        T *dst = (s & 1) ? buf0 : buf1;
#pragma unroll
        for (int j = 0; j < VPT; ++j) cur[j] = Op::op(cur[j], rd(src, o + j + (1 << s)));
#pragma unroll
        for (int j = 0; j < VPT; ++j) dst[pad(o + j)] = cur[j];
        __syncthreads();
      }
    }
  }
  store_tile<Op, VPT>(out, n - (uint64_t)w + 1, g, o, TO, vec, y);
}

// ------------------------------------------------------------------------------------------
// Prefix difference (invertible operators)
// ------------------------------------------------------------------------------------------
template <class Op>
struct Inverse;
template <>
struct Inverse<OpAddI32> {
  static __device__ __forceinline__ uint32_t undo(uint32_t total, uint32_t head) { return total - head; }
};
template <>
struct Inverse<OpXorI32> {
  static __device__ __forceinline__ uint32_t undo(uint32_t total, uint32_t head) { return total ^ head; }
};

template <class Op, int NT, int VPT>
__global__ void __launch_bounds__(NT) k_slide_pd(const uint32_t *__restrict__ in, uint32_t *__restrict__ out,
                                                 uint64_t n, int w, int TO) {
  constexpr int NW = NT / 32;
  constexpr int L = NT * VPT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint32_t *T = reinterpret_cast<uint32_t *>(smem_raw);  // running sums, padded (L + NT words)
  __shared__ uint32_t wtot[NW];
  auto pad = [](int i) { return i + i / VPT; };

  const uint64_t t0 = (uint64_t)blockIdx.x * (uint64_t)TO;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int o = threadIdx.x * VPT;
  const uint64_t g = t0 + (uint64_t)o;
  const bool vec = aligned16(in) && aligned16(out);
  uint32_t x[VPT];
  load_tile<Op, VPT>(in, n, g, vec, x);
#pragma unroll
  for (int j = 1; j < VPT; ++j) x[j] = Op::op(x[j - 1], x[j]);
  const uint32_t v = warp_seg_scan_fwd<Op>(x[VPT - 1], 0u, lane);
  if (lane == 31) wtot[warp] = v;
  __syncthreads();
  uint32_t carry = Op::identity();
  for (int i = 0; i < warp; ++i) carry = Op::op(carry, wtot[i]);
  const uint32_t ev = shfl_up_t(v, 1);
  if (lane > 0) carry = Op::op(carry, ev);
#pragma unroll
  for (int j = 0; j < VPT; ++j) {
    x[j] = Op::op(carry, x[j]);
    T[pad(o + j)] = x[j];
  }
  __syncthreads();
  uint32_t y[VPT];
#pragma unroll
  for (int j = 0; j < VPT; ++j) {
    int q = o + j + w - 1;
    q = q < L ? q : L - 1;
    const uint32_t head = (o + j == 0) ? Op::identity() : (j == 0 ? T[pad(o - 1)] : x[j - 1]);
    y[j] = Inverse<Op>::undo(T[pad(q)], head);
  }
  store_tile<Op, VPT>(out, n - (uint64_t)w + 1, g, o, TO, vec, y);
}

// ------------------------------------------------------------------------------------------
// Launch plumbing
// ------------------------------------------------------------------------------------------
template <class Cfg, int ESIZE>
struct Shape {
  static constexpr int NT = Cfg::NT;
  static constexpr int VPT = ESIZE == 4 ? Cfg::VPT4 : Cfg::VPT8;
  static constexpr int L = NT * VPT;
};

int tile_outputs(int L, int esize, int w) {
  const int align = 16 / esize;
  const int to = (L - (w - 1)) / align * align;
  return to >= align ? to : 0;
}

// The aligned block-combine applies when blocks are whole thread chunks, blocks of at most a
// warp divide the warp (or are whole warps), and a tile holds at least one block of outputs.
bool aligned_blocks_ok(int w, int vpt, int nt, int L) {
  if (w % vpt != 0) return false;
  const int G = w / vpt;
  const bool shape = (G <= 32 && 32 % G == 0) || (G % 32 == 0 && G / 32 <= nt / 32);
  return shape && (L - w + 1) / w >= 1;
}

template <class Kern>
cudaError_t set_smem(Kern kern, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// ---- persistent TMA-staged block-combine ---------------------------------------------------
using EncodeTiled = PFN_cuTensorMapEncodeTiled_v12000;

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime (no -lcuda).
EncodeTiled encode_tiled() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  });
  return fn;
}

int gcd_int(int a, int b) {
  while (b) {
    const int r = a % b;
    a = b;
    b = r;
  }
  return a;
}

// Outputs per tile of the streamed kernel: the largest multiple of lcm(w, elements per 128-byte
// row) that leaves the tile room for the following block; 0 when none fits.
int stream_tile_outputs(int L, int esize, int w) {
  const long long r = kStreamRowBytes / esize;
  const long long unit = (long long)w / gcd_int(w, (int)r) * r;
  return (int)((L - w + 1) / unit * unit);
}

template <class Op, int NT, int VPT, int MINB>
cudaError_t launch_stream(const void *in, void *out, uint64_t n, int w, int num_sms, int *err, cudaStream_t st,
                          bool quiet_unsupported) {
  using T = typename Op::T;
  constexpr int STAGES = 2;
  constexpr int L = NT * VPT;
  constexpr int ES = (int)sizeof(T);
  constexpr int ROW = VPT * ES / 16 + 1;
  static_assert(L * ES / kStreamRowBytes <= 256, "a TMA box has at most 256 rows");
  const int TO = stream_tile_outputs(L, ES, w);
  const uint64_t rows = n * ES / kStreamRowBytes;
  const uint64_t nout = n - (uint64_t)w + 1;
  const uint64_t tiles = TO > 0 ? (nout + (uint64_t)TO - 1) / (uint64_t)TO : 0;
  EncodeTiled enc = encode_tiled();
  if (TO == 0 || rows == 0 || rows > (1ull << 32) || (reinterpret_cast<uintptr_t>(in) & 15u) != 0 ||
      !aligned_blocks_ok(w, VPT, NT, L) || !enc || num_sms < 1 || err == nullptr ||
      tiles * (uint64_t)TO * ES / kStreamRowBytes > 0x7fffffffull)
    return quiet_unsupported ? cudaErrorNotSupported : cudaErrorInvalidValue;
  CUtensorMap map;
  const cuuint64_t gdim[2] = {kStreamRowBytes / 4, rows};
  const cuuint64_t gstride[1] = {kStreamRowBytes};
  const cuuint32_t box[2] = {kStreamRowBytes / 4, (cuuint32_t)(L * ES / kStreamRowBytes)};
  const cuuint32_t estr[2] = {1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void *>(in), gdim, gstride, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const size_t smem = (size_t)STAGES * L * ES + (size_t)NT * ROW * 16 + 1024;
  auto kern = k_slide_tma<Op, NT, VPT, STAGES, MINB>;
  // resident CTAs per SM, once per device (the attribute and the answer do not change)
  static int per_sm[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int nb = (dev >= 0 && dev < 64) ? per_sm[dev] : 0;
  if (nb == 0) {
    e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, NT, smem);
    if (e != cudaSuccess) return e;
    if (nb < 1) return cudaErrorInvalidConfiguration;
    if (dev >= 0 && dev < 64) per_sm[dev] = nb;
  }
  uint64_t grid = (uint64_t)num_sms * (uint64_t)nb;
  if (grid > tiles) grid = tiles;
  const uint64_t n_full = rows * kStreamRowBytes / ES;
  kern<<<(unsigned)grid, NT, smem, st>>>(map, static_cast<const T *>(in), static_cast<T *>(out), n, n_full, w, TO,
                                         tiles, err);
  return cudaGetLastError();
}

// Warp-private streaming block-combine: w = VPT * G, G a power of two <= 32.  The run shape
// (warps per CTA, warp-tiles per stage, stages) is chosen by G: narrow blocks want more bytes in
// flight per warp, wide blocks more warps (measured on GB300 over the sweep's operators).
template <class Op, int NWARP, int SW, int NSTAGE>
cudaError_t launch_warp_shape(const CUtensorMap &map, const void *in, void *out, uint64_t n, uint64_t n_full, int w,
                              uint64_t nwt, int num_sms, int *err, cudaStream_t st) {
  using T = typename Op::T;
  constexpr int VPT = kStreamRowBytes / 2 / (int)sizeof(T);
  constexpr int STAGE_BYTES = SW * 32 * VPT * (int)sizeof(T);
  const size_t smem = (size_t)NWARP * NSTAGE * STAGE_BYTES + 1024;
  auto kern = k_slide_warp<Op, VPT, NWARP, SW, NSTAGE>;
  static int per_sm[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int nb = (dev >= 0 && dev < 64) ? per_sm[dev] : 0;
  if (nb == 0) {
    e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, NWARP * 32, smem);
    if (e != cudaSuccess) return e;
    if (nb < 1) return cudaErrorInvalidConfiguration;
    if (dev >= 0 && dev < 64) per_sm[dev] = nb;
  }
  const uint64_t warps = (uint64_t)num_sms * nb * NWARP;
  const uint64_t per_warp = (nwt + warps - 1) / warps;
  const uint64_t grid = ((nwt + per_warp - 1) / per_warp + NWARP - 1) / NWARP;
  kern<<<(unsigned)grid, NWARP * 32, smem, st>>>(map, static_cast<const T *>(in), static_cast<T *>(out), n, n_full, w,
                                                 nwt, per_warp, err);
  return cudaGetLastError();
}

template <class Op, int M, int NWARP, int NSTAGE>
cudaError_t launch_wblk_shape(const void *in, void *out, uint64_t n, int num_sms, int *err, cudaStream_t st) {
  using T = typename Op::T;
  constexpr int ES = (int)sizeof(T);
  constexpr int VPT = kStreamRowBytes / 2 / ES;
  constexpr int BLK = M * 32 * VPT;
  constexpr int STAGE_BYTES = BLK * ES;
  static_assert(STAGE_BYTES / kStreamRowBytes <= 256, "a TMA box has at most 256 rows");
  const uint64_t rows = n * ES / kStreamRowBytes;
  const uint64_t nout = n - (uint64_t)BLK + 1;
  const uint64_t nob = (nout + BLK - 1) / BLK;  // output blocks; input blocks 0 .. nob
  if ((nob + 1) * (uint64_t)(STAGE_BYTES / kStreamRowBytes) > 0x7fffffffull) return cudaErrorNotSupported;
  EncodeTiled enc = encode_tiled();
  CUtensorMap map;
  const cuuint64_t gdim[2] = {kStreamRowBytes / 4, rows};
  const cuuint64_t gstride[1] = {kStreamRowBytes};
  const cuuint32_t box[2] = {kStreamRowBytes / 4, (cuuint32_t)(STAGE_BYTES / kStreamRowBytes)};
  const cuuint32_t estr[2] = {1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void *>(in), gdim, gstride, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const size_t smem = (size_t)NWARP * NSTAGE * STAGE_BYTES + 1024;
  auto kern = k_slide_wblk<Op, VPT, M, NWARP, NSTAGE>;
  static int per_sm[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int nb = (dev >= 0 && dev < 64) ? per_sm[dev] : 0;
  if (nb == 0) {
    e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, NWARP * 32, smem);
    if (e != cudaSuccess) return e;
    if (nb < 1) return cudaErrorInvalidConfiguration;
    if (dev >= 0 && dev < 64) per_sm[dev] = nb;
  }
  const uint64_t warps = (uint64_t)num_sms * nb * NWARP;
  const uint64_t per_warp = (nob + warps - 1) / warps;
  const uint64_t grid = ((nob + per_warp - 1) / per_warp + NWARP - 1) / NWARP;
  const uint64_t n_full = rows * kStreamRowBytes / ES;
  kern<<<(unsigned)grid, NWARP * 32, smem, st>>>(map, static_cast<const T *>(in), static_cast<T *>(out), n, n_full, nob,
                                                 per_warp, err);
  return cudaGetLastError();
}

template <class Op>
cudaError_t launch_warp_stream(const void *in, void *out, uint64_t n, int w, int num_sms, int *err, cudaStream_t st,
                               bool quiet_unsupported, int shape) {
  using T = typename Op::T;
  constexpr int ES = (int)sizeof(T);
  constexpr int VPT = kStreamRowBytes / 2 / ES;  // 16 for 4-byte elements, 8 for affine pairs
  constexpr int WT = 32 * VPT;
  const int G = w % VPT == 0 ? w / VPT : 0;
  const uint64_t rows = n * ES / kStreamRowBytes;
  EncodeTiled enc = encode_tiled();
  const bool blocks_of_tiles = G == 64 || G == 128 || G == 256;
  if (G < 1 || G > 256 || (G & (G - 1)) != 0 || rows == 0 || rows > (1ull << 32) ||
      (reinterpret_cast<uintptr_t>(in) & 15u) != 0 || !enc || num_sms < 1 || err == nullptr)
    return quiet_unsupported ? cudaErrorNotSupported : cudaErrorInvalidValue;
  if (blocks_of_tiles) {  // blocks of 2, 4 or 8 whole warp-tiles
    if (G == 64) return launch_wblk_shape<Op, 2, 16, 3>(in, out, n, num_sms, err, st);
    if (G == 128) return launch_wblk_shape<Op, 4, 8, 3>(in, out, n, num_sms, err, st);
    return launch_wblk_shape<Op, 8, 4, 3>(in, out, n, num_sms, err, st);
  }
  // one warp-tile past the last full one: the lanes that emit a tile late need the next tile's
  // prefixes even when n is a multiple of the warp-tile (that tile is then all identity)
  const uint64_t nwt = n / WT + 1;
  if (nwt * (uint64_t)(WT * ES / kStreamRowBytes) > 0x7fffffffull) return cudaErrorNotSupported;
  // run shapes (warps per CTA, warp-tiles per stage, stages): 1 = 4 x 8 x 2, 2 = 8 x 4 x 2,
  // 3 = 16 x 2 x 3; by default narrow blocks take more bytes in flight per warp, wide ones more warps
  if (shape < 1 || shape > kWarpShapes) shape = G == 1 ? 1 : (G <= 4 ? 2 : 3);
  const int sw = shape == 1 ? 8 : (shape == 2 ? 4 : 2);  // warp-tiles per stage
  CUtensorMap map;
  const cuuint64_t gdim[2] = {kStreamRowBytes / 4, rows};
  const cuuint64_t gstride[1] = {kStreamRowBytes};
  const cuuint32_t box[2] = {kStreamRowBytes / 4, (cuuint32_t)(sw * WT * ES / kStreamRowBytes)};
  const cuuint32_t estr[2] = {1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void *>(in), gdim, gstride, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const uint64_t n_full = rows * kStreamRowBytes / ES;
  if (shape == 1) return launch_warp_shape<Op, 4, 8, 2>(map, in, out, n, n_full, w, nwt, num_sms, err, st);
  if (shape == 2) return launch_warp_shape<Op, 8, 4, 2>(map, in, out, n, n_full, w, nwt, num_sms, err, st);
  return launch_warp_shape<Op, 16, 2, 3>(map, in, out, n, n_full, w, nwt, num_sms, err, st);
}

template <class Op, class Cfg>
cudaError_t launch_op(const SlideLaunch &SL, const void *in, void *out, uint64_t n, int w, cudaStream_t st) {
  using T = typename Op::T;
  using S = Shape<Cfg, (int)sizeof(T)>;
  constexpr int MINB = 1024 / S::NT;
  const int variant = SL.variant;
  if (variant == SWS_VARIANT_BLOCK_COMBINE_STREAM)
    return launch_stream<Op, S::NT, S::VPT, MINB>(in, out, n, w, SL.num_sms, SL.err, st, true);
  if (variant == SWS_VARIANT_BLOCK_COMBINE_WARP)
    return launch_warp_stream<Op>(in, out, n, w, SL.num_sms, SL.err, st, true, SL.shape);
  if (variant == SWS_VARIANT_AUTO && !(w <= 8 && S::VPT % w == 0)) {
    // warp-private streaming when w's blocks fit a warp and the input fills the GPU a few times
    constexpr uint64_t WT = 32 * (kStreamRowBytes / 2 / sizeof(T));
    if (n / WT >= 64ull * (uint64_t)SL.num_sms) {
      const cudaError_t e = launch_warp_stream<Op>(in, out, n, w, SL.num_sms, SL.err, st, true, SL.shape);
      if (e != cudaErrorNotSupported) return e;
    }
    // streamed when the grid fills the GPU at least twice; the one-shot tiles otherwise
    const int TOs = stream_tile_outputs(S::L, (int)sizeof(T), w);
    if (TOs > 0 && (n - (uint64_t)w + 1) / (uint64_t)TOs >= 2ull * (uint64_t)SL.num_sms * (uint64_t)MINB) {
      const cudaError_t e = launch_stream<Op, S::NT, S::VPT, MINB>(in, out, n, w, SL.num_sms, SL.err, st, true);
      if (e != cudaErrorNotSupported) return e;
    }
  }
  const int TO = tile_outputs(S::L, (int)sizeof(T), w);
  if (TO == 0) return cudaErrorInvalidValue;
  const uint64_t nout = n - (uint64_t)w + 1;
  const uint64_t tiles = (nout + (uint64_t)TO - 1) / (uint64_t)TO;
  if (tiles > 0x7fffffffull) return cudaErrorInvalidValue;
  const T *pin = static_cast<const T *>(in);
  T *pout = static_cast<T *>(out);
  if (variant == SWS_VARIANT_DOUBLING) {
    const size_t sm = 2 * (size_t)(S::L + S::NT) * sizeof(T);
    auto kern = k_slide_dbl<Op, S::NT, S::VPT>;
    cudaError_t e = set_smem(kern, sm);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)tiles, S::NT, sm, st>>>(pin, pout, n, w, TO);
  } else if (w <= 8 && S::VPT % w == 0) {
    const uint64_t chunks = (nout + S::VPT - 1) / S::VPT;
    const uint64_t blocks = (chunks + 255) / 256;
    if (blocks > 0x7fffffffull) return cudaErrorInvalidValue;
    switch (w) {
      case 1: k_slide_small<Op, 1, S::VPT><<<(unsigned)blocks, 256, 0, st>>>(pin, pout, n); break;
      case 2: k_slide_small<Op, 2, S::VPT><<<(unsigned)blocks, 256, 0, st>>>(pin, pout, n); break;
      case 4: k_slide_small<Op, 4, S::VPT><<<(unsigned)blocks, 256, 0, st>>>(pin, pout, n); break;
      default: k_slide_small<Op, 8, S::VPT><<<(unsigned)blocks, 256, 0, st>>>(pin, pout, n); break;
    }
  } else if (aligned_blocks_ok(w, S::VPT, S::NT, S::L)) {
    const int TOa = (S::L - w + 1) / w * w;
    const uint64_t tiles_a = (nout + (uint64_t)TOa - 1) / (uint64_t)TOa;
    if (tiles_a > 0x7fffffffull) return cudaErrorInvalidValue;
    constexpr int ROW = S::VPT * (int)sizeof(T) / 16 + 1;
    const size_t sm = (size_t)S::NT * ROW * 16;
    auto kern = k_slide_al<Op, S::NT, S::VPT>;
    cudaError_t e = set_smem(kern, sm);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)tiles_a, S::NT, sm, st>>>(pin, pout, n, w, TOa);
  } else {
    const size_t sm = sizeof(typename BlockCombine<Op, S::NT, S::VPT>::Shared);
    auto kern = k_slide_bc<Op, S::NT, S::VPT>;
    cudaError_t e = set_smem(kern, sm);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)tiles, S::NT, sm, st>>>(pin, pout, n, w, TO);
  }
  return cudaGetLastError();
}

template <class Op, class Cfg>
cudaError_t launch_pd(const void *in, void *out, uint64_t n, int w, cudaStream_t st) {
  using S = Shape<Cfg, 4>;
  const int TO = tile_outputs(S::L, 4, w);
  if (TO == 0) return cudaErrorInvalidValue;
  const uint64_t nout = n - (uint64_t)w + 1;
  const uint64_t tiles = (nout + (uint64_t)TO - 1) / (uint64_t)TO;
  if (tiles > 0x7fffffffull) return cudaErrorInvalidValue;
  const size_t sm = (size_t)(S::L + S::NT) * 4;
  auto kern = k_slide_pd<Op, S::NT, S::VPT>;
  cudaError_t e = set_smem(kern, sm);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)tiles, S::NT, sm, st>>>(static_cast<const uint32_t *>(in), static_cast<uint32_t *>(out), n, w, TO);
  return cudaGetLastError();
}

template <class Cfg>
cudaError_t launch_cfg(const SlideLaunch &L, const void *in, void *out, uint64_t n, int w, cudaStream_t st) {
  if (L.variant == SWS_VARIANT_PREFIX_DIFF) {
    if (L.op == SWS_OP_ADD_I32) return launch_pd<OpAddI32, Cfg>(in, out, n, w, st);
    if (L.op == SWS_OP_XOR_I32) return launch_pd<OpXorI32, Cfg>(in, out, n, w, st);
    return cudaErrorInvalidValue;
  }
  switch (L.op) {
    case SWS_OP_ADD_I32: return launch_op<OpAddI32, Cfg>(L, in, out, n, w, st);
    case SWS_OP_MIN_I32: return launch_op<OpMinI32, Cfg>(L, in, out, n, w, st);
    case SWS_OP_MAX_I32: return launch_op<OpMaxI32, Cfg>(L, in, out, n, w, st);
    case SWS_OP_XOR_I32: return launch_op<OpXorI32, Cfg>(L, in, out, n, w, st);
    case SWS_OP_AFFINE_U32: return launch_op<OpAffineU32, Cfg>(L, in, out, n, w, st);
    case SWS_OP_ADD_F32: return launch_op<OpAddF32, Cfg>(L, in, out, n, w, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

namespace {
// A splitmix-style finaliser of the word index: any fixed pattern works for timing.
__global__ void k_fill_pattern(uint32_t *__restrict__ dst, uint64_t words) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (uint64_t)gridDim.x * blockDim.x) {
    unsigned long long z = i * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    dst[i] = (uint32_t)(z ^ (z >> 31)) & 0x00FFFFFFu;  // small values: no float specials
  }
}
}  // namespace

cudaError_t launch_fill_pattern(void *dst, uint64_t bytes, cudaStream_t st) {
  const uint64_t words = bytes / 4;
  if (words == 0) return cudaSuccess;
  k_fill_pattern<<<1024, 256, 0, st>>>(static_cast<uint32_t *>(dst), words);
  return cudaGetLastError();
}

int slide_tile_len(int cfg, int esize) {
  if (cfg == CFG_SMALL) return esize == 4 ? Shape<CfgSmall, 4>::L : Shape<CfgSmall, 8>::L;
  return esize == 4 ? Shape<CfgLarge, 4>::L : Shape<CfgLarge, 8>::L;
}

int slide_tile_outputs(int cfg, int esize, int w) { return tile_outputs(slide_tile_len(cfg, esize), esize, w); }

cudaError_t launch_sliding_sum(const SlideLaunch &L, const void *in, void *out, uint64_t n, int w,
                               cudaStream_t stream) {
  if (L.cfg == CFG_SMALL) return launch_cfg<CfgSmall>(L, in, out, n, w, stream);
  return launch_cfg<CfgLarge>(L, in, out, n, w, stream);
}

}  // namespace sws
