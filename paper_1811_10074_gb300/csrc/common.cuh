// common.cuh -- device building blocks shared by the library's kernels: the associative
// operators of the sliding sum (Eq. 2), warp shuffles for any element type, segmented
// warp/CTA scans, and the block-combine tile routine.
//
// Block-combine (a GPU restatement of the "Vector Input" scheme, Alg. 2 of Sec. 3.1, with the
// block length chosen equal to w): cut the sequence into blocks of w elements aligned at
// global multiples of w.  A window [p, p+w-1] is the suffix of p's block from p plus the prefix
// of the next block up to p+w-1, so
//     y_p = S_p (+) P_{p+w-1}      (S = in-block suffix sums, P = in-block prefix sums),
// and y_p = S_p when p starts a block.  Both scans need only associativity and keep operand
// order, so non-commutative operators (affine maps) are exact; each output costs O(1) (+).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sws {

constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------------------------------------------
// Operators: T, op(left, right) with left = earlier elements, identity().
// ------------------------------------------------------------------------------------------
struct OpAddI32 {
  using T = uint32_t;
  static __device__ __forceinline__ T op(T l, T r) { return l + r; }
  static __device__ __forceinline__ T identity() { return 0u; }
};
struct OpMinI32 {
  using T = int32_t;
  static __device__ __forceinline__ T op(T l, T r) { return r < l ? r : l; }
  static __device__ __forceinline__ T identity() { return 0x7fffffff; }
};
struct OpMaxI32 {
  using T = int32_t;
  static __device__ __forceinline__ T op(T l, T r) { return r > l ? r : l; }
  static __device__ __forceinline__ T identity() { return (int32_t)0x80000000; }
};
struct OpXorI32 {
  using T = uint32_t;
  static __device__ __forceinline__ T op(T l, T r) { return l ^ r; }
  static __device__ __forceinline__ T identity() { return 0u; }
};
// Affine map x -> a*x + b (mod 2^32) as uint2{a, b}; op(l, r) = "apply l, then r".
struct OpAffineU32 {
  using T = uint2;
  static __device__ __forceinline__ T op(T l, T r) { return make_uint2(r.x * l.x, r.x * l.y + r.y); }
  static __device__ __forceinline__ T identity() { return make_uint2(1u, 0u); }
};
struct OpAddF32 {
  using T = float;
  static __device__ __forceinline__ T op(T l, T r) { return l + r; }
  static __device__ __forceinline__ T identity() { return 0.0f; }
};
// Minimizer key with a hash of at most 32 bits: (hash << 32) | position; min = least hash,
// leftmost position on ties.
struct OpMinKey64 {
  using T = unsigned long long;
  static __device__ __forceinline__ T op(T l, T r) { return r < l ? r : l; }
  static __device__ __forceinline__ T identity() { return ~0ull; }
};
// Minimizer key with a hash of up to 64 bits: compared as (hash, position).
struct Key96 {
  uint32_t hlo, hhi, pos;
};
struct OpMinKey96 {
  using T = Key96;
  static __device__ __forceinline__ unsigned long long h(const T &a) {
    return ((unsigned long long)a.hhi << 32) | a.hlo;
  }
  static __device__ __forceinline__ T op(T l, T r) {
    unsigned long long hl = h(l), hr = h(r);
    return (hr < hl || (hr == hl && r.pos < l.pos)) ? r : l;
  }
  static __device__ __forceinline__ T identity() { return Key96{~0u, ~0u, ~0u}; }
};

// ------------------------------------------------------------------------------------------
// Shuffles for any 4-byte-multiple element type.
// ------------------------------------------------------------------------------------------
template <class T>
struct Words {
  static constexpr int N = (int)(sizeof(T) / 4);
  static_assert(sizeof(T) % 4 == 0, "element must be a multiple of 4 bytes");
};

template <class T>
__device__ __forceinline__ T shfl_up_t(T v, unsigned d) {
  uint32_t u[Words<T>::N];
  memcpy(u, &v, sizeof(T));
#pragma unroll
  for (int i = 0; i < Words<T>::N; ++i) u[i] = __shfl_up_sync(kFull, u[i], d);
  T r;
  memcpy(&r, u, sizeof(T));
  return r;
}
template <class T>
__device__ __forceinline__ T shfl_down_t(T v, unsigned d) {
  uint32_t u[Words<T>::N];
  memcpy(u, &v, sizeof(T));
#pragma unroll
  for (int i = 0; i < Words<T>::N; ++i) u[i] = __shfl_down_sync(kFull, u[i], d);
  T r;
  memcpy(&r, u, sizeof(T));
  return r;
}
template <class T>
__device__ __forceinline__ T shfl_idx_t(T v, int src) {
  uint32_t u[Words<T>::N];
  memcpy(u, &v, sizeof(T));
#pragma unroll
  for (int i = 0; i < Words<T>::N; ++i) u[i] = __shfl_sync(kFull, u[i], src);
  T r;
  memcpy(&r, u, sizeof(T));
  return r;
}

__device__ __forceinline__ unsigned lanemask_le(int lane) { return lane == 31 ? kFull : ((2u << lane) - 1u); }
__device__ __forceinline__ unsigned lanemask_lt(int lane) { return (1u << lane) - 1u; }

// Inclusive segmented scan over the lanes of a warp, left to right.  `flag` marks lanes whose
// value begins a new segment; each lane ends with the (+) of the values from its segment's
// first lane up to itself.
template <class Op>
__device__ __forceinline__ typename Op::T warp_seg_scan_fwd(typename Op::T v, unsigned flags, int lane) {
  int h = 31 - __clz(flags & lanemask_le(lane));  // -1 when no flagged lane <= lane
  if (h < 0) h = 0;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    typename Op::T u = shfl_up_t(v, d);
    if (lane - d >= h) v = Op::op(u, v);
  }
  return v;
}

// Mirror image: right to left; `flags` marks lanes whose value ends a segment.
template <class Op>
__device__ __forceinline__ typename Op::T warp_seg_scan_bwd(typename Op::T v, unsigned flags, int lane) {
  int h = __ffs(flags & ~lanemask_lt(lane)) - 1;  // -1 when no flagged lane >= lane
  if (h < 0) h = 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    typename Op::T u = shfl_down_t(v, d);
    if (lane + d <= h) v = Op::op(v, u);
  }
  return v;
}

// ------------------------------------------------------------------------------------------
// Block-combine over one CTA tile of NT*VPT consecutive elements (thread t holds elements
// t*VPT .. t*VPT+VPT-1 of the tile in registers).
// ------------------------------------------------------------------------------------------
template <class Op, int NT, int VPT>
struct BlockCombine {
  using T = typename Op::T;
  static constexpr int NW = NT / 32;
  static constexpr int L = NT * VPT;
  static constexpr int PADL = L + NT;  // one pad slot per VPT elements: conflict-free shifted reads
  static_assert(NT % 32 == 0 && NW <= 32, "NT must be a multiple of 32, at most 1024");
  static_assert(VPT >= 1 && VPT <= 32, "VPT must be in [1, 32]");

  struct Shared {
    T P[PADL];
    T wf[NW];
    T wb[NW];
    unsigned char wflag[NW];  // bit 0: the warp holds a block start; bit 1: a block end
  };

  static __device__ __forceinline__ int pad(int i) { return i + i / VPT; }

  // x: this thread's elements; r0: position of x[0] inside its block of w (0 <= r0 < w).
  // On return y[j] holds the window sum of the w elements starting at tile index
  // t*VPT + j, for every j with t*VPT + j + w - 1 < L.  Ends with the shared P array written
  // and one __syncthreads() after it; the caller must sync before reusing `sh`.
  static __device__ __forceinline__ void run(Shared &sh, const T (&x)[VPT], int r0, int w, T (&y)[VPT]) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    T P[VPT], S[VPT];
    unsigned smask = 0;
    int r = r0;
#pragma unroll
    for (int j = 0; j < VPT; ++j) {
      const bool s = (r == 0);
      smask |= (unsigned)s << j;
      if (j == 0) P[0] = x[0];
      else P[j] = s ? x[j] : Op::op(P[j - 1], x[j]);
      r = (r + 1 == w) ? 0 : r + 1;
    }
    // element j ends a block iff element j+1 starts one; the last element ends one iff the
    // element after the thread's run (phase r) starts one.
    const unsigned emask = (smask >> 1) | ((unsigned)(r == 0) << (VPT - 1));
    S[VPT - 1] = x[VPT - 1];
#pragma unroll
    for (int j = VPT - 2; j >= 0; --j) S[j] = ((emask >> j) & 1u) ? x[j] : Op::op(x[j], S[j + 1]);

    // Warp-level segmented scans of the per-thread tails (forward) and heads (backward).
    const unsigned fb = __ballot_sync(kFull, smask != 0);
    const unsigned bb = __ballot_sync(kFull, emask != 0);
    const T vf = warp_seg_scan_fwd<Op>(P[VPT - 1], fb, lane);
    const T vb = warp_seg_scan_bwd<Op>(S[0], bb, lane);
    if (lane == 31) sh.wf[warp] = vf;
    if (lane == 0) {
      sh.wb[warp] = vb;
      sh.wflag[warp] = (unsigned char)((fb != 0u) | ((bb != 0u) << 1));
    }
    __syncthreads();
    const unsigned char wfl = lane < NW ? sh.wflag[lane] : (unsigned char)0;
    const unsigned wff = __ballot_sync(kFull, wfl & 1);
    const unsigned wbf = __ballot_sync(kFull, wfl & 2);

    // Carry into this warp from earlier warps (forward) and later warps (backward), each
    // warp computing its own with a lane-per-warp segmented scan.
    T cwf = Op::identity(), cwb = Op::identity();
    if (NW > 1) {
      if (warp > 0) {
        T v = lane < warp ? sh.wf[lane] : Op::identity();
        const unsigned f = wff & ((1u << warp) - 1u);
        v = warp_seg_scan_fwd<Op>(v, f, lane);
        cwf = shfl_idx_t(v, warp - 1);
      }
      if (warp < NW - 1) {
        T v = (lane > warp && lane < NW) ? sh.wb[lane] : Op::identity();
        const unsigned f = wbf & ~((2u << warp) - 1u);
        v = warp_seg_scan_bwd<Op>(v, f | (NW < 32 ? (1u << (NW - 1)) : 0u), lane);
        cwb = shfl_idx_t(v, warp + 1);
      }
    }

    // Exclusive carries into this thread.
    const T ef = shfl_up_t(vf, 1);
    const T eb = shfl_down_t(vb, 1);
    T cP, cS;
    bool hasP, hasS;
    if (lane == 0) {
      cP = cwf;
      hasP = warp > 0;
    } else if (fb & lanemask_lt(lane)) {
      cP = ef;
      hasP = true;
    } else {
      cP = warp > 0 ? Op::op(cwf, ef) : ef;
      hasP = true;
    }
    if (lane == 31) {
      cS = cwb;
      hasS = warp < NW - 1;
    } else if (bb & ~lanemask_le(lane)) {
      cS = eb;
      hasS = true;
    } else {
      cS = warp < NW - 1 ? Op::op(eb, cwb) : eb;
      hasS = true;
    }
#pragma unroll
    for (int j = 0; j < VPT; ++j) {
      if (hasP && (smask & ((2u << j) - 1u)) == 0u) P[j] = Op::op(cP, P[j]);
      if (hasS && (emask >> j) == 0u) S[j] = Op::op(S[j], cS);
    }

#pragma unroll
    for (int j = 0; j < VPT; ++j) sh.P[pad(t * VPT + j)] = P[j];
    __syncthreads();
    r = r0;
#pragma unroll
    for (int j = 0; j < VPT; ++j) {
      const int q = t * VPT + j + w - 1;
      y[j] = (r == 0 || q >= L) ? S[j] : Op::op(S[j], sh.P[pad(q)]);
      r = (r + 1 == w) ? 0 : r + 1;
    }
  }
};

// ------------------------------------------------------------------------------------------
// Raw vector memory access helpers.
// ------------------------------------------------------------------------------------------
template <class T, int VPT>
__device__ __forceinline__ void load_vec(const T *__restrict__ src, T (&x)[VPT]) {
  static_assert((sizeof(T) * VPT) % 16 == 0, "vector load needs a multiple of 16 bytes");
  constexpr int NV = (int)(sizeof(T) * VPT / 16);
  uint4 v[NV];
  const uint4 *s = reinterpret_cast<const uint4 *>(src);
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = __ldg(s + i);
  memcpy(x, v, sizeof(T) * VPT);
}

template <class T, int VPT>
__device__ __forceinline__ void store_vec(T *__restrict__ dst, const T (&y)[VPT]) {
  constexpr int NV = (int)(sizeof(T) * VPT / 16);
  uint4 v[NV];
  memcpy(v, y, sizeof(T) * VPT);
  uint4 *d = reinterpret_cast<uint4 *>(dst);
#pragma unroll
  for (int i = 0; i < NV; ++i) __stcs(d + i, v[i]);
}

}  // namespace sws
