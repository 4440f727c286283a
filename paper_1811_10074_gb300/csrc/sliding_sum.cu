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
//   prefix-diff    for invertible operators (add mod 2^32, xor): y_p = T_{p+w-1} (-) T_{p-1},
//                  with T the running sum from the tile start (the "recurrent" sliding sums of
//                  Sec. 5), O(1) per output and independent of w.
#include <cstdio>

#include "../../include/sws.h"
#include "common.cuh"
#include "internal.h"

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
  constexpr int PADL = L + NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint32_t *T = reinterpret_cast<uint32_t *>(smem_raw);  // running sums, padded
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

template <class Kern>
cudaError_t set_smem(Kern kern, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <class Op, class Cfg>
cudaError_t launch_op(int variant, const void *in, void *out, uint64_t n, int w, cudaStream_t st) {
  using T = typename Op::T;
  using S = Shape<Cfg, (int)sizeof(T)>;
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
    case SWS_OP_ADD_I32: return launch_op<OpAddI32, Cfg>(L.variant, in, out, n, w, st);
    case SWS_OP_MIN_I32: return launch_op<OpMinI32, Cfg>(L.variant, in, out, n, w, st);
    case SWS_OP_MAX_I32: return launch_op<OpMaxI32, Cfg>(L.variant, in, out, n, w, st);
    case SWS_OP_XOR_I32: return launch_op<OpXorI32, Cfg>(L.variant, in, out, n, w, st);
    case SWS_OP_AFFINE_U32: return launch_op<OpAffineU32, Cfg>(L.variant, in, out, n, w, st);
    case SWS_OP_ADD_F32: return launch_op<OpAddF32, Cfg>(L.variant, in, out, n, w, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

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
