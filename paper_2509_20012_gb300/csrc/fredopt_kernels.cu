// Kernels of the superiorized simultaneous feasibility-seeking loop
// (arXiv 2509.20012, Sec. 2.4.3: Fig. 2 in simultaneous form, Fig. 3, Eq. 2)
// for sm_103a.  Memory-bound sparse work: no tensor cores.
//
//   K1 k_forward     fused Dx / Lx over one shared CSR index stream, 16-byte
//                    streaming loads of col / D / L, x staged in shared
//                    memory by one bulk (TMA) copy, warp per row, rows
//                    assigned to warps in nnz-balanced contiguous ranges;
//                    fused epilogues: objective residual (Eq. 2), line-search
//                    coefficients, FP64 final outputs.
//   K2 k_constraints per-row half-space evaluation and relaxed projection
//                    coefficients (Fig. 2), FP64 norms and divides.
//   K3 k_backward    transposed product over the CSC copy, split into
//                    fixed-size column chunks, one warp per chunk range;
//                    every chunk sum is a fixed-order warp reduction (no
//                    float atomics, deterministic).
//   K3b k_colfinish  per spot: sum of its chunks in order, then the
//                    gradient, or the clip w <- max(0, x + u) (Fig. 2, last
//                    loop); closes the iteration (log entry, k).
//   K4 k_finish      64 blocks, then the last one: deterministic two-level
//                    reduction of the partials and the closed-form
//                    non-ascent trial loop (Fig. 3) in one warp.
//   K5 setup         validation, row gather, quantisation, FP64 moments,
//                    blocked stable transpose (CSR -> CSC) 16 rows a step.
#include "fredopt.h"
#include "fredopt_internal.cuh"

#include <algorithm>

#include <cstdio>
#include <type_traits>

namespace fo {

constexpr unsigned kFull = 0xffffffffu;
// Launch shape and streaming depth (compile-time; the defaults were chosen
// by measurement on GB300).
#ifndef FO_FWD_UNROLL
#define FO_FWD_UNROLL 1
#endif
#ifndef FO_BWD_UNROLL
#define FO_BWD_UNROLL 2
#endif
#ifndef FO_PREFETCH_UNITS
#define FO_PREFETCH_UNITS 1
#endif
#ifndef FO_BWD_MIN_BLOCKS
#define FO_BWD_MIN_BLOCKS 4
#endif
#ifndef FO_FWD_XS
#define FO_FWD_XS 1
#endif
#ifndef FO_FWD_THREADS
#define FO_FWD_THREADS 1024
#endif
constexpr int kFwdThreads = FO_FWD_THREADS;
constexpr int kFwdUnroll = FO_FWD_UNROLL;
#ifndef FO_UNROLL16
#define FO_UNROLL16 2
#endif
#ifndef FO_BWD_UNROLL16
#define FO_BWD_UNROLL16 3
#endif
#ifndef FO_BWD_PP
#define FO_BWD_PP 0
#endif
constexpr int kFwdUnroll16 = FO_UNROLL16;
// Register units (blocks of 128 elements loaded together) of the transposed
// product per pass: FO_BWD_UNROLL16 for the 16-bit projection pass (D and L
// streams), FO_BWD_UNROLL16_G for the 16-bit gradient pass (L stream only),
// FO_BWD_UNROLL_G for the FP32 gradient pass.  The gradient passes carry
// fewer bytes per element, so more of their elements fit in the 64
// registers of a thread.  Clinical plan, per launch (mean of both passes):
// BF16 0.598 -> 0.535 ms, FP32 0.687 -> 0.672 ms against 2/2/2 units.
#ifndef FO_BWD_UNROLL16_G
#define FO_BWD_UNROLL16_G 4
#endif
#ifndef FO_BWD_UNROLL_G
#define FO_BWD_UNROLL_G 3
#endif
// 1: a pass that uses only the L components of the coefficient pairs gathers
// 4 bytes per element instead of the 8-byte pair (fewer registers)
#ifndef FO_BWD_GATHER_Y
#define FO_BWD_GATHER_Y 1
#endif
template <typename VT, bool UD>
__host__ __device__ constexpr int bwd_units() {
  return sizeof(VT) == 4 ? (UD ? FO_BWD_UNROLL : FO_BWD_UNROLL_G) : (UD ? FO_BWD_UNROLL16 : FO_BWD_UNROLL16_G);
}
constexpr bool kBwdPingPong = FO_BWD_PP != 0;
constexpr int kPrefetchUnits = FO_PREFETCH_UNITS;
constexpr int kBwdThreads = 256;
constexpr int kRowThreads = 256;
constexpr int kColThreads = 256;
constexpr int kMbarSpins = FREDOPT_WAIT_POLLS;
// Lane mapping of a block's 128 elements (element of value q of lane l):
//   0 contiguous  4l + q            (16-byte index / FP32 loads per lane)
//   1 strided     32q + l           (one gather instruction reads the
//                                    coefficients of 32 consecutive elements)
//   2 pairs       64(q/2) + 2l + q%2 (4-byte 16-bit loads; 64-element spans)
// The transposed product gathers a coefficient per element; consecutive CSC
// elements of a column are mostly neighbouring voxels, so mappings 1 and 2
// touch fewer L1 sectors per gather instruction.  Mapping 2 measured fastest
// for both value widths (clinical plan, per launch: FP32 0.687 ms against
// 0.707 strided and 0.728 contiguous; BF16 0.598 against 0.644 contiguous
// and 0.676 strided).
#ifndef FO_BWD_LM
#define FO_BWD_LM 2
#endif
#ifndef FO_BWD_LM16
#define FO_BWD_LM16 2
#endif
template <typename VT>
constexpr int kBwdLaneMap = sizeof(VT) == 4 ? FO_BWD_LM : FO_BWD_LM16;
template <int LM>
__device__ __forceinline__ int lane_pos(int lane, int q) {
  return LM == 0 ? lane * 4 + q : LM == 1 ? q * 32 + lane : (q >> 1) * 64 + 2 * lane + (q & 1);
}

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }

template <typename VT> struct VecOf;
template <> struct VecOf<float> { static constexpr int V = 4; };
// 16-bit values: 4 per lane too (8-byte value loads), so a block keeps the
// register footprint of the FP32 block and more blocks fit in a unit
template <> struct VecOf<__nv_bfloat16> { static constexpr int V = 4; };
template <> struct VecOf<__half> { static constexpr int V = 4; };

// 16-byte loads of the streamed arrays.  S = streaming (read once):
// FO_LOAD_KIND 0: ld.global.cs (evict-first in L1 and L2);
//              1: ld.global.L1::no_allocate;
//              2: ld.global.L1::no_allocate with an L2 evict-first policy;
//              3: ld.global.nc.L1::no_allocate.
// Otherwise (data reused across passes while it fits in L2): ld.global.nc.
#ifndef FO_LOAD_KIND
#define FO_LOAD_KIND 0
#endif
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ int4 ld_stream(const int4* p) {
  int4 v;
#if FO_LOAD_KIND == 0
  v = __ldcs(p);
#elif FO_LOAD_KIND == 1
  asm volatile("ld.global.L1::no_allocate.v4.s32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
#elif FO_LOAD_KIND == 2
  asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v4.s32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p), "l"(l2_evict_first_policy()));
#else
  asm volatile("ld.global.nc.L1::no_allocate.v4.s32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
#endif
  return v;
}
template <bool S>
__device__ __forceinline__ int4 ld16(const int4* p) {
  if (S) return ld_stream(p);
  return __ldg(p);
}
template <bool S>
__device__ __forceinline__ uint4 ld16(const uint4* p) {
  if (S) {
    const int4 v = ld_stream(reinterpret_cast<const int4*>(p));
    return make_uint4((unsigned)v.x, (unsigned)v.y, (unsigned)v.z, (unsigned)v.w);
  }
  return __ldg(p);
}

__device__ __forceinline__ void unpack(float, uint4 u, float* o) {
  o[0] = __uint_as_float(u.x);
  o[1] = __uint_as_float(u.y);
  o[2] = __uint_as_float(u.z);
  o[3] = __uint_as_float(u.w);
}
// 16-bit values: 4 per lane in the low 8 bytes (u.x, u.y)
__device__ __forceinline__ void unpack(__nv_bfloat16, uint4 u, float* o) {
  const uint32_t w[2] = {u.x, u.y};
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    o[2 * i] = __uint_as_float(w[i] << 16);
    o[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
}
__device__ __forceinline__ void unpack(__half, uint4 u, float* o) {
  const uint32_t w[2] = {u.x, u.y};
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    __half2 h = *reinterpret_cast<const __half2*>(&w[i]);
    float2 f = __half22float2(h);
    o[2 * i] = f.x;
    o[2 * i + 1] = f.y;
  }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// ---- double-float (double-word) accumulation ----
// A value hi + lo held in two FP32 numbers (|lo| <= ulp(hi) / 2): about 48
// significant bits at FP32 speed.  GB300's FP64 rate is a small fraction of
// its FP32 rate, so the final FP64-class pass accumulates in this form.
// Products are exact (TwoProd with an FMA); additions use the accurate
// double-word sum of Joldes, Muller and Popescu (ACM TOMS 44(2), 2017,
// relative error <= 3 * 2^-48), built from Knuth's TwoSum and Dekker's
// FastTwoSum.  Every operation is an explicitly rounded intrinsic, so the
// compiler cannot fuse or reorder any step.
struct DF {
  float hi, lo;
  __device__ DF() : hi(0.0f), lo(0.0f) {}
  __device__ explicit DF(float v) : hi(v), lo(0.0f) {}
  __device__ DF(float h, float l) : hi(h), lo(l) {}
  __device__ explicit operator double() const { return (double)hi + (double)lo; }
};
__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return DF(s, e);
}
__device__ __forceinline__ DF fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return DF(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ DF df_add(DF x, DF y) {
  const DF s = two_sum(x.hi, y.hi);
  const DF t = two_sum(x.lo, y.lo);
  const DF v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}
// c + a * b: the accumulation step of the streaming core for each accumulator type
__device__ __forceinline__ float acc_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ DF acc_fma(float a, float b, DF c) {
  const float p = __fmul_rn(a, b);
  return df_add(c, DF(p, __fmaf_rn(a, b, -p)));  // a * b = p + (a * b - p) exactly
}
template <>
__device__ __forceinline__ DF warp_sum(DF v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const DF w(__shfl_xor_sync(kFull, v.hi, o), __shfl_xor_sync(kFull, v.lo, o));
    v = df_add(v, w);
  }
  return v;
}

// ---- mbarrier + bulk copy (TMA engine, non-tensor form) ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// bulk prefetch of [src, src + bytes) into L2 (TMA engine; no registers or
// shared memory; bytes a multiple of 16, src 16-byte aligned)
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
// bounded wait on phase `parity`; true when the phase completed
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int max_spins) {
  const uint32_t a = smem_u32(bar);
  for (int i = 0; i < max_spins; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// ------------------------------------------------------------------ streaming core

// One block of the index stream and the two value streams, 4 elements per
// lane: 16 bytes of 32-bit indices (8 bytes of 16-bit ones, in c0.x, c0.y)
// and 16 bytes of FP32 values (8 bytes of 16-bit ones, in the low half).
template <typename VT>
struct Blk {
  int4 c0;      // 4 indices
  uint4 a, b;   // values of the two streams
  int hb;       // block header of based 16-bit indices (see BlockBase)
};

// Based 16-bit indices: the stream is cut into aligned blocks of 128
// elements; block k holds uint16 offsets from hdr[k] >= 0, or, when its
// indices span 65536 or more, hdr[k] = -1 - j and its 128 int32 indices are
// ovf[128 j .. 128 j + 127].
struct BlockBase {
  const int32_t* hdr;
  const int32_t* ovf;
  int32_t n_ovf;
};

// Checked builds (FO_CHECKED=1, a debug aid in place of a memory checker):
// the streaming kernels check every tile's element range against the
// allocated length, every gathered index against its table and every
// overflow slot, record a failure in bit 1 of the error word (reported as
// FREDOPT_ERR_PATTERN) and skip the access.  Results are otherwise
// bit-identical to the default build.
#ifndef FO_CHECKED
#define FO_CHECKED 0
#endif
struct SegCheck {
  int64_t n_elems;
  int* err;
};

template <bool S>
__device__ __forceinline__ int4 ld_idx(const int32_t* p) {
  return ld16<S>(reinterpret_cast<const int4*>(p));
}
template <bool S>
__device__ __forceinline__ int4 ld_idx(const uint16_t* p) {  // 4 x 16-bit = 8 bytes
  uint2 v;
  if (S) v = __ldcs(reinterpret_cast<const uint2*>(p));
  else v = __ldg(reinterpret_cast<const uint2*>(p));
  return make_int4((int)v.x, (int)v.y, 0, 0);
}
__device__ __forceinline__ void unpack_idx(int32_t, int4 c, int* cs) {
  cs[0] = c.x; cs[1] = c.y; cs[2] = c.z; cs[3] = c.w;
}
__device__ __forceinline__ void unpack_idx(uint16_t, int4 c, int* cs) {  // little-endian halves
  cs[0] = (int)((uint32_t)c.x & 0xffffu); cs[1] = (int)((uint32_t)c.x >> 16);
  cs[2] = (int)((uint32_t)c.y & 0xffffu); cs[3] = (int)((uint32_t)c.y >> 16);
}

template <bool S>
__device__ __forceinline__ uint4 ld_vals(const float* p) {
  return ld16<S>(reinterpret_cast<const uint4*>(p));
}
template <bool S, typename H>
__device__ __forceinline__ uint4 ld_vals(const H* p) {  // 4 x 16-bit = 8 bytes
  uint2 v;
  if (S) v = __ldcs(reinterpret_cast<const uint2*>(p));
  else v = __ldg(reinterpret_cast<const uint2*>(p));
  return make_uint4(v.x, v.y, 0u, 0u);
}

template <typename VT, bool S, bool USE_A, typename IT>
__device__ __forceinline__ void load_blk(Blk<VT>& k, const IT* idx, const VT* Av, const VT* Bv,
                                         int64_t p) {
  k.c0 = ld_idx<S>(idx + p);
  if (USE_A) k.a = ld_vals<S>(Av + p);
  k.b = ld_vals<S>(Bv + p);
}

// Lane-strided block: elements p, p + 32, p + 64, p + 96 (p = block start +
// lane), packed into the same registers as load_blk's 4 consecutive ones.
template <bool S, typename T>
__device__ __forceinline__ T ld1(const T* p) {
  if (S) return __ldcs(p);
  return __ldg(p);
}
template <bool S, typename T>
__device__ __forceinline__ uint4 ld_strided(const T* p) {
  if constexpr (sizeof(T) == 4) {
    const unsigned* q = reinterpret_cast<const unsigned*>(p);
    return make_uint4(ld1<S>(q), ld1<S>(q + 32), ld1<S>(q + 64), ld1<S>(q + 96));
  } else {
    const unsigned short* q = reinterpret_cast<const unsigned short*>(p);
    const uint32_t e0 = ld1<S>(q), e1 = ld1<S>(q + 32), e2 = ld1<S>(q + 64), e3 = ld1<S>(q + 96);
    return make_uint4(e0 | (e1 << 16), e2 | (e3 << 16), 0u, 0u);
  }
}
template <typename VT, bool S, bool USE_A, typename IT>
__device__ __forceinline__ void load_blk_strided(Blk<VT>& k, const IT* idx, const VT* Av, const VT* Bv,
                                                 int64_t p) {
  const uint4 c = ld_strided<S>(idx + p);
  k.c0 = make_int4((int)c.x, (int)c.y, (int)c.z, (int)c.w);
  if (USE_A) k.a = ld_strided<S>(Av + p);
  k.b = ld_strided<S>(Bv + p);
}
// Pair block: elements p, p + 1, p + 64, p + 65 (p = block start + 2 lane).
template <bool S, typename T>
__device__ __forceinline__ uint4 ld_pairs(const T* p) {
  if constexpr (sizeof(T) == 4) {
    const uint2* q = reinterpret_cast<const uint2*>(p);
    const uint2 a = ld1<S>(q), b = ld1<S>(q + 32);
    return make_uint4(a.x, a.y, b.x, b.y);
  } else {
    const unsigned* q = reinterpret_cast<const unsigned*>(p);
    return make_uint4(ld1<S>(q), ld1<S>(q + 32), 0u, 0u);
  }
}
template <typename VT, bool S, bool USE_A, typename IT>
__device__ __forceinline__ void load_blk_pairs(Blk<VT>& k, const IT* idx, const VT* Av, const VT* Bv,
                                               int64_t p) {
  const uint4 c = ld_pairs<S>(idx + p);
  k.c0 = make_int4((int)c.x, (int)c.y, (int)c.z, (int)c.w);
  if (USE_A) k.a = ld_pairs<S>(Av + p);
  k.b = ld_pairs<S>(Bv + p);
}

// Streams the elements [ptr[r0], ptr[r1]) of one warp as consecutive blocks
// of 32*V elements (lane l holds elements l*V .. l*V+V-1 of a block; every
// load is 16 bytes; the next unit of U blocks is in flight while the
// current one is consumed) and splits the stream into the segments
// [ptr[r], ptr[r+1]).  For element i with index c: sA += A_i * g(c).x and
// sB += B_i * g(c).y.  A finished segment is summed over the warp in a fixed
// butterfly; lane (r - base) keeps it; every 32 segments (and at the end)
// flush(base, count, mine_A, mine_B) runs with lane j < count owning segment
// base + j.  Deterministic: the split depends only on ptr, r0, r1.  The index
// stream is int32 or uint16 (IT), the latter plain or BASED on per-block
// headers (bb); the sums do not depend on the encoding.  LM: lane mapping
// of a block's elements (lane_pos; mapping 0 is the one described above).
// The arrays must be readable (zero padded) up to
// round_up(ptr[r1], 32*V) + U*32*V elements (a prefetch starts below ptr[r1]
// and covers U*32*V elements, within the same bound).
template <typename VT, typename Acc, bool S, bool USE_A, int U, bool BASED = false, int LM = 0,
          typename IT, class Gather, class Flush, int PF = kPrefetchUnits, bool PP = false>
__device__ __forceinline__ void stream_segments(const IT* __restrict__ idx,
                                                const VT* __restrict__ Av, const VT* __restrict__ Bv,
                                                const int64_t* __restrict__ ptr, int64_t r0, int64_t r1,
                                                int lane, Gather gather, Flush flush,
                                                BlockBase bbase = BlockBase{nullptr, nullptr, 0},
                                                SegCheck chk = SegCheck{0, nullptr}) {
  constexpr int V = VecOf<VT>::V;
  constexpr int BLK = 32 * V;
  constexpr int UB = U * BLK;
  static_assert(!BASED || (BLK == 128 && sizeof(IT) == 2), "based indices: 16-bit, 128-element blocks");
  if (r0 >= r1) return;
#if FO_CHECKED
  if (chk.err) {
    const int64_t p0 = ptr[r0], p1 = ptr[r1];
    if (p0 < 0 || p1 < p0 || (p1 + BLK - 1) / BLK * BLK + UB > chk.n_elems) {
      if (lane == 0) atomicOr(chk.err, 2);
      return;
    }
  }
#endif
  // 32-bit offsets from the block-aligned start of the warp's range (a
  // warp's range is far below 2^31 elements)
  const int64_t start = ptr[r0] & ~(int64_t)(BLK - 1);
  const int32_t* __restrict__ hdr = BASED ? bbase.hdr + start / BLK : nullptr;
  idx += start;
  if (USE_A) Av += start;
  Bv += start;
  const int pb = (int)(ptr[r0] - start), pe = (int)(ptr[r1] - start);
  const int nrows = (int)(r1 - r0);
  int row = 0, base = 0;  // relative to r0
  int ends = (lane < nrows) ? (int)(ptr[r0 + 1 + lane] - start) : pe;
  int e_cur = __shfl_sync(kFull, ends, 0);
  Acc sA{}, sB{}, myA{}, myB{};
  bool done = false;

  // consume the U blocks of one unit starting at offset b
  auto consume = [&](const Blk<VT>* unit, int b) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (done) return;
      const int bb = b + u * BLK;
      int cs[V];
      float av[V], bv[V];
      unpack_idx(IT(), unit[u].c0, cs);
      if (BASED) {
        const int hb = unit[u].hb;
        if (hb >= 0) {
#pragma unroll
          for (int q = 0; q < V; ++q) cs[q] += hb;
        } else {  // wide block: its int32 indices from the overflow table
          int slot = -1 - hb;
#if FO_CHECKED
          if (slot >= bbase.n_ovf) {
            if (chk.err) atomicOr(chk.err, 2);
            slot = 0;
          }
#endif
          const int32_t* ov = bbase.ovf + (int64_t)slot * BLK;
          if (LM == 1) {
#pragma unroll
            for (int q = 0; q < V; ++q) cs[q] = __ldg(ov + q * 32 + lane);
          } else if (LM == 2) {
            const int2 w0 = __ldg(reinterpret_cast<const int2*>(ov) + lane);
            const int2 w1 = __ldg(reinterpret_cast<const int2*>(ov + 64) + lane);
            cs[0] = w0.x; cs[1] = w0.y; cs[2] = w1.x; cs[3] = w1.y;
          } else {
            const int4 w = __ldg(reinterpret_cast<const int4*>(ov) + lane);
            cs[0] = w.x; cs[1] = w.y; cs[2] = w.z; cs[3] = w.w;
          }
        }
      }
      if (USE_A) unpack(VT(), unit[u].a, av);
      unpack(VT(), unit[u].b, bv);
      float2 gv[V];
#pragma unroll
      for (int q = 0; q < V; ++q) gv[q] = gather(cs[q]);
      int lo = bb > pb ? bb : pb;
      while (true) {
        const int hi = e_cur < bb + BLK ? e_cur : bb + BLK;
#pragma unroll
        for (int q = 0; q < V; ++q) {
          const int e = bb + lane_pos<LM>(lane, q);
          if (e >= lo && e < hi) {
            if (USE_A) sA = acc_fma(av[q], gv[q].x, sA);
            sB = acc_fma(bv[q], gv[q].y, sB);
          }
        }
        if (e_cur > bb + BLK) break;  // the open segment continues in the next block
        const Acc tA = warp_sum(sA), tB = warp_sum(sB);
        sA = Acc{}; sB = Acc{};
        if (lane == row - base) { myA = tA; myB = tB; }
        ++row;
        if (row - base == 32 || row == nrows) {
          flush(r0 + base, row - base, myA, myB);
          myA = Acc{}; myB = Acc{};
          if (row == nrows) { done = true; return; }
          base = row;
          ends = (base + lane < nrows) ? (int)(ptr[r0 + base + 1 + lane] - start) : pe;
        }
        e_cur = __shfl_sync(kFull, ends, row - base);
        lo = hi;
        if (lo >= bb + BLK) break;
      }
    }
  };
  // lane 0 asks the TMA engine to bring the unit PF units ahead into L2, so
  // the demand loads of the warp mostly wait on L2 rather than DRAM
  auto prefetch_unit = [&](int q) {
    if (PF > 0 && lane == 0 && q < pe) {
      bulk_prefetch_l2(idx + q, (uint32_t)(UB * sizeof(IT)));
      if (USE_A) bulk_prefetch_l2(Av + q, (uint32_t)(UB * sizeof(VT)));
      bulk_prefetch_l2(Bv + q, (uint32_t)(UB * sizeof(VT)));
    }
  };
  auto load_unit = [&](Blk<VT>* unit, int b) {
    prefetch_unit(b + PF * UB);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (LM == 1) load_blk_strided<VT, S, USE_A, IT>(unit[u], idx, Av, Bv, b + u * BLK + lane);
      else if (LM == 2) load_blk_pairs<VT, S, USE_A, IT>(unit[u], idx, Av, Bv, b + u * BLK + 2 * lane);
      else load_blk<VT, S, USE_A, IT>(unit[u], idx, Av, Bv, b + u * BLK + lane * V);
      if (BASED) unit[u].hb = __ldg(hdr + (b + u * BLK) / BLK);
    }
  };

  int b = 0;
#pragma unroll
  for (int k = 1; k < PF; ++k) prefetch_unit(b + k * UB);
  if (PP) {
    // ping-pong between two register units: while one is consumed the loads
    // of the other are in flight (no register copies of pending loads)
    Blk<VT> ua[U], ub[U];
    load_unit(ua, b);
    while (true) {
      if (b + UB < pe) load_unit(ub, b + UB);
      consume(ua, b);
      if (done) break;
      b += UB;
      if (b + UB < pe) load_unit(ua, b + UB);
      consume(ub, b);
      if (done) break;
      b += UB;
    }
  } else {
    // one register unit: its U blocks are loaded together, then consumed;
    // latency is hidden by the other warps of the SM
    Blk<VT> ua[U];
    while (!done) {
      load_unit(ua, b);
      consume(ua, b);
      b += UB;
    }
  }
}

// ------------------------------------------------------------------ K1

// Objective of one row (Eq. 2 terms of the structures the voxel is in):
// f_i = sum w (q - T)^2 ; residual rD = sum_DOSE 2w(Dx - T), rL = sum_CDL 2wc(cLx - T).
__device__ __forceinline__ void row_objective(const Tables& t, uint32_t m, double Dx, double Lx,
                                              double& f, double& rD, double& rL) {
  f = 0.0; rD = 0.0; rL = 0.0;
  for (int i = 0; i < t.n_obj; ++i) {
    const ObjEntry& o = t.obj[i];
    if (!((m >> o.bit) & 1u)) continue;
    if (o.q == 0) {
      const double d = Dx - o.target;
      f += o.weight * d * d;
      rD += 2.0 * o.weight * d;
    } else {
      const double d = t.c * Lx - o.target;
      f += o.weight * d * d;
      rL += 2.0 * o.weight * t.c * d;
    }
  }
}

template <typename IT> __device__ __forceinline__ const IT* fwd_col(const FwdArgs& a);
template <> __device__ __forceinline__ const int32_t* fwd_col<int32_t>(const FwdArgs& a) { return a.col; }
template <> __device__ __forceinline__ const uint16_t* fwd_col<uint16_t>(const FwdArgs& a) { return a.col16; }

// Fused Dx, Lx over the warp's nonempty rows [warp_row[2w], warp_row[2w+1]).
// IT: width of the column indices (uint16_t only with x in shared memory).
template <typename VT, int EPI, bool XS, bool S, typename IT>
__global__ void __launch_bounds__(kFwdThreads, 1024 / kFwdThreads) k_forward(FwdArgs a, Tables t) {
  extern __shared__ __align__(128) unsigned char smem[];
  using Acc = typename std::conditional<EPI == EPI_FINAL, DF, float>::type;
  const float* __restrict__ x = a.x;
  if (XS) {
    float* xs = reinterpret_cast<float*>(smem);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + (size_t)a.n_x_pad * sizeof(float));
    if (threadIdx.x == 0) {
      mbar_init(bar, 1);
      fence_mbar_init();
    }
    __syncthreads();
    const uint32_t bytes = (uint32_t)a.n_x_pad * (uint32_t)sizeof(float);
    if (threadIdx.x == 0) {
      mbar_expect_tx(bar, bytes);
      bulk_g2s(xs, a.x, bytes, bar);
    }
    if (!mbar_wait(bar, 0, kMbarSpins)) {
      if (threadIdx.x == 0) atomicOr(&a.st->err, 1);
      mbar_wait(bar, 0, kMbarSpins);  // let the copy in flight land before leaving
      return;
    }
    x = xs;
  }
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  // Tiles: a warp streams tile `warp` (static schedule) or claims tiles in
  // order from a counter (a.sched[0]) until none is left, so that faster SMs
  // stream more of them; a.sched[1] counts the warps that are done and the
  // last one resets both counters for the next launch.  A tile's sums do not
  // depend on which warp streams it.
  auto claim = [&]() -> int {
    unsigned j = 0;
    if (lane == 0) j = atomicAdd(&a.sched[0], 1u);
    return (int)__shfl_sync(kFull, j, 0);
  };
  int job = a.sched ? claim() : warp;
  const VT* __restrict__ Dv = reinterpret_cast<const VT*>(a.Dv);
  const VT* __restrict__ Lv = reinterpret_cast<const VT*>(a.Lv);
  double acc0 = 0.0, acc1 = 0.0;  // per-lane partials of the epilogue reductions
  auto gather = [&](int c) {
#if FO_CHECKED
    if ((unsigned)c >= (unsigned)a.n_x) {
      atomicOr(&a.st->err, 2);
      c = 0;
    }
#endif
    const float v = x[c];
    return make_float2(v, v);
  };
  auto flush = [&](int64_t base, int cnt, Acc myD, Acc myL) {
    if (lane >= cnt) return;
    const int64_t r = base + lane;
    const double sd = a.sD ? (double)a.sD[r] : 1.0;
    const double sl = a.sL ? (double)a.sL[r] : 1.0;
    if (EPI == EPI_FINAL) {
      const double Dx = (double)myD * sd, Lx = (double)myL * sl;
      a.y64[r] = make_double2(Dx, Lx);
      const int64_t v = a.voxel ? a.voxel[r] : r;
      if (a.dose_out) a.dose_out[v] = (float)Dx;
      if (a.letd_out) a.letd_out[v] = Dx > 0.0 ? (float)(Lx / Dx) : 0.0f;
    } else {
      const float Dx = (float)((double)myD * sd), Lx = (float)((double)myL * sl);
      a.y[r] = make_float2(Dx, Lx);
      if (EPI == EPI_OBJ) {
        double f, rD, rL;
        row_objective(t, a.mask[r], Dx, Lx, f, rD, rL);
        a.r_out[r] = make_float2((float)(rD * sd), (float)(rL * sl));
        acc0 += f;
      } else if (EPI == EPI_BC) {
        // B' = sum w (q(x) - T) q(g) = 1/2 (rD Dg + rL Lg); C' = sum w q(g)^2
        const float2 rin = a.r_in[r];  // already multiplied by the row scales
        acc0 += 0.5 * ((double)rin.x * (double)myD + (double)rin.y * (double)myL);
        const uint32_t m = a.mask[r];
        double PD = 0.0, PL = 0.0;
        for (int i = 0; i < t.n_obj; ++i) {
          if (!((m >> t.obj[i].bit) & 1u)) continue;
          if (t.obj[i].q == 0) PD += t.obj[i].weight;
          else PL += t.obj[i].weight;
        }
        acc1 += PD * (double)Dx * (double)Dx + PL * t.c * t.c * (double)Lx * (double)Lx;
      }
    }
  };
  while (job < a.n_warps) {
    const int64_t r0 = a.warp_row[2 * job], r1 = a.warp_row[2 * job + 1];
    acc0 = 0.0;
    acc1 = 0.0;
    stream_segments<VT, Acc, S, true, (sizeof(VT) == 4 ? kFwdUnroll : kFwdUnroll16)>(
        fwd_col<IT>(a), Dv, Lv, a.rp, r0, r1, lane, gather, flush, BlockBase{nullptr, nullptr, 0},
        SegCheck{a.n_elems, FO_CHECKED ? &a.st->err : nullptr});
    if (EPI == EPI_OBJ || EPI == EPI_BC) {  // partials per tile, summed later in tile order
      const double s0 = warp_sum(acc0), s1 = warp_sum(acc1);
      if (lane == 0) {
        a.part[job] = s0;
        if (EPI == EPI_BC) a.part[a.n_warps + job] = s1;
      }
    }
    if (!a.sched) break;
    job = claim();
  }
  if (a.sched && lane == 0) {
    __threadfence();
    const unsigned total = (gridDim.x * blockDim.x) >> 5;
    if (atomicAdd(&a.sched[1], 1u) == total - 1) {
      a.sched[0] = 0u;
      a.sched[1] = 0u;
    }
  }
}



// ------------------------------------------------------------------ K3

// Chunk sums of the transposed product: chunk c = nonzeros [chunk_ptr[c],
// chunk_ptr[c+1]) of one column; sum_i D_ij coef_i.x + L_ij coef_i.y.
// NB: row indices as based 16-bit offsets (BwdArgs.row16/hdr/ovf).
template <typename VT, bool S, bool UD, bool NB>
__global__ void __launch_bounds__(kBwdThreads, FO_BWD_MIN_BLOCKS) k_backward(BwdArgs a) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const VT* __restrict__ Dv = reinterpret_cast<const VT*>(a.Dv);
  const VT* __restrict__ Lv = reinterpret_cast<const VT*>(a.Lv);
  const float2* __restrict__ cf = a.coef;
  auto gather = [&](int r) {
#if FO_CHECKED
    if ((uint64_t)(int64_t)r >= (uint64_t)a.n_rows) {
      atomicOr(&a.st->err, 2);
      r = 0;
    }
#endif
    if (!UD && FO_BWD_GATHER_Y) return make_float2(0.0f, __ldg(&cf[r].y));
    return __ldg(&cf[r]);
  };
  float* out = a.chunk_sum;
  auto flush = [&](int64_t base, int cnt, float mA, float mB) {
    if (lane < cnt) out[base + lane] = UD ? mA + mB : mB;
  };
  // tiles of column chunks, static (tile = warp) or claimed from a counter as
  // in the forward product; a chunk's sum does not depend on its warp
  auto claim = [&]() -> int {
    unsigned j = 0;
    if (lane == 0) j = atomicAdd(&a.sched[0], 1u);
    return (int)__shfl_sync(kFull, j, 0);
  };
  int job = a.sched ? claim() : warp;
  while (job < a.n_warps) {
    if (NB)
      stream_segments<VT, float, S, UD, bwd_units<VT, UD>(), true, kBwdLaneMap<VT>,
                      uint16_t, decltype(gather), decltype(flush), kPrefetchUnits, kBwdPingPong>(
          a.row16, Dv, Lv, a.chunk_ptr, a.warp_chunk[job], a.warp_chunk[job + 1], lane, gather, flush,
          BlockBase{a.hdr, a.ovf, a.n_ovf}, SegCheck{a.n_elems, FO_CHECKED ? &a.st->err : nullptr});
    else
      stream_segments<VT, float, S, UD, bwd_units<VT, UD>(), false, kBwdLaneMap<VT>,
                      int32_t, decltype(gather), decltype(flush), kPrefetchUnits, kBwdPingPong>(
          a.row, Dv, Lv, a.chunk_ptr, a.warp_chunk[job], a.warp_chunk[job + 1], lane, gather, flush,
          BlockBase{nullptr, nullptr, 0}, SegCheck{a.n_elems, FO_CHECKED ? &a.st->err : nullptr});
    if (!a.sched) break;
    job = claim();
  }
  if (a.sched && lane == 0) {
    __threadfence();
    const unsigned total = (gridDim.x * blockDim.x) >> 5;
    if (atomicAdd(&a.sched[1], 1u) == total - 1) {
      a.sched[0] = 0u;
      a.sched[1] = 0u;
    }
  }
}

// ------------------------------------------------------------------ block reductions

// Block reductions of one double per thread (blockDim = 256), in a fixed
// order: a warp butterfly, then thread 0 adds the 8 warp results in warp
// order.  GB300 runs FP64 at a small fraction of its FP32 rate, and every
// FP64 warp instruction costs the same however few of its lanes are active,
// so: a warp whose lanes all hold zero skips its butterfly (its sum is that
// zero), maxima are of non-negative doubles, whose bit patterns order as
// signed 64-bit integers (integer compares), and counts held in doubles are
// added as 64-bit integers (exact, so in any order).
__device__ __forceinline__ double warp_sum_nz(double v) {
  if (!__any_sync(kFull, v != 0.0)) return v;
  return warp_sum(v);
}
__device__ __forceinline__ long long warp_max_bits(long long b) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long c = __shfl_xor_sync(kFull, b, o);
    b = c > b ? c : b;
  }
  return b;
}
__device__ __forceinline__ double warp_max_nonneg(double v) {
  return __longlong_as_double(warp_max_bits(__double_as_longlong(v)));
}
__device__ __forceinline__ long long warp_isum(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
// red: at least 9 doubles of shared memory; every thread returns the result
__device__ __forceinline__ double block_sum256(double v, double* red) {
  v = warp_sum_nz(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = red[0];
#pragma unroll
    for (int w = 1; w < 8; ++w) r += red[w];
    red[8] = r;
  }
  __syncthreads();
  // red[8] is rewritten only after the next call's first barrier, which
  // every thread reaches after this read
  return red[8];
}
// v >= 0
__device__ __forceinline__ double block_max256(double v, double* red) {
  long long* rb = reinterpret_cast<long long*>(red);
  const long long b = warp_max_bits(__double_as_longlong(v));
  if ((threadIdx.x & 31) == 0) rb[threadIdx.x >> 5] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long r = rb[0];
#pragma unroll
    for (int w = 1; w < 8; ++w) r = rb[w] > r ? rb[w] : r;
    rb[8] = r;
  }
  __syncthreads();
  return __longlong_as_double(rb[8]);
}
// integers held in doubles (|v| < 2^53), added exactly
__device__ __forceinline__ double block_count256(long long v, double* red) {
  long long* rb = reinterpret_cast<long long*>(red);
  v = warp_isum(v);
  if ((threadIdx.x & 31) == 0) rb[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long r = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) r += rb[w];
    rb[8] = r;
  }
  __syncthreads();
  return (double)rb[8];
}
// Sum of n doubles in a fixed order (strided per thread, then block_sum256).
__device__ __forceinline__ double block_sum_array(const double* p, int n, double* red) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) v += p[i];
  return block_sum256(v, red);
}
// p[i] >= 0
__device__ __forceinline__ double block_max_array(const double* p, int n, double* red) {
  long long v = 0;
  for (int i = threadIdx.x; i < n; i += 256) {
    const long long b = __double_as_longlong(p[i]);
    v = b > v ? b : v;
  }
  return block_max256(__longlong_as_double(v), red);
}
__device__ __forceinline__ double block_count_array(const double* p, int n, double* red) {
  long long v = 0;
  for (int i = threadIdx.x; i < n; i += 256) v += (long long)p[i];
  return block_count256(v, red);
}

// ------------------------------------------------------------------ K3b

// The end of an iteration (block-wide): its log entry (violated rows and
// largest violation from the constraint partials, the solve state written by
// the scalar finish) and k <- k + 1.
__device__ __forceinline__ void close_iteration(const ColArgs& a, double* red) {
  const double nviol = block_count_array(a.k2part + a.k2_blocks, a.k2_blocks, red);
  const double mxv = block_max_array(a.k2part + 2 * a.k2_blocks, a.k2_blocks, red);
  if (threadIdx.x == 0) {
    DevState* st = a.st;
    if (st->log_cap > 0) {
      LogEntry e;
      e.k = st->k;
      e.s = st->s;
      e.accepted = st->accepted;
      e.n_violated = (int)nviol;
      e.beta = st->beta_acc;
      e.f_start = st->f_start;
      e.f_end = st->f_cur;
      e.gnorm = st->gnorm;
      e.max_violation = mxv;
      a.log[st->k % st->log_cap] = e;
    }
    st->k += 1;
  }
}

template <int MODE>
__global__ void __launch_bounds__(kColThreads) k_colfinish(ColArgs a) {
  __shared__ double red[kColThreads];
  __shared__ double sh_scale;
  __shared__ bool sh_last;
  // COL_PROJ with log_block: the launch's last block closes the iteration,
  // concurrently with the others (nothing else in the launch reads k), and
  // the other blocks split the columns
  const int nb = (int)gridDim.x - (MODE == COL_PROJ ? a.log_block : 0);
  if (MODE == COL_PROJ && a.log_block && (int)blockIdx.x == nb) {
    close_iteration(a, red);
    return;
  }
  double scale = a.scale;  // COL_PROJ with has_scale: lam ps / W from the host
  if (MODE == COL_PROJ && !a.has_scale) {
    double W = a.W_all;
    if (a.norm == 1) W = block_sum_array(a.k2part, a.k2_blocks, red);
    if (threadIdx.x == 0) {
      const double ps = a.in_solve ? (a.st->eta == 1.0 ? 1.0 : pow(a.st->eta, (double)a.st->k)) : a.prio_scale;
      sh_scale = W > 0.0 ? a.lam * ps / W : 0.0;
    }
    __syncthreads();
    scale = sh_scale;
  }
  const double coef = (MODE == COL_PROJ && a.use_coef) ? a.st->coef : 0.0;
  const int per = (a.n + nb - 1) / nb;
  const int j0 = blockIdx.x * per, j1 = min(a.n, j0 + per);
  double acc = 0.0;
  for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
    float s = 0.0f;
    if (a.use_u) {
      // the chunk sums of the column in chunk order (loads unrolled ahead of
      // the sequential additions)
      const int c1 = a.col_chunk[j + 1];
#pragma unroll 8
      for (int c = a.col_chunk[j]; c < c1; ++c) s += __ldcg(&a.chunk_sum[c]);
    }
    if (MODE == COL_OUT) {
      a.out[j] = s;
    } else if (MODE == COL_GRAD) {
      a.out[j] = s;
      acc += (double)s * (double)s;
    } else {
      double xj = (double)a.w[j];
      if (a.use_coef) xj += coef * (double)a.g[j];
      const double wn = xj + scale * (double)s;
      a.w[j] = wn > 0.0 ? (float)wn : 0.0f;
    }
  }
  if (MODE == COL_GRAD) {
    acc = block_sum256(acc, red);
    if (threadIdx.x == 0) a.part[blockIdx.x] = acc;
  }
  if (MODE == COL_PROJ && a.in_solve && !a.log_block) {
    // the last block to finish closes the iteration: log entry, k <- k + 1
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned prev = atomicAdd(&a.st->done, 1u);
      sh_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (sh_last) {
      __threadfence();
      close_iteration(a, red);
      if (threadIdx.x == 0) a.st->done = 0u;
    }
  }
}

// ------------------------------------------------------------------ K2

__global__ void __launch_bounds__(kRowThreads) k_constraints(ConArgs a, Tables t) {
  // block b evaluates a contiguous slice of the rows: of [r0, n_hot), or of
  // the listed rows
  const int64_t lo = a.rows ? 0 : a.r0, hi = a.rows ? a.n_list : a.n_hot;
  const int64_t per = (hi - lo + gridDim.x - 1) / gridDim.x;
  const int64_t j0 = lo + (int64_t)blockIdx.x * per;
  const int64_t j1 = min(hi, j0 + per);
  const double coef = a.use_coef ? a.st->coef : 0.0;
  double psum = 0.0, mx = 0.0, preach = 0.0;
  long long nv = 0;
  for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
    const int64_t i = a.rows ? a.rows[j] : j;
    const uint32_t m = a.mask[i];
    float2 out = make_float2(0.f, 0.f);
    if (m) {
      const float2 w2 = a.yw[i];
      double xd = w2.x, xl = w2.y;
      if (a.use_coef) {
        const float2 g2 = a.yg[i];
        xd += coef * (double)g2.x;
        xl += coef * (double)g2.y;
      }
      double gD = 0.0, gL = 0.0;
      for (int q = 0; q < t.n_con; ++q) {
        const ConEntry& c = t.con[q];
        if (!((m >> c.bit) & 1u)) continue;
        double v, n2, b;
        const int fam = c.kind >> 1;  // 0 dose, 1 cDL, 2 LETd
        if (fam == 0) {
          v = xd; n2 = a.dd[i]; b = c.bound;
        } else if (fam == 1) {
          v = t.c * xl; n2 = t.c * t.c * a.ll[i]; b = c.bound;
        } else {
          v = xl - c.bound * xd;
          n2 = a.ll[i] - 2.0 * c.bound * a.dl[i] + c.bound * c.bound * a.dd[i];
          b = 0.0;
        }
        if (!(n2 > 0.0)) continue;  // unreachable row
        preach += c.prio;
        const bool upper = (c.kind & 1) != 0;
        const double viol = upper ? v - b : b - v;
        if (viol > 0.0) {
          const double tt = c.prio * (b - v) / n2;
          if (fam == 0) gD += tt;
          else if (fam == 1) gL += t.c * tt;
          else { gD -= c.bound * tt; gL += tt; }
          psum += c.prio;
          nv += 1;
          const double vu = (fam == 2) ? (xd > 0.0 ? viol / xd : 0.0) : viol;  // LETd in keV/um
          mx = vu > mx ? vu : mx;
        }
      }
      const double sd = a.sD ? (double)a.sD[i] : 1.0;
      const double sl = a.sL ? (double)a.sL[i] : 1.0;
      out = make_float2((float)(gD * sd), (float)(gL * sl));
    }
    a.gam[i] = out;
  }
  // the block's two sums, its violated-row count and its largest violation
  // (>= 0): warp reductions (the FP64 butterflies skipped by warps without
  // violated or reachable rows), then the warp results in warp order
  __shared__ double wred[3][kRowThreads / 32];
  __shared__ long long wcnt[kRowThreads / 32];
  psum = warp_sum_nz(psum);
  preach = warp_sum_nz(preach);
  nv = warp_isum(nv);
  mx = warp_max_nonneg(mx);
  if ((threadIdx.x & 31) == 0) {
    const int wi = threadIdx.x >> 5;
    wred[0][wi] = psum;
    wred[1][wi] = preach;
    wred[2][wi] = mx;
    wcnt[wi] = nv;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    const int k = threadIdx.x;
    double t;
    if (k == 1) {
      long long c = 0;
#pragma unroll
      for (int w = 0; w < kRowThreads / 32; ++w) c += wcnt[w];
      t = (double)c;
    } else if (k == 2) {
      long long b = 0;
#pragma unroll
      for (int w = 0; w < kRowThreads / 32; ++w) {
        const long long x = __double_as_longlong(wred[2][w]);
        b = x > b ? x : b;
      }
      t = __longlong_as_double(b);
    } else {
      const int src = k == 0 ? 0 : 1;
      t = wred[src][0];
#pragma unroll
      for (int w = 1; w < kRowThreads / 32; ++w) t += wred[src][w];
    }
    // partial slices: sum of priorities of violated rows, violated rows,
    // largest violation, sum of priorities of reachable rows
    a.part[k * gridDim.x + blockIdx.x] = t;
  }
}

// ------------------------------------------------------------------ K4

// The partial sums (one per forward tile: tens of thousands) are added in
// two fixed levels: every CTA sums one slice of each array, and the last CTA
// to finish adds the slice sums in order and runs the trial loop.  GB300's
// FP64 rate is low and an FP64 warp instruction costs the same with one
// active lane or 32, so each sum is laid out to need few of them: within a
// CTA, warps 2k and 2k + 1 add array k (lane l of warp 2k + h takes the
// elements 64 t + 32 h + l of the slice), each warp's lanes by a butterfly,
// the two warps' results in warp order; the last CTA adds the 64 slice sums
// of array k in warp k.  The solve state and the first trial steps are
// loaded at the start, so that the last CTA's chain of dependent loads is
// short.
__global__ void __launch_bounds__(256) k_finish(int step, const double* part_f, int nf,
                                                const double* part_bc, int nbc, const double* part_g,
                                                int ng, DevState* st, double* stage, const double* btab,
                                                long long n_btab) {
  __shared__ double wred[4][2];
  __shared__ double tot_sh[4];
  __shared__ bool sh_last;
  const int G = gridDim.x, b = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // state read by the last CTA (written only by it, at its end, in this kernel)
  const long long s0 = st->s;
  const int max_trials = st->max_trials;
  const int grad_normalize = st->grad_normalize;
  const double f_empty = st->f_empty;
  double beta_pre = 0.0;  // step of trial `lane` (first round)
  if (wid == 0 && lane < max_trials) {
    const long long si = s0 + lane;
    if (si < n_btab) beta_pre = btab[si];
  }
  {
    const int k = wid >> 1, h = wid & 1;
    const double* arr = k == 0 ? part_f : k == 1 ? part_bc : k == 2 ? part_bc + nbc : part_g;
    const int len = k == 0 ? nf : k == 3 ? ng : nbc;
    const int per = (len + G - 1) / G;
    const int i0 = min(len, b * per), i1 = min(len, i0 + per);
    double v = 0.0;
    for (int i = i0 + 32 * h + lane; i < i1; i += 64) v += arr[i];
    v = warp_sum_nz(v);
    if (lane == 0) wred[k][h] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) stage[threadIdx.x * G + b] = wred[threadIdx.x][0] + wred[threadIdx.x][1];
  if (threadIdx.x == 0) {
    __threadfence();
    sh_last = atomicAdd(&st->done_fin, 1u) == (unsigned)G - 1;
  }
  __syncthreads();
  if (!sh_last) return;
  __threadfence();
  // the slice sums, written by other CTAs of this launch: read past L1
  if (wid < 4) {
    double v = 0.0;
    for (int i = lane; i < G; i += 32) v += __ldcg(&stage[wid * G + i]);
    v = warp_sum_nz(v);
    if (lane == 0) tot_sh[wid] = v;
  }
  __syncthreads();
  if (wid != 0) return;
  const double f = tot_sh[0] + (step == 0 ? f_empty : 0.0);
  const double Bp = tot_sh[1];
  const double Cp = tot_sh[2];
  const double gn2 = tot_sh[3];
  // The trial loop of Fig. 3 (beta = beta0 alpha^s, s advancing on every
  // trial, accept the first trial that does not ascend, at most max_trials):
  // the warp evaluates 32 consecutive trials at once, one per lane, and takes
  // the lowest accepting lane, so the decision and s are those of the trials
  // taken in turn.  The steps beta0 alpha^s come from the table filled at
  // fredopt_begin (s < n_btab), else from the same FP64 expression.
  const double gn = gn2 > 0.0 ? sqrt(gn2) : 0.0;
  const double ig = gn2 > 0.0 ? 1.0 / gn : 0.0;  // one FP64 division for B, C and the step
  double B = 0.0, C = 0.0;
  if (gn2 > 0.0) {
    if (grad_normalize) { B = -Bp * ig; C = Cp * ig * ig; }
    else { B = -Bp; C = Cp; }
  }
  int first = max_trials;  // index of the accepted trial, max_trials if none
  double beta_acc = 0.0;
  if (gn2 > 0.0) {
    for (int base = 0; base < max_trials; base += 32) {
      const int tr = base + lane;
      double beta = 0.0;
      bool ok = false;
      if (tr < max_trials) {
        const long long si = s0 + tr;
        beta = base == 0 && si < n_btab ? beta_pre
             : si < n_btab              ? btab[si]
                                        : st->beta0 * pow(st->alpha, (double)si);
        const double df = beta * (2.0 * B + beta * C);  // f(x + beta v) - f(x), Eq. 2 is quadratic
        ok = df <= 0.0;
      }
      const unsigned acc = __ballot_sync(kFull, ok);
      if (acc) {
        const int l = __ffs(acc) - 1;
        first = base + l;
        beta_acc = __shfl_sync(kFull, beta, l);
        break;
      }
    }
  }
  if (lane != 0) return;
  st->done_fin = 0u;
  if (step == 0) {
    st->f_start = f;
    st->accepted = 0;
    st->beta_acc = 0.0;
  }
  double fc = f;
  double coef = 0.0;
  long long s = s0;
  if (gn2 > 0.0) {
    st->gnorm = gn;
    if (first < max_trials) {
      const double beta = beta_acc;
      coef = grad_normalize ? -beta * ig : -beta;
      st->accepted += 1;
      st->accepted_total += 1;
      st->beta_acc = beta;
      fc = f + beta * (2.0 * B + beta * C);
      s = s0 + first + 1;
    } else {
      s = s0 + max_trials;
    }
  } else {
    st->gnorm = 0.0;
  }
  st->s = s;
  st->coef = coef;
  st->f_cur = fc;
}

// x <- x + coef g for the next perturbation step (reductions > 1)
__global__ void k_apply_step(int64_t n_hot, int n, float* w, const float* g, float2* yw,
                             const float2* yg, const DevState* st) {
  const double coef = st->coef;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) w[i] = (float)((double)w[i] + coef * (double)g[i]);
  if (i < n_hot) {
    const float2 a = yw[i], b = yg[i];
    yw[i] = make_float2((float)((double)a.x + coef * b.x), (float)((double)a.y + coef * b.y));
  }
}

__global__ void __launch_bounds__(kRowThreads) k_row_objective(Tables t, const float2* yw,
                                                              const uint32_t* mask, const float* sD,
                                                              const float* sL, int64_t n_hot,
                                                              float2* r_out, double* part) {
  __shared__ double red[kRowThreads];
  const int64_t per = (n_hot + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * per, i1 = min(n_hot, i0 + per);
  double acc = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const float2 y = yw[i];
    double f, rD, rL;
    row_objective(t, mask[i], y.x, y.y, f, rD, rL);
    const double sd = sD ? (double)sD[i] : 1.0, sl = sL ? (double)sL[i] : 1.0;
    r_out[i] = make_float2((float)(rD * sd), (float)(rL * sl));
    acc += f;
  }
  acc = block_sum256(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// FP64 check at the final point: per block [max violation per kind (6), n violated, f]
__global__ void __launch_bounds__(kRowThreads) k_final_check(Tables t, const double2* y64,
                                                            const uint32_t* mask, const double* dd,
                                                            const double* ll, const double* dl,
                                                            int64_t n_hot, double* part) {
  __shared__ double red[kRowThreads];
  const int64_t per = (n_hot + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * per, i1 = min(n_hot, i0 + per);
  double mk[6] = {0, 0, 0, 0, 0, 0};
  double nv = 0.0, fo = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const uint32_t m = mask[i];
    if (!m) continue;
    const double2 y = y64[i];
    for (int q = 0; q < t.n_con; ++q) {
      const ConEntry& c = t.con[q];
      if (!((m >> c.bit) & 1u)) continue;
      const int fam = c.kind >> 1;
      double v, n2, b;
      if (fam == 0) { v = y.x; n2 = dd[i]; b = c.bound; }
      else if (fam == 1) { v = t.c * y.y; n2 = ll[i]; b = c.bound; }
      else {
        v = y.y - c.bound * y.x;
        n2 = ll[i] - 2.0 * c.bound * dl[i] + c.bound * c.bound * dd[i];
        b = 0.0;
      }
      if (!(n2 > 0.0)) continue;
      const double viol = (c.kind & 1) ? v - b : b - v;
      if (viol > 0.0) {
        nv += 1.0;
        const double vu = (fam == 2) ? (y.x > 0.0 ? viol / y.x : 0.0) : viol;
        mk[c.kind] = fmax(mk[c.kind], vu);
      }
    }
    double f, rD, rL;
    row_objective(t, m, y.x, y.y, f, rD, rL);
    fo += f;
  }
  for (int q = 0; q < 6; ++q) {
    const double v = block_max256(mk[q], red);
    if (threadIdx.x == 0) part[blockIdx.x * 8 + q] = v;
  }
  nv = block_sum256(nv, red);
  fo = block_sum256(fo, red);
  if (threadIdx.x == 0) {
    part[blockIdx.x * 8 + 6] = nv;
    part[blockIdx.x * 8 + 7] = fo;
  }
}

__global__ void k_begin_state(DevState* st) {
  st->k = 0;
  st->s = 0;
  st->accepted_total = 0;
  st->accepted = 0;
  st->coef = 0.0;
  st->f_start = st->f_cur = st->gnorm = st->beta_acc = 0.0;
  st->err = 0;
  st->done = 0u;
}

// ------------------------------------------------------------------ K5 setup

__global__ void k_validate(const int64_t* rp, const int32_t* col, const float* D, const float* L,
                           int64_t n_rows, int32_t n_cols, int* err) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_rows; r += nw) {
    const int64_t s = rp[r], e = rp[r + 1];
    int bad = 0;
    for (int64_t p = s + lane; p < e; p += 32) {
      const int c = col[p];
      if (c < 0 || c >= n_cols) bad |= 1;
      if (p > s && col[p - 1] >= c) bad |= 1;
      if (!isfinite(D[p]) || !isfinite(L[p])) bad |= 2;
    }
    bad = __reduce_or_sync(kFull, bad);
    if (bad && lane == 0) atomicOr(err, bad);
  }
}

__global__ void k_gather_rows(const int64_t* rp_src, const int64_t* src_row, const int64_t* rp_dst,
                              int64_t n_rows, const int32_t* col_src, const float* D_src,
                              const float* L_src, int32_t* col_dst, float* D_dst, float* L_dst) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_rows; r += nw) {
    const int64_t sr = src_row[r];
    const int64_t s = rp_src[sr], e = rp_src[sr + 1], d = rp_dst[r];
    for (int64_t p = s + lane; p < e; p += 32) {
      col_dst[d + (p - s)] = col_src[p];
      D_dst[d + (p - s)] = D_src[p];
      L_dst[d + (p - s)] = L_src[p];
    }
  }
}

// Power-of-two scale so that scale * q is exact in binary32:
// BF16: max|q| in (1/2, 1]; FP16: max|q| in (2^13, 2^14] (all normal values
// down to 2^-28 of the row maximum keep 11 significant bits).
__device__ __forceinline__ float pow2_scale(float amax, int fmt) {
  if (!(amax > 0.0f)) return 1.0f;
  int ex;
  frexpf(amax, &ex);  // amax in [2^(ex-1), 2^ex)
  return ldexpf(1.0f, fmt == 2 ? ex - 14 : ex);
}

template <typename VT>
__device__ __forceinline__ VT from_f(float v);
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }

template <typename VT>
__global__ void k_quantize(int fmt, const int64_t* rp, int64_t n_rows, const float* D, const float* L,
                           VT* qD, VT* qL, float* sD, float* sL) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_rows; r += nw) {
    const int64_t s = rp[r], e = rp[r + 1];
    float mD = 0.f, mL = 0.f;
    for (int64_t p = s + lane; p < e; p += 32) {
      mD = fmaxf(mD, fabsf(D[p]));
      mL = fmaxf(mL, fabsf(L[p]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mD = fmaxf(mD, __shfl_xor_sync(kFull, mD, o));
      mL = fmaxf(mL, __shfl_xor_sync(kFull, mL, o));
    }
    const float scD = pow2_scale(mD, fmt), scL = pow2_scale(mL, fmt);
    for (int64_t p = s + lane; p < e; p += 32) {
      qD[p] = from_f<VT>(D[p] / scD);
      qL[p] = from_f<VT>(L[p] / scL);
    }
    if (lane == 0) { sD[r] = scD; sL[r] = scL; }
  }
}

// FP64-accurate row moments |D_i|^2, |L_i|^2, <D_i, L_i> of the stored
// values in double-float (exact products, accurate double-word sums: relative
// error <= 3 * 2^-48 per addition of these nonnegative terms), at FP32 speed;
// the power-of-two row scales are applied at the end, exactly.
template <typename VT>
__global__ void k_moments(const int64_t* rp, int64_t n_rows, const VT* Dv, const VT* Lv,
                          const float* sD, const float* sL, double* dd, double* ll, double* dl) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_rows; r += nw) {
    const int64_t s = rp[r], e = rp[r + 1];
    DF a, b, c;
    for (int64_t p = s + lane; p < e; p += 32) {
      const float d = to_f(Dv[p]), l = to_f(Lv[p]);
      a = acc_fma(d, d, a);
      b = acc_fma(l, l, b);
      c = acc_fma(d, l, c);
    }
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    if (lane == 0) {
      const double sd = sD ? (double)sD[r] : 1.0, sl = sL ? (double)sL[r] : 1.0;
      dd[r] = (double)a * (sd * sd);
      ll[r] = (double)b * (sl * sl);
      dl[r] = (double)c * (sd * sl);
    }
  }
}

// blocked counting transpose: block b owns rows [blk_row[b], blk_row[b+1])
template <bool SMEM>
__global__ void k_csc_count(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const int64_t* __restrict__ blk_row, int32_t n_cols, int32_t* __restrict__ cnt) {
  extern __shared__ int32_t sh_cnt[];
  const int b = blockIdx.x;
  const int64_t s = rp[blk_row[b]], e = rp[blk_row[b + 1]];
  int32_t* c = cnt + (int64_t)b * n_cols;
  if (SMEM) {  // a shared-memory histogram, then one coalesced write of the block's row
    for (int j = threadIdx.x; j < n_cols; j += blockDim.x) sh_cnt[j] = 0;
    __syncthreads();
    for (int64_t p = s + threadIdx.x; p < e; p += blockDim.x) atomicAdd(&sh_cnt[col[p]], 1);
    __syncthreads();
    for (int j = threadIdx.x; j < n_cols; j += blockDim.x) c[j] = sh_cnt[j];
  } else {
    for (int64_t p = s + threadIdx.x; p < e; p += blockDim.x) atomicAdd(&c[col[p]], 1);
  }
}

__global__ void k_csc_colsum(const int32_t* cnt, int n_blk, int32_t n_cols, int64_t* tot) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_cols) return;
  int64_t s = 0;
  for (int b = 0; b < n_blk; ++b) s += cnt[(int64_t)b * n_cols + j];
  tot[j] = s;
}

// cnt[b][j] <- first output position of block b's entries of column j
__global__ void k_csc_offsets(int32_t* cnt, int n_blk, int32_t n_cols, const int64_t* cp) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_cols) return;
  int64_t run = cp[j];
  for (int b = 0; b < n_blk; ++b) {
    const int64_t i = (int64_t)b * n_cols + j;
    const int32_t t = cnt[i];
    cnt[i] = (int32_t)run;  // positions < 2^31 (checked on the host)
    run += t;
  }
}

// Rows of a block in ascending order; within a row all columns differ, so
// the cursor updates of one row never collide; a barrier separates rows,
// which keeps the rows of every column ascending (a stable transpose).
// The block's nonzeros reach shared memory by bulk copies (TMA engine) in
// windows of W elements, two buffers deep: while the rows of one window are
// scattered the next window is in flight, and a block barrier does not wait
// for bulk copies, so a row costs shared-memory reads, a cursor update and a
// barrier.  Row pointers are staged in chunks of kFillRows rows.  A bounded
// wait that gives up sets bit 0 of *err; the block lets its copies land and
// stops (the load then fails with a timeout).
constexpr int kFillThreads = 1024;
constexpr int kFillRows = 2048;
constexpr int64_t kFillAlign = 8;  // window starts and lengths: 16 bytes of every array
constexpr size_t kFillRpBytes = ((kFillRows + 1) * sizeof(int64_t) + 15) & ~(size_t)15;

template <typename VT>
size_t csc_fill_smem(int W, int32_t n_cols, bool smem_cursors) {
  return 2 * (size_t)W * (sizeof(int32_t) + 2 * sizeof(VT)) + kFillRpBytes +
         (smem_cursors ? (((size_t)n_cols * sizeof(int32_t) + 15) & ~(size_t)15) : 0) + 2 * sizeof(uint64_t);
}

template <typename VT, bool SMEM>
__global__ void __launch_bounds__(kFillThreads) k_csc_fill(
    const int64_t* __restrict__ rp, const int32_t* __restrict__ col, const VT* __restrict__ Dv,
    const VT* __restrict__ Lv, const int64_t* __restrict__ blk_row, int32_t n_cols, int32_t* __restrict__ cursor,
    int32_t* __restrict__ row_out, VT* __restrict__ DT, VT* __restrict__ LT, int W, int* err) {
  extern __shared__ __align__(16) unsigned char fill_sh[];
  const int b = blockIdx.x;
  const int64_t r0 = blk_row[b], r1 = blk_row[b + 1];
  if (r0 >= r1) return;
  const size_t win_bytes = (size_t)W * (sizeof(int32_t) + 2 * sizeof(VT));
  int64_t* sh_rp = reinterpret_cast<int64_t*>(fill_sh + 2 * win_bytes);
  int32_t* sh_cur = reinterpret_cast<int32_t*>(fill_sh + 2 * win_bytes + kFillRpBytes);
  const size_t cur_bytes = SMEM ? (((size_t)n_cols * sizeof(int32_t) + 15) & ~(size_t)15) : 0;
  uint64_t* bar = reinterpret_cast<uint64_t*>(fill_sh + 2 * win_bytes + kFillRpBytes + cur_bytes);
  auto wcol = [&](int j) { return reinterpret_cast<int32_t*>(fill_sh + j * win_bytes); };
  auto wD = [&](int j) { return reinterpret_cast<VT*>(fill_sh + j * win_bytes + sizeof(int32_t) * (size_t)W); };
  auto wL = [&](int j) {
    return reinterpret_cast<VT*>(fill_sh + j * win_bytes + (sizeof(int32_t) + sizeof(VT)) * (size_t)W);
  };
  int32_t* cur = cursor + (int64_t)b * n_cols;
  if (SMEM) {  // the block's cursors stay in shared memory for the whole pass
    for (int j = threadIdx.x; j < n_cols; j += blockDim.x) sh_cur[j] = cur[j];
    cur = sh_cur;
  }
  // window k = elements [EA + k W, min(EA + (k + 1) W, EZ)); the arrays are
  // zero padded past nnz to a multiple of 256 elements, so EZ is in bounds
  const int64_t EA = rp[r0] & ~(kFillAlign - 1);
  const int64_t EZ = (rp[r1] + kFillAlign - 1) & ~(kFillAlign - 1);
  const int64_t n_win = (EZ - EA + W - 1) / W;
  auto issue = [&](int64_t k) {  // thread 0: window k into buffer k & 1
    const int j = (int)(k & 1);
    const int64_t ws = EA + k * W;
    const uint32_t n = (uint32_t)(EZ - ws < W ? EZ - ws : W);
    mbar_expect_tx(&bar[j], n * (uint32_t)(sizeof(int32_t) + 2 * sizeof(VT)));
    bulk_g2s(wcol(j), col + ws, n * (uint32_t)sizeof(int32_t), &bar[j]);
    bulk_g2s(wD(j), Dv + ws, n * (uint32_t)sizeof(VT), &bar[j]);
    bulk_g2s(wL(j), Lv + ws, n * (uint32_t)sizeof(VT), &bar[j]);
  };
  // window k's phase on its buffer is the (k >> 1)-th; the outcome is made uniform over the block
  auto wait_win = [&](int64_t k) -> bool {
    const bool ok = mbar_wait(&bar[k & 1], (uint32_t)((k >> 1) & 1), kMbarSpins);
    return __syncthreads_and(ok) != 0;
  };
  auto land = [&](int64_t k) {  // let windows k and k + 1 (issued ones) arrive
    if (k < n_win) mbar_wait(&bar[k & 1], (uint32_t)((k >> 1) & 1), kMbarSpins);
    if (k + 1 < n_win) mbar_wait(&bar[(k + 1) & 1], (uint32_t)(((k + 1) >> 1) & 1), kMbarSpins);
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    issue(0);
    if (n_win > 1) issue(1);
  }
  int64_t k = 0;
  if (!wait_win(0)) {
    if (threadIdx.x == 0) atomicOr(err, 1);
    land(0);
    return;
  }
  int64_t ws = EA, we = EA + W < EZ ? EA + W : EZ;
  for (int64_t c0 = r0; c0 < r1; c0 += kFillRows) {
    const int nr = (int)(r1 - c0 < kFillRows ? r1 - c0 : kFillRows);
    __syncthreads();  // the previous chunk is done with sh_rp
    for (int i = threadIdx.x; i <= nr; i += blockDim.x) sh_rp[i] = rp[c0 + i];
    __syncthreads();
    for (int i = 0; i < nr; ++i) {
      int64_t sp = sh_rp[i];
      const int64_t ep = sh_rp[i + 1];
      const int32_t r = (int32_t)(c0 + i);
      while (true) {
        const int64_t hi = ep < we ? ep : we;
        const int j = (int)(k & 1);
        const int32_t* cc = wcol(j);
        const VT* dd = wD(j);
        const VT* ll = wL(j);
        for (int64_t p = sp + threadIdx.x; p < hi; p += kFillThreads) {
          const int o = (int)(p - ws);
          const int c = cc[o];
          const int32_t pos = cur[c];
          cur[c] = pos + 1;
          row_out[pos] = r;
          DT[pos] = dd[o];
          LT[pos] = ll[o];
        }
        if (ep <= we) break;
        // the row continues in window k + 1: free buffer k & 1 for window k + 2
        __syncthreads();
        if (threadIdx.x == 0 && k + 2 < n_win) issue(k + 2);
        ++k;
        if (!wait_win(k)) {
          if (threadIdx.x == 0) atomicOr(err, 1);
          land(k);
          return;
        }
        ws += W;
        we = ws + W < EZ ? ws + W : EZ;
        sp = hi;
      }
      __syncthreads();  // the row's cursor updates are done
    }
  }
  land(k + 1);  // nothing is normally in flight here; never leave with a copy pending
}

template <typename VT>
__global__ void k_dequant_csc(const int64_t* cp, int32_t n_cols, const int32_t* row, const VT* DT,
                              const VT* LT, const float* sD, const float* sL, float* Dout, float* Lout) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n_cols; j += nw) {
    for (int64_t p = cp[j] + lane; p < cp[j + 1]; p += 32) {
      const int r = row[p];
      Dout[p] = (sD ? sD[r] : 1.0f) * to_f(DT[p]);
      Lout[p] = (sL ? sL[r] : 1.0f) * to_f(LT[p]);
    }
  }
}

__global__ void k_scale_coef(int64_t n, const float* aD, const float* aL, const int64_t* voxel,
                             const float* sD, const float* sL, float2* coef) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t v = voxel ? voxel[i] : i;
  const float d = aD ? aD[v] : 0.0f, l = aL ? aL[v] : 0.0f;
  coef[i] = make_float2(sD ? d * sD[i] : d, sL ? l * sL[i] : l);
}


// reachable constraint rows (|a_r|^2 > 0): per block [count, unreachable, sum of priorities]
__global__ void __launch_bounds__(kRowThreads) k_count_rows(Tables t, const uint32_t* mask,
                                                           const double* dd, const double* ll,
                                                           const double* dl, int64_t n_hot,
                                                           double* part) {
  __shared__ double red[kRowThreads];
  const int64_t per = (n_hot + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * per, i1 = min(n_hot, i0 + per);
  double nr = 0.0, nu = 0.0, W = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const uint32_t m = mask[i];
    if (!m) continue;
    for (int q = 0; q < t.n_con; ++q) {
      const ConEntry& c = t.con[q];
      if (!((m >> c.bit) & 1u)) continue;
      const int fam = c.kind >> 1;
      const double n2 = fam == 0 ? dd[i]
                      : fam == 1 ? ll[i]
                                 : ll[i] - 2.0 * c.bound * dl[i] + c.bound * c.bound * dd[i];
      if (n2 > 0.0) { nr += 1.0; W += c.prio; }
      else nu += 1.0;
    }
  }
  nr = block_sum256(nr, red);
  nu = block_sum256(nu, red);
  W = block_sum256(W, red);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = nr;
    part[3 * blockIdx.x + 1] = nu;
    part[3 * blockIdx.x + 2] = W;
  }
}

__global__ void k_scatter_y(const float2* y, const int64_t* voxel, int64_t n, float* a, float* b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t v = voxel ? voxel[i] : i;
  const float2 t = y[i];
  if (a) a[v] = t.x;
  if (b) b[v] = t.y;
}

// ------------------------------------------------------------------ launch wrappers

template <typename VT, int EPI, bool XS, bool S, typename IT = int32_t>
static void fwd_inst(const Geometry& g, const FwdArgs& a, const Tables& t, cudaStream_t s) {
  const size_t smem = XS ? (size_t)a.n_x_pad * sizeof(float) + 16 : 0;
  // only the CTAs that hold scheduled warps (all of them for a full pass)
  const int wpb = g.fwd_threads / 32;
  const int blocks = std::max(1, std::min(g.fwd_blocks, (a.n_warps + wpb - 1) / wpb));
  k_forward<VT, EPI, XS, S, IT><<<blocks, g.fwd_threads, smem, s>>>(a, t);
}

template <typename VT, int EPI>
static void fwd_dispatch_xs(const Geometry& g, bool xs, bool st, const FwdArgs& a, const Tables& t,
                            cudaStream_t s) {
  if (a.col16) {  // the load keeps 16-bit indices only when x fits shared memory
    if (EPI == EPI_FINAL || !st) fwd_inst<VT, EPI, true, false, uint16_t>(g, a, t, s);
    else fwd_inst<VT, EPI, true, true, uint16_t>(g, a, t, s);
    return;
  }
  if (EPI == EPI_FINAL) {
    if (xs) fwd_inst<VT, EPI, true, false>(g, a, t, s);
    else fwd_inst<VT, EPI, false, false>(g, a, t, s);
    return;
  }
  if (xs) {
    if (st) fwd_inst<VT, EPI, true, true>(g, a, t, s);
    else fwd_inst<VT, EPI, true, false>(g, a, t, s);
  } else {
    if (st) fwd_inst<VT, EPI, false, true>(g, a, t, s);
    else fwd_inst<VT, EPI, false, false>(g, a, t, s);
  }
}

template <typename VT>
static void fwd_dispatch_epi(const Geometry& g, int epi, bool xs, bool st, const FwdArgs& a,
                             const Tables& t, cudaStream_t s) {
  switch (epi) {
    case EPI_STORE: fwd_dispatch_xs<VT, EPI_STORE>(g, xs, st, a, t, s); break;
    case EPI_OBJ: fwd_dispatch_xs<VT, EPI_OBJ>(g, xs, st, a, t, s); break;
    case EPI_BC: fwd_dispatch_xs<VT, EPI_BC>(g, xs, st, a, t, s); break;
    default: fwd_dispatch_xs<VT, EPI_FINAL>(g, xs, st, a, t, s); break;
  }
}

bool forward_uses_smem(const Geometry& g, int n_x_pad) {
  return FO_FWD_XS && (size_t)n_x_pad * sizeof(float) + 16 <= g.smem_limit;
}

void launch_forward(const Geometry& g, int fmt, int epi, bool stream_hint, const FwdArgs& a,
                    const Tables& t, cudaStream_t s) {
  const bool xs = forward_uses_smem(g, a.n_x_pad);
  if (fmt == 1) fwd_dispatch_epi<__nv_bfloat16>(g, epi, xs, stream_hint, a, t, s);
  else if (fmt == 2) fwd_dispatch_epi<__half>(g, epi, xs, stream_hint, a, t, s);
  else fwd_dispatch_epi<float>(g, epi, xs, stream_hint, a, t, s);
}

template <typename VT, bool NB>
static void bwd_dispatch_nb(const Geometry& g, bool st, bool ud, const BwdArgs& a, cudaStream_t s) {
  if (st) {
    if (ud) k_backward<VT, true, true, NB><<<g.bwd_blocks, g.bwd_threads, 0, s>>>(a);
    else k_backward<VT, true, false, NB><<<g.bwd_blocks, g.bwd_threads, 0, s>>>(a);
  } else {
    if (ud) k_backward<VT, false, true, NB><<<g.bwd_blocks, g.bwd_threads, 0, s>>>(a);
    else k_backward<VT, false, false, NB><<<g.bwd_blocks, g.bwd_threads, 0, s>>>(a);
  }
}
template <typename VT>
static void bwd_dispatch(const Geometry& g, bool st, bool ud, const BwdArgs& a, cudaStream_t s) {
  if (a.row16) bwd_dispatch_nb<VT, true>(g, st, ud, a, s);
  else bwd_dispatch_nb<VT, false>(g, st, ud, a, s);
}

void launch_backward(const Geometry& g, int fmt, bool stream_hint, bool use_D, const BwdArgs& a,
                     cudaStream_t s) {
  if (fmt == 1) bwd_dispatch<__nv_bfloat16>(g, stream_hint, use_D, a, s);
  else if (fmt == 2) bwd_dispatch<__half>(g, stream_hint, use_D, a, s);
  else bwd_dispatch<float>(g, stream_hint, use_D, a, s);
}

void launch_colfinish(const Geometry& g, int mode, const ColArgs& a, cudaStream_t s) {
  if (mode == COL_OUT) k_colfinish<COL_OUT><<<g.col_blocks, kColThreads, 0, s>>>(a);
  else if (mode == COL_GRAD) k_colfinish<COL_GRAD><<<g.col_blocks, kColThreads, 0, s>>>(a);
  else k_colfinish<COL_PROJ><<<g.col_blocks + a.log_block, kColThreads, 0, s>>>(a);
}

void launch_constraints(const Geometry& g, const Tables& t, const ConArgs& a, cudaStream_t s, int grid) {
  k_constraints<<<grid > 0 ? grid : g.row_blocks, kRowThreads, 0, s>>>(a, t);
}

__global__ void k_beta_table(double* out, long long n, double beta0, double alpha) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = beta0 * pow(alpha, (double)i);
}

void launch_beta_table(double* out, long long n, double beta0, double alpha, cudaStream_t s) {
  if (n > 0) k_beta_table<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n, beta0, alpha);
}

void launch_finish(int step, const double* part_f, int nf, const double* part_bc, int nbc,
                   const double* part_g, int ng, DevState* st, double* stage, const double* btab,
                   long long n_btab, cudaStream_t s) {
  k_finish<<<kFinishBlocks, 256, 0, s>>>(step, part_f, nf, part_bc, nbc, part_g, ng, st, stage, btab, n_btab);
}

void launch_apply_step(int64_t n_hot, int n, float* w, const float* g, float2* yw, const float2* yg,
                       const DevState* st, cudaStream_t s) {
  const int64_t m = n_hot > n ? n_hot : n;
  if (m == 0) return;
  k_apply_step<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(n_hot, n, w, g, yw, yg, st);
}

void launch_row_objective(const Geometry& g, const Tables& t, const float2* yw, const uint32_t* mask,
                          const float* sD, const float* sL, int64_t n_hot, float2* r_out,
                          double* part, cudaStream_t s) {
  k_row_objective<<<g.row_blocks, kRowThreads, 0, s>>>(t, yw, mask, sD, sL, n_hot, r_out, part);
}

void launch_final_check(const Geometry& g, const Tables& t, const double2* y64, const uint32_t* mask,
                        const double* dd, const double* ll, const double* dl, int64_t n_hot,
                        double* part, cudaStream_t s) {
  k_final_check<<<g.row_blocks, kRowThreads, 0, s>>>(t, y64, mask, dd, ll, dl, n_hot, part);
}

void launch_begin_state(DevState* st, cudaStream_t s) { k_begin_state<<<1, 1, 0, s>>>(st); }

void launch_count_rows(const Geometry& g, const Tables& t, const uint32_t* mask, const double* dd,
                       const double* ll, const double* dl, int64_t n_hot, double* part,
                       cudaStream_t s) {
  k_count_rows<<<g.row_blocks, kRowThreads, 0, s>>>(t, mask, dd, ll, dl, n_hot, part);
}

void launch_scatter_y(const float2* y, const int64_t* voxel, int64_t n, float* a, float* b,
                      cudaStream_t s) {
  if (n == 0) return;
  k_scatter_y<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(y, voxel, n, a, b);
}

static unsigned grid_for(int64_t work, int per_block, int cap) {
  int64_t b = (work + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

void launch_validate(const int64_t* rp, const int32_t* col, const float* D, const float* L,
                     int64_t n_rows, int32_t n_cols, int64_t, int* err, cudaStream_t s) {
  if (n_rows == 0) return;
  k_validate<<<grid_for(n_rows, 8, 65535), 256, 0, s>>>(rp, col, D, L, n_rows, n_cols, err);
}

void launch_gather_rows(const int64_t* rp_src, const int64_t* src_row, const int64_t* rp_dst,
                        int64_t n_rows, const int32_t* col_src, const float* D_src,
                        const float* L_src, int32_t* col_dst, float* D_dst, float* L_dst,
                        cudaStream_t s) {
  if (n_rows == 0) return;
  k_gather_rows<<<grid_for(n_rows, 8, 65535), 256, 0, s>>>(rp_src, src_row, rp_dst, n_rows, col_src,
                                                          D_src, L_src, col_dst, D_dst, L_dst);
}

void launch_quantize(int fmt, const int64_t* rp, int64_t n_rows, const float* D, const float* L,
                     void* qD, void* qL, float* sD, float* sL, cudaStream_t s) {
  if (n_rows == 0) return;
  const unsigned gb = grid_for(n_rows, 8, 65535);
  if (fmt == 1)
    k_quantize<__nv_bfloat16><<<gb, 256, 0, s>>>(fmt, rp, n_rows, D, L, (__nv_bfloat16*)qD,
                                                  (__nv_bfloat16*)qL, sD, sL);
  else
    k_quantize<__half><<<gb, 256, 0, s>>>(fmt, rp, n_rows, D, L, (__half*)qD, (__half*)qL, sD, sL);
}

void launch_moments(int fmt, const int64_t* rp, int64_t n_rows, const void* Dv, const void* Lv,
                    const float* sD, const float* sL, double* dd, double* ll, double* dl,
                    cudaStream_t s) {
  if (n_rows == 0) return;
  const unsigned gb = grid_for(n_rows, 8, 65535);
  if (fmt == 1)
    k_moments<__nv_bfloat16><<<gb, 256, 0, s>>>(rp, n_rows, (const __nv_bfloat16*)Dv,
                                                 (const __nv_bfloat16*)Lv, sD, sL, dd, ll, dl);
  else if (fmt == 2)
    k_moments<__half><<<gb, 256, 0, s>>>(rp, n_rows, (const __half*)Dv, (const __half*)Lv, sD, sL, dd,
                                          ll, dl);
  else
    k_moments<float><<<gb, 256, 0, s>>>(rp, n_rows, (const float*)Dv, (const float*)Lv, sD, sL, dd,
                                         ll, dl);
}

constexpr size_t kCscSmemMax = 200 * 1024;  // per-block column table kept in shared memory

void launch_csc_count(const int64_t* rp, const int32_t* col, const int64_t* blk_row, int n_blk,
                      int32_t n_cols, int32_t* cnt, cudaStream_t s) {
  const size_t smem = (size_t)n_cols * sizeof(int32_t);
  if (smem <= kCscSmemMax) {
    cudaFuncSetAttribute(k_csc_count<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_csc_count<true><<<n_blk, 1024, smem, s>>>(rp, col, blk_row, n_cols, cnt);
  } else {
    k_csc_count<false><<<n_blk, 1024, 0, s>>>(rp, col, blk_row, n_cols, cnt);
  }
}

void launch_csc_colsum(const int32_t* cnt, int n_blk, int32_t n_cols, int64_t* tot, cudaStream_t s) {
  k_csc_colsum<<<(n_cols + 255) / 256, 256, 0, s>>>(cnt, n_blk, n_cols, tot);
}

void launch_csc_offsets(int32_t* cnt, int n_blk, int32_t n_cols, const int64_t* cp, cudaStream_t s) {
  k_csc_offsets<<<(n_cols + 255) / 256, 256, 0, s>>>(cnt, n_blk, n_cols, cp);
}

// The same stable transpose, rows taken kFillWinRows at a time: the order of
// a column's entries within a window of rows is recovered from a per-column
// bit mask of the window rows that hold the column, so a window costs three
// block barriers instead of one per row.  For each window:
//   A  every entry (row r, column c) sets bit r - g0 of mask[c] (atomic OR,
//      order-independent);
//   B  it goes to position cur[c] + popc(mask[c] below bit r - g0): the rows
//      of the window before r that hold c come first, as in row order;
//   C  the first entry of each column advances cur[c] by popc(mask[c]) and
//      clears the mask.
// Two 16-bit masks share a 32-bit word.  Shared memory: the block's cursors
// and masks (6 bytes per column) and a chunk of row pointers.  The result
// equals k_csc_fill's bit for bit.
constexpr int kFillWinRows = 16;
constexpr int kFillK = 2;  // entries per thread a window holds in registers (else the loop form)
#ifndef FO_FILL_WIN
#define FO_FILL_WIN 1  // 0: the row-by-row k_csc_fill for every plan
#endif
#ifndef FO_FILL_REC
#define FO_FILL_REC 1  // 1: the window fill stores records, then k_csc_split
#endif

__device__ __forceinline__ int fill_win_row(const int64_t* wrp, int nr, int64_t p) {
  int lo = 0, hi = nr - 1;  // the window row r with wrp[r] <= p < wrp[r + 1]
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (wrp[mid] <= p) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// With `rec`, an entry is one record store (row and both values: 16 bytes
// for FP32, 8 for 16-bit values) instead of three scattered 4- or 2-byte
// stores, and k_csc_split writes the three arrays afterwards with coalesced
// stores: scattered stores are limited by their count, not their bytes.
template <typename VT> struct FillRec;
template <> struct FillRec<float> { using T = int4; };
template <> struct FillRec<uint16_t> { using T = uint2; };
__device__ __forceinline__ int4 fill_rec(int32_t r, float d, float l) {
  return make_int4(r, __float_as_int(d), __float_as_int(l), 0);
}
__device__ __forceinline__ uint2 fill_rec(int32_t r, uint16_t d, uint16_t l) {
  return make_uint2((uint32_t)r, (uint32_t)d | ((uint32_t)l << 16));
}

template <typename VT>
__global__ void k_csc_split(const typename FillRec<VT>::T* __restrict__ rec, int64_t n, int32_t* __restrict__ row_out,
                            VT* __restrict__ DT, VT* __restrict__ LT) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const auto v = rec[i];
  if constexpr (sizeof(VT) == 4) {
    row_out[i] = v.x;
    DT[i] = __int_as_float(v.y);
    LT[i] = __int_as_float(v.z);
  } else {
    row_out[i] = (int32_t)v.x;
    DT[i] = (uint16_t)(v.y & 0xffffu);
    LT[i] = (uint16_t)(v.y >> 16);
  }
}

template <typename VT>
__global__ void __launch_bounds__(kFillThreads) k_csc_fill_win(
    const int64_t* __restrict__ rp, const int32_t* __restrict__ col, const VT* __restrict__ Dv,
    const VT* __restrict__ Lv, const int64_t* __restrict__ blk_row, int32_t n_cols,
    const int32_t* __restrict__ cursor, int32_t* __restrict__ row_out, VT* __restrict__ DT,
    VT* __restrict__ LT, typename FillRec<VT>::T* __restrict__ rec) {
  extern __shared__ __align__(16) unsigned char fill_sh[];
  int32_t* cur = reinterpret_cast<int32_t*>(fill_sh);
  uint32_t* mask = reinterpret_cast<uint32_t*>(fill_sh + (size_t)n_cols * sizeof(int32_t));
  int64_t* srp = reinterpret_cast<int64_t*>(
      fill_sh + (((size_t)n_cols * sizeof(int32_t) + (size_t)((n_cols + 1) / 2) * sizeof(uint32_t) + 15) & ~(size_t)15));
  const int b = blockIdx.x;
  const int64_t r0 = blk_row[b], r1 = blk_row[b + 1];
  if (r0 >= r1) return;
  const int32_t* gcur = cursor + (int64_t)b * n_cols;
  for (int j = threadIdx.x; j < n_cols; j += blockDim.x) cur[j] = gcur[j];
  for (int j = threadIdx.x; j < (n_cols + 1) / 2; j += blockDim.x) mask[j] = 0u;
  // row pointers staged kFillRows rows at a time; windows of kFillWinRows rows
  for (int64_t c0 = r0; c0 < r1; c0 += kFillRows) {
    const int nc = (int)(r1 - c0 < kFillRows ? r1 - c0 : kFillRows);
    __syncthreads();  // the previous chunk is done with srp, cur and mask
    for (int i = threadIdx.x; i <= nc; i += blockDim.x) srp[i] = rp[c0 + i];
    __syncthreads();
    for (int w0 = 0; w0 < nc; w0 += kFillWinRows) {
      const int nr = nc - w0 < kFillWinRows ? nc - w0 : kFillWinRows;
      const int64_t* wrp = srp + w0;
      const int64_t g0 = c0 + w0;
      const int64_t e0 = wrp[0], e1 = wrp[nr];
      if (w0 > 0) __syncthreads();  // the previous window's C is done with cur and mask
      if (e1 - e0 <= (int64_t)kFillK * kFillThreads) {
        // the window's entries in registers: one round of loads, then the
        // three steps on shared memory only
        int cc[kFillK], rr[kFillK];
        VT dv[kFillK], lv[kFillK];
#pragma unroll
        for (int k = 0; k < kFillK; ++k) {
          const int64_t p = e0 + threadIdx.x + (int64_t)k * kFillThreads;
          cc[k] = -1;
          if (p < e1) {
            cc[k] = col[p];
            dv[k] = Dv[p];
            lv[k] = Lv[p];
            rr[k] = fill_win_row(wrp, nr, p);
          }
        }
#pragma unroll
        for (int k = 0; k < kFillK; ++k)
          if (cc[k] >= 0) atomicOr(&mask[cc[k] >> 1], 1u << ((cc[k] & 1) * 16 + rr[k]));
        __syncthreads();
        uint32_t mk[kFillK];
#pragma unroll
        for (int k = 0; k < kFillK; ++k) {
          if (cc[k] < 0) continue;
          const int c = cc[k], r = rr[k];
          mk[k] = (mask[c >> 1] >> ((c & 1) * 16)) & 0xffffu;
          const int32_t pos = cur[c] + __popc(mk[k] & ((1u << r) - 1u));
          if (rec) {
            rec[pos] = fill_rec((int32_t)(g0 + r), dv[k], lv[k]);
          } else {
            row_out[pos] = (int32_t)(g0 + r);
            DT[pos] = dv[k];
            LT[pos] = lv[k];
          }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kFillK; ++k) {
          if (cc[k] < 0) continue;
          const int c = cc[k];
          if ((mk[k] & ((1u << rr[k]) - 1u)) == 0u) {  // the column's first row in the window
            cur[c] += __popc(mk[k]);
            atomicAnd(&mask[c >> 1], ~(0xffffu << ((c & 1) * 16)));
          }
        }
        continue;
      }
      // A: the window rows that hold each column
      for (int64_t p = e0 + threadIdx.x; p < e1; p += kFillThreads) {
        const int c = col[p];
        const int r = fill_win_row(wrp, nr, p);
        atomicOr(&mask[c >> 1], 1u << ((c & 1) * 16 + r));
      }
      __syncthreads();
      // B: each entry to its place
      for (int64_t p = e0 + threadIdx.x; p < e1; p += kFillThreads) {
        const int c = col[p];
        const int r = fill_win_row(wrp, nr, p);
        const uint32_t m = (mask[c >> 1] >> ((c & 1) * 16)) & 0xffffu;
        const int32_t pos = cur[c] + __popc(m & ((1u << r) - 1u));
        if (rec) {
          rec[pos] = fill_rec((int32_t)(g0 + r), Dv[p], Lv[p]);
        } else {
          row_out[pos] = (int32_t)(g0 + r);
          DT[pos] = Dv[p];
          LT[pos] = Lv[p];
        }
      }
      __syncthreads();
      // C: advance the cursors past the window, clear the masks
      for (int64_t p = e0 + threadIdx.x; p < e1; p += kFillThreads) {
        const int c = col[p];
        const int r = fill_win_row(wrp, nr, p);
        const uint32_t m = (mask[c >> 1] >> ((c & 1) * 16)) & 0xffffu;
        if ((m & ((1u << r) - 1u)) == 0u) {  // the column's first row in the window
          cur[c] += __popc(m);
          atomicAnd(&mask[c >> 1], ~(0xffffu << ((c & 1) * 16)));
        }
      }
    }
  }
}

template <typename VT>
size_t csc_fill_win_smem(int32_t n_cols) {
  return (((size_t)n_cols * sizeof(int32_t) + (size_t)((n_cols + 1) / 2) * sizeof(uint32_t) + 15) & ~(size_t)15) +
         (kFillRows + 1) * sizeof(int64_t);
}

// Window length W (a multiple of kFillAlign, at most 8192) from the shared
// memory left after the row-pointer chunk and, when they fit with W >= 1024,
// the block's cursors.
template <typename VT>
static void fill_inst(const Geometry& g, const int64_t* rp, const int32_t* col, const void* Dv, const void* Lv,
                      const int64_t* blk_row, int n_blk, int32_t n_cols, int32_t* cursor, int32_t* row_out,
                      void* DT, void* LT, int* err, void* rec, int64_t n_out, cudaStream_t s) {
  const size_t limit = g.smem_limit;
  if (FO_FILL_WIN && csc_fill_win_smem<VT>(n_cols) <= limit) {
    using R = typename FillRec<VT>::T;
    const size_t smem = csc_fill_win_smem<VT>(n_cols);
    cudaFuncSetAttribute(k_csc_fill_win<VT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_csc_fill_win<VT><<<n_blk, kFillThreads, smem, s>>>(rp, col, (const VT*)Dv, (const VT*)Lv, blk_row, n_cols,
                                                          cursor, row_out, (VT*)DT, (VT*)LT, (R*)rec);
    if (rec && n_out > 0)
      k_csc_split<VT><<<(unsigned)((n_out + 255) / 256), 256, 0, s>>>((const R*)rec, n_out, row_out, (VT*)DT,
                                                                       (VT*)LT);
    return;
  }
  const size_t per_w = 2 * (sizeof(int32_t) + 2 * sizeof(VT));
  auto w_for = [&](bool sc) -> int {
    const size_t fixed = csc_fill_smem<VT>(0, n_cols, sc);
    if (fixed >= limit) return 0;
    const size_t w = std::min<size_t>((limit - fixed) / per_w, 8192) & ~(size_t)(kFillAlign - 1);
    return (int)w;
  };
  bool sc = true;
  int W = w_for(true);
  if (W < 1024) {
    sc = false;
    W = w_for(false);
  }
  const size_t smem = csc_fill_smem<VT>(W, n_cols, sc);
  if (sc) {
    cudaFuncSetAttribute(k_csc_fill<VT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_csc_fill<VT, true><<<n_blk, kFillThreads, smem, s>>>(rp, col, (const VT*)Dv, (const VT*)Lv, blk_row, n_cols,
                                                            cursor, row_out, (VT*)DT, (VT*)LT, W, err);
  } else {
    cudaFuncSetAttribute(k_csc_fill<VT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_csc_fill<VT, false><<<n_blk, kFillThreads, smem, s>>>(rp, col, (const VT*)Dv, (const VT*)Lv, blk_row, n_cols,
                                                             cursor, row_out, (VT*)DT, (VT*)LT, W, err);
  }
}

size_t csc_fill_rec_bytes(const Geometry& g, int fmt, int32_t n_cols) {
  if (!FO_FILL_WIN || !FO_FILL_REC) return 0;
  if (fmt == 0) return csc_fill_win_smem<float>(n_cols) <= g.smem_limit ? sizeof(int4) : 0;
  return csc_fill_win_smem<uint16_t>(n_cols) <= g.smem_limit ? sizeof(uint2) : 0;
}

void launch_csc_fill(const Geometry& g, int fmt, const int64_t* rp, const int32_t* col, const void* Dv,
                     const void* Lv, const int64_t* blk_row, int n_blk, int32_t n_cols, int32_t* cursor,
                     int32_t* row_out, void* DT, void* LT, int* err, void* rec, int64_t n_out, cudaStream_t s) {
  if (fmt == 0)
    fill_inst<float>(g, rp, col, Dv, Lv, blk_row, n_blk, n_cols, cursor, row_out, DT, LT, err, rec, n_out, s);
  else
    fill_inst<uint16_t>(g, rp, col, Dv, Lv, blk_row, n_blk, n_cols, cursor, row_out, DT, LT, err, rec, n_out, s);
}

void launch_dequant_csc(int fmt, const int64_t* cp, int32_t n_cols, const int32_t* row, const void* DT,
                        const void* LT, const float* sD, const float* sL, float* Dout, float* Lout,
                        cudaStream_t s) {
  const unsigned gb = grid_for(n_cols, 8, 65535);
  if (fmt == 1)
    k_dequant_csc<__nv_bfloat16><<<gb, 256, 0, s>>>(cp, n_cols, row, (const __nv_bfloat16*)DT,
                                                     (const __nv_bfloat16*)LT, sD, sL, Dout, Lout);
  else if (fmt == 2)
    k_dequant_csc<__half><<<gb, 256, 0, s>>>(cp, n_cols, row, (const __half*)DT, (const __half*)LT, sD,
                                              sL, Dout, Lout);
  else
    k_dequant_csc<float><<<gb, 256, 0, s>>>(cp, n_cols, row, (const float*)DT, (const float*)LT, sD,
                                             sL, Dout, Lout);
}

void launch_scale_coef(int64_t n, const float* aD, const float* aL, const int64_t* voxel,
                       const float* sD, const float* sL, float2* coef, cudaStream_t s) {
  if (n == 0) return;
  k_scale_coef<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, aD, aL, voxel, sD, sL, coef);
}

// ------------------------------------------------------------------ init

template <typename VT, int EPI, typename IT>
static cudaError_t set_smem_attr_it(int bytes) {
  cudaError_t e = cudaFuncSetAttribute(k_forward<VT, EPI, true, false, IT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  if (EPI != EPI_FINAL)
    e = cudaFuncSetAttribute(k_forward<VT, EPI, true, true, IT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}
template <typename VT, int EPI>
static cudaError_t set_smem_attr(int bytes) {
  cudaError_t e = set_smem_attr_it<VT, EPI, int32_t>(bytes);
  if (e != cudaSuccess) return e;
  return set_smem_attr_it<VT, EPI, uint16_t>(bytes);
}

template <typename VT>
static cudaError_t set_smem_all(int bytes) {
  cudaError_t e;
  if ((e = set_smem_attr<VT, EPI_STORE>(bytes)) != cudaSuccess) return e;
  if ((e = set_smem_attr<VT, EPI_OBJ>(bytes)) != cudaSuccess) return e;
  if ((e = set_smem_attr<VT, EPI_BC>(bytes)) != cudaSuccess) return e;
  return set_smem_attr<VT, EPI_FINAL>(bytes);
}

cudaError_t kernel_arch(int* fwd_binary, int* bwd_binary, int* ptx_version) {
  cudaFuncAttributes fa, ba;
  cudaError_t e = cudaFuncGetAttributes(&fa, k_forward<float, EPI_OBJ, true, true, uint16_t>);
  if (e != cudaSuccess) return e;
  e = cudaFuncGetAttributes(&ba, k_backward<float, true, true, true>);
  if (e != cudaSuccess) return e;
  if (fwd_binary) *fwd_binary = fa.binaryVersion;
  if (bwd_binary) *bwd_binary = ba.binaryVersion;
  if (ptx_version) *ptx_version = fa.ptxVersion;
  return cudaSuccess;
}

int init_kernels(Geometry* g, int device) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return -1;
  g->n_sms = prop.multiProcessorCount;
  g->smem_limit = prop.sharedMemPerBlockOptin;
  g->fwd_threads = kFwdThreads;
  // 1024 threads per SM: one CTA when x is staged in shared memory (120 KB
  // for 30000 spots); smaller CTAs only when it is read through L1 instead
  g->fwd_blocks = g->n_sms * (FO_FWD_XS ? 1 : 1024 / kFwdThreads);
  g->fwd_warps = g->fwd_blocks * (kFwdThreads / 32);
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_backward<float, true, true, false>, kBwdThreads, 0);
  if (occ < 1) occ = 1;
  g->bwd_threads = kBwdThreads;
  g->bwd_blocks = g->n_sms * occ;
  g->bwd_warps = g->bwd_blocks * (kBwdThreads / 32);
  g->row_threads = kRowThreads;
  g->row_blocks = g->n_sms * 4;
  g->col_threads = kColThreads;
  g->col_blocks = g->n_sms * 2;
  const int bytes = (int)g->smem_limit;
  if (set_smem_all<float>(bytes) != cudaSuccess) return -2;
  if (set_smem_all<__nv_bfloat16>(bytes) != cudaSuccess) return -2;
  if (set_smem_all<__half>(bytes) != cudaSuccess) return -2;
  return 0;
}

// ------------------------------------------------------------------ block-iterative sweep

// x = w + coef * g (the perturbed point; coef = 0 without perturbation), and
// the sweep's violation counters cleared.
__global__ void k_sweep_start(int n, const float* __restrict__ w, const float* __restrict__ g, int use_coef,
                              float* __restrict__ x, DevState* st) {
  const double coef = use_coef ? st->coef : 0.0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    x[j] = use_coef ? (float)((double)w[j] + coef * (double)g[j]) : w[j];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->sweep_nv = 0.0;
    st->sweep_mx = 0.0;
  }
}

// pos[t * n + j] = first CSC position of column j whose row is >= bounds[t].
__global__ void k_sweep_pos(const int64_t* __restrict__ cp, const int32_t* __restrict__ row, int32_t n,
                            const int64_t* __restrict__ bounds, int n_bounds, int64_t* __restrict__ pos) {
  const int64_t total = (int64_t)n_bounds * n;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(idx / n);
    const int j = (int)(idx - (int64_t)t * n);
    const int64_t target = bounds[t];
    int64_t lo = cp[j], hi = cp[j + 1];
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if ((int64_t)row[mid] < target) lo = mid + 1;
      else hi = mid;
    }
    pos[idx] = lo;
  }
}

// One block of the sweep: u_j = sum over the block's CSC entries of column j
// of D_ij gamma_D[i] + L_ij gamma_L[i] (one warp per column, fixed order), then
// x_j += lam * scale / W_B * u_j.  W_B and the violation counts come from the
// block's constraint partials.
template <typename VT>
__global__ void __launch_bounds__(256) k_sweep_update(SweepArgs a) {
  __shared__ double red[256];
  __shared__ double sh_scale;
  const double W = block_sum_array(a.k2part + (a.norm == 1 ? 0 : 3 * a.k2_blocks), a.k2_blocks, red);
  if (a.in_solve && blockIdx.x == 0) {
    const double nv = block_count_array(a.k2part + a.k2_blocks, a.k2_blocks, red);
    const double mx = block_max_array(a.k2part + 2 * a.k2_blocks, a.k2_blocks, red);
    if (threadIdx.x == 0) {
      a.st->sweep_nv += nv;
      a.st->sweep_mx = fmax(a.st->sweep_mx, mx);
    }
  }
  if (threadIdx.x == 0) {
    const double ps = a.in_solve ? (a.st->eta == 1.0 ? 1.0 : pow(a.st->eta, (double)a.st->k)) : a.prio_scale;
    sh_scale = W > 0.0 ? a.lam * ps / W : 0.0;
  }
  __syncthreads();
  const double scale = sh_scale;
  if (scale == 0.0) return;
  const VT* __restrict__ Dv = reinterpret_cast<const VT*>(a.Dv);
  const VT* __restrict__ Lv = reinterpret_cast<const VT*>(a.Lv);
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < a.n; j += nw) {
    const int64_t p0 = a.pos0[j], p1 = a.pos1[j];
    if (p1 <= p0) continue;
    float acc = 0.0f;
    for (int64_t p = p0 + lane; p < p1; p += 32) {
      const float2 c = a.gam[a.row[p]];
      acc = fmaf(to_f(Dv[p]), c.x, acc);
      acc = fmaf(to_f(Lv[p]), c.y, acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) a.x[j] = (float)((double)a.x[j] + scale * (double)acc);
  }
}

// out = max(0, x); in a solve the last block writes the log entry and advances k.
__global__ void __launch_bounds__(256) k_sweep_finish(int n, const float* __restrict__ x, float* __restrict__ out,
                                                      int in_solve, DevState* st, LogEntry* log) {
  __shared__ bool sh_last;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    out[j] = x[j] > 0.0f ? x[j] : 0.0f;
  if (!in_solve) return;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&st->done, 1u);
    sh_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (sh_last && threadIdx.x == 0) {
    __threadfence();
    if (st->log_cap > 0) {
      LogEntry e;
      e.k = st->k;
      e.s = st->s;
      e.accepted = st->accepted;
      e.n_violated = (int)st->sweep_nv;
      e.beta = st->beta_acc;
      e.f_start = st->f_start;
      e.f_end = st->f_cur;
      e.gnorm = st->gnorm;
      e.max_violation = st->sweep_mx;
      log[st->k % st->log_cap] = e;
    }
    st->k += 1;
    st->done = 0u;
  }
}

void launch_sweep_start(int n, const float* w, const float* g, int use_coef, float* x, DevState* st,
                        cudaStream_t s) {
  k_sweep_start<<<std::max(1, std::min(1024, (n + 255) / 256)), 256, 0, s>>>(n, w, g, use_coef, x, st);
}

void launch_sweep_pos(const int64_t* cp, const int32_t* row, int32_t n, const int64_t* bounds, int n_bounds,
                      int64_t* pos, cudaStream_t s) {
  const int64_t total = (int64_t)n_bounds * n;
  if (total == 0) return;
  const unsigned gb = (unsigned)std::min<int64_t>((total + 255) / 256, 65535);
  k_sweep_pos<<<gb, 256, 0, s>>>(cp, row, n, bounds, n_bounds, pos);
}

void launch_sweep_update(const Geometry& g, int fmt, const SweepArgs& a, cudaStream_t s) {
  const unsigned gb = (unsigned)std::max(1, std::min(g.n_sms * 8, (a.n + 7) / 8));
  if (fmt == 1)
    k_sweep_update<__nv_bfloat16><<<gb, 256, 0, s>>>(a);
  else if (fmt == 2)
    k_sweep_update<__half><<<gb, 256, 0, s>>>(a);
  else
    k_sweep_update<float><<<gb, 256, 0, s>>>(a);
}

void launch_sweep_finish(const Geometry& g, int n, const float* x, float* out, int in_solve, DevState* st,
                         LogEntry* log, cudaStream_t s) {
  const unsigned gb = (unsigned)std::max(1, std::min(g.n_sms, (n + 255) / 256));
  k_sweep_finish<<<gb, 256, 0, s>>>(n, x, out, in_solve, st, log);
}

__global__ void __launch_bounds__(256) k_narrow_idx(const int4* __restrict__ in, uint2* __restrict__ out, int64_t n4) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
    const int4 v = __ldcs(in + i);
    out[i] = make_uint2(((uint32_t)v.x & 0xffffu) | ((uint32_t)v.y << 16),
                        ((uint32_t)v.z & 0xffffu) | ((uint32_t)v.w << 16));
  }
}

void launch_narrow_idx(const int32_t* in, uint16_t* out, int64_t n, cudaStream_t s) {
  const int64_t n4 = n / 4;
  if (n4 == 0) return;
  const unsigned grid = (unsigned)std::min<int64_t>((n4 + 255) / 256, 152 * 8);
  k_narrow_idx<<<grid, 256, 0, s>>>(reinterpret_cast<const int4*>(in), reinterpret_cast<uint2*>(out), n4);
}

// Based 16-bit row indices of the CSC (see BlockBase): one warp per block of
// 128 elements.  Pass 1 writes the block's base and offsets when its rows
// span less than 65536, else marks it -1 and counts it; pass 2 gives every
// marked block an overflow slot and copies its 128 int32 rows there.
__global__ void __launch_bounds__(256) k_narrow_rows(const int32_t* __restrict__ row, int64_t n_blk,
                                                     uint16_t* __restrict__ row16, int32_t* __restrict__ hdr,
                                                     unsigned int* n_wide) {
  const int lane = threadIdx.x & 31;
  const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n_blk; k += wstride) {
    const int4 v = __ldg(reinterpret_cast<const int4*>(row + k * 128) + lane);
    int lo = min(min(v.x, v.y), min(v.z, v.w)), hi = max(max(v.x, v.y), max(v.z, v.w));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = min(lo, __shfl_xor_sync(kFull, lo, o));
      hi = max(hi, __shfl_xor_sync(kFull, hi, o));
    }
    if ((int64_t)hi - (int64_t)lo < 65536) {
      reinterpret_cast<uint2*>(row16 + k * 128)[lane] =
          make_uint2((uint32_t)(v.x - lo) | ((uint32_t)(v.y - lo) << 16),
                     (uint32_t)(v.z - lo) | ((uint32_t)(v.w - lo) << 16));
      if (lane == 0) hdr[k] = lo;
    } else {
      reinterpret_cast<uint2*>(row16 + k * 128)[lane] = make_uint2(0u, 0u);
      if (lane == 0) {
        hdr[k] = -1;
        atomicAdd(n_wide, 1u);
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_narrow_rows_wide(const int32_t* __restrict__ row, int64_t n_blk,
                                                          int32_t* __restrict__ hdr, int32_t* __restrict__ ovf,
                                                          unsigned int* slot, unsigned int n_wide) {
  const int lane = threadIdx.x & 31;
  const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n_blk; k += wstride) {
    if (hdr[k] != -1) continue;
    unsigned j = 0;
    if (lane == 0) j = atomicAdd(slot, 1u);
    j = __shfl_sync(kFull, j, 0);
    if (j >= n_wide) continue;  // cannot happen: pass 1 counted every marked block
    reinterpret_cast<int4*>(ovf + (int64_t)j * 128)[lane] = __ldg(reinterpret_cast<const int4*>(row + k * 128) + lane);
    __syncwarp();
    if (lane == 0) hdr[k] = -1 - (int32_t)j;
  }
}

void launch_narrow_rows(const int32_t* row, int64_t n_blk, uint16_t* row16, int32_t* hdr, unsigned int* n_wide,
                        cudaStream_t s) {
  if (n_blk == 0) return;
  const unsigned grid = (unsigned)std::min<int64_t>((n_blk + 7) / 8, 152 * 8);
  k_narrow_rows<<<grid, 256, 0, s>>>(row, n_blk, row16, hdr, n_wide);
}

void launch_narrow_rows_wide(const int32_t* row, int64_t n_blk, int32_t* hdr, int32_t* ovf, unsigned int* slot,
                             unsigned int n_wide, cudaStream_t s) {
  if (n_blk == 0 || n_wide == 0) return;
  const unsigned grid = (unsigned)std::min<int64_t>((n_blk + 7) / 8, 152 * 8);
  k_narrow_rows_wide<<<grid, 256, 0, s>>>(row, n_blk, hdr, ovf, slot, n_wide);
}

// Failure detection without a fault: one CTA polls an mbarrier phase with the
// same bounded wait the bulk copies use.  With `arrive` set, thread 0 arrives
// first and the phase completes; otherwise nothing arrives, every poll fails,
// and after `spins` polls the CTA records the give-up in the error word and
// returns.  No copy is ever issued on this barrier.
__global__ void k_wait_check(int arrive, int spins, DevState* st) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (arrive && threadIdx.x == 0) mbar_expect_tx(&bar, 0u);
  if (!mbar_wait(&bar, 0, spins) && threadIdx.x == 0) atomicOr(&st->err, 1);
}

void launch_wait_check(int arrive, int spins, DevState* st, cudaStream_t s) {
  k_wait_check<<<1, 32, 0, s>>>(arrive, spins > 0 ? spins : kMbarSpins, st);
}

}  // namespace fo
