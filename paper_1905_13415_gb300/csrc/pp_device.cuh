// pp_device.cuh -- device-side building blocks of the GB300 ParPaRaw parser.
//
// Inline PTX for sm_103a (TMA bulk copies through mbarriers, acquire/release
// accesses for the decoupled look-back, %globaltimer for bounded waits), the
// packed state-transition vector with its composite operator (Sec. 3.1), warp
// and block scans, and the look-back over tile status words (single-pass
// scan after Merrill & Garland, which the paper builds on, Sec. 2).
#pragma once
#include <cstdint>

#include "pp_types.h"

namespace pp {

// ------------------------------------------------------------------ PTX ---

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// global -> shared bulk copy (TMA, non-tensor); 16-byte aligned, size % 16 == 0
__device__ __forceinline__ void tma_load_1d(void* sdst, const void* gsrc, uint32_t bytes,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(sdst)),
      "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// global -> L2 bulk prefetch (no destination, no completion); 16-byte
// aligned, size % 16 == 0
__device__ __forceinline__ void prefetch_l2_bulk(const void* gsrc, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(gsrc), "r"(bytes) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ------------------------------------------------------------- bit masks ---

__device__ __forceinline__ uint64_t bits_below(int n) {
  return n <= 0 ? 0ull : (n >= 64 ? ~0ull : ((1ull << n) - 1ull));
}
// bits [lo, hi) of a 64-bit word (both may fall outside 0..64)
__device__ __forceinline__ uint64_t bit_range(int lo, int hi) {
  return bits_below(hi) & ~bits_below(lo);
}

// ------------------------------------------- state-transition vectors ---
//
// A vector (Sec. 3.1) holds, for every start state i < 8, the state reached
// after a chunk; entry i is byte i of a 64-bit word (values < 8).  The
// composite a o b ("a's chunk, then b's", (a o b)_i = b[a_i]) is two byte
// permutes whose selectors are a's entries packed as nibbles.

constexpr uint64_t kIdentityVec = 0x0706050403020100ull;

// entries e0..e3 (bytes) -> nibbles in bits 0..15; bits 16..31 are not defined
__device__ __forceinline__ uint32_t nibble_selector(uint32_t bytes4) {
  uint32_t y = bytes4 | (bytes4 >> 4);  // byte0 = e0 | e1<<4, byte2 = e2 | e3<<4
  return __byte_perm(y, 0u, 0x0020u);
}
__device__ __forceinline__ uint64_t vcompose(uint64_t a, uint64_t b) {
  const uint32_t blo = static_cast<uint32_t>(b), bhi = static_cast<uint32_t>(b >> 32);
  const uint32_t rlo = __byte_perm(blo, bhi, nibble_selector(static_cast<uint32_t>(a)));
  const uint32_t rhi = __byte_perm(blo, bhi, nibble_selector(static_cast<uint32_t>(a >> 32)));
  return (static_cast<uint64_t>(rhi) << 32) | rlo;
}
__device__ __forceinline__ uint32_t vget(uint64_t v, uint32_t i) {
  return static_cast<uint32_t>(v >> (8 * i)) & 0xFFu;
}
// 32-bit nibble form of a vector, for status words
__device__ __forceinline__ uint32_t vpack(uint64_t v) {
  return (nibble_selector(static_cast<uint32_t>(v)) & 0xFFFFu) |
         (nibble_selector(static_cast<uint32_t>(v >> 32)) << 16);
}
__device__ __forceinline__ uint32_t nib4_to_bytes(uint32_t x) {
  x &= 0xFFFFu;
  x = (x | (x << 8)) & 0x00FF00FFu;
  x = (x | (x << 4)) & 0x0F0F0F0Fu;
  return x;
}
__device__ __forceinline__ uint64_t vunpack(uint32_t p) {
  return (static_cast<uint64_t>(nib4_to_bytes(p >> 16)) << 32) | nib4_to_bytes(p);
}

// --------------------------------------------- record / column offsets ---
//
// Per chunk: the records it closes and its column offset, absolute (the chunk
// has a record delimiter: field delimiters after the last one) or relative
// (field delimiters seen).  The scan operator (Sec. 3.2) keeps b when b is
// absolute, else adds b's offset to a's; counts saturate at kColSat.

constexpr uint32_t kColSat = 0x7FFFu;

// block-level packing (32 bits): [31] abs, [30:16] column offset, [15:0] records
__device__ __forceinline__ uint32_t rc_pack(uint32_t rec, uint32_t col, bool abs) {
  return (abs ? 0x80000000u : 0u) | (min(col, kColSat) << 16) | rec;
}
__device__ __forceinline__ uint32_t rc_combine(uint32_t a, uint32_t b) {
  const uint32_t rec = (a & 0xFFFFu) + (b & 0xFFFFu);
  uint32_t colpart;
  if (b & 0x80000000u) {
    colpart = b & 0xFFFF0000u;
  } else {
    const uint32_t col = min(((a >> 16) & kColSat) + ((b >> 16) & kColSat), kColSat);
    colpart = (a & 0x80000000u) | (col << 16);
  }
  return colpart | (rec & 0xFFFFu);
}

// tile-level packing (62 bits payload): [61] abs, [60:40] column, [39:0] records
constexpr uint64_t kRecMask = (1ull << 40) - 1;
__device__ __forceinline__ uint64_t tc_pack(uint64_t rec, uint32_t col, bool abs) {
  return (abs ? (1ull << 61) : 0ull) | (static_cast<uint64_t>(min(col, kColSat)) << 40) |
         (rec & kRecMask);
}
__device__ __forceinline__ uint64_t tc_combine(uint64_t a, uint64_t b) {
  const uint64_t rec = ((a & kRecMask) + (b & kRecMask)) & kRecMask;
  if (b & (1ull << 61)) return (b & ~kRecMask) | rec;
  const uint32_t col =
      min(static_cast<uint32_t>((a >> 40) & 0x1FFFFF) + static_cast<uint32_t>((b >> 40) & 0x1FFFFF),
          kColSat);
  return (a & (1ull << 61)) | (static_cast<uint64_t>(col) << 40) | rec;
}

// ------------------------------------------------------------ warp scans ---

template <class T, class Op>
__device__ __forceinline__ T warp_inclusive_scan(T v, Op op, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const T o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v = op(o, v);
  }
  return v;
}

// Block-wide exclusive scan of one value per thread with an associative
// (not necessarily commutative) operator.  `wsum` is NT/32 words of shared
// memory; the caller separates successive uses with __syncthreads().
template <int NT, class T, class Op>
__device__ __forceinline__ T block_exclusive_scan(T v, Op op, T identity, T* wsum, T* total) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T inc = warp_inclusive_scan(v, op, lane);
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T w = lane < NW ? wsum[lane] : identity;
    w = warp_inclusive_scan(w, op, lane);
    if (lane < NW) wsum[lane] = w;
  }
  __syncthreads();
  T ex = __shfl_up_sync(0xffffffffu, inc, 1);
  if (lane == 0) ex = identity;
  const T wp = warp > 0 ? wsum[warp - 1] : identity;
  *total = wsum[NW - 1];
  return warp > 0 ? op(wp, ex) : ex;
}


}  // namespace pp
