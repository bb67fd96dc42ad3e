// pp_kernel.cuh -- the single-pass ParPaRaw tile kernel for sm_103a.
//
// One block owns one tile of T = NT * B input bytes at a time (B = 16 * VPT
// bytes per thread, the paper's per-thread chunk, Sec. 3) and takes tiles
// from a device work counter, so a tile's predecessors always belong to
// blocks that are already running.  Per tile:
//
//   load    TMA bulk copy of the tile into shared memory (ragged ends by
//           plain loads); 16-byte vector reads per thread.  The tile a block
//           will take one tile-time later is bulk-prefetched into L2.
//   a1, a2  symbol matching (SWAR zero-byte tests against the symbols,
//           Sec. 4.5) and multi-state simulation of the chunk: one DFA
//           instance per state, packed as a state-transition vector
//           (Sec. 3.1).  Runs of catch-all symbols collapse into one
//           transition when the catch-all transition is idempotent.
//   a3      exclusive o-scan of the vectors: block scan, then decoupled
//           look-back over the tiles' status words (chain 1).
//   a4      re-simulation from the chunk's start state emitting the data /
//           field / record / control tags as bit masks (Sec. 3.1).
//   a5      record counts (popcount), absolute/relative column offsets, data
//           bytes and delimiters per chunk (Sec. 3.2): one block scan, then
//           look-back (chain 2) for the tile's first record and column.
//           The field list: every delimiter of the tile (and the open field
//           after the last one) becomes an entry with its end, column and
//           record; per-column string bytes summed over equal shares of the
//           entries, block-scanned, then look-back (chain 3) for each
//           column's output base.  Tiles with more fields than the list
//           holds are processed in rounds.
//   a6      stable partition (Sec. 3.3): over equal shares of the entries,
//           each string field's running offset and its data bytes straight
//           from the tile to the column (long fields queued, then copied in
//           512-byte pieces taken by free warps, 16-byte stores); Arrow
//           int64 offsets per record.
//   a7      numeric fields are converted by G threads per record (G chosen
//           per round to balance the threads), lanes of a warp on
//           consecutive records, column by column (Sec. 3.3).
//   a8      invalid transitions, field-count mismatches and conversion
//           failures are recorded; the finalize kernel turns them into
//           validity bitmaps and the result.
//
// Every spin (mbarrier, look-back) is bounded by %globaltimer and reports
// PP_E_TIMEOUT instead of hanging.
#pragma once
#include <cstddef>
#include <cstdint>

#include "pp_convert.cuh"
#include "pp_device.cuh"
#include "pp_types.h"

// Opt-in instrumentation (profiling builds only, -DPP_PHASE_TIMING): thread 0
// accumulates the cycles between block-wide synchronisation points per phase
// (counters 0-15); every warp times its own share of a step between two
// marks, and each tile adds the slowest warp's time (16 + s) and the sum
// over warps (24 + s) of span s.
#ifdef PP_PHASE_TIMING
#define PP_PHASE(k)                        \
  do {                                     \
    if (tid == 0) {                        \
      const long long _now = clock64();    \
      H->ph_cycles[k] += _now - ph_last;   \
      ph_last = _now;                      \
    }                                      \
  } while (0)
#define PP_WMARK() \
  do {             \
    __syncwarp();  \
    w_t0 = clock64(); \
  } while (0)
#define PP_WSPAN(s)                                                              \
  do {                                                                           \
    __syncwarp();                                                                \
    if (lane == 0) {                                                             \
      const unsigned long long _d = static_cast<unsigned long long>(clock64() - w_t0); \
      atomicMax(&H->w_max[s], _d);                                               \
      atomicAdd(&H->w_sum[s], _d);                                               \
    }                                                                            \
  } while (0)
#else
#define PP_PHASE(k) \
  do {              \
  } while (0)
#define PP_WMARK() \
  do {             \
  } while (0)
#define PP_WSPAN(s) \
  do {              \
  } while (0)
#endif

namespace pp {

template <int NT_, int VPT_, int MINB_ = 1>
struct TileShape {
  static constexpr int NT = NT_;
  static constexpr int VPT = VPT_;
  static constexpr int MINB = MINB_;       // resident blocks per SM asked of ptxas
  static constexpr int B = 16 * VPT;       // bytes per thread (chunk)
  static constexpr int T = NT * B;         // bytes per tile
  static constexpr int MW = (B + 63) / 64; // 64-bit mask words per chunk
  static constexpr int NW = NT / 32;
  static_assert(T < 65536, "tile positions are 16-bit field-list entries");
};

// A field-list entry: [15:0] the field's end position in the tile (its
// delimiter, or the tile's end for the open field), [23:16] its column
// (saturated), [24] the open field (after the tile's last delimiter), [25]
// the field ends a record.
constexpr uint32_t kEntPos = 0xFFFFu;
constexpr uint32_t kEntOpen = 1u << 24;
constexpr uint32_t kEntRec = 1u << 25;

// A piece of a long string field, copied by whichever warp is free; 16
// bytes, so that a warp reads it with one shared-memory vector load.
//   dst  contiguous piece: destination of its first byte; gapped: the
//        field's destination
//   x0   first tile position of the piece
//   len  contiguous piece: bytes; gapped: tile positions it spans
//   fd   gapped: the field's first data position (ranks count from it);
//        kContiguousPiece for a contiguous piece
//   nb   gapped: the field's data bytes (the destination's extent)
struct alignas(16) Piece {
  uint8_t* dst;
  uint16_t x0, len, fd, nb;
};
static_assert(sizeof(Piece) == 16, "one 16-byte load per piece");
constexpr uint16_t kContiguousPiece = 0xFFFF;
constexpr uint32_t kMaxPieces = 128;  // pieces queued per round (fields that do not fit are copied where found)
constexpr uint32_t kPiece = 512;  // queued long fields are copied in pieces of this many tile bytes

struct SmemHead {
  uint64_t mbar;
  unsigned long long item;
  uint32_t job;
  int32_t tables_loaded;
  uint64_t prefix_vec;   // chain 1 exclusive prefix of this tile
  uint64_t prefix_rc;    // chain 2 exclusive prefix of this tile
  int64_t col_base[PP_MAX_STRING_COLUMNS];   // chain 3 exclusive prefix
  uint32_t tile_tot[PP_MAX_STRING_COLUMNS];
  uint64_t wsum64[32];
  uint32_t wsum32[32];
  uint32_t wsumk[PP_MAX_STRING_COLUMNS / 2][32];
  Tables tab;
  uint8_t str_col[PP_MAX_STRING_COLUMNS];  // slot -> column
  int32_t job_loaded;
  unsigned long long tile_last_rd;  // partial inputs: last record delimiter + 1
  uint32_t eof_rd;                  // the input's last byte is a record delimiter
  // field list of the current round (fields [f0, f0 + nwin) of the tile)
  int32_t prev_pos;      // end of field f0 - 1 (the start of the tile's data - 1 for f0 = 0)
  uint32_t rr0;          // record of field f0, relative to the tile's first record
  uint32_t rr_last;      // record of the round's last field
  int32_t next_prev_pos;
  uint32_t rr_next;
  uint32_t round_tot[PP_MAX_STRING_COLUMNS];   // string bytes of the round per slot
  uint32_t round_base[PP_MAX_STRING_COLUMNS];  // string bytes of the earlier rounds
  uint32_t npieces;       // pieces claimed in the queue
  uint32_t npieces_ok;    // pieces written (a prefix of the queue)
  uint32_t w2_g;         // threads per record of the round's step (2)
  uint32_t piece_next;   // the next long-field piece to copy
  uint32_t w2_next;      // the next run of step (2) work items
  alignas(16) Piece pieces[kMaxPieces];  // read with 16-byte loads
#ifdef PP_PHASE_TIMING
  long long ph_cycles[32];  // profiling builds only
  unsigned long long w_max[8], w_sum[8];
#endif
  Job jd;                  // the current job and its columns, staged from the
  Col cd[PP_MAX_COLUMNS];  // launch parameters / global memory once per job
};

static_assert(offsetof(SmemHead, pieces) % 16 == 0, "16-byte loads of the piece queue");

template <class Shape>
struct SmemLayout {
  static constexpr size_t kHead = (sizeof(SmemHead) + 127) & ~size_t(127);
  static constexpr size_t kTile = kHead;
  static constexpr size_t kDm = kTile + ((Shape::T + 64 + 127) & ~size_t(127));
  static constexpr size_t kCnt = kDm + sizeof(uint64_t) * Shape::NT * Shape::MW;
  static constexpr size_t kDex = kCnt + sizeof(uint16_t) * Shape::NT * PP_MAX_STRING_COLUMNS;
  static constexpr size_t kFe = kDex + ((sizeof(uint16_t) * (Shape::NT + 1) + 15) & ~size_t(15));
  // Field-list capacity: what an SM's shared memory (228 KB, 1 KB reserved
  // per block) leaves at the shape's residency (at least 2 blocks), within
  // [T/32, T/4] and at most 4960 entries of 8 bytes.  Tiles with more fields
  // are processed in rounds.
  static constexpr int kBlocks = Shape::MINB > 2 ? Shape::MINB : 2;
  static constexpr long kPerBlock = 233472 / kBlocks - 1024;
  static constexpr long kFit = (kPerBlock - static_cast<long>(kFe)) / 8;
  static constexpr long kLo = kFit > Shape::T / 32 ? kFit : Shape::T / 32;
  static constexpr long kHi = Shape::T / 4 < 4960 ? Shape::T / 4 : 4960;
  static constexpr int kFcap = static_cast<int>(((kLo < kHi ? kLo : kHi) & ~31L) < 64 ? 64 : ((kLo < kHi ? kLo : kHi) & ~31L));
  static constexpr size_t kFo = kFe + sizeof(uint32_t) * kFcap;
  static constexpr size_t kRec = kFo + sizeof(uint16_t) * kFcap;
  static constexpr size_t kBytes = kRec + sizeof(uint16_t) * kFcap;
};

// ---------------------------------------------------- look-back (1 word) ---

struct StatePolicy {  // chain 1: state-transition vectors, composite operator
  static __device__ __forceinline__ uint64_t to_word(uint64_t v) { return vpack(v); }
  static __device__ __forceinline__ uint64_t from_word(uint64_t w) {
    return vunpack(static_cast<uint32_t>(w));
  }
  static __device__ __forceinline__ uint64_t combine(uint64_t a, uint64_t b) { return vcompose(a, b); }
  static constexpr uint64_t kIdentity = kIdentityVec;
};
struct RcPolicy {  // chain 2: records and column offsets
  static __device__ __forceinline__ uint64_t to_word(uint64_t v) { return v; }
  static __device__ __forceinline__ uint64_t from_word(uint64_t w) { return w & ~kFlagMask; }
  static __device__ __forceinline__ uint64_t combine(uint64_t a, uint64_t b) { return tc_combine(a, b); }
  static constexpr uint64_t kIdentity = 0;
};

// How many lanes of a look-back window (lane i = tile idx - i) can be
// combined: up to and including the nearest inclusive prefix, as soon as
// every lane before it has published; 32 when all published without an
// inclusive prefix; 0 while the window must wait.  *done: an inclusive
// prefix was reached.
__device__ __forceinline__ int window_take(uint32_t valid, uint32_t inc, bool* done) {
  const int fi = valid == 0xffffffffu ? 32 : __ffs(~valid) - 1;
  const int fc = inc ? __ffs(inc) - 1 : 32;
  *done = fc < fi;
  if (fc < fi) return fc + 1;
  return fi == 32 ? 32 : 0;
}

// Look-back windows: each lane loads kLbRounds status words at once, so one
// round trip to L2 covers 32 * kLbRounds predecessors (32 / slots * kLbRounds
// per byte-count chain).  One word per lane measured fastest: an inclusive
// prefix is nearly always within reach, and wider windows cost registers in
// the whole kernel.
constexpr int kLbRounds = 1;
constexpr int kLbRoundsSums = 1;  // the same for the per-slot byte counts

// Called by one full warp.  Publishes the tile's aggregate, walks back over
// predecessors until an inclusive prefix is found, publishes the tile's
// inclusive prefix and returns the exclusive one.  `first` is the prefix of
// tile 0.  All waits end at `deadline` (then PP_E_TIMEOUT).
template <class P>
__device__ uint64_t lookback_word(uint64_t* st, uint64_t t, uint64_t agg, uint64_t first,
                                  uint64_t deadline, Misc* misc) {
  const int lane = threadIdx.x & 31;
  // flag and payload share one 64-bit word, so relaxed accesses suffice
  if (t == 0) {
    if (lane == 0) st_relaxed_u64(&st[0], kFlagInc | P::to_word(P::combine(first, agg)));
    return first;
  }
  if (lane == 0) st_relaxed_u64(&st[t], kFlagAgg | P::to_word(agg));
  uint64_t acc = P::kIdentity;
  int64_t base = static_cast<int64_t>(t) - 1;
  bool done = false;
  while (!done) {
    uint64_t w[kLbRounds];
#pragma unroll
    for (int j = 0; j < kLbRounds; ++j) {
      const int64_t mine = base - (32 * j + lane);
      w[j] = mine >= 0 ? ld_relaxed_u64(&st[mine]) : (kFlagInc | P::to_word(P::kIdentity));
    }
#pragma unroll
    for (int j = 0; j < kLbRounds; ++j) {
      if (!done) {
        const int64_t mine = base - (32 * j + lane);
        int take;
        for (;;) {
          take = window_take(__ballot_sync(0xffffffffu, (w[j] & kFlagMask) != 0),
                             __ballot_sync(0xffffffffu, (w[j] & kFlagMask) == kFlagInc), &done);
          if (take > 0) break;
          const bool expired = __shfl_sync(0xffffffffu, globaltimer_ns() > deadline ? 1 : 0, 0) != 0;
          if (expired) {
            if (lane == 0) atomicOr(&misc->timeout, 1u);
            done = true;
            take = 0;
            break;
          }
          __nanosleep(20);
          if ((w[j] & kFlagMask) == 0) w[j] = ld_relaxed_u64(&st[mine]);
        }
        uint64_t v = lane < take ? P::from_word(w[j]) : P::kIdentity;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const uint64_t o = __shfl_down_sync(0xffffffffu, v, off);
          if (lane + off < 32) v = P::combine(o, v);  // o holds earlier tiles
        }
        v = __shfl_sync(0xffffffffu, v, 0);
        acc = P::combine(v, acc);
      }
    }
    base -= 32 * kLbRounds;
  }
  if (lane == 0) st_relaxed_u64(&st[t], kFlagInc | P::to_word(P::combine(acc, agg)));
  return acc;
}

// Look-back over several independent additive chains at once (one status
// word per tile and chain: flag | count).  Lanes are grouped by chain: with G
// = ns rounded up to a power of two, lane l serves chain l % G and the
// (l / G)-th predecessor of each sub-window, so every chain advances over
// 32 / G predecessors per sub-window and kLbRounds sub-windows per round
// trip.  Returns, in lane k < ns, the exclusive prefix of chain k.
static __device__ int64_t lookback_sums(uint64_t* st, uint64_t t, uint32_t ns, const uint32_t* tile_tot,
                                 uint64_t deadline, Misc* misc) {
  const int lane = threadIdx.x & 31;
  uint32_t G = 1;
  while (G < ns) G <<= 1;
  const int per = 32 / static_cast<int>(G);          // predecessors per sub-window
  const uint32_t k = static_cast<uint32_t>(lane) & (G - 1);  // this lane's chain
  const int i = lane / static_cast<int>(G);          // this lane's predecessor offset
  uint32_t lanes_k = 0;                               // lanes serving chain k
  for (int l = static_cast<int>(k); l < 32; l += static_cast<int>(G)) lanes_k |= 1u << l;
  const bool active = k < ns;
  if (lane < static_cast<int>(ns)) st_relaxed_u64(&st[t * ns + lane], (t == 0 ? kFlagInc : kFlagAgg) | tile_tot[lane]);
  int64_t acc = 0;
  if (t > 0) {
    bool mydone = !active;  // this lane's chain found its inclusive prefix
    int64_t base = static_cast<int64_t>(t) - 1;
    while (__any_sync(0xffffffffu, !mydone)) {
      uint64_t w[kLbRoundsSums];
#pragma unroll
      for (int j = 0; j < kLbRoundsSums; ++j) {
        const int64_t mine = base - (per * j + i);
        w[j] = (active && mine >= 0) ? ld_relaxed_u64(&st[mine * ns + k]) : kFlagInc;
      }
#pragma unroll
      for (int j = 0; j < kLbRoundsSums; ++j) {
        const int64_t mine = base - (per * j + i);
        int limit = -1;  // include lanes of chain k up to this lane index
        bool done_now = false;
        for (;;) {
          const uint32_t valid = __ballot_sync(0xffffffffu, (w[j] & kFlagMask) != 0);
          const uint32_t inc = __ballot_sync(0xffffffffu, (w[j] & kFlagMask) == kFlagInc);
          const uint32_t bad = ~valid & lanes_k, incs = inc & lanes_k;
          const int fi = bad ? __ffs(bad) - 1 : 32;
          const int fc = incs ? __ffs(incs) - 1 : 32;
          bool ready = true;
          done_now = false;
          if (mydone) {
            limit = -1;
          } else if (fc < fi) {
            limit = fc;
            done_now = true;
          } else if (fi == 32) {
            limit = 31;
          } else {
            ready = false;
          }
          if (__all_sync(0xffffffffu, ready)) break;
          const bool expired = __shfl_sync(0xffffffffu, globaltimer_ns() > deadline ? 1 : 0, 0) != 0;
          if (expired) {
            if (lane == 0) atomicOr(&misc->timeout, 1u);
            mydone = true;
            limit = -1;
            done_now = false;
            break;
          }
          __nanosleep(20);
          if ((w[j] & kFlagMask) == 0 && active && mine >= 0) w[j] = ld_relaxed_u64(&st[mine * ns + k]);
        }
        long long x = (!mydone && lane <= limit) ? static_cast<long long>(w[j] & ~kFlagMask) : 0ll;
        for (int off = static_cast<int>(G); off < 32; off <<= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        acc += x;
        if (done_now) mydone = true;
      }
      base -= per * kLbRoundsSums;
    }
  }
  if (lane < static_cast<int>(ns))
    st_relaxed_u64(&st[t * ns + lane], kFlagInc | static_cast<uint64_t>(acc + tile_tot[lane]));
  return acc;
}

// ------------------------------------------------------ mask helpers ---

template <int MW>
__device__ __forceinline__ void set_range(uint64_t (&m)[MW], int lo, int hi) {
#pragma unroll
  for (int w = 0; w < MW; ++w) m[w] |= bit_range(lo - 64 * w, hi - 64 * w);
}
template <int MW>
__device__ __forceinline__ bool test_bit(const uint64_t (&m)[MW], int p) {
  bool r = false;
#pragma unroll
  for (int w = 0; w < MW; ++w)
    if ((p >> 6) == w) r = (m[w] >> (p & 63)) & 1ull;
  return r;
}

// shared -> shared or global byte copy: bytes up to a 4-byte aligned destination, then
// 32-bit words assembled with funnel shifts, four per step (the source loads
// of a step are independent).  May read up to 20 bytes past the source end.
__device__ __forceinline__ void smem_copy(uint8_t* dst, const uint8_t* src, int n) {
  while (n > 0 && (reinterpret_cast<uintptr_t>(dst) & 3)) {
    *dst++ = *src++;
    --n;
  }
  const int nw = n >> 2;
  if (nw > 0) {
    const uint32_t sh = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(src) & 3) * 8;
    const uint32_t* s = reinterpret_cast<const uint32_t*>(reinterpret_cast<uintptr_t>(src) & ~uintptr_t(3));
    uint32_t* d = reinterpret_cast<uint32_t*>(dst);
    uint32_t lo = s[0];
    int k = 0;
    for (; k + 4 <= nw; k += 4) {
      const uint32_t a = s[k + 1], b = s[k + 2], c = s[k + 3], e = s[k + 4];
      d[k] = __funnelshift_r(lo, a, sh);
      d[k + 1] = __funnelshift_r(a, b, sh);
      d[k + 2] = __funnelshift_r(b, c, sh);
      d[k + 3] = __funnelshift_r(c, e, sh);
      lo = e;
    }
    for (; k < nw; ++k) {
      const uint32_t hi = s[k + 1];
      d[k] = __funnelshift_r(lo, hi, sh);
      lo = hi;
    }
    dst += 4 * nw;
    src += 4 * nw;
    n -= 4 * nw;
  }
  while (n-- > 0) *dst++ = *src++;
}

// Warp-wide copy of n bytes from shared to global memory: 16-byte aligned
// destination vectors assembled with funnel shifts, the ragged ends byte by
// byte.  May read up to 20 bytes past the source end.
__device__ __forceinline__ void warp_copy_out(uint8_t* dst, const uint8_t* src, int n, int lane) {
  const int head = min(n, static_cast<int>((16u - (reinterpret_cast<uintptr_t>(dst) & 15u)) & 15u));
  if (lane < head) dst[lane] = src[lane];
  dst += head;
  src += head;
  n -= head;
  const int nv = n >> 4;
  const uintptr_t sa = reinterpret_cast<uintptr_t>(src);
  const uint32_t* s = reinterpret_cast<const uint32_t*>(sa & ~uintptr_t(3));
  const uint32_t sh = static_cast<uint32_t>(sa & 3u) * 8u;
  uint4* d = reinterpret_cast<uint4*>(dst);
  for (int k = lane; k < nv; k += 32) {
    const uint32_t* q = s + 4 * k;
    const uint32_t w0 = q[0], w1 = q[1], w2 = q[2], w3 = q[3], w4 = q[4];
    d[k] = make_uint4(__funnelshift_r(w0, w1, sh), __funnelshift_r(w1, w2, sh), __funnelshift_r(w2, w3, sh),
                      __funnelshift_r(w3, w4, sh));
  }
  if (lane < (n & 15)) dst[16 * nv + lane] = src[16 * nv + lane];
}

// String fields with more data bytes in a tile than this are queued and
// copied by the block's warps together.
constexpr uint32_t kLongField = 40;

__device__ __forceinline__ void store_value(const Col& col, uint32_t type, uint64_t r, uint64_t v) {
  if (type == PP_INT32 || type == PP_DATE_D)
    static_cast<uint32_t*>(col.values)[r] = static_cast<uint32_t>(v);
  else
    static_cast<uint64_t*>(col.values)[r] = v;
}

// ------------------------------------------------------------- kernel ---

// INFER: the inference form (parparaw_infer): the same pipeline, but each
// record's field count and each field's narrowest numeric type are reduced
// per tile in shared memory (the per-column sums, unused then) and folded into
// the job's Misc; nothing is written to the columns.
// UNITS: the form that also reads UTF-16LE code units (Sec. 4.2) for parsers
// whose tables ask for it; byte-only launches use the form without, whose
// code has no branch on the symbol width.
template <class Shape, int NSPEC, bool INFER = false, bool UNITS = false>
__global__ void __launch_bounds__(Shape::NT, Shape::MINB) pp_tile_kernel(const __grid_constant__ Launch L) {
  constexpr int NT = Shape::NT, VPT = Shape::VPT, B = Shape::B, T = Shape::T, MW = Shape::MW;
  using Lay = SmemLayout<Shape>;
  extern __shared__ __align__(128) uint8_t smem[];
  SmemHead* H = reinterpret_cast<SmemHead*>(smem);
  uint8_t* s_tile = smem + Lay::kTile;
  uint64_t* s_dm = reinterpret_cast<uint64_t*>(smem + Lay::kDm);
  uint16_t* s_cnt = reinterpret_cast<uint16_t*>(smem + Lay::kCnt);
  uint16_t* s_dex = reinterpret_cast<uint16_t*>(smem + Lay::kDex);  // data bytes before each chunk
  uint32_t* s_fe = reinterpret_cast<uint32_t*>(smem + Lay::kFe);    // field list (one round)
  uint16_t* s_fo = reinterpret_cast<uint16_t*>(smem + Lay::kFo);
  uint16_t* s_rec = reinterpret_cast<uint16_t*>(smem + Lay::kRec);
  const Tables& TB = H->tab;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    mbar_init(&H->mbar, 1);
    fence_mbar_init();
    H->tables_loaded = -1;
    H->job_loaded = -1;
  }
  __syncthreads();
  uint32_t phase = 0;
#ifdef PP_PHASE_TIMING
  if (tid == 0) {
    for (int k = 0; k < 32; ++k) H->ph_cycles[k] = 0;
    for (int k = 0; k < 8; ++k) H->w_max[k] = H->w_sum[k] = 0;
  }
  long long ph_last = clock64();
  long long w_t0 = 0;
#endif

  for (;;) {
    // ------------------------------------------------------------ work item
    if (tid == 0) {
      const unsigned long long item = atomicAdd(L.work_counter, 1ull);
      uint32_t j = 0;
      if (L.jobs != nullptr && item < L.total_tiles) {
        uint32_t lo = 0, hi = L.njobs - 1;
        while (lo < hi) {
          const uint32_t mid = (lo + hi + 1) >> 1;
          if (L.jobs[mid].tile_base <= item) lo = mid; else hi = mid - 1;
        }
        j = lo;
      }
      H->item = item;
      H->job = j;
      H->tile_last_rd = 0;
      H->eof_rd = 0;
      H->npieces = H->npieces_ok = 0;
    }
    if (tid < PP_MAX_STRING_COLUMNS) H->round_base[tid] = 0;
    __syncthreads();
    const unsigned long long item = H->item;
    if (item >= L.total_tiles) break;
    uint32_t* s_inf = reinterpret_cast<uint32_t*>(s_cnt);  // INFER: ranks [0, 64), min / max fields
    if constexpr (INFER) {
      if (tid < PP_MAX_COLUMNS + 2) s_inf[tid] = tid == PP_MAX_COLUMNS ? 0xFFFFFFFFu : 0u;
    }
    if (H->job_loaded != static_cast<int32_t>(H->job)) {
      const Job& src = L.jobs ? L.jobs[H->job] : L.job0;
      const Col* csrc = L.jobs ? (L.cols + src.col0) : L.cols0;
      const uint32_t* s32 = reinterpret_cast<const uint32_t*>(&src);
      uint32_t* d32 = reinterpret_cast<uint32_t*>(&H->jd);
      for (int i = tid; i < static_cast<int>(sizeof(Job) / 4); i += NT) d32[i] = s32[i];
      const uint32_t ncol = (L.jobs ? L.tables[src.tables] : L.tables0).num_columns;
      const uint64_t* c64 = reinterpret_cast<const uint64_t*>(csrc);
      uint64_t* e64 = reinterpret_cast<uint64_t*>(H->cd);
      for (uint32_t i = tid; i < ncol * (sizeof(Col) / 8); i += NT) e64[i] = c64[i];
      __syncthreads();
      if (tid == 0) H->job_loaded = static_cast<int32_t>(H->job);
    }
    const Job& J = H->jd;
    const Col* cols = H->cd;
    const uint64_t deadline = globaltimer_ns() + L.timeout_ns;

    if (H->tables_loaded != static_cast<int32_t>(J.tables)) {
      const Tables* src = L.jobs ? &L.tables[J.tables] : &L.tables0;
      __syncthreads();
      const uint32_t* s32 = reinterpret_cast<const uint32_t*>(src);
      uint32_t* d32 = reinterpret_cast<uint32_t*>(&H->tab);
      for (int i = tid; i < static_cast<int>(sizeof(Tables) / 4); i += NT) d32[i] = s32[i];
      __syncthreads();
      if (tid < PP_MAX_STRING_COLUMNS) {
        uint8_t col = 0xFF;
        for (int c = 0; c < H->tab.num_columns; ++c)
          if (H->tab.str_slot[c] == tid) col = static_cast<uint8_t>(c);
        H->str_col[tid] = col;
      }
      if (tid == 0) H->tables_loaded = static_cast<int32_t>(J.tables);
      __syncthreads();
    }
    PP_PHASE(0);

    // ------------------------------------------------------- load the tile
    const uint64_t t = item - J.tile_base;
    const uint64_t VL = J.head + J.len;  // virtual length (16-byte aligned origin)
    const uint64_t v0 = t * T;
    const uint64_t v1 = min(v0 + T, VL);
    const uint8_t* vbase = J.input - J.head;
    const uint64_t a16 = max(v0, (J.head + 15) & ~uint64_t(15));
    const uint64_t b16 = min(v1, VL & ~uint64_t(15));
    const uint32_t bulk = b16 > a16 ? static_cast<uint32_t>(b16 - a16) : 0u;
    if (tid == 0 && bulk > 0) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&H->mbar, bulk);
      tma_load_1d(s_tile + (a16 - v0), vbase + a16, bulk, &H->mbar);
      // The tile a block will take about one tile from now (tiles go out in
      // order, one per resident block per tile time) is pulled into L2, so
      // its load waits on L2 rather than HBM.
      const uint64_t tn = t + gridDim.x;
      if (tn < J.ntiles) {
        const uint64_t pa = max(tn * T, (J.head + 15) & ~uint64_t(15));
        const uint64_t pb = min(tn * T + T, VL & ~uint64_t(15));
        if (pb > pa) prefetch_l2_bulk(vbase + pa, static_cast<uint32_t>(pb - pa));
      }
    }
    {
      const uint64_t lo_v = max(v0, J.head);
      if (bulk == 0) {
        for (uint64_t x = lo_v + tid; x < v1; x += NT) s_tile[x - v0] = vbase[x];
      } else if (tid < 32) {
        const uint64_t x = tid < 16 ? lo_v + tid : b16 + (tid - 16);
        const bool in_head = tid < 16 && x < a16 && x < v1;
        const bool in_tail = tid >= 16 && x < v1;
        if (in_head || in_tail) s_tile[x - v0] = vbase[x];
      }
    }
    bool load_expired = false;
    if (bulk > 0) {
      while (!mbar_try_wait(&H->mbar, phase)) {
        if (globaltimer_ns() > deadline + 1000000000ull) {
          load_expired = true;
          break;
        }
      }
    }
    if (__syncthreads_or(load_expired)) {
      // The tile did not arrive in time.  The block stops: it reports the
      // timeout, gives the copy in flight one more bounded wait so that
      // nothing still writes into its shared memory when it exits, and
      // neither re-arms the barrier nor reuses the tile buffer.  The tiles
      // behind this one time out in their look-backs.
      if (tid == 0) atomicOr(&J.misc->timeout, 1u);
      const uint64_t last = globaltimer_ns() + 1000000000ull;
      while (!mbar_try_wait(&H->mbar, phase) && globaltimer_ns() < last) {
      }
      return;
    }
    if (bulk > 0) phase ^= 1u;
    PP_PHASE(1);
    PP_WMARK();

    // valid bytes of this thread's chunk, chunk-relative [lo, hi)
    const int64_t cv0 = static_cast<int64_t>(v0) + static_cast<int64_t>(tid) * B;
    int lo = static_cast<int>(min(max(static_cast<int64_t>(J.head) - cv0, int64_t(0)), int64_t(B)));
    int hi = static_cast<int>(min(max(static_cast<int64_t>(VL) - cv0, int64_t(0)), int64_t(B)));
    if (hi < lo) hi = lo;
    const uint8_t* chunk = s_tile + tid * B;

    // --------------------------------------------- a1: symbol matching
    uint64_t spec[MW];
#pragma unroll
    for (int w = 0; w < MW; ++w) spec[w] = 0;
    if (!TB.idempotent) {
      set_range(spec, lo, hi);  // every symbol is simulated on its own
    } else if (TB.num_symbols > 0) {
      uint32_t rep[NSPEC];
#pragma unroll
      for (int s = 0; s < NSPEC; ++s) rep[s] = TB.rep[s < TB.num_symbols ? s : 0];
      const uint4* src = reinterpret_cast<const uint4*>(chunk);
      if (UNITS && TB.unit2) {
        // UTF-16LE code units (Sec. 4.2): the same test on 16-bit lanes
        // against the symbols' code units 0x00bb; a flag lands on the unit's
        // first byte
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
          const uint4 q = src[v];
          const uint32_t wd[4] = {q.x, q.y, q.z, q.w};
          uint32_t acc[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            acc[k] = 0;
#pragma unroll
            for (int s = 0; s < NSPEC; ++s) {
              const uint32_t x = wd[k] ^ (rep[s] & 0x00FF00FFu);
              acc[k] |= (x - 0x00010001u) & ~x;
            }
          }
          if ((acc[0] | acc[1] | acc[2] | acc[3]) & 0x80008000u) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const uint32_t bits4 = ((acc[k] >> 15) & 1u) | ((acc[k] >> 29) & 4u);
              const int pos = 16 * v + 4 * k;
              spec[pos >> 6] |= static_cast<uint64_t>(bits4) << (pos & 63);
            }
          }
        }
      } else {
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
          const uint4 q = src[v];
          const uint32_t wd[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            // zero-byte test of the word against every symbol; a flagged
            // byte that is not a symbol (borrow from a zero byte below) is
            // harmless: it is simulated on its own with the catch-all
            // transition
            uint32_t acc = 0;
#pragma unroll
            for (int s = 0; s < NSPEC; ++s) {
              const uint32_t x = wd[k] ^ rep[s];
              acc |= (x - 0x01010101u) & ~x;
            }
            acc &= 0x80808080u;
            const uint32_t bits4 = (((acc >> 7) * 0x00204081u) >> 21) & 0xFu;
            const int pos = 16 * v + 4 * k;
            spec[pos >> 6] |= static_cast<uint64_t>(bits4) << (pos & 63);
          }
        }
      }
#pragma unroll
      for (int w = 0; w < MW; ++w) spec[w] &= bit_range(lo - 64 * w, hi - 64 * w);
    }

    const int P0 = static_cast<int>(min(max(static_cast<int64_t>(J.head) - static_cast<int64_t>(v0), int64_t(0)),
                                        static_cast<int64_t>(T)));
    const int PE = static_cast<int>(v1 - v0);  // end of the tile's bytes
    // ------------------------------------ a2: multi-state simulation
    // Symbols are W bytes: 1, or 2 for UTF-16LE code units (a code unit above
    // U+00FF is in the catch-all group).
    const int W = (UNITS && TB.unit2) ? 2 : 1;
    auto group_at = [&](int p) -> uint32_t {
      return (W == 2 && chunk[p + 1] != 0) ? TB.catch_all : TB.group_of[chunk[p]];
    };
    uint64_t vec = kIdentityVec;
    {
      int prev = -W;
#pragma unroll
      for (int w = 0; w < MW; ++w) {  // the symbols in order, one mask word at a time
        for (uint64_t sw = spec[w]; sw; sw &= sw - 1) {
          const int p = 64 * w + __ffsll(static_cast<long long>(sw)) - 1;
          const bool run = max(prev + W, lo) < p;
          const uint32_t g = group_at(p);
          vec = vcompose(vec, run ? TB.trans_run[g] : TB.trans[g]);
          prev = p;
        }
      }
      if (max(prev + W, lo) < hi) vec = vcompose(vec, TB.trans[TB.catch_all]);
    }

    // ------------------------------------------- a3: o-scan + chain 1
    PP_WSPAN(0);
    uint64_t tile_vec;
    const uint64_t vex = block_exclusive_scan<NT>(
        vec, [](uint64_t a, uint64_t b) { return vcompose(a, b); }, kIdentityVec, H->wsum64,
        &tile_vec);
    PP_PHASE(2);
    if (warp == 0) {
      const uint64_t pre =
          lookback_word<StatePolicy>(J.st_state, t, tile_vec, kIdentityVec, deadline, J.misc);
      if (lane == 0) H->prefix_vec = pre;
    }
    __syncthreads();
    PP_PHASE(3);
    const uint32_t tile_s0 = vget(H->prefix_vec, TB.start_state);
    const uint32_t tile_send = vget(tile_vec, tile_s0);
    const uint32_t s_start = vget(vex, tile_s0);

    // ------------------------------------------- a4: re-simulation, tags
    PP_WMARK();
    uint64_t dm[MW], fm[MW], rm[MW];
#pragma unroll
    for (int w = 0; w < MW; ++w) {  // runs are data unless fixed below (a symbol's bytes in one word)
      dm[w] = bit_range(lo - 64 * w, hi - 64 * w) & ~(spec[w] | (W == 2 ? spec[w] << 1 : 0ull));
      fm[w] = rm[w] = 0;
    }
    {
      const uint32_t inv = TB.invalid_state;
      const uint32_t ca = TB.catch_all;
      const uint32_t e_ca = TB.emit[ca];
      const uint64_t t_ca = TB.trans[ca];
      uint32_t s = s_start;
      int prev = -W, inv_pos = -1;
      auto run = [&](int rs, int re) {
        const uint32_t s1 = vget(t_ca, s);
        const uint32_t tag0 = (e_ca >> (2 * s)) & 3u, tagr = (e_ca >> (2 * s1)) & 3u;
        if (s != inv && s1 == inv && inv_pos < 0) inv_pos = rs;
        if ((tag0 | tagr) != PP_TAG_DATA) {  // rare: a run that is not all data
#pragma unroll
          for (int w = 0; w < MW; ++w) {
            const uint64_t b0 = bit_range(rs - 64 * w, rs + W - 64 * w);  // the run's first symbol
            const uint64_t br = bit_range(rs + W - 64 * w, re - 64 * w);
            dm[w] &= ~((tag0 != PP_TAG_DATA ? b0 : 0) | (tagr != PP_TAG_DATA ? br : 0));
            fm[w] |= (tag0 == PP_TAG_FIELD ? b0 : 0) | (tagr == PP_TAG_FIELD ? br : 0);
            rm[w] |= (tag0 == PP_TAG_RECORD ? b0 : 0) | (tagr == PP_TAG_RECORD ? br : 0);
          }
        }
        s = s1;
      };
#pragma unroll
      for (int w = 0; w < MW; ++w) {  // the symbols in order, one mask word at a time
        // this word's symbols that are data, field and record delimiters
        // (or-ed in after the word: run() touches only bits before the
        // current symbol, never an earlier symbol's)
        uint64_t dw = 0, fw = 0, rw = 0;
        for (uint64_t sw = spec[w]; sw; sw &= sw - 1) {
          const int b = __ffsll(static_cast<long long>(sw)) - 1;
          const int p = 64 * w + b;
          const int rs = max(prev + W, lo);
          const uint32_t g = group_at(p);
          // one lookup for the catch-all run before the symbol (if any) and
          // the symbol itself; runs that are not all data take the
          // byte-exact path
          uint32_t st = TB.step[rs < p ? 1 : 0][g][s];
          if (st & kStepSlow) {
            run(rs, p);
            st = TB.step[0][g][s];
          }
          const uint32_t tag = (st >> 3) & 3u;
          if ((st & kStepInv) && inv_pos < 0) inv_pos = p;
          // a special symbol is never data unless its tag says so;
          // delimiters are marked at their first byte (a UTF-16 unit starts
          // at an even position, so its second byte is in the same word)
          const uint64_t bit = 1ull << b;
          if (tag == PP_TAG_DATA) dw |= bit | (W == 2 ? bit << 1 : 0ull);
          else if (tag == PP_TAG_FIELD) fw |= bit;
          else if (tag == PP_TAG_RECORD) rw |= bit;
          s = st & 7u;
          prev = p;
        }
        dm[w] |= dw;
        fm[w] |= fw;
        rm[w] |= rw;
      }
      {
        const int rs = max(prev + W, lo);
        if (rs < hi && (TB.step[1][0][s] & kStepSlow)) run(rs, hi);  // else all data
      }
      if (inv_pos >= 0)
        atomicMin(&J.misc->first_invalid,
                  static_cast<unsigned long long>(cv0 + inv_pos - static_cast<int64_t>(J.head)));
    }
#pragma unroll
    for (int w = 0; w < MW; ++w) s_dm[tid * MW + w] = dm[w];

    // ---------------------------------- a5: records, columns + chain 2
    // Per chunk: records, column offset (abs/rel), data bytes and
    // delimiters; one block scan carries all four (records and columns with
    // the (+, oplus) pair, data bytes and delimiters as plain sums).
    uint32_t nrec = 0, ncol = 0, ndl = 0, ndat = 0;
    {
      int last_rd = -1;
#pragma unroll
      for (int w = 0; w < MW; ++w) {
        nrec += __popcll(rm[w]);
        ndl += __popcll(fm[w] | rm[w]);
        ndat += __popcll(dm[w]);
        if (rm[w]) last_rd = 64 * w + 63 - __clzll(static_cast<long long>(rm[w]));
      }
#pragma unroll
      for (int w = 0; w < MW; ++w) ncol += __popcll(fm[w] & ~bits_below(last_rd + 1 - 64 * w));
      if (TB.partial && last_rd >= 0)  // the record ends after its delimiter's W bytes
        atomicMax(&H->tile_last_rd, static_cast<unsigned long long>(cv0 + last_rd + W - static_cast<int64_t>(J.head)));
      if (lo < hi && cv0 + hi == static_cast<int64_t>(VL) && test_bit(rm, hi - W)) H->eof_rd = 1u;
    }
    PP_WSPAN(1);
    uint64_t sc_tile;
    const uint64_t sc_ex = block_exclusive_scan<NT>(
        static_cast<uint64_t>(rc_pack(nrec, ncol, nrec > 0)) | (static_cast<uint64_t>(ndat | (ndl << 16)) << 32),
        [](uint64_t a, uint64_t b) {
          return static_cast<uint64_t>(rc_combine(static_cast<uint32_t>(a), static_cast<uint32_t>(b))) |
                 (((a >> 32) + (b >> 32)) << 32);
        },
        uint64_t(0), H->wsum64, &sc_tile);
    const uint32_t rc_ex = static_cast<uint32_t>(sc_ex), rc_tile = static_cast<uint32_t>(sc_tile);
    const uint32_t dat_ex = static_cast<uint32_t>(sc_ex >> 32) & 0xFFFFu;
    const uint32_t dl_ex = static_cast<uint32_t>(sc_ex >> 48);
    const uint32_t ND = static_cast<uint32_t>(sc_tile >> 48);  // delimiters of the tile
    s_dex[tid] = static_cast<uint16_t>(dat_ex);
    if (tid == NT - 1) s_dex[NT] = static_cast<uint16_t>((sc_tile >> 32) & 0xFFFFu);
    PP_PHASE(4);
    if (TB.partial && tid == 0 && H->tile_last_rd)  // after the scan's barriers
      atomicMax(&J.misc->last_record_end, H->tile_last_rd);
    if (warp == 0) {
      const uint64_t agg = tc_pack(rc_tile & 0xFFFFu, (rc_tile >> 16) & kColSat, (rc_tile >> 31) != 0);
      const uint64_t pre = lookback_word<RcPolicy>(J.st_rc, t, agg, tc_pack(0, 0, true), deadline, J.misc);
      if (lane == 0) H->prefix_rc = pre;
    }
    __syncthreads();
    PP_PHASE(5);
    // Skipping records (Sec. 4.3): record i of the input (from 0) leaves row
    // i - S, and nothing at all for i < S.  The tile's first record is row
    // row0 (mod 2^64).
    const uint64_t row0 = (H->prefix_rc & kRecMask) - TB.skip_records;
    const uint32_t tile_col0 = static_cast<uint32_t>((H->prefix_rc >> 40) & 0x1FFFFF);
    const uint32_t row_start = rc_ex & 0xFFFFu;  // relative to the tile's first record
    const uint32_t col_start = (rc_ex >> 31) ? ((rc_ex >> 16) & kColSat)
                                             : min(tile_col0 + ((rc_ex >> 16) & kColSat), kColSat);
    // the tile's open field (after its last delimiter): record and column
    const uint32_t rec_tile = rc_tile & 0xFFFFu;
    const uint32_t col_end = (rc_tile >> 31) ? ((rc_tile >> 16) & kColSat)
                                             : min(tile_col0 + ((rc_tile >> 16) & kColSat), kColSat);

    const uint32_t C = TB.num_columns;
    const uint32_t NS = TB.num_str;
    const bool last_tile = (t + 1 == J.ntiles);
    const uint64_t rows_cap = J.rows_cap;
    // The field after the last delimiter ends at the input's end when the
    // input ends here.  If the input's last byte is a record delimiter that
    // field does not exist; otherwise it closes a trailing record when the
    // final state accepts (and the input is whole).
    const bool open_dead = last_tile && H->eof_rd;
    const bool trailing =
        last_tile && !TB.partial && !H->eof_rd && ((TB.accept_mask >> tile_send) & 1u) && PE > P0;
    const uint32_t NF = ND + 1;  // fields of the tile, the open one included
    constexpr uint32_t FCAP = static_cast<uint32_t>(Lay::kFcap);
    const uint32_t nrounds = (NF + FCAP - 1) / FCAP;

    // Data bytes of the tile before tile position p (p in [0, T]).
    auto data_before = [&](int p) -> uint32_t {
      if constexpr (B % 64 == 0) {  // whole mask words per chunk: word p / 64 of the tile holds p
        const int wi = p >> 6, u = wi / MW, w = wi - u * MW;
        uint32_t n = s_dex[u];
#pragma unroll
        for (int k = 0; k + 1 < MW; ++k)
          if (k < w) n += __popcll(s_dm[u * MW + k]);
        if (p & 63) n += __popcll(s_dm[wi] & ((1ull << (p & 63)) - 1ull));
        return n;
      } else {
        const int u = p / B;
        const int off = p - u * B;
        uint32_t n = s_dex[u];
        if (off > 0) {
#pragma unroll
          for (int w = 0; w < MW; ++w) n += __popcll(s_dm[u * MW + w] & bits_below(off - 64 * w));
        }
        return n;
      }
    };

    // First data position in [p, e), else e.  Mask bits at or past B are
    // never set.
    auto first_data = [&](int p, int e) -> int {
      while (p < e) {
        const int u = p / B, i = p - u * B;
        const uint64_t w = s_dm[u * MW + (i >> 6)] & ~bits_below(i & 63);
        if (w) return min(u * B + (i & ~63) + __ffsll(static_cast<long long>(w)) - 1, e);
        p = (i & ~63) + 64 >= B ? (u + 1) * B : u * B + (i & ~63) + 64;
      }
      return e;
    };

    // Field list of one round: entry i describes field f0 + i of the tile
    // (the kEnt* layout: end position, column, open field, ends a record).
    // s_rec[k] = first entry of the round's k-th record.  The thread that
    // writes the round's last entry leaves the next round's starting point.
    // The start of a round: the end of its field f0 - 1 (the tile's data start
    // - 1 for f0 = 0) and the record of field f0.  Round 0 starts at the
    // tile's start; later rounds read what the previous round left in H.
    struct RoundStart {
      int prev_pos;
      uint32_t rr0;
    };
    const RoundStart first_round{P0 - 1, 0u};
    // Skipped records of a round (of nrec records from the tile's record
    // rr0), and the round's first entry of a kept record (after
    // build_round's barrier): 0 unless the round starts among the skipped
    // records.  The per-entry and per-record loops start there, so they
    // carry no test of their own.
    auto round_skip = [&](uint32_t rr0, uint32_t nrec) -> uint32_t {
      const uint64_t rec = (H->prefix_rc & kRecMask) + rr0;
      const uint64_t S = TB.skip_records;
      return rec >= S ? 0u : (S - rec < nrec ? static_cast<uint32_t>(S - rec) : nrec);
    };
    auto first_kept = [&](uint32_t rr0, uint32_t nwin) -> uint32_t {
      const uint32_t nrec = H->rr_last - rr0 + 1;
      const uint32_t k = round_skip(rr0, nrec);
      return k == 0 ? 0u : (k < nrec ? s_rec[k] : nwin);
    };
    auto build_round = [&](uint32_t f0, uint32_t f1, RoundStart r0) {
      const uint32_t rr0 = r0.rr0;
      if (tid == 0) s_rec[0] = 0;
      if (dl_ex < f1 && dl_ex + ndl > f0) {
        uint32_t g = dl_ex, c = col_start, rr = row_start;
#pragma unroll
        for (int w = 0; w < MW; ++w) {  // the delimiters in order, one mask word at a time
          for (uint64_t dw = fm[w] | rm[w]; dw && g < f1; dw &= dw - 1, ++g) {
            const int b = __ffsll(static_cast<long long>(dw)) - 1;
            const bool rd = (rm[w] >> b) & 1ull;
            if (g >= f0) {
              const int pos = tid * B + 64 * w + b;
              s_fe[g - f0] = static_cast<uint32_t>(pos) | (rd ? kEntRec : 0u) | (min(c, 255u) << 16);
              if (rd && g + 1 < f1) s_rec[rr + 1 - rr0] = static_cast<uint16_t>(g + 1 - f0);
              if (g + 1 == f1) {
                H->rr_last = rr;
                H->rr_next = rr + (rd ? 1u : 0u);
                H->next_prev_pos = pos;
              }
            }
            if (rd) {
              ++rr;
              c = 0;
            } else {
              c = min(c + 1, kColSat);
            }
          }
        }
      }
      if (tid == NT - 1 && ND >= f0 && ND < f1) {
        s_fe[ND - f0] = static_cast<uint32_t>(PE) | (trailing ? kEntRec : 0u) | (min(col_end, 255u) << 16) |
                        kEntOpen;
        H->rr_last = rec_tile;
      }
      __syncthreads();
    };

    // Block scan of the per-thread, per-slot counts in s_cnt (two 16-bit
    // slots per word; a slot's total is at most T < 2^16): leaves the
    // exclusive per-thread sums in s_cnt and the totals in round_tot.
    auto scan_counts = [&]() {
      const uint32_t K = (NS + 1) / 2;
      uint32_t incl[PP_MAX_STRING_COLUMNS / 2], own[PP_MAX_STRING_COLUMNS / 2];
#pragma unroll
      for (int k = 0; k < PP_MAX_STRING_COLUMNS / 2; ++k) {
        if (k < static_cast<int>(K)) {
          own[k] = s_cnt[(2 * k) * NT + tid] |
                   (2 * k + 1 < static_cast<int>(NS) ? (static_cast<uint32_t>(s_cnt[(2 * k + 1) * NT + tid]) << 16) : 0u);
          incl[k] = warp_inclusive_scan(own[k], [](uint32_t a, uint32_t b) { return a + b; }, lane);
          if (lane == 31) H->wsumk[k][warp] = incl[k];
        }
      }
      __syncthreads();
      if (warp == 0) {
        for (uint32_t k = 0; k < K; ++k) {
          uint32_t x = lane < Shape::NW ? H->wsumk[k][lane] : 0u;
          x = warp_inclusive_scan(x, [](uint32_t a, uint32_t b) { return a + b; }, lane);
          if (lane < Shape::NW) H->wsumk[k][lane] = x;
        }
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < PP_MAX_STRING_COLUMNS / 2; ++k) {
        if (k < static_cast<int>(K)) {
          const uint32_t ex = incl[k] - own[k] + (warp > 0 ? H->wsumk[k][warp - 1] : 0u);
          s_cnt[(2 * k) * NT + tid] = static_cast<uint16_t>(ex & 0xFFFFu);
          if (2 * k + 1 < static_cast<int>(NS)) s_cnt[(2 * k + 1) * NT + tid] = static_cast<uint16_t>(ex >> 16);
          if (tid == 0) {
            const uint32_t tot = H->wsumk[k][Shape::NW - 1];
            H->round_tot[2 * k] = tot & 0xFFFFu;
            if (2 * k + 1 < static_cast<int>(NS)) H->round_tot[2 * k + 1] = tot >> 16;
          }
        }
      }
      // each thread reads back only its own sums; round_tot is written by
      // thread 0 and read by warp 0
      __syncwarp();
    };

    // Per-slot string bytes of the round's fields; each thread takes an
    // equal share of consecutive entries, then the counts are scanned.
    auto count_round = [&](uint32_t nwin, RoundStart r0) {
      const uint32_t per = (nwin + NT - 1) / NT;
      const uint32_t b1 = min(tid * per + per, nwin);
      const uint32_t b0 = min(max(tid * per, first_kept(r0.rr0, nwin)), b1);
      for (uint32_t k = 0; k < NS; ++k) s_cnt[k * NT + tid] = 0;
      int eprev = b0 == 0 ? r0.prev_pos : static_cast<int>(s_fe[b0 - 1] & kEntPos);
      for (uint32_t g = b0; g < b1; ++g) {  // data bytes are counted for string fields only
        const uint32_t fe = s_fe[g];
        const int e = static_cast<int>(fe & kEntPos);
        const uint32_t c = (fe >> 16) & 0xFFu;
        if (c < C && TB.str_slot[c] != 0xFF)
          s_cnt[TB.str_slot[c] * NT + tid] += static_cast<uint16_t>(data_before(e) - data_before(eprev + 1));
        eprev = e;
      }
      scan_counts();
    };

    // The tile's per-slot string bytes without a field list (for tiles of
    // several rounds, whose lists are built again when emitted): each thread
    // splits its chunk at its delimiters and adds each piece's data bytes to
    // the slot of the field it belongs to -- the field open at the chunk's
    // start has the column and record the o-scan gave it.  Fields of skipped
    // records count nothing.  The totals land in round_tot.
    auto count_chunks = [&]() {
      for (uint32_t k = 0; k < NS; ++k) s_cnt[k * NT + tid] = 0;
      const uint64_t rec0 = H->prefix_rc & kRecMask;
      const uint64_t S = TB.skip_records;
      uint32_t c = col_start, rr = row_start, done = 0, base = 0;
      auto add = [&](uint32_t upto) {  // data bytes up to here belong to field (rr, c)
        if (upto > done && c < C && TB.str_slot[c] != 0xFF && rec0 + rr >= S)
          s_cnt[TB.str_slot[c] * NT + tid] += static_cast<uint16_t>(upto - done);
        done = upto;
      };
#pragma unroll
      for (int w = 0; w < MW; ++w) {  // the delimiters in order, one mask word at a time
        const uint64_t dmw = s_dm[tid * MW + w];
        for (uint64_t dw = fm[w] | rm[w]; dw; dw &= dw - 1) {
          const int b = __ffsll(static_cast<long long>(dw)) - 1;
          add(base + __popcll(dmw & bits_below(b)));
          if ((rm[w] >> b) & 1ull) {
            ++rr;
            c = 0;
          } else {
            c = min(c + 1, kColSat);
          }
        }
        base += __popcll(dmw);
      }
      add(base);
      scan_counts();
    };

    auto round_start = [&](uint32_t r) -> RoundStart {  // after next_round's barrier for r > 0
      return r == 0 ? first_round : RoundStart{H->prev_pos, H->rr0};
    };
    auto next_round = [&]() {  // after a barrier that follows the round's last use of its list
      if (tid == 0) {
        H->prev_pos = H->next_prev_pos;
        H->rr0 = H->rr_next;
        H->npieces = H->npieces_ok = 0;
      }
      if (tid < static_cast<int>(NS)) H->round_base[tid] += H->round_tot[tid];
      __syncthreads();
    };

    // ------------------------ pass 1: string bytes per column + chain 3
    if (NS > 0) {
      if (nrounds == 1) {  // the round stays in place for pass 2
        build_round(0, NF, first_round);
        PP_PHASE(13);
        count_round(NF, first_round);
      } else {
        count_chunks();
      }
      if (tid < static_cast<int>(NS)) H->tile_tot[tid] = H->round_tot[tid];
      __syncwarp();  // written and read by warp 0 (NS <= 32)
      PP_PHASE(6);
      // chain 3: per-slot byte counts, summed over the predecessors; all
      // slots advance together
      if (warp == 0) {
        const int64_t base_k = lookback_sums(J.st_bytes, t, NS, H->tile_tot, deadline, J.misc);
        if (lane < static_cast<int>(NS)) H->col_base[lane] = base_k;
      }
      __syncthreads();
      PP_PHASE(7);
    }

    // ----------------- a6 / a7 / a8: offsets, gather, conversion, rejects
    // Converts numeric field (r, c) occupying tile positions [a, e); `ended`:
    // the field ends there (else it continues past the tile, and its data
    // bytes are gathered from global memory by re-simulating from the
    // tile's end state).
    auto convert_field = [&](uint64_t r, uint32_t c, int a, int e, bool ended) {
      const uint32_t type = TB.col_type[c];
      uint64_t val = 0;
      int st;
      const int n_in = static_cast<int>(data_before(e) - data_before(a));
      if (ended && n_in == e - a && W == 1) {
        st = n_in > kNumericMaxLen ? kConvFail : convert_value(type, s_tile + a, n_in, &val);
      } else {
        uint8_t buf[kNumericMaxLen + 2];
        int m = 0;
        for (int y = a; y < e && m <= kNumericMaxLen; ++y) {
          const int u = y / B, i = y - u * B;
          if ((s_dm[u * MW + (i >> 6)] >> (i & 63)) & 1ull) buf[m++] = s_tile[y];
        }
        if (!ended && m <= kNumericMaxLen) {  // the rest of the field, past the tile
          uint32_t s = tile_send;
          for (uint64_t g = v1; g + W <= VL; g += W) {
            const uint32_t unit = W == 2 ? (vbase[g] | (vbase[g + 1] << 8)) : vbase[g];
            const uint32_t grp = unit <= 0xFFu ? TB.group_of[unit] : TB.catch_all;
            const uint32_t tag = (TB.emit[grp] >> (2 * s)) & 3u;
            s = vget(TB.trans[grp], s);
            if (tag == PP_TAG_DATA) {
              buf[m++] = vbase[g];
              if (W == 2) buf[m++] = vbase[g + 1];
              if (m > kNumericMaxLen) break;
            } else if (tag != PP_TAG_CONTROL) {
              break;
            }
            if (s == TB.invalid_state) break;
          }
        }
        if (W == 2 && m <= kNumericMaxLen) {  // UTF-16LE text converts when it is ASCII
          bool ascii = (m & 1) == 0;
          for (int k = 0; ascii && 2 * k < m; ++k) {
            ascii = buf[2 * k + 1] == 0 && buf[2 * k] < 0x80;
            buf[k] = buf[2 * k];
          }
          m = ascii ? m / 2 : kNumericMaxLen + 1;
        }
        st = m > kNumericMaxLen ? kConvFail : convert_value(type, buf, m, &val);
      }
      store_value(cols[c], type, r, val);
      if (st != kConvOk) {
        const uint32_t bit = 1u << (r & 31);
        atomicOr(&J.null_bits[TB.num_slot[c] * J.bit_words + (r >> 5)], bit);
        if (st == kConvFail) atomicOr(&J.fail_bits[r >> 5], bit);
      }
    };

    // ------------------------------------------- pass 2: emit, by rounds
    if (NS > 0 && nrounds > 1) {  // the rounds again from the first (else pass 1's only round is in place)
      if (tid < static_cast<int>(NS)) H->round_base[tid] = 0;
      __syncthreads();
    }
    for (uint32_t r = 0; r < nrounds; ++r) {
      const uint32_t f0 = r * FCAP, f1 = min(f0 + FCAP, NF), nwin = f1 - f0;
      const RoundStart rs = round_start(r);
      if (NS == 0 || nrounds > 1) {
        build_round(f0, f1, rs);
        if (NS > 0) count_round(nwin, rs);
        PP_PHASE(14);
      }
      const uint32_t rr0 = rs.rr0;
      const uint32_t nrec_win = H->rr_last - rr0 + 1;
      const int prev_pos = rs.prev_pos;

      // (1) equal shares of consecutive entries: per-slot running byte
      // positions -> s_fo (field end minus data bytes before it, mod 2^16);
      // string field bytes to their columns (a lane copies a short field,
      // the warp the long ones together; nothing past a column's capacity);
      // records with a wrong field count (rare)
      PP_WMARK();
      if (tid == 0) {
        // step (2) gives G threads to a record, each taking every G-th field:
        // the G, from min(C, NT / records) up, that leaves the busiest
        // thread the fewest fields
        uint32_t g = max(1u, min(C, static_cast<uint32_t>(NT) / nrec_win));
        uint32_t best = ((nrec_win * g + NT - 1) / NT) * ((C + g - 1) / g);
        for (uint32_t g2 = g + 1, ge = min(C, g + 4); g2 <= ge; ++g2) {
          const uint32_t cost = ((nrec_win * g2 + NT - 1) / NT) * ((C + g2 - 1) / g2);
          if (cost < best) {
            best = cost;
            g = g2;
          }
        }
        H->w2_g = g;
        H->piece_next = 0;
        H->w2_next = 0;
      }
      {
        const uint32_t per = (nwin + NT - 1) / NT;
        const uint32_t b1 = min(tid * per + per, nwin);
        const uint32_t b0 = min(max(tid * per, first_kept(rr0, nwin)), b1);
        for (uint32_t k = 0; k < NS; ++k) s_cnt[k * NT + tid] = static_cast<uint16_t>(s_cnt[k * NT + tid] + H->round_base[k]);
        // the entries of the share with work: string fields, and records that
        // end with the wrong number of fields (rare); the others need nothing
        static_assert(Shape::B / 4 <= 64, "a share has at most 64 entries");
        uint64_t work = 0;
        for (uint32_t g = b0; g < b1; ++g) {
          const uint32_t fe = s_fe[g];
          const uint32_t c = (fe >> 16) & 0xFFu;
          const bool str = NS > 0 && c < C && TB.str_slot[c] != 0xFF;
          const bool rej = !INFER && (fe & kEntRec) && c + 1 != C && !((fe & kEntOpen) != 0 && open_dead);
          if (str || rej) work |= 1ull << (g - b0);
        }
        const int trips = __reduce_max_sync(0xffffffffu, static_cast<unsigned>(__popcll(work)));
        for (int it = 0; it < trips; ++it) {  // the same trip count in every lane (warp-wide copies)
          bool is_long = false, contiguous = true;
          int fd = 0, e_cur = 0;
          uint32_t nb = 0;
          uint8_t* gdst = nullptr;
          if (work) {
          const uint32_t g = b0 + static_cast<uint32_t>(__ffsll(static_cast<long long>(work)) - 1);
          work &= work - 1;
          const int eprev = g == 0 ? prev_pos : static_cast<int>(s_fe[g - 1] & kEntPos);
          const uint32_t fe = s_fe[g];
          const int e = static_cast<int>(fe & kEntPos);
          e_cur = e;
          const uint32_t c = (fe >> 16) & 0xFFu;
          if (NS > 0) {
            if (c < C && TB.str_slot[c] != 0xFF) {  // data bytes are counted for string fields only
              const uint32_t de = data_before(e), dprev = data_before(eprev + 1);
              const uint32_t slot = TB.str_slot[c];
              const uint16_t run = static_cast<uint16_t>(s_cnt[slot * NT + tid] + (de - dprev));
              s_cnt[slot * NT + tid] = run;
              s_fo[g] = static_cast<uint16_t>(run - de);
              if (de > dprev && !(((fe & kEntOpen) != 0) && open_dead)) {
                const uint64_t off = static_cast<uint64_t>(H->col_base[slot]) + static_cast<uint16_t>(run - (de - dprev));
                const uint64_t cap = cols[c].values_cap;
                nb = off >= cap ? 0u : static_cast<uint32_t>(min(static_cast<uint64_t>(de - dprev), cap - off));
                if (nb > 0) {
                  gdst = static_cast<uint8_t*>(cols[c].values) + off;
                  fd = first_data(eprev + 1, e);
                  contiguous = data_before(fd + static_cast<int>(nb)) == dprev + nb;
                  if (nb > kLongField) {  // queued in pieces for the block, else (queue full) copied by this warp below
                    const uint32_t span = contiguous ? nb : static_cast<uint32_t>(e - fd);
                    const uint32_t np = (span + kPiece - 1) / kPiece;
                    const uint32_t q = atomicAdd(&H->npieces, np);
                    if (q + np <= kMaxPieces) {  // the pieces written form a prefix of the queue
                      for (uint32_t k = 0; k < np; ++k) {
                        const uint32_t x0 = static_cast<uint32_t>(fd) + k * kPiece;
                        H->pieces[q + k] =
                            contiguous ? Piece{gdst + k * kPiece, static_cast<uint16_t>(x0),
                                               static_cast<uint16_t>(min(kPiece, nb - k * kPiece)), kContiguousPiece, 0}
                                       : Piece{gdst, static_cast<uint16_t>(x0),
                                               static_cast<uint16_t>(min(kPiece, static_cast<uint32_t>(e) - x0)),
                                               static_cast<uint16_t>(fd), static_cast<uint16_t>(nb)};
                      }
                      atomicMax(&H->npieces_ok, q + np);
                    } else {
                      is_long = true;
                    }
                  } else if (contiguous) {
                    smem_copy(gdst, s_tile + fd, static_cast<int>(nb));
                  } else {
                    uint32_t m = 0;
                    for (int x = fd; x < e && m < nb; ++x)
                      if ((s_dm[(x / B) * MW + ((x % B) >> 6)] >> ((x % B) & 63)) & 1ull) gdst[m++] = s_tile[x];
                  }
                }
              }
            }
          }
          if (!INFER && (fe & kEntRec) && c + 1 != C && !((fe & kEntOpen) != 0 && open_dead)) {
            // the record ends with the wrong number of fields: reject it and
            // give the missing columns their defaults
            uint32_t klo = 0, khi = nrec_win - 1;
            while (klo < khi) {
              const uint32_t mid = (klo + khi + 1) >> 1;
              if (s_rec[mid] <= g) klo = mid; else khi = mid - 1;
            }
            const uint64_t row = row0 + rr0 + klo;
            if (row < rows_cap) {
              atomicOr(&J.fail_bits[row >> 5], 1u << (row & 31));
              for (uint32_t c2 = c + 1; c2 < C; ++c2) {
                const uint32_t slot = TB.str_slot[c2];
                if (slot != 0xFF)
                  cols[c2].offsets[row + 1] = H->col_base[slot] + s_cnt[slot * NT + tid];
                else if (TB.num_slot[c2] != 0xFF)
                  store_value(cols[c2], TB.col_type[c2], row, 0);
              }
            }
          }
          }
          if (NS > 0) {
            uint32_t longs = __ballot_sync(0xffffffffu, is_long);
            while (longs) {
              const int src = __ffs(static_cast<int>(longs)) - 1;
              longs &= longs - 1;
              const int lfd = __shfl_sync(0xffffffffu, fd, src);
              const uint32_t lnb = __shfl_sync(0xffffffffu, nb, src);
              uint8_t* ldst = reinterpret_cast<uint8_t*>(
                  __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(gdst), src));
              if (__shfl_sync(0xffffffffu, contiguous, src)) {
                warp_copy_out(ldst, s_tile + lfd, static_cast<int>(lnb), lane);
              } else {  // data bytes with gaps: each lane places the bytes it holds by their rank
                const int le = __shfl_sync(0xffffffffu, e_cur, src);  // the field's end
                const uint32_t d0 = data_before(lfd);
                for (int u = lfd / B; u * B < le; ++u) {
                  for (int x = u * B + lane; x < (u + 1) * B; x += 32) {
                    if (x < lfd || x >= le) continue;
                    const int ix = x - u * B;
                    if ((s_dm[u * MW + (ix >> 6)] >> (ix & 63)) & 1ull) {
                      const uint32_t rank = data_before(x) - d0;
                      if (rank < lnb) ldst[rank] = s_tile[x];
                    }
                  }
                }
              }
            }
          }
        }
      }
      PP_WSPAN(2);
      __syncthreads();
      PP_PHASE(10);
      PP_WMARK();
      // the queued pieces of long fields, taken by whichever warp is free (a
      // whole field per warp leaves one warp copying a long text while the
      // block waits for it)
      {
        const uint32_t total = H->npieces_ok;
        uint32_t pn = 0;
        if (lane == 0) pn = atomicAdd(&H->piece_next, 1u);
        for (uint32_t p = __shfl_sync(0xffffffffu, pn, 0); p < total; p = __shfl_sync(0xffffffffu, pn, 0)) {
          // the next claim is issued before this piece is copied, so its
          // latency is hidden behind the copy
          if (lane == 0) pn = atomicAdd(&H->piece_next, 1u);
          const uint4 raw = reinterpret_cast<const uint4*>(H->pieces)[p];
          uint8_t* dst = reinterpret_cast<uint8_t*>((static_cast<uint64_t>(raw.y) << 32) | raw.x);
          const int x0 = static_cast<int>(raw.z & 0xFFFFu), len = static_cast<int>(raw.z >> 16);
          const uint32_t fd = raw.w & 0xFFFFu, nb = raw.w >> 16;
          if (fd == kContiguousPiece) {
            warp_copy_out(dst, s_tile + x0, len, lane);
          } else {
            // data bytes with gaps (a doubled quote, say): the runs between
            // the piece's non-data bytes, in order.  Each lane reads the
            // data bits of 16 aligned positions (inside one mask word of one
            // chunk); the warp walks the non-data positions it found.
            const int x1 = x0 + len;
            uint32_t rank = data_before(x0) - data_before(static_cast<int>(fd));  // of run start a
            int a = x0;
            for (int q0 = x0 & ~15; q0 < x1 && rank < nb; q0 += 512) {
              const int q = q0 + 16 * lane;
              uint32_t gap = 0;
              if (q < x1) {
                const int u = q / B, i = q - u * B;
                gap = ~static_cast<uint32_t>(s_dm[u * MW + (i >> 6)] >> (i & 63)) & 0xFFFFu;
                if (q < x0) gap &= ~((1u << (x0 - q)) - 1u);
                if (x1 - q < 16) gap &= (1u << (x1 - q)) - 1u;
              }
              for (uint32_t ls = __ballot_sync(0xffffffffu, gap != 0); ls && rank < nb; ls &= ls - 1) {
                const int src = __ffs(static_cast<int>(ls)) - 1;
                for (uint32_t gm = __shfl_sync(0xffffffffu, gap, src); gm && rank < nb; gm &= gm - 1) {
                  const int g = q0 + 16 * src + __ffs(static_cast<int>(gm)) - 1;
                  if (g > a) {
                    warp_copy_out(dst + rank, s_tile + a, min(g - a, static_cast<int>(nb - rank)), lane);
                    rank += static_cast<uint32_t>(g - a);
                  }
                  a = g + 1;
                }
              }
            }
            if (a < x1 && rank < nb) warp_copy_out(dst + rank, s_tile + a, min(x1 - a, static_cast<int>(nb - rank)), lane);
          }
        }
      }

      PP_WSPAN(3);
      PP_WMARK();
      // (2) string offsets and numeric conversions, record by record: G
      // threads per record take every G-th field (G chosen in step (1)).
      // Work item j is share j / nk of record j % nk, so the lanes of a warp
      // take consecutive records and store each column side by side.
      const uint32_t G = H->w2_g;  // written before the barrier after step (1)
      const uint32_t ks = round_skip(rr0, nrec_win);  // skipped records lead the round
      const uint32_t nk = nrec_win - ks;
      if constexpr (INFER) {
        // (2') inference: the fields of each record that ends here, and the
        // narrowest type of every non-empty field that starts here
        for (uint32_t j = tid; j < nk * G; j += NT) {
          const uint32_t sub = j / nk, k = ks + (j - sub * nk);
          const uint32_t gb = s_rec[k], ge = k + 1 < nrec_win ? s_rec[k + 1] : nwin;
          if (sub == 0 && ge > gb) {
            const uint32_t fl = s_fe[ge - 1];
            if ((fl & kEntRec) && !(((fl & kEntOpen) != 0) && open_dead)) {
              const uint32_t n = min(((fl >> 16) & 0xFFu) + 1u, static_cast<uint32_t>(PP_INFER_MAX_FIELDS));
              atomicMin(&s_inf[PP_MAX_COLUMNS], n);
              atomicMax(&s_inf[PP_MAX_COLUMNS + 1], n);
            }
          }
          for (uint32_t g = gb + sub; g < ge; g += G) {
            const uint32_t fe = s_fe[g];
            const uint32_t c = (fe >> 16) & 0xFFu;
            const bool open = (fe & kEntOpen) != 0;
            if (c >= PP_MAX_COLUMNS || (open && open_dead)) break;
            if (!(f0 + g > 0 || t == 0)) continue;  // started in an earlier tile, typed there
            const int e = static_cast<int>(fe & kEntPos);
            const int a = g > 0 ? static_cast<int>(s_fe[g - 1] & kEntPos) + 1 : (f0 == 0 ? P0 : prev_pos + 1);
            const bool ended = !open || last_tile;
            // the field's data bytes (as in convert_field), then the first
            // type of int32, int64, float64 that takes them, else string
            const int n_in = static_cast<int>(data_before(e) - data_before(a));
            uint8_t buf[kNumericMaxLen + 1];
            const uint8_t* txt = buf;
            int m = 0;
            if (ended && n_in == e - a) {
              txt = s_tile + a;
              m = n_in;
            } else {
              for (int y = a; y < e && m <= kNumericMaxLen; ++y) {
                const int u = y / B, i = y - u * B;
                if ((s_dm[u * MW + (i >> 6)] >> (i & 63)) & 1ull) buf[m++] = s_tile[y];
              }
              if (!ended && m <= kNumericMaxLen) {
                uint32_t s = tile_send;
                for (uint64_t gg = v1; gg < VL; ++gg) {
                  const uint8_t b = vbase[gg];
                  const uint32_t grp = TB.group_of[b];
                  const uint32_t tag = (TB.emit[grp] >> (2 * s)) & 3u;
                  s = vget(TB.trans[grp], s);
                  if (tag == PP_TAG_DATA) {
                    buf[m++] = b;
                    if (m > kNumericMaxLen) break;
                  } else if (tag != PP_TAG_CONTROL) {
                    break;
                  }
                  if (s == TB.invalid_state) break;
                }
              }
            }
            if (m == 0) continue;  // empty: no type
            uint32_t rank = 4;
            uint64_t v;
            if (m <= kNumericMaxLen) {
              if (convert_value(PP_INT32, txt, m, &v) == kConvOk) rank = 1;
              else if (convert_value(PP_INT64, txt, m, &v) == kConvOk) rank = 2;
              else if (convert_value(PP_FLOAT64, txt, m, &v) == kConvOk) rank = 3;
            }
            atomicMax(&s_inf[c], rank);
          }
        }
      } else {
        // work items in runs of 32 taken by whichever warp is free (a warp
        // that copied long pieces late takes fewer), so the tile's last
        // barrier waits less; a run keeps a warp's lanes on consecutive
        // records
        for (uint32_t jn = lane == 0 ? atomicAdd(&H->w2_next, 32u) : 0u, j0 = __shfl_sync(0xffffffffu, jn, 0);
             j0 < nk * G; j0 = __shfl_sync(0xffffffffu, jn, 0)) {
          if (lane == 0) jn = atomicAdd(&H->w2_next, 32u);  // the next run's claim, ahead of this one's work
          const uint32_t j = j0 + static_cast<uint32_t>(lane);
          if (j >= nk * G) continue;
          const uint32_t sub = j / nk, k = ks + (j - sub * nk);
          const uint64_t row = row0 + rr0 + k;
          if (row >= rows_cap) continue;
          const uint32_t gb = s_rec[k], ge = k + 1 < nrec_win ? s_rec[k + 1] : nwin;
          for (uint32_t g = gb + sub; g < ge; g += G) {
            const uint32_t fe = s_fe[g];
            const uint32_t c = (fe >> 16) & 0xFFu;
            const bool open = (fe & kEntOpen) != 0;
            if (c >= C || (open && open_dead)) break;
            const int e = static_cast<int>(fe & kEntPos);
            const uint32_t slot = TB.str_slot[c];
            if (slot != 0xFF) {
              if (!open || (fe & kEntRec))
                cols[c].offsets[row + 1] =
                    H->col_base[slot] + static_cast<uint16_t>(s_fo[g] + data_before(e));
            } else if (TB.num_slot[c] != 0xFF && (f0 + g > 0 || t == 0)) {
              const int a = g > 0 ? static_cast<int>(s_fe[g - 1] & kEntPos) + 1 : (f0 == 0 ? P0 : prev_pos + 1);
              convert_field(row, c, a, e, !open || last_tile);
            }
          }
        }
      }

      PP_WSPAN(4);
      PP_PHASE(11);
      __syncthreads();
      PP_PHASE(12);
      if (r + 1 < nrounds) next_round();
    }
    if constexpr (INFER) {  // after the round loop's last barrier
      if (tid < PP_MAX_COLUMNS && s_inf[tid]) atomicMax(&J.misc->inf_rank[tid], s_inf[tid]);
      if (tid == PP_MAX_COLUMNS && s_inf[tid] != 0xFFFFFFFFu) atomicMin(&J.misc->inf_min_fields, s_inf[tid]);
      if (tid == PP_MAX_COLUMNS + 1 && s_inf[tid]) atomicMax(&J.misc->inf_max_fields, s_inf[tid]);
    }
    if (last_tile && tid == 0) {
      const uint64_t recs = (H->prefix_rc & kRecMask) + rec_tile + (trailing ? 1u : 0u);  // of the input
      J.misc->rows = static_cast<int64_t>(recs > TB.skip_records ? recs - TB.skip_records : 0u);  // read by the finalize kernel only
      J.misc->final_state = static_cast<int32_t>(tile_send);
      for (uint32_t k = 0; k < NS; ++k) J.misc->bytes_total[k] = H->col_base[k] + H->tile_tot[k];
      J.misc->done = 1u;
    }

    PP_PHASE(9);  // the last barrier of the round loop ends the tile
#ifdef PP_PHASE_TIMING
    if (tid == 0) {  // every warp's spans of this tile ended before that barrier
      for (int k = 0; k < 8; ++k) {
        H->ph_cycles[16 + k] += static_cast<long long>(H->w_max[k]);
        H->ph_cycles[24 + k] += static_cast<long long>(H->w_sum[k]);
        H->w_max[k] = H->w_sum[k] = 0;
      }
    }
#endif
  }
#ifdef PP_PHASE_TIMING
  if (tid == 0 && L.phase_cycles != nullptr)
    for (int k = 0; k < 32; ++k) atomicAdd(&L.phase_cycles[k], static_cast<unsigned long long>(H->ph_cycles[k]));
#endif
}

}  // namespace pp
