// Skipping rows (Sec. 4.3): the pruning pass that drops whole physical lines
// from the raw input before a parse (the C ABI in include/parparaw.h).
//
// Positions are virtual: the input starts `head` bytes into a 16-byte aligned
// origin, so every 16-byte vector load is aligned; bytes outside the input
// are never read (partial vectors are read byte by byte).  The virtual range
// is cut into chunks of kChunk bytes, one block each, kSeg bytes per thread:
//   1. every block counts the line terminators of its chunk;
//   2. one block scans the counts: the row number at each chunk's start;
//   3. every block numbers the rows of each thread's segment and counts the
//      bytes that stay;
//   4. one block scans those counts: each chunk's output position;
//   5. every block compacts the bytes that stay into shared memory and
//      writes them out with 4-byte stores.
// A segment is described by 64-bit masks (valid bytes, terminators); a
// cursor into the sorted list of dropped rows, placed by a binary search at
// the segment's first row, tells which of its rows go.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/parparaw.h"

namespace {

constexpr int kThreads = 256;
constexpr int kSeg = 64;                 // bytes per thread: one 64-bit mask
constexpr int kChunk = kThreads * kSeg;  // bytes per block
constexpr int kScanThreads = 1024;

struct Input {
  const uint8_t* vbase;  // 16-byte aligned; the input is [head, vlen) from here
  uint64_t head, vlen;
};

__device__ __forceinline__ uint64_t bits_below(int n) {
  return n <= 0 ? 0ull : (n >= 64 ? ~0ull : ((1ull << n) - 1ull));
}

// Inclusive sum over the block of one value per thread; returns it and
// leaves the block total in *total.  `ws` is kThreads / 32 words.
__device__ uint64_t block_inclusive_sum(uint64_t v, uint64_t* ws, uint64_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += o;
  }
  if (lane == 31) ws[warp] = v;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = lane < kThreads / 32 ? ws[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t o = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += o;
    }
    if (lane < kThreads / 32) ws[lane] = w;
  }
  __syncthreads();
  const uint64_t r = v + (warp > 0 ? ws[warp - 1] : 0);
  *total = ws[kThreads / 32 - 1];
  __syncthreads();  // ws may be reused
  return r;
}

// The first index of rows[0..n) holding a row >= r.
__device__ uint64_t lower_bound(const uint64_t* rows, uint64_t n, uint64_t r) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (rows[mid] < r) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// This thread's segment: its bytes (zero outside the input), which of them
// are input bytes, which are terminators.
struct Segment {
  uint4 q[kSeg / 16];
  uint64_t valid, term;
};

__device__ Segment load_segment(const Input& in, uint64_t v0, uint8_t terminator) {
  Segment s;
  const int lo = static_cast<int>(in.head > v0 ? (in.head - v0 < kSeg ? in.head - v0 : kSeg) : 0);
  const int hi = static_cast<int>(in.vlen > v0 ? (in.vlen - v0 < kSeg ? in.vlen - v0 : kSeg) : 0);
  s.valid = lo < hi ? bits_below(hi) & ~bits_below(lo) : 0ull;
  const uint32_t rep = 0x01010101u * terminator;
  s.term = 0;
#pragma unroll
  for (int k = 0; k < kSeg / 16; ++k) {
    const uint64_t a = v0 + 16u * k;
    if (a >= in.head && a + 16 <= in.vlen) {
      s.q[k] = *reinterpret_cast<const uint4*>(in.vbase + a);
    } else {  // a partial vector: only its input bytes are read
      uint32_t w[4] = {0u, 0u, 0u, 0u};
      for (int i = 0; i < 16; ++i)
        if (a + i >= in.head && a + i < in.vlen) w[i >> 2] |= static_cast<uint32_t>(in.vbase[a + i]) << (8 * (i & 3));
      s.q[k] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    const uint32_t wd[4] = {s.q[k].x, s.q[k].y, s.q[k].z, s.q[k].w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      // exact zero-byte test of word ^ terminator: the high bit of each byte
      // is set iff that byte equals the terminator
      const uint32_t x = wd[j] ^ rep;
      const uint32_t z = ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x | 0x7F7F7F7Fu);
      const uint32_t bits4 = (((z >> 7) * 0x00204081u) >> 21) & 0xFu;
      s.term |= static_cast<uint64_t>(bits4) << (16 * k + 4 * j);
    }
  }
  s.term &= s.valid;
  return s;
}

// The bytes of a segment that stay: its rows start at row `row` (the row of
// its first input byte); a row ends with its terminator, and a row listed in
// rows[0..n) loses all its bytes.  The common segment touches no dropped row
// and keeps every input byte.
__device__ uint64_t keep_mask(const Segment& s, uint64_t row, const uint64_t* rows, uint64_t n) {
  const int m = __popcll(s.term);  // the segment holds rows row .. row + m
  uint64_t p = lower_bound(rows, n, row);
  uint64_t keep = s.valid;
  for (; p < n && rows[p] <= row + static_cast<uint64_t>(m); ++p) {
    // row row + k spans the bits after its segment's k-th terminator up to
    // and including the (k+1)-th
    const int k = static_cast<int>(rows[p] - row);
    uint64_t rest = s.term;  // the terminators from the (k+1)-th on
    for (int j = 0; j < k; ++j) rest &= rest - 1;
    const uint64_t done = s.term & ~rest;  // the first k terminators
    const int b0 = k == 0 ? 0 : 64 - __clzll(static_cast<long long>(done));
    const int b1 = rest ? __ffsll(static_cast<long long>(rest)) : 64;
    keep &= ~(bits_below(b1) & ~bits_below(b0));
  }
  return keep;
}

// 2. / 4. exclusive scan of n counts by one block; *total = the sum
__global__ void __launch_bounds__(kScanThreads) rows_scan_kernel(const uint32_t* in, uint64_t* out, uint64_t n,
                                                                 uint64_t* total) {
  __shared__ uint64_t ws[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t per = (n + kScanThreads - 1) / kScanThreads;
  const uint64_t lo = threadIdx.x * per < n ? threadIdx.x * per : n;
  const uint64_t hi = lo + per < n ? lo + per : n;
  uint64_t s = 0;
  for (uint64_t i = lo; i < hi; ++i) s += in[i];
  uint64_t v = s;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += o;
  }
  if (lane == 31) ws[warp] = v;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = ws[lane];  // kScanThreads / 32 == 32 warps
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t o = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += o;
    }
    ws[lane] = w;
  }
  __syncthreads();
  uint64_t run = v - s + (warp > 0 ? ws[warp - 1] : 0);
  for (uint64_t i = lo; i < hi; ++i) {
    out[i] = run;
    run += in[i];
  }
  if (threadIdx.x == 0) *total = ws[31];
}

__device__ __forceinline__ uint64_t segment_start(int t) {
  return static_cast<uint64_t>(blockIdx.x) * kChunk + static_cast<uint64_t>(t) * kSeg;
}

// 1. terminators per chunk
__global__ void __launch_bounds__(kThreads) rows_count_kernel(Input in, uint8_t term, uint32_t* cnt) {
  __shared__ uint64_t ws[kThreads / 32];
  const Segment s = load_segment(in, segment_start(threadIdx.x), term);
  uint64_t total;
  block_inclusive_sum(static_cast<uint64_t>(__popcll(s.term)), ws, &total);
  if (threadIdx.x == 0) cnt[blockIdx.x] = static_cast<uint32_t>(total);
}

// A thread's segment with its first row and the bytes of it that stay
// (rows numbered by the scan of the chunk counts).
struct Kept {
  Segment s;
  uint64_t keep;
};

__device__ Kept segment_keep(const Input& in, uint8_t term, const uint64_t* rows, uint64_t nrows,
                             const uint64_t* row0, uint64_t* ws) {
  Kept k;
  k.s = load_segment(in, segment_start(threadIdx.x), term);
  const uint64_t t = static_cast<uint64_t>(__popcll(k.s.term));
  uint64_t total;
  const uint64_t inc = block_inclusive_sum(t, ws, &total);
  k.keep = keep_mask(k.s, row0[blockIdx.x] + inc - t, rows, nrows);
  return k;
}

// 3. bytes that stay, per chunk
__global__ void __launch_bounds__(kThreads) rows_keep_kernel(Input in, uint8_t term, const uint64_t* rows,
                                                             uint64_t nrows, const uint64_t* row0, uint32_t* kept) {
  __shared__ uint64_t ws[kThreads / 32];
  const Kept k = segment_keep(in, term, rows, nrows, row0, ws);
  uint64_t total;
  block_inclusive_sum(static_cast<uint64_t>(__popcll(k.keep)), ws, &total);
  if (threadIdx.x == 0) kept[blockIdx.x] = static_cast<uint32_t>(total);
}

// 5. the bytes that stay, compacted in shared memory, then stored with
// 4-byte stores at the chunk's output position
__global__ void __launch_bounds__(kThreads) rows_write_kernel(Input in, uint8_t term, const uint64_t* rows,
                                                              uint64_t nrows, const uint64_t* row0,
                                                              const uint64_t* out0, uint8_t* out) {
  __shared__ uint64_t ws[kThreads / 32];
  __shared__ __align__(16) uint8_t tile[kChunk];
  __shared__ __align__(16) uint8_t buf[kChunk + 16];
  const Kept k = segment_keep(in, term, rows, nrows, row0, ws);
  const uint64_t nk = static_cast<uint64_t>(__popcll(k.keep));
  uint64_t total;
  const uint32_t o = static_cast<uint32_t>(block_inclusive_sum(nk, ws, &total) - nk);  // first position in buf
  const uint32_t w[16] = {k.s.q[0].x, k.s.q[0].y, k.s.q[0].z, k.s.q[0].w, k.s.q[1].x, k.s.q[1].y,
                          k.s.q[1].z, k.s.q[1].w, k.s.q[2].x, k.s.q[2].y, k.s.q[2].z, k.s.q[2].w,
                          k.s.q[3].x, k.s.q[3].y, k.s.q[3].z, k.s.q[3].w};
  if (k.keep == ~0ull) {
    // the whole segment stays: byte i goes to buf[o + i]; whole words by
    // funnel shifts, the partial first and last words byte by byte (their
    // other bytes belong to the neighbouring segments)
    const uint32_t a = o & 3u, base = o - a;
    uint32_t* b32 = reinterpret_cast<uint32_t*>(buf + base);
    if (a == 0) {
#pragma unroll
      for (int d = 0; d < 16; ++d) b32[d] = w[d];
    } else {
      for (uint32_t c = a; c < 4; ++c) buf[base + c] = static_cast<uint8_t>(w[0] >> (8 * (c - a)));
#pragma unroll
      for (int d = 1; d < 16; ++d) b32[d] = __funnelshift_l(w[d - 1], w[d], 8 * a);
      for (uint32_t c = 0; c < a; ++c) buf[base + 64 + c] = static_cast<uint8_t>(w[15] >> (8 * (4 - a + c)));
    }
  } else if (k.keep) {  // some bytes go: the segment's own copy in `tile`, then byte by byte
    uint4* t4 = reinterpret_cast<uint4*>(tile + threadIdx.x * kSeg);
#pragma unroll
    for (int j = 0; j < kSeg / 16; ++j) t4[j] = k.s.q[j];
    const uint8_t* src = tile + threadIdx.x * kSeg;
    uint32_t at = o;
    for (uint64_t m = k.keep; m; m &= m - 1) buf[at++] = src[__ffsll(static_cast<long long>(m)) - 1];
  }
  __syncthreads();
  const uint32_t n = static_cast<uint32_t>(total);
  uint8_t* dst = out + out0[blockIdx.x];
  const uint32_t head = min(n, static_cast<uint32_t>((4u - (reinterpret_cast<uintptr_t>(dst) & 3u)) & 3u));
  if (threadIdx.x < head) dst[threadIdx.x] = buf[threadIdx.x];
  const uint32_t nw = (n - head) >> 2, sh = 8u * (head & 3u);
  const uint32_t* s32 = reinterpret_cast<const uint32_t*>(buf);  // reads may pass n by up to 4 bytes
  uint32_t* d32 = reinterpret_cast<uint32_t*>(dst + head);
  for (uint32_t i = threadIdx.x; i < nw; i += kThreads) {
    const uint32_t x = (head >> 2) + i;  // head < 4: buf word i holds bytes 4i .. 4i + 3
    d32[i] = __funnelshift_r(s32[x], s32[x + 1], sh);
  }
  const uint32_t tail = head + 4 * nw;
  if (threadIdx.x < n - tail) dst[tail + threadIdx.x] = buf[tail + threadIdx.x];
}

uint64_t num_chunks(uint64_t vlen) { return (vlen + kChunk - 1) / kChunk; }

}  // namespace

// Scratch: per chunk a row number, an output position, a terminator count
// and a kept count; then the two totals.  Sized for the worst alignment.
extern "C" uint64_t parparaw_skip_rows_scratch_bytes(uint64_t len) {
  const uint64_t nb = num_chunks(len + 15);
  return nb * (8 + 8 + 4 + 4) + 16 + 64;
}

extern "C" pp_status parparaw_skip_rows(const uint8_t* input, uint64_t len, const uint64_t* rows, uint64_t nrows,
                                        uint8_t terminator, uint8_t* output, uint64_t* output_len, void* scratch,
                                        uint64_t scratch_bytes, void* stream_) {
  if (output_len == nullptr) return PP_E_ARG;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  if (len == 0) {
    return cudaMemsetAsync(output_len, 0, sizeof(uint64_t), stream) == cudaSuccess ? PP_OK : PP_E_CUDA;
  }
  if (input == nullptr || output == nullptr || scratch == nullptr || (nrows > 0 && rows == nullptr))
    return PP_E_ARG;
  if (scratch_bytes < parparaw_skip_rows_scratch_bytes(len) || (reinterpret_cast<uintptr_t>(scratch) & 15u))
    return PP_E_ARG;
  Input in;
  in.head = reinterpret_cast<uintptr_t>(input) & 15u;
  in.vbase = input - in.head;
  in.vlen = in.head + len;
  const uint64_t nb = num_chunks(in.vlen);
  if (nb > 0x7FFFFFFFull) return PP_E_UNSUPPORTED;
  uint64_t* row0 = static_cast<uint64_t*>(scratch);
  uint64_t* out0 = row0 + nb;
  uint64_t* totals = out0 + nb;  // [0] terminators, [1] bytes kept
  uint32_t* cnt = reinterpret_cast<uint32_t*>(totals + 2);
  uint32_t* kept = cnt + nb;
  const unsigned grid = static_cast<unsigned>(nb);
  rows_count_kernel<<<grid, kThreads, 0, stream>>>(in, terminator, cnt);
  rows_scan_kernel<<<1, kScanThreads, 0, stream>>>(cnt, row0, nb, &totals[0]);
  rows_keep_kernel<<<grid, kThreads, 0, stream>>>(in, terminator, rows, nrows, row0, kept);
  rows_scan_kernel<<<1, kScanThreads, 0, stream>>>(kept, out0, nb, &totals[1]);
  rows_write_kernel<<<grid, kThreads, 0, stream>>>(in, terminator, rows, nrows, row0, out0, output);
  if (cudaMemcpyAsync(output_len, &totals[1], sizeof(uint64_t), cudaMemcpyDeviceToDevice, stream) != cudaSuccess)
    return PP_E_CUDA;
  return cudaGetLastError() == cudaSuccess ? PP_OK : PP_E_CUDA;
}
