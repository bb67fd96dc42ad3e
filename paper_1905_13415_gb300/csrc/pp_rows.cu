// Skipping rows (Sec. 4.3): the pruning pass that drops whole physical lines
// from the raw input before a parse (the C ABI in include/parparaw.h).  The
// input is cut into chunks of kChunk bytes, one block each:
//   1. every block counts the line terminators of its chunk;
//   2. one block scans the counts: the row number at each chunk's start;
//   3. every block stages its chunk in shared memory, numbers the rows of
//      each thread's segment and counts the bytes that stay;
//   4. one block scans those counts: each chunk's output position;
//   5. every block writes the bytes that stay, each thread its segment.
// A thread walks its segment with a cursor into the sorted list of dropped
// rows (a binary search places it at the segment's first row).
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/parparaw.h"

namespace {

constexpr int kThreads = 256;
constexpr int kSeg = 64;                      // bytes per thread
constexpr int kChunk = kThreads * kSeg;       // bytes per block
constexpr int kScanThreads = 1024;

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

// 1. terminators per chunk (coalesced byte loads)
__global__ void __launch_bounds__(kThreads) rows_count_kernel(const uint8_t* in, uint64_t len, uint8_t term,
                                                              uint32_t* cnt) {
  __shared__ uint64_t ws[kThreads / 32];
  const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kChunk;
  const uint64_t end = base + kChunk < len ? base + kChunk : len;
  uint64_t n = 0;
  for (uint64_t i = base + threadIdx.x; i < end; i += kThreads) n += in[i] == term;
  uint64_t total;
  block_inclusive_sum(n, ws, &total);
  if (threadIdx.x == 0) cnt[blockIdx.x] = static_cast<uint32_t>(total);
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

// The first index of rows[0..n) holding a row >= r.
__device__ uint64_t lower_bound(const uint64_t* rows, uint64_t n, uint64_t r) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (rows[mid] < r) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// A cursor into the sorted list of dropped rows, for rows visited in
// ascending order; `next` caches the first listed row not below the last
// one asked about.
struct Cursor {
  const uint64_t* rows;
  uint64_t n, p, next;
  __device__ Cursor(const uint64_t* r, uint64_t nr, uint64_t row) : rows(r), n(nr), p(lower_bound(r, nr, row)) {
    next = p < n ? rows[p] : ~0ull;
  }
  __device__ bool dropped(uint64_t row) {
    while (next < row) {
      ++p;
      next = p < n ? rows[p] : ~0ull;
    }
    return next == row;
  }
};

// The chunk in shared memory, and each thread's segment [s0, s1) of it with
// the row number at its start.
struct Segment {
  int s0, s1;
  uint64_t row;
};

__device__ Segment stage(const uint8_t* in, uint64_t len, uint8_t term, const uint64_t* row0, uint8_t* tile,
                         uint64_t* ws) {
  const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kChunk;
  const int n = static_cast<int>(base + kChunk < len ? kChunk : len - base);
  for (int i = threadIdx.x; i < n; i += kThreads) tile[i] = in[base + i];
  __syncthreads();
  Segment sg;
  sg.s0 = min(static_cast<int>(threadIdx.x) * kSeg, n);
  sg.s1 = min(sg.s0 + kSeg, n);
  uint64_t t = 0;
  for (int i = sg.s0; i < sg.s1; ++i) t += tile[i] == term;
  uint64_t total;
  const uint64_t inc = block_inclusive_sum(t, ws, &total);
  sg.row = row0[blockIdx.x] + inc - t;
  return sg;
}

// 3. bytes that stay, per chunk
__global__ void __launch_bounds__(kThreads) rows_keep_kernel(const uint8_t* in, uint64_t len, uint8_t term,
                                                             const uint64_t* rows, uint64_t nrows,
                                                             const uint64_t* row0, uint32_t* kept) {
  __shared__ uint8_t tile[kChunk];
  __shared__ uint64_t ws[kThreads / 32];
  const Segment sg = stage(in, len, term, row0, tile, ws);
  Cursor cur(rows, nrows, sg.row);
  uint64_t row = sg.row, k = 0;
  for (int i = sg.s0; i < sg.s1; ++i) {
    k += !cur.dropped(row);
    row += tile[i] == term;
  }
  uint64_t total;
  block_inclusive_sum(k, ws, &total);
  if (threadIdx.x == 0) kept[blockIdx.x] = static_cast<uint32_t>(total);
}

// 5. the bytes that stay, to their output positions
__global__ void __launch_bounds__(kThreads) rows_write_kernel(const uint8_t* in, uint64_t len, uint8_t term,
                                                              const uint64_t* rows, uint64_t nrows,
                                                              const uint64_t* row0, const uint64_t* out0,
                                                              uint8_t* out) {
  __shared__ uint8_t tile[kChunk];
  __shared__ uint64_t ws[kThreads / 32];
  const Segment sg = stage(in, len, term, row0, tile, ws);
  const Cursor first(rows, nrows, sg.row);
  Cursor cur = first;
  uint64_t row = sg.row, k = 0;
  for (int i = sg.s0; i < sg.s1; ++i) {  // count first, for this thread's output position
    k += !cur.dropped(row);
    row += tile[i] == term;
  }
  uint64_t total;
  const uint64_t inc = block_inclusive_sum(k, ws, &total);
  uint8_t* dst = out + out0[blockIdx.x] + (inc - k);
  row = sg.row;
  cur = first;
  for (int i = sg.s0; i < sg.s1; ++i) {
    if (!cur.dropped(row)) *dst++ = tile[i];
    row += tile[i] == term;
  }
}

uint64_t num_chunks(uint64_t len) { return (len + kChunk - 1) / kChunk; }

}  // namespace

// Scratch: per chunk a terminator count, a row number, a kept count and an
// output position; then the two totals.
extern "C" uint64_t parparaw_skip_rows_scratch_bytes(uint64_t len) {
  const uint64_t nb = num_chunks(len);
  return nb * (4 + 8 + 4 + 8) + 16 + 64;
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
  const uint64_t nb = num_chunks(len);
  if (nb > 0x7FFFFFFFull) return PP_E_UNSUPPORTED;
  uint8_t* s = static_cast<uint8_t*>(scratch);
  uint64_t* row0 = reinterpret_cast<uint64_t*>(s);
  uint64_t* out0 = row0 + nb;
  uint64_t* totals = out0 + nb;  // [0] terminators, [1] bytes kept
  uint32_t* cnt = reinterpret_cast<uint32_t*>(totals + 2);
  uint32_t* kept = cnt + nb;
  const unsigned grid = static_cast<unsigned>(nb);
  rows_count_kernel<<<grid, kThreads, 0, stream>>>(input, len, terminator, cnt);
  rows_scan_kernel<<<1, kScanThreads, 0, stream>>>(cnt, row0, nb, &totals[0]);
  rows_keep_kernel<<<grid, kThreads, 0, stream>>>(input, len, terminator, rows, nrows, row0, kept);
  rows_scan_kernel<<<1, kScanThreads, 0, stream>>>(kept, out0, nb, &totals[1]);
  rows_write_kernel<<<grid, kThreads, 0, stream>>>(input, len, terminator, rows, nrows, row0, out0, output);
  if (cudaMemcpyAsync(output_len, &totals[1], sizeof(uint64_t), cudaMemcpyDeviceToDevice, stream) != cudaSuccess)
    return PP_E_CUDA;
  return cudaGetLastError() == cudaSuccess ? PP_OK : PP_E_CUDA;
}
