// pp_stream.cu -- end-to-end streaming parse of host-resident input (Sec. 4.4)
// behind the C ABI: parparaw_stream_create / _parse / _destroy, declared in
// include/parparaw.h.
//
// Two device input buffers alternate.  While partition k is parsed out of one
// (stream s_parse), partition k+1 is copied into the other (s_h2d) and the
// columns of partition k-1 are copied to the caller's host arena (s_d2h).
// Each buffer holds a carry-over region in front of its partition: the bytes
// of partition k after its last record delimiter (the device reports where
// they start as `consumed`) are copied there, device to device, and parsed
// again at the start of partition k+1.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <initializer_list>
#include <new>

#include "pp_parser.h"

namespace {

constexpr uint64_t kArenaAlign = 64;

uint32_t value_width(uint32_t type) {
  return (type == PP_INT32 || type == PP_DATE_D) ? 4u : 8u;
}

// One set of device output columns and its descriptor.
struct OutSet {
  uint64_t rows_cap = 0;
  uint64_t caps[PP_MAX_COLUMNS] = {};
  pp_columns desc;
  bool allocated = false;
};

pp_status map_cuda(cudaError_t e) {
  if (e == cudaSuccess) return PP_OK;
  return e == cudaErrorMemoryAllocation ? PP_E_NOMEM : PP_E_CUDA;
}

}  // namespace

struct pp_streamer {
  pp_parser parser;  // a copy: options of the caller's parser at create time
  uint64_t part = 0, carry = 0;
  uint8_t* buf[2] = {nullptr, nullptr};
  OutSet out[2];
  pp_parse_result* res_dev = nullptr;   // the two sets' results (device)
  pp_parse_result* res_host = nullptr;  // their pinned host copies
  cudaStream_t s_h2d = nullptr, s_parse = nullptr, s_d2h = nullptr;
  cudaEvent_t h2d_done[2] = {}, parse_done[2] = {}, d2h_done[2] = {}, carry_done = nullptr;
  // the starts of each set's copy in, parse and copy out (timed against the
  // *_done events above, for the partitions' device times)
  cudaEvent_t h2d_start[2] = {}, parse_start[2] = {}, d2h_start[2] = {};
  uint8_t* scratch[2] = {nullptr, nullptr};  // each output set's parse scratch, sized with it
  size_t scratch_cap[2] = {0, 0};
};

namespace {

void free_outset(OutSet& o) {
  if (!o.allocated) return;
  for (uint32_t c = 0; c < o.desc.num_columns; ++c) {
    cudaFree(o.desc.cols[c].values);
    cudaFree(o.desc.cols[c].offsets);
    cudaFree(o.desc.cols[c].validity);
  }
  cudaFree(o.desc.row_valid);
  std::memset(&o.desc, 0, sizeof(o.desc));
  o.allocated = false;
}

// Device columns for rows_cap rows, string columns with the capacities in caps.
pp_status alloc_outset(pp_streamer* S, int b, uint64_t rows_cap, const uint64_t* caps) {
  OutSet& o = S->out[b];
  free_outset(o);
  std::memset(&o.desc, 0, sizeof(o.desc));
  const pp_parser& P = S->parser;
  const uint32_t C = P.tab.num_columns;
  const uint64_t nbits = (rows_cap + 7) / 8;
  o.desc.num_columns = C;
  o.desc.rows_cap = rows_cap;
  o.allocated = true;  // partial allocations are freed by free_outset
  cudaError_t e = cudaSuccess;
  for (uint32_t c = 0; c < C && e == cudaSuccess; ++c) {
    const uint32_t t = P.types[c];
    pp_column& col = o.desc.cols[c];
    if (t == PP_SKIP) continue;
    if (t == PP_STRING) {
      o.caps[c] = std::max<uint64_t>(caps[c], 1);
      col.values_cap = o.caps[c];
      e = cudaMalloc(&col.values, o.caps[c]);
      if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&col.offsets), 8 * (rows_cap + 1));
    } else {
      e = cudaMalloc(&col.values, std::max<uint64_t>(rows_cap, 1) * value_width(t));
    }
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&col.validity), std::max<uint64_t>(nbits, 1));
  }
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&o.desc.row_valid), std::max<uint64_t>(nbits, 1));
  if (e != cudaSuccess) {
    free_outset(o);
    return map_cuda(e);
  }
  o.rows_cap = rows_cap;
  o.desc.result = S->res_dev + b;
  // the parse scratch for a whole buffer into this set (status words, bitmaps)
  const size_t need = pp_parse_scratch_bytes(&S->parser, S->carry + S->part, rows_cap);
  if (need > S->scratch_cap[b]) {
    cudaFree(S->scratch[b]);
    S->scratch[b] = nullptr;
    S->scratch_cap[b] = 0;
    if ((e = cudaMalloc(reinterpret_cast<void**>(&S->scratch[b]), need)) != cudaSuccess) {
      free_outset(o);
      return map_cuda(e);
    }
    S->scratch_cap[b] = need;
  }
  return PP_OK;
}

// Parses buf[b][start, start + length) into output set b on s_parse, copies
// its result to pinned host memory and marks the set's parse as done.
pp_status enqueue_parse(pp_streamer* S, int b, uint64_t start, uint64_t length, bool last, bool first) {
  cudaError_t e0 = cudaEventRecord(S->parse_start[b], S->s_parse);
  if (e0 != cudaSuccess) return map_cuda(e0);
  pp_parser local = S->parser;
  local.tab.partial = last ? 0 : 1;
  local.tab.skip_records = first ? S->parser.tab.skip_records : 0;
  local.ev_start = local.ev_stop = nullptr;
  pp_status st = pp_parse_with_scratch(&local, length ? S->buf[b] + start : nullptr, length, &S->out[b].desc,
                                       S->s_parse, S->scratch[b], S->scratch_cap[b]);
  if (st != PP_OK) return st;
  cudaError_t e = cudaMemcpyAsync(S->res_host + b, S->res_dev + b, sizeof(pp_parse_result), cudaMemcpyDeviceToHost,
                                  S->s_parse);
  if (e == cudaSuccess) e = cudaEventRecord(S->parse_done[b], S->s_parse);
  return map_cuda(e);
}

// Bytes of the arena that a partition with this result needs.
uint64_t partition_arena_bytes(const pp_parser& P, const pp_parse_result& r) {
  const uint64_t rows = static_cast<uint64_t>(r.rows), nb = (rows + 7) / 8;
  auto up = [](uint64_t x) { return (x + kArenaAlign - 1) / kArenaAlign * kArenaAlign; };
  uint64_t n = up(nb);
  for (uint32_t c = 0; c < P.tab.num_columns; ++c) {
    const uint32_t t = P.types[c];
    if (t == PP_SKIP) continue;
    if (t == PP_STRING)
      n += up(std::max<uint64_t>(static_cast<uint64_t>(r.values_bytes_needed[c]), 1)) + up(8 * (rows + 1));
    else
      n += up(std::max<uint64_t>(rows, 1) * value_width(t));
    n += up(std::max<uint64_t>(nb, 1));
  }
  return n;
}

// Carves partition columns from the arena and enqueues their copies out of
// output set b on s_d2h (after the set's parse).
pp_status enqueue_copy_out(pp_streamer* S, int b, const pp_parse_result& r, uint8_t* arena, uint64_t* used,
                           pp_host_partition* part) {
  const pp_parser& P = S->parser;
  const OutSet& o = S->out[b];
  const uint64_t rows = static_cast<uint64_t>(r.rows), nb = (rows + 7) / 8;
  auto take = [&](uint64_t n) {
    uint8_t* p = arena + *used;
    *used += (std::max<uint64_t>(n, 1) + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
    return p;
  };
  cudaError_t e = cudaStreamWaitEvent(S->s_d2h, S->parse_done[b], 0);
  if (e == cudaSuccess) e = cudaEventRecord(S->d2h_start[b], S->s_d2h);
  auto copy = [&](void* dst, const void* src, uint64_t n) {
    if (e == cudaSuccess && n > 0) e = cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, S->s_d2h);
  };
  std::memset(part->cols, 0, sizeof(part->cols));
  part->rows = r.rows;
  for (uint32_t c = 0; c < P.tab.num_columns; ++c) {
    const uint32_t t = P.types[c];
    pp_column& h = part->cols[c];
    if (t == PP_SKIP) continue;
    if (t == PP_STRING) {
      const uint64_t bytes = static_cast<uint64_t>(r.values_bytes_needed[c]);
      h.values = take(bytes);
      h.values_cap = bytes;
      copy(h.values, o.desc.cols[c].values, bytes);
      h.offsets = reinterpret_cast<int64_t*>(take(8 * (rows + 1)));
      copy(h.offsets, o.desc.cols[c].offsets, 8 * (rows + 1));
    } else {
      h.values = take(rows * value_width(t));
      copy(h.values, o.desc.cols[c].values, rows * value_width(t));
    }
    h.validity = take(nb);
    copy(h.validity, o.desc.cols[c].validity, nb);
  }
  part->row_valid = take(nb);
  copy(part->row_valid, o.desc.row_valid, nb);
  if (e == cudaSuccess) e = cudaEventRecord(S->d2h_done[b], S->s_d2h);
  return map_cuda(e);
}

// Waits for set b's parse and returns its result; on PP_E_CAPACITY the set
// is regrown to the reported sizes (with headroom, so later partitions fit
// too) and the partition parsed again.
pp_status settle(pp_streamer* S, int b, uint64_t start, uint64_t length, bool last, bool first,
                 pp_parse_result* r) {
  cudaError_t e = cudaEventSynchronize(S->parse_done[b]);
  if (e != cudaSuccess) return map_cuda(e);
  *r = S->res_host[b];
  if (r->status != PP_E_CAPACITY) return PP_OK;
  if ((e = cudaEventSynchronize(S->d2h_done[b])) != cudaSuccess) return map_cuda(e);  // the set's last copy-out
  uint64_t caps[PP_MAX_COLUMNS];
  for (uint32_t c = 0; c < PP_MAX_COLUMNS; ++c) {
    const uint64_t need = static_cast<uint64_t>(std::max<int64_t>(r->values_bytes_needed[c], 1));
    caps[c] = std::max(S->out[b].caps[c], need + need / 4);
  }
  const uint64_t rows = std::max(S->out[b].rows_cap, static_cast<uint64_t>(r->rows) + static_cast<uint64_t>(r->rows) / 4 + 1);
  pp_status st = alloc_outset(S, b, rows, caps);
  if (st != PP_OK) return st;
  if ((st = enqueue_parse(S, b, start, length, last, first)) != PP_OK) return st;
  if ((e = cudaEventSynchronize(S->parse_done[b])) != cudaSuccess) return map_cuda(e);
  *r = S->res_host[b];
  return r->status == PP_E_CAPACITY ? PP_E_CUDA : PP_OK;  // exact sizes cannot fall short
}

void drain(pp_streamer* S) {
  cudaStreamSynchronize(S->s_h2d);
  cudaStreamSynchronize(S->s_parse);
  cudaStreamSynchronize(S->s_d2h);
}

}  // namespace

extern "C" void parparaw_stream_destroy(pp_streamer* S) {
  if (S == nullptr) return;
  if (S->s_parse) drain(S);
  for (int b = 0; b < 2; ++b) {
    free_outset(S->out[b]);
    cudaFree(S->buf[b]);
    cudaFree(S->scratch[b]);
    if (S->h2d_done[b]) cudaEventDestroy(S->h2d_done[b]);
    if (S->parse_done[b]) cudaEventDestroy(S->parse_done[b]);
    if (S->d2h_done[b]) cudaEventDestroy(S->d2h_done[b]);
    if (S->h2d_start[b]) cudaEventDestroy(S->h2d_start[b]);
    if (S->parse_start[b]) cudaEventDestroy(S->parse_start[b]);
    if (S->d2h_start[b]) cudaEventDestroy(S->d2h_start[b]);
  }
  if (S->carry_done) cudaEventDestroy(S->carry_done);
  if (S->s_h2d) cudaStreamDestroy(S->s_h2d);
  if (S->s_parse) cudaStreamDestroy(S->s_parse);
  if (S->s_d2h) cudaStreamDestroy(S->s_d2h);
  if (S->res_host) cudaFreeHost(S->res_host);
  cudaFree(S->res_dev);
  delete S;
}

extern "C" pp_status parparaw_stream_create(const pp_parser* parser, uint64_t partition_bytes, uint64_t carry_bytes,
                                            pp_streamer** out) {
  if (out == nullptr) return PP_E_ARG;
  *out = nullptr;
  if (parser == nullptr || partition_bytes == 0) return PP_E_ARG;
  if (parser->tab.unit2 && (partition_bytes % 2 != 0 || carry_bytes % 2 != 0)) return PP_E_ARG;  // whole code units
  pp_streamer* S = new (std::nothrow) pp_streamer();
  if (S == nullptr) return PP_E_NOMEM;
  S->parser = *parser;
  S->part = partition_bytes;
  S->carry = carry_bytes ? carry_bytes : partition_bytes;
  const uint64_t span = S->carry + S->part;
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = cudaMalloc(reinterpret_cast<void**>(&S->buf[b]), span);
    for (cudaEvent_t* ev : {&S->h2d_done[b], &S->parse_done[b], &S->d2h_done[b], &S->h2d_start[b],
                            &S->parse_start[b], &S->d2h_start[b]})
      if (e == cudaSuccess) e = cudaEventCreate(ev);  // timed: the partitions' device times
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->carry_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->s_h2d, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->s_parse, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->s_d2h, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&S->res_dev), 2 * sizeof(pp_parse_result));
  if (e == cudaSuccess)
    e = cudaHostAlloc(reinterpret_cast<void**>(&S->res_host), 2 * sizeof(pp_parse_result), cudaHostAllocDefault);
  pp_status st = map_cuda(e);
  if (st == PP_OK) {
    uint64_t caps[PP_MAX_COLUMNS];
    for (auto& c : caps) c = span;
    const uint64_t rows = std::max<uint64_t>(1024, span / 16);
    for (int b = 0; b < 2 && st == PP_OK; ++b) st = alloc_outset(S, b, rows, caps);
  }
  if (st != PP_OK) {
    parparaw_stream_destroy(S);
    return st;
  }
  *out = S;
  return PP_OK;
}

extern "C" pp_status parparaw_stream_parse(pp_streamer* S, const uint8_t* input, uint64_t len, uint8_t* arena,
                                           uint64_t arena_bytes, pp_host_partition* parts, uint64_t max_parts,
                                           pp_stream_result* result) {
  if (S == nullptr || result == nullptr || parts == nullptr || (input == nullptr && len > 0) ||
      (arena == nullptr && arena_bytes > 0))
    return PP_E_ARG;
  const uint64_t nparts = std::max<uint64_t>(1, (len + S->part - 1) / S->part);
  if (max_parts < nparts) return PP_E_ARG;
  std::memset(result, 0, sizeof(*result));
  result->first_invalid_offset = -1;
  const pp_parser& P = S->parser;

  cudaError_t e = cudaSuccess;
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {  // every wait below is satisfied until re-recorded
    e = cudaEventRecord(S->parse_done[b], S->s_parse);
    if (e == cudaSuccess) e = cudaEventRecord(S->d2h_done[b], S->s_parse);
    if (e == cudaSuccess) e = cudaEventRecord(S->h2d_done[b], S->s_parse);
  }
  // device times: a partition's copy in and parse are complete when its
  // result is settled; its copy out when the next partition of the same
  // set is settled (that parse waits for it), or after the final drain
  int64_t d2h_pending[2] = {-1, -1};  // the partition whose copy-out time set b still owes
  auto elapsed = [](cudaEvent_t a, cudaEvent_t z) {
    float ms = 0.f;
    return cudaEventElapsedTime(&ms, a, z) == cudaSuccess ? ms : -1.f;
  };
  auto take_d2h = [&](int b) {
    if (d2h_pending[b] >= 0 && cudaEventSynchronize(S->d2h_done[b]) == cudaSuccess)
      parts[d2h_pending[b]].d2h_ms = elapsed(S->d2h_start[b], S->d2h_done[b]);
    d2h_pending[b] = -1;
  };
  if (e == cudaSuccess) e = cudaEventRecord(S->carry_done, S->s_parse);
  if (e != cudaSuccess) return map_cuda(e);

  // partition k's fresh bytes go behind buffer k % 2's carry-over region,
  // once the carry-over out of that buffer (into the other one) is taken
  auto h2d = [&](uint64_t k) -> cudaError_t {
    const int b = static_cast<int>(k % 2);
    const uint64_t lo = k * S->part, ln = std::min(S->part, len - lo);
    cudaError_t r = cudaStreamWaitEvent(S->s_h2d, S->carry_done, 0);
    if (r == cudaSuccess) r = cudaEventRecord(S->h2d_start[b], S->s_h2d);
    if (r == cudaSuccess && ln > 0)
      r = cudaMemcpyAsync(S->buf[b] + S->carry, input + lo, ln, cudaMemcpyHostToDevice, S->s_h2d);
    if (r == cudaSuccess) r = cudaEventRecord(S->h2d_done[b], S->s_h2d);
    return r;
  };

  struct Pending {
    int b;
    uint64_t start, length, offset;  // in the buffer; in the input
    bool first, last;
  } prev{};
  bool have_prev = false;
  uint64_t used = 0;
  int64_t row0 = 0;
  pp_status st = PP_OK;

  // takes partition k-1's result, queues its copy-out; returns the carry-over
  // length, or sets st and stops
  auto retire = [&](const Pending& q, uint64_t* carry_len) -> bool {
    pp_parse_result r;
    st = settle(S, q.b, q.start, q.length, q.last, q.first, &r);
    if (st != PP_OK) return false;
    take_d2h(q.b);  // the set's previous partition, copied out before this parse
    if (r.status == PP_E_TIMEOUT || r.status == PP_E_INVALID_INPUT || r.status == PP_E_UNTERMINATED ||
        r.status == PP_OK) {
      const uint64_t need = partition_arena_bytes(P, r);
      if (used + need > arena_bytes) {
        result->status = PP_E_CAPACITY;
        result->arena_bytes = used + need;
        return false;
      }
      pp_host_partition& hp = parts[result->num_partitions];
      hp.row0 = row0;
      hp.input_offset = q.offset;
      hp.input_bytes = q.length;
      hp.h2d_ms = elapsed(S->h2d_start[q.b], S->h2d_done[q.b]);
      hp.parse_ms = elapsed(S->parse_start[q.b], S->parse_done[q.b]);
      hp.d2h_ms = 0.f;
      if ((st = enqueue_copy_out(S, q.b, r, arena, &used, &hp)) != PP_OK) return false;
      d2h_pending[q.b] = static_cast<int64_t>(result->num_partitions);
      result->num_partitions += 1;
      result->rows += r.rows;
      result->n_rejected += r.n_rejected;
      row0 += r.rows;
      result->arena_bytes = used;
    }
    if (r.status != PP_OK) {
      result->status = r.status;
      if (r.first_invalid_offset >= 0)
        result->first_invalid_offset = static_cast<int64_t>(q.offset) + r.first_invalid_offset;
      return false;
    }
    *carry_len = q.length - static_cast<uint64_t>(r.consumed);
    if (*carry_len > S->carry) {
      result->status = PP_E_UNSUPPORTED;  // a record longer than the carry-over region
      return false;
    }
    return true;
  };

  bool ok = (e = h2d(0)) == cudaSuccess;
  if (!ok) st = map_cuda(e);
  for (uint64_t k = 0; ok && k < nparts; ++k) {
    const int b = static_cast<int>(k % 2);
    const bool last = k + 1 == nparts;
    uint64_t carry_len = 0;
    if (have_prev) {
      if (!(ok = retire(prev, &carry_len))) break;
      // the incomplete record of partition k-1, in front of partition k
      e = cudaStreamWaitEvent(S->s_parse, S->h2d_done[b], 0);
      if (e == cudaSuccess && carry_len > 0)
        e = cudaMemcpyAsync(S->buf[b] + S->carry - carry_len, S->buf[prev.b] + prev.start + (prev.length - carry_len),
                            carry_len, cudaMemcpyDeviceToDevice, S->s_parse);
      if (e == cudaSuccess) e = cudaEventRecord(S->carry_done, S->s_parse);
    }
    const uint64_t fresh = std::min(S->part, len - std::min(len, k * S->part));
    Pending cur{b, S->carry - carry_len, carry_len + fresh, k * S->part - carry_len, k == 0, last};
    if (e == cudaSuccess) e = cudaStreamWaitEvent(S->s_parse, S->h2d_done[b], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(S->s_parse, S->d2h_done[b], 0);  // the set's last copy-out
    if (e != cudaSuccess) {
      st = map_cuda(e);
      break;
    }
    if ((st = enqueue_parse(S, b, cur.start, cur.length, last, k == 0)) != PP_OK) break;
    if (!last) e = h2d(k + 1);
    if (e != cudaSuccess) {
      st = map_cuda(e);
      break;
    }
    prev = cur;
    have_prev = true;
  }
  if (ok && st == PP_OK && have_prev) {
    uint64_t unused = 0;
    retire(prev, &unused);
  }
  drain(S);
  take_d2h(0);
  take_d2h(1);
  return st;
}
