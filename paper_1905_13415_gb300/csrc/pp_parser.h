// pp_parser.h -- the host-side parser object behind the opaque pp_parser
// handle of include/parparaw.h (host code only).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "pp_types.h"

struct pp_parser {
  pp::Tables tab;
  uint32_t types[PP_MAX_COLUMNS];
  int tile_config = 0;
  uint64_t timeout_ns = 2000000000ull;
  int64_t grid_limit = 0;
  uint32_t first_item = 0;
  cudaEvent_t ev_start = nullptr, ev_stop = nullptr;
};

// Internal (not in include/parparaw.h): a parse whose scratch comes from the
// caller's device block of scratch_cap bytes (PP_E_UNSUPPORTED when too
// small), or is allocated stream-ordered when scratch_block is null; and the
// scratch bytes a parse of len bytes into rows_cap rows needs.
pp_status pp_parse_with_scratch(const pp_parser* P, const uint8_t* input, uint64_t len, const pp_columns* out,
                                cudaStream_t stream, uint8_t* scratch_block, size_t scratch_cap);
size_t pp_parse_scratch_bytes(const pp_parser* P, uint64_t len, uint64_t rows_cap);
