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
