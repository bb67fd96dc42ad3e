// pp_tile_inst.cuh -- defines the launch entry of one tile shape for every
// supported symbol count (4, 8, 16 SWAR comparisons per word).
#pragma once
#include <cuda_runtime.h>

#include "pp_kernel.cuh"
#include "pp_launch.h"

#define PP_DEFINE_SHAPE(NAME, NT_, VPT_, MINB_)                                                         \
  namespace pp {                                                                                 \
  using Shape_##NAME = TileShape<NT_, VPT_, MINB_>;                                                     \
  static const void* kernel_ptr_##NAME(int nspec) {                                              \
    if (nspec <= 4) return reinterpret_cast<const void*>(&pp_tile_kernel<Shape_##NAME, 4>);      \
    if (nspec <= 8) return reinterpret_cast<const void*>(&pp_tile_kernel<Shape_##NAME, 8>);      \
    return reinterpret_cast<const void*>(&pp_tile_kernel<Shape_##NAME, 16>);                     \
  }                                                                                              \
  ShapeInfo shape_info_##NAME() {                                                                \
    ShapeInfo s;                                                                                 \
    s.threads = NT_;                                                                             \
    s.tile_bytes = Shape_##NAME::T;                                                              \
    s.smem_bytes = SmemLayout<Shape_##NAME>::kBytes;                                             \
    s.kernel = &kernel_ptr_##NAME;                                                               \
    return s;                                                                                    \
  }                                                                                              \
  }
