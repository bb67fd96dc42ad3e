// pp_tile_inst.cuh -- defines the launch entry of one tile shape for every
// supported symbol count (4, 8, 16 SWAR comparisons per word); the default
// shape also defines the inference form of the kernel, and it and the two
// small shapes the form that reads UTF-16LE code units.
#pragma once
#include <cuda_runtime.h>

#include "pp_kernel.cuh"
#include "pp_launch.h"

#define PP_SHAPE_COMMON(NAME, NT_, VPT_, MINB_)                                                      \
  using Shape_##NAME = TileShape<NT_, VPT_, MINB_>;                                                 \
  static const void* kernel_ptr_##NAME(int nspec) {                                                \
    if (nspec <= 4) return reinterpret_cast<const void*>(&pp_tile_kernel<Shape_##NAME, 4>);        \
    if (nspec <= 8) return reinterpret_cast<const void*>(&pp_tile_kernel<Shape_##NAME, 8>);        \
    return reinterpret_cast<const void*>(&pp_tile_kernel<Shape_##NAME, 16>);                       \
  }

#define PP_SHAPE_INFO(NAME, NT_, INFER_FN, UNITS_FN)                                                 \
  ShapeInfo shape_info_##NAME() {                                                                  \
    ShapeInfo s;                                                                                   \
    s.threads = NT_;                                                                               \
    s.tile_bytes = Shape_##NAME::T;                                                                \
    s.smem_bytes = SmemLayout<Shape_##NAME>::kBytes;                                               \
    s.kernel = &kernel_ptr_##NAME;                                                                 \
    s.infer_kernel = INFER_FN;                                                                     \
    s.units_kernel = UNITS_FN;                                                                     \
    return s;                                                                                      \
  }

// the form that also reads UTF-16LE code units
#define PP_SHAPE_UNITS(NAME)                                                                               \
  static const void* units_ptr_##NAME(int nspec) {                                                       \
    if (nspec <= 4) return reinterpret_cast<const void*>(&pp_tile_kernel<Shape_##NAME, 4, false, true>); \
    if (nspec <= 8) return reinterpret_cast<const void*>(&pp_tile_kernel<Shape_##NAME, 8, false, true>); \
    return reinterpret_cast<const void*>(&pp_tile_kernel<Shape_##NAME, 16, false, true>);                \
  }

#define PP_DEFINE_SHAPE(NAME, NT_, VPT_, MINB_) \
  namespace pp {                                \
  PP_SHAPE_COMMON(NAME, NT_, VPT_, MINB_)       \
  PP_SHAPE_INFO(NAME, NT_, nullptr, nullptr)    \
  }

#define PP_DEFINE_SHAPE_WITH_UNITS(NAME, NT_, VPT_, MINB_) \
  namespace pp {                                           \
  PP_SHAPE_COMMON(NAME, NT_, VPT_, MINB_)                  \
  PP_SHAPE_UNITS(NAME)                                     \
  PP_SHAPE_INFO(NAME, NT_, nullptr, &units_ptr_##NAME)     \
  }

#define PP_DEFINE_SHAPE_WITH_INFER(NAME, NT_, VPT_, MINB_)                                           \
  namespace pp {                                                                                   \
  PP_SHAPE_COMMON(NAME, NT_, VPT_, MINB_)                                                          \
  PP_SHAPE_UNITS(NAME)                                                                             \
  static const void* infer_ptr_##NAME(int nspec) {                                                 \
    if (nspec <= 4) return reinterpret_cast<const void*>(&pp_tile_kernel<Shape_##NAME, 4, true>);  \
    if (nspec <= 8) return reinterpret_cast<const void*>(&pp_tile_kernel<Shape_##NAME, 8, true>);  \
    return reinterpret_cast<const void*>(&pp_tile_kernel<Shape_##NAME, 16, true>);                 \
  }                                                                                                \
  PP_SHAPE_INFO(NAME, NT_, &infer_ptr_##NAME, &units_ptr_##NAME)                                   \
  }
