// pp_launch.h -- host-side view of the compiled tile shapes.
#pragma once
#include <cstddef>
#include <cstdint>

namespace pp {

struct ShapeInfo {
  int threads = 0;
  int tile_bytes = 0;
  size_t smem_bytes = 0;
  const void* (*kernel)(int nspec) = nullptr;  // pp_tile_kernel<Shape, NSPEC>
  const void* (*infer_kernel)(int nspec) = nullptr;  // its inference form (default shape only)
  const void* (*units_kernel)(int nspec) = nullptr;  // its form for UTF-16LE code units (some shapes)
};

// tile configurations selectable with PP_OPT_TILE_CONFIG
ShapeInfo shape_info_tiny();    // 32 threads x 16 B   =   512 B tiles
ShapeInfo shape_info_small();   // 64 threads x 48 B   =  3 KiB tiles
ShapeInfo shape_info_mid();     // 256 threads x 112 B = 28 KiB tiles
ShapeInfo shape_info_wide();    // 128 threads x 208 B = 26 KiB tiles
ShapeInfo shape_info_m128();    // 128 threads x 112 B = 14 KiB tiles, 4 blocks / SM
ShapeInfo shape_info_m128x6();  // 128 threads x 112 B = 14 KiB tiles, 6 blocks / SM
ShapeInfo shape_info_s128();    // 128 threads x 48 B  =  6 KiB tiles, 8 blocks / SM
ShapeInfo shape_info_mid3();    // 256 threads x 80 B  = 20 KiB tiles, 3 blocks / SM
ShapeInfo shape_info_y96();     // 256 threads x 96 B  = 24 KiB tiles, 3 blocks / SM
ShapeInfo shape_info_t448();    // 448 threads x 64 B  = 28 KiB tiles, 2 blocks / SM
ShapeInfo shape_info_w48();     // 512 threads x 48 B  = 24 KiB tiles, 2 blocks / SM
ShapeInfo shape_info_big3();    // 256 threads x 112 B = 28 KiB tiles, 3 blocks / SM
ShapeInfo shape_info_q384();    // 384 threads x 128 B = 48 KiB tiles, 2 blocks / SM
ShapeInfo shape_info_q448();    // 448 threads x 128 B = 56 KiB tiles, 2 blocks / SM

}  // namespace pp
