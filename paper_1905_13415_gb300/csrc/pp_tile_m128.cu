// Tile shape "m128": 128 threads x 112 bytes per thread, >= 4 blocks per SM.
#include "pp_tile_inst.cuh"
PP_DEFINE_SHAPE(m128, 128, 7, 4)
