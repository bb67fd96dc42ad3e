// Tile shape "m128x6": 128 threads x 112 bytes per thread, >= 6 blocks per SM.
#include "pp_tile_inst.cuh"
PP_DEFINE_SHAPE(m128x6, 128, 7, 6)
