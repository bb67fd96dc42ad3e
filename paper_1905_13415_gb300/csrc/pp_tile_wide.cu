// Tile shape "wide": 128 threads x 208 bytes per thread, >= 1 blocks per SM.
#include "pp_tile_inst.cuh"
PP_DEFINE_SHAPE(wide, 128, 13, 1)
