// Tile shape "s128": 128 threads x 48 bytes per thread, >= 8 blocks per SM.
#include "pp_tile_inst.cuh"
PP_DEFINE_SHAPE(s128, 128, 3, 8)
