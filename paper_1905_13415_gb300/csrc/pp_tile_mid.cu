// Tile shape "mid": 256 threads x 112 bytes per thread, >= 1 blocks per SM.
#include "pp_tile_inst.cuh"
PP_DEFINE_SHAPE(mid, 256, 7, 2)
