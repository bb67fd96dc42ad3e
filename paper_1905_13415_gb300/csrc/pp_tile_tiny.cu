// Tile shape "tiny": 32 threads x 16 bytes per thread, >= 1 blocks per SM.
#include "pp_tile_inst.cuh"
PP_DEFINE_SHAPE_WITH_UNITS(tiny, 32, 1, 1)
