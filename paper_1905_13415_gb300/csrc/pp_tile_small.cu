// Tile shape "small": 64 threads x 48 bytes per thread, >= 1 blocks per SM.
#include "pp_tile_inst.cuh"
PP_DEFINE_SHAPE_WITH_UNITS(small, 64, 3, 1)
