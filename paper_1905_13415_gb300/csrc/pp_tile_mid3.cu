// Tile shape "mid3": 256 threads x 80 bytes per thread, >= 3 blocks per SM.
#include "pp_tile_inst.cuh"
PP_DEFINE_SHAPE(mid3, 256, 5, 3)
