// pp_tile_y96.cu -- tile shape 256 threads x 96 B, 3 blocks per SM.
#include "pp_tile_inst.cuh"
PP_DEFINE_SHAPE(y96, 256, 6, 3)
