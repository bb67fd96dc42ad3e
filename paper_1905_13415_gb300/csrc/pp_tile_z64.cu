// pp_tile_z64.cu -- tile shape 256 threads x 64 B, 4 blocks per SM.
#include "pp_tile_inst.cuh"
PP_DEFINE_SHAPE(z64, 256, 4, 4)
