// pp_tile_big3.cu -- tile shape 256 threads x 112 B, 3 blocks per SM.
#include "pp_tile_inst.cuh"
PP_DEFINE_SHAPE(big3, 256, 7, 3)
