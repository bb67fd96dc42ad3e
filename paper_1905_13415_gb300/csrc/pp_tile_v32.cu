// pp_tile_v32.cu -- tile shape 256 threads x 32 B.
#include "pp_tile_inst.cuh"
PP_DEFINE_SHAPE(v32, 256, 2, 4)
