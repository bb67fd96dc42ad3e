// pp_tile_v48.cu -- tile shape 256 threads x 48 B.
#include "pp_tile_inst.cuh"
PP_DEFINE_SHAPE(v48, 256, 3, 3)
