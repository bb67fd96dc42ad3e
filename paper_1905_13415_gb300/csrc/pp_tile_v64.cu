// pp_tile_v64.cu -- tile shape 256 threads x 64 B.
#include "pp_tile_inst.cuh"
PP_DEFINE_SHAPE(v64, 256, 4, 3)
