// pp_tile_w48.cu -- tile shape 512 threads x 48 B.
#include "pp_tile_inst.cuh"
PP_DEFINE_SHAPE(w48, 512, 3, 2)
