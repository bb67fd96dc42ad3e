// pp_tile_t448.cu -- tile shape 448 threads x 64 B, 2 blocks per SM (the default).
#include "pp_tile_inst.cuh"
PP_DEFINE_SHAPE(t448, 448, 4, 2)
