// pp_tile_t448.cu -- tile shape 448 threads x 64 B, 2 blocks per SM (the default,
// with the inference form).
#include "pp_tile_inst.cuh"
PP_DEFINE_SHAPE_WITH_INFER(t448, 448, 4, 2)
