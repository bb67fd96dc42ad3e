// Tile shape "q448": 448 threads x 128 bytes per thread = 56 KiB tiles, 2 blocks per SM.
#include "pp_tile_inst.cuh"
PP_DEFINE_SHAPE(q448, 448, 8, 2)
