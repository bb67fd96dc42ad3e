// Tile shape "q384": 384 threads x 128 bytes per thread = 48 KiB tiles, 2 blocks per SM.
#include "pp_tile_inst.cuh"
PP_DEFINE_SHAPE(q384, 384, 8, 2)
