// Instantiates the batch iterate kernel for float arithmetic and the VEGAS_GAUSS_MIX2
// integrand (and its big-block adapting variant).
#include "batch_kernel.cuh"

VEGAS_BATCH_TABLE(batch_table_f32_mix2, float, VEGAS_GAUSS_MIX2)
VEGAS_BATCH_TABLE_BIG(batch_table_big_f32_mix2, VEGAS_GAUSS_MIX2)
