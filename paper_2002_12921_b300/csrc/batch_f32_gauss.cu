// Instantiates the batch iterate kernel for float arithmetic and the VEGAS_GAUSS
// integrand (and its big-block adapting variant).
#include "batch_kernel.cuh"

VEGAS_BATCH_TABLE(batch_table_f32_gauss, float, VEGAS_GAUSS)
VEGAS_BATCH_TABLE_BIG(batch_table_big_f32_gauss, VEGAS_GAUSS)
