// Instantiates the batch iterate kernel for float arithmetic and the VEGAS_GENZ_DISC
// integrand (and its big-block adapting variant).
#include "batch_kernel.cuh"

VEGAS_BATCH_TABLE(batch_table_f32_genz_disc, float, VEGAS_GENZ_DISC)
VEGAS_BATCH_TABLE_BIG(batch_table_big_f32_genz_disc, VEGAS_GENZ_DISC)
