// Instantiates the batch iterate kernel for float arithmetic and the VEGAS_GENZ_DISC
// integrand.
#include "batch_kernel.cuh"

VEGAS_BATCH_TABLE(batch_table_f32_genz_disc, float, VEGAS_GENZ_DISC)
