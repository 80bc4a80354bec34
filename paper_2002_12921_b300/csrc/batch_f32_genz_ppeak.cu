// Instantiates the batch iterate kernel for float arithmetic and the VEGAS_GENZ_PPEAK
// integrand.
#include "batch_kernel.cuh"

VEGAS_BATCH_TABLE(batch_table_f32_genz_ppeak, float, VEGAS_GENZ_PPEAK)
