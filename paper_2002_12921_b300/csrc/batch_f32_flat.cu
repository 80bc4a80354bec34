// Instantiates the batch iterate kernel for float arithmetic and the VEGAS_FLAT
// integrand.
#include "batch_kernel.cuh"

VEGAS_BATCH_TABLE(batch_table_f32_flat, float, VEGAS_FLAT)
