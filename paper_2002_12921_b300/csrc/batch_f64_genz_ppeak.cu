// Instantiates the batch iterate kernel for double arithmetic and the VEGAS_GENZ_PPEAK
// integrand.
#include "batch_kernel.cuh"

VEGAS_BATCH_TABLE(batch_table_f64_genz_ppeak, double, VEGAS_GENZ_PPEAK)
