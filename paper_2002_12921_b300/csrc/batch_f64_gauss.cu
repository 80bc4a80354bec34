// Instantiates the batch iterate kernel for double arithmetic and the VEGAS_GAUSS
// integrand.
#include "batch_kernel.cuh"

VEGAS_BATCH_TABLE(batch_table_f64_gauss, double, VEGAS_GAUSS)
