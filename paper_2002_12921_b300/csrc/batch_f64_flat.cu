// Instantiates the batch iterate kernel for double arithmetic and the VEGAS_FLAT
// integrand.
#include "batch_kernel.cuh"

VEGAS_BATCH_TABLE(batch_table_f64_flat, double, VEGAS_FLAT)
