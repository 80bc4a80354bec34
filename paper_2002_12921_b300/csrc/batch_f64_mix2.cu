// Instantiates the batch iterate kernel for double arithmetic and the VEGAS_GAUSS_MIX2
// integrand.
#include "batch_kernel.cuh"

VEGAS_BATCH_TABLE(batch_table_f64_mix2, double, VEGAS_GAUSS_MIX2)
