// Instantiates the batch iterate kernel for double arithmetic and the VEGAS_GENZ_DISC
// integrand.
#include "batch_kernel.cuh"

VEGAS_BATCH_TABLE(batch_table_f64_genz_disc, double, VEGAS_GENZ_DISC)
