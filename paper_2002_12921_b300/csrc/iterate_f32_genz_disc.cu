// Instantiates the fused iterate kernel for float arithmetic and the VEGAS_GENZ_DISC
// integrand, dimensions 1..20, with and without the refinement histogram.
#include "iterate_kernel.cuh"

VEGAS_KERNEL_TABLE(iterate_table_f32_genz_disc, float, VEGAS_GENZ_DISC)
