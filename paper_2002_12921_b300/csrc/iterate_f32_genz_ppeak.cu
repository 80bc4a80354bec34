// Instantiates the fused iterate kernel for float arithmetic and the VEGAS_GENZ_PPEAK
// integrand, dimensions 1..20, with and without the refinement histogram.
#include "iterate_kernel.cuh"

VEGAS_KERNEL_TABLE(iterate_table_f32_genz_ppeak, float, VEGAS_GENZ_PPEAK)
