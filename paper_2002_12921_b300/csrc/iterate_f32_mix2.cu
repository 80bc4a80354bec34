// Instantiates the fused iterate kernel for float arithmetic and the VEGAS_GAUSS_MIX2
// integrand, dimensions 1..20, with and without the refinement histogram.
#include "iterate_kernel.cuh"

VEGAS_KERNEL_TABLE(iterate_table_f32_mix2, float, VEGAS_GAUSS_MIX2)
