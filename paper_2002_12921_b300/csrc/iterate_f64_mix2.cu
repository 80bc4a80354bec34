// Instantiates the fused iterate kernel for double arithmetic and the VEGAS_GAUSS_MIX2
// integrand, dimensions 1..20, with and without the refinement histogram.
#include "iterate_kernel.cuh"

VEGAS_KERNEL_TABLE(iterate_table_f64_mix2, double, VEGAS_GAUSS_MIX2)
