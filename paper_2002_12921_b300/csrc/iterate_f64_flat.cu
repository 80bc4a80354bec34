// Instantiates the fused iterate kernel for double arithmetic and the VEGAS_FLAT
// integrand, dimensions 1..20, with and without the refinement histogram.
#include "iterate_kernel.cuh"

VEGAS_KERNEL_TABLE(iterate_table_f64_flat, double, VEGAS_FLAT)
