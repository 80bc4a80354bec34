// Instantiates the big-block adapting iterate kernel (float arithmetic, one
// block of up to kBigBlockThreads per SM) and the default-shape one with the
// run-time histogram copy count for the VEGAS_FLAT integrand, dimensions
// 1..20.
#include "iterate_kernel.cuh"

VEGAS_KERNEL_TABLE_BIG(iterate_table_big_f32_flat, VEGAS_FLAT)
VEGAS_KERNEL_TABLE_FEW(iterate_table_few_f32_flat, VEGAS_FLAT)
