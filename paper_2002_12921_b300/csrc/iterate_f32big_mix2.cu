// Instantiates the big-block adapting iterate kernel (float arithmetic, one
// block of up to kBigBlockThreads per SM) and the default-shape one with the
// run-time histogram copy count for the VEGAS_GAUSS_MIX2 integrand, dimensions
// 1..20.
#include "iterate_kernel.cuh"

VEGAS_KERNEL_TABLE_BIG(iterate_table_big_f32_mix2, VEGAS_GAUSS_MIX2)
VEGAS_KERNEL_TABLE_FEW(iterate_table_few_f32_mix2, VEGAS_GAUSS_MIX2)
