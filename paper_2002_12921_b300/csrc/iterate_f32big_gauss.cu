// Instantiates, for the VEGAS_GAUSS integrand in float arithmetic: the big-block
// adapting iterate kernel (one block of up to kBigBlockThreads per SM) and the
// default-shape adapting one with the run-time histogram copy count, for
// dimensions 1..20; and the fixed-grid kernels compiled for kFixedBins bins,
// for dimensions 1..kFixedBinsMaxDim.
#include "iterate_kernel.cuh"

VEGAS_KERNEL_TABLE_BIG(iterate_table_big_f32_gauss, VEGAS_GAUSS)
VEGAS_KERNEL_TABLE_FEW(iterate_table_few_f32_gauss, VEGAS_GAUSS)
VEGAS_KERNEL_TABLE_NB(iterate_table_nb_f32_gauss, VEGAS_GAUSS)
