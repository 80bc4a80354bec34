// The batch iterate kernels for double arithmetic, by integrand (one
// instantiation file per integrand: batch_f64_*.cu).
#include "batch_kernel.cuh"

namespace vegas {
const void* batch_table_f64_gauss(bool adapt, int block);
const void* batch_table_f64_mix2(bool adapt, int block);
const void* batch_table_f64_flat(bool adapt, int block);
const void* batch_table_f64_genz_disc(bool adapt, int block);
const void* batch_table_f64_genz_ppeak(bool adapt, int block);

const void* batch_iterate_kernel_f64(int integrand, bool adapt, int block) {
    switch (integrand) {
    case VEGAS_GAUSS: return batch_table_f64_gauss(adapt, block);
    case VEGAS_GAUSS_MIX2: return batch_table_f64_mix2(adapt, block);
    case VEGAS_FLAT: return batch_table_f64_flat(adapt, block);
    case VEGAS_GENZ_DISC: return batch_table_f64_genz_disc(adapt, block);
    case VEGAS_GENZ_PPEAK: return batch_table_f64_genz_ppeak(adapt, block);
    default: return nullptr;
    }
}
}  // namespace vegas
