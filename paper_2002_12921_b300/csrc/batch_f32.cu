// The batch iterate kernels for float arithmetic, by integrand (one
// instantiation file per integrand: batch_f32_*.cu).
#include "batch_kernel.cuh"

namespace vegas {
const void* batch_table_f32_gauss(bool adapt, int block);
const void* batch_table_f32_mix2(bool adapt, int block);
const void* batch_table_f32_flat(bool adapt, int block);
const void* batch_table_f32_genz_disc(bool adapt, int block);
const void* batch_table_f32_genz_ppeak(bool adapt, int block);

const void* batch_iterate_kernel_f32(int integrand, bool adapt, int block) {
    switch (integrand) {
    case VEGAS_GAUSS: return batch_table_f32_gauss(adapt, block);
    case VEGAS_GAUSS_MIX2: return batch_table_f32_mix2(adapt, block);
    case VEGAS_FLAT: return batch_table_f32_flat(adapt, block);
    case VEGAS_GENZ_DISC: return batch_table_f32_genz_disc(adapt, block);
    case VEGAS_GENZ_PPEAK: return batch_table_f32_genz_ppeak(adapt, block);
    default: return nullptr;
    }
}
const void* batch_table_big_f32_gauss();
const void* batch_table_big_f32_mix2();
const void* batch_table_big_f32_flat();
const void* batch_table_big_f32_genz_disc();
const void* batch_table_big_f32_genz_ppeak();

const void* batch_iterate_kernel_f32_big(int integrand) {
    switch (integrand) {
    case VEGAS_GAUSS: return batch_table_big_f32_gauss();
    case VEGAS_GAUSS_MIX2: return batch_table_big_f32_mix2();
    case VEGAS_FLAT: return batch_table_big_f32_flat();
    case VEGAS_GENZ_DISC: return batch_table_big_f32_genz_disc();
    case VEGAS_GENZ_PPEAK: return batch_table_big_f32_genz_ppeak();
    default: return nullptr;
    }
}
}  // namespace vegas
