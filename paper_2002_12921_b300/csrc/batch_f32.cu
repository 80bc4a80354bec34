// Instantiates the batch iterate kernel for float arithmetic.
#include "batch_kernel.cuh"

namespace vegas {
const void* batch_iterate_kernel_f32(bool adapt) {
    return adapt ? (const void*)&batch_iterate_kernel<float, true>
                 : (const void*)&batch_iterate_kernel<float, false>;
}
}  // namespace vegas
