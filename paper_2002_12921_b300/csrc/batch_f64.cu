// Instantiates the batch iterate kernel for double arithmetic.
#include "batch_kernel.cuh"

namespace vegas {
const void* batch_iterate_kernel_f64(bool adapt) {
    return adapt ? (const void*)&batch_iterate_kernel<double, true>
                 : (const void*)&batch_iterate_kernel<double, false>;
}
}  // namespace vegas
