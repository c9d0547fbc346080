// flb_batch_k2.cu -- instantiations of the batched step kernel for the
// look-up-table f-norm (one translation unit per basis, compiled in parallel).
#include "flb_batch_kernel.cuh"

namespace flb {

const void* batch_kernel_lut(int variant, bool sample) {
    switch (variant) {
        case 0:
            return sample ? (const void*)batch_step_kernel<2, true, 128, 2>
                          : (const void*)batch_step_kernel<2, false, 128, 2>;
        case 1:
            return sample ? (const void*)batch_step_kernel<2, true, 64, 2>
                          : (const void*)batch_step_kernel<2, false, 64, 2>;
        case 2:
            return sample ? (const void*)batch_step_kernel<2, true, 128, 1>
                          : (const void*)batch_step_kernel<2, false, 128, 1>;
        case 3:
            return sample ? (const void*)batch_step_kernel<2, true, 128, 2, kBatchNWTensor>
                          : (const void*)batch_step_kernel<2, false, 128, 2, kBatchNWTensor>;
        case 4:
            return sample ? (const void*)batch_step_kernel<2, true, 64, 2, kBatchNWTensor>
                          : (const void*)batch_step_kernel<2, false, 64, 2, kBatchNWTensor>;
        case 5:
            return sample ? (const void*)batch_step_kernel<2, true, kMixedTW, 2, kBatchNWTensor>
                          : (const void*)batch_step_kernel<2, false, kMixedTW, 2, kBatchNWTensor>;
        default:
            return nullptr;
    }
}

}  // namespace flb
