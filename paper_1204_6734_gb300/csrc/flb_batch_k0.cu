// flb_batch_k0.cu -- instantiations of the batched step kernel for the
// Hermite-norm (standard) basis (one translation unit per basis, compiled in parallel).
#include "flb_batch_kernel.cuh"

namespace flb {

const void* batch_kernel_std(int variant, bool sample) {
    switch (variant) {
        case 0:
            return sample ? (const void*)batch_step_kernel<0, true, 128, 2>
                          : (const void*)batch_step_kernel<0, false, 128, 2>;
        case 1:
            return sample ? (const void*)batch_step_kernel<0, true, 64, 2>
                          : (const void*)batch_step_kernel<0, false, 64, 2>;
        case 2:
            return sample ? (const void*)batch_step_kernel<0, true, 128, 1>
                          : (const void*)batch_step_kernel<0, false, 128, 1>;
        case 3:
            return sample ? (const void*)batch_step_kernel<0, true, 128, 2, kBatchNWTensor>
                          : (const void*)batch_step_kernel<0, false, 128, 2, kBatchNWTensor>;
        case 4:
            return sample ? (const void*)batch_step_kernel<0, true, 64, 2, kBatchNWTensor>
                          : (const void*)batch_step_kernel<0, false, 64, 2, kBatchNWTensor>;
        case 5:
            return sample ? (const void*)batch_step_kernel<0, true, kMixedTW, 2, kBatchNWTensor>
                          : (const void*)batch_step_kernel<0, false, kMixedTW, 2, kBatchNWTensor>;
        default:
            return nullptr;
    }
}

}  // namespace flb

namespace flb {

// Every tile shape fits the 227 KB of shared memory a CTA may take.
static_assert(BatchShape<128, 2>::smem_bytes() <= 227 * 1024 && BatchShape<64, 2>::smem_bytes() <= 227 * 1024 &&
                  BatchShape<128, 1>::smem_bytes() <= 227 * 1024 &&
                  BatchShape<128, 2, kBatchNWTensor>::smem_bytes() <= 227 * 1024 &&
                  BatchShape<64, 2, kBatchNWTensor>::smem_bytes() <= 227 * 1024 &&
                  BatchShape<kMixedTW, 2, kBatchNWTensor>::smem_bytes() <= 227 * 1024,
              "batch shapes");

size_t batch_smem_bytes(int variant) {
    switch (variant) {
        case 0: return BatchShape<128, 2>::smem_bytes();
        case 1: return BatchShape<64, 2>::smem_bytes();
        case 2: return BatchShape<128, 1>::smem_bytes();
        case 3: return BatchShape<128, 2, kBatchNWTensor>::smem_bytes();
        case 4: return BatchShape<64, 2, kBatchNWTensor>::smem_bytes();
        case 5: return BatchShape<kMixedTW, 2, kBatchNWTensor>::smem_bytes();
        default: return 0;
    }
}

}  // namespace flb
