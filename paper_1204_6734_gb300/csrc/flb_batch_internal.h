// flb_batch_internal.h -- what the request server (flb_server.cu) uses of a
// batch beyond the C ABI: asynchronous read-out of one replica's sums and
// error record, and the pool's occupancy.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/flb.h"
#include "flb_kernels.cuh"

namespace flb {

// Enqueue on the batch's stream the copy of replica `slot`'s kSums running
// sums and its error record into host memory (page-locked for an asynchronous
// copy). The values are those after every step enqueued so far.
int batch_enqueue_readout(flb_batch b, int slot, double* acc_out, DevError* err_out);

// Number of sampled node-steps of replica `slot` so far (host bookkeeping).
int64_t batch_samples(flb_batch b, int slot);

// Replica time after every step enqueued so far.
int64_t batch_replica_time(flb_batch b, int slot);

cudaStream_t batch_stream(flb_batch b);

}  // namespace flb
