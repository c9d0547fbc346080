// flb_runtime.h -- what the request server (flb_server.cu) and the batch code
// use of batches and lattice handles beyond the C ABI: creation without a host
// synchronisation, asynchronous read-out of a replica's sums and error record,
// bookkeeping, the finalisation of correlation sums.
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

// flb_create without the final stream synchronisation (errors of the
// initialisation kernels then surface at the next synchronising call).
int lattice_create(const flb_params* p, void* dev_workspace, size_t workspace_bytes,
                   cudaStream_t stream, bool sync, flb_lattice* out);

// As batch_enqueue_readout, for a lattice handle.
int lattice_enqueue_readout(flb_lattice h, double* acc_out, DevError* err_out);
int64_t lattice_samples(flb_lattice h);
int64_t lattice_time(flb_lattice h);

// Device addresses of the look-up-table f-norm's velocity tables (FP32 and
// FP64) on the current device, built on first use (synchronously, on a stream
// of its own). Either pointer may be NULL.
int lut_tables(const float** t32, const double** t64);

// Free the host side of a handle whose workspace the caller owns, without
// waiting for its stream: the caller orders any reuse of the workspace after
// the handle's last enqueued work.
void lattice_forget(flb_lattice h);

// <df df>, <dM dM> and the mean deviation from kSums running sums over nsamp
// node-samples taken relative to f^0(rho0, u0) (as flb_correlations, with the
// measurement basis at (ux0, uy0)); on a scratch buffer of its own, ordered on
// stream st, synchronous. Any output pointer may be NULL.
int finalize_sums(const double* acc, int64_t nsamp, int32_t measure_basis, double ux0, double uy0,
                  cudaStream_t st, double* Cff, double* CMM, double* mean_dev);

}  // namespace flb
