// flb_batch.cu -- host side of batches: many independent FP32 lattices
// ("replicas") stepped together by one persistent launch of the batched
// pipelined kernel (flb_batch_kernel.cuh) per step.
//
// Device memory of a batch:
//  * the pool: one allocation made at open time; every replica's two
//    population buffers are carved out of it by a first-fit arena
//    (flb_arena.h), so adding and removing replicas never allocates;
//  * the metadata: replica descriptors (tensor maps + hot block), the tile
//    table, the control block {step, ticket, ntiles}, per-replica running sums
//    and error records.
// Membership changes (add, remove, tile shape) rewrite descriptors and the
// tile table with stream-ordered copies, so they take effect at the next
// launch, and a captured CUDA graph of k launches stays valid across them.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/flb.h"
#include "flb_arena.h"
#include "flb_batch_kernel.cuh"
#include "flb_host.h"
#include "flb_internal.h"
#include "flb_io.cuh"
#include "flb_runtime.h"

using namespace flb;

namespace {

struct BatchSlot {
    bool used = false;
    flb_params p;
    Geometry geo;
    size_t off = 0, bytes = 0;     // pool range: buffer 0, then buffer 1
    int64_t join = 0, tend = 0;    // batch step at which it joined; time limit
    int64_t warmup = 0, every = 0, nsamp = 0;
    float* buf[2] = {nullptr, nullptr};
};

}  // namespace

struct flb_batch_s {
    int basis = 0, cap = 0;
    const float* lut = nullptr;   // velocity table (look-up-table f-norm)
    cudaStream_t stream = nullptr;
    char* pool = nullptr;
    Arena arena;
    char* meta = nullptr;
    ReplicaDesc* desc = nullptr;   // [cap]
    uint32_t* tiles = nullptr;     // [max_tiles]
    size_t max_tiles = 0;
    BatchCtl* ctl = nullptr;
    double* acc = nullptr;         // [cap][kSums]
    DevError* err = nullptr;       // [cap]
    std::vector<BatchSlot> slots;
    std::vector<ReplicaDesc> hdesc;
    std::vector<uint32_t> htiles;
    int tile = 0;                  // FLB_TILE_*
    int grid = 1, sms = 1;
    int64_t step = 0;              // launches enqueued
    bool table_dirty = true;
    int graph_steps = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};   // [sample]
};

namespace {

constexpr int kMaxSide = 8192;

size_t buffer_bytes(const Geometry& g) { return Arena::round_up((size_t)9 * g.plane * sizeof(float)); }

int tile_rows(int tile) { return kBatchVariants[tile].th(); }
int tile_cols(int tile) { return kBatchVariants[tile].mixed() ? kind_tw(0) : kBatchVariants[tile].tw; }

// Column bands of the mixed tiling: nc[k] columns of kind k, the 128-wide
// ones first; the rest w of the width takes one column of the narrowest kind
// that covers it, or a 64-wide and a 32-wide column when 64 < w <= 96.
struct Bands {
    int nc[kKinds];
    int64_t tiles[kKinds];
};

Bands mixed_bands(int Lx, int Ly) {
    Bands b{};
    b.nc[0] = Lx / kind_tw(0);
    const int w = Lx - b.nc[0] * kind_tw(0);
    if (w > kind_tw(0) - kind_tw(2)) {
        ++b.nc[0];
    } else if (w > kind_tw(1)) {
        b.nc[1] = b.nc[2] = 1;
    } else if (w > kind_tw(2)) {
        b.nc[1] = 1;
    } else if (w > 0) {
        b.nc[2] = 1;
    }
    for (int k = 0; k < kKinds; ++k) b.tiles[k] = (int64_t)b.nc[k] * ((Ly + kind_th(k) - 1) / kind_th(k));
    return b;
}

int64_t replica_tiles(const flb_params& p, int tile) {
    if (kBatchVariants[tile].mixed()) {
        const Bands b = mixed_bands(p.Lx, p.Ly);
        return b.tiles[0] + b.tiles[1] + b.tiles[2];
    }
    return (int64_t)((p.Lx + tile_cols(tile) - 1) / tile_cols(tile)) *
           ((p.Ly + tile_rows(tile) - 1) / tile_rows(tile));
}

int64_t count_sampled(int64_t ta, int64_t tb, int64_t warmup, int64_t every) {
    if (every <= 0) return 0;
    const int64_t lo = std::max(ta, warmup);
    if (lo >= tb) return 0;
    const int64_t first = warmup + (lo - warmup + every - 1) / every * every;
    if (first >= tb) return 0;
    return (tb - 1 - first) / every + 1;
}

int64_t slot_time(const flb_batch_s* b, const BatchSlot& s) {
    return std::min<int64_t>(b->step - s.join, s.tend);
}

const void* kernel_of(int basis, int variant, bool sample) {
    return basis == FLB_BASIS_STANDARD ? batch_kernel_std(variant, sample)
           : basis == FLB_BASIS_LOCAL  ? batch_kernel_loc(variant, sample)
                                       : batch_kernel_lut(variant, sample);
}

const void* kernel_for(const flb_batch_s* b, bool sample) { return kernel_of(b->basis, b->tile, sample); }

cudaError_t launch(flb_batch_s* b, bool sample, cudaStream_t s) {
    BatchArgs a;
    a.desc = b->desc;
    a.tiles = b->tiles;
    a.ctl = b->ctl;
    a.lut = b->lut;
    void* params[1] = {(void*)&a};
    const BatchVariant& v = kBatchVariants[b->tile];
    const int warps = v.nw + (sample && !v.tensor() ? kSamplers : 1);
    return cudaLaunchKernel(kernel_for(b, sample), dim3(b->grid), dim3(warps * 32), params,
                            batch_smem_bytes(b->tile), s);
}

void drop_graphs(flb_batch_s* b) {
    for (auto& g : b->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

// Tensor maps of the replica's two buffers for boxes of the tile shape, and
// the tile-grid width the producer decodes tile indices with.
cudaError_t encode_maps(ReplicaDesc& d, const BatchSlot& s, int tile) {
    if (kBatchVariants[tile].mixed()) {
        const Bands bd = mixed_bands(s.p.Lx, s.p.Ly);
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < kKinds && e == cudaSuccess; ++k)
            for (int j = 0; j < 2 && e == cudaSuccess; ++j)
                e = tma_encode_planes(&d.map[2 * k + j], s.buf[j], s.geo, kind_bw(k), kind_th(k));
        d.hot.tiles_x = bd.nc[0];
        d.hot.kt0 = (int)bd.tiles[0];
        d.hot.kt01 = (int)(bd.tiles[0] + bd.tiles[1]);
        d.hot.kx1 = bd.nc[0] * kind_tw(0);
        d.hot.kx2 = d.hot.kx1 + bd.nc[1] * kind_tw(1);
        return e;
    }
    const int bw = tile_cols(tile) + 8, th = tile_rows(tile);
    cudaError_t e = tma_encode_planes(&d.map[0], s.buf[0], s.geo, bw, th);
    if (e == cudaSuccess) e = tma_encode_planes(&d.map[1], s.buf[1], s.geo, bw, th);
    d.hot.tiles_x = (s.p.Lx + tile_cols(tile) - 1) / tile_cols(tile);
    return e;
}

cudaError_t upload_desc(flb_batch_s* b, int slot) {
    return cudaMemcpyAsync(b->desc + slot, &b->hdesc[slot], sizeof(ReplicaDesc),
                           cudaMemcpyHostToDevice, b->stream);
}

// Rebuild the tile table from the live replicas (slot order) and upload it
// with the tile count; takes effect at the next launch.
cudaError_t upload_table(flb_batch_s* b) {
    if (!b->table_dirty) return cudaSuccess;
    b->htiles.clear();
    for (int k = 0; k < b->cap; ++k) {
        const BatchSlot& s = b->slots[k];
        if (!s.used) continue;
        const int n = (int)replica_tiles(s.p, b->tile);
        for (int t = 0; t < n; ++t) b->htiles.push_back(((uint32_t)k << kLocalBits) | (uint32_t)t);
    }
    if (b->htiles.size() > b->max_tiles) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    if (!b->htiles.empty())
        e = cudaMemcpyAsync(b->tiles, b->htiles.data(), sizeof(uint32_t) * b->htiles.size(),
                            cudaMemcpyHostToDevice, b->stream);
    const int n = (int)b->htiles.size();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&b->ctl->ntiles, &n, sizeof(int), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) b->table_dirty = false;
    return e;
}

bool slot_ok(const flb_batch_s* b, int slot) {
    return b && slot >= 0 && slot < b->cap && b->slots[slot].used;
}

int read_status(flb_batch_s* b, int slot) {
    DevError e;
    cudaError_t ce = cudaMemcpyAsync(&e, b->err + slot, sizeof(e), cudaMemcpyDeviceToHost, b->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(b->stream);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return FLB_ERR_CUDA;
    }
    return map_status(e.code);
}

}  // namespace

namespace flb {

int batch_enqueue_readout(flb_batch b, int slot, double* acc_out, DevError* err_out) {
    if (!slot_ok(b, slot)) return FLB_ERR_ARG;
    cudaError_t ce = cudaMemcpyAsync(acc_out, b->acc + (size_t)slot * kSums, sizeof(double) * kSums,
                                     cudaMemcpyDeviceToHost, b->stream);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(err_out, b->err + slot, sizeof(DevError), cudaMemcpyDeviceToHost,
                             b->stream);
    return ce == cudaSuccess ? FLB_OK : FLB_ERR_CUDA;
}

int64_t batch_samples(flb_batch b, int slot) { return slot_ok(b, slot) ? b->slots[slot].nsamp : 0; }

int64_t batch_replica_time(flb_batch b, int slot) {
    return slot_ok(b, slot) ? slot_time(b, b->slots[slot]) : -1;
}

cudaStream_t batch_stream(flb_batch b) { return b->stream; }

}  // namespace flb

extern "C" {

size_t flb_batch_replica_bytes(const flb_params* p) {
    if (!valid_params(p) || p->precision != FLB_FP32 || p->Lx > kMaxSide || p->Ly > kMaxSide)
        return 0;
    return 2 * buffer_bytes(make_geometry(p->Lx, p->Ly));
}

size_t flb_batch_workspace_bytes(const flb_params* p, int32_t n) {
    if (!p || n < 1) return 0;
    size_t total = 0;
    for (int k = 0; k < n; ++k) {
        const size_t r = flb_batch_replica_bytes(p + k);
        if (r == 0 || p[k].basis != p[0].basis) return 0;
        total += r;
    }
    return total;
}

int flb_batch_open(int32_t basis, int32_t max_replicas, size_t pool_bytes, void* stream,
                   flb_batch* out) {
    if (!out) return FLB_ERR_ARG;
    *out = nullptr;
    if ((basis != FLB_BASIS_STANDARD && basis != FLB_BASIS_LOCAL && basis != FLB_BASIS_LOCAL_LUT) ||
        max_replicas < 1 ||
        max_replicas > kMaxBatchReplicas || pool_bytes < Arena::kAlign)
        return FLB_ERR_ARG;
    flb_batch b = new (std::nothrow) flb_batch_s();
    if (!b) return FLB_ERR_OOM;
    b->basis = basis;
    b->cap = max_replicas;
    b->stream = (cudaStream_t)stream;
    b->slots.resize(max_replicas);
    b->hdesc.resize(max_replicas);
    std::memset((void*)b->hdesc.data(), 0, sizeof(ReplicaDesc) * b->hdesc.size());
    // a replica of B pool bytes has at most B / 9216 tiles of 128 x 2 nodes
    b->max_tiles = pool_bytes / 9216 + (size_t)max_replicas;
    const size_t desc_bytes = Arena::round_up(sizeof(ReplicaDesc) * max_replicas);
    const size_t tile_bytes = Arena::round_up(sizeof(uint32_t) * b->max_tiles);
    const size_t ctl_bytes = Arena::round_up(sizeof(BatchCtl));
    const size_t acc_bytes = Arena::round_up(sizeof(double) * kSums * max_replicas);
    const size_t err_bytes = Arena::round_up(sizeof(DevError) * max_replicas);
    const size_t meta_bytes = desc_bytes + tile_bytes + ctl_bytes + acc_bytes + err_bytes;
    void *pool = nullptr, *meta = nullptr;
    if (cudaMalloc(&pool, pool_bytes) != cudaSuccess || cudaMalloc(&meta, meta_bytes) != cudaSuccess) {
        cudaGetLastError();
        if (pool) cudaFree(pool);
        delete b;
        return FLB_ERR_OOM;
    }
    b->pool = (char*)pool;
    b->arena.reset(pool_bytes);
    b->meta = (char*)meta;
    char* m = b->meta;
    b->desc = (ReplicaDesc*)m;
    m += desc_bytes;
    b->tiles = (uint32_t*)m;
    m += tile_bytes;
    b->ctl = (BatchCtl*)m;
    m += ctl_bytes;
    b->acc = (double*)m;
    m += acc_bytes;
    b->err = (DevError*)m;

    int dev = 0;
    cudaError_t ce = cudaMemsetAsync(b->meta, 0, meta_bytes, b->stream);
    if (ce == cudaSuccess) ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    if (ce == cudaSuccess && b->basis == FLB_BASIS_LOCAL_LUT && lut_tables(&b->lut, nullptr) != FLB_OK)
        ce = cudaErrorUnknown;
    for (int v = 0; v < kNumBatchVariants && ce == cudaSuccess; ++v)
        for (int smp = 0; smp < 2 && ce == cudaSuccess; ++smp) {
            const void* fn = kernel_of(b->basis, v, smp);
            ce = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)batch_smem_bytes(v));
        }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(b->stream);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        cudaFree(b->pool);
        cudaFree(b->meta);
        delete b;
        return FLB_ERR_CUDA;
    }
    b->grid = std::max(1, b->sms);   // persistent: one CTA per SM
    *out = b;
    return FLB_OK;
}

int flb_batch_add(flb_batch b, const flb_params* p, int64_t nsteps, int32_t* slot) {
    if (!b || !slot || nsteps < 0 || nsteps >= INT_MAX) return FLB_ERR_ARG;
    if (!valid_params(p) || p->precision != FLB_FP32 || p->basis != b->basis ||
        p->Lx > kMaxSide || p->Ly > kMaxSide)
        return FLB_ERR_ARG;
    // the tensor-core shapes stage deviations in FP16: every replica must allow it
    if (kBatchVariants[b->tile].tensor() && !tensor_sampling_ok(p)) return FLB_ERR_ARG;
    int k = 0;
    while (k < b->cap && b->slots[k].used) ++k;
    if (k == b->cap) return FLB_ERR_OOM;
    BatchSlot s;
    s.p = *p;
    s.geo = make_geometry(p->Lx, p->Ly);
    const size_t half = buffer_bytes(s.geo);
    s.bytes = 2 * half;
    if (!b->arena.alloc(s.bytes, &s.off)) return FLB_ERR_OOM;
    s.buf[0] = (float*)(b->pool + s.off);
    s.buf[1] = (float*)(b->pool + s.off + half);
    s.used = true;
    s.join = b->step;
    s.tend = nsteps > 0 ? nsteps : INT_MAX;

    ReplicaDesc& d = b->hdesc[k];
    std::memset((void*)&d, 0, sizeof(d));
    ReplicaHot& h = d.hot;
    h.cc = collide_const<float>(p);
    double ref[9];
    feq_host(p->rho0, p->ux0, p->uy0, ref);
    Vec9 v;
    for (int i = 0; i < 9; ++i) {
        h.ref[i] = (float)ref[i];
        v.v[i] = ref[i];
    }
    h.Lx = p->Lx;
    h.Ly = p->Ly;
    h.gram_s = tensor_sampling_ok(p) ? (float)gram_scale(p) : 0.f;
    h.gram_inv = h.gram_s > 0.f ? (float)(1.0 / gram_scale(p)) : 0.f;
    for (int q = 0; q < 6; ++q) {
        h.pc.nomega[q] = make_float2(h.cc.nomega[q], h.cc.nomega[q]);
        h.pc.namp[q] = make_float2(-h.cc.amp[q], -h.cc.amp[q]);
    }
    h.sinv = make_float2(h.gram_inv, h.gram_inv);
    for (int i = 0; i < 9; ++i) {
        const float v = -h.ref[i] * h.gram_inv;   // the FP32 product the kernel formed before
        h.snref[i] = make_float2(v, v);
    }
    h.t0 = 0;
    h.join = (int)(unsigned)b->step;
    h.warmup = 0;
    h.every = 0;
    h.pitch = s.geo.pitch;
    h.plane = s.geo.plane;
    h.buf[0] = s.buf[0];
    h.buf[1] = s.buf[1];
    h.acc = b->acc + (size_t)k * kSums;
    h.err = b->err + k;
    h.tend = (int)s.tend;
    cudaError_t ce = encode_maps(d, s, b->tile);
    if (ce == cudaSuccess) {
        fill_kernel<float><<<grid_for(9 * s.geo.plane), 256, 0, b->stream>>>(s.buf[0], s.geo, v);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess)
        ce = cudaMemsetAsync(b->acc + (size_t)k * kSums, 0, sizeof(double) * kSums, b->stream);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(b->err + k, 0, sizeof(DevError), b->stream);
    if (ce == cudaSuccess) ce = upload_desc(b, k);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        b->arena.release(s.off);
        return FLB_ERR_CUDA;
    }
    b->slots[k] = s;
    b->table_dirty = true;
    *slot = k;
    return FLB_OK;
}

int flb_batch_remove(flb_batch b, int32_t slot) {
    if (!slot_ok(b, slot)) return FLB_ERR_ARG;
    // work already enqueued still uses the buffers; later users of the range
    // are ordered after it on the same stream
    b->arena.release(b->slots[slot].off);
    b->slots[slot] = BatchSlot();
    b->table_dirty = true;
    return FLB_OK;
}

int flb_batch_create(const flb_params* p, int32_t n, void* stream, flb_batch* out) {
    if (!out) return FLB_ERR_ARG;
    *out = nullptr;
    const size_t bytes = flb_batch_workspace_bytes(p, n);
    if (bytes == 0) return FLB_ERR_ARG;
    flb_batch b = nullptr;
    int rc = flb_batch_open(p[0].basis, n, bytes, stream, &b);
    for (int k = 0; k < n && rc == FLB_OK; ++k) {
        int32_t slot = -1;
        rc = flb_batch_add(b, p + k, 0, &slot);
        if (rc == FLB_OK && slot != k) rc = FLB_ERR_STATE;
    }
    if (rc == FLB_OK) {
        const cudaError_t ce = cudaStreamSynchronize(b->stream);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            rc = FLB_ERR_CUDA;
        }
    }
    if (rc != FLB_OK) {
        flb_batch_destroy(b);
        return rc;
    }
    *out = b;
    return FLB_OK;
}

int flb_batch_destroy(flb_batch b) {
    if (!b) return FLB_OK;
    cudaError_t ce = cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    const cudaError_t e1 = cudaFree(b->pool), e2 = cudaFree(b->meta);
    if (ce == cudaSuccess) ce = e1 != cudaSuccess ? e1 : e2;
    delete b;
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return FLB_ERR_CUDA;
    }
    return FLB_OK;
}

int flb_batch_set_sampling(flb_batch b, int32_t slot, int64_t warmup, int64_t every) {
    if (!b || warmup < 0 || every < 0 || warmup >= INT_MAX || every >= INT_MAX) return FLB_ERR_ARG;
    if (slot != -1 && !slot_ok(b, slot)) return FLB_ERR_ARG;
    cudaError_t ce = cudaSuccess;
    for (int k = 0; k < b->cap && ce == cudaSuccess; ++k) {
        if (!b->slots[k].used || (slot != -1 && k != slot)) continue;
        BatchSlot& s = b->slots[k];
        s.warmup = warmup;
        s.every = every;
        s.nsamp = 0;
        b->hdesc[k].hot.warmup = (int)warmup;
        b->hdesc[k].hot.every = (int)every;
        ce = upload_desc(b, k);
        if (ce == cudaSuccess)
            ce = cudaMemsetAsync(b->acc + (size_t)k * kSums, 0, sizeof(double) * kSums, b->stream);
    }
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return FLB_ERR_CUDA;
    }
    return FLB_OK;
}

int flb_batch_set_graph(flb_batch b, int32_t steps) {
    if (!b || steps < 0 || steps > 100000) return FLB_ERR_ARG;
    drop_graphs(b);
    b->graph_steps = steps;
    return FLB_OK;
}

// Whether every replica of the batch allows the tensor-core sums.
static bool batch_tensor_ok(const flb_batch_s* b) {
    for (const BatchSlot& s : b->slots)
        if (s.used && !tensor_sampling_ok(&s.p)) return false;
    return true;
}

int flb_batch_set_tile(flb_batch b, int32_t tile) {
    if (!b || tile < 0 || tile >= kNumBatchVariants) return FLB_ERR_ARG;
    if (tile == b->tile) return FLB_OK;
    if (kBatchVariants[tile].tensor() && !batch_tensor_ok(b)) return FLB_ERR_ARG;
    b->tile = tile;
    cudaError_t ce = cudaSuccess;
    for (int k = 0; k < b->cap && ce == cudaSuccess; ++k) {
        if (!b->slots[k].used) continue;
        ce = encode_maps(b->hdesc[k], b->slots[k], tile);
        if (ce == cudaSuccess) ce = upload_desc(b, k);
    }
    drop_graphs(b);
    b->table_dirty = true;
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return FLB_ERR_CUDA;
    }
    return FLB_OK;
}

int flb_batch_get_tile(flb_batch b, int32_t* tile) {
    if (!b || !tile) return FLB_ERR_ARG;
    *tile = b->tile;
    return FLB_OK;
}

int flb_batch_step(flb_batch b, int64_t n) {
    if (!b || n < 0) return FLB_ERR_ARG;
    if (n == 0) return FLB_OK;
    cudaError_t ce = upload_table(b);
    bool sample = false;
    for (const BatchSlot& s : b->slots)
        if (s.used && s.every > 0 && b->step - s.join < s.tend) sample = true;
    int64_t done = 0;
    if (ce == cudaSuccess && b->graph_steps > 0 && n >= b->graph_steps) {
        cudaGraphExec_t& ge = b->graph[sample ? 1 : 0];
        if (!ge) {
            cudaStream_t cs = nullptr;
            cudaGraph_t g = nullptr;
            ce = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
            if (ce == cudaSuccess) ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (ce == cudaSuccess) {
                for (int k = 0; k < b->graph_steps && ce == cudaSuccess; ++k) ce = launch(b, sample, cs);
                const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
                if (ce == cudaSuccess) ce = e2;
            }
            if (ce == cudaSuccess) ce = cudaGraphInstantiate(&ge, g, 0);
            if (g) cudaGraphDestroy(g);
            if (cs) cudaStreamDestroy(cs);
        }
        while (ce == cudaSuccess && n - done >= b->graph_steps) {
            ce = cudaGraphLaunch(ge, b->stream);
            done += b->graph_steps;
        }
    }
    for (; done < n && ce == cudaSuccess; ++done) ce = launch(b, sample, b->stream);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return FLB_ERR_CUDA;
    }
    for (BatchSlot& s : b->slots) {
        if (!s.used) continue;
        const int64_t ta = std::min<int64_t>(b->step - s.join, s.tend);
        const int64_t tb = std::min<int64_t>(b->step + n - s.join, s.tend);
        s.nsamp += count_sampled(ta, tb, s.warmup, s.every) * (int64_t)s.p.Lx * s.p.Ly;
    }
    b->step += n;
    return FLB_OK;
}

int flb_batch_autotune(flb_batch b, int32_t trial_steps, int32_t* tile, double* ms_per_step) {
    if (!b || trial_steps < 1 || trial_steps > 100000) return FLB_ERR_ARG;
    const int keep_graph = b->graph_steps;
    b->graph_steps = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    int best = b->tile, rc = FLB_OK;
    float best_ms = 0.f;
    for (int v = 0; v < kNumBatchVariants && ce == cudaSuccess && rc == FLB_OK; ++v) {
        if (kBatchVariants[v].tensor() && !batch_tensor_ok(b)) {   // not a candidate
            if (ms_per_step) ms_per_step[v] = -1.0;
            continue;
        }
        rc = flb_batch_set_tile(b, v);
        if (rc == FLB_OK) rc = flb_batch_step(b, 2);   // upload the table, warm the caches
        if (rc != FLB_OK) break;
        ce = cudaEventRecord(e0, b->stream);
        if (ce == cudaSuccess) rc = flb_batch_step(b, trial_steps);
        if (ce == cudaSuccess && rc == FLB_OK) ce = cudaEventRecord(e1, b->stream);
        if (ce == cudaSuccess && rc == FLB_OK) ce = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (ce == cudaSuccess && rc == FLB_OK) ce = cudaEventElapsedTime(&ms, e0, e1);
        ms /= (float)trial_steps;
        if (ms_per_step) ms_per_step[v] = ms;
        if (v == 0 || ms < best_ms) {
            best_ms = ms;
            best = v;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    b->graph_steps = keep_graph;
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return FLB_ERR_CUDA;
    }
    if (rc != FLB_OK) return rc;
    rc = flb_batch_set_tile(b, best);
    if (tile) *tile = best;
    return rc;
}

int flb_batch_sync(flb_batch b) {
    if (!b) return FLB_ERR_ARG;
    std::vector<DevError> e(b->cap);
    cudaError_t ce = cudaMemcpyAsync(e.data(), b->err, sizeof(DevError) * b->cap,
                                     cudaMemcpyDeviceToHost, b->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(b->stream);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return FLB_ERR_CUDA;
    }
    for (int k = 0; k < b->cap; ++k)
        if (b->slots[k].used && e[k].code) return map_status(e[k].code);
    return FLB_OK;
}

int flb_batch_status(flb_batch b, int32_t slot) {
    if (!slot_ok(b, slot)) return FLB_ERR_ARG;
    return read_status(b, slot);
}

int flb_batch_time(flb_batch b, int64_t* step) {
    if (!b || !step) return FLB_ERR_ARG;
    *step = b->step;
    return FLB_OK;
}

int flb_batch_replica_time(flb_batch b, int32_t slot, int64_t* t) {
    if (!slot_ok(b, slot) || !t) return FLB_ERR_ARG;
    *t = slot_time(b, b->slots[slot]);
    return FLB_OK;
}

int flb_batch_info(flb_batch b, int32_t* replicas, int64_t* tiles, size_t* pool_used,
                   size_t* pool_size) {
    if (!b) return FLB_ERR_ARG;
    int32_t n = 0;
    int64_t t = 0;
    for (const BatchSlot& s : b->slots)
        if (s.used) {
            ++n;
            t += replica_tiles(s.p, b->tile);
        }
    if (replicas) *replicas = n;
    if (tiles) *tiles = t;
    if (pool_used) *pool_used = b->arena.used();
    if (pool_size) *pool_size = b->arena.size();
    return FLB_OK;
}

int flb_batch_raw_sums(flb_batch b, int32_t slot, double* S1, double* S2, int64_t* n_samples) {
    if (!slot_ok(b, slot)) return FLB_ERR_ARG;
    double acc[kSums];
    cudaError_t ce = cudaMemcpyAsync(acc, b->acc + (size_t)slot * kSums, sizeof(acc),
                                     cudaMemcpyDeviceToHost, b->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(b->stream);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return FLB_ERR_CUDA;
    }
    const int rc = read_status(b, slot);
    if (rc) return rc;
    if (S1)
        for (int i = 0; i < 9; ++i) S1[i] = acc[i];
    if (S2) {
        int k = 9;
        for (int i = 0; i < 9; ++i)
            for (int j = i; j < 9; ++j, ++k) S2[i * 9 + j] = S2[j * 9 + i] = acc[k];
    }
    if (n_samples) *n_samples = b->slots[slot].nsamp;
    return FLB_OK;
}

int flb_batch_correlations(flb_batch b, int32_t n, const int32_t* slots, int32_t measure_basis,
                           double* Cff, double* CMM, double* mean_dev, int64_t* n_samples) {
    if (!b || n < 1 || !slots) return FLB_ERR_ARG;
    for (int32_t q = 0; q < n; ++q) {
        if (!slot_ok(b, slots[q])) return FLB_ERR_ARG;
        const flb_params& a = b->slots[slots[0]].p;
        const flb_params& c = b->slots[slots[q]].p;
        if (c.rho0 != a.rho0 || c.ux0 != a.ux0 || c.uy0 != a.uy0) return FLB_ERR_ARG;
    }
    double pooled[kSums] = {0.0};
    int64_t ns = 0;
    for (int32_t q = 0; q < n; ++q) {
        double acc[kSums];
        cudaError_t ce = cudaMemcpyAsync(acc, b->acc + (size_t)slots[q] * kSums, sizeof(acc),
                                         cudaMemcpyDeviceToHost, b->stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(b->stream);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            return FLB_ERR_CUDA;
        }
        const int rc = read_status(b, slots[q]);
        if (rc) return rc;
        for (int k = 0; k < kSums; ++k) pooled[k] += acc[k];
        ns += b->slots[slots[q]].nsamp;
    }
    if (n_samples) *n_samples = ns;
    const flb_params& p = b->slots[slots[0]].p;
    return finalize_sums(pooled, ns, measure_basis, p.ux0, p.uy0, b->stream, Cff, CMM, mean_dev);
}

int flb_batch_get_populations(flb_batch b, int32_t slot, double* host_out) {
    if (!slot_ok(b, slot) || !host_out) return FLB_ERR_ARG;
    const BatchSlot& s = b->slots[slot];
    const size_t n = (size_t)9 * s.p.Lx * s.p.Ly;
    double* tmp = nullptr;
    if (cudaMalloc(&tmp, n * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return FLB_ERR_OOM;
    }
    const float* src = s.buf[slot_time(b, s) & 1];
    gather_state_kernel<float><<<grid_for((long long)s.p.Lx * s.p.Ly), 256, 0, b->stream>>>(
        src, s.geo, tmp);
    cudaError_t ce = cudaGetLastError();
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(host_out, tmp, n * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(b->stream);
    cudaFree(tmp);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return FLB_ERR_CUDA;
    }
    return read_status(b, slot);
}

int flb_batch_set_populations(flb_batch b, int32_t slot, const double* host_in) {
    if (!slot_ok(b, slot) || !host_in) return FLB_ERR_ARG;
    const BatchSlot& s = b->slots[slot];
    const size_t n = (size_t)9 * s.p.Lx * s.p.Ly;
    double* tmp = nullptr;
    if (cudaMalloc(&tmp, n * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return FLB_ERR_OOM;
    }
    float* dst = s.buf[slot_time(b, s) & 1];
    cudaError_t ce = cudaMemcpyAsync(tmp, host_in, n * sizeof(double), cudaMemcpyHostToDevice,
                                     b->stream);
    if (ce == cudaSuccess) {
        scatter_state_kernel<float><<<grid_for((long long)s.p.Lx * s.p.Ly), 256, 0, b->stream>>>(
            tmp, s.geo, dst);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(b->stream);
    cudaFree(tmp);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return FLB_ERR_CUDA;
    }
    return FLB_OK;
}

}  // extern "C"
