// The library context behind the opaque lbm_ctx handle of include/lbm.h,
// shared by the API and adjoint translation units.
#pragma once

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "body.cuh"

// launch orders of a step whose band is known ahead (see lbm_step); the
// first TRIAL_STEPS steps after lbm_set_geometry alternate them, the first
// pair warming up, the other two pairs timed
enum { ORDER_UNDECIDED = LBM_ORDER_AUTO, ORDER_SPLIT = LBM_ORDER_SPLIT, ORDER_SEQUENTIAL = LBM_ORDER_SEQUENTIAL };
constexpr int TRIAL_STEPS = 6;

struct lbm_ctx {
    lbm::Lattice L;
    int storage = 0;
    size_t elem = 0;
    void *f[2] = {nullptr, nullptr};
    int cur = 0;
    uint8_t *flags = nullptr;
    cudaStream_t stream = nullptr;
    lbm::GeomParams G{};
    bool has_body = false;
    bool initialised = false;
    lbm::Scratch S{};
    int bcur = 0;                 // body copy holding the latest state
    cudaStream_t side = nullptr;  // boundary + force kernels, overlapping the bulk kernel
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    double *plane = nullptr;      // N doubles for the host codec
    double *tot_partials = nullptr;
    int tot_blocks = 608;
    int64_t launches = 0;
    // asynchronous force records: a copy stream, one event per ring entry,
    // the record each ticket writes, and per body slot the last copy out of it
    cudaStream_t copy = nullptr;
    cudaEvent_t ev_step = nullptr;
    cudaEvent_t ev_copy[LBM_RECORD_DEPTH] = {};
    lbm_force_record *rec[LBM_RECORD_DEPTH] = {};
    cudaEvent_t ev_slot[2] = {nullptr, nullptr};
    bool slot_pending[2] = {false, false};
    int64_t next_ticket = 0;
    // launch order of steps whose band is known ahead (lbm_step): 0 not yet
    // chosen, 1 split, 2 sequential; the trial steps that time both and the
    // events around them; whether the last step ran split
    int order = 0;
    int order_request = 0;  // LBM_ORDER_* asked for by the caller
    int trial = 0;
    cudaEvent_t ev_trial[5] = {};
    bool last_split = false;
    std::vector<cudaEvent_t> prof;  // start/stop pairs around bulk launches
    int prof_used = 0;
    bool prof_open = false;
    std::string err;
    // slab of a box split along z (lbm_set_slab); zper = 0: none
    int slab_zoff = 0, slab_zper = 0, slab_own_lo = 0, slab_own_hi = 0;
    // lbm_step_interior has enqueued the interior layers of a step that
    // lbm_step_edges completes
    bool interior_pending = false;
    // caller's device allocator for the scratch (lbm_set_allocator; null:
    // cudaMalloc / cudaFree) and the number of live blocks taken through
    // ctx_malloc
    lbm_alloc_fn dev_alloc = nullptr;
    lbm_release_fn dev_release = nullptr;
    void *alloc_user = nullptr;
    long long live_blocks = 0;
};

// device scratch of a context, through the caller's allocator when one is set
inline cudaError_t ctx_malloc(lbm_ctx *ctx, void **p, size_t bytes)
{
    if (bytes == 0) bytes = 1;
    if (ctx->dev_alloc) {
        *p = ctx->dev_alloc(bytes, (void *)ctx->stream, ctx->alloc_user);
        if (!*p) return cudaErrorMemoryAllocation;
        // the kernels' vector accesses need the alignment cudaMalloc gives
        if (reinterpret_cast<uintptr_t>(*p) & 255u) {
            ctx->dev_release(*p, (void *)ctx->stream, ctx->alloc_user);
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
    } else {
        const cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            *p = nullptr;
            return e;
        }
    }
    ctx->live_blocks++;
    return cudaSuccess;
}
template <typename T>
inline cudaError_t ctx_alloc(lbm_ctx *ctx, T **p, size_t count)
{
    void *v = nullptr;
    const cudaError_t e = ctx_malloc(ctx, &v, count * sizeof(T));
    *p = static_cast<T *>(v);
    return e;
}
inline void ctx_release(lbm_ctx *ctx, void *p)
{
    if (!p) return;
    if (ctx->dev_release) ctx->dev_release(p, (void *)ctx->stream, ctx->alloc_user);
    else cudaFree(p);
    ctx->live_blocks--;
}

// An NVTX range over one library call or phase, named after it: ncu and
// nsys can select the kernels enqueued inside it (ncu --nvtx --nvtx-include
// "lbm_refine_step/"); without a tool attached the push and pop do nothing.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// records the start (which = 0) or stop (1) event of a profiled bulk launch
// on the context stream while a profile (lbm_profile_begin) is open
cudaError_t ctx_prof_mark(lbm_ctx *ctx, int which);

// One step t -> t+1 of ctx in the sequential launch order (the body's
// geometry and refill, then its boundary nodes and force beside one
// flag-aware bulk launch), with the bookkeeping of lbm_step: the context's
// current state buffer and body slot advance.  Adds its launches to
// *launches.  Used by the refined step for a fine level that carries a body.
cudaError_t ctx_step_flagged(lbm_ctx *ctx, int *launches);

// waits on the host for the asynchronous force-record copies that may still
// read the body slots (before a call that rewrites the slots)
inline cudaError_t drain_records(lbm_ctx *ctx)
{
    if (!ctx->copy) return cudaSuccess;
    ctx->slot_pending[0] = ctx->slot_pending[1] = false;
    return cudaStreamSynchronize(ctx->copy);
}

