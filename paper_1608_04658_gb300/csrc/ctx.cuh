// The library context behind the opaque lbm_ctx handle of include/lbm.h,
// shared by the API and adjoint translation units.
#pragma once

#include <string>
#include <vector>

#include "body.cuh"

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
    std::vector<cudaEvent_t> prof;  // start/stop pairs around bulk launches
    int prof_used = 0;
    bool prof_open = false;
    std::string err;
};

