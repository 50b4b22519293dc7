// kmc_handle.h -- host-side state of one device (one kmc_handle) shared by
// the single-device runtime (kmc_capi.cu) and the batch runtime (kmc_batch.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>
#include <vector>

#include "kmc_internal.h"

namespace kmc {

// Device allocator in effect when a handle was created.
struct Allocator {
    kmc_alloc_fn alloc = nullptr;
    kmc_free_fn free_fn = nullptr;
    void *ctx = nullptr;
};

}  // namespace kmc

struct kmc_handle {
    kmc_params p{};
    cudaStream_t stream = nullptr;
    int64_t n_total = 0;
    int64_t t = 0;
    int64_t stride = 0;
    kmc::Allocator al;
    std::vector<std::pair<void *, size_t>> allocs;

    uint8_t *occ = nullptr;
    double *V = nullptr;
    int32_t *N0 = nullptr;
    double *P0site = nullptr;
    float *P0f = nullptr;
    float2 *P0bnd = nullptr;
    double2 *bgd = nullptr;                   // [R][Z] backgrounds of the FP64 decision paths
    kmc::DevConst *K = nullptr;
    unsigned long long *J = nullptr;
    unsigned long long *Zc = nullptr;
    kmc_log_entry *log = nullptr;
    unsigned long long *misc = nullptr;  // [0] log count, [1..3] counters, [4] scratch count
    kmc::SweepArgs *args_dev = nullptr;       // device copy of args for the kernels' rare paths
    int64_t log_cap = 4096;
    uint8_t *occ_init = nullptr;              // occupancy at step 0: the gradient pass's checkpoint
    int64_t *Jr = nullptr;                    // [R] per-rail net leftward crossings so far

    // gradient pass (allocated at the first kmc_grad)
    uint8_t *g_occ = nullptr;                 // replayed occupancy
    double *g_state = nullptr;                // [R][kGradState]
    double *g_wJ = nullptr;                   // weight of J_t per step
    double *g_fJab = nullptr;                 // per step (aJ, bJ): baselined current share
    double *g_fZa = nullptr, *g_fZb = nullptr;  // per step aZ[Z], bZ: baselined zone share
    int32_t *g_fZr = nullptr;                   // per step range of zones with a nonzero aZ
    double *g_out = nullptr;                  // [8] sums and standard errors
    unsigned long long *g_misc = nullptr;     // log count and counters of the replay
    kmc::SweepArgs *g_args_dev = nullptr;
    double *g_etab = nullptr;                 // exp tables of the zone sums (1024 + nH doubles)
    int32_t g_etM = -1;                       // their range, or -1 when not built

    kmc::SweepArgs args{};
    kmc::SweepLaunch launch{};
    int warps_req = 0;
    int flush_req = 0;
    int accept_req = -1;   // accept path: -1 automatic, 0 off, 1 on

    void *alloc(size_t bytes)
    {
        void *ptr = nullptr;
        if (bytes == 0) bytes = 16;
        if (al.alloc) {
            ptr = al.alloc(bytes, (void *)stream, al.ctx);
        } else if (cudaMallocAsync(&ptr, bytes, stream) != cudaSuccess) {
            cudaGetLastError();
            ptr = nullptr;
        }
        if (ptr) allocs.emplace_back(ptr, bytes);
        return ptr;
    }
    void release_all()
    {
        for (auto &a : allocs) {
            if (al.free_fn) al.free_fn(a.first, a.second, (void *)stream, al.ctx);
            else cudaFreeAsync(a.first, stream);
        }
        allocs.clear();
        cudaStreamSynchronize(stream);
    }
};

namespace kmc {
// Host side of the gradient pass (kmc_capi.cu), shared with the batch runtime.
int grad_prepare(kmc_handle *h, const double *dLoss_dJ, const double *dLoss_dZc, SweepArgs *ga);
int grad_reduce_out(kmc_handle *h, double *out_host);
void grad_outputs(const kmc_handle *h, const double out[8], double grad_out[4], double stderr_out[4]);
}  // namespace kmc
