// kmc_batch.cu -- many devices advanced together: per chunk of steps, one
// persistent launch per tile shape over all devices' rail tiles of that shape,
// replayed as a CUDA graph, with the CTA size and the steps per launch chosen
// by a measuring autotuner.
//
// Each device of a batch is an ordinary handle (kmc_create), so placement,
// per-device constants and observables are exactly those of a single device;
// the batch adds the work list, the shared step counter and the graph.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <string>
#include <vector>

#include "kmc_handle.h"
#include "kmc_internal.h"

using namespace kmc;

struct kmc_batch {
    std::vector<kmc_handle *> dev;       // one handle per device
    cudaStream_t user = nullptr;         // caller's stream
    cudaStream_t work = nullptr;         // stream the graph is captured and replayed on
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int64_t t = 0;                       // current absolute step
    int64_t n_total = 0;
    SweepArgs *inst = nullptr;           // device copies of the handles' arguments
    BatchItem *items = nullptr;          // grouped by kernel shape, longest tiles first in each
    unsigned *work_ctr = nullptr;        // [kShapeKinds] next work item of each shape
    int64_t *t0 = nullptr;
    int n_items = 0;
    int warps = 8;
    int steps_per_launch = 512;
    int flush = 256;
    int acc_req = -1;                    // accept path: -1 automatic, 0 off, 1 on
    int acc = 0;                         // accept path in effect
    BatchPlan plan{};                    // CTAs and shared memory of each shape's launch
    int cls_off[kShapeKinds + 1] = {};   // items of shape k: [cls_off[k], cls_off[k + 1])
    uint32_t rk0[10], rk1[10];
    cudaGraphExec_t graph = nullptr;     // one launch of steps_per_launch steps + advance
    int graph_warps = 0, graph_steps = 0, graph_acc = -1;
};

namespace {

int fail(int code, const std::string &msg)
{
    kmc_internal_set_error(msg.c_str());
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(e == cudaErrorMemoryAllocation ? KMC_E_NOMEM : KMC_E_CUDA,
                std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

#define BCK(call, what)                                    \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

void drop_graph(kmc_batch *b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_warps = b->graph_steps = 0;
    b->graph_acc = -1;
}

// Work list for a CTA size: one item per tile of 32/LPR * warps rails, larger
// tiles (longer rails) first so that the dynamic schedule ends evenly.
// Work items of a list of devices: every device's rails cut into tiles of
// (32 / lanes per rail) x warps rails, grouped by kernel shape and, within a
// shape, longest tiles first.  Returns the items and the shape offsets.
void make_items(const std::vector<const kmc_params *> &devs, const std::vector<int> &inst, int warps,
                std::vector<BatchItem> &sorted, int *cls_off)
{
    std::vector<BatchItem> items;
    std::vector<int64_t> cost;
    for (size_t i = 0; i < devs.size(); ++i) {
        const kmc_params &p = *devs[i];
        int wpl = 1;
        const int lpr = sweep_pick_lpr(p.n_sites, &wpl);
        const int64_t tile = (int64_t)(32 / lpr) * warps;
        for (int64_t r0 = 0; r0 < p.n_rails; r0 += tile) {
            BatchItem it;
            it.inst = inst[i];
            it.kind = sweep_kind(lpr, wpl);
            it.tile_rail0 = r0;
            items.push_back(it);
            cost.push_back(std::min<int64_t>(tile, p.n_rails - r0) * p.n_sites);
        }
    }
    std::vector<size_t> order(items.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
        return items[x].kind != items[y].kind ? items[x].kind < items[y].kind : cost[x] > cost[y];
    });
    sorted.resize(items.size());
    for (size_t i = 0; i < order.size(); ++i) sorted[i] = items[order[i]];
    for (int k = 0; k <= kShapeKinds; ++k) cls_off[k] = 0;
    for (const BatchItem &it : sorted) ++cls_off[it.kind + 1];
    for (int k = 0; k < kShapeKinds; ++k) cls_off[k + 1] += cls_off[k];
}

int build_items(kmc_batch *b, int warps)
{
    if (b->work) cudaStreamSynchronize(b->work);   // launches in flight may read the old list
    int dev = 0, max_smem = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (max_smem <= 0) max_smem = 48 * 1024;
    max_smem = std::min(max_smem, 200 * 1024);
    float p0max = 0.0f;
    for (const kmc_handle *h : b->dev) p0max = std::max(p0max, h->args.P0f_scalar);
    const int acc = b->acc_req >= 0 ? b->acc_req : (p0max >= kAcceptAutoP0 ? 1 : 0);
    // shared memory of each shape's CTAs: the largest of its devices' tiles
    BatchPlan plan{};
    std::vector<const kmc_params *> devs;
    std::vector<int> inst;
    for (size_t i = 0; i < b->dev.size(); ++i) {
        const kmc_params &p = b->dev[i]->p;
        int wpl = 1;
        const int lpr = sweep_pick_lpr(p.n_sites, &wpl);
        const int k = sweep_kind(lpr, wpl);
        plan.smem[k] = std::max(plan.smem[k], sweep_smem_bytes(lpr, wpl, p.n_zones, p.n_sites, warps,
                                                               b->flush, acc != 0));
        devs.push_back(&p);
        inst.push_back((int)i);
    }
    for (int k = 0; k < kShapeKinds; ++k)
        if (plan.smem[k] + 1024 > (size_t)max_smem)
            return fail(KMC_E_ARG, "batch: shared memory for this CTA size exceeds the device limit");
    std::vector<BatchItem> sorted;
    int cls_off[kShapeKinds + 1];
    make_items(devs, inst, warps, sorted, cls_off);
    if (b->items) cudaFreeAsync(b->items, b->user);
    b->items = nullptr;
    BCK(cudaMallocAsync((void **)&b->items, sizeof(BatchItem) * std::max<size_t>(1, sorted.size()),
                        b->user),
        "cudaMallocAsync(items)");
    BCK(cudaMemcpyAsync(b->items, sorted.data(), sizeof(BatchItem) * sorted.size(),
                        cudaMemcpyHostToDevice, b->user),
        "copy items");
    BCK(cudaStreamSynchronize(b->user), "batch items");
    b->n_items = (int)sorted.size();
    b->warps = warps;
    b->acc = acc;
    // one persistent grid per shape: every SM full (as many CTAs as its
    // registers and shared memory allow), at most one CTA per item
    for (int k = 0; k < kShapeKinds; ++k) {
        const int n = cls_off[k + 1] - cls_off[k];
        b->cls_off[k] = cls_off[k];
        plan.grid[k] = n > 0 ? std::min(n, sms * batch_ctas_per_sm(k, acc, warps, plan.smem[k])) : 0;
    }
    b->cls_off[kShapeKinds] = cls_off[kShapeKinds];
    b->plan = plan;
    drop_graph(b);
    return KMC_OK;
}

BatchArgs batch_args(const kmc_batch *b, int n_steps)
{
    BatchArgs a;
    memset(&a, 0, sizeof(a));
    a.inst = b->inst;
    a.items = b->items;
    a.n_items = b->n_items;
    for (int k = 0; k <= kShapeKinds; ++k) a.cls_off[k] = b->cls_off[k];
    a.n_steps = n_steps;
    a.flush = b->flush;
    a.n_inst = (int32_t)b->dev.size();
    a.max_z = 1;
    for (const kmc_handle *h : b->dev) a.max_z = std::max(a.max_z, (int32_t)h->p.n_zones);
    a.work = b->work_ctr;
    a.t0 = b->t0;
    a.t0_mut = b->t0;
    for (int i = 0; i < 10; ++i) {
        a.rk0[i] = b->rk0[i];
        a.rk1[i] = b->rk1[i];
    }
    return a;
}

// n_steps (<= 2^30) on the work stream: a graph replay when n_steps is the
// tuned chunk, a direct launch otherwise.
int run_chunk(kmc_batch *b, int n_steps)
{
    if (n_steps == b->steps_per_launch) {
        if (!b->graph || b->graph_warps != b->warps || b->graph_steps != n_steps ||
            b->graph_acc != b->acc) {
            drop_graph(b);
            cudaGraph_t g = nullptr;
            BCK(cudaStreamBeginCapture(b->work, cudaStreamCaptureModeThreadLocal), "begin capture");
            cudaError_t le = batch_launch(batch_args(b, n_steps), b->plan, b->warps, b->acc != 0,
                                          b->work);
            cudaError_t ce = cudaStreamEndCapture(b->work, &g);
            if (le != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return cuda_fail(le, "batched launch (capture)");
            }
            BCK(ce, "end capture");
            cudaError_t ie = cudaGraphInstantiate(&b->graph, g, 0);
            cudaGraphDestroy(g);
            BCK(ie, "cudaGraphInstantiate");
            b->graph_warps = b->warps;
            b->graph_steps = n_steps;
            b->graph_acc = b->acc;
        }
        BCK(cudaGraphLaunch(b->graph, b->work), "cudaGraphLaunch");
        return KMC_OK;
    }
    BCK(batch_launch(batch_args(b, n_steps), b->plan, b->warps, b->acc != 0, b->work),
        "batched launch");
    return KMC_OK;
}

int step_impl(kmc_batch *b, int64_t n_steps)
{
    BCK(cudaEventRecord(b->ev_in, b->user), "event");
    BCK(cudaStreamWaitEvent(b->work, b->ev_in, 0), "wait");
    int64_t left = n_steps;
    while (left > 0) {
        const int n = (int)std::min<int64_t>(left, b->steps_per_launch);
        int rc = run_chunk(b, n);
        if (rc) return rc;
        left -= n;
    }
    BCK(cudaEventRecord(b->ev_out, b->work), "event");
    BCK(cudaStreamWaitEvent(b->user, b->ev_out, 0), "wait");
    b->t += n_steps;
    for (kmc_handle *h : b->dev) h->t = b->t;
    return KMC_OK;
}

}  // namespace

extern "C" {

int kmc_batch_create(const kmc_params *params, int32_t n_inst, const double *const *V_per_step,
                     int64_t n_steps_total, const uint8_t *const *init_occ_or_null,
                     const double *const *Ea_site_or_null, void *cuda_stream, kmc_batch **out)
{
    if (!out) return fail(KMC_E_ARG, "out is NULL");
    *out = nullptr;
    if (!params || n_inst < 1) return fail(KMC_E_ARG, "batch needs params and n_inst >= 1");
    if (!V_per_step) return fail(KMC_E_ARG, "V_per_step is NULL");
    for (int i = 1; i < n_inst; ++i)
        if (params[i].seed != params[0].seed)
            return fail(KMC_E_ARG, "all devices of a batch share one seed (Philox key); "
                                   "they are told apart by their instance words");
    kmc_batch *b = new kmc_batch();
    b->user = (cudaStream_t)cuda_stream;
    b->n_total = n_steps_total;
    int rc = KMC_OK;
    for (int i = 0; i < n_inst && rc == KMC_OK; ++i) {
        kmc_handle *h = nullptr;
        rc = kmc_create(&params[i], V_per_step[i], n_steps_total,
                        init_occ_or_null ? init_occ_or_null[i] : nullptr,
                        Ea_site_or_null ? Ea_site_or_null[i] : nullptr, cuda_stream, &h);
        if (rc == KMC_OK) b->dev.push_back(h);
    }
    auto bail = [&](int code) {
        std::string msg = kmc_last_error();
        kmc_batch_destroy(b);
        kmc_internal_set_error(msg.c_str());
        return code;
    };
    if (rc != KMC_OK) return bail(rc);
    uint32_t k0 = (uint32_t)(params[0].seed & 0xffffffffu), k1 = (uint32_t)(params[0].seed >> 32);
    for (int i = 0; i < 10; ++i) {
        b->rk0[i] = k0;
        b->rk1[i] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&b->work, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming)) != cudaSuccess ||
        (e = batch_set_smem_limit()) != cudaSuccess)
        return bail(cuda_fail(e, "batch streams"));
    std::vector<SweepArgs> host(n_inst);
    for (int i = 0; i < n_inst; ++i) host[i] = b->dev[i]->args;
    if ((e = cudaMallocAsync((void **)&b->inst, sizeof(SweepArgs) * n_inst, b->user)) != cudaSuccess ||
        (e = cudaMallocAsync((void **)&b->work_ctr, sizeof(unsigned) * kShapeKinds, b->user)) != cudaSuccess ||
        (e = cudaMallocAsync((void **)&b->t0, sizeof(int64_t) * 2, b->user)) != cudaSuccess)
        return bail(cuda_fail(e, "batch allocation"));
    if ((e = cudaMemcpyAsync(b->inst, host.data(), sizeof(SweepArgs) * n_inst, cudaMemcpyHostToDevice,
                             b->user)) != cudaSuccess ||
        (e = cudaMemsetAsync(b->work_ctr, 0, sizeof(unsigned) * kShapeKinds, b->user)) != cudaSuccess ||
        (e = cudaMemsetAsync(b->t0, 0, sizeof(int64_t) * 2, b->user)) != cudaSuccess)
        return bail(cuda_fail(e, "batch set-up"));
    rc = build_items(b, b->warps);
    if (rc) return bail(rc);
    *out = b;
    return KMC_OK;
}

int kmc_batch_step_n(kmc_batch *b, int64_t n_steps)
{
    if (!b) return fail(KMC_E_ARG, "batch is NULL");
    if (n_steps < 0) return fail(KMC_E_ARG, "n_steps must be >= 0");
    if (b->t + n_steps > b->n_total)
        return fail(KMC_E_RANGE, "steps exceed the voltage tables of the batch");
    if (n_steps == 0) return KMC_OK;
    return step_impl(b, n_steps);
}

int kmc_batch_observables(kmc_batch *b, int32_t inst, int64_t first_step, int64_t count,
                          int64_t *J_out, int64_t *zone_counts_out, uint8_t *occ_out_or_null)
{
    if (!b) return fail(KMC_E_ARG, "batch is NULL");
    if (inst < 0 || inst >= (int32_t)b->dev.size()) return fail(KMC_E_ARG, "device index out of range");
    cudaError_t e = cudaStreamSynchronize(b->user);
    if (e != cudaSuccess) return cuda_fail(e, "batch sync");
    return kmc_observables(b->dev[inst], first_step, count, J_out, zone_counts_out, occ_out_or_null);
}

int kmc_batch_rail_current(kmc_batch *b, int32_t inst, int64_t *J_rail_out)
{
    if (!b) return fail(KMC_E_ARG, "batch is NULL");
    if (inst < 0 || inst >= (int32_t)b->dev.size()) return fail(KMC_E_ARG, "device index out of range");
    cudaError_t e = cudaStreamSynchronize(b->user);
    if (e != cudaSuccess) return cuda_fail(e, "batch sync");
    return kmc_rail_current(b->dev[inst], J_rail_out);
}

int kmc_batch_set_launch(kmc_batch *b, int32_t warps_per_cta, int32_t steps_per_launch)
{
    if (!b) return fail(KMC_E_ARG, "batch is NULL");
    if (warps_per_cta != 1 && warps_per_cta != 2 && warps_per_cta != 4 && warps_per_cta != 8)
        return fail(KMC_E_ARG, "warps_per_cta must be 1, 2, 4 or 8");
    if (steps_per_launch < 1 || steps_per_launch > (1 << 20))
        return fail(KMC_E_ARG, "steps_per_launch must be in [1, 2^20]");
    b->steps_per_launch = steps_per_launch;
    if (warps_per_cta != b->warps) return build_items(b, warps_per_cta);
    drop_graph(b);
    return KMC_OK;
}

int kmc_batch_tune(kmc_batch *b, int64_t probe_steps, int32_t *warps_out, int32_t *steps_out)
{
    if (!b) return fail(KMC_E_ARG, "batch is NULL");
    if (probe_steps < 1) return fail(KMC_E_ARG, "probe_steps must be >= 1");
    if (b->t + probe_steps > b->n_total)
        return fail(KMC_E_RANGE, "probe steps exceed the voltage tables of the batch");
    // save every device's state (occupancy, counters, per-rail current); the
    // probes advance real steps from it and it is restored after every probe
    cudaError_t e = cudaStreamSynchronize(b->user);
    if (e != cudaSuccess) return cuda_fail(e, "batch sync");
    std::vector<void *> saved(b->dev.size(), nullptr);
    auto cleanup = [&]() {
        for (void *p : saved)
            if (p) cudaFreeAsync(p, b->user);
        cudaStreamSynchronize(b->user);
    };
    for (size_t i = 0; i < b->dev.size(); ++i) {
        kmc_handle *h = b->dev[i];
        const size_t occ_b = (size_t)h->stride * h->p.n_rails;
        const size_t bytes = occ_b + sizeof(unsigned long long) * 8 + sizeof(int64_t) * h->p.n_rails;
        if ((e = cudaMallocAsync(&saved[i], bytes, b->user)) != cudaSuccess) {
            cleanup();
            return cuda_fail(e, "tune: save buffer");
        }
        cudaMemcpyAsync(saved[i], h->occ, occ_b, cudaMemcpyDeviceToDevice, b->user);
        cudaMemcpyAsync((char *)saved[i] + occ_b, h->misc, sizeof(unsigned long long) * 8,
                        cudaMemcpyDeviceToDevice, b->user);
        cudaMemcpyAsync((char *)saved[i] + occ_b + sizeof(unsigned long long) * 8, h->Jr,
                        sizeof(int64_t) * h->p.n_rails, cudaMemcpyDeviceToDevice, b->user);
    }
    auto restore = [&]() {
        cudaStreamSynchronize(b->work);
        for (size_t i = 0; i < b->dev.size(); ++i) {
            kmc_handle *h = b->dev[i];
            const size_t occ_b = (size_t)h->stride * h->p.n_rails;
            cudaMemcpyAsync(h->occ, saved[i], occ_b, cudaMemcpyDeviceToDevice, b->user);
            cudaMemcpyAsync(h->misc, (char *)saved[i] + occ_b, sizeof(unsigned long long) * 8,
                            cudaMemcpyDeviceToDevice, b->user);
            cudaMemcpyAsync(h->Jr, (char *)saved[i] + occ_b + sizeof(unsigned long long) * 8,
                            sizeof(int64_t) * h->p.n_rails, cudaMemcpyDeviceToDevice, b->user);
            cudaMemsetAsync(h->J + b->t, 0, sizeof(int64_t) * (size_t)probe_steps, b->user);
            cudaMemsetAsync(h->Zc + b->t * h->p.n_zones, 0,
                            sizeof(int64_t) * (size_t)probe_steps * h->p.n_zones, b->user);
        }
        const int64_t t = b->t;
        cudaMemcpyAsync(b->t0, &t, sizeof(int64_t), cudaMemcpyHostToDevice, b->user);
        cudaStreamSynchronize(b->user);
    };
    const int cand_warps[] = {4, 8};
    const int cand_steps[] = {64, 128, 256, 512, 1024, 2048};
    double best = -1.0;
    int best_w = b->warps, best_s = b->steps_per_launch;
    const int64_t t_start = b->t;
    const int acc_req = b->acc_req;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // steps per second of the current items at sp steps per launch
    auto probe = [&](int sp) {
        b->steps_per_launch = sp;
        const int64_t n = probe_steps / sp * sp;
        run_chunk(b, sp);  // warm-up (captures the graph)
        restore();
        cudaEventRecord(e0, b->work);
        for (int64_t k = 0; k < n; k += sp) run_chunk(b, sp);
        cudaEventRecord(e1, b->work);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        restore();
        return (double)n / (ms > 0 ? ms : 1e-3);
    };
    for (int w : cand_warps) {
        int rc = build_items(b, w);
        if (rc) continue;  // this CTA size does not fit
        for (int sp : cand_steps) {
            if (sp > probe_steps) continue;
            const double rate = probe(sp);
            if (rate > best) {
                best = rate;
                best_w = w;
                best_s = sp;
            }
        }
    }
    // with the automatic accept path, try the other kernel at the best shape
    int best_acc = -1;
    if (acc_req < 0 && best > 0.0) {
        int rc = build_items(b, best_w);
        const int auto_acc = b->acc;
        if (rc == KMC_OK) {
            b->acc_req = 1 - auto_acc;
            if (build_items(b, best_w) == KMC_OK && probe(best_s) > best) best_acc = 1 - auto_acc;
        }
        b->acc_req = acc_req;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->t = t_start;
    cleanup();
    b->steps_per_launch = best_s;
    if (best_acc >= 0) b->acc_req = best_acc;
    int rc = build_items(b, best_w);
    if (rc) return rc;
    if (warps_out) *warps_out = best_w;
    if (steps_out) *steps_out = best_s;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "tune");
    return KMC_OK;
}

int kmc_batch_set_accept_path(kmc_batch *b, int32_t mode)
{
    if (!b) return fail(KMC_E_ARG, "batch is NULL");
    if (mode < -1 || mode > 1) return fail(KMC_E_ARG, "mode must be -1, 0 or 1");
    b->acc_req = mode;
    return build_items(b, b->warps);
}

int kmc_batch_accept_path(const kmc_batch *b) { return b ? b->acc : -1; }

int kmc_batch_grad(kmc_batch *b, int32_t inst, const double *dLoss_dJ, const double *dLoss_dZc,
                   double grad_out[4], double stderr_out[4])
{
    if (!b) return fail(KMC_E_ARG, "batch is NULL");
    if (inst < 0 || inst >= (int32_t)b->dev.size()) return fail(KMC_E_ARG, "device index out of range");
    cudaError_t e = cudaStreamSynchronize(b->user);
    if (e != cudaSuccess) return cuda_fail(e, "batch sync");
    return kmc_grad(b->dev[inst], dLoss_dJ, dLoss_dZc, grad_out, stderr_out);
}

int kmc_batch_grad_all(kmc_batch *b, const double *const *dLoss_dJ, const double *const *dLoss_dZc,
                       double *grad_out, double *stderr_out)
{
    if (!b || !grad_out) return fail(KMC_E_ARG, "batch or grad_out is NULL");
    cudaError_t e = cudaStreamSynchronize(b->user);
    if (e != cudaSuccess) return cuda_fail(e, "batch sync");
    const int n_inst = (int)b->dev.size();
    std::vector<double> out((size_t)n_inst * 8, 0.0);
    std::vector<SweepArgs> gargs((size_t)n_inst);
    std::vector<char> active((size_t)n_inst, 0);
    int dev = 0, max_smem = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (max_smem <= 0) max_smem = 48 * 1024;
    max_smem = std::min(max_smem, 200 * 1024);
    int n_active = 0;
    for (int i = 0; i < n_inst && b->t > 0; ++i) {
        const double *wJ = dLoss_dJ ? dLoss_dJ[i] : nullptr;
        const double *wZ = dLoss_dZc ? dLoss_dZc[i] : nullptr;
        if (!wJ && !wZ) continue;
        int rc = grad_prepare(b->dev[i], wJ, wZ, &gargs[(size_t)i]);
        if (rc) return rc;
        active[(size_t)i] = 1;
        ++n_active;
    }
    if (n_active > 0) {
        // CTA size: 8 warps unless some device's tile needs less shared memory
        int warps = 8;
        auto smem_for = [&](int w) {
            size_t m = 0;
            for (int i = 0; i < n_inst; ++i)
                if (active[(size_t)i]) {
                    const kmc_params &p = b->dev[(size_t)i]->p;
                    int wpl = 1;
                    const int lpr = sweep_pick_lpr(p.n_sites, &wpl);
                    m = std::max(m, grad_smem_bytes(lpr, wpl, p.n_zones, p.n_sites, w));
                }
            return m;
        };
        while (warps > 1 && smem_for(warps) > (size_t)max_smem) warps >>= 1;
        if (smem_for(warps) > (size_t)max_smem)
            return fail(KMC_E_ARG, "batched gradient pass: shared memory exceeds the device limit");
        // work items grouped by shape, longest tiles first in each; one
        // persistent launch per shape, its shared memory the largest tile's
        std::vector<const kmc_params *> devs;
        std::vector<int> inst;
        BatchPlan plan{};
        for (int i = 0; i < n_inst; ++i) {
            if (!active[(size_t)i]) continue;
            const kmc_params &p = b->dev[(size_t)i]->p;
            int wpl = 1;
            const int lpr = sweep_pick_lpr(p.n_sites, &wpl);
            const int k = sweep_kind(lpr, wpl);
            plan.smem[k] = std::max(plan.smem[k], grad_smem_bytes(lpr, wpl, p.n_zones, p.n_sites, warps));
            devs.push_back(&p);
            inst.push_back(i);
        }
        std::vector<BatchItem> sorted;
        int cls_off[kShapeKinds + 1];
        make_items(devs, inst, warps, sorted, cls_off);
        for (int k = 0; k < kShapeKinds; ++k) {
            const int n = cls_off[k + 1] - cls_off[k];
            plan.grid[k] = n > 0 ? std::min(n, sms * batch_ctas_per_sm(k, 2, warps, plan.smem[k])) : 0;
        }
        SweepArgs *ginst = nullptr;
        BatchItem *gitems = nullptr;
        BCK(cudaMallocAsync((void **)&ginst, sizeof(SweepArgs) * (size_t)n_inst, b->user), "grad args");
        e = cudaMallocAsync((void **)&gitems, sizeof(BatchItem) * sorted.size(), b->user);
        if (e != cudaSuccess) {
            cudaFreeAsync(ginst, b->user);
            return cuda_fail(e, "grad items");
        }
        BatchArgs a = batch_args(b, (int)b->t);
        a.inst = ginst;
        a.items = gitems;
        a.n_items = (int)sorted.size();
        for (int k = 0; k <= kShapeKinds; ++k) a.cls_off[k] = cls_off[k];
        if ((e = cudaMemcpyAsync(ginst, gargs.data(), sizeof(SweepArgs) * (size_t)n_inst,
                                 cudaMemcpyHostToDevice, b->user)) == cudaSuccess &&
            (e = cudaMemcpyAsync(gitems, sorted.data(), sizeof(BatchItem) * sorted.size(),
                                 cudaMemcpyHostToDevice, b->user)) == cudaSuccess &&
            (e = cudaMemsetAsync(b->work_ctr, 0, sizeof(unsigned) * kShapeKinds, b->user)) == cudaSuccess &&
            (e = batch_grad_launch(a, plan, warps, b->user)) == cudaSuccess)
            // re-arm for the forward
            e = cudaMemsetAsync(b->work_ctr, 0, sizeof(unsigned) * kShapeKinds, b->user);
        cudaFreeAsync(gitems, b->user);
        cudaFreeAsync(ginst, b->user);
        if (e != cudaSuccess) return cuda_fail(e, "batched gradient pass");
        for (int i = 0; i < n_inst; ++i)
            if (active[(size_t)i]) {
                int rc = grad_reduce_out(b->dev[(size_t)i], &out[(size_t)i * 8]);
                if (rc) return rc;
            }
        BCK(cudaStreamSynchronize(b->user), "batched gradient pass");
    }
    for (int i = 0; i < n_inst; ++i)
        grad_outputs(b->dev[(size_t)i], &out[(size_t)i * 8], grad_out + 4 * (size_t)i,
                     stderr_out ? stderr_out + 4 * (size_t)i : nullptr);
    return KMC_OK;
}

int64_t kmc_batch_current_step(const kmc_batch *b) { return b ? b->t : -1; }

void kmc_batch_destroy(kmc_batch *b)
{
    if (!b) return;
    if (b->user) cudaStreamSynchronize(b->user);
    if (b->work) cudaStreamSynchronize(b->work);
    drop_graph(b);
    cudaStream_t s = b->user;
    if (b->inst) cudaFreeAsync(b->inst, s);
    if (b->items) cudaFreeAsync(b->items, s);
    if (b->work_ctr) cudaFreeAsync(b->work_ctr, s);
    if (b->t0) cudaFreeAsync(b->t0, s);
    cudaStreamSynchronize(s);
    for (kmc_handle *h : b->dev) kmc_destroy(h);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->work) cudaStreamDestroy(b->work);
    delete b;
}

}  // extern "C"
