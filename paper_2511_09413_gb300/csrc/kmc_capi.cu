// kmc_capi.cu -- host runtime behind the C ABI of include/kmc.h: parameter
// validation, device memory, initial placement, launch configuration and
// observable readback.  All compute runs in the kernels of kmc_sweep.cu and
// kmc_setup.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "kmc_handle.h"
#include "kmc_internal.h"

using namespace kmc;

namespace {

thread_local std::string g_err;

Allocator g_alloc;
std::mutex g_alloc_mu;
std::once_flag g_attr_once;
cudaError_t g_attr_err = cudaSuccess;

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(e == cudaErrorMemoryAllocation ? KMC_E_NOMEM : KMC_E_CUDA, "%s: %s (%s)", what,
                cudaGetErrorName(e), cudaGetErrorString(e));
}

}  // namespace

void kmc::kmc_internal_set_error(const char *msg) { g_err = msg ? msg : ""; }


namespace {

bool finite_pos(double x) { return isfinite(x) && x > 0.0; }

int validate(const kmc_params *p, const double *V, int64_t n_total, const uint8_t *occ0)
{
    if (!p) return fail(KMC_E_ARG, "params is NULL");
    if (p->n_rails < 1) return fail(KMC_E_ARG, "n_rails must be >= 1 (got %d)", p->n_rails);
    if (p->n_sites < 2 || p->n_sites > KMC_MAX_SITES)
        return fail(KMC_E_ARG, "n_sites must be in [2, %d] (got %d)", KMC_MAX_SITES, p->n_sites);
    if (p->n_zones < 1 || p->n_zones > KMC_MAX_ZONES || p->n_zones > p->n_sites)
        return fail(KMC_E_ARG, "n_zones must be in [1, min(n_sites, %d)] (got %d)", KMC_MAX_ZONES,
                    p->n_zones);
    if (p->electrodes != 0 && p->electrodes != 1)
        return fail(KMC_E_ARG, "electrodes must be 0 or 1 (got %d)", p->electrodes);
    if (!finite_pos(p->site_spacing_nm)) return fail(KMC_E_ARG, "site_spacing_nm must be > 0");
    if (!finite_pos(p->dt_s)) return fail(KMC_E_ARG, "dt_s must be > 0");
    if (!finite_pos(p->T_K)) return fail(KMC_E_ARG, "T_K must be > 0");
    if (!(isfinite(p->nu_Hz) && p->nu_Hz >= 0.0)) return fail(KMC_E_ARG, "nu_Hz must be >= 0");
    if (!isfinite(p->Ea_eV)) return fail(KMC_E_ARG, "Ea_eV must be finite");
    if (!isfinite(p->alpha_V) || !isfinite(p->kappa))
        return fail(KMC_E_ARG, "alpha_V and kappa must be finite");
    if (p->electrodes == 1) {
        if (!(isfinite(p->k_electrode_Hz) && p->k_electrode_Hz >= 0.0))
            return fail(KMC_E_ARG, "k_electrode_Hz must be >= 0");
        if (!(p->rho_electrode >= 0.0 && p->rho_electrode <= 1.0))
            return fail(KMC_E_ARG, "rho_electrode must be in [0, 1]");
    }
    if (p->update_rule != 0 && p->update_rule != 1)
        return fail(KMC_E_ARG, "update_rule must be 0 or 1 (got %d)", p->update_rule);
    if (p->rail_base < 0 || (int64_t)p->rail_base + p->n_rails > (int64_t)INT32_MAX)
        return fail(KMC_E_ARG, "rail_base must be >= 0 with rail_base + n_rails <= 2^31 - 1");
    if (p->rail_base != 0 && p->init_mode == 0)
        return fail(KMC_E_ARG, "init_mode 0 (exact ion count) is defined over a whole device: "
                               "it needs rail_base 0 (place a part with init_mode 1 or 2)");
    if (n_total < 0 || n_total >= (int64_t)kInitStep)
        return fail(KMC_E_ARG, "n_steps_total must be in [0, 2^32 - 1)");
    if (n_total > 0 && !V) return fail(KMC_E_ARG, "V_per_step is NULL");
    const int64_t nsites = (int64_t)p->n_rails * p->n_sites;
    switch (p->init_mode) {
    case 0:
        if (p->n_ions < 0 || p->n_ions > nsites)
            return fail(KMC_E_ARG, "n_ions must be in [0, n_rails * n_sites]");
        break;
    case 1:
        if (!(p->fill >= 0.0 && p->fill <= 1.0)) return fail(KMC_E_ARG, "fill must be in [0, 1]");
        break;
    case 2:
        if (!occ0) return fail(KMC_E_ARG, "init_mode 2 needs init_occ_or_null");
        break;
    default:
        return fail(KMC_E_ARG, "init_mode must be 0, 1 or 2 (got %d)", p->init_mode);
    }
    for (int64_t i = 0; i < n_total; ++i)
        if (!isfinite(V[i])) return fail(KMC_E_ARG, "V_per_step[%lld] is not finite", (long long)i);
    return KMC_OK;
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

int pick_launch(kmc_handle *h)
{
    const kmc_params &p = h->p;
    SweepLaunch l{};
    l.lpr = sweep_pick_lpr(p.n_sites, &l.wpl);
    const int G = 32 / l.lpr;
    int flush = h->flush_req > 0 ? h->flush_req : 256;
    int warps = h->warps_req > 0 ? h->warps_req : 8;
    warps = std::min(warps, 8);
    int dev = 0, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (max_smem <= 0) max_smem = 48 * 1024;
    max_smem = std::min(max_smem, 200 * 1024);
    l.acc = h->accept_req >= 0 ? h->accept_req : (h->args.P0f_scalar >= kAcceptAutoP0 ? 1 : 0);
    const bool acc = l.acc != 0;
    while (warps > 1 && sweep_smem_bytes(l.lpr, l.wpl, p.n_zones, p.n_sites, warps, flush,
                                         acc) > (size_t)max_smem)
        warps >>= 1;
    while (flush > 1 && sweep_smem_bytes(l.lpr, l.wpl, p.n_zones, p.n_sites, warps, flush,
                                         acc) > (size_t)max_smem)
        flush >>= 1;
    l.warps = warps;
    l.smem = sweep_smem_bytes(l.lpr, l.wpl, p.n_zones, p.n_sites, warps, flush, acc);
    const int64_t rails_per_cta = (int64_t)G * warps;
    l.grid = (int)((p.n_rails + rails_per_cta - 1) / rails_per_cta);
    h->launch = l;
    h->args.flush = flush;
    return KMC_OK;
}

void fill_args(kmc_handle *h)
{
    const kmc_params &p = h->p;
    SweepArgs &a = h->args;
    a.occ = h->occ;
    a.stride = h->stride;
    a.R = p.n_rails;
    a.L = p.n_sites;
    a.Z = p.n_zones;
    a.electrodes = p.electrodes;
    a.instance = p.instance;
    a.rail_base = (uint32_t)p.rail_base;
    uint32_t k0 = (uint32_t)(p.seed & 0xffffffffu), k1 = (uint32_t)(p.seed >> 32);
    for (int i = 0; i < 10; ++i) {
        a.rk0[i] = k0;
        a.rk1[i] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    a.V = h->V;
    a.N0 = h->N0;
    a.P0site = h->P0site;
    a.P0f = h->P0f;
    a.P0bnd = h->P0bnd;
    a.bgd = h->bgd;
    a.K = h->K;
    a.self = h->args_dev;
    a.J = h->J;
    a.Zc = h->Zc;
    a.log = h->log;
    a.log_count = h->misc;
    a.log_cap = h->log_cap;
    a.counters = h->misc + 1;
    a.Jr = (long long *)h->Jr;
    const int L = p.n_sites, Z = p.n_zones;
    int bnd[KMC_MAX_ZONES + 1];
    for (int z = 0; z <= Z; ++z) bnd[z] = (int)(((int64_t)z * L) / Z);
    for (int z = 0; z <= KMC_MAX_ZONES; ++z) a.bnd[z] = z <= Z ? bnd[z] : L;
    double H = 0.0;
    for (int z = 0; z < Z; ++z) H += (double)(bnd[z + 1] - bnd[z]) * (double)(bnd[z] + bnd[z + 1]);
    for (int z = 0; z <= KMC_MAX_ZONES; ++z) {
        int w_prev = (z >= 1 && z <= Z) ? bnd[z] - bnd[z - 1] : 0;
        int w_cur = (z < Z) ? bnd[z + 1] - bnd[z] : 0;
        a.wsum[z] = w_prev + w_cur;
    }
    for (int z = 0; z < KMC_MAX_ZONES; ++z)
        a.cz[z] = z < Z ? (float)(((double)(bnd[z] + bnd[z + 1]) - H / L) / (2.0 * L)) : 0.0f;
    const double kT = 8.6173e-5 * p.T_K;
    a.inv_L = (float)(1.0 / L);
    a.inv_LkT = (float)(1.0 / ((double)L * kT));
    a.ka_f = (float)(p.kappa * p.alpha_V);
    a.delta = 1.0f / 1024.0f;
    a.rule = p.update_rule;
}

int init_exact_count(kmc_handle *h)
{
    const kmc_params &p = h->p;
    const int64_t n = p.n_ions;
    const int64_t nsites = (int64_t)p.n_rails * p.n_sites;
    unsigned long long *dcount = h->misc + 4;
    auto count = [&](uint64_t bound, int mode, int64_t idx, unsigned long long *out) -> int {
        CK(cudaMemsetAsync(dcount, 0, sizeof(unsigned long long), h->stream), "memset");
        CK(setup_count_keys(p, bound, mode, idx, dcount, h->stream), "count_keys launch");
        CK(cudaMemcpyAsync(out, dcount, sizeof(*out), cudaMemcpyDeviceToHost, h->stream), "copy");
        CK(cudaStreamSynchronize(h->stream), "count_keys");
        return KMC_OK;
    };
    if (n == 0) {
        CK(setup_mark_smallest(p, 0, 0, 1, h->occ, h->stride, h->stream), "mark launch");
        return KMC_OK;
    }
    // smallest key K* with #(key <= K*) >= n
    uint64_t lo = 0, hi = ~0ull;
    unsigned long long c = 0;
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo) / 2;
        int rc = count(mid, 0, 0, &c);
        if (rc) return rc;
        if ((int64_t)c >= n) hi = mid;
        else lo = mid + 1;
    }
    const uint64_t kstar = lo;
    unsigned long long below = 0;
    if (kstar > 0) {
        int rc = count(kstar - 1, 0, 0, &below);
        if (rc) return rc;
    }
    const int64_t m = n - (int64_t)below;  // sites with key == K* still to take, by index
    int64_t ilo = 0, ihi = nsites - 1;
    while (ilo < ihi) {
        const int64_t mid = ilo + (ihi - ilo) / 2;
        int rc = count(kstar, 1, mid, &c);
        if (rc) return rc;
        if ((int64_t)c >= m) ihi = mid;
        else ilo = mid + 1;
    }
    CK(setup_mark_smallest(p, kstar, ilo, 0, h->occ, h->stride, h->stream), "mark launch");
    return KMC_OK;
}

int create_impl(const kmc_params *params, const double *V, int64_t n_total, const uint8_t *occ0,
                const double *Ea, void *stream, kmc_handle *h)
{
    int rc = validate(params, V, n_total, occ0);
    if (rc) return rc;
    h->p = *params;
    h->stream = (cudaStream_t)stream;
    h->n_total = n_total;
    h->t = 0;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        h->al = g_alloc;
    }
    std::call_once(g_attr_once, [] { g_attr_err = sweep_set_smem_limits(); });
    if (g_attr_err != cudaSuccess) return cuda_fail(g_attr_err, "cudaFuncSetAttribute");

    const kmc_params &p = h->p;
    const int64_t R = p.n_rails, L = p.n_sites, Z = p.n_zones;
    h->stride = (L + 15) / 16 * 16;
    const size_t occ_bytes = (size_t)(R * h->stride);
    h->occ = (uint8_t *)h->alloc(occ_bytes);
    h->V = (double *)h->alloc(sizeof(double) * (size_t)std::max<int64_t>(n_total, 1));
    h->N0 = (int32_t *)h->alloc(sizeof(int32_t) * (size_t)R);
    h->K = (DevConst *)h->alloc(sizeof(DevConst));
    h->J = (unsigned long long *)h->alloc(sizeof(int64_t) * (size_t)std::max<int64_t>(n_total, 1));
    h->Zc = (unsigned long long *)h->alloc(sizeof(int64_t) * (size_t)std::max<int64_t>(n_total, 1) *
                                           (size_t)Z);
    h->log = (kmc_log_entry *)h->alloc(sizeof(kmc_log_entry) * (size_t)h->log_cap);
    h->misc = (unsigned long long *)h->alloc(sizeof(unsigned long long) * 8);
    h->args_dev = (SweepArgs *)h->alloc(sizeof(SweepArgs));
    h->occ_init = (uint8_t *)h->alloc(occ_bytes);
    h->Jr = (int64_t *)h->alloc(sizeof(int64_t) * (size_t)R);
    h->bgd = (double2 *)h->alloc(sizeof(double2) * (size_t)R * (size_t)Z);
    if (!h->bgd || !h->Jr || !h->occ_init || !h->args_dev || !h->occ || !h->V || !h->N0 || !h->K || !h->J || !h->Zc || !h->log || !h->misc)
        return fail(KMC_E_NOMEM, "device allocation failed");
    if (Ea) {
        h->P0site = (double *)h->alloc(sizeof(double) * (size_t)(R * L));
        h->P0f = (float *)h->alloc(sizeof(float) * (size_t)(R * L));
        h->P0bnd = (float2 *)h->alloc(sizeof(float2) * (size_t)(R * Z));
        if (!h->P0site || !h->P0f || !h->P0bnd)
            return fail(KMC_E_NOMEM, "device allocation failed (P0 table)");
    }
    cudaStream_t s = h->stream;
    CK(cudaMemsetAsync(h->misc, 0, sizeof(unsigned long long) * 8, s), "memset");
    CK(cudaMemsetAsync(h->J, 0, sizeof(int64_t) * (size_t)std::max<int64_t>(n_total, 1), s), "memset");
    CK(cudaMemsetAsync(h->Zc, 0, sizeof(int64_t) * (size_t)std::max<int64_t>(n_total, 1) * (size_t)Z, s),
       "memset");
    CK(cudaMemsetAsync(h->occ, 0, occ_bytes, s), "memset");
    CK(cudaMemsetAsync(h->Jr, 0, sizeof(int64_t) * (size_t)R, s), "memset");
    CK(setup_constants(p, h->K, s), "constants launch");
    if (n_total > 0)
        CK(cudaMemcpyAsync(h->V, V, sizeof(double) * (size_t)n_total, cudaMemcpyHostToDevice, s),
           "copy V");

    // initial placement
    if (p.init_mode == 2) {
        CK(cudaMemcpy2DAsync(h->occ, (size_t)h->stride, occ0, (size_t)L, (size_t)L, (size_t)R,
                             cudaMemcpyHostToDevice, s),
           "copy occupancy");
    } else if (p.init_mode == 1) {
        CK(setup_init_bernoulli(p, h->occ, h->stride, s), "bernoulli launch");
    } else {
        rc = init_exact_count(h);
        if (rc) return rc;
    }
    unsigned long long *bad = h->misc + 5;
    CK(setup_row_counts(h->occ, h->stride, (int32_t)R, (int32_t)L, h->N0, bad, s), "row counts");
    CK(setup_background(h->N0, (int32_t)R, (int32_t)L, (int32_t)Z, h->K, h->bgd, s), "background");
    CK(cudaMemcpyAsync(h->occ_init, h->occ, occ_bytes, cudaMemcpyDeviceToDevice, s), "checkpoint");

    int *p0bad = (int *)(h->misc + 6);
    if (Ea) {
        CK(cudaMemcpyAsync(h->P0site, Ea, sizeof(double) * (size_t)(R * L), cudaMemcpyHostToDevice, s),
           "copy Ea");
        CK(setup_p0_table(p, h->P0site, h->P0site, R * L, p0bad, s), "P0 table");
        CK(setup_p0_bounds(h->P0site, (int32_t)R, (int32_t)L, (int32_t)Z, h->K, h->P0bnd, s),
           "P0 bounds");
        CK(setup_p0_float(h->P0site, R * L, h->P0f, s), "P0 float table");
    }
    // check derived values
    DevConst kc;
    unsigned long long flags[8];
    CK(cudaMemcpyAsync(&kc, h->K, sizeof(kc), cudaMemcpyDeviceToHost, s), "copy constants");
    CK(cudaMemcpyAsync(flags, h->misc, sizeof(flags), cudaMemcpyDeviceToHost, s), "copy flags");
    CK(cudaStreamSynchronize(s), "create");
    if (kc.status == KMC_E_PROB)
        return fail(KMC_E_PROB, "derived probability outside [0, 1]: P0=%g E_in=%g E_out=%g", kc.P0,
                    kc.E_in, kc.E_out);
    if (kc.status != 0) return fail(kc.status, "invalid derived constants");
    if (flags[5] != 0)
        return fail(KMC_E_ARG, "initial occupancy has %llu bytes that are not 0 or 1", flags[5]);
    if (Ea && (int)(flags[6] & 0xffffffffu) != 0)
        return fail(KMC_E_PROB, "per-site base probability outside [0, 1] (check Ea_site)");
    CK(cudaMemsetAsync(h->misc, 0, sizeof(unsigned long long) * 8, s), "memset");
    fill_args(h);
    h->args.P0f_scalar = kc.P0f;
    h->args.E_inf = kc.E_inf;
    h->args.E_outf = kc.E_outf;
    rc = pick_launch(h);
    if (rc) return rc;
    CK(cudaMemcpyAsync(h->args_dev, &h->args, sizeof(SweepArgs), cudaMemcpyHostToDevice, s),
       "copy args");
    CK(cudaStreamSynchronize(s), "create");
    return KMC_OK;
}

}  // namespace

// Gradient pass, host side (shared by kmc_grad and kmc_batch_grad_all):
// validate, allocate the pass's buffers at the first call, upload the
// observable's per-step coefficients (with the forward's totals for the
// leave-one-out baselines), copy the step-0 checkpoint to the replay
// buffer, clear the per-rail state, and fill the replay's arguments.
int kmc::grad_prepare(kmc_handle *h, const double *dLoss_dJ, const double *dLoss_dZc, SweepArgs *gout)
{
    if (h->P0site)
        return fail(KMC_E_ARG, "kmc_grad needs a scalar barrier (the handle has per-site Ea)");
    if (h->p.update_rule != 0)
        return fail(KMC_E_ARG, "kmc_grad follows the synchronous update (update_rule 0)");
    const kmc_params &p = h->p;
    const int64_t R = p.n_rails, L = p.n_sites, Z = p.n_zones, n = h->t;
    if (n > ((int64_t)1 << 30)) return fail(KMC_E_RANGE, "gradient pass over more than 2^30 steps");
    cudaStream_t s = h->stream;
    const size_t occ_bytes = (size_t)(R * h->stride);
    const size_t nt = (size_t)std::max<int64_t>(h->n_total, 1);
    if (!h->g_occ) {
        h->g_occ = (uint8_t *)h->alloc(occ_bytes);
        h->g_state = (double *)h->alloc(sizeof(double) * kGradState * (size_t)std::max<int64_t>(R, 1));
        h->g_wJ = (double *)h->alloc(sizeof(double) * nt);
        h->g_fJab = (double *)h->alloc(sizeof(double) * 2 * nt);
        h->g_fZa = (double *)h->alloc(sizeof(double) * nt * (size_t)Z);
        h->g_fZb = (double *)h->alloc(sizeof(double) * nt);
        h->g_fZr = (int32_t *)h->alloc(sizeof(int32_t) * nt);
        h->g_out = (double *)h->alloc(sizeof(double) * 8);
        h->g_misc = (unsigned long long *)h->alloc(sizeof(unsigned long long) * 8);
        h->g_args_dev = (SweepArgs *)h->alloc(sizeof(SweepArgs));
        if (!h->g_occ || !h->g_state || !h->g_wJ || !h->g_fJab || !h->g_fZa || !h->g_fZb || !h->g_fZr ||
            !h->g_out || !h->g_misc || !h->g_args_dev)
            return fail(KMC_E_NOMEM, "device allocation failed (gradient pass)");
    }
    for (int64_t i = 0; i < n; ++i)
        if (dLoss_dJ && !isfinite(dLoss_dJ[i]))
            return fail(KMC_E_ARG, "dLoss_dJ[%lld] is not finite", (long long)i);
    if (dLoss_dZc)
        for (int64_t i = 0; i < n * Z; ++i)
            if (!isfinite(dLoss_dZc[i]))
                return fail(KMC_E_ARG, "dLoss_dZc[%lld] is not finite", (long long)i);
    // the forward's totals give each step's leave-one-out baseline:
    //   fJ = wJ (J_r - (J_t - J_r) / (R - 1)) = aJ J_r - bJ, and likewise fZ
    std::vector<int64_t> Jt((size_t)n), Zt;
    CK(cudaMemcpyAsync(Jt.data(), h->J, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToHost, s),
       "copy J");
    if (dLoss_dZc) {
        Zt.resize((size_t)(n * Z));
        CK(cudaMemcpyAsync(Zt.data(), h->Zc, sizeof(int64_t) * (size_t)(n * Z),
                           cudaMemcpyDeviceToHost, s),
           "copy Zc");
    }
    CK(cudaStreamSynchronize(s), "totals");
    const double loo = R > 1 ? (double)(R - 1) : 0.0;
    const double scale = R > 1 ? (double)R / loo : 1.0;
    std::vector<double> fJab, fZa, fZb;
    std::vector<int32_t> fZr;
    if (dLoss_dJ) {
        fJab.resize((size_t)(2 * n));
        for (int64_t i = 0; i < n; ++i) {
            fJab[2 * i] = dLoss_dJ[i] * scale;
            fJab[2 * i + 1] = loo > 0.0 ? dLoss_dJ[i] * ((double)Jt[i] / loo) : 0.0;
        }
        CK(cudaMemcpyAsync(h->g_wJ, dLoss_dJ, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, s),
           "copy dLoss_dJ");
        CK(cudaMemcpyAsync(h->g_fJab, fJab.data(), sizeof(double) * (size_t)(2 * n),
                           cudaMemcpyHostToDevice, s),
           "copy fJ coefficients");
    }
    if (dLoss_dZc) {
        fZa.resize((size_t)(n * Z));
        fZb.assign((size_t)n, 0.0);
        fZr.assign((size_t)n, 0);
        for (int64_t i = 0; i < n; ++i) {
            int lo = (int)Z, hi = 0;
            for (int64_t z = 0; z < Z; ++z) {
                const double w = dLoss_dZc[i * Z + z];
                fZa[(size_t)(i * Z + z)] = w * scale;
                if (loo > 0.0) fZb[(size_t)i] += w * ((double)Zt[(size_t)(i * Z + z)] / loo);
                if (w != 0.0) {
                    lo = std::min(lo, (int)z);
                    hi = (int)z + 1;
                }
            }
            // the replay skips the zones outside [lo, hi), and the whole step
            // when no weight is set (its share is then zero)
            if (hi > 0) fZr[(size_t)i] = lo | (hi << 8);
        }
        CK(cudaMemcpyAsync(h->g_fZa, fZa.data(), sizeof(double) * (size_t)(n * Z),
                           cudaMemcpyHostToDevice, s),
           "copy fZ coefficients");
        CK(cudaMemcpyAsync(h->g_fZb, fZb.data(), sizeof(double) * (size_t)n,
                           cudaMemcpyHostToDevice, s),
           "copy fZ offsets");
        CK(cudaMemcpyAsync(h->g_fZr, fZr.data(), sizeof(int32_t) * (size_t)n,
                           cudaMemcpyHostToDevice, s),
           "copy fZ zone ranges");
    }
    CK(cudaMemcpyAsync(h->g_occ, h->occ_init, occ_bytes, cudaMemcpyDeviceToDevice, s), "checkpoint");
    CK(cudaMemsetAsync(h->g_state, 0, sizeof(double) * kGradState * (size_t)std::max<int64_t>(R, 1), s),
       "memset");
    CK(cudaMemsetAsync(h->g_misc, 0, sizeof(unsigned long long) * 8, s), "memset");
    // the replay: same trajectory (same counters), no traces, no log
    SweepArgs ga = h->args;
    ga.occ = h->g_occ;
    ga.self = h->g_args_dev;
    ga.J = nullptr;
    ga.Zc = nullptr;
    ga.log = h->log;
    ga.log_cap = 0;
    ga.log_count = h->g_misc;
    ga.counters = h->g_misc + 1;
    ga.Jr = nullptr;
    ga.wJ = dLoss_dJ ? h->g_wJ : nullptr;
    ga.fJab = dLoss_dJ ? (const double2 *)h->g_fJab : nullptr;
    ga.fZa = dLoss_dZc ? h->g_fZa : nullptr;
    ga.fZb = dLoss_dZc ? h->g_fZb : nullptr;
    ga.fZr = dLoss_dZc ? h->g_fZr : nullptr;
    ga.gstate = h->g_state;
    ga.alpha = p.alpha_V;
    const double kT = 8.6173e-5 * p.T_K;
    ga.tdev_kT = ((double)L * p.site_spacing_nm) * kT;
    // exp tables of the integer zone sums: |cm m| <= kappa alpha / kT over
    // |m| <= 2 L^2; built once per handle, used while every factor is finite
    ga.etL = ga.etH = nullptr;
    ga.etM = 0;
    const double ka = p.kappa * p.alpha_V;
    if (fabs(ka) / kT < 600.0) {
        const int32_t M = (int32_t)(2 * L * L);
        const int32_t nH = 2 * M / 1024 + 2;
        if (!h->g_etab) {
            h->g_etab = (double *)h->alloc(sizeof(double) * (size_t)(1024 + nH));
            if (!h->g_etab) return fail(KMC_E_NOMEM, "device allocation failed (exp tables)");
        }
        if (h->g_etM != M) {
            const double cm = ka / (2.0 * (double)L * (double)L * kT);
            CK(setup_exp_tables(cm, M, h->g_etab, h->g_etab + 1024, nH, s), "exp tables");
            h->g_etM = M;
        }
        ga.etL = h->g_etab;
        ga.etH = h->g_etab + 1024;
        ga.etM = M;
    }
    CK(cudaMemcpyAsync(h->g_args_dev, &ga, sizeof(SweepArgs), cudaMemcpyHostToDevice, s),
       "copy args");
    ga.t0 = 0;
    ga.n_steps = (int32_t)n;
    ga.flush = (int32_t)n;
    *gout = ga;
    return KMC_OK;
}

// Per-rail sums and standard errors into out[8] (enqueued on the handle's stream).
int kmc::grad_reduce_out(kmc_handle *h, double *out_host)
{
    const kmc_params &p = h->p;
    const bool has_rho = p.init_mode == 1 && p.fill > 0.0 && p.fill < 1.0;
    const double kT = 8.6173e-5 * p.T_K;
    // d ln P0 / d Ea and d ln P0 / d nu (Eq. 1, P0 = 1 - exp(-x), x = 2 Gamma0 dt)
    const double x = 2.0 * (p.nu_Hz * exp(-p.Ea_eV / kT)) * p.dt_s;
    const double P0 = -expm1(-x);
    const double cEa = -((x / kT) * exp(-x)) / P0;
    const double cnu = ((x / p.nu_Hz) * exp(-x)) / P0;
    CK(grad_reduce(h->g_state, p.n_rails, h->N0, p.n_sites, p.fill, has_rho ? 1 : 0, cEa, cnu,
                   h->g_out, h->stream),
       "gradient reduce launch");
    CK(cudaMemcpyAsync(out_host, h->g_out, sizeof(double) * 8, cudaMemcpyDeviceToHost, h->stream),
       "copy gradient");
    return KMC_OK;
}

// grad_out / stderr_out from the reduced sums; the fill entry is NaN unless
// the placement was Bernoulli(fill).
void kmc::grad_outputs(const kmc_handle *h, const double out[8], double grad_out[4],
                       double stderr_out[4])
{
    const kmc_params &p = h->p;
    const bool has_rho = p.init_mode == 1 && p.fill > 0.0 && p.fill < 1.0;
    for (int i = 0; i < 4; ++i) {
        grad_out[i] = out[i];
        if (stderr_out) stderr_out[i] = out[4 + i];
    }
    if (!has_rho) {
        grad_out[3] = NAN;
        if (stderr_out) stderr_out[3] = NAN;
    }
}

extern "C" {

int kmc_set_allocator(kmc_alloc_fn alloc, kmc_free_fn free_fn, void *ctx)
{
    if ((alloc == nullptr) != (free_fn == nullptr))
        return fail(KMC_E_ARG, "alloc and free must both be set or both be NULL");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc.alloc = alloc;
    g_alloc.free_fn = free_fn;
    g_alloc.ctx = alloc ? ctx : nullptr;
    return KMC_OK;
}

int kmc_create(const kmc_params *params, const double *V_per_step, int64_t n_steps_total,
               const uint8_t *init_occ_or_null, const double *Ea_site_or_null, void *cuda_stream,
               kmc_handle **out)
{
    if (!out) return fail(KMC_E_ARG, "out is NULL");
    *out = nullptr;
    kmc_handle *h = new (std::nothrow) kmc_handle();
    if (!h) return fail(KMC_E_NOMEM, "host allocation failed");
    int rc = create_impl(params, V_per_step, n_steps_total, init_occ_or_null, Ea_site_or_null,
                         cuda_stream, h);
    if (rc != KMC_OK) {
        std::string msg = g_err;
        h->release_all();
        delete h;
        cudaGetLastError();
        g_err = msg;
        return rc;
    }
    *out = h;
    g_err.clear();
    return KMC_OK;
}

int kmc_step_n(kmc_handle *h, int64_t n_steps)
{
    if (!h) return fail(KMC_E_ARG, "handle is NULL");
    if (n_steps < 0) return fail(KMC_E_ARG, "n_steps must be >= 0");
    if (h->t + n_steps > h->n_total)
        return fail(KMC_E_RANGE, "steps [%lld, %lld) exceed the voltage table (%lld steps)",
                    (long long)h->t, (long long)(h->t + n_steps), (long long)h->n_total);
    while (n_steps > 0) {
        const int64_t n = std::min<int64_t>(n_steps, 1 << 30);
        h->args.t0 = h->t;
        h->args.n_steps = (int32_t)n;
        cudaError_t e = sweep_launch(h->args, h->launch, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "sweep launch");
        e = zone_scan(h->Zc, h->t, (int)n, h->p.n_zones, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "zone-count scan launch");
        h->t += n;
        n_steps -= n;
    }
    return KMC_OK;
}

int kmc_observables(kmc_handle *h, int64_t first_step, int64_t count, int64_t *J_out,
                    int64_t *zone_counts_out, uint8_t *occ_out_or_null)
{
    if (!h) return fail(KMC_E_ARG, "handle is NULL");
    if (first_step < 0 || count < 0 || first_step + count > h->t)
        return fail(KMC_E_RANGE, "steps [%lld, %lld) not simulated yet (current step %lld)",
                    (long long)first_step, (long long)(first_step + count), (long long)h->t);
    cudaStream_t s = h->stream;
    if (count > 0 && J_out)
        CK(cudaMemcpyAsync(J_out, h->J + first_step, sizeof(int64_t) * (size_t)count,
                           cudaMemcpyDeviceToHost, s),
           "copy J");
    if (count > 0 && zone_counts_out)
        CK(cudaMemcpyAsync(zone_counts_out, h->Zc + first_step * h->p.n_zones,
                           sizeof(int64_t) * (size_t)count * (size_t)h->p.n_zones,
                           cudaMemcpyDeviceToHost, s),
           "copy zone counts");
    if (occ_out_or_null)
        CK(cudaMemcpy2DAsync(occ_out_or_null, (size_t)h->p.n_sites, h->occ, (size_t)h->stride,
                             (size_t)h->p.n_sites, (size_t)h->p.n_rails, cudaMemcpyDeviceToHost, s),
           "copy occupancy");
    CK(cudaStreamSynchronize(s), "observables");
    return KMC_OK;
}

int kmc_rail_current(kmc_handle *h, int64_t *J_rail_out)
{
    if (!h || !J_rail_out) return fail(KMC_E_ARG, "handle or J_rail_out is NULL");
    CK(cudaMemcpyAsync(J_rail_out, h->Jr, sizeof(int64_t) * (size_t)h->p.n_rails,
                       cudaMemcpyDeviceToHost, h->stream),
       "copy per-rail current");
    CK(cudaStreamSynchronize(h->stream), "rail current");
    return KMC_OK;
}

int kmc_set_voltage(kmc_handle *h, int64_t first_step, int64_t count, const double *V_host)
{
    if (!h) return fail(KMC_E_ARG, "handle is NULL");
    if (first_step < 0 || count < 0 || first_step + count > h->n_total)
        return fail(KMC_E_RANGE, "steps [%lld, %lld) outside the voltage table",
                    (long long)first_step, (long long)(first_step + count));
    if (count == 0) return KMC_OK;
    if (!V_host) return fail(KMC_E_ARG, "V_host is NULL");
    for (int64_t i = 0; i < count; ++i)
        if (!isfinite(V_host[i])) return fail(KMC_E_ARG, "V_host[%lld] is not finite", (long long)i);
    CK(cudaMemcpyAsync(h->V + first_step, V_host, sizeof(double) * (size_t)count,
                       cudaMemcpyHostToDevice, h->stream),
       "copy V");
    return KMC_OK;
}

int kmc_near_threshold_log(kmc_handle *h, kmc_log_entry *out, int64_t cap, int64_t *n_total)
{
    if (!h || !n_total) return fail(KMC_E_ARG, "handle or n_total is NULL");
    unsigned long long n = 0;
    CK(cudaMemcpyAsync(&n, h->misc, sizeof(n), cudaMemcpyDeviceToHost, h->stream), "copy count");
    CK(cudaStreamSynchronize(h->stream), "log");
    *n_total = (int64_t)n;
    const int64_t k = std::min<int64_t>(std::min<int64_t>((int64_t)n, h->log_cap), cap);
    if (k > 0 && out) {
        CK(cudaMemcpyAsync(out, h->log, sizeof(kmc_log_entry) * (size_t)k, cudaMemcpyDeviceToHost,
                           h->stream),
           "copy log");
        CK(cudaStreamSynchronize(h->stream), "log");
    }
    return KMC_OK;
}

int kmc_philox_probe(void *cuda_stream, double *blocks_per_s)
{
    if (!blocks_per_s) return fail(KMC_E_ARG, "blocks_per_s is NULL");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev), "cudaGetDevice");
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    const int grid = sms * 8, iters = 20000;   // 8 CTAs of 256 threads per SM
    uint32_t *sink = nullptr;
    CK(cudaMallocAsync((void **)&sink, sizeof(uint32_t) * (size_t)grid * 256, s), "probe buffer");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = philox_probe(grid, iters / 10, sink, s);      // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = philox_probe(grid, iters, sink, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(sink, s);
    cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "Philox probe");
    *blocks_per_s = (double)grid * 256.0 * 4.0 * (double)iters / ((double)ms * 1e-3);
    return KMC_OK;
}

int kmc_counters(kmc_handle *h, uint64_t out[3])
{
    if (!h || !out) return fail(KMC_E_ARG, "handle or out is NULL");
    unsigned long long c[3];
    CK(cudaMemcpyAsync(c, h->misc + 1, sizeof(c), cudaMemcpyDeviceToHost, h->stream), "copy");
    CK(cudaStreamSynchronize(h->stream), "counters");
    for (int i = 0; i < 3; ++i) out[i] = c[i];
    return KMC_OK;
}

int kmc_set_launch(kmc_handle *h, int warps_per_cta, int flush_steps)
{
    if (!h) return fail(KMC_E_ARG, "handle is NULL");
    if (warps_per_cta < 0 || warps_per_cta > 32)
        return fail(KMC_E_ARG, "warps_per_cta must be in [0, 32]");
    if (flush_steps < 0 || flush_steps > 1024)
        return fail(KMC_E_ARG, "flush_steps must be in [0, 1024]");
    h->warps_req = warps_per_cta;
    h->flush_req = flush_steps;
    return pick_launch(h);
}

int kmc_grad(kmc_handle *h, const double *dLoss_dJ, const double *dLoss_dZc, double grad_out[4],
             double stderr_out[4])
{
    if (!h || !grad_out) return fail(KMC_E_ARG, "handle or grad_out is NULL");
    if (h->P0site)
        return fail(KMC_E_ARG, "kmc_grad needs a scalar barrier (the handle has per-site Ea)");
    if (h->p.update_rule != 0)
        return fail(KMC_E_ARG, "kmc_grad follows the synchronous update (update_rule 0)");
    const kmc_params &p = h->p;
    const int64_t R = p.n_rails, L = p.n_sites, Z = p.n_zones, n = h->t;
    double out[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    cudaStream_t s = h->stream;
    if (n > 0 && (dLoss_dJ || dLoss_dZc)) {
        SweepArgs ga;
        int rc = grad_prepare(h, dLoss_dJ, dLoss_dZc, &ga);
        if (rc) return rc;
        SweepLaunch l = h->launch;
        int dev = 0, max_smem = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (max_smem <= 0) max_smem = 48 * 1024;
        max_smem = std::min(max_smem, 200 * 1024);
        int warps = 8;
        while (warps > 1 && grad_smem_bytes(l.lpr, l.wpl, (int)Z, (int)L, warps) > (size_t)max_smem)
            warps >>= 1;
        if (grad_smem_bytes(l.lpr, l.wpl, (int)Z, (int)L, warps) > (size_t)max_smem)
            return fail(KMC_E_ARG, "gradient pass: shared memory exceeds the device limit");
        l.warps = warps;
        l.smem = grad_smem_bytes(l.lpr, l.wpl, (int)Z, (int)L, warps);
        const int64_t rails_per_cta = (int64_t)(32 / l.lpr) * warps;
        l.grid = (int)((R + rails_per_cta - 1) / rails_per_cta);
        CK(grad_launch(ga, l, s), "gradient pass launch");
        rc = grad_reduce_out(h, out);
        if (rc) return rc;
        CK(cudaStreamSynchronize(s), "gradient pass");
    }
    grad_outputs(h, out, grad_out, stderr_out);
    return KMC_OK;
}

int kmc_set_accept_path(kmc_handle *h, int mode)
{
    if (!h) return fail(KMC_E_ARG, "handle is NULL");
    if (mode < -1 || mode > 1) return fail(KMC_E_ARG, "mode must be -1, 0 or 1");
    h->accept_req = mode;
    return pick_launch(h);
}

int kmc_accept_path(const kmc_handle *h) { return h ? h->launch.acc : -1; }

int64_t kmc_current_step(const kmc_handle *h) { return h ? h->t : -1; }

void kmc_destroy(kmc_handle *h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    h->release_all();
    delete h;
}

const char *kmc_last_error(void) { return g_err.c_str(); }

}  // extern "C"
