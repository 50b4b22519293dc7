// kmc_noalloc.cu -- kmc_sweep_noalloc: the sweep kernel driven from memory the
// caller already owns, for callers that cannot allocate device memory.
//
// The sweep needs a little working memory besides its inputs and outputs: the
// derived constants block, a device copy of the launch arguments, counters, a
// near-threshold log and the per-rail background ion count.  Here that memory
// is one file-scope __device__ array, so the entry point itself allocates
// nothing.  Every GPU that loads the library holds the array until the process
// exits.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <mutex>

#include "kmc_internal.h"

using namespace kmc;

namespace {

// Scratch layout (bytes): constants | argument copy | counters | log | N0[R].
constexpr size_t kOffConst = 0;
constexpr size_t kOffArgs = 256;
constexpr size_t kOffMisc = 2048;                 // 8 x uint64: [0] log count, [1..3] counters,
                                                  // [5] bytes of the occupancy that are not 0/1
constexpr size_t kOffLog = 2048 + 64;
constexpr int kLogCap = 64;
constexpr size_t kOffN0 = 8192;
constexpr int64_t kMaxRails = KMC_NOALLOC_MAX_RAILS;
constexpr size_t kScratchBytes = kOffN0 + sizeof(int32_t) * (size_t)kMaxRails;
static_assert(sizeof(DevConst) <= kOffArgs - kOffConst, "constants block too large");
static_assert(sizeof(SweepArgs) <= kOffMisc - kOffArgs, "argument copy too large");
static_assert(kOffLog + sizeof(kmc_log_entry) * kLogCap <= kOffN0, "log too large");

__device__ __align__(256) static unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};  // device address of g_scratch, per device

int fail(int code, const char *msg)
{
    kmc_internal_set_error(msg);
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
    kmc_internal_set_error(buf);
    return e == cudaErrorMemoryAllocation ? KMC_E_NOMEM : KMC_E_CUDA;
}

// Device address of the scratch array for the current device; the first call
// on a device looks it up (and raises the kernels' shared-memory limit).
int scratch_for_current_device(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(KMC_E_ARG, "device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        e = sweep_set_smem_limits();
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
        g_scratch_addr[dev] = ptr;
    }
    *out = (unsigned char *)g_scratch_addr[dev];
    return KMC_OK;
}

bool finite_pos(double x) { return isfinite(x) && x > 0.0; }

// Writes the launch arguments into the scratch array from the kernel's own
// parameter space, so that no host buffer has to outlive the call (a copy
// from host memory would read the caller's stack frame when it executes).
__global__ void store_args_kernel(const SweepArgs a, SweepArgs *dst)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *dst = a;
}

}  // namespace

extern "C" int kmc_sweep_noalloc(const kmc_params *p, uint8_t *occ_dev, int64_t row_stride,
                                 const int32_t *N0_dev_or_null, const double *V_dev, int64_t t0,
                                 int64_t n_steps, int64_t *J_dev, int64_t *zone_counts_dev,
                                 void *cuda_stream)
{
    // ---- host-side checks (nothing is launched on a failed check)
    if (!p) return fail(KMC_E_ARG, "params is NULL");
    if (p->n_rails < 1 || p->n_rails > kMaxRails)
        return fail(KMC_E_ARG, "kmc_sweep_noalloc: n_rails must be in [1, KMC_NOALLOC_MAX_RAILS]");
    if (p->n_sites < 2 || p->n_sites > KMC_MAX_SITES)
        return fail(KMC_E_ARG, "n_sites must be in [2, 2048]");
    if (p->n_zones < 1 || p->n_zones > KMC_MAX_ZONES || p->n_zones > p->n_sites)
        return fail(KMC_E_ARG, "n_zones must be in [1, min(n_sites, 32)]");
    if (p->electrodes != 0 && p->electrodes != 1) return fail(KMC_E_ARG, "electrodes must be 0 or 1");
    if (p->update_rule != 0 && p->update_rule != 1) return fail(KMC_E_ARG, "update_rule must be 0 or 1");
    if (p->rail_base < 0 || (int64_t)p->rail_base + p->n_rails > (int64_t)INT32_MAX)
        return fail(KMC_E_ARG, "rail_base must be >= 0 with rail_base + n_rails <= 2^31 - 1");
    if (!finite_pos(p->site_spacing_nm) || !finite_pos(p->dt_s) || !finite_pos(p->T_K))
        return fail(KMC_E_ARG, "site_spacing_nm, dt_s and T_K must be > 0");
    if (!(isfinite(p->nu_Hz) && p->nu_Hz >= 0.0) || !isfinite(p->Ea_eV) || !isfinite(p->alpha_V) ||
        !isfinite(p->kappa))
        return fail(KMC_E_ARG, "nu_Hz, Ea_eV, alpha_V and kappa must be finite (nu_Hz >= 0)");
    if (p->electrodes == 1 && (!(isfinite(p->k_electrode_Hz) && p->k_electrode_Hz >= 0.0) ||
                               !(p->rho_electrode >= 0.0 && p->rho_electrode <= 1.0)))
        return fail(KMC_E_ARG, "k_electrode_Hz must be >= 0 and rho_electrode in [0, 1]");
    if (t0 < 0 || n_steps < 0 || t0 + n_steps >= (int64_t)kInitStep)
        return fail(KMC_E_ARG, "steps must satisfy 0 <= t0, 0 <= n_steps, t0 + n_steps < 2^32 - 1");
    if (row_stride < p->n_sites || row_stride % 16 != 0)
        return fail(KMC_E_ARG, "row_stride must be a multiple of 16 and >= n_sites");
    if (!occ_dev || ((uintptr_t)occ_dev & 15u) != 0)
        return fail(KMC_E_ARG, "occ_dev must be a 16-byte aligned device pointer");
    if (n_steps > 0 && (!V_dev || !J_dev || !zone_counts_dev))
        return fail(KMC_E_ARG, "V_dev, J_dev and zone_counts_dev are required when n_steps > 0");
    // derived probabilities (Eq. 1 and the electrode exchange), checked on the host
    const double kT = 8.6173e-5 * p->T_K;
    const double P0 = -expm1(-(2.0 * (p->nu_Hz * exp(-p->Ea_eV / kT)) * p->dt_s));
    const double E = -expm1(-(2.0 * p->k_electrode_Hz * p->dt_s));
    const double E_in = E * p->rho_electrode, E_out = E * (1.0 - p->rho_electrode);
    if (!(P0 >= 0.0 && P0 <= 1.0) ||
        (p->electrodes == 1 && !(E_in >= 0.0 && E_in <= 1.0 && E_out >= 0.0 && E_out <= 1.0)))
        return fail(KMC_E_PROB, "derived probability outside [0, 1]");
    if (n_steps == 0) return KMC_OK;

    unsigned char *scr = nullptr;
    int rc = scratch_for_current_device(&scr);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    DevConst *K = (DevConst *)(scr + kOffConst);
    SweepArgs *args_dev = (SweepArgs *)(scr + kOffArgs);
    unsigned long long *misc = (unsigned long long *)(scr + kOffMisc);
    kmc_log_entry *log = (kmc_log_entry *)(scr + kOffLog);
    int32_t *N0s = (int32_t *)(scr + kOffN0);

    const int R = p->n_rails, L = p->n_sites, Z = p->n_zones;
    cudaError_t e;
    // counters and outputs start at zero (the kernel accumulates into them)
    if ((e = cudaMemsetAsync(misc, 0, 8 * sizeof(unsigned long long), s)) != cudaSuccess)
        return cuda_fail(e, "cudaMemsetAsync");
    if ((e = cudaMemsetAsync(J_dev, 0, sizeof(int64_t) * (size_t)n_steps, s)) != cudaSuccess)
        return cuda_fail(e, "cudaMemsetAsync");
    if ((e = cudaMemsetAsync(zone_counts_dev, 0, sizeof(int64_t) * (size_t)n_steps * Z, s)) !=
        cudaSuccess)
        return cuda_fail(e, "cudaMemsetAsync");
    if ((e = setup_constants(*p, K, s)) != cudaSuccess) return cuda_fail(e, "constants launch");
    const int32_t *N0 = N0_dev_or_null;
    if (!N0) {
        if ((e = setup_row_counts(occ_dev, row_stride, R, L, N0s, misc + 5, s)) != cudaSuccess)
            return cuda_fail(e, "row counts launch");
        N0 = N0s;
    }

    // ---- launch arguments (same derivation as for a handle)
    SweepArgs a;
    memset(&a, 0, sizeof(a));
    a.occ = occ_dev;
    a.stride = row_stride;
    a.R = R;
    a.L = L;
    a.Z = Z;
    a.electrodes = p->electrodes;
    a.instance = p->instance;
    a.rail_base = (uint32_t)p->rail_base;
    uint32_t k0 = (uint32_t)(p->seed & 0xffffffffu), k1 = (uint32_t)(p->seed >> 32);
    for (int i = 0; i < 10; ++i) {
        a.rk0[i] = k0;
        a.rk1[i] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    // the kernel indexes V and the traces by absolute step; the caller's arrays
    // start at step t0
    a.t0 = t0;
    a.n_steps = (int32_t)std::min<int64_t>(n_steps, 1 << 30);
    a.V = V_dev - t0;
    a.N0 = N0;
    a.K = K;
    a.self = args_dev;
    a.J = (unsigned long long *)J_dev - t0;
    a.Zc = (unsigned long long *)zone_counts_dev - t0 * Z;
    a.log = log;
    a.log_count = misc;
    a.log_cap = kLogCap;
    a.counters = misc + 1;
    a.Jr = nullptr;     // no per-rail current on this path
    a.bgd = nullptr;    // no background table: undecided draws take the exact path
    int bnd[KMC_MAX_ZONES + 1];
    for (int z = 0; z <= Z; ++z) bnd[z] = (int)(((int64_t)z * L) / Z);
    for (int z = 0; z <= KMC_MAX_ZONES; ++z) a.bnd[z] = z <= Z ? bnd[z] : L;
    double H = 0.0;
    for (int z = 0; z < Z; ++z) H += (double)(bnd[z + 1] - bnd[z]) * (double)(bnd[z] + bnd[z + 1]);
    for (int z = 0; z <= KMC_MAX_ZONES; ++z) {
        const int w_prev = (z >= 1 && z <= Z) ? bnd[z] - bnd[z - 1] : 0;
        const int w_cur = (z < Z) ? bnd[z + 1] - bnd[z] : 0;
        a.wsum[z] = w_prev + w_cur;
    }
    for (int z = 0; z < KMC_MAX_ZONES; ++z)
        a.cz[z] = z < Z ? (float)(((double)(bnd[z] + bnd[z + 1]) - H / L) / (2.0 * L)) : 0.0f;
    a.inv_L = (float)(1.0 / L);
    a.inv_LkT = (float)(1.0 / ((double)L * kT));
    a.ka_f = (float)(p->kappa * p->alpha_V);
    a.delta = 1.0f / 1024.0f;
    a.rule = p->update_rule;
    // FP32 images of the base probabilities; the band factors absorb their rounding
    a.P0f_scalar = (float)P0;
    a.E_inf = (float)E_in;
    a.E_outf = (float)E_out;

    // ---- launch shape: as many warps per CTA (up to 8) as shared memory allows
    SweepLaunch l{};
    l.lpr = sweep_pick_lpr(L, &l.wpl);
    int dev = 0, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (max_smem <= 0) max_smem = 48 * 1024;
    max_smem = std::min(max_smem, 200 * 1024);
    int warps = 8, flush = 256;
    l.acc = P0 >= kAcceptAutoP0 ? 1 : 0;
    const bool acc = l.acc != 0;
    while (warps > 1 &&
           sweep_smem_bytes(l.lpr, l.wpl, Z, L, warps, flush, acc) > (size_t)max_smem)
        warps >>= 1;
    while (flush > 1 &&
           sweep_smem_bytes(l.lpr, l.wpl, Z, L, warps, flush, acc) > (size_t)max_smem)
        flush >>= 1;
    l.warps = warps;
    l.smem = sweep_smem_bytes(l.lpr, l.wpl, Z, L, warps, flush, acc);
    const int64_t rails_per_cta = (int64_t)(32 / l.lpr) * warps;
    l.grid = (int)((R + rails_per_cta - 1) / rails_per_cta);
    a.flush = flush;

    store_args_kernel<<<1, 32, 0, s>>>(a, args_dev);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "argument store launch");
    int64_t left = n_steps;
    while (left > 0) {
        const int64_t n = std::min<int64_t>(left, 1 << 30);
        a.n_steps = (int32_t)n;
        if ((e = sweep_launch(a, l, s)) != cudaSuccess) return cuda_fail(e, "sweep launch");
        if ((e = zone_scan(a.Zc, a.t0, (int)n, Z, s)) != cudaSuccess)
            return cuda_fail(e, "zone-count scan launch");
        a.t0 += n;
        left -= n;
    }
    return KMC_OK;
}
