// kmc_internal.h -- device-side data structures shared by the kernels
// (kmc_sweep.cu, kmc_setup.cu) and the host runtime (kmc_capi.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kmc.h"

namespace kmc {

constexpr uint32_t kInitStep = 0xFFFFFFFFu;   // Philox step word of the placement stream
constexpr int kMaxZones = KMC_MAX_ZONES;
constexpr int kMaxSites = KMC_MAX_SITES;

// Per-device constants derived from kmc_params on the device (setup kernel):
// exact FP64 values used by the exact decision path and their FP32 images
// used by the bounded fast path.
struct DevConst {
    double P0;      // -expm1(-2 Gamma0 dt), Gamma0 = nu exp(-Ea / kT)   (Eq. 1)
    double E_in;    // E rho_e,        E = -expm1(-2 k_e dt)
    double E_out;   // E (1 - rho_e)
    double ka;      // kappa * alpha
    double kT;      // k_B T, k_B = 8.6173e-5 eV/K (Eq. 4)
    double d;       // hop distance
    double t_dev;   // L d
    double xs;      // -d / (t_dev kT): dV -> the exponent of Eq. 4 (fast FP64 band)
    double half_invL; // 0.5 / L
    float P0f, E_inf, E_outf, pad;
    int32_t status; // 0 ok, else a KMC_E_* code found while deriving
    int32_t pad2;
    int32_t bnd[kMaxZones + 1];  // zone boundaries floor(z L / Z), z = 0..Z
};

// Everything one sweep launch needs.  Passed by value (kernel parameter space).
struct SweepArgs {
    uint8_t *occ;              // [R][stride] occupancy bytes
    int64_t stride;            // bytes per rail (L rounded up to 16)
    int32_t R, L, Z, electrodes;
    uint32_t instance;
    uint32_t rail_base;        // global index of local rail 0 (Philox counter word 1, log)
    uint32_t rk0[10], rk1[10]; // Philox round keys (seed words plus Weyl increments)
    int64_t t0;                // absolute step of the first step of this launch
    int32_t n_steps;
    int32_t flush;             // steps between trace flushes
    const double *V;           // [n_steps_total]
    const int32_t *N0;         // [R] background (initial) ion count per rail
    const double *P0site;      // [R][L] or null
    const float *P0f;          // [R][L] P0site rounded to FP32, or null
    const float2 *P0bnd;       // [R][Z] (min, max) of P0site over the zone, or null
    const double2 *bgd;        // [R][Z] (N0 w_z / L, D'_z) in FP64 for the FP64 paths, or null
    const DevConst *K;
    const SweepArgs *self;     // copy of these arguments in device memory (rare paths)
    unsigned long long *J;     // [n_steps_total] int64 two's complement
    unsigned long long *Zc;    // [n_steps_total][Z]
    kmc_log_entry *log;
    unsigned long long *log_count;
    int64_t log_cap;
    unsigned long long *counters; // [3] philox blocks, exact decisions, moves
    long long *Jr;                // [R] per-rail net leftward crossings, accumulated, or null
    int32_t bnd[kMaxZones + 1];   // zone boundaries floor(z L / Z)
    int32_t wsum[kMaxZones + 1];  // w_{z-1} + w_z (w_{-1} = w_Z = 0)
    float cz[kMaxZones];          // ((b_z + b_{z+1}) - H / L) / (2 L), H = sum w_z (b_z + b_{z+1})
    float inv_L;                  // 1 / L
    float inv_LkT;                // 1 / (L kT)
    float ka_f;                   // kappa alpha
    float delta;                  // relative half-width of the FP32 probability band
    float P0f_scalar;             // scalar P0 in FP32 (host copy of DevConst::P0f)
    float E_inf, E_outf;          // electrode base probabilities in FP32
    int32_t rule;                 // 0 synchronous update, 1 brick-wall (even/odd bonds)

    // likelihood-ratio gradient pass only (unused by the forward sweep)
    // With the forward's totals J_t, Zc_t and the leave-one-out divisor R - 1,
    // a rail's baselined share of the observable's step-t terms is
    //   fJ = aJ J_rt - bJ,  aJ = wJ_t R / (R - 1),  bJ = wJ_t J_t / (R - 1),
    //   fZ = sum_z aZ_z N_rz - bZ,  aZ_z = wZ_tz R / (R - 1),  bZ = sum_z wZ_tz Zc_tz / (R - 1)
    // (aJ = wJ_t, bJ = 0 and the like when R == 1), precomputed on the host.
    const double *wJ;                    // [n_steps_total] weight of J_t, or null
    const double2 *fJab;                 // [n_steps_total] (aJ, bJ)
    const double *fZa;                   // [n_steps_total][Z] aZ, or null
    const double *fZb;                   // [n_steps_total] bZ
    const int32_t *fZr;                  // [n_steps_total] zones [lo, hi) that hold every
                                         // nonzero aZ of the step, as lo | hi << 8 (0: none)
    double *gstate;                      // [R][kGradState] per-rail accumulators
    double alpha;                        // space-charge volts per excess ion
    double tdev_kT;                      // t_dev kB T (d ln B / d kappa denominator)
    // exp(cm m) for the integer zone sums m = L (Pb_z + Pb_z+1) - F in [-etM, etM]
    // as etH[(m + etM) >> 10] * etL[(m + etM) & 1023], cm = kappa alpha / (2 L^2 kT)
    // (null: the gradient pass evaluates exp directly)
    const double *etL;                   // [1024]
    const double *etH;                   // [2 etM / 1024 + 1]
    int32_t etM;
    int32_t et_pad;
};

// Per-rail state of the gradient pass: cumulative inner-trial weight W (the
// Ea and nu scores are W times d ln P0 / d theta), cumulative kappa score K,
// and the estimator sums G_W, G_K, G_1 (the rho term is G_1 times the rail's
// initial-placement score).
constexpr int kGradState = 5;

// One work item of a batched launch: a tile of rails of one device.
struct BatchItem {
    int32_t inst;        // device index in the batch
    int32_t kind;        // kernel shape (shape_kind of the device's lanes per rail)
    int64_t tile_rail0;  // first rail of the tile
};

// Kernel shapes of the tile body: lanes per rail 1, 2, 4, 8, 16, 32 with one
// 32-bit word per lane (kinds 0-5), and 32 lanes of two words (kind 6).
constexpr int kShapeKinds = 7;
__host__ __device__ constexpr int shape_kind(int lpr, int wpl)
{
    return wpl == 2 ? 6 : lpr == 1 ? 0 : lpr == 2 ? 1 : lpr == 4 ? 2 : lpr == 8 ? 3 : lpr == 16 ? 4 : 5;
}

// Per-shape launches of a batch: CTAs and dynamic shared memory of each
// shape's persistent launch (grid 0: the batch has no items of that shape).
struct BatchPlan {
    int grid[kShapeKinds];
    size_t smem[kShapeKinds];
};

// Arguments of one batched launch.
struct BatchArgs {
    const SweepArgs *inst;   // [n_inst] per-device arguments (device memory)
    const BatchItem *items;  // [n_items] grouped by shape, longest tiles first in each
    int32_t cls_off[kShapeKinds + 1];  // items of shape k: [cls_off[k], cls_off[k + 1])
    int32_t n_items;
    int32_t n_steps;         // steps of this launch
    int32_t flush;           // steps between flushes of the warps' counters
    int32_t n_inst;          // devices
    int32_t max_z;           // the largest zone count of the devices
    int32_t pad2;
    unsigned *work;          // [kShapeKinds] next work item of each shape (reset by the
                             // advance kernel)
    const int64_t *t0;       // absolute step of the launch's first step
    int64_t *t0_mut;         // the same counter, advanced after the launch
    uint32_t rk0[10], rk1[10];
};

// Launch configuration chosen on the host.
struct SweepLaunch {
    int lpr;      // lanes per rail (1..32)
    int wpl;      // 32-bit words per lane (1 or 2)
    int warps;    // warps per CTA
    size_t smem;  // dynamic shared memory bytes
    int grid;
    int acc;      // 1: kernel with accept-sure tables and the inline accept path
};

// Automatic choice of the accept path: on when the scalar hop probability P0
// (Eq. 1 at the device's mean barrier) is at least this large.
constexpr double kAcceptAutoP0 = 1.0 / 128.0;

size_t sweep_smem_bytes(int lpr, int wpl, int Z, int L, int warps, int flush, bool acc);
int sweep_pick_lpr(int L, int *wpl);
cudaError_t sweep_launch(const SweepArgs &a, const SweepLaunch &l, cudaStream_t s);
// zone-count trace of steps [t0, t0 + n): per-step changes -> counts (after a sweep)
cudaError_t zone_scan(unsigned long long *Zc, int64_t t0, int n, int Z, cudaStream_t s);
cudaError_t sweep_set_smem_limits();
// gradient passes of a batch: one persistent launch per shape over its
// (device, tile) items, whose per-device arguments (b.inst) are gradient-pass
// arguments
cudaError_t batch_grad_launch(const BatchArgs &b, const BatchPlan &plan, int warps, cudaStream_t s);
// resident CTAs per SM of a shape's batched kernel (mode 0 forward, 1 forward
// with the accept path, 2 gradient pass) at this CTA size and shared memory
int batch_ctas_per_sm(int kind, int mode, int warps, size_t smem);
// Philox-only probe: grid CTAs of 256 threads, each thread 4 x iters blocks
cudaError_t philox_probe(int grid, int iters, uint32_t *sink, cudaStream_t s);
// gradient pass: shared memory of a launch, the launch, and the final sum
size_t grad_smem_bytes(int lpr, int wpl, int Z, int L, int warps);
cudaError_t grad_launch(const SweepArgs &a, const SweepLaunch &l, cudaStream_t s);
cudaError_t grad_reduce(const double *gstate, int64_t R, const int32_t *N0, int L, double fill,
                        int has_rho, double cEa, double cnu, double *out, cudaStream_t s);
int sweep_kind(int lpr, int wpl);
cudaError_t batch_set_smem_limit();
// launches the batched sweep (one launch per shape), the zone-count scans, and
// then advances *t0 by n_steps and re-arms the work counters
cudaError_t batch_launch(const BatchArgs &b, const BatchPlan &plan, int warps, bool acc,
                         cudaStream_t s);

// Sets the message returned by kmc_last_error() on this thread (kmc_capi.cu).
void kmc_internal_set_error(const char *msg);

// setup kernels (kmc_setup.cu)
cudaError_t setup_constants(const kmc_params &p, DevConst *K, cudaStream_t s);
cudaError_t setup_p0_table(const kmc_params &p, const double *Ea, double *P0, int64_t n, int *bad,
                           cudaStream_t s);
cudaError_t setup_p0_bounds(const double *P0, int32_t R, int32_t L, int32_t Z, const DevConst *K,
                            float2 *out, cudaStream_t s);
cudaError_t setup_p0_float(const double *P0, int64_t n, float *out, cudaStream_t s);
cudaError_t setup_row_counts(const uint8_t *occ, int64_t stride, int32_t R, int32_t L,
                             int32_t *N0, unsigned long long *bad, cudaStream_t s);
// bgd[r][z] = (N0[r] w_z / L in the oracle's FP64 order, D'_z): the background
// of zone z of rail r and its part of Q_z - Qbar (S2.1.8 reading)
cudaError_t setup_background(const int32_t *N0, int32_t R, int32_t L, int32_t Z, const DevConst *K,
                             double2 *bgd, cudaStream_t s);
cudaError_t setup_init_bernoulli(const kmc_params &p, uint8_t *occ, int64_t stride,
                                 cudaStream_t s);
// mode 0: count init keys <= key_bound; mode 1: keys == key_bound with linear index <= idx_bound
cudaError_t setup_count_keys(const kmc_params &p, uint64_t key_bound, int mode, int64_t idx_bound,
                             unsigned long long *count, cudaStream_t s);
cudaError_t setup_mark_smallest(const kmc_params &p, uint64_t key_star, int64_t idx_star,
                                int select_none, uint8_t *occ, int64_t stride, cudaStream_t s);
// exp(cm (j 1024 - M)) for j < nH into etH and exp(cm i) for i < 1024 into etL
cudaError_t setup_exp_tables(double cm, int32_t M, double *etL, double *etH, int32_t nH,
                             cudaStream_t s);

}  // namespace kmc
