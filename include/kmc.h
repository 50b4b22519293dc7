/*
 * kmc.h -- C ABI of the GB300 rail-based kinetic Monte Carlo ion-migration
 * sweep (arXiv 2511.09413).
 *
 * One simulated device ("instance") is a lattice of n_rails independent rails
 * of n_sites sites each (Supplementary S1.2, S2.1.1).  Every time step sweeps
 * every rail and site (S2.1.2 - S2.1.7): zone counts, the space-charge field
 * (S2.1.8), the energy gap of Eq. 3, the Boltzmann factor of Eq. 4, the hop
 * probabilities of Eqs. 5-6 (with the base probability from Eq. 1), two
 * uniforms per ion from a keyed Philox4x32-10 stream, exclusion, conflict
 * cancellation, electrode exchange, and the net-crossing current.
 *
 * Conventions shared by every entry point:
 *  - Return value: KMC_OK (0) on success, a negative KMC_E_* code otherwise.
 *    No exception crosses this boundary.  kmc_last_error() returns a
 *    human-readable message for the last failure on the calling thread.
 *  - Host pointers are plain CPU memory owned by the caller; they are read or
 *    written before the call returns unless stated otherwise.  Device memory
 *    is owned by the handle.
 *  - Occupancy layout: uint8 [n_rails][n_sites], row-major, values 0 or 1
 *    (site 0 is next to the electrode the cations drift to at V > 0).
 *  - Step indices are absolute: step t of a handle uses V[t] and Philox
 *    counter word 2 = t; kmc_step_n continues from the handle's current step.
 */
#ifndef KMC_H
#define KMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KMC_OK 0
#define KMC_E_ARG (-1)     /* invalid argument (size, range, null pointer) */
#define KMC_E_PROB (-2)    /* a derived probability is outside [0, 1] or not finite */
#define KMC_E_NOMEM (-3)   /* device allocation failed */
#define KMC_E_CUDA (-4)    /* a CUDA runtime call or kernel launch failed */
#define KMC_E_TIMEOUT (-5) /* a bounded device-side wait gave up */
#define KMC_E_RANGE (-6)   /* steps beyond the voltage table */

#define KMC_MAX_SITES 2048
#define KMC_MAX_ZONES 32

/* Physical and numerical parameters of one device (one instance).
 * Units: nm, s, K, eV, Hz, V.  See Table S1 for the paper's defaults. */
typedef struct kmc_params {
    int32_t n_rails;          /* R >= 1: rails (Table S1 dimension_y)                     */
    int32_t n_sites;          /* L in [2, 2048]: sites per rail (Table S1 dimension_x)      */
    int32_t n_zones;          /* Z in [1, min(L, 32)]: spatial zones (S2.1.5; paper uses 10)*/
    int32_t electrodes;       /* 0 blocking, 1 injecting/extracting                         */
    double site_spacing_nm;   /* d_hop of Eq. 3; the device thickness is t_dev = L d_hop     */
    double dt_s;              /* time step                                                   */
    double T_K;               /* temperature (Eqs. 1, 4)                                     */
    double Ea_eV;             /* migration barrier of Eq. 1 (used when no per-site table)    */
    double nu_Hz;             /* attempt frequency of Eq. 1                                  */
    double alpha_V;           /* space-charge volts per excess ion on a rail (S2.1.8)       */
    double kappa;             /* dimensionless space-charge coupling                         */
    double k_electrode_Hz;    /* electrode exchange rate (electrodes == 1)                   */
    double rho_electrode;     /* electrode reservoir density in [0, 1] (electrodes == 1)     */
    uint64_t seed;            /* Philox key: (seed & 0xffffffff, seed >> 32)                 */
    uint32_t instance;        /* Philox counter word 3                                       */
    int32_t init_mode;        /* 0: n_ions ions on the sites with the smallest init keys;
                                 1: Bernoulli(fill) per site; 2: caller occupancy            */
    int64_t n_ions;           /* init_mode 0                                                 */
    double fill;              /* init_mode 1                                                 */
    int32_t update_rule;      /* 0: the paper's synchronous update (S2.1.6-S2.1.7);
                                 1: brick-wall variant, not in the paper: at step t only
                                 bonds (b, b+1) with b = t mod 2 are active (the left
                                 electrode's bond is b = -1), each ion makes at most one
                                 trial, across its active bond, and no hops conflict    */
    int32_t rail_base;        /* global index of rail 0 of this device, >= 0 (default 0):
                                 rail r draws with Philox counter word 1 = rail_base + r
                                 and places its ions with that index, so a device of
                                 n_rails rails starting at rail_base advances exactly
                                 rows [rail_base, rail_base + n_rails) of a larger
                                 device with the same seed and instance (rails are
                                 independent, S1.2, S2.1.1).  rail_base + n_rails must
                                 not exceed 2^31 - 1; init_mode 0 needs rail_base 0   */
} kmc_params;

/* One decision whose uniform fell within 1e-12 of its threshold. */
typedef struct kmc_log_entry {
    int32_t rail;   /* global rail index: rail_base + the rail's row in the device */
    uint32_t step;
    int32_t site;
    int32_t dir;  /* 0 right trial, 1 left trial */
    int32_t kind; /* 0 inner hop, 1 injection, 2 extraction */
    int32_t pad;
    double diff;  /* u - p */
} kmc_log_entry;

typedef struct kmc_handle kmc_handle;

/* Optional device allocator (for example a framework's caching allocator).
 * alloc returns device memory of at least `bytes` usable on `stream`, or NULL.
 * free receives the pointer, its size and the stream it was used on.
 * Passing NULL functions restores the default (cudaMallocAsync/cudaFreeAsync).
 * Affects handles created afterwards.  Not thread-safe against kmc_create. */
typedef void *(*kmc_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*kmc_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
int kmc_set_allocator(kmc_alloc_fn alloc, kmc_free_fn free_fn, void *ctx);

/* Create a device: validates parameters, allocates device state on
 * `cuda_stream` (a cudaStream_t, NULL = legacy default stream), copies the
 * voltage table V_per_step[n_steps_total] (S2.2: protocol as V(t) table),
 * places ions (init_mode, S2.1.1; init_occ_or_null is read when init_mode is 2),
 * and, if Ea_site_or_null is given (double [R][L], eV), uses a per-site
 * barrier for hops leaving each site instead of Ea_eV.
 * Errors: KMC_E_ARG for bad sizes or values, KMC_E_PROB if P0 or the electrode
 * probabilities are not in [0, 1], KMC_E_NOMEM, KMC_E_CUDA.  On error *out is
 * NULL and nothing is leaked.  Synchronizes the stream before returning. */
int kmc_create(const kmc_params *params, const double *V_per_step, int64_t n_steps_total,
               const uint8_t *init_occ_or_null, const double *Ea_site_or_null,
               void *cuda_stream, kmc_handle **out);

/* Advance n_steps >= 0 steps from the handle's current step (asynchronous on
 * the handle's stream).  Each step is the synchronous sweep of S2.1.2 - S2.1.7
 * over every rail and site: zone counts (S2.1.5), the space-charge field
 * (S2.1.8) and the energy gap of Eq. 3, the Boltzmann factor of Eq. 4, the hop
 * probabilities of Eqs. 5-6 with the base probability from Eq. 1, two uniforms
 * per ion compared with "u <= p" (S2.1.6 - S2.1.7), exclusion against the
 * step-start occupancy, conflict cancellation, electrode exchange, and the
 * net-crossing current.  The occupancy and traces stay on the device.
 * KMC_E_RANGE if the voltage table is too short; KMC_E_CUDA if a launch fails. */
int kmc_step_n(kmc_handle *h, int64_t n_steps);

/* Read observables (synchronizes the stream):
 *  J_out[count]            net leftward bond crossings per step, all rails and
 *                          bonds including the electrode bonds (may be NULL):
 *                          the ionic current of each step, counted exactly as
 *                          the moves of S2.1.7 that cross a bond;
 *  zone_counts_out[count][Z] ions per zone at the start of each step, summed
 *                          over rails (may be NULL): with Z = 10 the deciles
 *                          whose ion fractions the paper converts to
 *                          conductance and current (S3: first decile at V > 0,
 *                          tenth at V < 0; zones as in S2.1.5);
 *  occ_out_or_null[R][L]   current occupancy (may be NULL).
 * Steps [first_step, first_step + count) must already have been simulated
 * (KMC_E_RANGE otherwise).  Host buffers are caller-owned. */
int kmc_observables(kmc_handle *h, int64_t first_step, int64_t count, int64_t *J_out,
                    int64_t *zone_counts_out, uint8_t *occ_out_or_null);

/* Per-rail current: J_rail_out[R] receives, for each rail of the device, its
 * net leftward bond crossings (electrode bonds included) summed over every
 * step simulated so far; the sum over rails of J_rail_out equals the sum of
 * kmc_observables' J_out over those steps.  Host buffer of n_rails int64,
 * caller-owned.  Synchronizes the stream.  Errors: KMC_E_ARG for NULL
 * arguments, KMC_E_CUDA. */
int kmc_rail_current(kmc_handle *h, int64_t *J_rail_out);

/* Overwrite V for steps [first_step, first_step + count) from host memory
 * (asynchronous copy on the handle's stream; the host buffer must stay valid
 * until the next synchronizing call). */
int kmc_set_voltage(kmc_handle *h, int64_t first_step, int64_t count, const double *V_host);

/* Copy up to `cap` near-threshold log entries (|u - p| < 1e-12) to `out` and
 * report the total number logged in *n_total (synchronizes). */
int kmc_near_threshold_log(kmc_handle *h, kmc_log_entry *out, int64_t cap, int64_t *n_total);

/* Device counters since creation: [0] Philox blocks drawn, [1] decisions
 * resolved by the exact FP64 path, [2] accepted moves (synchronizes). */
int kmc_counters(kmc_handle *h, uint64_t out[3]);

/* Launch shape: warps per CTA (1..32, 0 = automatic) and steps between the
 * warps' flushes of their counters and per-rail current (1..1024, 0 =
 * automatic; the traces are written as the steps run).  Results do not
 * depend on either. */
int kmc_set_launch(kmc_handle *h, int warps_per_cta, int flush_steps);

/* Accept path: mode 1 selects the kernel that also keeps accept-sure bounds
 * per zone and decides inner hops whose draw is not rejected outright inside
 * the draw loop (faster where P0 is of order 1e-2 or more), 0 the kernel
 * without them, -1 (the default) picks 1 when P0 at the device's Ea is at
 * least 1/128.  Results do not depend on the mode (every decision is still
 * u <= p in FP64, Eq. 5-6).  kmc_accept_path returns the mode in effect. */
int kmc_set_accept_path(kmc_handle *h, int mode);
int kmc_accept_path(const kmc_handle *h);

/* Likelihood-ratio gradient of an observable's expectation.  The paper's
 * method has no derivative; this is the score-function (likelihood-ratio)
 * estimator over the same stochastic dynamics (Eqs. 1, 3-6 give every trial's
 * probability p, S2.1.6-S2.1.7 its Bernoulli outcome a).  For the steps
 * 0 .. t-1 simulated so far (t = kmc_current_step) and the observable
 *     F = sum_s dLoss_dJ[s] J_s + sum_{s,z} dLoss_dZc[s][z] Zc_s[z]
 * (J, Zc as kmc_observables returns them), grad_out receives an unbiased
 * estimate of dE[F]/d(Ea_eV, nu_Hz, kappa, fill):
 *     sum over rails r, steps s of  f_rs * S_r(s),
 * where S_r(s) is the score of rail r's trajectory up to step s (the sum over
 * its performed trials of (a - p)/(1 - p) d ln p, plus d/dfill of the
 * Bernoulli placement) and f_rs is the rail's share of F's step-s term minus
 * the mean share of the other rails (a baseline that leaves the estimate
 * unbiased).  Zone counts, recorded at the start of step s, pair with the
 * score of steps < s; the current of step s with that of steps <= s, less
 * dLoss_dJ[s] eta_rs times the score of steps < s, where eta_rs (the sum over
 * the rail's left trials of a - p minus that over its right trials) is the
 * part of the rail's current that the step's own draws add: a control
 * variate of zero mean that removes most of the estimator's variance.
 * stderr_out (may be NULL) receives the standard error of each entry from the
 * spread of the independent per-rail terms.
 *
 * The backward pass replays the trajectory from the initial occupancy kept at
 * kmc_create (the Philox counters (site, rail, step, instance) are the only
 * other checkpoint) with every trial's outcome recomputed, and accumulates the
 * estimator in FP64 on the device; the forward state is not touched.
 *  dLoss_dJ    host double [t] or NULL;  dLoss_dZc  host double [t][Z] or NULL.
 * The fill entry is NaN unless the placement was Bernoulli(fill) (init_mode 1).
 * The Ea and nu entries refer to the scalar barrier: handles created with
 * per-site barriers are rejected (KMC_E_ARG).  Electrode exchange enters only
 * through kappa (rho_electrode and k_electrode_Hz are held fixed).  The first
 * call allocates the pass's buffers (an occupancy, R x 5 doubles, and weight
 * tables of n_steps_total entries).  Synchronizes the stream.
 * Errors: KMC_E_ARG, KMC_E_NOMEM, KMC_E_CUDA. */
int kmc_grad(kmc_handle *h, const double *dLoss_dJ, const double *dLoss_dZc, double grad_out[4],
             double stderr_out[4]);

/* Measurement aid: the GPU's throughput of Philox4x32-10 blocks as the sweep
 * draws them (same routine, the two words the draw loop consumes), with no
 * other work, in blocks per second; the integer-pipe ceiling of kmc_step_n.
 * Runs about 50 ms on cuda_stream (allocates a small buffer; synchronizes). */
int kmc_philox_probe(void *cuda_stream, double *blocks_per_s);

/* Current absolute step of the handle. */
int64_t kmc_current_step(const kmc_handle *h);

/* Release all device memory of the handle (synchronizes its stream). */
void kmc_destroy(kmc_handle *h);

/* Message of the last failure on this thread ("" if none). */
const char *kmc_last_error(void);

/* ---- Batches: many devices advanced by persistent launches.
 * A batch holds n_inst independent devices (each as kmc_create would make it,
 * with its own sizes, parameters, voltage table and occupancy) that advance
 * together.  Every chunk of steps covers all devices with one persistent
 * launch per tile shape (lanes per rail): its CTAs take (device, rail tile)
 * work items of that shape, longest tiles first, from a shared counter, so
 * devices of very different sizes keep the GPU full.  The launches of
 * steps_per_launch steps, the zone-count scans and the advance of the
 * batch's step counter are captured once as a CUDA graph and replayed.  Results per device are identical to kmc_step_n on that
 * device alone.  All devices share one seed (the Philox key) and are told
 * apart by their instance words (counter word 3); give them distinct ones.
 * V_per_step[i] is device i's host voltage table of n_steps_total entries;
 * init_occ_or_null may be NULL or hold NULL entries (for init_mode != 2);
 * Ea_site_or_null may be NULL or hold NULL entries, and a non-NULL entry i is
 * device i's per-site barrier table as kmc_create's Ea_site_or_null (host,
 * FP64 [n_rails][n_sites], copied).  Devices with per-site barriers advance
 * exactly as with kmc_create; their gradient passes are not available
 * (kmc_grad's scalar-barrier rule).  Errors as kmc_create. */
typedef struct kmc_batch kmc_batch;
int kmc_batch_create(const kmc_params *params, int32_t n_inst, const double *const *V_per_step,
                     int64_t n_steps_total, const uint8_t *const *init_occ_or_null,
                     const double *const *Ea_site_or_null, void *cuda_stream, kmc_batch **out);
/* Advance every device by n_steps (asynchronous on the batch's stream). */
int kmc_batch_step_n(kmc_batch *b, int64_t n_steps);
/* kmc_observables for device `inst` of the batch (synchronizes). */
int kmc_batch_observables(kmc_batch *b, int32_t inst, int64_t first_step, int64_t count,
                          int64_t *J_out, int64_t *zone_counts_out, uint8_t *occ_out_or_null);
/* kmc_rail_current for device `inst` of the batch (synchronizes). */
int kmc_batch_rail_current(kmc_batch *b, int32_t inst, int64_t *J_rail_out);
/* Launch shape: warps per CTA (1, 2, 4, 8) and steps per launch (graph size). */
int kmc_batch_set_launch(kmc_batch *b, int32_t warps_per_cta, int32_t steps_per_launch);
/* Autotuner: times every candidate launch shape (warps per CTA in {4, 8},
 * steps per launch in {64 ... 2048} up to probe_steps, and the accept path,
 * see below) on probe_steps real
 * steps from the current state, restores the state after each probe (the
 * simulation is unchanged), and keeps the fastest.  Synchronizes. */
int kmc_batch_tune(kmc_batch *b, int64_t probe_steps, int32_t *warps_out, int32_t *steps_out);
/* Accept path of the batch kernel (as kmc_set_accept_path; automatic mode
 * looks at the largest P0 of the batch).  With the automatic mode,
 * kmc_batch_tune also times the other kernel at the best shape and keeps it
 * when faster.  kmc_batch_accept_path returns the mode in effect. */
int kmc_batch_set_accept_path(kmc_batch *b, int32_t mode);
int kmc_batch_accept_path(const kmc_batch *b);
/* Likelihood-ratio gradient for device inst of the batch over the steps the
 * batch has simulated: as kmc_grad on that device (same arguments, same
 * estimator; the device's trajectory is replayed from its own initial
 * occupancy).  Synchronizes the batch's stream. */
int kmc_batch_grad(kmc_batch *b, int32_t inst, const double *dLoss_dJ, const double *dLoss_dZc,
                   double grad_out[4], double stderr_out[4]);
/* The gradient passes of every device of the batch, one persistent launch
 * per tile shape (the devices' rail tiles as work items, as the forward
 * batch).  For device
 * i, dLoss_dJ[i] and dLoss_dZc[i] are as kmc_grad's (either array of pointers,
 * or an entry, may be NULL); grad_out[i][4] and stderr_out[i][4] (may be NULL)
 * receive what kmc_grad would return for that device alone.  Synchronizes. */
int kmc_batch_grad_all(kmc_batch *b, const double *const *dLoss_dJ, const double *const *dLoss_dZc,
                       double *grad_out, double *stderr_out);
int64_t kmc_batch_current_step(const kmc_batch *b);
void kmc_batch_destroy(kmc_batch *b);

/* ---- Sweep without any device allocation.
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory: applications whose framework allocator owns
 * all of the GPU's memory and forbids side allocations, latency-bound loops
 * where cudaMalloc's implicit synchronisation is unacceptable, and services
 * that must keep the device footprint fixed after start-up.
 *
 * Advances n_steps steps, starting at absolute step t0, of a device whose
 * state is caller-owned device memory:
 *   occ_dev          uint8 [n_rails][row_stride] occupancy (0/1 in the first
 *                    n_sites bytes of each row; padding is rewritten as 0),
 *                    16-byte aligned, row_stride a multiple of 16, updated in place;
 *                    the bytes are not checked (checking would need a
 *                    synchronisation), and any byte other than 0 or 1 gives
 *                    undefined results;
 *   N0_dev_or_null   int32 [n_rails] background ion count per rail (the count at
 *                    the device's first step), or NULL to take it from occ_dev
 *                    at this call (right for a device's first call, and for any
 *                    call with blocking electrodes, where counts are conserved);
 *   V_dev            double [n_steps]: V of steps t0 .. t0 + n_steps - 1;
 *   J_dev            int64 [n_steps] output, as kmc_observables' J_out;
 *   zone_counts_dev  int64 [n_steps][n_zones] output, as zone_counts_out.
 * Only the scalar barrier Ea_eV is used (no per-site table); init_mode, n_ions
 * and fill are ignored; rail_base is honoured; the near-threshold log and the
 * per-rail current are not returned.  Results are identical to kmc_step_n on a
 * handle in the same state.
 *
 * Working memory is one static device array of about 4 MiB that every GPU
 * loading the library holds until the process exits; it limits n_rails to
 * KMC_NOALLOC_MAX_RAILS (larger sizes return KMC_E_ARG).  The first call on
 * a device looks up that array's device address and raises the kernels'
 * shared-memory limit (host-side, once per device).  All calls share
 * the array: calls that overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  The entry point zeroes
 * what has to start at zero (its counters, J_dev, zone_counts_dev) on
 * cuda_stream, calls no allocator, and is asynchronous.  Errors: KMC_E_ARG or
 * KMC_E_PROB before anything is launched, KMC_E_CUDA if a launch fails. */
#define KMC_NOALLOC_MAX_RAILS (1 << 20)
int kmc_sweep_noalloc(const kmc_params *params, uint8_t *occ_dev, int64_t row_stride,
                      const int32_t *N0_dev_or_null, const double *V_dev, int64_t t0,
                      int64_t n_steps, int64_t *J_dev, int64_t *zone_counts_dev,
                      void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* KMC_H */
