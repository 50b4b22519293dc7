/*
 * kmc_oracle.h -- interface of the plain FP64 CPU oracle (test infrastructure
 * only; see kmc_oracle.c for the readings of the paper it implements).
 * This header belongs to the oracle alone; the CUDA path does not include it.
 */
#ifndef KMC_ORACLE_H
#define KMC_ORACLE_H

#include <stdint.h>

#define ORC_MAX_ZONES 32
/* step index of the initial-placement stream (never a simulated step) */
#define ORC_INIT_STEP 0xFFFFFFFFu

typedef struct {
    int32_t R;          /* rails */
    int32_t L;          /* sites per rail */
    int32_t Z;          /* zones (S2.1.5) */
    int32_t electrodes; /* 0 blocking, 1 injecting/extracting */
    double d;           /* hop distance d_hop (nm) */
    double dt;          /* time step (s) */
    double T;           /* temperature (K) */
    double Ea;          /* migration barrier (eV), Eq. 1 */
    double nu;          /* attempt frequency (Hz), Eq. 1 */
    double alpha;       /* volts per excess ion of the rail-local space charge */
    double kappa;       /* dimensionless coupling of the space-charge term */
    double k_e;         /* electrode exchange rate (Hz) */
    double rho_e;       /* reservoir density in [0, 1] */
    uint64_t seed;      /* Philox key */
    uint32_t instance;  /* fourth Philox counter word */
    int32_t rule;       /* 0 synchronous update (S2.1.7), 1 brick-wall (even/odd bonds) */
} orc_params;

typedef struct {
    int32_t rail;
    uint32_t step;
    int32_t site;
    int32_t dir;  /* 0 right trial, 1 left trial */
    int32_t kind; /* 0 inner hop, 1 injection, 2 extraction */
    int32_t pad;
    double diff;  /* u - p */
} orc_log_entry;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
int orc_zone_of(int k, int L, int Z);
void orc_zone_widths(int L, int Z, int32_t *w);
double orc_gamma0(double nu, double Ea, double T);
double orc_p0(double nu, double Ea, double T, double dt);
void orc_p0_table(const orc_params *P, const double *Ea_site, double *P0);
void orc_hop_probs(double base, double B, double inv, double *p_left, double *p_right);
void orc_zone_field(const orc_params *P, const int32_t *Nz, int32_t N0, double V, double *dV,
                    double *B, double *inv);
/* rail_ids (optional, Bernoulli mode only): global rail index of each local rail */
int orc_init_occupancy(const orc_params *P, int mode, int64_t n_ions, double fill,
                       const int32_t *rail_ids, uint8_t *occ);
/* rail_ids (optional): global rail index (Philox counter word 1) of each local
 * rail, so that a sample of a large device can be advanced on its own */
int orc_run(const orc_params *P, const double *V, int64_t t0, int64_t n_steps, uint8_t *occ,
            const int32_t *N0, const double *P0site, const int32_t *rail_ids, int64_t *J_out,
            int64_t *Zc_out, int64_t *J_rail, orc_log_entry *log, int64_t log_cap,
            int64_t *log_count, int nthreads);
int orc_max_threads(void);
/* Likelihood-ratio gradient (scalar barrier only) of the observable
 *     F = sum_s [ wJ[s] J_s + sum_z wZ[s][z] Zc_s[z] ]
 * over steps t0 .. t0 + n_steps - 1 (s relative to t0), replaying the run from
 * occ (rails 0 .. R-1, updated in place).  Per rail r it keeps the cumulative
 * score S_cum[r] = (d/dEa, d/dnu, d/dkappa, d/drho) log-probability of the
 * rail's trajectory so far (entry 3, the initial-placement score, is set by
 * the caller and left unchanged), and adds to G[r]
 *     (fZ_s - wJ[s] eta_rs) S_cum(before step s) + fJ_s S_cum(after step s),
 *     fJ_s = wJ[s] (J_rs - (J_tot[s] - J_rs) / (R - 1)),
 *     eta_rs = sum over the rail's left trials of (a - p) - same over right trials,
 *     fZ_s = sum_z wZ[s][z] (N_rz(s) - (Zc_tot[s][z] - N_rz(s)) / (R - 1)),
 * with the totals J_tot, Zc_tot of the same run (leave-one-out baselines;
 * none when R == 1).  The sum of G over rails estimates dE[F]/dtheta without
 * bias (the eta term is a control variate: eta_rs has zero mean given the
 * state at the start of step s, and S_cum before step s is fixed by then).  loglik[r] (optional) accumulates the log-probability of the same
 * trial outcomes under parameters Pe.  J_out (optional) receives J_s.
 *
 * Control-variate features (optional, cv_out non-NULL, cv_window >= 1): for
 * rail r, score entry e (0: Ea, 1: kappa), window k = s / cv_window and
 * feature f, cv_out[((r * 2 + e) * K + k) * F + f] (K = ceil(n_steps /
 * cv_window), F = Z + 2) accumulates psi_e(s) phi_f(s): psi_e(s) is the
 * rail-step's score increment of entry e, and phi(s) = (1, sum_k k occ[k] / L,
 * N_0 .. N_{Z-1}) is taken from the step-start occupancy.  psi has zero mean
 * given the step-start state, so every feature sum has zero mean, and any
 * combination of them with coefficients fixed independently of the rail can
 * be subtracted from the rail's term G without bias.  (The ν score is the Ea
 * score times a constant, so the Ea features serve it too.) */
int orc_run_lr(const orc_params *P, const orc_params *Pe, const double *V, int64_t t0,
               int64_t n_steps, uint8_t *occ, const int32_t *N0, const double *wJ,
               const double *wZ, const int64_t *J_tot, const int64_t *Zc_tot, double *S_cum,
               double *G, double *loglik, int64_t *J_out, int nthreads, int64_t cv_window,
               double *cv_out);

#endif
