/*
 * kmc_oracle.c -- plain FP64 CPU oracle of the rail-based kinetic Monte Carlo
 * ion-migration step (arXiv 2511.09413, Supplementary Information S2.1).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and
 * bench.py's CPU-baseline leg and reference arm (--impl reference) may load
 * this library.  It shares no code, header, table or constant generator with
 * the CUDA path.
 *
 * Parity unpinned: the magnitude of the space-charge coupling (alpha, kappa
 * below).  The paper prints no value or figure data that fixes it; its
 * structure (zero for a uniform rail, the Dirichlet constraint, the discrete
 * Gauss law, mirror symmetry, the sign of the response) is pinned.
 *
 * The method is a stochastic iteration, so the oracle is the algorithm itself
 * written out step by step: one loop per step, per rail, per site, in FP64,
 * in the order of S2.1.2 - S2.1.7.  It is compiled with -ffp-contract=off so
 * that every FP64 operation is a single IEEE-rounded operation.
 *
 * Readings of the paper used here (the paper is silent on these points):
 *  - state: occupancy occ[r][k] in {0,1} instead of the ion-indexed matrix X
 *    of S2.1.5; equivalent because ions never pass each other.
 *  - zone of site k (0-based): z = ceil((k+1) Z / L) - 1   (S2.1.5 with X = k+1).
 *  - space charge (S2.1.8, "Mapping to the code" in Sec. 3): rail-local,
 *    zone-coarse-grained 1-D Gauss law with a fixed anion background equal to
 *    the rail's initial ion count N0 and Dirichlet electrodes:
 *        C_z = N_z - N0 w_z / L,  Q_z = sum_{z'<z} C_z' + C_z / 2,
 *        Qbar = sum_z w_z Q_z / L,  dV_z = V - kappa alpha (Q_z - Qbar).
 *  - Eq. 3 with q = 1 e and t_dev = L d:  dE_z = dV_z d / t_dev  (eV).
 *  - P0 = 1 - exp(-2 Gamma0 dt) with Gamma0 from Eq. 1, so that
 *    p_left = p_right = P0/2 ~ Gamma0 dt at zero bias.
 *  - draws: Philox4x32-10 (Salmon et al., SC'11), key = (seed lo, seed hi),
 *    counter = (site, rail, step, instance); u = (53 high bits of the 64-bit
 *    word pair) * 2^-53; accept iff u <= p (S2.1.7).
 *  - exclusion is tested against the step-start occupancy; an ion whose two
 *    trials both succeed stays (X + M_right - M_left = X); two ions entering
 *    the same empty site are both cancelled.
 *  - electrodes: blocking (no hop out of the lattice) or open: extraction is
 *    an outward hop with base probability E_out = E (1 - rho_e), injection into
 *    an empty boundary site uses that site's own draw with base probability
 *    E_in = E rho_e, E = 1 - exp(-2 k_e dt); the Boltzmann split of Eqs. 5-6
 *    is applied to both, exactly as to an inner hop.
 *  - current J_t = (number of leftward bond crossings) - (rightward), over all
 *    bonds of all rails including the two electrode bonds.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "kmc_oracle.h"

/* Boltzmann constant in eV/K exactly as printed next to Eq. 4. */
static const double ORC_KB = 8.6173e-5;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies, the    */
/* high halves xor-ed with the other two counter words and the round key;   */
/* the key is bumped by the Weyl constants between rounds.                  */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t prod0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* The two uniforms of one site and step: u_right from words (x1:x0), u_left
 * from words (x3:x2), each the 53 high bits of the 64-bit pair times 2^-53. */
static void site_uniforms(const orc_params *P, uint32_t site, uint32_t rail, uint32_t step,
                          double *u_right, double *u_left)
{
    uint32_t ctr[4] = {site, rail, step, P->instance};
    uint32_t key[2] = {(uint32_t)(P->seed & 0xffffffffu), (uint32_t)(P->seed >> 32)};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    uint64_t wr = ((uint64_t)x[1] << 32) | x[0];
    uint64_t wl = ((uint64_t)x[3] << 32) | x[2];
    *u_right = (double)(wr >> 11) * 0x1.0p-53;
    *u_left = (double)(wl >> 11) * 0x1.0p-53;
}

/* ------------------------------------------------------------------------ */
/* Zones (S2.1.5): Z equal-width zones, z = ceil(X / (L/Z)) with X = k + 1.  */
/* ------------------------------------------------------------------------ */
int orc_zone_of(int k, int L, int Z)
{
    /* ceil((k+1) Z / L) - 1 in integer arithmetic */
    return (int)(((int64_t)(k + 1) * Z + L - 1) / L) - 1;
}

void orc_zone_widths(int L, int Z, int32_t *w)
{
    for (int z = 0; z < Z; ++z) w[z] = 0;
    for (int k = 0; k < L; ++k) w[orc_zone_of(k, L, Z)] += 1;
}

/* ------------------------------------------------------------------------ */
/* Eq. 1 and the base hop probability P0.                                    */
/* ------------------------------------------------------------------------ */
double orc_gamma0(double nu, double Ea, double T)
{
    double kT = ORC_KB * T;
    return nu * exp(-Ea / kT); /* Eq. 1 */
}

double orc_p0(double nu, double Ea, double T, double dt)
{
    double g = orc_gamma0(nu, Ea, T);
    double x = 2.0 * g * dt;
    return -expm1(-x);
}

void orc_p0_table(const orc_params *P, const double *Ea_site, double *P0)
{
    int64_t n = (int64_t)P->R * P->L;
    for (int64_t i = 0; i < n; ++i) P0[i] = orc_p0(P->nu, Ea_site[i], P->T, P->dt);
}

/* ------------------------------------------------------------------------ */
/* Space-charge field per zone (S2.1.8) and Eqs. 3-4 plus 1/(1+B).          */
/* ------------------------------------------------------------------------ */
/* Enclosed charge of zone z relative to its rail mean, Q_z - Qbar (S2.1.8). */
static void zone_charge(const orc_params *P, const int32_t *Nz, int32_t N0, double *dq)
{
    const int L = P->L, Z = P->Z;
    int32_t w[ORC_MAX_ZONES];
    double C[ORC_MAX_ZONES], Q[ORC_MAX_ZONES];
    orc_zone_widths(L, Z, w);
    /* excess ions per zone over the fixed background N0 w_z / L */
    for (int z = 0; z < Z; ++z) C[z] = (double)Nz[z] - ((double)N0 * (double)w[z]) / (double)L;
    /* charge enclosed up to the middle of zone z */
    double run = 0.0;
    for (int z = 0; z < Z; ++z) {
        Q[z] = run + 0.5 * C[z];
        run = run + C[z];
    }
    /* Dirichlet constraint: the field averages to V / L over the rail */
    double acc = 0.0;
    for (int z = 0; z < Z; ++z) acc = acc + (double)w[z] * Q[z];
    double Qbar = acc / (double)L;
    for (int z = 0; z < Z; ++z) dq[z] = Q[z] - Qbar;
}

void orc_zone_field(const orc_params *P, const int32_t *Nz, int32_t N0, double V,
                    double *dV, double *B, double *inv)
{
    const int L = P->L, Z = P->Z;
    double dq[ORC_MAX_ZONES];
    zone_charge(P, Nz, N0, dq);
    double ka = P->kappa * P->alpha;
    double kT = ORC_KB * P->T;
    double t_dev = (double)L * P->d;
    for (int z = 0; z < Z; ++z) {
        dV[z] = V - ka * dq[z];
        double dE = (dV[z] * P->d) / t_dev;   /* Eq. 3, q = 1 e */
        B[z] = exp(-dE / kT);                 /* Eq. 4 */
        inv[z] = 1.0 / (1.0 + B[z]);          /* Eqs. 5-6 denominator */
    }
}

/* Eqs. 5-6: left and right hop probabilities from a base probability and the
 * zone's Boltzmann factor; p_right / p_left = B and p_left + p_right = base. */
void orc_hop_probs(double base, double B, double inv, double *p_left, double *p_right)
{
    *p_left = base * inv;     /* Eq. 5 */
    *p_right = *p_left * B;   /* Eq. 6 */
}

/* ------------------------------------------------------------------------ */
/* Initial occupancy (S2.1.1): uniform random placement from the init       */
/* stream, counter (site, rail, 0xFFFFFFFF, instance).                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t key;
    int64_t idx;
} orc_keyed;

static int keyed_cmp(const void *a, const void *b)
{
    const orc_keyed *x = (const orc_keyed *)a, *y = (const orc_keyed *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

static uint64_t init_key(const orc_params *P, uint32_t site, uint32_t rail)
{
    uint32_t ctr[4] = {site, rail, ORC_INIT_STEP, P->instance};
    uint32_t key[2] = {(uint32_t)(P->seed & 0xffffffffu), (uint32_t)(P->seed >> 32)};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    return ((uint64_t)x[1] << 32) | x[0];
}

int orc_init_occupancy(const orc_params *P, int mode, int64_t n_ions, double fill,
                       const int32_t *rail_ids, uint8_t *occ)
{
    const int R = P->R, L = P->L;
    const int64_t n = (int64_t)R * L;
    if (mode == 0) {
        if (rail_ids) return -1; /* the exact count is defined over the whole device */
        /* exactly n_ions ions on the sites with the smallest init keys */
        if (n_ions < 0 || n_ions > n) return -1;
        orc_keyed *all = (orc_keyed *)malloc((size_t)n * sizeof(orc_keyed));
        if (!all) return -2;
        for (int r = 0; r < R; ++r)
            for (int k = 0; k < L; ++k) {
                all[(int64_t)r * L + k].key = init_key(P, (uint32_t)k, (uint32_t)r);
                all[(int64_t)r * L + k].idx = (int64_t)r * L + k;
            }
        qsort(all, (size_t)n, sizeof(orc_keyed), keyed_cmp);
        memset(occ, 0, (size_t)n);
        for (int64_t i = 0; i < n_ions; ++i) occ[all[i].idx] = 1;
        free(all);
        return 0;
    }
    if (mode == 1) {
        /* independent Bernoulli(fill) per site */
        for (int r = 0; r < R; ++r)
            for (int k = 0; k < L; ++k) {
                uint32_t rail = rail_ids ? (uint32_t)rail_ids[r] : (uint32_t)r;
                double u = (double)(init_key(P, (uint32_t)k, rail) >> 11) * 0x1.0p-53;
                occ[(int64_t)r * L + k] = (u < fill) ? 1 : 0;
            }
        return 0;
    }
    return -1;
}

/* ------------------------------------------------------------------------ */
/* One synchronous step of one rail (S2.1.2 - S2.1.7).                       */
/* ------------------------------------------------------------------------ */
static void log_near(orc_log_entry *log, int64_t cap, int64_t *count, int32_t rail, uint32_t step,
                     int32_t site, int32_t dir, int32_t kind, double diff)
{
    int64_t slot;
#ifdef _OPENMP
#pragma omp atomic capture
#endif
    slot = (*count)++;
    if (log && slot < cap) {
        log[slot].rail = rail;
        log[slot].step = step;
        log[slot].site = site;
        log[slot].dir = dir;
        log[slot].kind = kind;
        log[slot].diff = diff;
    }
}

/* decision u <= p with near-threshold logging (|u - p| < 1e-12) */
static int trial(double u, double p, orc_log_entry *log, int64_t cap, int64_t *count,
                 int32_t rail, uint32_t step, int32_t site, int32_t dir, int32_t kind)
{
    double diff = u - p;
    if (fabs(diff) < 1e-12) log_near(log, cap, count, rail, step, site, dir, kind, diff);
    return u <= p;
}

/* ------------------------------------------------------------------------ */
/* Likelihood-ratio score of the trials of one rail-step (not part of the    */
/* paper's method: the derivative of the log-probability of the trajectory   */
/* that a likelihood-ratio gradient of an observable needs).  Every trial is  */
/* a Bernoulli(p) draw, so its outcome a contributes                         */
/*     a d ln p + (1 - a) d ln(1 - p)  =  (a - p) / (1 - p) * d ln p         */
/* with, for p = base B^s / (1 + B) (s = 1 right, 0 left, Eqs. 5-6):          */
/*     d ln p / d kappa = (s - B / (1 + B)) d ln B / d kappa,                */
/*     d ln B / d kappa = alpha (Q_z - Qbar) d / (t_dev kB T)    (Eqs. 3-4), */
/* and for an inner hop (base P0 = 1 - exp(-x), x = 2 nu exp(-Ea/kT) dt):     */
/*     d ln P0 / d Ea = -(x / kT) exp(-x) / P0,                              */
/*     d ln P0 / d nu = (x / nu) exp(-x) / P0.                               */
/* Electrode trials do not depend on Ea or nu.  The accumulator also sums   */
/* the innovation of the step's current, eta = sum over left trials of      */
/* (a - p) minus the same over right trials (zero mean given the step-start */
/* state), and the log-probability of the same outcomes under a second     */
/* parameter set Pe (for checking the derivatives by differences).          */
/* ------------------------------------------------------------------------ */
typedef struct {
    const orc_params *Pe;
    double dlnP0[2];                         /* d ln P0 / d Ea, d ln P0 / d nu at P */
    double P0e, Ein_e, Eout_e;               /* base probabilities at Pe */
    double inv[ORC_MAX_ZONES], c[ORC_MAX_ZONES];      /* 1/(1+B), d ln B / d kappa at P */
    double Be[ORC_MAX_ZONES], inve[ORC_MAX_ZONES];    /* B, 1/(1+B) at Pe */
    double s[3];                             /* score of the rail-step: Ea, nu, kappa */
    double ll;                               /* log-probability at Pe */
    double eta;                              /* innovation of the step's current */
    int32_t Nz[ORC_MAX_ZONES];               /* zone counts of the step-start occupancy */
} orc_trial_acc;

static void acc_begin(orc_trial_acc *a, const orc_params *P, const int32_t *Nz, int32_t N0,
                      double V, const double *inv)
{
    const int Z = P->Z;
    double dq[ORC_MAX_ZONES], dVe[ORC_MAX_ZONES];
    zone_charge(P, Nz, N0, dq);
    const double kT = ORC_KB * P->T;
    const double t_dev = (double)P->L * P->d;
    for (int z = 0; z < Z; ++z) {
        a->inv[z] = inv[z];
        a->c[z] = (P->alpha * dq[z] * P->d) / (t_dev * kT);
        a->Nz[z] = Nz[z];
    }
    orc_zone_field(a->Pe, Nz, N0, V, dVe, a->Be, a->inve);
    a->s[0] = a->s[1] = a->s[2] = 0.0;
    a->ll = 0.0;
    a->eta = 0.0;
}

static void acc_trial(orc_trial_acc *a, int z, int dir, int kind, double p, int hit)
{
    const double w = (p < 1.0) ? ((double)hit - p) / (1.0 - p) : 1.0;
    const double dk = dir == 0 ? a->inv[z] * a->c[z] : -(1.0 - a->inv[z]) * a->c[z];
    if (kind == 0) {
        a->s[0] += w * a->dlnP0[0];
        a->s[1] += w * a->dlnP0[1];
    }
    a->s[2] += w * dk;
    /* a left trial that succeeds is a leftward crossing (+1 in J), a right one -1 */
    a->eta += dir == 1 ? ((double)hit - p) : -((double)hit - p);
    const double base = kind == 0 ? a->P0e : (kind == 1 ? a->Ein_e : a->Eout_e);
    double pl, pr;
    orc_hop_probs(base, a->Be[z], a->inve[z], &pl, &pr);
    const double pe = dir == 0 ? pr : pl;
    a->ll += hit ? log(pe) : log1p(-pe);
}

static void rail_step(const orc_params *P, int r, uint32_t t, double V, uint8_t *occ, int32_t N0,
                      const double *P0row, double P0scalar, double E_in, double E_out,
                      int8_t *mvR, int8_t *mvL, uint8_t *next, int64_t *J_acc, int64_t *zc_acc,
                      orc_log_entry *log, int64_t cap, int64_t *count, orc_trial_acc *acc)
{
    const int L = P->L, Z = P->Z;
    const int open = P->electrodes == 1;
    if (L < 2) return;
    int32_t Nz[ORC_MAX_ZONES];
    double dV[ORC_MAX_ZONES], B[ORC_MAX_ZONES], inv[ORC_MAX_ZONES];

    /* zone counts of the step-start occupancy */
    for (int z = 0; z < Z; ++z) Nz[z] = 0;
    for (int k = 0; k < L; ++k)
        if (occ[k]) Nz[orc_zone_of(k, L, Z)] += 1;
    for (int z = 0; z < Z; ++z) zc_acc[z] += Nz[z];

    /* field, Eq. 3, Eq. 4 per zone */
    orc_zone_field(P, Nz, N0, V, dV, B, inv);
    if (acc) acc_begin(acc, P, Nz, N0, V, inv);

    /* trials (S2.1.6 - S2.1.7) */
    int injR = 0, injL = 0; /* injection into site 0 / site L-1 */
    for (int k = 0; k < L; ++k) {
        mvR[k] = 0;
        mvL[k] = 0;
        const int z = orc_zone_of(k, L, Z);
        double uR, uL;
        if (occ[k]) {
            int okR = (k + 1 < L) ? (occ[k + 1] == 0) : open;
            int okL = (k - 1 >= 0) ? (occ[k - 1] == 0) : open;
            if (!okR && !okL) continue;
            site_uniforms(P, (uint32_t)k, (uint32_t)r, t, &uR, &uL);
            double P0k = P0row ? P0row[k] : P0scalar;
            double pL, pR, eL, eR;
            orc_hop_probs(P0k, B[z], inv[z], &pL, &pR);
            orc_hop_probs(E_out, B[z], inv[z], &eL, &eR);
            int kindR = 0, kindL = 0;
            if (k == L - 1 && open) {      /* extraction through the right electrode */
                pR = eR;
                kindR = 2;
            }
            if (k == 0 && open) {          /* extraction through the left electrode */
                pL = eL;
                kindL = 2;
            }
            int aR = 0, aL = 0;
            if (okR) {
                aR = trial(uR, pR, log, cap, count, r, t, k, 0, kindR);
                if (acc) acc_trial(acc, z, 0, kindR, pR, aR);
            }
            if (okL) {
                aL = trial(uL, pL, log, cap, count, r, t, k, 1, kindL);
                if (acc) acc_trial(acc, z, 1, kindL, pL, aL);
            }
            /* X + M_right - M_left: both trials succeeding leaves the ion in place */
            if (aR && !aL) mvR[k] = 1;
            if (aL && !aR) mvL[k] = 1;
        } else if (open && (k == 0 || k == L - 1)) {
            double iL, iR;
            orc_hop_probs(E_in, B[z], inv[z], &iL, &iR);
            site_uniforms(P, (uint32_t)k, (uint32_t)r, t, &uR, &uL);
            if (k == 0) { /* a rightward hop from the left reservoir into site 0 */
                injR = trial(uR, iR, log, cap, count, r, t, k, 0, 1);
                if (acc) acc_trial(acc, z, 0, 1, iR, injR);
            }
            if (k == L - 1) { /* a leftward hop from the right reservoir into site L-1 */
                injL = trial(uL, iL, log, cap, count, r, t, k, 1, 1);
                if (acc) acc_trial(acc, z, 1, 1, iL, injL);
            }
        }
    }

    /* conflicts: two hops into the same empty site cancel each other */
    for (int k = 0; k < L; ++k) {
        if (occ[k]) continue;
        int fromLeft = (k > 0) ? mvR[k - 1] : injR;
        int fromRight = (k < L - 1) ? mvL[k + 1] : injL;
        if (fromLeft && fromRight) {
            if (k > 0) mvR[k - 1] = 0; else injR = 0;
            if (k < L - 1) mvL[k + 1] = 0; else injL = 0;
        }
    }

    /* synchronous update and net crossings (leftward +1, rightward -1) */
    int64_t J = 0;
    memcpy(next, occ, (size_t)L);
    for (int k = 0; k < L; ++k) {
        if (mvR[k]) {
            next[k] = 0;
            if (k + 1 < L) next[k + 1] = 1;
            J -= 1;
        }
        if (mvL[k]) {
            next[k] = 0;
            if (k - 1 >= 0) next[k - 1] = 1;
            J += 1;
        }
    }
    if (injR) {
        next[0] = 1;
        J -= 1;
    }
    if (injL) {
        next[L - 1] = 1;
        J += 1;
    }
    memcpy(occ, next, (size_t)L);
    *J_acc += J;
}

/* ------------------------------------------------------------------------ */
/* Brick-wall variant (not the paper's rule; an optional alternative).  At   */
/* step t only the bonds (b, b+1) with b = t (mod 2) are active; the bond    */
/* (-1, 0) to the left reservoir has b = -1 (odd) and (L-1, L) to the right  */
/* one b = L-1.  Every site belongs to exactly one active bond, so an ion    */
/* makes at most one trial per step and no two hops can target one site.   */
/* An active inner bond holding one ion tries that ion's hop across it with */
/* the probability and the draw of Eqs. 5-6 (right hop: the right draw of   */
/* the ion's site, left hop: its left draw); the electrode bonds exchange   */
/* ions as in the synchronous rule.                                         */
/* ------------------------------------------------------------------------ */
static void rail_step_brick(const orc_params *P, int r, uint32_t t, double V, uint8_t *occ,
                            int32_t N0, const double *P0row, double P0scalar, double E_in,
                            double E_out, uint8_t *next, int64_t *J_acc, int64_t *zc_acc,
                            orc_log_entry *log, int64_t cap, int64_t *count)
{
    const int L = P->L, Z = P->Z;
    const int open = P->electrodes == 1;
    int32_t Nz[ORC_MAX_ZONES];
    double dV[ORC_MAX_ZONES], B[ORC_MAX_ZONES], inv[ORC_MAX_ZONES];
    for (int z = 0; z < Z; ++z) Nz[z] = 0;
    for (int k = 0; k < L; ++k)
        if (occ[k]) Nz[orc_zone_of(k, L, Z)] += 1;
    for (int z = 0; z < Z; ++z) zc_acc[z] += Nz[z];
    orc_zone_field(P, Nz, N0, V, dV, B, inv);

    const int par = (int)(t & 1u);
    int64_t J = 0;
    memcpy(next, occ, (size_t)L);
    for (int b = -1; b <= L - 1; ++b) {
        if (((b % 2) + 2) % 2 != par) continue;   /* inactive bond this step */
        double uR, uL, pl, pr;
        if (b == -1) {                            /* left reservoir | site 0 */
            if (!open) continue;
            const int z = orc_zone_of(0, L, Z);
            site_uniforms(P, 0u, (uint32_t)r, t, &uR, &uL);
            if (occ[0]) {                         /* extraction: leftward out of site 0 */
                orc_hop_probs(E_out, B[z], inv[z], &pl, &pr);
                if (trial(uL, pl, log, cap, count, r, t, 0, 1, 2)) {
                    next[0] = 0;
                    J += 1;
                }
            } else {                              /* injection: rightward into site 0 */
                orc_hop_probs(E_in, B[z], inv[z], &pl, &pr);
                if (trial(uR, pr, log, cap, count, r, t, 0, 0, 1)) {
                    next[0] = 1;
                    J -= 1;
                }
            }
        } else if (b == L - 1) {                  /* site L-1 | right reservoir */
            if (!open) continue;
            const int k = L - 1;
            const int z = orc_zone_of(k, L, Z);
            site_uniforms(P, (uint32_t)k, (uint32_t)r, t, &uR, &uL);
            if (occ[k]) {                         /* extraction: rightward out of L-1 */
                orc_hop_probs(E_out, B[z], inv[z], &pl, &pr);
                if (trial(uR, pr, log, cap, count, r, t, k, 0, 2)) {
                    next[k] = 0;
                    J -= 1;
                }
            } else {                              /* injection: leftward into L-1 */
                orc_hop_probs(E_in, B[z], inv[z], &pl, &pr);
                if (trial(uL, pl, log, cap, count, r, t, k, 1, 1)) {
                    next[k] = 1;
                    J += 1;
                }
            }
        } else if (occ[b] && !occ[b + 1]) {       /* the ion at b hops right */
            const int z = orc_zone_of(b, L, Z);
            site_uniforms(P, (uint32_t)b, (uint32_t)r, t, &uR, &uL);
            orc_hop_probs(P0row ? P0row[b] : P0scalar, B[z], inv[z], &pl, &pr);
            if (trial(uR, pr, log, cap, count, r, t, b, 0, 0)) {
                next[b] = 0;
                next[b + 1] = 1;
                J -= 1;
            }
        } else if (!occ[b] && occ[b + 1]) {       /* the ion at b+1 hops left */
            const int k = b + 1;
            const int z = orc_zone_of(k, L, Z);
            site_uniforms(P, (uint32_t)k, (uint32_t)r, t, &uR, &uL);
            orc_hop_probs(P0row ? P0row[k] : P0scalar, B[z], inv[z], &pl, &pr);
            if (trial(uL, pl, log, cap, count, r, t, k, 1, 0)) {
                next[k] = 0;
                next[b] = 1;
                J += 1;
            }
        }
    }
    memcpy(occ, next, (size_t)L);
    *J_acc += J;
}

int orc_run(const orc_params *P, const double *V, int64_t t0, int64_t n_steps, uint8_t *occ,
            const int32_t *N0, const double *P0site, const int32_t *rail_ids, int64_t *J_out,
            int64_t *Zc_out, int64_t *J_rail, orc_log_entry *log, int64_t log_cap,
            int64_t *log_count, int nthreads)
{
    const int R = P->R, L = P->L, Z = P->Z;
    if (L < 2 || Z < 1 || Z > ORC_MAX_ZONES || Z > L || R < 0) return -1;
    if (P->rule != 0 && P->rule != 1) return -1;
    if (t0 < 0 || t0 + n_steps > (int64_t)ORC_INIT_STEP) return -1;
    const double P0scalar = orc_p0(P->nu, P->Ea, P->T, P->dt);
    const double E = -expm1(-(2.0 * P->k_e * P->dt));
    const double E_in = E * P->rho_e;
    const double E_out = E * (1.0 - P->rho_e);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    for (int64_t s = 0; s < n_steps; ++s) {
        const uint32_t t = (uint32_t)(t0 + s);
        int64_t J = 0;
        int64_t zc[ORC_MAX_ZONES];
        for (int z = 0; z < Z; ++z) zc[z] = 0;
#ifdef _OPENMP
#pragma omp parallel reduction(+ : J) reduction(+ : zc[:ORC_MAX_ZONES])
#endif
        {
            int8_t *mvR = (int8_t *)malloc((size_t)L);
            int8_t *mvL = (int8_t *)malloc((size_t)L);
            uint8_t *next = (uint8_t *)malloc((size_t)L);
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
            for (int r = 0; r < R; ++r) {
                int64_t Jr = 0;
                const int rail = rail_ids ? rail_ids[r] : r;
                if (P->rule == 1)
                    rail_step_brick(P, rail, t, V[t], occ + (int64_t)r * L, N0[r],
                                    P0site ? P0site + (int64_t)r * L : NULL, P0scalar, E_in,
                                    E_out, next, &Jr, zc, log, log_cap, log_count);
                else
                    rail_step(P, rail, t, V[t], occ + (int64_t)r * L, N0[r],
                              P0site ? P0site + (int64_t)r * L : NULL, P0scalar, E_in, E_out,
                              mvR, mvL, next, &Jr, zc, log, log_cap, log_count, NULL);
                J += Jr;
                if (J_rail) J_rail[r] += Jr;
            }
            free(mvR);
            free(mvL);
            free(next);
        }
        if (J_out) J_out[s] = J;
        if (Zc_out)
            for (int z = 0; z < Z; ++z) Zc_out[s * Z + z] = zc[z];
    }
    return 0;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Likelihood-ratio gradient of a linear observable of the traces.          */
/* ------------------------------------------------------------------------ */
int orc_run_lr(const orc_params *P, const orc_params *Pe, const double *V, int64_t t0,
               int64_t n_steps, uint8_t *occ, const int32_t *N0, const double *wJ,
               const double *wZ, const int64_t *J_tot, const int64_t *Zc_tot, double *S_cum,
               double *G, double *loglik, int64_t *J_out, int nthreads, int64_t cv_window,
               double *cv_out)
{
    const int R = P->R, L = P->L, Z = P->Z;
    if (L < 2 || Z < 1 || Z > ORC_MAX_ZONES || Z > L || R < 0) return -1;
    if (P->rule != 0) return -1;   /* the score hook follows the synchronous rule */
    if (t0 < 0 || t0 + n_steps > (int64_t)ORC_INIT_STEP) return -1;
    if ((wJ && !J_tot) || (wZ && !Zc_tot)) return -1;
    if (cv_out && cv_window < 1) return -1;
    const int64_t cvK = cv_out ? (n_steps + cv_window - 1) / cv_window : 0;
    const int cvF = Z + 2;   /* features: 1, first moment / L, zone counts */
    const double P0scalar = orc_p0(P->nu, P->Ea, P->T, P->dt);
    const double E = -expm1(-(2.0 * P->k_e * P->dt));
    const double E_in = E * P->rho_e;
    const double E_out = E * (1.0 - P->rho_e);
    const double kT = ORC_KB * P->T;
    const double x = 2.0 * orc_gamma0(P->nu, P->Ea, P->T) * P->dt;
    const double dlnP0_dEa = -((x / kT) * exp(-x)) / P0scalar;
    const double dlnP0_dnu = ((x / P->nu) * exp(-x)) / P0scalar;
    const double Ee = -expm1(-(2.0 * Pe->k_e * Pe->dt));
    const double P0e = orc_p0(Pe->nu, Pe->Ea, Pe->T, Pe->dt);
    const double loo = R > 1 ? (double)(R - 1) : 0.0;   /* leave-one-out baseline divisor */
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    for (int64_t s = 0; s < n_steps; ++s) {
        const uint32_t t = (uint32_t)(t0 + s);
        int64_t J = 0;
#ifdef _OPENMP
#pragma omp parallel reduction(+ : J)
#endif
        {
            int8_t *mvR = (int8_t *)malloc((size_t)L);
            int8_t *mvL = (int8_t *)malloc((size_t)L);
            uint8_t *next = (uint8_t *)malloc((size_t)L);
            orc_trial_acc acc;
            acc.Pe = Pe;
            acc.dlnP0[0] = dlnP0_dEa;
            acc.dlnP0[1] = dlnP0_dnu;
            acc.P0e = P0e;
            acc.Ein_e = Ee * Pe->rho_e;
            acc.Eout_e = Ee * (1.0 - Pe->rho_e);
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
            for (int r = 0; r < R; ++r) {
                int64_t Jr = 0;
                int64_t zc[ORC_MAX_ZONES];
                for (int z = 0; z < Z; ++z) zc[z] = 0;
                /* first moment of the step-start occupancy (control-variate feature) */
                double m1 = 0.0;
                if (cv_out) {
                    const uint8_t *o = occ + (int64_t)r * L;
                    for (int k = 0; k < L; ++k) m1 += (double)(k * o[k]);
                    m1 /= (double)L;
                }
                rail_step(P, r, t, V[t], occ + (int64_t)r * L, N0[r], NULL, P0scalar, E_in, E_out,
                          mvR, mvL, next, &Jr, zc, NULL, 0, NULL, &acc);
                if (cv_out) {
                    /* score increments of this rail-step times the step-start features */
                    const int64_t k = s / cv_window;
                    for (int e = 0; e < 2; ++e) {
                        const double psi = acc.s[e == 0 ? 0 : 2];
                        double *cv = cv_out + (((int64_t)r * 2 + e) * cvK + k) * cvF;
                        cv[0] += psi;
                        cv[1] += psi * m1;
                        for (int z = 0; z < Z; ++z) cv[2 + z] += psi * (double)acc.Nz[z];
                    }
                }
                double *Sr = S_cum + 4 * (int64_t)r;
                double *Gr = G + 4 * (int64_t)r;
                /* zone counts at the start of step t pair with the score of steps < t */
                if (wZ) {
                    double fZ = 0.0;
                    for (int z = 0; z < Z; ++z) {
                        const double b = loo > 0.0 ? (double)(Zc_tot[s * Z + z] - acc.Nz[z]) / loo : 0.0;
                        fZ += wZ[s * Z + z] * ((double)acc.Nz[z] - b);
                    }
                    for (int i = 0; i < 4; ++i) Gr[i] += fZ * Sr[i];
                }
                /* control variate: the innovation of J_rs times the score before step s
                 * has zero mean; removing it leaves the predictable part of the
                 * current paired with the past score */
                if (wJ) {
                    const double c = wJ[s] * acc.eta;
                    for (int i = 0; i < 4; ++i) Gr[i] -= c * Sr[i];
                }
                for (int i = 0; i < 3; ++i) Sr[i] += acc.s[i];
                /* the current of step t pairs with the score of steps <= t */
                if (wJ) {
                    const double b = loo > 0.0 ? (double)(J_tot[s] - Jr) / loo : 0.0;
                    const double fJ = wJ[s] * ((double)Jr - b);
                    for (int i = 0; i < 4; ++i) Gr[i] += fJ * Sr[i];
                }
                if (loglik) loglik[r] += acc.ll;
                J += Jr;
            }
            free(mvR);
            free(mvL);
            free(next);
        }
        if (J_out) J_out[s] = J;
    }
    return 0;
}
