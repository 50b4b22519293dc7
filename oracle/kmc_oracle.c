/*
 * kmc_oracle.c -- plain FP64 CPU oracle of the rail-based kinetic Monte Carlo
 * ion-migration step (arXiv 2511.09413, Supplementary Information S2.1).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path.
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
void orc_zone_field(const orc_params *P, const int32_t *Nz, int32_t N0, double V,
                    double *dV, double *B, double *inv)
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
    double ka = P->kappa * P->alpha;
    double kT = ORC_KB * P->T;
    double t_dev = (double)L * P->d;
    for (int z = 0; z < Z; ++z) {
        dV[z] = V - ka * (Q[z] - Qbar);
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

static void rail_step(const orc_params *P, int r, uint32_t t, double V, uint8_t *occ, int32_t N0,
                      const double *P0row, double P0scalar, double E_in, double E_out,
                      int8_t *mvR, int8_t *mvL, uint8_t *next, int64_t *J_acc, int64_t *zc_acc,
                      orc_log_entry *log, int64_t cap, int64_t *count)
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
            int aR = okR && trial(uR, pR, log, cap, count, r, t, k, 0, kindR);
            int aL = okL && trial(uL, pL, log, cap, count, r, t, k, 1, kindL);
            /* X + M_right - M_left: both trials succeeding leaves the ion in place */
            if (aR && !aL) mvR[k] = 1;
            if (aL && !aR) mvL[k] = 1;
        } else if (open && (k == 0 || k == L - 1)) {
            double iL, iR;
            orc_hop_probs(E_in, B[z], inv[z], &iL, &iR);
            site_uniforms(P, (uint32_t)k, (uint32_t)r, t, &uR, &uL);
            if (k == 0) /* a rightward hop from the left reservoir into site 0 */
                injR = trial(uR, iR, log, cap, count, r, t, k, 0, 1);
            if (k == L - 1) /* a leftward hop from the right reservoir into site L-1 */
                injL = trial(uL, iL, log, cap, count, r, t, k, 1, 1);
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

int orc_run(const orc_params *P, const double *V, int64_t t0, int64_t n_steps, uint8_t *occ,
            const int32_t *N0, const double *P0site, const int32_t *rail_ids, int64_t *J_out,
            int64_t *Zc_out, int64_t *J_rail, orc_log_entry *log, int64_t log_cap,
            int64_t *log_count, int nthreads)
{
    const int R = P->R, L = P->L, Z = P->Z;
    if (L < 2 || Z < 1 || Z > ORC_MAX_ZONES || Z > L || R < 0) return -1;
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
                rail_step(P, rail, t, V[t], occ + (int64_t)r * L, N0[r],
                          P0site ? P0site + (int64_t)r * L : NULL, P0scalar, E_in, E_out,
                          mvR, mvL, next, &Jr, zc, log, log_cap, log_count);
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
