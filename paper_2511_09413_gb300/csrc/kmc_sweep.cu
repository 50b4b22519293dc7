// kmc_sweep.cu -- the per-time-step sweep over every rail and site
// (arXiv 2511.09413, Supplementary S2.1.2 - S2.1.7), hand-written for sm_103a.
//
// Design (GB300):
//  * A rail lives in registers as a bitmask: lane l of a rail's lane segment
//    holds sites [32 l WPL, 32 (l + 1) WPL).  LPR lanes per rail, 32 / LPR rails
//    per warp.  The occupancy is read from HBM once per launch (uint8 rows,
//    16-byte vector loads), kept resident for all steps of the launch, and
//    written back once.
//  * Zone counts come from a segmented warp scan of popcounts; the field of
//    S2.1.8 and Eqs. 3-6 are evaluated once per (rail, zone) per step.
//  * GB300's FP64 rate is a small fraction of its FP32 rate, so each decision
//    u <= p (S2.1.7) is first made against an FP32 interval [p_lo, p_hi] that
//    provably contains the exact FP64 p: a draw whose high 32 bits lie below
//    p_lo 2^32 - 1 is accepted and one above p_hi 2^32 is rejected without
//    any FP64 work.  Only draws inside the interval (about 1e-6 of them) take
//    the exact path, which recomputes p in FP64 with the oracle's operation
//    order and compares u <= p exactly.  Decisions are therefore identical to
//    an all-FP64 evaluation.
//  * Philox4x32-10 is evaluated only for sites whose decision can matter
//    (occupied with a free neighbour, or an electrode site), after a warp-wide
//    compaction so that all 32 lanes draw.  The draw loop itself is lean: one
//    Philox block, one zone-threshold load and two compares; hops are rare
//    (p ~ 1e-4), so acceptance, electrodes and per-site refinement live on a
//    rarely taken branch, and the exact FP64 path runs after the loop.
//  * Moves are rare per step, so the move/conflict/apply phase runs only when
//    the warp accepted at least one hop.
//  * Per-step current and zone-count changes go straight to the int64 traces
//    with one global reduction per warp and nonzero value (only steps that
//    moved an ion have any); a prefix sum over the launch's steps
//    (zone_scan_kernel) turns the zone-count changes into counts.  No CTA
//    barrier: the warps of a CTA advance independently.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <type_traits>

#include "kmc_internal.h"

namespace kmc {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kDeferCap = 64;           // deferred (exact-path) candidates per warp and step
// Philox blocks in flight per lane per iteration of the draw loop.  One is
// fastest on both loops: the kernel gains more from resident warps than from
// ILP (the accept-table loop at 4 CTAs per SM, the reject-only loop at 5).
constexpr int kDrawIlpAcc = 1;
constexpr int kDrawIlpReject = 1;

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): per round two 32x32->64
// multiplies; the high halves are xor-ed with the other counter words and the
// round key.  The ten round keys are precomputed on the host.
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        const uint32_t *rk0, const uint32_t *rk1)
{
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        // one widening multiply per product (both halves at once): 1 % faster
        // in the sweep and 2.5 % in the Philox-only probe than separate
        // low and high multiplies
        uint64_t p0, p1;
        asm("mul.wide.u32 %0, %1, %2;" : "=l"(p0) : "r"(c0), "r"(0xD2511F53u));
        asm("mul.wide.u32 %0, %1, %2;" : "=l"(p1) : "r"(c2), "r"(0xCD9E8D57u));
        const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
        const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
        c0 = hi1 ^ c1 ^ rk0[i];
        c1 = lo1;
        c2 = hi0 ^ c3 ^ rk1[i];
        c3 = lo0;
    }
    return make_uint4(c0, c1, c2, c3);
}

// 16 occupancy bytes (values 0/1) -> 16 bits; byte i -> bit i.
__device__ __forceinline__ uint32_t pack4(uint32_t v)
{
    return (((v & 0x01010101u) * 0x00204081u) >> 21) & 0xFu;
}
__device__ __forceinline__ uint32_t pack16(uint4 q)
{
    return pack4(q.x) | (pack4(q.y) << 4) | (pack4(q.z) << 8) | (pack4(q.w) << 12);
}
// 4 bits -> 4 bytes of 0/1
__device__ __forceinline__ uint32_t unpack4(uint32_t n)
{
    return (n * 0x00204081u) & 0x01010101u;
}
__device__ __forceinline__ uint4 unpack16(uint32_t b)
{
    return make_uint4(unpack4(b & 0xF), unpack4((b >> 4) & 0xF), unpack4((b >> 8) & 0xF),
                      unpack4((b >> 12) & 0xF));
}

// Site masks of the 32-site word starting at site s0 of an L-site rail: the
// sites that exist, site 0, site L-1.  Recomputed where needed rather than
// held in registers through the step.
__device__ __forceinline__ uint32_t valid_mask(int s0, int L)
{
    return s0 >= L ? 0u : (s0 + 32 <= L ? 0xffffffffu : ((1u << (L - s0)) - 1u));
}
__device__ __forceinline__ uint32_t first_mask(int s0) { return s0 == 0 ? 1u : 0u; }
__device__ __forceinline__ uint32_t last_mask(int s0, int L)
{
    return (L - 1 >= s0 && L - 1 < s0 + 32) ? (1u << (L - 1 - s0)) : 0u;
}

// Conservative integer thresholds on the high 32 bits h of a 64-bit draw w
// (u = (w >> 11) 2^-53):  h < acc_thr(p_lo) implies u <= p;  h > rej_thr(p_hi)
// implies u > p, for any p in [p_lo, p_hi].
__device__ __forceinline__ uint32_t acc_thr(float p_lo)
{
    const uint32_t f = __float2uint_rd(p_lo * 4294967296.0f);
    return f > 0u ? f - 1u : 0u;
}
__device__ __forceinline__ uint32_t rej_thr(float p_hi)
{
    return __float2uint_ru(p_hi * 4294967296.0f);
}

// ---------------------------------------------------------------- shared memory
// One warp's block: a fixed part whose offsets are compile-time constants and a
// part that scales with G * Z (offsets from one runtime stride), so that the
// kernel keeps only a base address and that stride in registers.
__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

template <int LPR, int WPL>
struct Layout {
    static constexpr int G = 32 / LPR;
    static constexpr int W = 32 * WPL;                 // words per warp
    static constexpr int LIST = 1024 * WPL + 2 * G;    // candidate slots
    static constexpr size_t MVR = 0;
    static constexpr size_t MVL = MVR + align16(4 * W);
    static constexpr size_t FR = MVL + align16(4 * W);
    static constexpr size_t FL = FR + align16(4 * W);
    static constexpr size_t OW = FL + align16(4 * W);
    static constexpr size_t INJ = OW + align16(4 * W);         // int [2][G]
    static constexpr size_t N0S = INJ + align16(4 * 2 * G);    // int [G]
    static constexpr size_t FS = N0S + align16(4 * G);         // int [G]
    static constexpr size_t JR = FS + align16(4 * G);          // int [G]: per-rail current
    static constexpr size_t NDEF = JR + align16(4 * G);        // int [4]
    static constexpr size_t CNT = NDEF + 16;                   // uint32 [4]: draws, moves
    static constexpr size_t DEF = CNT + 16;                    // uint16 [kDeferCap]
    static constexpr size_t LST = DEF + align16(2 * 64);       // uint16 [LIST]
    static constexpr size_t FIXED = LST + align16(2 * LIST);
    // variable part: rm [G Z + 2 G] (zones, then the two electrode sites of each
    // rail): uint2 reject-sure bounds (R, L) on the draw's high word, or, with the
    // accept tables, uint4 (reject R, reject L, accept R, accept L), zf and P0b float2 [G][Z] (gz8 = align16(8 G Z) bytes each),
    // Pb int [G][Z+1]
    __host__ __device__ static size_t rm_bytes(int Z, bool acc)
    {
        return align16((size_t)(acc ? 16 : 8) * G * (Z + 2));
    }
    __host__ __device__ static size_t gz8(int Z) { return align16((size_t)8 * G * Z); }
    // Pb int [G][Z+1], then the zone counts last written to the trace int [G][Z]
    __host__ __device__ static size_t pb_only(int Z) { return align16((size_t)4 * G * (Z + 1)); }
    __host__ __device__ static size_t pb_bytes(int Z) { return pb_only(Z) + align16((size_t)4 * G * Z); }
    __host__ __device__ static size_t bytes(int Z, bool acc)
    {
        return FIXED + rm_bytes(Z, acc) + 2 * gz8(Z) + pb_bytes(Z);
    }
    // gradient pass, appended: accepted-trial masks accR, accL uint32 [W] each;
    // per (rail, zone) (gzq = align16(8 G Z) bytes per double): Q_z double,
    // N0 w_z / L double, and the cached (p_R, p_L), (1/(1-p_R), 1/(1-p_L)),
    // (d ln p_R / d kappa, d ln p_L / d kappa), (p_R/(1-p_R), p_L/(1-p_L))
    // double2; per rail double [G][16]
    // (state, Qbar, V of the cache, electrode probabilities and reciprocals);
    // per rail int [G][Z+2] (zone prefix counts of the cache, changed flag)
    __host__ __device__ static size_t grad_bytes(int Z)
    {
        return 2 * align16(4 * W) + 10 * align16((size_t)8 * G * Z) + align16((size_t)128 * G) +
               align16((size_t)4 * G * (Z + 2));
    }
};

// Candidate-list entries (uint16): the site in the low bits and, above it,
// the rail slot (several rails per warp) or, with one rail per warp, the row
// of the entry's decision bounds in rm (its zone).  Rails of at most 1,024
// sites in one word per lane need only 10 site bits, which leaves 6 bits for
// rows up to G Z + 1, so the electrode entries carry their rows too and the
// draw loop reads every row straight from the entry.
template <int LPR, int WPL>
struct ListCode {
    static constexpr bool kRow = LPR == 32 && WPL == 1;
    static constexpr int kShift = kRow ? 10 : 11;
    static constexpr uint32_t kSite = (1u << kShift) - 1u;
};

template <int LPR, int WPL>
struct WarpSmem {
    using Ly = Layout<LPR, WPL>;
    uint8_t *b;     // block base (shared memory)
    uint32_t rz;    // Layout::rm_bytes(Z, acc)
    uint32_t gz;    // Layout::gz8(Z)
    uint32_t pbz;   // Layout::pb_bytes(Z)
    uint32_t npo;   // offset of the zone counts last written to the trace
    uint32_t goff;  // Layout::bytes(Z, acc): start of the gradient-pass region
    uint32_t gzq;   // align16(8 G Z)
    __device__ uint32_t *mvR() const { return (uint32_t *)(b + Ly::MVR); }
    __device__ uint32_t *mvL() const { return (uint32_t *)(b + Ly::MVL); }
    __device__ uint32_t *fR() const { return (uint32_t *)(b + Ly::FR); }
    __device__ uint32_t *fL() const { return (uint32_t *)(b + Ly::FL); }
    __device__ uint32_t *ow() const { return (uint32_t *)(b + Ly::OW); }
    __device__ int32_t *inj() const { return (int32_t *)(b + Ly::INJ); }
    __device__ int32_t *N0s() const { return (int32_t *)(b + Ly::N0S); }
    __device__ int32_t *Fs() const { return (int32_t *)(b + Ly::FS); }
    // net leftward crossings of each rail of the warp since the last flush
    __device__ int32_t *jr() const { return (int32_t *)(b + Ly::JR); }
    __device__ int32_t *ndef() const { return (int32_t *)(b + Ly::NDEF); }
    // window mid voltage (FP32) and band factors (flo, fhi), stored next to
    // the deferral counter
    __device__ float &vmid_ref() const { return *(float *)(b + Ly::NDEF + 4); }
    __device__ float2 &band() const { return *(float2 *)(b + Ly::NDEF + 8); }
    // Philox blocks drawn and hops applied by the warp since the last flush
    __device__ uint32_t *cnt() const { return (uint32_t *)(b + Ly::CNT); }
    __device__ uint16_t *def() const { return (uint16_t *)(b + Ly::DEF); }
    __device__ uint16_t *list() const { return (uint16_t *)(b + Ly::LST); }
    __device__ uint2 *rm() const { return (uint2 *)(b + Ly::FIXED); }
    __device__ uint4 *rm4() const { return (uint4 *)(b + Ly::FIXED); }
    __device__ float2 *zf() const { return (float2 *)(b + Ly::FIXED + rz); }
    __device__ float2 *P0b() const { return (float2 *)(b + Ly::FIXED + rz + gz); }
    __device__ int32_t *Pb() const { return (int32_t *)(b + Ly::FIXED + rz + 2 * gz); }
    __device__ int32_t *Np() const { return (int32_t *)(b + npo); }
    __device__ uint32_t *accR() const { return (uint32_t *)(b + goff); }
    __device__ uint32_t *accL() const { return (uint32_t *)(b + goff + align16(4 * Ly::W)); }
    __device__ uint8_t *gbase() const { return b + goff + 2 * align16(4 * Ly::W); }
    // exp(gXV ka D'_z): the background factor of B_z (exp tables on)
    __device__ double *gEe() const { return (double *)gbase(); }
    __device__ double *gCz() const { return (double *)(gbase() + gzq); }
    __device__ double2 *gP() const { return (double2 *)(gbase() + 2 * gzq); }
    __device__ double2 *gR1() const { return (double2 *)(gbase() + 4 * gzq); }
    __device__ double2 *gDK() const { return (double2 *)(gbase() + 6 * gzq); }
    __device__ double2 *gPQ() const { return (double2 *)(gbase() + 8 * gzq); }
    __device__ double *gS() const { return (double *)(gbase() + 10 * gzq); }
    __device__ int32_t *gPb() const { return (int32_t *)(gbase() + 10 * gzq + align16(128 * Ly::G)); }
};

// --------------------------------------------------------- exact FP64 path
// Exact FP64 zone quantities (B_z, 1/(1+B_z)) for zone zt of one rail, with
// the operation order of the oracle: excess C_z, enclosed charge Q_z, mean
// Qbar, dV_z (S2.1.8), dE_z (Eq. 3), B_z (Eq. 4).  Every operation is an
// explicitly rounded intrinsic so that no contraction changes the result.
__device__ __forceinline__ void exact_zone(const int32_t *Pb, const DevConst *Kp, int Z, int L,
                                        int32_t n0, const double2 *bgd, double V, int zt, double *B,
                                        double *inv)
{
    const DevConst &K = *Kp;
    const double Ld = (double)L;
    double run = 0.0, acc = 0.0, Qt = 0.0;
    for (int z = 0; z < Z; ++z) {
        const int w = K.bnd[z + 1] - K.bnd[z];
        const int Nz = Pb[z + 1] - Pb[z];
        // background N0 w_z / L: the rail's precomputed row when there is one
        const double bz = bgd ? bgd[z].x : __ddiv_rn(__dmul_rn((double)n0, (double)w), Ld);
        const double C = __dsub_rn((double)Nz, bz);
        const double Q = __dadd_rn(run, __dmul_rn(0.5, C));
        run = __dadd_rn(run, C);
        acc = __dadd_rn(acc, __dmul_rn((double)w, Q));
        if (z == zt) Qt = Q;
    }
    const double Qbar = __ddiv_rn(acc, Ld);
    const double dV = __dsub_rn(V, __dmul_rn(K.ka, __dsub_rn(Qt, Qbar)));
    const double dE = __ddiv_rn(__dmul_rn(dV, K.d), K.t_dev);
    const double b = exp(__ddiv_rn(-dE, K.kT));
    *B = b;
    *inv = __ddiv_rn(1.0, __dadd_rn(1.0, b));
}

// Exact decision u <= p for the 64-bit word w, with near-threshold logging.
__device__ __forceinline__ bool exact_trial(uint64_t w, double p, kmc_log_entry *log,
                                         unsigned long long *log_count, int64_t log_cap,
                                         int32_t rail, uint32_t step, int32_t site, int32_t dir,
                                         int32_t kind)
{
    const double u = __dmul_rn((double)(w >> 11), 0x1.0p-53);
    const double diff = __dsub_rn(u, p);
    if (fabs(diff) < 1e-12) {
        const unsigned long long slot = atomicAdd(log_count, 1ull);
        if ((int64_t)slot < log_cap) {
            kmc_log_entry e;
            e.rail = rail;
            e.step = step;
            e.site = site;
            e.dir = dir;
            e.kind = kind;
            e.pad = 0;
            e.diff = diff;
            log[slot] = e;
        }
    }
    return u <= p;
}

// ------------------------------------------------------------ one decision
// Bounded decision of one candidate from the step-start state kept in shared
// memory: dR, dL in {0 reject (or direction blocked), 1 accept, 2 undecided},
// the move kinds (0 inner hop, 1 injection, 2 extraction), and where to record
// the move.  Thresholds come from the zone's FP32 (B, 1/(1+B)) and the band
// factors (flo, fhi); electrode and per-site base probabilities are applied here.
struct Decision {
    int dR, dL, kindR, kindL;
    bool occd;
    int idx;
    uint32_t bit;
};

// Band factors: p_lo = p flo, p_hi = p fhi bracket the exact p.
__device__ __forceinline__ int bounded(uint32_t h, float p, float flo, float fhi)
{
    return h < acc_thr(p * flo) ? 1 : (h > rej_thr(p * fhi) ? 0 : 2);
}

template <int LPR, int WPL>
__device__ __forceinline__ Decision decide(const WarpSmem<LPR, WPL> &S, const SweepArgs *g,
                                           uint4 x, int site, int g2, int z, bool isE,
                                           bool persite, float flo, float fhi, int64_t r2)
{
    const int L = g->L, Z = g->Z;
    Decision D;
    D.idx = g2 * LPR * WPL + (site >> 5);
    D.bit = 1u << (site & 31);
    D.occd = (S.ow()[D.idx] & D.bit) != 0;
    // an occupied site tries a direction whose neighbour (or open electrode) is
    // free; at an empty electrode site the same mask bits say whether an
    // injection is tried (set when the masks are built)
    const bool tryR = (S.fR()[D.idx] & D.bit) != 0;
    const bool tryL = (S.fL()[D.idx] & D.bit) != 0;
    const float2 bi = S.zf()[g2 * Z + z];          // (B, 1/(1+B)); (0, 0) when undecidable
    const bool ok = bi.y > 0.0f;
    const float sR = bi.y * bi.x, sL = bi.y;
    D.kindR = 0;
    D.kindL = 0;
    // base probability of each trial: P0 (scalar or this site's), or electrode
    // exchange.  The slow path is rare, so a site's P0 is read from global memory
    // (rail r2) rather than staged in shared memory.
    float bR = persite ? __ldg(g->P0f + r2 * L + site) : g->K->P0f;
    float bL = bR;
    if (isE) {
        if (!D.occd) {              // injection: site 0 via the right draw, L-1 via the left
            if (site == 0) {
                bR = g->K->E_inf;
                D.kindR = 1;
            } else {
                bL = g->K->E_inf;
                D.kindL = 1;
            }
        } else {                    // extraction through the adjacent electrode
            if (site == 0) {
                bL = g->K->E_outf;
                D.kindL = 2;
            }
            if (site == L - 1) {
                bR = g->K->E_outf;
                D.kindR = 2;
            }
        }
    }
    D.dR = tryR ? (ok ? bounded(x.y, bR * sR, flo, fhi) : 2) : 0;
    D.dL = tryL ? (ok ? bounded(x.w, bL * sL, flo, fhi) : 2) : 0;
    return D;
}

// Record an accepted net move (both trials accepted: the ion stays, S2.1.7).
// The gradient pass also marks every accepted trial.
template <int LPR, int WPL, bool GRAD = false>
__device__ __forceinline__ bool record_move(const WarpSmem<LPR, WPL> &S, const Decision &D, int g2)
{
    constexpr int G = 32 / LPR;
    if constexpr (GRAD) {
        if (D.dR == 1) atomicOr(&S.accR()[D.idx], D.bit);
        if (D.dL == 1) atomicOr(&S.accL()[D.idx], D.bit);
    }
    if (D.dR == 1 && D.dL != 1) {
        if (!D.occd) S.inj()[g2] = 1;               // injection into site 0
        else atomicOr(&S.mvR()[D.idx], D.bit);
        return true;
    }
    if (D.dL == 1 && D.dR != 1) {
        if (!D.occd) S.inj()[G + g2] = 1;           // injection into site L-1
        else atomicOr(&S.mvL()[D.idx], D.bit);
        return true;
    }
    return false;
}

// Slow path of one candidate (taken for roughly one draw in a thousand):
// recomputes the draw, decides against the FP32 band and records the move.
// With exact == false an undecided candidate is queued for the exact pass;
// with exact == true only undecided candidates are handled, by recomputing p
// in FP64 with the oracle's operation order (exact_zone) and comparing u <= p.
// Reads the launch arguments through their copy in global memory (g), which
// keeps the parameter block in the constant bank for the draw loop.
template <int LPR, int WPL, bool GRAD = false>
__device__ __forceinline__ bool slow_candidate(WarpSmem<LPR, WPL> S, const SweepArgs *g, int i,
                                            int n_inner, int64_t rail0, uint32_t t,
                                            const uint8_t *zone_tab, bool persite, bool exact,
                                            uint32_t xy, uint32_t xw)
{
    const float2 band = S.band();
    const float flo = band.x, fhi = band.y;
    const uint16_t dsc = S.list()[i];
    const int site = dsc & ListCode<LPR, WPL>::kSite, g2 = LPR == 32 ? 0 : dsc >> 11;
    const int64_t r2 = rail0 + g2;                      // the rail's row in this device
    const uint32_t rg = g->rail_base + (uint32_t)r2;    // its global index (Philox, log)
    // the bounded decision needs only the high words (x1, x3) of the draw; the
    // exact pass recomputes the whole block
    const uint4 x = exact ? philox((uint32_t)site, rg, t, g->instance, g->rk0, g->rk1)
                          : make_uint4(0u, xy, 0u, xw);
    const int z = zone_tab[site];
    const bool isE = i >= n_inner;
    Decision D = decide<LPR, WPL>(S, g, x, site, g2, z, isE, persite, flo, fhi, r2);
    const bool undecided = D.dR == 2 || D.dL == 2;
    if (!exact) {
        if (undecided) {
            const int slot = atomicAdd(S.ndef(), 1);
            if (slot < kDeferCap) S.def()[slot] = (uint16_t)i;
            return false;
        }
        return record_move<LPR, WPL, GRAD>(S, D, g2);
    }
    if (!undecided) return false;   // decided (and applied) in the draw loop
    const DevConst *K = g->K;
    const int L = g->L, Z = g->Z;
    const double V = g->V[t];
    const double P0k = persite ? g->P0site[r2 * L + site] : K->P0;
    const double baseR = D.kindR == 1 ? K->E_in : (D.kindR == 2 ? K->E_out : P0k);
    const double baseL = D.kindL == 1 ? K->E_in : (D.kindL == 2 ? K->E_out : P0k);
    const uint64_t wR = ((uint64_t)x.y << 32) | x.x, wL = ((uint64_t)x.w << 32) | x.z;
    unsigned ne = 0;
    // FP64 band: p from Q_z - Qbar = m_z / (2 L) - D'_z (integer m_z, the rail's
    // D'_z) in a dozen FP64 operations.  Its relative error is below 1e-13 for
    // every exponent |x| < 600 (a few roundings of x, each moving p by at most
    // |x| ulp), so a draw more than 1e-11 from it has the exact p on the same
    // side and is not a near-threshold decision (|u - p| > 1e-12).  Only draws
    // within 1e-11 take the exact path below.
    if (g->bgd) {
        const int32_t *Pb = S.Pb() + g2 * (Z + 1);
        const int m = L * (Pb[z] + Pb[z + 1]) - S.Fs()[g2];
        const double dq = __fma_rn((double)m, K->half_invL, -g->bgd[r2 * Z + z].y);
        const double xx = __dmul_rn(__fma_rn(-K->ka, dq, V), K->xs);
        if (fabs(xx) < 600.0) {
            const double Bf = exp(xx);
            const double invf = 1.0 / (1.0 + Bf);
            if (D.dR == 2) {
                const double d = __dsub_rn(__dmul_rn((double)(wR >> 11), 0x1.0p-53),
                                           __dmul_rn(__dmul_rn(baseR, invf), Bf));
                if (fabs(d) > 1e-11) {
                    D.dR = d <= 0.0 ? 1 : 0;
                    ++ne;
                }
            }
            if (D.dL == 2) {
                const double d = __dsub_rn(__dmul_rn((double)(wL >> 11), 0x1.0p-53),
                                           __dmul_rn(baseL, invf));
                if (fabs(d) > 1e-11) {
                    D.dL = d <= 0.0 ? 1 : 0;
                    ++ne;
                }
            }
        }
    }
    if (D.dR == 2 || D.dL == 2) {
        // exact path: p in FP64 with the oracle's operation order, u <= p
        double B, inv;
        exact_zone(S.Pb() + g2 * (Z + 1), K, Z, L, S.N0s()[g2], g->bgd ? g->bgd + r2 * Z : nullptr,
                   V, z, &B, &inv);
        if (D.dR == 2) {
            const double p = __dmul_rn(__dmul_rn(baseR, inv), B);   // Eq. 6
            D.dR = exact_trial(wR, p, g->log, g->log_count, g->log_cap, (int32_t)rg, t, site, 0,
                               D.kindR) ? 1 : 0;
            ++ne;
        }
        if (D.dL == 2) {
            const double p = __dmul_rn(baseL, inv);                  // Eq. 5
            D.dL = exact_trial(wL, p, g->log, g->log_count, g->log_cap, (int32_t)rg, t, site, 1,
                               D.kindL) ? 1 : 0;
            ++ne;
        }
    }
    atomicAdd(&g->counters[1], (unsigned long long)ne);
    return record_move<LPR, WPL, GRAD>(S, D, g2);
}

// ------------------------------------------------- likelihood-ratio score
// Summed score weight of n Bernoulli(p) trials of which A succeeded: each
// trial contributes (a - p) / (1 - p) times d ln p, so the sum is
// A r1 - n q with r1 = 1 / (1 - p) and q = p / (1 - p), kept with p; a
// certain trial (p >= 1) contributes d ln p, and is cached as r1 = 1, q = 0.
__device__ __forceinline__ double trial_weight(int A, int n, double r1, double q)
{
    return __fma_rn(-(double)n, q, __dmul_rn((double)A, r1));
}
// Tests on a double's bit pattern, on the integer pipe (FP64 compares take
// the FP64 pipe, the gradient pass's bottleneck): x != 0 (NaN counts as
// nonzero, as the FP64 test does), equality of two values that are never NaN
// (+0 and -0 differ: a stale mark at worst), and lo < x < hi for lo, hi
// positive and finite (positive doubles order as their bit patterns; negative
// values and NaN fall outside).
__device__ __forceinline__ bool nonzero_bits(double x)
{
    return ((unsigned long long)__double_as_longlong(x) << 1) != 0ull;
}
__device__ __forceinline__ bool same_bits(double x, double y)
{
    return __double_as_longlong(x) == __double_as_longlong(y);
}
__device__ __forceinline__ bool inside_bits(double x, double lo, double hi)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned long long l = (unsigned long long)__double_as_longlong(lo);
    const unsigned long long h = (unsigned long long)__double_as_longlong(hi);
    return u - (l + 1ull) < h - (l + 1ull);
}

// 1 / d for d > 0 (normal, finite) by Newton-Raphson on f(r) = 1/r - d from the
// hardware approximation (rcp.approx.ftz.f64, about 2^-22 relative): each
// step r <- r + r (1 - d r) squares the relative error, so two give full FP64
// accuracy up to a few ulp, enough for score weights.
__device__ __forceinline__ double recip_newton(double d)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
    double e = __fma_rn(-d, r, 1.0);
    r = __fma_rn(r, e, r);
    e = __fma_rn(-d, r, 1.0);
    return __fma_rn(r, e, r);
}

// Score weight of one electrode trial of probability p, outcome hit, with
// r1 = 1 / (1 - p) (0 when p >= 1)
__device__ __forceinline__ double et_weight(int hit, double p, double r1)
{
    if (p >= 1.0) return (double)hit;
    return __fma_rn(-1.0, __dmul_rn(p, r1), __dmul_rn((double)hit, r1));
}
// r1 and q of a trial of probability p (cached for inner trials)
__device__ __forceinline__ double2 trial_factors(double p, double r1_if_uncertain)
{
    return p >= 1.0 ? make_double2(1.0, 0.0) : make_double2(r1_if_uncertain, __dmul_rn(p, r1_if_uncertain));
}

// Score of one step for the rails of a warp (gradient pass).  Trials are
// grouped per (rail, zone): inner hops of a zone share p (scalar barrier), so
// their summed weight needs only the counts of performed and accepted trials
// from the step-start masks ow, fR, fL and the accepted-trial masks; the
// electrode trials of the two boundary sites are added one by one.  Lane sl
// of rail slot seg takes zones sl, sl + W2, ... (W2, a power of two <= LPR,
// lanes per rail take part) and returns its own zones' Ws, the summed
// inner-trial weight (times d ln P0 / d theta it is the Ea and nu score), and
// Ks, the kappa score with d ln p / d kappa = (s - B/(1+B)) d ln B / d kappa
// (s = 1 right, 0 left); Es, the innovation of the rail's current (left
// trials' a - p minus right trials' a - p), is summed over the rail's lanes
// (and left at zero when the current carries no weight).  The per-zone probabilities (Eqs. 3-6, FP64) are cached until the rail's
// zone counts or V change.  With the exp tables,
//   B_z = exp(gXV V) exp(gXV ka D'_z) exp(cm m_z),  m_z = L (Pb_z + Pb_z+1) - F,
// three factors of which only the last changes with the zone counts, looked
// up by the integer m_z; the probabilities and the reciprocals 1/(1+B),
// 1/(1-p_R), 1/(1-p_L) then take one FP64 reciprocal.
template <int LPR, int WPL>
__device__ __forceinline__ void grad_step_score(const SweepArgs &a, const WarpSmem<LPR, WPL> &S,
                                                uint32_t t, int nact, bool open, int seg, int sl,
                                                int W2, double gInvL, double gXV, double gKC,
                                                double &Ws, double &Ks, double &Es)
{
    const int L = a.L, Z = a.Z;
    const DevConst &K = *a.K;
    const double V = a.V[t];
    const bool act = seg < nact;
    const bool wantE = a.wJ != nullptr;   // the innovation pairs with the current's weight only
    // A. is the rail's cache stale (V or a zone count changed)?  The rail's
    //    lanes compare the prefix counts side by side; a ballot joins them.
    bool changed;
    {
        const int32_t *Pb = S.Pb() + seg * (Z + 1);
        int32_t *Pc = S.gPb() + seg * (Z + 2);
        double *rs = S.gS() + seg * 16;
        bool diff = false;
        if (act) {
            for (int z = sl; z <= Z; z += LPR) diff |= Pb[z] != Pc[z];
            if (sl == 0) diff |= !same_bits(rs[6], V);
        }
        const uint32_t mine = LPR == 32 ? FULL : (((1u << (LPR & 31)) - 1u) << (seg * LPR));
        changed = (__ballot_sync(FULL, diff) & mine) != 0u;
        if (changed) {
            for (int z = sl; z <= Z; z += LPR) Pc[z] = Pb[z];
            if (sl == 0) {
                if (!same_bits(rs[6], V)) rs[15] = exp(__dmul_rn(gXV, V));   // exp(gXV V)
                rs[6] = V;
            }
        }
    }
    __syncwarp();
    double Wp = 0.0, Kp = 0.0, Ep = 0.0;
    if (act && sl < W2) {
        double *rs = S.gS() + seg * 16;
        for (int z = sl; z < Z; z += W2) {
            const int pi = seg * Z + z;
            if (changed) {
                // Q_z - Qbar (S2.1.8) = m_z / (2 L) - D'_z with the integer
                // m_z = L (Pb_z + Pb_z+1) - F, F = sum_z w_z (Pb_z + Pb_z+1)
                const int32_t *Pb = S.Pb() + seg * (Z + 1);
                const int m = L * (Pb[z] + Pb[z + 1]) - S.Fs()[seg];
                const double dq = __fma_rn(0.5 * gInvL, (double)m, -S.gCz()[pi]);
                double B;                                             // Eqs. 3-4
                if (a.etL != nullptr && fabs(__dmul_rn(gXV, V)) < 600.0) {
                    const int u = m + a.etM;
                    B = __dmul_rn(__dmul_rn(rs[15], S.gEe()[pi]),
                                  __dmul_rn(__ldg(a.etH + (u >> 10)), __ldg(a.etL + (u & 1023))));
                } else {
                    B = exp(__dmul_rn(__fma_rn(-K.ka, dq, V), gXV));
                }
                const double c = __dmul_rn(gKC, dq);                 // d ln B / d kappa
                // x1 = 1 + B; y2 = x1 (1 - p_R), y3 = x1 (1 - p_L) with p_L = P0 / x1
                const double x1 = __dadd_rn(1.0, B);
                const double y2 = __fma_rn(-K.P0, B, x1), y3 = __dsub_rn(x1, K.P0);
                const double y23 = __dmul_rn(y2, y3);
                double inv, pL, pR;
                const double xd = __dmul_rn(x1, y23);
                if (inside_bits(xd, 1e-300, 1e300)) {                  // both trials uncertain
                    const double rp = recip_newton(xd);                // 1 / (x1 y2 y3)
                    const double x1rp = __dmul_rn(x1, rp), x1x1rp = __dmul_rn(x1, x1rp);
                    inv = __dmul_rn(y23, rp);
                    pL = __dmul_rn(K.P0, inv);                          // Eq. 5
                    pR = __dmul_rn(pL, B);                              // Eq. 6
                    const double r1R = __dmul_rn(y3, x1x1rp), r1L = __dmul_rn(y2, x1x1rp);  // x1/y2, x1/y3
                    S.gR1()[pi] = make_double2(r1R, r1L);
                    S.gPQ()[pi] = make_double2(__dmul_rn(pR, r1R), __dmul_rn(pL, r1L));
                } else {                                               // a certain trial, or B out of range
                    inv = __drcp_rn(x1);
                    pL = __dmul_rn(K.P0, inv);
                    pR = __dmul_rn(pL, B);
                    const double2 fR = trial_factors(pR, pR < 1.0 ? __drcp_rn(__dsub_rn(1.0, pR)) : 0.0);
                    const double2 fL = trial_factors(pL, pL < 1.0 ? __drcp_rn(__dsub_rn(1.0, pL)) : 0.0);
                    S.gR1()[pi] = make_double2(fR.x, fL.x);
                    S.gPQ()[pi] = make_double2(fR.y, fL.y);
                }
                S.gP()[pi] = make_double2(pR, pL);
                // d ln p / d kappa: right (1 - B/(1+B)) c = inv c, left -(B/(1+B)) c = inv c - c
                const double dkR = __dmul_rn(inv, c);
                S.gDK()[pi] = make_double2(dkR, __dsub_rn(dkR, c));
                if (open && z == 0) {
                    const double pin = __dmul_rn(__dmul_rn(K.E_in, inv), B);   // injection into 0
                    const double pout = __dmul_rn(K.E_out, inv);               // extraction at 0
                    rs[7] = pin;
                    rs[8] = pout;
                    rs[11] = pin < 1.0 ? __drcp_rn(__dsub_rn(1.0, pin)) : 0.0;
                    rs[12] = pout < 1.0 ? __drcp_rn(__dsub_rn(1.0, pout)) : 0.0;
                }
                if (open && z == Z - 1) {
                    const double pout = __dmul_rn(__dmul_rn(K.E_out, inv), B);  // extraction at L-1
                    const double pin = __dmul_rn(K.E_in, inv);                  // injection into L-1
                    rs[9] = pout;
                    rs[10] = pin;
                    rs[13] = pout < 1.0 ? __drcp_rn(__dsub_rn(1.0, pout)) : 0.0;
                    rs[14] = pin < 1.0 ? __drcp_rn(__dsub_rn(1.0, pin)) : 0.0;
                }
            }
            // inner trials of the zone's sites [lo, hi); at an open rail the
            // outward trials of sites 0 and L-1 are electrode trials, below
            const int lo = K.bnd[z], hi = K.bnd[z + 1];
            int nR = 0, nL = 0, aR = 0, aL = 0;
            for (int w = lo >> 5; w <= (hi - 1) >> 5; ++w) {
                const int s0 = 32 * w;
                uint32_t m = FULL;
                if (lo > s0) m &= FULL << (lo - s0);
                if (hi < s0 + 32) m &= (1u << (hi - s0)) - 1u;
                const int idx = seg * LPR * WPL + w;
                const uint32_t o = S.ow()[idx] & m;
                uint32_t fR = S.fR()[idx], fL = S.fL()[idx];
                if (open) {
                    if (L - 1 >= s0 && L - 1 < s0 + 32) fR &= ~(1u << ((L - 1) - s0));
                    if (s0 == 0) fL &= ~1u;
                }
                nR += __popc(o & fR);
                nL += __popc(o & fL);
                aR += __popc(o & fR & S.accR()[idx]);
                aL += __popc(o & fL & S.accL()[idx]);
            }
            if (nR | nL) {
                const double2 p = S.gP()[pi], r1 = S.gR1()[pi], q = S.gPQ()[pi], dk = S.gDK()[pi];
                const double wR = trial_weight(aR, nR, r1.x, q.x);
                const double wL = trial_weight(aL, nL, r1.y, q.y);
                Wp = __dadd_rn(Wp, __dadd_rn(wR, wL));
                Kp = __fma_rn(wR, dk.x, __fma_rn(wL, dk.y, Kp));
                // left trials' a - p minus right trials' a - p: the integer part
                // aL - aR and nR p_R - nL p_L
                if (wantE)
                    Ep = __dadd_rn(Ep, __fma_rn((double)nR, p.x,
                                                __fma_rn(-(double)nL, p.y, (double)(aL - aR))));
            }
            if (open && z == 0) {
                const double dkR = S.gDK()[pi].x, dkL = S.gDK()[pi].y;
                const int idx = seg * LPR * WPL;
                if (S.ow()[idx] & 1u) {        // extraction through the left electrode
                    const int hit = (S.accL()[idx] & 1u) ? 1 : 0;
                    Kp = __fma_rn(et_weight(hit, rs[8], rs[12]), dkL, Kp);
                    if (wantE) Ep = __dadd_rn(Ep, __dsub_rn((double)hit, rs[8]));
                } else {                       // injection into site 0
                    const int hit = (S.accR()[idx] & 1u) ? 1 : 0;
                    Kp = __fma_rn(et_weight(hit, rs[7], rs[11]), dkR, Kp);
                    if (wantE) Ep = __dsub_rn(Ep, __dsub_rn((double)hit, rs[7]));
                }
            }
            if (open && z == Z - 1) {
                const double dkR = S.gDK()[pi].x, dkL = S.gDK()[pi].y;
                const int idx = seg * LPR * WPL + ((L - 1) >> 5);
                const uint32_t bit = 1u << ((L - 1) & 31);
                if (S.ow()[idx] & bit) {       // extraction through the right electrode
                    const int hit = (S.accR()[idx] & bit) ? 1 : 0;
                    Kp = __fma_rn(et_weight(hit, rs[9], rs[13]), dkR, Kp);
                    if (wantE) Ep = __dsub_rn(Ep, __dsub_rn((double)hit, rs[9]));
                } else {                       // injection into site L-1
                    const int hit = (S.accL()[idx] & bit) ? 1 : 0;
                    Kp = __fma_rn(et_weight(hit, rs[10], rs[14]), dkL, Kp);
                    if (wantE) Ep = __dadd_rn(Ep, __dsub_rn((double)hit, rs[10]));
                }
            }
        }
    }
    // the rail's innovation, summed over its W2 zone lanes
    if (wantE)
        for (int off = W2 >> 1; off >= 1; off >>= 1) Ep = __dadd_rn(Ep, __shfl_xor_sync(FULL, Ep, off, W2));
    Ws = Wp;
    Ks = Kp;
    Es = Ep;
}

template <int LPR, int WPL, bool ACC, bool GRAD = false>
// One CTA's tile of rails advanced through steps [t0, t0 + n_steps): the whole
// sweep of S2.1.2 - S2.1.7 for rails [tile_rail0, tile_rail0 + G * warps).
// `a` describes one device (in the kernel's parameter space for a single
// device, in shared memory for a batch); rk0 / rk1 are the Philox round keys.
// ACC adds accept-sure bounds to the zone tables and decides inner hops whose
// draw is not rejected outright inside the draw loop; it pays when hop
// probabilities are large (P0 of order 1e-2 and above), where most steps
// carry several such draws per warp, and costs a few per cent otherwise.
__device__ __forceinline__ void sweep_tile(const SweepArgs &a, const uint32_t *rk0,
                                           const uint32_t *rk1, int64_t t0, int n_steps,
                                           int flush, int64_t tile_rail0, uint8_t *smem)
{
    constexpr int G = 32 / LPR;
    constexpr int VWIN = 32;              // steps per voltage window of the FP32 bounds
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int seg = lane / LPR;
    const int sl = lane % LPR;
    const int wbase = sl * WPL;
    const int L = a.L, Z = a.Z;
    const uint32_t instance = a.instance;
    const bool open = a.electrodes == 1;
    const bool persite = a.P0bnd != nullptr;
    const int64_t rail0 = tile_rail0 + (int64_t)warp * G;
    const int64_t rail = rail0 + seg;
    // Philox counter word 1 of the warp's first rail: the global rail index
    const uint32_t prail0 = a.rail_base + (uint32_t)rail0;
    const bool active = rail < a.R;
    const int nact = (int)max((int64_t)0, min((int64_t)G, (int64_t)a.R - rail0));

    using Ly = Layout<LPR, WPL>;
    const size_t wb0 = Ly::bytes(Z, ACC);
    const size_t wb = wb0 + (GRAD ? Ly::grad_bytes(Z) : 0);
    WarpSmem<LPR, WPL> S;
    S.b = smem + (size_t)warp * wb;
    S.rz = (uint32_t)Ly::rm_bytes(Z, ACC);
    S.gz = (uint32_t)Ly::gz8(Z);
    S.pbz = (uint32_t)Ly::pb_bytes(Z);
    S.npo = (uint32_t)(Ly::FIXED + S.rz + 2 * S.gz + Ly::pb_only(Z));
    S.goff = (uint32_t)wb0;
    S.gzq = (uint32_t)align16((size_t)8 * G * Z);
    uint8_t *zone_tab = smem + (size_t)nwarps * wb;

    // ---- per-CTA tables and per-warp staging
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        int z = 0;
        while (a.bnd[z + 1] <= k) ++z;
        zone_tab[k] = (uint8_t)z;
    }
    for (int pi = lane; pi < G * Z; pi += 32) S.Np()[pi] = 0;
    if (lane == 0) {
        S.cnt()[0] = 0;
        S.cnt()[1] = 0;
        S.band() = make_float2(1.0f - a.delta, 1.0f + a.delta);
    }
    for (int i = lane; i < 32 * WPL; i += 32) {
        S.mvR()[i] = 0;
        S.mvL()[i] = 0;
        if constexpr (GRAD) {
            S.accR()[i] = 0;
            S.accL()[i] = 0;
        }
    }
    // gradient pass: lanes per rail that take zones (a power of two <= LPR)
    int gW2 = 1;
    while (gW2 < Z && gW2 < LPR) gW2 <<= 1;
    // 1 / L; dV_z -> ln B_z = -dV_z d / (t_dev kT) (Eqs. 3-4); dq -> d ln B_z / d kappa
    double gInvL = 0.0, gXV = 0.0, gKC = 0.0;
    // gradient pass: this lane's share of the rail's cumulative inner-trial
    // weight W, kappa score K and estimator sums G_W, G_K (its zones' terms;
    // the rail's values are the sums over its lanes, formed at the end)
    double aW = 0.0, aK = 0.0, aGW = 0.0, aGK = 0.0;
    if constexpr (GRAD) {
        gInvL = 1.0 / (double)L;
        gXV = -(a.K->d / a.K->t_dev) / a.K->kT;
        gKC = (a.alpha * a.K->d) / a.tdev_kT;
        // D'_z = D_z - sum_z' w_z' D_z' / L with D_z = sum_{z'<z} c_z' + c_z / 2,
        // c_z = N0 w_z / L: the background part of Q_z - Qbar, fixed per rail
        if (sl == 0) {
            const int32_t n0 = active ? a.N0[rail] : 0;
            double run = 0.0, acc = 0.0;
            for (int z = 0; z < Z; ++z) {
                const int w = a.bnd[z + 1] - a.bnd[z];
                const double cz = ((double)n0 * (double)w) / (double)L;
                const double D = run + 0.5 * cz;
                run += cz;
                acc += (double)w * D;
                S.gCz()[seg * Z + z] = D;
            }
            const double mean = acc / (double)L;
            for (int z = 0; z < Z; ++z) {
                S.gCz()[seg * Z + z] -= mean;
                // the background factor exp(gXV ka D'_z) of B_z (exp tables)
                if (a.etL) S.gEe()[seg * Z + z] = exp(__dmul_rn(__dmul_rn(gXV, a.K->ka),
                                                                  S.gCz()[seg * Z + z]));
            }
        }
        if (sl == 0) S.gS()[seg * 16 + 6] = __longlong_as_double(0x7FF8000000000000ll);  // no cache
        if (sl == 0 && active) {
            const double *g0 = a.gstate + rail * kGradState;
            aW = g0[0];
            aK = g0[1];
            aGW = g0[2];
            aGK = g0[3];
            S.gS()[seg * 16 + 4] = g0[4];
        } else if (sl == 0) {
            S.gS()[seg * 16 + 4] = 0.0;
        }
    }
    for (int i = lane; i < 2 * G; i += 32) S.inj()[i] = 0;
    if (sl == 0) S.N0s()[seg] = active ? a.N0[rail] : 0;
    if (sl == 0) S.jr()[seg] = 0;
    if (persite) {
        for (int pi = lane; pi < G * Z; pi += 32) {
            const int64_t r2 = rail0 + pi / Z;
            S.P0b()[pi] = r2 < a.R ? a.P0bnd[r2 * Z + pi % Z] : make_float2(0.0f, 0.0f);
        }
    }

    // ---- the rail's occupancy words: read once from HBM, kept in shared memory
    //      (S.ow) for the whole launch; only the move phase changes them
    {
        const uint8_t *row = a.occ + (active ? rail : 0) * a.stride;
#pragma unroll
        for (int j = 0; j < WPL; ++j) {
            const int s0 = 32 * (wbase + j);
            uint32_t bits = 0;
            if (active) {
                if (s0 < a.stride) bits |= pack16(*(const uint4 *)(row + s0));
                if (s0 + 16 < a.stride) bits |= pack16(*(const uint4 *)(row + s0 + 16)) << 16;
            }
            S.ow()[seg * LPR * WPL + wbase + j] = bits & valid_mask(s0, L);
        }
    }
    // interior zone boundaries z in [zlo, zhi] that lie in this lane's words,
    // packed as zlo | zhi << 8
    int zb = 1;
    {
        const int lo = 32 * wbase, hi = 32 * (wbase + WPL);
        int zlo = 1, zhi = 0;
        bool first = true;
        for (int z = 1; z < Z; ++z) {
            const int b = a.bnd[z];
            if (b >= lo && b < hi) {
                if (first) {
                    zlo = z;
                    first = false;
                }
                zhi = z;
            }
        }
        zb = zlo | (zhi << 8);
    }
    bool dirty = true;      // occupancy changed since the candidate list was built
    int n_inner = 0, nlist = 0;
    __syncthreads();

    for (int c0 = 0; c0 < n_steps; c0 += flush) {
        const int c1 = min(n_steps, c0 + flush);
        for (int s = c0; s < c1; ++s) {
            const uint32_t t = (uint32_t)(t0 + s);

            // the brick-wall rule's active bonds alternate: its candidates change
            // every step even when the occupancy does not
            const bool rebuilt = dirty || a.rule != 0;
            if (rebuilt) {
                uint32_t o[WPL];
#pragma unroll
                for (int j = 0; j < WPL; ++j) o[j] = S.ow()[seg * LPR * WPL + wbase + j];
                // ---- 1. zone counts: segmented scan of popcounts
                int cnt = 0;
#pragma unroll
                for (int j = 0; j < WPL; ++j) cnt += __popc(o[j]);
                int incl = cnt;
#pragma unroll
                for (int off2 = 1; off2 < LPR; off2 <<= 1) {
                    const int v = __shfl_up_sync(FULL, incl, off2, LPR);
                    if (sl >= off2) incl += v;
                }
                const int excl = incl - cnt;
                const int total = __shfl_sync(FULL, incl, LPR - 1, LPR);
                int fpart = 0;
                for (int z = zb & 0xFF; z <= (zb >> 8); ++z) {
                    const int b = a.bnd[z];
                    const int j = (b >> 5) - wbase;
                    const uint32_t below = (1u << (b & 31)) - 1u;
                    int P = excl;
                    if (WPL == 2) {
                        if (j == 1) P += __popc(o[0]) + __popc(o[WPL - 1] & below);
                        else P += __popc(o[0] & below);
                    } else {
                        P += __popc(o[0] & below);
                    }
                    S.Pb()[seg * (Z + 1) + z] = P;
                    fpart += P * a.wsum[z];
                }
                if (sl == 0) S.Pb()[seg * (Z + 1)] = 0;
                if (sl == LPR - 1) {
                    S.Pb()[seg * (Z + 1) + Z] = total;
                    fpart += total * a.wsum[Z];
                }
#pragma unroll
                for (int off2 = LPR / 2; off2 >= 1; off2 >>= 1)
                    fpart += __shfl_xor_sync(FULL, fpart, off2, LPR);
                if (sl == 0) S.Fs()[seg] = fpart;

                // ---- 3. candidates: occupied sites with a free neighbour; the two
                //         electrode sites of an open rail are listed separately
                uint32_t cand[WPL];
                {
                    uint32_t f[WPL];
#pragma unroll
                    for (int j = 0; j < WPL; ++j) f[j] = ~o[j] & valid_mask(32 * (wbase + j), L);
                    const uint32_t f_prev = __shfl_up_sync(FULL, f[WPL - 1], 1, LPR);
                    const uint32_t f_next = __shfl_down_sync(FULL, f[0], 1, LPR);
#pragma unroll
                    for (int j = 0; j < WPL; ++j) {
                        const uint32_t cp = j > 0 ? (f[j > 0 ? j - 1 : 0] >> 31)
                                                  : (sl > 0 ? (f_prev >> 31) : (open ? 1u : 0u));
                        const uint32_t cn = j < WPL - 1 ? (f[j < WPL - 1 ? j + 1 : 0] & 1u)
                                                        : (sl < LPR - 1 ? (f_next & 1u) : 0u);
                        const int s0 = 32 * (wbase + j);
                        const uint32_t firstm = first_mask(s0), lastm = last_mask(s0, L);
                        uint32_t fL = (f[j] << 1) | cp;
                        uint32_t fR = (f[j] >> 1) | (cn << 31);
                        if (open) fR |= lastm;
                        // brick-wall rule: only bonds (b, b+1) with b = t (mod 2) are
                        // active; a site of the parity of t faces its active bond on
                        // the right, the others on the left (site parity = bit parity)
                        bool inj0 = open, injL = open;
                        if (a.rule != 0) {
                            const uint32_t rmask = (t & 1u) ? 0xAAAAAAAAu : 0x55555555u;
                            fR &= rmask;
                            fL &= ~rmask;
                            inj0 = open && (t & 1u);                       // bond -1 active
                            injL = open && (((uint32_t)(L - 1) ^ t) & 1u) == 0u;  // bond L-1
                        }
                        // empty electrode sites: the right bit of site 0 and the left bit
                        // of site L-1 mark an injection trial, the other bits are clear
                        const uint32_t e0 = firstm & ~o[j], eL = lastm & ~o[j];
                        fR = (fR & ~(e0 | eL)) | (inj0 ? e0 : 0u);
                        fL = (fL & ~(e0 | eL)) | (injL ? eL : 0u);
                        const int wi = seg * LPR * WPL + wbase + j;
                        S.fR()[wi] = fR;
                        S.fL()[wi] = fL;
                        uint32_t c = o[j] & (fL | fR);
                        if (open) c &= ~(firstm | lastm);
                        cand[j] = active ? c : 0u;
                    }
                }

                // ---- 4. warp-wide compaction of candidates
                int nc = 0;
#pragma unroll
                for (int j = 0; j < WPL; ++j) nc += __popc(cand[j]);
                int ic = nc;
#pragma unroll
                for (int off2 = 1; off2 < 32; off2 <<= 1) {
                    const int v = __shfl_up_sync(FULL, ic, off2);
                    if (lane >= off2) ic += v;
                }
                int pos = ic - nc;
                n_inner = __shfl_sync(FULL, ic, 31);
#pragma unroll
                for (int j = 0; j < WPL; ++j) {
                    uint32_t m = cand[j];
                    const uint32_t base = (uint32_t)(32 * (wbase + j)) | ((uint32_t)seg << 11);
                    while (m) {
                        const uint32_t site = base + (uint32_t)(__ffs(m) - 1);
                        // with one rail per warp the rail-slot bits carry the zone
                        S.list()[pos++] = (uint16_t)(G == 1 ? site | ((uint32_t)zone_tab[site]
                                                                      << ListCode<LPR, WPL>::kShift)
                                                            : site);
                        m &= m - 1;
                    }
                }
                if (open && seg < nact) {
                    // electrode entries: rows G Z + 2 seg (site 0) and + 1 (site L-1)
                    // in the entry when it has room, else the rail slot
                    constexpr bool kRow = ListCode<LPR, WPL>::kRow;
                    const uint32_t r0 = kRow ? (uint32_t)(G * Z + 2 * seg) << ListCode<LPR, WPL>::kShift
                                             : (uint32_t)seg << 11;
                    const uint32_t r1 = kRow ? (uint32_t)(G * Z + 2 * seg + 1) << ListCode<LPR, WPL>::kShift
                                             : (uint32_t)seg << 11;
                    if (sl == 0) S.list()[n_inner + 2 * seg] = (uint16_t)r0;
#pragma unroll
                    for (int j = 0; j < WPL; ++j)
                        if (last_mask(32 * (wbase + j), L))
                            S.list()[n_inner + 2 * seg + 1] = (uint16_t)(r1 | (uint32_t)(L - 1));
                }
                nlist = n_inner + (open ? 2 * nact : 0);
                __syncwarp();
            }

            // ---- 2. field and FP32 decision bands per (rail, zone), valid for
            //         every step of the voltage window while the occupancy holds
            const bool win_start = (s & (VWIN - 1)) == 0;   // windows of VWIN steps from c0 = 0
            if (dirty || win_start) {
                if (win_start) {
                    const int win_end = min(s + VWIN, n_steps);
                    const int k = min(lane, win_end - 1 - s);
                    const double v = a.V[t + k];
                    float vlo = __double2float_rd(v), vhi = __double2float_ru(v);
#pragma unroll
                    for (int off2 = 16; off2 >= 1; off2 >>= 1) {
                        vlo = fminf(vlo, __shfl_xor_sync(FULL, vlo, off2));
                        vhi = fmaxf(vhi, __shfl_xor_sync(FULL, vhi, off2));
                    }
                    // Evaluating at the window's mid voltage moves the exponent x of
                    // Eq. 4 by at most h = (vhi - vlo) / (2 L kT); B/(1+B) and 1/(1+B)
                    // have logarithmic derivatives in [-1, 1] with respect to x, so
                    // both change by a factor within [e^-h, e^h].  FP32 evaluation
                    // errors (about 1e-5 relative for |x| <= 40) are covered by delta.
                    const float h = 0.5f * (vhi - vlo) * a.inv_LkT;
                    const float eh = __expf(h) * (1.0f + 1.0f / 65536.0f);
                    // every lane writes the same values and reads back its own
                    S.band() = make_float2((1.0f - a.delta) / eh, (1.0f + a.delta) * eh);
                    S.vmid_ref() = 0.5f * (vlo + vhi);
                }
                const float Vf = S.vmid_ref();
                const float2 band = S.band();
                const float flo = band.x, fhi = band.y;
                for (int pi = lane; pi < G * Z; pi += 32) {
                    const int g2 = pi / Z;
                    const int z = pi - g2 * Z;
                    float2 zf = make_float2(0.0f, 0.0f);
                    uint4 rm = make_uint4(FULL, FULL, 0u, 0u);
                    if (g2 < nact) {
                        const int Pz = S.Pb()[g2 * (Z + 1) + z];
                        const int Pz1 = S.Pb()[g2 * (Z + 1) + z + 1];
                        const float qd = 0.5f * ((float)(Pz + Pz1) - (float)S.Fs()[g2] * a.inv_L) -
                                         (float)S.N0s()[g2] * a.cz[z];
                        const float dV = Vf - a.ka_f * qd;
                        const float x = -dV * a.inv_LkT;
                        if (fabsf(x) <= 40.0f) {
                            const float B = __expf(x);
                            const float inv = __fdividef(1.0f, 1.0f + B);
                            float blo = a.P0f_scalar, bhi = a.P0f_scalar;
                            if (persite) {
                                const float2 pb = S.P0b()[pi];
                                blo = pb.x;
                                bhi = pb.y;
                            }
                            rm.x = rej_thr(bhi * inv * B * fhi);
                            rm.y = rej_thr(bhi * inv * fhi);
                            if constexpr (ACC) {
                                rm.z = acc_thr(blo * inv * B * flo);
                                rm.w = acc_thr(blo * inv * flo);
                            }
                            zf = make_float2(B, inv);
                        }
                    }
                    // rm: reject-sure bounds for inner hops; (FULL, FULL) sends every
                    // draw of the zone to the slow path (zf == 0 marks it undecidable)
                    if constexpr (ACC) S.rm4()[pi] = rm;
                    else S.rm()[pi] = make_uint2(rm.x, rm.y);
                    S.zf()[pi] = zf;
                    if (open && g2 < nact && (z == 0 || z == Z - 1)) {
                        // reject-sure bounds of the electrode sites: an occupied site 0
                        // can hop right (inner) or leave left (extraction); an empty one
                        // can only receive an injection through its right draw.  Site
                        // L-1 mirrors this.  A bound of 0 marks a direction never tried.
                        const float sR = zf.y * zf.x, sL = zf.y;
                        const bool ok = zf.y > 0.0f;
                        const float bhi = persite ? S.P0b()[pi].y : a.P0f_scalar;
                        const float Ein = a.E_inf, Eout = a.E_outf;
                        if (z == 0) {
                            const bool occ0 = (S.ow()[g2 * LPR * WPL] & 1u) != 0;
                            uint2 e = occ0 ? make_uint2(rej_thr(bhi * sR * fhi), rej_thr(Eout * sL * fhi))
                                           : make_uint2(rej_thr(Ein * sR * fhi), 0u);
                            if (!ok) e = make_uint2(FULL, FULL);
                            if constexpr (ACC) S.rm4()[G * Z + 2 * g2] = make_uint4(e.x, e.y, 0u, 0u);
                            else S.rm()[G * Z + 2 * g2] = e;
                        }
                        if (z == Z - 1) {
                            const int wl = g2 * LPR * WPL + ((L - 1) >> 5);
                            const bool occl = (S.ow()[wl] >> ((L - 1) & 31)) & 1u;
                            uint2 e = occl ? make_uint2(rej_thr(Eout * sR * fhi), rej_thr(bhi * sL * fhi))
                                           : make_uint2(0u, rej_thr(Ein * sL * fhi));
                            if (!ok) e = make_uint2(FULL, FULL);
                            if constexpr (ACC) S.rm4()[G * Z + 2 * g2 + 1] = make_uint4(e.x, e.y, 0u, 0u);
                            else S.rm()[G * Z + 2 * g2 + 1] = e;
                        }
                    }
                }
                __syncwarp();
            }

            // ---- zone counts of the step-start occupancy into the trace, as
            //      changes (the launch's first step: the counts themselves):
            //      they can only change when the occupancy was rebuilt, and a
            //      prefix sum over the launch's steps (zone_scan) turns them
            //      into counts
            if constexpr (!GRAD) {
                if (rebuilt) {
                    for (int pi = lane; pi < G * Z; pi += 32) {
                        const int g2 = pi / Z;
                        const int z = pi - g2 * Z;
                        const int nz = S.Pb()[g2 * (Z + 1) + z + 1] - S.Pb()[g2 * (Z + 1) + z];
                        const int dz = nz - S.Np()[pi];
                        if (dz != 0) {
                            atomicAdd(&a.Zc[(t0 + s) * Z + z], (unsigned long long)(long long)dz);
                            S.Np()[pi] = nz;
                        }
                    }
                }
            }
            if (lane == 0) {
                S.ndef()[0] = 0;
                S.cnt()[0] += (uint32_t)nlist;
            }
            __syncwarp();

            // ---- 5. draws: one Philox block per lane per iteration; everything
            //         but the reject-sure (and, with ACC, the accept-sure) test
            //         is on the slow path
            bool moved = false;
            if constexpr (ACC) {
                for (int i0 = lane; i0 < nlist; i0 += 32 * kDrawIlpAcc) {
                    uint32_t xy[kDrawIlpAcc], xw[kDrawIlpAcc];
                    uint4 th[kDrawIlpAcc];
                    int sites[kDrawIlpAcc], gs[kDrawIlpAcc];
                    bool at[kDrawIlpAcc];
#pragma unroll
                    for (int q = 0; q < kDrawIlpAcc; ++q) {
                        const int i = i0 + 32 * q;
                        const bool has = i < nlist;
                        const uint16_t d = S.list()[has ? i : i0];
                        const int site = d & ListCode<LPR, WPL>::kSite, g = G == 1 ? 0 : d >> 11;
                        const uint4 x = philox((uint32_t)site, prail0 + (uint32_t)g, t, instance,
                                               rk0, rk1);
                        const int ts = ListCode<LPR, WPL>::kRow
                                           ? (int)(d >> ListCode<LPR, WPL>::kShift)
                                           : (i >= n_inner ? G * Z + (i - n_inner)
                                                           : (G == 1 ? (d >> 11) : g * Z + zone_tab[site]));
                        th[q] = S.rm4()[ts];
                        xy[q] = x.y;
                        xw[q] = x.w;
                        sites[q] = site;
                        gs[q] = g;
                        at[q] = has && (x.y <= th[q].x || x.w <= th[q].y);
                    }
#pragma unroll
                    for (int q = 0; q < kDrawIlpAcc; ++q) {
                        if (!at[q]) continue;
                        const int i = i0 + 32 * q;
                        bool slow = i >= n_inner;   // electrode sites
                        if (!slow) {
                            // inner hop (the site is occupied): accept-sure and
                            // reject-sure bounds of the zone and the free neighbours
                            const int idx = gs[q] * LPR * WPL + (sites[q] >> 5);
                            const uint32_t bit = 1u << (sites[q] & 31);
                            const bool tR = (S.fR()[idx] & bit) != 0;
                            const bool tL = (S.fL()[idx] & bit) != 0;
                            const int dR = tR ? (xy[q] < th[q].z ? 1 : (xy[q] > th[q].x ? 0 : 2)) : 0;
                            const int dL = tL ? (xw[q] < th[q].w ? 1 : (xw[q] > th[q].y ? 0 : 2)) : 0;
                            if constexpr (GRAD) {
                                if (dR != 2 && dL != 2) {
                                    if (dR == 1) atomicOr(&S.accR()[idx], bit);
                                    if (dL == 1) atomicOr(&S.accL()[idx], bit);
                                }
                            }
                            if (dR == 2 || dL == 2) {
                                slow = true;        // per-site refinement or the exact pass
                            } else if (dR == 1 && dL != 1) {
                                atomicOr(&S.mvR()[idx], bit);
                                moved = true;
                            } else if (dL == 1 && dR != 1) {
                                atomicOr(&S.mvL()[idx], bit);
                                moved = true;
                            }                       // both accepted: the ion stays
                        }
                        if (slow)
                            moved |= slow_candidate<LPR, WPL, GRAD>(S, a.self, i, n_inner, rail0, t,
                                                              zone_tab, persite, false, xy[q], xw[q]);
                    }
                }
            } else {
                for (int i0 = lane; i0 < nlist; i0 += 32 * kDrawIlpReject) {
                    // kDrawIlpReject independent Philox blocks per lane per iteration
                    uint32_t xy[kDrawIlpReject], xw[kDrawIlpReject];
                    bool at[kDrawIlpReject];
    #pragma unroll
                    for (int q = 0; q < kDrawIlpReject; ++q) {
                        const int i = i0 + 32 * q;
                        const bool has = i < nlist;
                        const uint16_t d = S.list()[has ? i : i0];
                        // with one rail per warp the rail slot is 0: the rail, step and
                        // instance words are then warp-uniform and the compiler hoists
                        // the parts of the first two Philox rounds that depend only on them
                        const int site = d & ListCode<LPR, WPL>::kSite, g = G == 1 ? 0 : d >> 11;
                        const uint4 x = philox((uint32_t)site, prail0 + (uint32_t)g, t, instance,
                                               rk0, rk1);
                        // electrode sites have their own rows after the G Z zone rows
                        const int ts = ListCode<LPR, WPL>::kRow
                                           ? (int)(d >> ListCode<LPR, WPL>::kShift)
                                           : (i >= n_inner ? G * Z + (i - n_inner)
                                                           : (G == 1 ? (d >> 11) : g * Z + zone_tab[site]));
                        const uint2 rm = S.rm()[ts];
                        xy[q] = x.y;
                        xw[q] = x.w;
                        at[q] = has && (x.y <= rm.x || x.w <= rm.y);
                    }
    #pragma unroll
                    for (int q = 0; q < kDrawIlpReject; ++q)
                        if (at[q])
                            moved |= slow_candidate<LPR, WPL, GRAD>(S, a.self, i0 + 32 * q, n_inner, rail0, t,
                                                              zone_tab, persite, false, xy[q], xw[q]);
                }
            }
            __syncwarp();

            // ---- 5b. exact FP64 resolution of undecided candidates (rare)
            const int nd = S.ndef()[0];
            if (nd > 0) {
                const bool overflow = nd > kDeferCap;
                const int cnt2 = overflow ? nlist : nd;
                for (int k = lane; k < cnt2; k += 32) {
                    const int i = overflow ? k : (int)S.def()[k];
                    moved |= slow_candidate<LPR, WPL, GRAD>(S, a.self, i, n_inner, rail0, t, zone_tab,
                                                      persite, true, 0u, 0u);
                }
            }

            // ---- 5c. gradient pass: score of this step's trials
            if constexpr (GRAD) {
                __syncwarp();
                double Ws, Ks, Es;
                grad_step_score<LPR, WPL>(a, S, t, nact, open, seg, sl, gW2, gInvL, gXV, gKC,
                                          Ws, Ks, Es);
                // coefficient of the score before this step: the zone counts at
                // the start of step t, less the current's innovation (a control
                // variate of zero mean); formed by the rail's first lane, applied
                // by every lane to its share of the score
                double d = 0.0;
                if (sl == 0 && seg < nact) {
                    // zones outside [lo, hi) have zero weight and add nothing;
                    // a step without weights has a zero share
                    const int zr = a.fZa ? a.fZr[t] : 0;
                    if (zr != 0) {
                        double fZ = -a.fZb[t];
                        for (int z = zr & 255; z < (zr >> 8); ++z) {
                            const int nz = S.Pb()[seg * (Z + 1) + z + 1] - S.Pb()[seg * (Z + 1) + z];
                            fZ = __fma_rn(a.fZa[(int64_t)t * Z + z], (double)nz, fZ);
                        }
                        d = fZ;
                    }
                    if (a.wJ) d = __fma_rn(-a.wJ[t], Es, d);
                    if (nonzero_bits(d)) S.gS()[seg * 16 + 4] = __dadd_rn(S.gS()[seg * 16 + 4], d);   // G_1
                }
                d = __shfl_sync(FULL, d, 0, LPR);
                if (nonzero_bits(d)) {
                    aGW = __fma_rn(d, aW, aGW);
                    aGK = __fma_rn(d, aK, aGK);
                }
                aW = __dadd_rn(aW, Ws);
                aK = __dadd_rn(aK, Ks);
#pragma unroll
                for (int j = 0; j < WPL; ++j) {
                    S.accR()[seg * LPR * WPL + wbase + j] = 0u;
                    S.accL()[seg * LPR * WPL + wbase + j] = 0u;
                }
            }

            // ---- 6. conflicts, synchronous update, current
            int Jrail = 0;   // this rail's J_t (gradient pass)
            dirty = __any_sync(FULL, moved);
            if (dirty) {
                __syncwarp();
                uint32_t mR[WPL], mL[WPL], tR[WPL], tL[WPL], cf[WPL];
#pragma unroll
                for (int j = 0; j < WPL; ++j) {
                    mR[j] = S.mvR()[seg * LPR * WPL + wbase + j];
                    mL[j] = S.mvL()[seg * LPR * WPL + wbase + j];
                }
                const int iR = S.inj()[seg], iL = S.inj()[G + seg];
                const uint32_t mR_prev = __shfl_up_sync(FULL, mR[WPL - 1], 1, LPR);
                const uint32_t mL_next = __shfl_down_sync(FULL, mL[0], 1, LPR);
#pragma unroll
                for (int j = 0; j < WPL; ++j) {
                    const uint32_t cp = j > 0 ? (mR[j > 0 ? j - 1 : 0] >> 31)
                                              : (sl > 0 ? (mR_prev >> 31) : (iR ? 1u : 0u));
                    const uint32_t cn = j < WPL - 1 ? (mL[j < WPL - 1 ? j + 1 : 0] & 1u)
                                                    : (sl < LPR - 1 ? (mL_next & 1u) : 0u);
                    const int s0 = 32 * (wbase + j);
                    const uint32_t vm = valid_mask(s0, L);
                    tR[j] = ((mR[j] << 1) | cp) & vm;
                    tL[j] = ((mL[j] >> 1) | (cn << 31)) & vm;
                    if (iL) tL[j] |= last_mask(s0, L);
                    cf[j] = tR[j] & tL[j];
                }
                const uint32_t c_prev = __shfl_up_sync(FULL, cf[WPL - 1], 1, LPR);
                const uint32_t c_next = __shfl_down_sync(FULL, cf[0], 1, LPR);
                int Jl = 0, nm = 0;
#pragma unroll
                for (int j = 0; j < WPL; ++j) {
                    const int s0 = 32 * (wbase + j);
                    const uint32_t lastm = last_mask(s0, L);
                    const int wi = seg * LPR * WPL + wbase + j;
                    const uint32_t cn = j < WPL - 1 ? (cf[j < WPL - 1 ? j + 1 : 0] & 1u)
                                                    : (sl < LPR - 1 ? (c_next & 1u) : 0u);
                    const uint32_t cp = j > 0 ? (cf[j > 0 ? j - 1 : 0] >> 31)
                                              : (sl > 0 ? (c_prev >> 31) : 0u);
                    mR[j] &= ~((cf[j] >> 1) | (cn << 31));
                    mL[j] &= ~((cf[j] << 1) | cp);
                    tR[j] &= ~cf[j];
                    tL[j] &= ~cf[j];
                    Jl += __popc(mL[j]) - __popc(mR[j]);
                    S.ow()[wi] = (S.ow()[wi] & ~(mR[j] | mL[j])) | tR[j] | tL[j];
                    nm += __popc(mR[j]) + __popc(mL[j]);
                    if (iR && s0 == 0 && !(cf[j] & 1u)) {            // injected at site 0
                        Jl -= 1;
                        nm += 1;
                    }
                    if (iL && lastm && !(cf[j] & lastm)) {           // injected at L-1
                        Jl += 1;
                        nm += 1;
                    }
                }
                nm = __reduce_add_sync(FULL, nm);
                if (lane == 0) S.cnt()[1] += (uint32_t)nm;
                __syncwarp();
#pragma unroll
                for (int j = 0; j < WPL; ++j) {
                    S.mvR()[seg * LPR * WPL + wbase + j] = 0u;
                    S.mvL()[seg * LPR * WPL + wbase + j] = 0u;
                }
                if (sl == 0) {
                    S.inj()[seg] = 0;
                    S.inj()[G + seg] = 0;
                }
                if constexpr (GRAD) {
                    int v = Jl;
#pragma unroll
                    for (int off2 = LPR / 2; off2 >= 1; off2 >>= 1)
                        v += __shfl_xor_sync(FULL, v, off2, LPR);
                    Jrail = v;
                } else {
                    const int Jw = __reduce_add_sync(FULL, Jl);
                    if (lane == 0 && Jw != 0)
                        atomicAdd(&a.J[t0 + s], (unsigned long long)(long long)Jw);
                    // per-rail current: the rail's own sum (the warp's when G == 1)
                    if (a.Jr) {
                        if (G == 1) {
                            if (lane == 0 && Jw != 0) S.jr()[0] += Jw;
                        } else {
                            int v = Jl;
#pragma unroll
                            for (int off2 = LPR / 2; off2 >= 1; off2 >>= 1)
                                v += __shfl_xor_sync(FULL, v, off2, LPR);
                            if (sl == 0 && v != 0) S.jr()[seg] += v;
                        }
                    }
                }
            }
            if constexpr (GRAD) {
                // the current of step t pairs with the score of steps <= t;
                // every lane of the rail holds its J_t (Jrail)
                if (a.wJ) {
                    const double2 ab = a.fJab[t];
                    if (nonzero_bits(ab.x) || nonzero_bits(ab.y)) {
                        const double fJ = __fma_rn(ab.x, (double)Jrail, -ab.y);
                        aGW = __fma_rn(fJ, aW, aGW);
                        aGK = __fma_rn(fJ, aK, aGK);
                        if (sl == 0 && seg < nact)
                            S.gS()[seg * 16 + 4] = __dadd_rn(S.gS()[seg * 16 + 4], fJ);
                    }
                }
            }
            __syncwarp();
        }
        // ---- flush this warp's counters and per-rail current (no CTA barrier:
        //      warps advance independently through the launch)
        if constexpr (GRAD) continue;
        if (lane == 0) {
            const uint32_t nd = S.cnt()[0], nmv = S.cnt()[1];
            if (nd) atomicAdd(&a.counters[0], (unsigned long long)nd);
            if (nmv) atomicAdd(&a.counters[2], (unsigned long long)nmv);
            S.cnt()[0] = 0;
            S.cnt()[1] = 0;
        }
        // the rail's current of this chunk (at most (L + 1) flush per rail: no
        // int32 overflow) into its int64 total; each rail belongs to one warp
        if (a.Jr && active && sl == 0) {
            const int v = S.jr()[seg];
            if (v != 0) a.Jr[rail] += v;
            S.jr()[seg] = 0;
        }
        __syncwarp();
    }

    if constexpr (GRAD) {
        // the rail's W, K, G_W, G_K: sums of its lanes' shares
#pragma unroll
        for (int off2 = LPR / 2; off2 >= 1; off2 >>= 1) {
            aW = __dadd_rn(aW, __shfl_xor_sync(FULL, aW, off2, LPR));
            aK = __dadd_rn(aK, __shfl_xor_sync(FULL, aK, off2, LPR));
            aGW = __dadd_rn(aGW, __shfl_xor_sync(FULL, aGW, off2, LPR));
            aGK = __dadd_rn(aGK, __shfl_xor_sync(FULL, aGK, off2, LPR));
        }
        if (active && sl == 0) {
            double *g0 = a.gstate + rail * kGradState;
            g0[0] = aW;
            g0[1] = aK;
            g0[2] = aGW;
            g0[3] = aGK;
            g0[4] = S.gS()[seg * 16 + 4];
        }
    }

    // ---- write the rail back
    if (active) {
        uint8_t *wrow = a.occ + rail * a.stride;
#pragma unroll
        for (int j = 0; j < WPL; ++j) {
            const int s0 = 32 * (wbase + j);
            const uint32_t o = S.ow()[seg * LPR * WPL + wbase + j];
            if (s0 < a.stride) *(uint4 *)(wrow + s0) = unpack16(o & 0xFFFFu);
            if (s0 + 16 < a.stride) *(uint4 *)(wrow + s0 + 16) = unpack16(o >> 16);
        }
    }
}

template <int LPR, int WPL, bool ACC>
// 4 CTAs of 256 threads per SM (64 registers) with the accept tables, 5 (48
// registers) without: the kernel is bound by instruction latency more than by
// any one pipe, and the extra resident warps outweigh the spills (mostly on
// the slow and exact paths) that the caps cause.  With 80 registers and 3 CTAs
// the hysteresis device runs 4.5 % slower.
__global__ void __launch_bounds__(256, ACC ? 4 : 5) sweep_kernel(const SweepArgs a)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int64_t tile_rail0 = (int64_t)blockIdx.x * (blockDim.x >> 5) * (32 / LPR);
    sweep_tile<LPR, WPL, ACC>(a, a.rk0, a.rk1, a.t0, a.n_steps, a.flush, tile_rail0, smem);
}

// Gradient pass: the forward sweep replayed from a checkpoint with the
// likelihood-ratio score accumulated per rail (3 CTAs of 256 threads per SM:
// 80 registers; 2 CTAs at 128 registers run 5 % slower, 4 at 64 no faster).
template <int LPR, int WPL>
__global__ void __launch_bounds__(256, 3) sweep_grad_kernel(const SweepArgs a)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int64_t tile_rail0 = (int64_t)blockIdx.x * (blockDim.x >> 5) * (32 / LPR);
    sweep_tile<LPR, WPL, true, true>(a, a.rk0, a.rk1, a.t0, a.n_steps, a.flush, tile_rail0, smem);
}

// Per-rail gradient terms (d/dEa, d/dnu, d/dkappa, d/drho) from the state.
__device__ __forceinline__ void rail_grad_terms(const double *gs, const int32_t *N0, int64_t r,
                                                int L, double fill, int has_rho, double cEa,
                                                double cnu, double v[4])
{
    const double *st = gs + r * kGradState;
    v[0] = __dmul_rn(cEa, st[2]);
    v[1] = __dmul_rn(cnu, st[2]);
    v[2] = st[3];
    v[3] = 0.0;
    if (has_rho) {
        // score of the rail's Bernoulli(fill) placement: (N0 - L fill) / (fill (1 - fill))
        const double s0 = __ddiv_rn(__dsub_rn((double)N0[r], __dmul_rn((double)L, fill)),
                                    __dmul_rn(fill, __dsub_rn(1.0, fill)));
        v[3] = __dmul_rn(s0, st[4]);
    }
}

// Deterministic sum of v over the 1024 threads of the block (result in thread 0).
__device__ __forceinline__ void block_sum4(double v[4], double (*part)[4])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 4; ++i)
        for (int off = 16; off >= 1; off >>= 1) v[i] = __dadd_rn(v[i], __shfl_down_sync(FULL, v[i], off));
    if (lane == 0)
        for (int i = 0; i < 4; ++i) part[warp][i] = v[i];
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        for (int i = 0; i < 4; ++i) {
            double x = lane < nw ? part[lane][i] : 0.0;
            for (int off = 16; off >= 1; off >>= 1) x = __dadd_rn(x, __shfl_down_sync(FULL, x, off));
            v[i] = x;
        }
    }
    __syncthreads();
}

// Sum over rails of the per-rail terms (out[0..3]) and their standard error
// sqrt(R / (R - 1) sum_r (G_r - mean)^2) (out[4..7]); one block, fixed order.
__global__ void __launch_bounds__(1024) grad_reduce_kernel(const double *gs, int64_t R,
                                                           const int32_t *N0, int L, double fill,
                                                           int has_rho, double cEa, double cnu,
                                                           double *out)
{
    __shared__ double part[32][4];
    __shared__ double mean[4];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t r = threadIdx.x; r < R; r += blockDim.x) {
        double v[4];
        rail_grad_terms(gs, N0, r, L, fill, has_rho, cEa, cnu, v);
        for (int i = 0; i < 4; ++i) acc[i] = __dadd_rn(acc[i], v[i]);
    }
    block_sum4(acc, part);
    if (threadIdx.x == 0)
        for (int i = 0; i < 4; ++i) {
            out[i] = acc[i];
            mean[i] = R > 0 ? __ddiv_rn(acc[i], (double)R) : 0.0;
        }
    __syncthreads();
    double sq[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t r = threadIdx.x; r < R; r += blockDim.x) {
        double v[4];
        rail_grad_terms(gs, N0, r, L, fill, has_rho, cEa, cnu, v);
        for (int i = 0; i < 4; ++i) {
            const double dv = __dsub_rn(v[i], mean[i]);
            sq[i] = __dadd_rn(sq[i], __dmul_rn(dv, dv));
        }
    }
    block_sum4(sq, part);
    if (threadIdx.x == 0)
        for (int i = 0; i < 4; ++i)
            out[4 + i] = R > 1 ? sqrt(__dmul_rn(__ddiv_rn((double)R, (double)(R - 1)), sq[i])) : 0.0;
}

// Batch of devices: one persistent launch per kernel shape (lanes per rail,
// words per lane), so that each shape gets the registers of its own tile
// body.  The launch's CTAs take (device, rail tile) items of that shape from
// the shape's own counter and run the tile body with the device's arguments
// copied to shared memory.  The step index lives in device memory so that the
// launches and their advance can be replayed as a CUDA graph.
template <bool ACC, int LPR, int WPL>
__global__ void __launch_bounds__(256, ACC ? 4 : 5) sweep_batch_kernel(const BatchArgs b)
{
    constexpr int kind = shape_kind(LPR, WPL);
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ SweepArgs ia;
    __shared__ int s_item;
    const int64_t t0 = *b.t0;
    const int first = b.cls_off[kind], end = b.cls_off[kind + 1];
    for (;;) {
        if (threadIdx.x == 0) s_item = first + (int)atomicAdd(b.work + kind, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= end) break;
        const BatchItem it = b.items[item];
        const uint32_t *src = (const uint32_t *)&b.inst[it.inst];
        for (int i = threadIdx.x; i < (int)(sizeof(SweepArgs) / 4); i += blockDim.x)
            ((uint32_t *)&ia)[i] = src[i];
        __syncthreads();
        sweep_tile<LPR, WPL, ACC>(ia, b.rk0, b.rk1, t0, b.n_steps, b.flush, it.tile_rail0, smem);
        __syncthreads();
    }
}

// Gradient passes of a batch of devices, one persistent launch per kernel
// shape: CTAs take (device, rail tile) items of that shape and replay that
// device's steps 0 .. n_steps-1 with its gradient-pass arguments (the same
// tile body as sweep_grad_kernel, at its 3 CTAs per SM).
template <int LPR, int WPL>
__global__ void __launch_bounds__(256, 3) sweep_batch_grad_kernel(const BatchArgs b)
{
    constexpr int kind = shape_kind(LPR, WPL);
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ SweepArgs ia;
    __shared__ int s_item;
    const int first = b.cls_off[kind], end = b.cls_off[kind + 1];
    for (;;) {
        if (threadIdx.x == 0) s_item = first + (int)atomicAdd(b.work + kind, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= end) break;
        const BatchItem it = b.items[item];
        const uint32_t *src = (const uint32_t *)&b.inst[it.inst];
        for (int i = threadIdx.x; i < (int)(sizeof(SweepArgs) / 4); i += blockDim.x)
            ((uint32_t *)&ia)[i] = src[i];
        __syncthreads();
        const int n = ia.n_steps;
        sweep_tile<LPR, WPL, true, true>(ia, b.rk0, b.rk1, 0, n, n, it.tile_rail0, smem);
        __syncthreads();
    }
}

// Zone-count traces of steps [t0, t0 + n): the sweep leaves there, for every
// step, the change of each zone's count (the first step: the counts), and an
// inclusive prefix sum over the steps turns them into counts.  One block per
// zone (blockIdx.x), 1,024 steps per pass.
__device__ __forceinline__ void scan_zone_trace(unsigned long long *Zc, int64_t t0, int n, int Z,
                                                int z)
{
    __shared__ long long part[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long carry = 0;
    for (int base = 0; base < n; base += 1024) {
        const int i = base + threadIdx.x;
        long long v = i < n ? (long long)Zc[(t0 + i) * Z + z] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const long long u = __shfl_up_sync(FULL, v, off);
            if (lane >= off) v += u;
        }
        if (lane == 31) part[warp] = v;
        __syncthreads();
        if (warp == 0) {
            long long w = part[lane];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const long long u = __shfl_up_sync(FULL, w, off);
                if (lane >= off) w += u;
            }
            part[lane] = w;
        }
        __syncthreads();
        if (warp > 0) v += part[warp - 1];
        if (i < n) Zc[(t0 + i) * Z + z] = (unsigned long long)(v + carry);
        carry += part[31];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) zone_scan_kernel(unsigned long long *Zc, int64_t t0, int n,
                                                         int Z)
{
    scan_zone_trace(Zc, t0, n, Z, blockIdx.x);
}

// The same for every device of a batch after a launch (grid: max Z x devices).
__global__ void __launch_bounds__(1024) batch_zone_scan_kernel(const BatchArgs b)
{
    const SweepArgs &ia = b.inst[blockIdx.y];
    if ((int)blockIdx.x >= ia.Z || ia.Zc == nullptr) return;
    scan_zone_trace(ia.Zc, *b.t0, b.n_steps, ia.Z, blockIdx.x);
}

// Advance the batch's step counter and re-arm the shapes' work counters.
__global__ void batch_advance_kernel(int64_t *t0, unsigned *work, int n_steps)
{
    if (blockIdx.x == 0) {
        if (threadIdx.x == 0) *t0 += n_steps;
        if (threadIdx.x < kShapeKinds) work[threadIdx.x] = 0u;
    }
}

template <int LPR, int WPL>
cudaError_t launch_t(const SweepArgs &a, const SweepLaunch &l, cudaStream_t s)
{
    if (l.acc) sweep_kernel<LPR, WPL, true><<<l.grid, l.warps * 32, l.smem, s>>>(a);
    else sweep_kernel<LPR, WPL, false><<<l.grid, l.warps * 32, l.smem, s>>>(a);
    return cudaGetLastError();
}

template <int LPR, int WPL>
cudaError_t grad_launch_t(const SweepArgs &a, const SweepLaunch &l, cudaStream_t s)
{
    sweep_grad_kernel<LPR, WPL><<<l.grid, l.warps * 32, l.smem, s>>>(a);
    return cudaGetLastError();
}

template <int LPR, int WPL>
cudaError_t smem_attr()
{
    cudaError_t e = cudaFuncSetAttribute(sweep_kernel<LPR, WPL, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(sweep_kernel<LPR, WPL, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(sweep_grad_kernel<LPR, WPL>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

// Philox-only throughput probe: the draw loop's Philox4x32-10 blocks and
// nothing else (counter (i, thread, 0, 0), the two high words consumed as in
// the draw loop), four independent blocks per iteration.  Measures the
// integer-pipe ceiling that the sweep's roofline refers to.
__global__ void __launch_bounds__(256) philox_probe_kernel(int iters, uint32_t k0, uint32_t k1,
                                                           uint32_t *sink)
{
    uint32_t rk0[10], rk1[10];
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        rk0[i] = k0 + 0x9E3779B9u * (uint32_t)i;
        rk1[i] = k1 + 0xBB67AE85u * (uint32_t)i;
    }
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 x = philox((uint32_t)(4 * it + q), tid, 0u, 0u, rk0, rk1);
            acc ^= x.y + x.w;
        }
    }
    if (acc == 0x12345678u) sink[tid] = acc;   // keeps the work; practically never stores
}

}  // namespace

size_t sweep_smem_bytes(int lpr, int wpl, int Z, int L, int warps, int flush, bool acc)
{
    size_t wb = 0;
    if (wpl == 2) wb = Layout<32, 2>::bytes(Z, acc);
    else if (lpr == 1) wb = Layout<1, 1>::bytes(Z, acc);
    else if (lpr == 2) wb = Layout<2, 1>::bytes(Z, acc);
    else if (lpr == 4) wb = Layout<4, 1>::bytes(Z, acc);
    else if (lpr == 8) wb = Layout<8, 1>::bytes(Z, acc);
    else if (lpr == 16) wb = Layout<16, 1>::bytes(Z, acc);
    else wb = Layout<32, 1>::bytes(Z, acc);
    (void)flush;   // the flush interval no longer needs shared memory
    return (size_t)warps * wb + align16((size_t)L);
}

size_t grad_smem_bytes(int lpr, int wpl, int Z, int L, int warps)
{
    size_t wb = 0;
    if (wpl == 2) wb = Layout<32, 2>::bytes(Z, true) + Layout<32, 2>::grad_bytes(Z);
    else if (lpr == 1) wb = Layout<1, 1>::bytes(Z, true) + Layout<1, 1>::grad_bytes(Z);
    else if (lpr == 2) wb = Layout<2, 1>::bytes(Z, true) + Layout<2, 1>::grad_bytes(Z);
    else if (lpr == 4) wb = Layout<4, 1>::bytes(Z, true) + Layout<4, 1>::grad_bytes(Z);
    else if (lpr == 8) wb = Layout<8, 1>::bytes(Z, true) + Layout<8, 1>::grad_bytes(Z);
    else if (lpr == 16) wb = Layout<16, 1>::bytes(Z, true) + Layout<16, 1>::grad_bytes(Z);
    else wb = Layout<32, 1>::bytes(Z, true) + Layout<32, 1>::grad_bytes(Z);
    return (size_t)warps * wb + align16((size_t)L);
}

cudaError_t grad_launch(const SweepArgs &a, const SweepLaunch &l, cudaStream_t s)
{
    if (l.wpl == 2) return grad_launch_t<32, 2>(a, l, s);
    switch (l.lpr) {
    case 1: return grad_launch_t<1, 1>(a, l, s);
    case 2: return grad_launch_t<2, 1>(a, l, s);
    case 4: return grad_launch_t<4, 1>(a, l, s);
    case 8: return grad_launch_t<8, 1>(a, l, s);
    case 16: return grad_launch_t<16, 1>(a, l, s);
    default: return grad_launch_t<32, 1>(a, l, s);
    }
}

// Calls f(lpr, wpl) with the lanes per rail and words per lane of shape kind
// k as integral constants (the tile body's template arguments).
template <class F>
cudaError_t with_shape(int k, F &&f)
{
    using std::integral_constant;
    switch (k) {
    case 0: return f(integral_constant<int, 1>(), integral_constant<int, 1>());
    case 1: return f(integral_constant<int, 2>(), integral_constant<int, 1>());
    case 2: return f(integral_constant<int, 4>(), integral_constant<int, 1>());
    case 3: return f(integral_constant<int, 8>(), integral_constant<int, 1>());
    case 4: return f(integral_constant<int, 16>(), integral_constant<int, 1>());
    case 5: return f(integral_constant<int, 32>(), integral_constant<int, 1>());
    default: return f(integral_constant<int, 32>(), integral_constant<int, 2>());
    }
}

cudaError_t batch_grad_launch(const BatchArgs &b, const BatchPlan &plan, int warps, cudaStream_t s)
{
    for (int k = 0; k < kShapeKinds; ++k) {
        if (plan.grid[k] <= 0) continue;
        const cudaError_t e = with_shape(k, [&](auto lpr, auto wpl) {
            constexpr int P = decltype(lpr)::value, Q = decltype(wpl)::value;
            sweep_batch_grad_kernel<P, Q><<<plan.grid[k], warps * 32, plan.smem[k], s>>>(b);
            return cudaGetLastError();
        });
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int batch_ctas_per_sm(int kind, int mode, int warps, size_t smem)
{
    int n = 0;
    const cudaError_t e = with_shape(kind, [&](auto lpr, auto wpl) {
        constexpr int P = decltype(lpr)::value, Q = decltype(wpl)::value;
        if (mode == 2)
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_batch_grad_kernel<P, Q>,
                                                                 warps * 32, smem);
        if (mode == 1)
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_batch_kernel<true, P, Q>,
                                                                 warps * 32, smem);
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_batch_kernel<false, P, Q>,
                                                             warps * 32, smem);
    });
    return e == cudaSuccess && n > 0 ? n : 1;
}

cudaError_t philox_probe(int grid, int iters, uint32_t *sink, cudaStream_t s)
{
    philox_probe_kernel<<<grid, 256, 0, s>>>(iters, 0x243F6A88u, 0x85A308D3u, sink);
    return cudaGetLastError();
}

cudaError_t grad_reduce(const double *gstate, int64_t R, const int32_t *N0, int L, double fill,
                        int has_rho, double cEa, double cnu, double *out, cudaStream_t s)
{
    grad_reduce_kernel<<<1, 1024, 0, s>>>(gstate, R, N0, L, fill, has_rho, cEa, cnu, out);
    return cudaGetLastError();
}

int sweep_pick_lpr(int L, int *wpl)
{
    if (L > 1024) {
        *wpl = 2;
        return 32;
    }
    *wpl = 1;
    int lpr = 1;
    while (32 * lpr < L) lpr <<= 1;
    return lpr;
}

cudaError_t sweep_set_smem_limits()
{
    cudaError_t e = cudaSuccess;
    cudaError_t r;
    if ((r = smem_attr<1, 1>()) != cudaSuccess) e = r;
    if ((r = smem_attr<2, 1>()) != cudaSuccess) e = r;
    if ((r = smem_attr<4, 1>()) != cudaSuccess) e = r;
    if ((r = smem_attr<8, 1>()) != cudaSuccess) e = r;
    if ((r = smem_attr<16, 1>()) != cudaSuccess) e = r;
    if ((r = smem_attr<32, 1>()) != cudaSuccess) e = r;
    if ((r = smem_attr<32, 2>()) != cudaSuccess) e = r;
    return e;
}

int sweep_kind(int lpr, int wpl)
{
    return shape_kind(lpr, wpl);
}

cudaError_t batch_set_smem_limit()
{
    for (int k = 0; k < kShapeKinds; ++k) {
        const cudaError_t e = with_shape(k, [](auto lpr, auto wpl) {
            constexpr int P = decltype(lpr)::value, Q = decltype(wpl)::value;
            const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
            cudaError_t r = cudaFuncSetAttribute(sweep_batch_kernel<false, P, Q>, attr, 200 * 1024);
            if (r == cudaSuccess) r = cudaFuncSetAttribute(sweep_batch_kernel<true, P, Q>, attr, 200 * 1024);
            if (r == cudaSuccess) r = cudaFuncSetAttribute(sweep_batch_grad_kernel<P, Q>, attr, 200 * 1024);
            return r;
        });
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t batch_launch(const BatchArgs &b, const BatchPlan &plan, int warps, bool acc,
                         cudaStream_t s)
{
    cudaError_t e;
    for (int k = 0; k < kShapeKinds; ++k) {
        if (plan.grid[k] <= 0) continue;
        e = with_shape(k, [&](auto lpr, auto wpl) {
            constexpr int P = decltype(lpr)::value, Q = decltype(wpl)::value;
            if (acc) sweep_batch_kernel<true, P, Q><<<plan.grid[k], warps * 32, plan.smem[k], s>>>(b);
            else sweep_batch_kernel<false, P, Q><<<plan.grid[k], warps * 32, plan.smem[k], s>>>(b);
            return cudaGetLastError();
        });
        if (e != cudaSuccess) return e;
    }
    batch_zone_scan_kernel<<<dim3(b.max_z, b.n_inst), 1024, 0, s>>>(b);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    batch_advance_kernel<<<1, 32, 0, s>>>(b.t0_mut, b.work, b.n_steps);
    return cudaGetLastError();
}

cudaError_t zone_scan(unsigned long long *Zc, int64_t t0, int n, int Z, cudaStream_t s)
{
    zone_scan_kernel<<<Z, 1024, 0, s>>>(Zc, t0, n, Z);
    return cudaGetLastError();
}

cudaError_t sweep_launch(const SweepArgs &a, const SweepLaunch &l, cudaStream_t s)
{
    if (l.wpl == 2) return launch_t<32, 2>(a, l, s);
    switch (l.lpr) {
    case 1: return launch_t<1, 1>(a, l, s);
    case 2: return launch_t<2, 1>(a, l, s);
    case 4: return launch_t<4, 1>(a, l, s);
    case 8: return launch_t<8, 1>(a, l, s);
    case 16: return launch_t<16, 1>(a, l, s);
    default: return launch_t<32, 1>(a, l, s);
    }
}

}  // namespace kmc
