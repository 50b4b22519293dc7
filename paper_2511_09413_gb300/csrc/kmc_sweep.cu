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
//    (occupied with a free neighbour, or an empty electrode site), after a
//    warp-wide compaction so that all 32 lanes draw.
//  * Moves are rare per step, so the move/conflict/apply phase runs only when
//    the warp accepted at least one hop.
//  * Per-step current and zone counts are reduced per CTA in shared memory and
//    flushed to the int64 traces with one atomic per value every `flush` steps.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "kmc_internal.h"

namespace kmc {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): per round two 32x32->64
// multiplies; the high halves are xor-ed with the other counter words and the
// round key.  The ten round keys are precomputed on the host.
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        const uint32_t *rk0, const uint32_t *rk1)
{
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
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

struct WarpSmem {
    uint4 *thr;     // [G][Z]  {acc R, rej R, acc L, rej L}
    uint4 *thrE;    // [G][2]  electrode thresholds
    float2 *zf;     // [G][Z]  FP32 (B, 1/(1+B))
    int32_t *Pb;    // [G][Z+1] ions before each zone boundary
    int32_t *Fs;    // [G] sum_z w_z (Pb_z + Pb_{z+1})
    int32_t *inj;   // [2][G] injection flags (left electrode, right electrode)
    uint32_t *mvR;  // [32 WPL] right-move sources
    uint32_t *mvL;  // [32 WPL] left-move sources
    uint32_t *list; // candidates
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline size_t warp_block_bytes(int G, int Z, int wpl)
{
    size_t b = 0;
    b += align16(sizeof(uint4) * G * Z);
    b += align16(sizeof(uint4) * G * 2);
    b += align16(sizeof(float2) * G * Z);
    b += align16(sizeof(int32_t) * G * (Z + 1));
    b += align16(sizeof(int32_t) * G);
    b += align16(sizeof(int32_t) * 2 * G);
    b += align16(sizeof(uint32_t) * 2 * 32 * wpl);
    b += align16(sizeof(uint32_t) * (1024 * wpl + 2 * G));
    return b;
}

__device__ inline WarpSmem carve(uint8_t *base, int G, int Z, int wpl)
{
    WarpSmem w;
    size_t o = 0;
    w.thr = (uint4 *)(base + o);
    o += align16(sizeof(uint4) * G * Z);
    w.thrE = (uint4 *)(base + o);
    o += align16(sizeof(uint4) * G * 2);
    w.zf = (float2 *)(base + o);
    o += align16(sizeof(float2) * G * Z);
    w.Pb = (int32_t *)(base + o);
    o += align16(sizeof(int32_t) * G * (Z + 1));
    w.Fs = (int32_t *)(base + o);
    o += align16(sizeof(int32_t) * G);
    w.inj = (int32_t *)(base + o);
    o += align16(sizeof(int32_t) * 2 * G);
    w.mvR = (uint32_t *)(base + o);
    w.mvL = w.mvR + 32 * wpl;
    o += align16(sizeof(uint32_t) * 2 * 32 * wpl);
    w.list = (uint32_t *)(base + o);
    return w;
}

// Exact FP64 zone quantities (B_z, 1/(1+B_z)) for zone zt of one rail, with
// the operation order of the oracle: excess C_z, enclosed charge Q_z, mean
// Qbar, dV_z (S2.1.8), dE_z (Eq. 3), B_z (Eq. 4).  Every operation is an
// explicitly rounded intrinsic so that no contraction changes the result.
__device__ __noinline__ void exact_zone(const int32_t *Pb, const DevConst *Kp, int Z, int L,
                                        int32_t n0, double V, int zt, double *B, double *inv)
{
    const DevConst &K = *Kp;
    const double Ld = (double)L;
    double run = 0.0, acc = 0.0, Qt = 0.0;
    for (int z = 0; z < Z; ++z) {
        const int w = K.bnd[z + 1] - K.bnd[z];
        const int Nz = Pb[z + 1] - Pb[z];
        const double C = __dsub_rn((double)Nz, __ddiv_rn(__dmul_rn((double)n0, (double)w), Ld));
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
__device__ __noinline__ bool exact_trial(uint64_t w, double p, kmc_log_entry *log,
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

template <int LPR, int WPL>
__global__ void __launch_bounds__(256) sweep_kernel(const SweepArgs a)
{
    constexpr int G = 32 / LPR;
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int seg = lane / LPR;
    const int sl = lane % LPR;
    const int wbase = sl * WPL;
    const int L = a.L, Z = a.Z;
    const bool open = a.electrodes == 1;
    const int64_t rail0 = ((int64_t)blockIdx.x * nwarps + warp) * G;
    const int64_t rail = rail0 + seg;
    const bool active = rail < a.R;

    const size_t wb = warp_block_bytes(G, Z, WPL);
    WarpSmem S = carve(smem + (size_t)warp * wb, G, Z, WPL);
    int32_t *trace = (int32_t *)(smem + (size_t)nwarps * wb);
    uint8_t *zone_tab = (uint8_t *)(trace + (size_t)a.flush * (1 + Z));

    // ---- per-CTA tables
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        int z = 0;
        while (a.bnd[z + 1] <= k) ++z;
        zone_tab[k] = (uint8_t)z;
    }
    for (int i = threadIdx.x; i < a.flush * (1 + Z); i += blockDim.x) trace[i] = 0;
    for (int i = lane; i < 2 * 32 * WPL; i += 32) S.mvR[i] = 0;
    for (int i = lane; i < 2 * G; i += 32) S.inj[i] = 0;

    // ---- per-lane site masks and owned zone boundaries
    uint32_t vm[WPL], firstm[WPL], lastm[WPL], o[WPL];
    const uint8_t *row = a.occ + (active ? rail : 0) * a.stride;
#pragma unroll
    for (int j = 0; j < WPL; ++j) {
        const int s0 = 32 * (wbase + j);
        vm[j] = s0 >= L ? 0u : (s0 + 32 <= L ? FULL : ((1u << (L - s0)) - 1u));
        firstm[j] = (s0 == 0) ? 1u : 0u;
        lastm[j] = (L - 1 >= s0 && L - 1 < s0 + 32) ? (1u << (L - 1 - s0)) : 0u;
        uint32_t bits = 0;
        if (active) {
            if (s0 < a.stride) bits |= pack16(*(const uint4 *)(row + s0));
            if (s0 + 16 < a.stride) bits |= pack16(*(const uint4 *)(row + s0 + 16)) << 16;
        }
        o[j] = bits & vm[j];
    }
    int zlo = 1, zhi = 0;  // interior boundaries z in [zlo, zhi] lie in this lane's words
    {
        const int lo = 32 * wbase, hi = 32 * (wbase + WPL);
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
    }
    const int32_t n0_seg = active ? a.N0[rail] : 0;
    const float delta = a.delta;
    const DevConst *K = a.K;
    const float P0f = K->P0f, E_inf = K->E_inf, E_outf = K->E_outf;
    unsigned long long n_draw = 0, n_exact = 0, n_move = 0;
    __syncthreads();

    for (int c0 = 0; c0 < a.n_steps; c0 += a.flush) {
        const int c1 = min(a.n_steps, c0 + a.flush);
        for (int s = c0; s < c1; ++s) {
            const uint32_t t = (uint32_t)(a.t0 + s);
            const double Vd = a.V[t];
            const float Vf = (float)Vd;
            int32_t *tr = trace + (s - c0) * (1 + Z);

            // ---- 1. zone counts: segmented scan of popcounts
            int cnt = 0;
#pragma unroll
            for (int j = 0; j < WPL; ++j) cnt += __popc(o[j]);
            int incl = cnt;
#pragma unroll
            for (int off = 1; off < LPR; off <<= 1) {
                const int v = __shfl_up_sync(FULL, incl, off, LPR);
                if (sl >= off) incl += v;
            }
            const int excl = incl - cnt;
            const int total = __shfl_sync(FULL, incl, LPR - 1, LPR);
            int fpart = 0;
            for (int z = zlo; z <= zhi; ++z) {
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
                S.Pb[seg * (Z + 1) + z] = P;
                fpart += P * a.wsum[z];
            }
            if (sl == 0) S.Pb[seg * (Z + 1)] = 0;
            if (sl == LPR - 1) {
                S.Pb[seg * (Z + 1) + Z] = total;
                fpart += total * a.wsum[Z];
            }
#pragma unroll
            for (int off = LPR / 2; off >= 1; off >>= 1) fpart += __shfl_xor_sync(FULL, fpart, off, LPR);
            if (sl == 0) S.Fs[seg] = fpart;
            __syncwarp();

            // ---- 2. field and FP32 decision intervals per (rail, zone)
            for (int pi = lane; pi < G * Z; pi += 32) {
                const int g2 = pi / Z;
                const int z = pi - g2 * Z;
                const int64_t r2 = rail0 + g2;
                const int Pz = S.Pb[g2 * (Z + 1) + z];
                const int Pz1 = S.Pb[g2 * (Z + 1) + z + 1];
                if (Pz1 != Pz) atomicAdd(&tr[1 + z], Pz1 - Pz);
                if (r2 >= a.R) continue;
                const int32_t n0 = a.N0[r2];
                const float qd = 0.5f * ((float)(Pz + Pz1) - (float)S.Fs[g2] * a.inv_L) -
                                 (float)n0 * a.cz[z];
                const float dV = Vf - a.ka_f * qd;
                const float x = -dV * a.inv_LkT;
                uint4 th;
                if (!(fabsf(x) <= 40.0f)) {
                    th = make_uint4(0u, FULL, 0u, FULL);  // undecidable in FP32: exact path
                    S.zf[pi] = make_float2(0.0f, 0.0f);
                    if (open && z == 0) S.thrE[g2 * 2 + 0] = th;
                    if (open && z == Z - 1) S.thrE[g2 * 2 + 1] = th;
                } else {
                    const float B = expf(x);
                    const float inv = 1.0f / (1.0f + B);
                    const float lo = 1.0f - delta, hi = 1.0f + delta;
                    float blo = P0f, bhi = P0f;
                    if (a.P0bnd) {
                        const float2 pb = a.P0bnd[r2 * Z + z];
                        blo = pb.x;
                        bhi = pb.y;
                    }
                    const float sR = inv * B, sL = inv;
                    th = make_uint4(acc_thr(blo * sR * lo), rej_thr(bhi * sR * hi),
                                    acc_thr(blo * sL * lo), rej_thr(bhi * sL * hi));
                    S.zf[pi] = make_float2(B, inv);
                    if (open && z == 0)  // injection into site 0 (right), extraction from 0 (left)
                        S.thrE[g2 * 2 + 0] =
                            make_uint4(acc_thr(E_inf * sR * lo), rej_thr(E_inf * sR * hi),
                                       acc_thr(E_outf * sL * lo), rej_thr(E_outf * sL * hi));
                    if (open && z == Z - 1)  // extraction from L-1 (right), injection into L-1 (left)
                        S.thrE[g2 * 2 + 1] =
                            make_uint4(acc_thr(E_outf * sR * lo), rej_thr(E_outf * sR * hi),
                                       acc_thr(E_inf * sL * lo), rej_thr(E_inf * sL * hi));
                }
                S.thr[pi] = th;
            }
            __syncwarp();

            // ---- 3. candidates: occupied with a free neighbour, empty electrode sites
            uint32_t fL[WPL], fR[WPL], cand[WPL];
            {
                uint32_t f[WPL];
#pragma unroll
                for (int j = 0; j < WPL; ++j) f[j] = ~o[j] & vm[j];
                const uint32_t f_prev = __shfl_up_sync(FULL, f[WPL - 1], 1, LPR);
                const uint32_t f_next = __shfl_down_sync(FULL, f[0], 1, LPR);
#pragma unroll
                for (int j = 0; j < WPL; ++j) {
                    const uint32_t cp = j > 0 ? (f[j > 0 ? j - 1 : 0] >> 31)
                                              : (sl > 0 ? (f_prev >> 31) : (open ? 1u : 0u));
                    const uint32_t cn = j < WPL - 1 ? (f[j < WPL - 1 ? j + 1 : 0] & 1u)
                                                    : (sl < LPR - 1 ? (f_next & 1u) : 0u);
                    fL[j] = (f[j] << 1) | cp;
                    fR[j] = (f[j] >> 1) | (cn << 31);
                    if (open) fR[j] |= lastm[j];
                    const uint32_t inj = open ? ((firstm[j] | lastm[j]) & ~o[j]) : 0u;
                    cand[j] = active ? ((o[j] & (fL[j] | fR[j])) | inj) : 0u;
                }
            }

            // ---- 4. warp-wide compaction of candidates
            int nc = 0;
#pragma unroll
            for (int j = 0; j < WPL; ++j) nc += __popc(cand[j]);
            int ic = nc;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int v = __shfl_up_sync(FULL, ic, off);
                if (lane >= off) ic += v;
            }
            int pos = ic - nc;
            const int ntot = __shfl_sync(FULL, ic, 31);
#pragma unroll
            for (int j = 0; j < WPL; ++j) {
                uint32_t m = cand[j];
                while (m) {
                    const int b = __ffs(m) - 1;
                    m &= m - 1;
                    const uint32_t bit = 1u << b;
                    const bool occd = (o[j] & bit) != 0;
                    const bool tR = occd ? (fR[j] & bit) != 0 : (firstm[j] & bit) != 0;
                    const bool tL = occd ? (fL[j] & bit) != 0 : (lastm[j] & bit) != 0;
                    S.list[pos++] = (uint32_t)(32 * (wbase + j) + b) | ((uint32_t)seg << 11) |
                                    (tR ? (1u << 16) : 0u) | (tL ? (1u << 17) : 0u) |
                                    (occd ? 0u : (1u << 18));
                }
            }
            __syncwarp();
            if (lane == 0) n_draw += (unsigned long long)ntot;

            // ---- 5. draws and decisions
            bool moved = false;
            for (int i = lane; i < ntot; i += 32) {
                const uint32_t dsc = S.list[i];
                const int site = (int)(dsc & 0x7FFu);
                const int g2 = (int)((dsc >> 11) & 31u);
                const bool tryR = (dsc >> 16) & 1u, tryL = (dsc >> 17) & 1u;
                const bool empty = (dsc >> 18) & 1u;
                const uint32_t r2 = (uint32_t)(rail0 + g2);
                const uint4 x = philox((uint32_t)site, r2, t, a.instance, a.rk0, a.rk1);
                const int z = zone_tab[site];
                const uint4 th = S.thr[g2 * Z + z];
                uint32_t aR = th.x, rR = th.y, aL = th.z, rL = th.w;
                int kindR = 0, kindL = 0;
                bool siteP0 = a.P0bnd != nullptr;  // per-site base probability applies
                bool siteP0R = siteP0, siteP0L = siteP0;
                if (open) {
                    if (empty) {
                        if (site == 0) {
                            const uint4 e = S.thrE[g2 * 2 + 0];
                            aR = e.x;
                            rR = e.y;
                            kindR = 1;
                        } else {
                            const uint4 e = S.thrE[g2 * 2 + 1];
                            aL = e.z;
                            rL = e.w;
                            kindL = 1;
                        }
                        siteP0R = siteP0L = false;
                    } else {
                        if (site == 0) {
                            const uint4 e = S.thrE[g2 * 2 + 0];
                            aL = e.z;
                            rL = e.w;
                            kindL = 2;
                            siteP0L = false;
                        }
                        if (site == L - 1) {
                            const uint4 e = S.thrE[g2 * 2 + 1];
                            aR = e.x;
                            rR = e.y;
                            kindR = 2;
                            siteP0R = false;
                        }
                    }
                }
                // 0 reject, 1 accept, 2 undecided in FP32
                int dR = tryR ? (x.y < aR ? 1 : (x.y > rR ? 0 : 2)) : 0;
                int dL = tryL ? (x.w < aL ? 1 : (x.w > rL ? 0 : 2)) : 0;
                if ((dR == 2 && siteP0R) || (dL == 2 && siteP0L)) {
                    // refine with this site's own base probability
                    const float P0k = (float)a.P0site[(int64_t)r2 * L + site];
                    const float2 bi = S.zf[g2 * Z + z];
                    const float lo = 1.0f - delta, hi = 1.0f + delta;
                    if (dR == 2 && siteP0R && bi.y > 0.0f) {
                        const float p = P0k * bi.y * bi.x;
                        dR = x.y < acc_thr(p * lo) ? 1 : (x.y > rej_thr(p * hi) ? 0 : 2);
                    }
                    if (dL == 2 && siteP0L && bi.y > 0.0f) {
                        const float p = P0k * bi.y;
                        dL = x.w < acc_thr(p * lo) ? 1 : (x.w > rej_thr(p * hi) ? 0 : 2);
                    }
                }
                if (dR == 2 || dL == 2) {
                    double B, inv;
                    exact_zone(S.Pb + g2 * (Z + 1), K, Z, L, a.N0[r2], Vd, z, &B, &inv);
                    const double P0k = siteP0 ? a.P0site[(int64_t)r2 * L + site] : K->P0;
                    if (dR == 2) {
                        const double base = kindR == 1 ? K->E_in : (kindR == 2 ? K->E_out : P0k);
                        const double p = __dmul_rn(__dmul_rn(base, inv), B);
                        dR = exact_trial(((uint64_t)x.y << 32) | x.x, p, a.log, a.log_count,
                                         a.log_cap, (int32_t)r2, t, site, 0, kindR)
                                 ? 1
                                 : 0;
                        ++n_exact;
                    }
                    if (dL == 2) {
                        const double base = kindL == 1 ? K->E_in : (kindL == 2 ? K->E_out : P0k);
                        const double p = __dmul_rn(base, inv);
                        dL = exact_trial(((uint64_t)x.w << 32) | x.z, p, a.log, a.log_count,
                                         a.log_cap, (int32_t)r2, t, site, 1, kindL)
                                 ? 1
                                 : 0;
                        ++n_exact;
                    }
                }
                // X + M_right - M_left: both trials succeeding leaves the ion in place
                if (dR == 1 && dL != 1) {
                    moved = true;
                    if (empty) S.inj[g2] = 1;  // injection into site 0
                    else atomicOr(&S.mvR[g2 * LPR * WPL + (site >> 5)], 1u << (site & 31));
                } else if (dL == 1 && dR != 1) {
                    moved = true;
                    if (empty) S.inj[G + g2] = 1;  // injection into site L-1
                    else atomicOr(&S.mvL[g2 * LPR * WPL + (site >> 5)], 1u << (site & 31));
                }
            }

            // ---- 6. conflicts, synchronous update, current
            if (__any_sync(FULL, moved)) {
                __syncwarp();
                uint32_t mR[WPL], mL[WPL], tR[WPL], tL[WPL], cf[WPL];
#pragma unroll
                for (int j = 0; j < WPL; ++j) {
                    mR[j] = S.mvR[seg * LPR * WPL + wbase + j];
                    mL[j] = S.mvL[seg * LPR * WPL + wbase + j];
                }
                const int iR = S.inj[seg], iL = S.inj[G + seg];
                const uint32_t mR_prev = __shfl_up_sync(FULL, mR[WPL - 1], 1, LPR);
                const uint32_t mL_next = __shfl_down_sync(FULL, mL[0], 1, LPR);
#pragma unroll
                for (int j = 0; j < WPL; ++j) {
                    const uint32_t cp = j > 0 ? (mR[j > 0 ? j - 1 : 0] >> 31)
                                              : (sl > 0 ? (mR_prev >> 31) : (iR ? 1u : 0u));
                    const uint32_t cn = j < WPL - 1 ? (mL[j < WPL - 1 ? j + 1 : 0] & 1u)
                                                    : (sl < LPR - 1 ? (mL_next & 1u) : 0u);
                    tR[j] = ((mR[j] << 1) | cp) & vm[j];
                    tL[j] = ((mL[j] >> 1) | (cn << 31)) & vm[j];
                    if (iL) tL[j] |= lastm[j];
                    cf[j] = tR[j] & tL[j];
                }
                const uint32_t c_prev = __shfl_up_sync(FULL, cf[WPL - 1], 1, LPR);
                const uint32_t c_next = __shfl_down_sync(FULL, cf[0], 1, LPR);
                int Jl = 0;
#pragma unroll
                for (int j = 0; j < WPL; ++j) {
                    const uint32_t cn = j < WPL - 1 ? (cf[j < WPL - 1 ? j + 1 : 0] & 1u)
                                                    : (sl < LPR - 1 ? (c_next & 1u) : 0u);
                    const uint32_t cp = j > 0 ? (cf[j > 0 ? j - 1 : 0] >> 31)
                                              : (sl > 0 ? (c_prev >> 31) : 0u);
                    mR[j] &= ~((cf[j] >> 1) | (cn << 31));
                    mL[j] &= ~((cf[j] << 1) | cp);
                    tR[j] &= ~cf[j];
                    tL[j] &= ~cf[j];
                    Jl += __popc(mL[j]) - __popc(mR[j]);
                    o[j] = (o[j] & ~(mR[j] | mL[j])) | tR[j] | tL[j];
                    if (iR && firstm[j] && !(cf[j] & 1u)) Jl -= 1;          // injected at site 0
                    if (iL && lastm[j] && !(cf[j] & lastm[j])) Jl += 1;     // injected at L-1
                    n_move += (unsigned long long)(__popc(mR[j]) + __popc(mL[j]));
                }
                if (iR && sl == 0 && !(cf[0] & 1u)) n_move += 1;
#pragma unroll
                for (int j = 0; j < WPL; ++j)
                    if (iL && lastm[j] && !(cf[j] & lastm[j])) n_move += 1;
                __syncwarp();
#pragma unroll
                for (int j = 0; j < WPL; ++j) {
                    S.mvR[seg * LPR * WPL + wbase + j] = 0u;
                    S.mvL[seg * LPR * WPL + wbase + j] = 0u;
                }
                if (sl == 0) {
                    S.inj[seg] = 0;
                    S.inj[G + seg] = 0;
                }
                const int Jw = __reduce_add_sync(FULL, Jl);
                if (lane == 0 && Jw != 0) atomicAdd(&tr[0], Jw);
            }
            __syncwarp();
        }
        // ---- flush this chunk's traces
        __syncthreads();
        const int nval = (c1 - c0) * (1 + Z);
        for (int i = threadIdx.x; i < nval; i += blockDim.x) {
            const int v = trace[i];
            if (v != 0) {
                const int64_t step = a.t0 + c0 + i / (1 + Z);
                const int q = i % (1 + Z);
                const unsigned long long add = (unsigned long long)(long long)v;
                if (q == 0) atomicAdd(&a.J[step], add);
                else atomicAdd(&a.Zc[step * Z + (q - 1)], add);
            }
            trace[i] = 0;
        }
        __syncthreads();
    }

    // ---- write the rail back
    if (active) {
        uint8_t *wrow = a.occ + rail * a.stride;
#pragma unroll
        for (int j = 0; j < WPL; ++j) {
            const int s0 = 32 * (wbase + j);
            if (s0 < a.stride) *(uint4 *)(wrow + s0) = unpack16(o[j] & 0xFFFFu);
            if (s0 + 16 < a.stride) *(uint4 *)(wrow + s0 + 16) = unpack16(o[j] >> 16);
        }
    }
    // ---- counters
    if (lane == 0) {
        if (n_draw) atomicAdd(&a.counters[0], n_draw);
    }
    n_exact = __reduce_add_sync(FULL, (unsigned)n_exact);
    n_move = __reduce_add_sync(FULL, (unsigned)n_move);
    if (lane == 0) {
        if (n_exact) atomicAdd(&a.counters[1], n_exact);
        if (n_move) atomicAdd(&a.counters[2], n_move);
    }
}

template <int LPR, int WPL>
cudaError_t launch_t(const SweepArgs &a, const SweepLaunch &l, cudaStream_t s)
{
    sweep_kernel<LPR, WPL><<<l.grid, l.warps * 32, l.smem, s>>>(a);
    return cudaGetLastError();
}

template <int LPR, int WPL>
cudaError_t smem_attr()
{
    return cudaFuncSetAttribute(sweep_kernel<LPR, WPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                200 * 1024);
}

}  // namespace

size_t sweep_smem_bytes(int lpr, int wpl, int Z, int L, int warps, int flush)
{
    const int G = 32 / lpr;
    return (size_t)warps * warp_block_bytes(G, Z, wpl) + align16(sizeof(int32_t) * flush * (1 + Z)) +
           align16((size_t)L);
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
