// kmc_setup.cu -- one-off device kernels run when a device is created:
// derived constants (Eq. 1, electrode exchange), per-site base probabilities,
// their per-zone bounds, initial placement (S2.1.1) and per-rail ion counts.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "kmc_internal.h"

namespace kmc {

namespace {

constexpr double kBoltzmann = 8.6173e-5;  // eV/K, the value printed with Eq. 4

__device__ __forceinline__ uint4 philox_init(uint32_t site, uint32_t rail, uint32_t inst,
                                             uint32_t k0, uint32_t k1)
{
    uint32_t c0 = site, c1 = rail, c2 = kInitStep, c3 = inst;
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        if (i) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
    }
    return make_uint4(c0, c1, c2, c3);
}

__device__ __forceinline__ uint64_t init_key(const kmc_params &p, int64_t idx)
{
    const int64_t row = idx / p.n_sites;                       // the rail's row in this device
    const uint32_t site = (uint32_t)(idx - row * p.n_sites);
    const uint32_t rail = (uint32_t)p.rail_base + (uint32_t)row;  // its global index
    const uint4 x = philox_init(site, rail, p.instance, (uint32_t)(p.seed & 0xffffffffu),
                                (uint32_t)(p.seed >> 32));
    return ((uint64_t)x.y << 32) | x.x;
}

// P0 = -expm1(-2 Gamma0 dt), Gamma0 = nu exp(-Ea / kT): Eq. 1 and the
// per-step hop probability, in explicitly rounded FP64 operations.
__device__ __forceinline__ double base_probability(double nu, double Ea, double kT, double dt)
{
    const double g = __dmul_rn(nu, exp(__ddiv_rn(-Ea, kT)));
    const double x = __dmul_rn(__dmul_rn(2.0, g), dt);
    return -expm1(-x);
}

__global__ void constants_kernel(const kmc_params p, DevConst *K)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    DevConst c;
    const double kT = __dmul_rn(kBoltzmann, p.T_K);
    c.kT = kT;
    c.P0 = base_probability(p.nu_Hz, p.Ea_eV, kT, p.dt_s);
    const double E = -expm1(-__dmul_rn(__dmul_rn(2.0, p.k_electrode_Hz), p.dt_s));
    c.E_in = __dmul_rn(E, p.rho_electrode);
    c.E_out = __dmul_rn(E, __dsub_rn(1.0, p.rho_electrode));
    c.ka = __dmul_rn(p.kappa, p.alpha_V);
    c.d = p.site_spacing_nm;
    c.t_dev = __dmul_rn((double)p.n_sites, p.site_spacing_nm);
    c.xs = -(c.d / c.t_dev) / kT;
    c.half_invL = 0.5 / (double)p.n_sites;
    c.P0f = (float)c.P0;
    c.E_inf = (float)c.E_in;
    c.E_outf = (float)c.E_out;
    c.pad = 0.0f;
    c.pad2 = 0;
    int st = 0;
    if (!(c.P0 >= 0.0 && c.P0 <= 1.0)) st = KMC_E_PROB;
    if (p.electrodes == 1 && !(c.E_in >= 0.0 && c.E_in <= 1.0 && c.E_out >= 0.0 && c.E_out <= 1.0))
        st = KMC_E_PROB;
    if (!(isfinite(c.kT) && c.kT > 0.0 && isfinite(c.ka) && isfinite(c.t_dev) && c.t_dev > 0.0))
        st = KMC_E_ARG;
    c.status = st;
    for (int z = 0; z <= kMaxZones; ++z)
        c.bnd[z] = z <= p.n_zones ? (int32_t)(((int64_t)z * p.n_sites) / p.n_zones) : p.n_sites;
    *K = c;
}

__global__ void p0_table_kernel(const kmc_params p, double kT, const double *Ea, double *P0,
                                int64_t n, int *bad)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = base_probability(p.nu_Hz, Ea[i], kT, p.dt_s);
        if (!(v >= 0.0 && v <= 1.0)) atomicExch(bad, 1);
        P0[i] = v;
    }
}

// (min, max) of P0 over each zone of each rail, rounded outward to FP32.
__global__ void p0_bounds_kernel(const double *P0, int32_t R, int32_t L, int32_t Z,
                                 const DevConst *K, float2 *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)R * Z) return;
    const int64_t r = i / Z;
    const int z = (int)(i - r * Z);
    double lo = 1.0, hi = 0.0;
    for (int k = K->bnd[z]; k < K->bnd[z + 1]; ++k) {
        const double v = P0[r * L + k];
        lo = fmin(lo, v);
        hi = fmax(hi, v);
    }
    out[i] = make_float2(__double2float_rd(lo), __double2float_ru(hi));
}

__global__ void p0_float_kernel(const double *P0, int64_t n, float *out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)P0[i];
}

// One warp per rail: ion count, and a count of bytes that are not 0 or 1.
__global__ void row_counts_kernel(const uint8_t *occ, int64_t stride, int32_t R, int32_t L,
                                  int32_t *N0, unsigned long long *bad)
{
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= R) return;
    int c = 0, b = 0;
    for (int k = lane; k < L; k += 32) {
        const uint8_t v = occ[r * stride + k];
        c += v == 1;
        b += v > 1;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    b = __reduce_add_sync(0xffffffffu, b);
    if (lane == 0) {
        N0[r] = c;
        if (b) atomicAdd(bad, (unsigned long long)b);
    }
}

__global__ void bernoulli_kernel(const kmc_params p, uint8_t *occ, int64_t stride)
{
    const int64_t n = (int64_t)p.n_rails * p.n_sites;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double u = __dmul_rn((double)(init_key(p, i) >> 11), 0x1.0p-53);
        const int64_t r = i / p.n_sites;
        occ[r * stride + (i - r * p.n_sites)] = u < p.fill ? 1 : 0;
    }
}

// mode 0: count keys <= key_bound;  mode 1: count keys == key_bound with index <= idx_bound
__global__ void count_keys_kernel(const kmc_params p, uint64_t key_bound, int mode,
                                  int64_t idx_bound, unsigned long long *count)
{
    const int64_t n = (int64_t)p.n_rails * p.n_sites;
    unsigned c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = init_key(p, i);
        c += mode == 0 ? (k <= key_bound) : (k == key_bound && i <= idx_bound);
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, (unsigned long long)c);
}

__global__ void mark_smallest_kernel(const kmc_params p, uint64_t key_star, int64_t idx_star,
                                     int select_none, uint8_t *occ, int64_t stride)
{
    const int64_t n = (int64_t)p.n_rails * p.n_sites;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = init_key(p, i);
        const bool sel = !select_none && (k < key_star || (k == key_star && i <= idx_star));
        const int64_t r = i / p.n_sites;
        occ[r * stride + (i - r * p.n_sites)] = sel ? 1 : 0;
    }
}

// Tables of the gradient pass: exp(cm m) = etH[(m + M) >> 10] etL[(m + M) & 1023].
__global__ void exp_table_kernel(double cm, int32_t M, double *etL, double *etH, int32_t nH)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 1024) etL[i] = exp(__dmul_rn(cm, (double)i));
    if (i < nH) etH[i] = exp(__dmul_rn(cm, (double)((int64_t)i * 1024 - M)));
}

// Background of each zone of each rail for the FP64 decision paths (one
// thread per rail): c_z = N0 w_z / L, an exact product rounded once by the
// division, as the exact path uses it, and D'_z = D_z - sum_z' w_z' D_z' / L
// with D_z = sum_{z'<z} c_z' + c_z / 2, the background part of Q_z - Qbar
// (S2.1.8 reading), so that Q_z - Qbar = (L (Pb_z + Pb_z+1) - F) / (2 L) - D'_z.
__global__ void background_kernel(const int32_t *N0, int32_t R, int32_t L, int32_t Z,
                                  const DevConst *K, double2 *bgd)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    double run = 0.0, acc = 0.0;
    for (int z = 0; z < Z; ++z) {
        const int w = K->bnd[z + 1] - K->bnd[z];
        const double c = __ddiv_rn(__dmul_rn((double)N0[r], (double)w), (double)L);
        const double D = run + 0.5 * c;
        run += c;
        acc += (double)w * D;
        bgd[r * Z + z] = make_double2(c, D);
    }
    const double mean = acc / (double)L;
    for (int z = 0; z < Z; ++z) bgd[r * Z + z].y -= mean;
}

int grid_for(int64_t n, int block)
{
    int64_t g = (n + block - 1) / block;
    if (g > 152 * 32) g = 152 * 32;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

cudaError_t setup_constants(const kmc_params &p, DevConst *K, cudaStream_t s)
{
    constants_kernel<<<1, 32, 0, s>>>(p, K);
    return cudaGetLastError();
}

cudaError_t setup_p0_table(const kmc_params &p, const double *Ea, double *P0, int64_t n,
                           int *bad, cudaStream_t s)
{
    const double kT = kBoltzmann * p.T_K;  // same IEEE product as on the device
    p0_table_kernel<<<grid_for(n, 256), 256, 0, s>>>(p, kT, Ea, P0, n, bad);
    return cudaGetLastError();
}

cudaError_t setup_p0_bounds(const double *P0, int32_t R, int32_t L, int32_t Z, const DevConst *K,
                            float2 *out, cudaStream_t s)
{
    const int64_t n = (int64_t)R * Z;
    p0_bounds_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P0, R, L, Z, K, out);
    return cudaGetLastError();
}

cudaError_t setup_p0_float(const double *P0, int64_t n, float *out, cudaStream_t s)
{
    p0_float_kernel<<<grid_for(n, 256), 256, 0, s>>>(P0, n, out);
    return cudaGetLastError();
}

cudaError_t setup_exp_tables(double cm, int32_t M, double *etL, double *etH, int32_t nH,
                             cudaStream_t s)
{
    const int n = nH > 1024 ? nH : 1024;
    exp_table_kernel<<<(n + 255) / 256, 256, 0, s>>>(cm, M, etL, etH, nH);
    return cudaGetLastError();
}

cudaError_t setup_background(const int32_t *N0, int32_t R, int32_t L, int32_t Z, const DevConst *K,
                             double2 *bgd, cudaStream_t s)
{
    background_kernel<<<(unsigned)((R + 255) / 256), 256, 0, s>>>(N0, R, L, Z, K, bgd);
    return cudaGetLastError();
}

cudaError_t setup_row_counts(const uint8_t *occ, int64_t stride, int32_t R, int32_t L,
                             int32_t *N0, unsigned long long *bad, cudaStream_t s)
{
    const int warps = 8;
    row_counts_kernel<<<(unsigned)((R + warps - 1) / warps), warps * 32, 0, s>>>(occ, stride, R, L,
                                                                                N0, bad);
    return cudaGetLastError();
}

cudaError_t setup_init_bernoulli(const kmc_params &p, uint8_t *occ, int64_t stride, cudaStream_t s)
{
    const int64_t n = (int64_t)p.n_rails * p.n_sites;
    bernoulli_kernel<<<grid_for(n, 256), 256, 0, s>>>(p, occ, stride);
    return cudaGetLastError();
}

cudaError_t setup_count_keys(const kmc_params &p, uint64_t key_bound, int mode, int64_t idx_bound,
                             unsigned long long *count, cudaStream_t s)
{
    const int64_t n = (int64_t)p.n_rails * p.n_sites;
    count_keys_kernel<<<grid_for(n, 256), 256, 0, s>>>(p, key_bound, mode, idx_bound, count);
    return cudaGetLastError();
}

cudaError_t setup_mark_smallest(const kmc_params &p, uint64_t key_star, int64_t idx_star,
                                int select_none, uint8_t *occ, int64_t stride, cudaStream_t s)
{
    const int64_t n = (int64_t)p.n_rails * p.n_sites;
    mark_smallest_kernel<<<grid_for(n, 256), 256, 0, s>>>(p, key_star, idx_star, select_none, occ,
                                                          stride);
    return cudaGetLastError();
}

}  // namespace kmc
