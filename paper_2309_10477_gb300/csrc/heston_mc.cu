// heston_mc.cu -- GB300 (sm_103a) Monte Carlo Heston pricing with pathwise
// Greeks, behind the C ABI declared in include/heston_mc.h.
//
// Method (arXiv 2309.10477):
//   * Heston dynamics, Eq. (heston_eq), Sec. 2.1.
//   * Correlated normals, Algorithm "Generation of two correlated Normal
//     random variables" (Sec. 2.4.1): Z1 = Za, Z2 = rho Z1 + sqrt(1-rho^2) Zb.
//   * Milstein for ln S and V (Sec. 2.4.2): ln S += (r - V/2) dt + sqrt(V dt) Z1
//     (no correction term), V += kappa (theta - V) dt + xi sqrt(V dt) Z2
//     + xi^2 dt (Z2^2 - 1) / 4, with full truncation or the paper's floor.
//   * Monte Carlo average (Algorithm "Monte Carlo option pricing estimation",
//     Sec. 2.5) of the discounted payoff and of the pathwise Greeks of
//     Eq. (euro_pw) / Eq. (asian_pw); Gamma, Vega (d/dv0) and Theta (-d/dT),
//     which the paper only names (Sec. 2), come from a pathwise /
//     likelihood-ratio Gamma weight and tangent recursions run alongside
//     the path.
//
// GPU design: one lane carries two paths through all N steps in registers
// (Philox4x32-10 -> Box-Muller -> correlate -> Milstein step -> tangents ->
// Asian sums), in FP32 as f32x2 instructions on the pair; a warp owns 64-path
// tiles and reduces each tile's estimators with shuffles; tile rows go to a
// workspace and two fixed-order kernels reduce them in FP64.  No per-path or
// per-step data touches memory.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <algorithm>
#include <cstring>
#include <deque>
#include <map>
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "heston_mc.h"

#include "heston_device.cuh"

namespace {

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct DeviceGuard {
    int prev = -1;
    bool switched = false;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int dev)
    {
        if (dev < 0) return;
        err = cudaGetDevice(&prev);
        if (err == cudaSuccess && prev != dev) {
            err = cudaSetDevice(dev);
            switched = (err == cudaSuccess);
        }
    }
    ~DeviceGuard()
    {
        if (switched) cudaSetDevice(prev);
    }
};

// Stream-ordered scratch of the synchronous entry points: one pool per
// device, owned by the library, that keeps freed memory for the next call
// (release threshold unlimited) instead of unmapping it at every
// synchronisation as a pool with threshold 0 does.  heston_release_cached_memory
// trims it.
constexpr int kMaxPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxPoolDevices];

cudaMemPool_t scratch_pool(int dev, bool create)
{
    if (dev < 0 || dev >= kMaxPoolDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev] && create) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pool[dev] = pool;
    }
    return g_pool[dev];
}

cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t st)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaMemPool_t pool = scratch_pool(dev, true);
    if (!pool) return cudaMallocAsync(p, bytes, st);
    return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

struct Prepared {
    ContractSet<double> cs;
    ContractSet<float> csf;
    Coef<float> kf;
    Coef<double> kd{};
    heston_options opt;
    uint32_t N;
    bool gamma_nan;
};

template <typename R> const ContractSet<R> &cs_of(const Prepared &pp);
template <> const ContractSet<double> &cs_of<double>(const Prepared &pp) { return pp.cs; }
template <> const ContractSet<float> &cs_of<float>(const Prepared &pp) { return pp.csf; }

bool finite_nonneg(double x) { return std::isfinite(x) && x >= 0.0; }

// Every coefficient rounded once from its FP64 value.
template <typename D>
Coef<D> coef_cast(const Coef<double> &k)
{
    static_assert(sizeof(Coef<double>) % sizeof(double) == 0, "Coef holds doubles only");
    constexpr int n = (int)(sizeof(Coef<double>) / sizeof(double));
    static_assert(sizeof(Coef<D>) == n * sizeof(D), "Coef layout");
    const double *src = reinterpret_cast<const double *>(&k);
    Coef<D> out;
    D *dst = reinterpret_cast<D *>(&out);
    for (int i = 0; i < n; ++i) dst[i] = (D)src[i];
    return out;
}

int validate_and_prepare(const heston_params *p, const heston_contract *c, uint32_t nc,
                         uint64_t n_paths, uint32_t N, const heston_options *opts, Prepared &out)
{
    if (!p || !c || nc == 0 || nc > (uint32_t)kMaxC) return HESTON_ERR_INVALID_ARG;
    if (N == 0 || n_paths < 2 || n_paths > (1ull << 40)) return HESTON_ERR_INVALID_ARG;
    if (!(std::isfinite(p->S0) && p->S0 > 0.0)) return HESTON_ERR_INVALID_ARG;
    if (!finite_nonneg(p->v0) || !finite_nonneg(p->kappa) || !finite_nonneg(p->theta) ||
        !finite_nonneg(p->xi) || !std::isfinite(p->r))
        return HESTON_ERR_INVALID_ARG;
    if (!std::isfinite(p->rho) || std::fabs(p->rho) > 1.0) return HESTON_ERR_INVALID_ARG;

    heston_options o;
    if (opts) {
        o = *opts;
    } else {
        std::memset(&o, 0, sizeof(o));
        o.prec = HESTON_FP64;
        o.device = -1;
    }
    if (o.trunc != HESTON_TRUNC_FULL && o.trunc != HESTON_TRUNC_PAPER_FLOOR) return HESTON_ERR_INVALID_ARG;
    if (o.prec != HESTON_FP32 && o.prec != HESTON_FP64) return HESTON_ERR_INVALID_ARG;
    if (o.rng != HESTON_RNG_PHILOX && o.rng != HESTON_RNG_SOBOL_BB) return HESTON_ERR_INVALID_ARG;
    if (o.reserved != 0) return HESTON_ERR_INVALID_ARG;
    if (o.scheme != HESTON_SCHEME_MILSTEIN && o.scheme != HESTON_SCHEME_EULER && o.scheme != HESTON_SCHEME_QE)
        return HESTON_ERR_INVALID_ARG;
    if (o.scheme == HESTON_SCHEME_QE && !(p->kappa > 0.0 && p->theta > 0.0 && p->xi > 0.0))
        return HESTON_ERR_INVALID_ARG;
    if (o.scheme != HESTON_SCHEME_MILSTEIN && o.rng != HESTON_RNG_PHILOX) return HESTON_ERR_UNSUPPORTED;
    if (o.block_threads != 0 && (o.block_threads % 32 != 0 || o.block_threads > kPathBlock))
        return HESTON_ERR_INVALID_ARG;

    const double T = c[0].T;
    if (!(std::isfinite(T) && T > 0.0)) return HESTON_ERR_INVALID_ARG;
    ContractSet<double> cs;
    std::memset(&cs, 0, sizeof(cs));
    cs.n = (int32_t)nc;
    uint32_t M = 0;
    for (uint32_t i = 0; i < nc; ++i) {
        if (c[i].payoff != HESTON_EUROPEAN && c[i].payoff != HESTON_ASIAN_ARITH) return HESTON_ERR_INVALID_ARG;
        if (c[i].is_put != 0 && c[i].is_put != 1) return HESTON_ERR_INVALID_ARG;
        if (c[i].reserved != 0) return HESTON_ERR_INVALID_ARG;
        if (!finite_nonneg(c[i].K) || c[i].T != T) return HESTON_ERR_INVALID_ARG;
        if (c[i].payoff == HESTON_ASIAN_ARITH) {
            const uint32_t Mi = c[i].n_monitor ? c[i].n_monitor : N;
            if (N % Mi != 0) return HESTON_ERR_INVALID_ARG;
            if (M != 0 && Mi != M) return HESTON_ERR_INVALID_ARG;
            M = Mi;
            cs.has_asian = 1;
        }
        cs.payoff[i] = c[i].payoff;
        cs.is_put[i] = c[i].is_put;
        cs.K[i] = c[i].K;
    }
    if (M == 0) M = N;
    cs.M = M;
    cs.stride = N / M;
    cs.T = T;
    cs.D = std::exp(-p->r * T);
    cs.r = p->r;
    cs.S0 = p->S0;
    cs.inv_S0 = 1.0 / p->S0;
    cs.inv_S0sq = 1.0 / (p->S0 * p->S0);
    const double sq = std::sqrt(1.0 - p->rho * p->rho);
    cs.inv_sq = 1.0 / sq;           // inf at |rho| = 1: Gamma is then reported as NaN
    cs.S0_over_M = p->S0 / (double)M;
    cs.dAr_scale = p->S0 * T / ((double)M * (double)M);
    cs.Mp1 = (double)M + 1.0;
    ContractSet<float> csf;
    std::memset(&csf, 0, sizeof(csf));
    csf.n = cs.n; csf.has_asian = cs.has_asian; csf.M = cs.M; csf.stride = cs.stride;
    for (int i = 0; i < kMaxC; ++i) {
        csf.payoff[i] = cs.payoff[i];
        csf.is_put[i] = cs.is_put[i];
        csf.K[i] = (float)cs.K[i];
    }
    csf.T = (float)cs.T; csf.D = (float)cs.D; csf.r = (float)cs.r;
    csf.S0 = (float)cs.S0; csf.inv_S0 = (float)cs.inv_S0; csf.inv_S0sq = (float)cs.inv_S0sq;
    csf.inv_sq = (float)cs.inv_sq; csf.S0_over_M = (float)cs.S0_over_M;
    csf.dAr_scale = (float)cs.dAr_scale; csf.Mp1 = (float)cs.Mp1;

    const double dt = T / (double)N;
    const double ddt = 1.0 / (double)N;
    Coef<double> kd;
    kd.v0 = p->v0;
    kd.dt = dt;
    kd.ddt = ddt;
    kd.half_dt = 0.5 * dt;
    kd.r = p->r;
    kd.kdt = p->kappa * dt;
    kd.kth_dt = p->kappa * p->theta * dt;
    kd.kth_ddt = p->kappa * p->theta * ddt;
    kd.kappa_ddt = p->kappa * ddt;
    kd.xi = p->xi;
    kd.c4 = 0.25 * p->xi * p->xi * dt;
    kd.c4T = 0.25 * p->xi * p->xi * ddt;
    kd.rho = p->rho;
    kd.sq = sq;
    kd.kappa = p->kappa;
    kd.theta = p->theta;
    kd.xrho = p->xi * p->rho;
    kd.xsq = p->xi * sq;
    kd.xi2 = p->xi * p->xi;
    kd.qdt = 0.25 * dt;
    kd.qddt = 0.25 * ddt;
    kd.half_invT = 0.5 / T;
    // QE constants (zero unless the scheme is QE, which has kappa, theta, xi > 0)
    if (o.scheme == HESTON_SCHEME_QE) {
        const double kap = p->kappa, th = p->theta, xi2 = p->xi * p->xi;
        const double E = std::exp(-kap * dt), omE = -std::expm1(-kap * dt);
        const double E_T = -kap * E * ddt;                  // dE/dT
        const double g = omE / kap, g_T = E * ddt;          // (1 - E)/kappa and d/dT
        kd.qE = E;
        kd.qE_T = E_T;
        kd.qmth = th * omE;
        kd.qmth_T = -th * E_T;
        kd.qs1 = xi2 * E * g;
        kd.qs1_T = xi2 * (E_T * g + E * g_T);
        kd.qs0 = 0.5 * th * xi2 * omE * g;
        kd.qs0_T = 0.5 * th * xi2 * (-E_T * g + omE * g_T);
        const double kr = kap * p->rho / p->xi - 0.5;
        kd.qK0r = p->r * dt - p->rho * kap * th * dt / p->xi;
        kd.qK0r_T = p->r * ddt - p->rho * kap * th * ddt / p->xi;
        kd.qK1 = 0.5 * dt * kr - p->rho / p->xi;
        kd.qK2 = 0.5 * dt * kr + p->rho / p->xi;
        kd.qK12_T = 0.5 * ddt * kr;
        kd.qhdt = 0.5 * dt;
        kd.qhddt = 0.5 * ddt;
    }
    const Coef<float> kf = coef_cast<float>(kd);

    out.cs = cs;
    out.csf = csf;
    out.kd = kd;
    out.kf = kf;
    out.opt = o;
    out.N = N;
    out.gamma_nan = (std::fabs(p->rho) == 1.0) || (p->v0 == 0.0);
    return HESTON_OK;
}

uint64_t tiles_for(uint64_t n_paths) { return (n_paths + kTile - 1) / kTile; }
// Threads of a one-contract reduction block: one per (column, part) of the fixed-order sums.
constexpr int kOneContractSumThreads = 12 * kSumParts;
uint64_t groups_for(uint64_t n_tiles) { return (n_tiles + kGroupTiles - 1) / kGroupTiles; }
size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t workspace_bytes(uint32_t nc, uint64_t n_paths)
{
    const uint64_t nt = tiles_for(n_paths);
    const size_t w = 12u * nc * sizeof(double);
    return align256(nt * w) + align256(groups_for(nt) * w);
}

template <typename R, int STEP, int MON>
cudaError_t launch_paths_t(const Prepared &pp, const Coef<R> &k, const Launch &a, cudaStream_t st)
{
    auto kern = heston_paths_kernel<R, STEP, MON>;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int n_sm = 0;
    e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // FP32 launches (every scheme and truncation) of fewer than 3 tiles per
    // SM take the split kernel (two warps per tile, one path per lane): there
    // each packed warp's chain of dependent instructions sets the time, and
    // twice the warps with shorter chains win (2^14 paths: 0.068 -> 0.057 ms);
    // from about 6 tiles per SM the packed kernel's fewer instructions win
    // (2^16: 0.089 ms against 0.100).  An explicit launch shape keeps the
    // packed kernel.
    if constexpr (packed_f32<R, STEP>()) {
        if (!pp.opt.block_threads && !pp.opt.grid_ctas && a.n_tiles < 3u * (uint64_t)n_sm) {
            int per_sm_split = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_split, heston_paths_split_kernel<STEP, MON>,
                                                              64, 0);
            if (e != cudaSuccess) return e;
            {
                const uint64_t full = (uint64_t)n_sm * (uint64_t)(per_sm_split < 1 ? 1 : per_sm_split);
                const uint64_t grid = a.n_tiles < full ? a.n_tiles : full;
                heston_paths_split_kernel<STEP, MON><<<(unsigned)(grid < 1 ? 1 : grid), 64, 0, st>>>(k, cs_of<R>(pp), a);
                return cudaGetLastError();
            }
        }
    }
    int block = pp.opt.block_threads ? (int)pp.opt.block_threads : kPathBlock;
    uint64_t grid;
    if (pp.opt.grid_ctas) {
        grid = pp.opt.grid_ctas;
    } else {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, 0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        uint64_t warps_per_cta = (uint64_t)block / 32;
        uint64_t need = (a.n_tiles + warps_per_cta - 1) / warps_per_cta;
        uint64_t full = (uint64_t)n_sm * (uint64_t)per_sm;
        // A launch that does not fill the machine gets one-warp CTAs, so that its
        // tiles spread evenly over the SMs (4-warp CTAs leave some SMs one CTA
        // and others two).  Tile rows do not depend on the shape.
        if (!pp.opt.block_threads && need < full) {
            int per_sm1 = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm1, kern, 32, 0);
            if (e != cudaSuccess) return e;
            if (per_sm1 < 1) per_sm1 = 1;
            block = 32;
            warps_per_cta = 1;
            need = a.n_tiles;
            full = (uint64_t)n_sm * (uint64_t)per_sm1;
        }
        grid = need < full ? need : full;
    }
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, block, 0, st>>>(k, cs_of<R>(pp), a);
    return cudaGetLastError();
}

int mon_mode(const ContractSet<double> &cs)
{
    if (!cs.has_asian) return MON_NONE;
    return cs.stride == 1 ? MON_EVERY : MON_STRIDE;
}

// Kernel instantiation of the options' scheme and truncation.
int step_of(const heston_options &o)
{
    if (o.scheme == HESTON_SCHEME_QE) return STEP_QE;
    return (o.scheme == HESTON_SCHEME_EULER ? STEP_EUL_FULL : STEP_MIL_FULL) + (o.trunc & 1);
}

template <typename R, int STEP>
cudaError_t launch_paths_s(const Prepared &pp, const Coef<R> &k, const Launch &a, cudaStream_t st)
{
    const int mon = mon_mode(pp.cs);
    if (mon == MON_NONE) return launch_paths_t<R, STEP, MON_NONE>(pp, k, a, st);
    if (mon == MON_EVERY) return launch_paths_t<R, STEP, MON_EVERY>(pp, k, a, st);
    return launch_paths_t<R, STEP, MON_STRIDE>(pp, k, a, st);
}

template <typename R>
cudaError_t launch_paths_r(const Prepared &pp, const Coef<R> &k, const Launch &a, cudaStream_t st)
{
    switch (step_of(pp.opt)) {
    case STEP_MIL_FULL: return launch_paths_s<R, STEP_MIL_FULL>(pp, k, a, st);
    case STEP_MIL_FLOOR: return launch_paths_s<R, STEP_MIL_FLOOR>(pp, k, a, st);
    case STEP_EUL_FULL: return launch_paths_s<R, STEP_EUL_FULL>(pp, k, a, st);
    case STEP_EUL_FLOOR: return launch_paths_s<R, STEP_EUL_FLOOR>(pp, k, a, st);
    default: return launch_paths_s<R, STEP_QE>(pp, k, a, st);
    }
}

cudaError_t launch_paths(const Prepared &pp, const Launch &a, cudaStream_t st)
{
    if (pp.opt.prec == HESTON_FP32) return launch_paths_r<float>(pp, pp.kf, a, st);
    return launch_paths_r<double>(pp, pp.kd, a, st);
}

cudaError_t launch_reduce(const double *tile_sums, uint64_t n_tiles, int nc, uint64_t n_paths,
                          double *group_sums, bool gamma_nan, double *out, cudaStream_t st)
{
    const int width = 12 * nc;
    const uint64_t ng = groups_for(n_tiles);
    // one thread per (column, part) pair of the fixed-order sums: 8 x 12 per contract
    const int threads = std::min(1024, ((8 * width + 31) / 32) * 32);
    reduce_groups_kernel<<<(unsigned)ng, threads, 0, st>>>(tile_sums, n_tiles, width, group_sums);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_final_kernel<<<1, threads, 0, st>>>(group_sums, ng, nc, (double)n_paths, gamma_nan ? 1 : 0, out);
    return cudaGetLastError();
}

PhiloxKey key_of(uint64_t seed) { return PhiloxKey{(uint32_t)seed, (uint32_t)(seed >> 32)}; }

int enqueue(const Prepared &pp, uint64_t n_paths, uint64_t seed, void *ws, size_t ws_bytes,
            double *d_out, cudaStream_t st)
{
    const uint64_t nt = tiles_for(n_paths);
    const size_t w = 12u * (size_t)pp.cs.n * sizeof(double);
    if (!ws || ((uintptr_t)ws & 255u) || ws_bytes < workspace_bytes(pp.cs.n, n_paths) || !d_out)
        return HESTON_ERR_WORKSPACE;
    double *tile_sums = (double *)ws;
    double *group_sums = (double *)((char *)ws + align256(nt * w));
    Launch a;
    a.key = key_of(seed);
    a.path_begin = 0;
    a.n_paths = n_paths;
    a.n_tiles = nt;
    a.N = pp.N;
    a.tile_sums = tile_sums;
    if (launch_paths(pp, a, st) != cudaSuccess) return HESTON_ERR_CUDA;
    if (launch_reduce(tile_sums, nt, pp.cs.n, n_paths, group_sums, pp.gamma_nan, d_out, st) != cudaSuccess)
        return HESTON_ERR_CUDA;
    return HESTON_OK;
}

// Fill host results; returns the largest per-contract status (a warning
// for non-finite Vega / Theta outranks the Gamma one).
int fill_results(const double *h, uint32_t nc, uint64_t n_paths, int status, heston_result *out)
{
    int worst = status;
    for (uint32_t c = 0; c < nc; ++c) {
        heston_result &r = out[c];
        r.price = h[c * 12 + 0]; r.delta = h[c * 12 + 1]; r.gamma = h[c * 12 + 2];
        r.vega = h[c * 12 + 3];  r.rho = h[c * 12 + 4];   r.theta = h[c * 12 + 5];
        for (int j = 0; j < 6; ++j) r.se[j] = h[c * 12 + 6 + j];
        r.n_paths = n_paths;
        r.status = status;
        if (!std::isfinite(r.vega) || !std::isfinite(r.theta) || !std::isfinite(r.se[3]) ||
            !std::isfinite(r.se[5]))
            r.status = HESTON_WARN_TANGENT_UNSTABLE;
        if (r.status > worst) worst = r.status;
        r.reserved = 0;
    }
    return worst;
}


// ---------------------------------------------------------------------------
// Host: QMC tables (Sobol direction integers, per-tile low-bit table, bridge
// event plan), their layout in a caller buffer, and the QMC launch.
// ---------------------------------------------------------------------------
uint64_t gf2_mulmod(uint64_t a, uint64_t b, uint64_t mod, int deg)
{
    uint64_t r = 0;
    while (b) {
        if (b & 1u) r ^= a;
        b >>= 1;
        a <<= 1;
        if ((a >> deg) & 1u) a ^= mod;
    }
    return r;
}

uint64_t gf2_powmod(uint64_t base, uint64_t e, uint64_t mod, int deg)
{
    uint64_t r = 1;
    while (e) {
        if (e & 1u) r = gf2_mulmod(r, base, mod, deg);
        base = gf2_mulmod(base, base, mod, deg);
        e >>= 1;
    }
    return r;
}

int degree_of(uint32_t poly)
{
    int d = -1;
    while (poly) { ++d; poly >>= 1; }
    return d;
}

// Primitive over GF(2): constant term 1 and x of order 2^s - 1 modulo poly.
bool gf2_primitive(uint32_t poly)
{
    const int s = degree_of(poly);
    if (s < 1 || !(poly & 1u)) return false;
    if (s == 1) return poly == 3u;
    const uint64_t order = (1ull << s) - 1;
    if (gf2_powmod(2, order, poly, s) != 1) return false;
    uint64_t n = order;
    for (uint64_t q = 2; q * q <= n; ++q) {
        if (n % q) continue;
        if (gf2_powmod(2, order / q, poly, s) == 1) return false;
        while (n % q == 0) n /= q;
    }
    if (n > 1 && gf2_powmod(2, order / n, poly, s) == 1) return false;
    return true;
}

// Bratley-Fox recurrence from the initial m_1..m_s to v_1..v_32.
void sobol_recurrence(uint32_t poly, const uint32_t *m_init, uint32_t *v)
{
    const int s = degree_of(poly);
    uint64_t m[32];
    for (int k = 0; k < s && k < 32; ++k) m[k] = m_init[k];
    for (int k = s; k < 32; ++k) {
        uint64_t val = m[k - s] ^ (m[k - s] << s);
        for (int i = 1; i < s; ++i)
            if ((poly >> (s - i)) & 1u) val ^= m[k - i] << i;
        m[k] = val;
    }
    for (int k = 0; k < 32; ++k) v[k] = (uint32_t)(m[k] << (31 - k));
}

uint32_t first_digit_row(const uint32_t *v, int n_cols)
{
    uint32_t row = 0;
    for (int k = 0; k < n_cols; ++k) row |= ((v[k] >> 31) & 1u) << k;
    return row;
}

// GF(2) elimination: rows independent?
bool gf2_independent(std::vector<uint32_t> rows)
{
    for (size_t i = 0; i < rows.size(); ++i) {
        if (!rows[i]) return false;
        const uint32_t low = rows[i] & (~rows[i] + 1u);      // pivot: lowest set bit
        for (size_t j = i + 1; j < rows.size(); ++j)
            if (rows[j] & low) rows[j] ^= rows[i];
    }
    return true;
}

void sobol_directions_host(uint32_t D, uint32_t *V)
{
    for (int k = 0; k < 32; ++k) V[k] = 1u << (31 - k);
    uint32_t poly = 2;                                    // next candidate polynomial
    const PhiloxKey key{kSobolKey0, kSobolKey1};
    for (uint32_t j = 1; j < D; ++j) {
        while (!gf2_primitive(poly)) ++poly;
        const uint32_t P = poly++;
        const int s = degree_of(P);
        uint32_t v[32], v0[32];
        auto candidate = [&](uint32_t c, uint32_t *out) {
            uint32_t m[32];
            for (int k = 1; k <= s; ++k) {
                const uint4 w = philox4x32_10(make_uint4((uint32_t)(k - 1) / 4u, j, c, kSobolInitTag), key);
                const int sel = (k - 1) % 4;
                const uint32_t word = sel == 0 ? w.x : sel == 1 ? w.y : sel == 2 ? w.z : w.w;
                m[k - 1] = 2u * (word % (1u << (k - 1))) + 1u;
            }
            sobol_recurrence(P, m, out);
        };
        candidate(0, v0);
        const uint32_t *chosen = v0;
        if (j < 32) {
            const int n_cols = (int)j + 1;
            std::vector<uint32_t> rows;
            for (uint32_t i = 0; i < j; ++i) rows.push_back(first_digit_row(V + i * 32u, n_cols));
            for (uint32_t c = 0; c < 64; ++c) {
                candidate(c, v);
                rows.push_back(first_digit_row(v, n_cols));
                const bool ok = gf2_independent(rows);
                rows.pop_back();
                if (ok) { chosen = v; break; }
            }
        }
        std::memcpy(V + j * 32u, chosen, sizeof(uint32_t) * 32);
    }
}

struct BridgePlanHost {
    uint32_t N = 0;
    int depth = 0;
    std::vector<BridgeOp> ev;
    std::vector<int32_t> off;
};

// Breadth-first bisection (node indices, hence Sobol dimensions) and the
// time-ordered stack plan of pushes per step (see the device comment).
bool plan_bridge(uint32_t N, BridgePlanHost &out)
{
    if (N == 0 || N > kQmcMaxSteps) return false;
    struct Node { uint32_t m, l, r; };
    std::vector<Node> nodes;
    std::map<std::pair<uint32_t, uint32_t>, int> node_of;   // interval -> node index
    nodes.push_back({N, 0, N});
    std::deque<std::pair<uint32_t, uint32_t>> queue;
    queue.push_back({0, N});
    while (!queue.empty()) {
        const auto iv = queue.front();
        queue.pop_front();
        if (iv.second - iv.first < 2) continue;
        const uint32_t m = iv.first + (iv.second - iv.first) / 2;
        node_of[iv] = (int)nodes.size();
        nodes.push_back({m, iv.first, iv.second});
        queue.push_back({iv.first, m});
        queue.push_back({m, iv.second});
    }
    if (nodes.size() != N) return false;
    out.N = N;
    out.depth = 0;
    out.ev.clear();
    out.off.assign(N + 1, 0);
    std::vector<uint32_t> right;            // right ends of the open intervals (stack)
    for (uint32_t k = 0; k < N; ++k) {
        out.off[k] = (int32_t)out.ev.size();
        if (k == 0) {
            out.ev.push_back({0, 0.0f, (float)std::sqrt((double)N), 0});
            right.push_back(N);
        }
        uint32_t r = right.back();
        while (r - k >= 2) {
            const auto it = node_of.find({k, r});
            if (it == node_of.end()) return false;
            const double m = nodes[it->second].m;
            out.ev.push_back({it->second, (float)((m - k) / (double)(r - k)),
                              (float)std::sqrt((m - k) * (r - m) / (double)(r - k)), 0});
            right.push_back((uint32_t)m);
            r = (uint32_t)m;
        }
        if (r != k + 1) return false;
        if ((int)right.size() > out.depth) out.depth = (int)right.size();
        if (out.depth >= kQmcMaxLevels) return false;
        right.pop_back();
    }
    out.off[N] = (int32_t)out.ev.size();
    return true;
}

struct QmcLayout {
    size_t off_V, off_T, off_evoff, off_ev, total;
};

QmcLayout qmc_layout(uint32_t N, size_t n_ev)
{
    const size_t D = 2u * (size_t)N;
    QmcLayout L;
    L.off_V = 0;
    L.off_T = align256(L.off_V + D * 32 * sizeof(uint32_t));
    L.off_evoff = align256(L.off_T + D * 64 * sizeof(uint32_t));     // N nodes x 32 lanes x uint4
    L.off_ev = align256(L.off_evoff + (N + 1) * sizeof(int32_t));
    L.total = align256(L.off_ev + n_ev * sizeof(BridgeOp));
    return L;
}

QmcTables qmc_tables_at(const void *base, const QmcLayout &L)
{
    const char *b = (const char *)base;
    return QmcTables{(const uint32_t *)(b + L.off_V), (const uint4 *)(b + L.off_T),
                     (const BridgeOp *)(b + L.off_ev), (const int32_t *)(b + L.off_evoff)};
}

// QMC workspace: tile rows | group sums [R][gpr] | replicate averages [R][6 nc] |
// U [tpr][D] | shifts [R][D].
struct QmcWs {
    size_t off_rows, off_groups, off_rep, off_U, off_shift, total;
};

QmcWs qmc_ws_layout(uint32_t nc, uint64_t n_paths, uint32_t N, uint32_t R)
{
    const size_t w = 12u * nc * sizeof(double);
    const uint64_t tiles = tiles_for(n_paths);
    const uint64_t tpr = tiles / R;
    const size_t D = 2u * (size_t)N;
    QmcWs L;
    L.off_rows = 0;
    L.off_groups = align256(tiles * w);
    L.off_rep = L.off_groups + align256((size_t)R * groups_for(tpr) * w);
    L.off_U = L.off_rep + align256((size_t)R * 6u * nc * sizeof(double));
    L.off_shift = L.off_U + align256(tpr * D * sizeof(uint32_t));
    L.total = L.off_shift + align256((size_t)R * D * sizeof(uint32_t));
    return L;
}

int validate_qmc(uint64_t n_paths, uint32_t N, const Prepared &pp)
{
    if (pp.opt.prec != HESTON_FP32) return HESTON_ERR_UNSUPPORTED;
    const uint32_t R = pp.opt.n_shifts;
    if (R < 2 || n_paths % R) return HESTON_ERR_INVALID_ARG;
    const uint64_t ppr = n_paths / R;
    if (ppr % kTile || ppr > (1ull << 32)) return HESTON_ERR_INVALID_ARG;
    if (N > kQmcMaxSteps) return HESTON_ERR_UNSUPPORTED;
    return HESTON_OK;
}

template <int TRUNC, int MON>
cudaError_t launch_qmc_t(const Prepared &pp, const QmcLaunch &a, cudaStream_t st)
{
    auto kern = heston_qmc_kernel<TRUNC, MON>;
    const int block = pp.opt.block_threads ? (int)pp.opt.block_threads : kPathBlock;
    // the bridge plan, one row of D high-bit words per warp and (16-byte aligned)
    // one bridge stack of depth x 32 float4 per warp in shared memory
    const size_t smem = (size_t)(a.n_ev + 1u) * sizeof(BridgeOp) + (size_t)((a.N + 4u) & ~3u) * sizeof(int32_t)
                        + (size_t)(block / 32) * a.D * sizeof(uint32_t) + 16u
                        + (size_t)(block / 32) * a.depth * 32u * sizeof(float4);
    int dev = 0, n_sm = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess && smem > 48 * 1024)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const uint64_t warps_per_cta = (uint64_t)block / 32;
    uint64_t grid = pp.opt.grid_ctas ? pp.opt.grid_ctas
                                     : std::min<uint64_t>((a.n_tiles + warps_per_cta - 1) / warps_per_cta,
                                                          (uint64_t)n_sm * per_sm);
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, block, smem, st>>>(pp.kf, pp.csf, a);
    return cudaGetLastError();
}

int enqueue_qmc(const Prepared &pp, uint64_t n_paths, uint64_t seed, const void *d_tables,
                void *ws, size_t ws_bytes, double *d_out, cudaStream_t st)
{
    BridgePlanHost plan;
    if (!plan_bridge(pp.N, plan)) return HESTON_ERR_UNSUPPORTED;
    const QmcLayout TL = qmc_layout(pp.N, plan.ev.size());
    const uint32_t R = pp.opt.n_shifts;
    const QmcWs WL = qmc_ws_layout(pp.cs.n, n_paths, pp.N, R);
    if (!d_tables || ((uintptr_t)d_tables & 255u)) return HESTON_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws & 255u) || ws_bytes < WL.total || !d_out) return HESTON_ERR_WORKSPACE;
    char *b = (char *)ws;
    QmcLaunch a;
    a.tb = qmc_tables_at(d_tables, TL);
    a.n_ev = (uint32_t)plan.ev.size();
    a.depth = (uint32_t)plan.depth;
    a.D = 2u * pp.N;
    a.N = pp.N;
    a.n_tiles = tiles_for(n_paths);
    a.tpr = (uint32_t)(a.n_tiles / R);
    a.tile_sums = (double *)(b + WL.off_rows);
    uint32_t *U = (uint32_t *)(b + WL.off_U);
    uint32_t *shift = (uint32_t *)(b + WL.off_shift);
    a.U = U;
    a.shift = shift;
    const uint64_t n_setup = (uint64_t)a.tpr * a.D + (uint64_t)R * a.D;
    qmc_setup_kernel<<<(unsigned)((n_setup + 255) / 256), 256, 0, st>>>(a.tb.V, a.D, a.tpr, R,
                                                                       key_of(seed), U, shift);
    if (cudaGetLastError() != cudaSuccess) return HESTON_ERR_CUDA;
    const int mon = mon_mode(pp.cs);
    const bool full = pp.opt.trunc == HESTON_TRUNC_FULL;
    cudaError_t e;
    if (full) e = mon == MON_NONE ? launch_qmc_t<0, MON_NONE>(pp, a, st)
                : mon == MON_EVERY ? launch_qmc_t<0, MON_EVERY>(pp, a, st) : launch_qmc_t<0, MON_STRIDE>(pp, a, st);
    else      e = mon == MON_NONE ? launch_qmc_t<1, MON_NONE>(pp, a, st)
                : mon == MON_EVERY ? launch_qmc_t<1, MON_EVERY>(pp, a, st) : launch_qmc_t<1, MON_STRIDE>(pp, a, st);
    if (e != cudaSuccess) return HESTON_ERR_CUDA;
    const int width = 12 * pp.cs.n;
    const uint32_t gpr = (uint32_t)groups_for(a.tpr);
    double *groups = (double *)(b + WL.off_groups);
    // one thread per (column, part) pair of the fixed-order sums, as launch_reduce
    const int threads = std::min(1024, ((8 * width + 31) / 32) * 32);
    reduce_replicate_groups_kernel<<<(unsigned)((uint64_t)R * gpr), threads, 0, st>>>(a.tile_sums, a.tpr, gpr,
                                                                                      width, groups);
    if (cudaGetLastError() != cudaSuccess) return HESTON_ERR_CUDA;
    reduce_final_qmc_kernel<<<1, 256, 0, st>>>(groups, R, gpr, pp.cs.n, (double)(n_paths / R),
                                               pp.gamma_nan ? 1 : 0, (double *)(b + WL.off_rep), d_out);
    return cudaGetLastError() == cudaSuccess ? HESTON_OK : HESTON_ERR_CUDA;
}

// Build the tables on the host and copy them to d_tables (synchronous).
int build_qmc_tables(uint32_t N, void *d_tables, size_t bytes)
{
    BridgePlanHost plan;
    if (!plan_bridge(N, plan)) return HESTON_ERR_UNSUPPORTED;
    const QmcLayout L = qmc_layout(N, plan.ev.size());
    if (!d_tables || ((uintptr_t)d_tables & 255u) || bytes < L.total) return HESTON_ERR_WORKSPACE;
    const uint32_t D = 2u * N;
    std::vector<unsigned char> h(L.total, 0);
    uint32_t *V = (uint32_t *)(h.data() + L.off_V);
    uint32_t *T = (uint32_t *)(h.data() + L.off_T);
    sobol_directions_host(D, V);
    // interleaved per bridge node j and lane l: x_{2j}(l), x_{2j}(l + 32), x_{2j+1}(l), x_{2j+1}(l + 32),
    // low 8 bits cleared (the uniform uses the top 24 bits of a word)
    for (uint32_t d = 0; d < D; ++d)
        for (uint32_t p = 0; p < 64; ++p) {
            uint32_t x = 0;
            for (int b = 0; b < 6; ++b)
                if ((p >> b) & 1u) x ^= V[d * 32u + b];
            T[((d >> 1) * 32u + (p & 31u)) * 4u + (d & 1u) * 2u + (p >> 5)] = x & 0xFFFFFF00u;
        }
    std::memcpy(h.data() + L.off_evoff, plan.off.data(), plan.off.size() * sizeof(int32_t));
    std::memcpy(h.data() + L.off_ev, plan.ev.data(), plan.ev.size() * sizeof(BridgeOp));
    if (cudaMemcpy(d_tables, h.data(), L.total, cudaMemcpyHostToDevice) != cudaSuccess) return HESTON_ERR_CUDA;
    return HESTON_OK;
}


// ---------------------------------------------------------------------------
// Host: batched launch
// ---------------------------------------------------------------------------
struct BatchDescLayout {
    size_t off_items, off_work_begin, off_work_item, off_group_begin, total;
};

BatchDescLayout batch_desc_layout(uint32_t n)
{
    BatchDescLayout L;
    L.off_items = 0;
    L.off_work_begin = align256((size_t)n * sizeof(BatchItemDev));
    L.off_work_item = L.off_work_begin + align256((size_t)n * sizeof(uint64_t));
    L.off_group_begin = L.off_work_item + align256((size_t)n * sizeof(uint32_t));
    L.total = L.off_group_begin + align256((size_t)n * sizeof(uint64_t));
    return L;
}

// Workspace: counter | tile rows | group rows.
struct BatchWsLayout {
    size_t off_counter, off_rows, off_groups, total;
};

BatchWsLayout batch_ws_layout(uint64_t tiles, uint64_t groups)
{
    BatchWsLayout L;
    L.off_counter = 0;
    L.off_rows = 256;
    L.off_groups = L.off_rows + align256(tiles * 12u * sizeof(double));
    L.total = L.off_groups + align256(groups * 12u * sizeof(double));
    return L;
}

int batch_prepare_items(const heston_batch_item *items, uint32_t n, const heston_options *opts,
                        std::vector<BatchItemDev> *dev, heston_batch_plan *plan)
{
    if (!items || n == 0 || !plan) return HESTON_ERR_INVALID_ARG;
    heston_options o;
    if (opts) o = *opts; else { std::memset(&o, 0, sizeof(o)); o.device = -1; }
    if (o.prec != HESTON_FP32 || o.rng != HESTON_RNG_PHILOX || o.scheme != HESTON_SCHEME_MILSTEIN)
        return HESTON_ERR_UNSUPPORTED;
    uint64_t tiles = 0, groups = 0, ps = 0;
    if (dev) dev->resize(n);
    for (uint32_t i = 0; i < n; ++i) {
        if (items[i].reserved != 0) return HESTON_ERR_INVALID_ARG;
        Prepared pp;
        const int rc = validate_and_prepare(&items[i].params, &items[i].contract, 1, items[i].n_paths,
                                            items[i].n_steps, &o, pp);
        if (rc < 0) return rc;
        const uint64_t nt = tiles_for(items[i].n_paths);
        if (dev) {
            BatchItemDev &d = (*dev)[i];
            std::memset(&d, 0, sizeof(d));
            d.k = pp.kf;
            d.cs = pp.csf;
            d.key = key_of(items[i].rng_seed);
            d.n_paths = items[i].n_paths;
            d.n_tiles = nt;
            d.row_begin = tiles;
            d.group_begin = groups;
            d.N = items[i].n_steps;
            d.mon = mon_mode(pp.cs);
            d.gamma_nan = pp.gamma_nan ? 1 : 0;
        }
        tiles += nt;
        groups += groups_for(nt);
        ps += items[i].n_paths * (uint64_t)items[i].n_steps;
    }
    plan->total_tiles = tiles;
    plan->total_groups = groups;
    plan->total_path_steps = ps;
    plan->n_items = n;
    plan->trunc = o.trunc;
    plan->descriptor_bytes = batch_desc_layout(n).total;
    plan->workspace_bytes = batch_ws_layout(tiles, groups).total;
    return HESTON_OK;
}

int batch_prepare(const heston_batch_item *items, const heston_options *opts,
                  const heston_batch_plan *plan, void *d_desc)
{
    if (!plan || !d_desc || ((uintptr_t)d_desc & 255u)) return HESTON_ERR_INVALID_ARG;
    const uint32_t n = plan->n_items;
    std::vector<BatchItemDev> dev;
    heston_batch_plan check;
    int rc = batch_prepare_items(items, n, opts, &dev, &check);
    if (rc < 0) return rc;
    if (check.total_tiles != plan->total_tiles || check.total_groups != plan->total_groups)
        return HESTON_ERR_INVALID_ARG;
    // work order: most steps first (ties: caller order)
    std::vector<uint32_t> order(n);
    for (uint32_t i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t x, uint32_t y) { return dev[x].N > dev[y].N; });
    std::vector<uint64_t> wb(n), gb(n);
    uint64_t acc = 0;
    for (uint32_t p = 0; p < n; ++p) { wb[p] = acc; acc += dev[order[p]].n_tiles; }
    for (uint32_t i = 0; i < n; ++i) gb[i] = dev[i].group_begin;
    const BatchDescLayout L = batch_desc_layout(n);
    std::vector<unsigned char> h(L.total, 0);
    std::memcpy(h.data() + L.off_items, dev.data(), n * sizeof(BatchItemDev));
    std::memcpy(h.data() + L.off_work_begin, wb.data(), n * sizeof(uint64_t));
    std::memcpy(h.data() + L.off_work_item, order.data(), n * sizeof(uint32_t));
    std::memcpy(h.data() + L.off_group_begin, gb.data(), n * sizeof(uint64_t));
    if (cudaMemcpy(d_desc, h.data(), L.total, cudaMemcpyHostToDevice) != cudaSuccess) return HESTON_ERR_CUDA;
    return HESTON_OK;
}

template <int TRUNC>
cudaError_t launch_batch_t(const BatchLaunch &a, const heston_options &o, cudaStream_t st)
{
    auto kern = heston_batch_kernel<TRUNC>;
    int dev = 0, n_sm = 0, per_sm = 0;
    const int block = o.block_threads ? (int)o.block_threads : kPathBlock;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const uint64_t warps_per_cta = (uint64_t)block / 32;
    uint64_t grid = o.grid_ctas ? o.grid_ctas
                                : std::min<uint64_t>((a.total_work + warps_per_cta - 1) / warps_per_cta,
                                                     (uint64_t)n_sm * per_sm);
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

int batch_launch(const heston_batch_plan *plan, const void *d_desc, const heston_options *opts,
                 void *ws, double *d_out, int32_t *d_status)
{
    if (!plan || !d_desc || !ws || !d_out || ((uintptr_t)d_desc & 255u) || ((uintptr_t)ws & 255u))
        return HESTON_ERR_INVALID_ARG;
    heston_options o;
    if (opts) o = *opts; else { std::memset(&o, 0, sizeof(o)); o.device = -1; }
    if (o.block_threads != 0 && (o.block_threads % 32 != 0 || o.block_threads > kPathBlock))
        return HESTON_ERR_INVALID_ARG;
    DeviceGuard g(o.device);
    if (g.err != cudaSuccess) return HESTON_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)o.cuda_stream;
    const uint32_t n = plan->n_items;
    const BatchDescLayout L = batch_desc_layout(n);
    const BatchWsLayout W = batch_ws_layout(plan->total_tiles, plan->total_groups);
    const char *d = (const char *)d_desc;
    char *w = (char *)ws;
    BatchLaunch a;
    a.items = (const BatchItemDev *)(d + L.off_items);
    a.work_begin = (const uint64_t *)(d + L.off_work_begin);
    a.work_item = (const uint32_t *)(d + L.off_work_item);
    a.work_tile0 = nullptr;
    a.group_begin = (const uint64_t *)(d + L.off_group_begin);
    a.n_items = n;
    a.total_work = plan->total_tiles;
    a.counter = (unsigned long long *)(w + W.off_counter);
    a.status = d_status;
    a.rows = (double *)(w + W.off_rows);
    if (cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), st) != cudaSuccess) return HESTON_ERR_CUDA;
    const cudaError_t e = plan->trunc == HESTON_TRUNC_FULL ? launch_batch_t<0>(a, o, st) : launch_batch_t<1>(a, o, st);
    if (e != cudaSuccess) return HESTON_ERR_CUDA;
    double *groups = (double *)(w + W.off_groups);
    batch_reduce_groups_kernel<<<(unsigned)plan->total_groups, kOneContractSumThreads, 0, st>>>(a.items, a.group_begin, n,
                                                                            a.rows, groups);
    if (cudaGetLastError() != cudaSuccess) return HESTON_ERR_CUDA;
    batch_reduce_final_kernel<<<n, kOneContractSumThreads, 0, st>>>(a.items, groups, d_out);
    return cudaGetLastError() == cudaSuccess ? HESTON_OK : HESTON_ERR_CUDA;
}


// ---------------------------------------------------------------------------
// Host: adjoint gradient
// ---------------------------------------------------------------------------
struct AdjLayout {
    uint32_t C, n_seg;
    size_t off_ckpt, off_seed, off_rows, off_groups, total;
};

AdjLayout adj_layout(uint64_t n_paths, uint32_t N)
{
    AdjLayout L;
    L.C = (uint32_t)kAdjSeg;
    L.n_seg = (N + L.C - 1) / L.C;
    const uint64_t tiles = tiles_for(n_paths);
    L.off_ckpt = 0;
    L.off_seed = align256((size_t)L.n_seg * n_paths * sizeof(float2));
    L.off_rows = L.off_seed + align256(n_paths * sizeof(float2));
    L.off_groups = L.off_rows + align256(tiles * 14u * sizeof(double));
    L.total = L.off_groups + align256(groups_for(tiles) * 14u * sizeof(double));
    return L;
}

template <int MON>
cudaError_t launch_adj_t(bool backward, const Prepared &pp, const AdjLaunch &a, cudaStream_t st)
{
    int dev = 0, n_sm = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (backward) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, heston_adj_bwd_kernel<MON>,
                                                                    kPathBlock, 0);
    else          e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, heston_adj_fwd_kernel<MON>, kPathBlock, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    uint64_t grid = std::min<uint64_t>((a.n_tiles + 3) / 4, (uint64_t)n_sm * per_sm);
    if (pp.opt.grid_ctas) grid = pp.opt.grid_ctas;
    if (grid < 1) grid = 1;
    if (backward) heston_adj_bwd_kernel<MON><<<(unsigned)grid, kPathBlock, 0, st>>>(pp.kf, pp.csf, a, (float)pp.cs.T);
    else          heston_adj_fwd_kernel<MON><<<(unsigned)grid, kPathBlock, 0, st>>>(pp.kf, pp.csf, a);
    return cudaGetLastError();
}

int adjoint_enqueue(bool backward, const heston_params *params, const heston_contract *contract,
                    uint64_t n_paths, uint32_t N, uint64_t seed, const heston_options *opts,
                    void *ws, size_t ws_bytes, double *d_out, double *d_per_path = nullptr)
{
    Prepared pp;
    int rc = validate_and_prepare(params, contract, 1, n_paths, N, opts, pp);
    if (rc < 0) return rc;
    if (pp.opt.prec != HESTON_FP32 || pp.opt.trunc != HESTON_TRUNC_FULL || pp.opt.rng != HESTON_RNG_PHILOX ||
        pp.opt.scheme != HESTON_SCHEME_MILSTEIN)
        return HESTON_ERR_UNSUPPORTED;
    const AdjLayout L = adj_layout(n_paths, N);
    if (N > kAdjMaxSteps) return HESTON_ERR_UNSUPPORTED;
    if (!d_out) return HESTON_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws & 255u) || ws_bytes < L.total) return HESTON_ERR_WORKSPACE;
    DeviceGuard g(pp.opt.device);
    if (g.err != cudaSuccess) return HESTON_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)pp.opt.cuda_stream;
    char *b = (char *)ws;
    AdjLaunch a;
    a.key = key_of(seed);
    a.n_paths = n_paths;
    a.n_tiles = tiles_for(n_paths);
    a.N = N;
    a.C = L.C;
    a.n_seg = L.n_seg;
    a.ckpt = (float2 *)(b + L.off_ckpt);
    a.seed = (float2 *)(b + L.off_seed);
    a.rows = (double *)(b + L.off_rows);
    a.per_path = d_per_path;
    const int mon = mon_mode(pp.cs);
    cudaError_t e = mon == MON_NONE ? launch_adj_t<MON_NONE>(backward, pp, a, st)
                  : mon == MON_EVERY ? launch_adj_t<MON_EVERY>(backward, pp, a, st)
                                     : launch_adj_t<MON_STRIDE>(backward, pp, a, st);
    if (e != cudaSuccess) return HESTON_ERR_CUDA;
    const int width = backward ? 14 : 2;
    double *groups = (double *)(b + L.off_groups);
    const uint64_t ng = groups_for(a.n_tiles);
    reduce_groups_kernel<<<(unsigned)ng, 64, 0, st>>>(a.rows, a.n_tiles, width, groups);
    if (cudaGetLastError() != cudaSuccess) return HESTON_ERR_CUDA;
    reduce_generic_final_kernel<<<1, 32, 0, st>>>(groups, ng, width / 2, (double)n_paths, d_out);
    return cudaGetLastError() == cudaSuccess ? HESTON_OK : HESTON_ERR_CUDA;
}


// ---------------------------------------------------------------------------
// Serving engine: continuous batching over the persistent batch kernel
// ---------------------------------------------------------------------------
}  // namespace

struct heston_server {
    heston_server_config cfg;
    int device = 0;
    cudaStream_t strm[2] = {nullptr, nullptr};   // rounds alternate between two streams
    int n_sm = 0, per_sm = 0;
    // device buffers
    BatchItemDev *d_slots = nullptr;
    double *d_pool = nullptr;
    double *d_groups[2] = {nullptr, nullptr};    // group rows of the round's finishing requests
    char *d_pack[2] = {nullptr, nullptr};        // the round's work lists (RoundLayout)
    double *d_res[2] = {nullptr, nullptr};       // results of the finishing requests, in list order
    // pinned host staging
    BatchItemDev *h_slots = nullptr;
    char *h_pack[2] = {nullptr, nullptr};
    double *h_res[2] = {nullptr, nullptr};
    cudaEvent_t ev[2] = {nullptr, nullptr};      // round on buffer b done (results on the host)
    cudaEvent_t ev_copy[2] = {nullptr, nullptr}; // round's copies done
    cudaEvent_t ev_kern[2] = {nullptr, nullptr}; // round's path kernel done
    // host state
    struct Req {
        uint64_t ticket = 0;
        BatchItemDev dev;
        uint64_t tiles = 0, next_tile = 0;
        size_t bytes = 0, pool_off = 0;
        int slot = -1;
        std::chrono::steady_clock::time_point t_submit;
    };
    struct Done {
        heston_result res;
        double latency;
    };
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req> queue;
    std::vector<Req> slots;                     // by slot; ticket 0 = free
    std::vector<int> free_slots;
    std::vector<uint64_t> order;                // active tickets in admission order (slot ids)
    std::map<size_t, size_t> free_blocks;       // pool offset -> size (bytes)
    std::unordered_map<uint64_t, Done> done;
    std::vector<int> pending[2];                // slots finishing in the round on buffer b
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread th;
    heston_server_stats st{};
    size_t pool_bytes = 0;
};

namespace {

size_t srv_alloc(heston_server *s, size_t bytes)
{
    for (auto it = s->free_blocks.begin(); it != s->free_blocks.end(); ++it) {
        if (it->second >= bytes) {
            const size_t off = it->first, sz = it->second;
            s->free_blocks.erase(it);
            if (sz > bytes) s->free_blocks[off + bytes] = sz - bytes;
            return off;
        }
    }
    return (size_t)-1;
}

void srv_free(heston_server *s, size_t off, size_t bytes)
{
    auto it = s->free_blocks.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != s->free_blocks.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        s->free_blocks.erase(nx);
    }
    if (it != s->free_blocks.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            s->free_blocks.erase(it);
        }
    }
}

// Pool blocks are multiples of 768 bytes (lcm of the 96-byte tile row and
// 256-byte alignment), so every block starts on a whole tile row.
constexpr size_t kPoolUnit = 768;
size_t srv_req_bytes(uint64_t tiles)
{
    const size_t b = tiles * 12u * sizeof(double);
    return (b + kPoolUnit - 1) / kPoolUnit * kPoolUnit;
}

// One round's work lists in a single pinned buffer (one copy per round):
// the work counter (zero), then per position its first work index, first
// tile and slot, then per finishing request its first group row and slot.
struct RoundLayout {
    size_t wb, wt, wi, fg, fs, total;
};
RoundLayout round_layout(size_t n, size_t nf)
{
    RoundLayout L;
    L.wb = 8;
    L.wt = L.wb + 8 * n;
    L.wi = L.wt + 8 * n;
    L.fg = (L.wi + 4 * n + 7) & ~(size_t)7;
    L.fs = L.fg + 8 * nf;
    L.total = L.fs + 4 * nf;
    return L;
}

// Retire the requests whose reduction ran in the round on buffer b.
void srv_retire(heston_server *s, int b)
{
    if (s->pending[b].empty()) return;
    const bool failed = cudaEventSynchronize(s->ev[b]) != cudaSuccess;
    const auto now = std::chrono::steady_clock::now();
    std::lock_guard<std::mutex> lock(s->mu);
    for (size_t p = 0; p < s->pending[b].size(); ++p) {
        const int slot = s->pending[b][p];
        heston_server::Req &r = s->slots[slot];
        heston_server::Done d;
        const bool gn = r.dev.gamma_nan != 0;
        fill_results(s->h_res[b] + p * 12u, 1, r.dev.n_paths,
                     gn ? HESTON_WARN_GAMMA_UNDEFINED : HESTON_OK, &d.res);
        if (failed) d.res.status = HESTON_ERR_CUDA;
        d.latency = std::chrono::duration<double>(now - r.t_submit).count();
        s->done[r.ticket] = d;
        srv_free(s, r.pool_off, r.bytes);
        s->st.memory_in_use -= r.bytes;
        s->st.completed += 1;
        s->st.active -= 1;
        s->order.erase(std::find(s->order.begin(), s->order.end(), (uint64_t)slot));
        r.ticket = 0;
        s->free_slots.push_back(slot);
    }
    s->pending[b].clear();
    s->cv_done.notify_all();
}

void srv_loop(heston_server *s)
{
    cudaSetDevice(s->device);
    int b = 0;
    const uint64_t budget = s->cfg.tiles_per_round;
    for (;;) {
        std::vector<int> round_slots;
        std::vector<uint64_t> round_tiles;
        std::vector<int> finishing;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            // admission: FIFO while a slot and pool memory are free
            while (!s->queue.empty() && !s->free_slots.empty()) {
                heston_server::Req &q = s->queue.front();
                const size_t off = srv_alloc(s, q.bytes);
                if (off == (size_t)-1) break;
                const int slot = s->free_slots.back();
                s->free_slots.pop_back();
                q.pool_off = off;
                q.slot = slot;
                q.dev.row_begin = off / (12u * sizeof(double));
                s->h_slots[slot] = q.dev;
                cudaMemcpyAsync(s->d_slots + slot, s->h_slots + slot, sizeof(BatchItemDev),
                                cudaMemcpyHostToDevice, s->strm[b]);
                s->slots[slot] = q;
                s->order.push_back((uint64_t)slot);
                s->st.memory_in_use += q.bytes;
                if (s->st.memory_in_use > s->st.memory_peak) s->st.memory_peak = s->st.memory_in_use;
                s->st.active += 1;
                s->st.queued -= 1;
                s->queue.pop_front();
            }
            // round: share the tile budget among requests with tiles left, oldest first
            uint64_t n_want = 0;
            for (uint64_t sl : s->order)
                if (s->slots[sl].next_tile < s->slots[sl].tiles) ++n_want;
            if (n_want) {
                const uint64_t quota = std::max<uint64_t>(1, (budget + n_want - 1) / n_want);
                uint64_t left = budget;
                for (uint64_t sl : s->order) {
                    heston_server::Req &r = s->slots[sl];
                    if (r.next_tile >= r.tiles || left == 0) continue;
                    const uint64_t take = std::min(std::min(r.tiles - r.next_tile, quota), left);
                    round_slots.push_back((int)sl);
                    round_tiles.push_back(take);
                    left -= take;
                }
                // most steps first, so that short tiles fill the end of the round
                std::vector<size_t> idx(round_slots.size());
                for (size_t i = 0; i < idx.size(); ++i) idx[i] = i;
                std::stable_sort(idx.begin(), idx.end(), [&](size_t x, size_t y) {
                    return s->slots[round_slots[x]].dev.N > s->slots[round_slots[y]].dev.N;
                });
                std::vector<int> rs(idx.size());
                std::vector<uint64_t> rt(idx.size());
                for (size_t i = 0; i < idx.size(); ++i) { rs[i] = round_slots[idx[i]]; rt[i] = round_tiles[idx[i]]; }
                round_slots.swap(rs);
                round_tiles.swap(rt);
            }
            const bool busy = !round_slots.empty() || !s->pending[0].empty() || !s->pending[1].empty();
            if (!busy) {
                if (s->stop && s->queue.empty() && s->order.empty()) break;
                s->cv_work.wait_for(lock, std::chrono::milliseconds(2));
                continue;
            }
        }
        if (!round_slots.empty()) {
            // buffer b was last used two rounds ago: wait for that round, retire it
            srv_retire(s, b);
            cudaEventSynchronize(s->ev[b]);
            cudaStream_t st = s->strm[b];
            const uint32_t n = (uint32_t)round_slots.size();
            uint64_t acc = 0;
            for (uint32_t p = 0; p < n; ++p) {
                heston_server::Req &r = s->slots[round_slots[p]];
                r.next_tile += round_tiles[p];
                if (r.next_tile == r.tiles) finishing.push_back(round_slots[p]);
            }
            const uint32_t nf = (uint32_t)finishing.size();
            const RoundLayout L = round_layout(n, nf);
            char *hp = s->h_pack[b], *dp = s->d_pack[b];
            *(uint64_t *)hp = 0;
            uint64_t *hwb = (uint64_t *)(hp + L.wb), *hwt = (uint64_t *)(hp + L.wt);
            uint32_t *hwi = (uint32_t *)(hp + L.wi);
            for (uint32_t p = 0; p < n; ++p) {
                const heston_server::Req &r = s->slots[round_slots[p]];
                hwb[p] = acc;
                hwt[p] = r.next_tile - round_tiles[p];
                hwi[p] = (uint32_t)round_slots[p];
                acc += round_tiles[p];
            }
            uint64_t gacc = 0;
            uint64_t *hfg = (uint64_t *)(hp + L.fg);
            uint32_t *hfs = (uint32_t *)(hp + L.fs);
            for (uint32_t p = 0; p < nf; ++p) {
                hfs[p] = (uint32_t)finishing[p];
                hfg[p] = gacc;
                gacc += groups_for(s->slots[finishing[p]].tiles);
            }
            cudaMemcpyAsync(dp, hp, L.total, cudaMemcpyHostToDevice, st);
            // descriptors admitted for the previous round were copied on the other stream
            cudaStreamWaitEvent(st, s->ev_copy[1 - b], 0);
            cudaEventRecord(s->ev_copy[b], st);
            BatchLaunch a;
            a.items = s->d_slots;
            a.work_begin = (const uint64_t *)(dp + L.wb);
            a.work_item = (const uint32_t *)(dp + L.wi);
            a.work_tile0 = (const uint64_t *)(dp + L.wt);
            a.group_begin = nullptr;
            a.n_items = n;
            a.total_work = acc;
            a.counter = (unsigned long long *)dp;
            a.status = nullptr;
            a.rows = s->d_pool;
            const uint64_t grid = std::min<uint64_t>((acc + 3) / 4, (uint64_t)s->n_sm * s->per_sm);
            if (s->cfg.trunc == HESTON_TRUNC_FULL)
                heston_batch_kernel<0><<<(unsigned)std::max<uint64_t>(grid, 1), kPathBlock, 0, st>>>(a);
            else
                heston_batch_kernel<1><<<(unsigned)std::max<uint64_t>(grid, 1), kPathBlock, 0, st>>>(a);
            cudaEventRecord(s->ev_kern[b], st);
            // the requests that finished: one reduction launch per level for all of them,
            // after the previous round's tiles (other stream) too
            if (nf) {
                cudaStreamWaitEvent(st, s->ev_kern[1 - b], 0);
                server_reduce_groups_kernel<<<(unsigned)gacc, kOneContractSumThreads, 0, st>>>(
                    s->d_slots, (const uint32_t *)(dp + L.fs), (const uint64_t *)(dp + L.fg), nf, s->d_pool,
                    s->d_groups[b]);
                server_reduce_final_kernel<<<nf, kOneContractSumThreads, 0, st>>>(s->d_slots, (const uint32_t *)(dp + L.fs),
                                                              (const uint64_t *)(dp + L.fg), s->d_groups[b],
                                                              s->d_res[b]);
                cudaMemcpyAsync(s->h_res[b], s->d_res[b], (size_t)nf * 12u * sizeof(double),
                                cudaMemcpyDeviceToHost, st);
            }
            cudaEventRecord(s->ev[b], st);
            {
                std::lock_guard<std::mutex> lock(s->mu);
                s->pending[b] = finishing;
                s->st.rounds += 1;
                s->st.tiles_done += acc;
            }
            // retire the previous round while this one runs
            srv_retire(s, 1 - b);
            b = 1 - b;
        } else {
            srv_retire(s, b);
            srv_retire(s, 1 - b);
        }
    }
}

void srv_free_buffers(heston_server *s)
{
    cudaFree(s->d_slots); cudaFree(s->d_pool);
    for (int b = 0; b < 2; ++b) {
        cudaFree(s->d_groups[b]); cudaFree(s->d_pack[b]); cudaFree(s->d_res[b]);
        cudaFreeHost(s->h_pack[b]); cudaFreeHost(s->h_res[b]);
        if (s->ev[b]) cudaEventDestroy(s->ev[b]);
        if (s->ev_copy[b]) cudaEventDestroy(s->ev_copy[b]);
        if (s->ev_kern[b]) cudaEventDestroy(s->ev_kern[b]);
        if (s->strm[b]) cudaStreamDestroy(s->strm[b]);
    }
    cudaFreeHost(s->h_slots);
}

}  // namespace

// Static device scratch of heston_mc_launch_noalloc (see include/heston_mc.h):
// one array per device that loads the library, shared by every call on it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[HESTON_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kNoallocMaxDevices];   // device address of g_noalloc_scratch, per device

// Device address of the scratch array on the current device, looked up once.
int noalloc_scratch(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HESTON_ERR_CUDA;
    if (dev < 0 || dev >= kNoallocMaxDevices) return HESTON_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return HESTON_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return HESTON_OK;
}
}  // namespace

namespace {
// Synchronous randomised-QMC estimate: tables, workspace and output are
// allocated stream-ordered for this call and freed before it returns.
int qmc_price_sync(const Prepared &pp, uint64_t n_paths, uint64_t seed, heston_result *out)
{
    int rc = validate_qmc(n_paths, pp.N, pp);
    if (rc < 0) return rc;
    BridgePlanHost plan;
    if (!plan_bridge(pp.N, plan)) return HESTON_ERR_UNSUPPORTED;
    DeviceGuard g(pp.opt.device);
    if (g.err != cudaSuccess) return HESTON_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)pp.opt.cuda_stream;
    const size_t tb = qmc_layout(pp.N, plan.ev.size()).total;
    const size_t wb = qmc_ws_layout(pp.cs.n, n_paths, pp.N, pp.opt.n_shifts).total;
    const size_t ob = 12u * pp.cs.n * sizeof(double);
    char *buf = nullptr;
    if (scratch_alloc((void **)&buf, tb + wb + align256(ob), st) != cudaSuccess) {
        cudaGetLastError();
        return HESTON_ERR_NOMEM;
    }
    int e = cudaStreamSynchronize(st) == cudaSuccess ? HESTON_OK : HESTON_ERR_CUDA;
    if (e == HESTON_OK) e = build_qmc_tables(pp.N, buf, tb);
    double *d_out = (double *)(buf + tb + wb);
    double h[12 * kMaxC];
    if (e == HESTON_OK) e = enqueue_qmc(pp, n_paths, seed, buf, buf + tb, wb, d_out, st);
    if (e == HESTON_OK && cudaMemcpyAsync(h, d_out, ob, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        e = HESTON_ERR_CUDA;
    cudaFreeAsync(buf, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) e = HESTON_ERR_CUDA;
    if (e < 0) return e;
    const int status = pp.gamma_nan ? HESTON_WARN_GAMMA_UNDEFINED : HESTON_OK;
    return fill_results(h, (uint32_t)pp.cs.n, n_paths, status, out);
}
}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char *heston_status_string(int status)
{
    switch (status) {
    case HESTON_OK: return "ok";
    case HESTON_WARN_GAMMA_UNDEFINED: return "gamma undefined (|rho| == 1 or v0 == 0); set to NaN";
    case HESTON_WARN_TANGENT_UNSTABLE: return "vega / theta not finite: pathwise tangents unstable near V = 0";
    case HESTON_ERR_INVALID_ARG: return "invalid argument";
    case HESTON_ERR_CUDA: return "CUDA runtime error";
    case HESTON_ERR_NOMEM: return "device allocation failed";
    case HESTON_ERR_TIMEOUT: return "device wait timed out";
    case HESTON_ERR_CANCELLED: return "cancelled";
    case HESTON_ERR_UNSUPPORTED: return "option combination not supported";
    case HESTON_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    default: return "unknown status";
    }
}

int heston_mc_workspace_bytes(uint32_t n_contracts, uint64_t n_paths, size_t *bytes)
{
    if (!bytes || n_contracts == 0 || n_contracts > (uint32_t)kMaxC || n_paths < 1 ||
        n_paths > (1ull << 40))
        return HESTON_ERR_INVALID_ARG;
    *bytes = workspace_bytes(n_contracts, n_paths);
    return HESTON_OK;
}

int heston_mc_launch(const heston_params *params, const heston_contract *contracts,
                     uint32_t n_contracts, uint64_t n_paths, uint32_t n_steps, uint64_t rng_seed,
                     const heston_options *opts, void *d_workspace, size_t workspace_bytes_,
                     double *d_out)
{
    Prepared pp;
    int rc = validate_and_prepare(params, contracts, n_contracts, n_paths, n_steps, opts, pp);
    if (rc < 0) return rc;
    if (pp.opt.rng != HESTON_RNG_PHILOX) return HESTON_ERR_UNSUPPORTED;
    DeviceGuard g(pp.opt.device);
    if (g.err != cudaSuccess) return HESTON_ERR_CUDA;
    const int e = enqueue(pp, n_paths, rng_seed, d_workspace, workspace_bytes_, d_out,
                          (cudaStream_t)pp.opt.cuda_stream);
    if (e < 0) return e;
    return pp.gamma_nan ? HESTON_WARN_GAMMA_UNDEFINED : HESTON_OK;
}

int heston_mc_launch_noalloc(const heston_params *params, const heston_contract *contracts,
                             uint32_t n_contracts, uint64_t n_paths, uint32_t n_steps,
                             uint64_t rng_seed, const heston_options *opts, double *d_out)
{
    Prepared pp;
    int rc = validate_and_prepare(params, contracts, n_contracts, n_paths, n_steps, opts, pp);
    if (rc < 0) return rc;
    if (pp.opt.rng != HESTON_RNG_PHILOX) return HESTON_ERR_UNSUPPORTED;
    if (!d_out) return HESTON_ERR_INVALID_ARG;
    if (workspace_bytes(n_contracts, n_paths) > (size_t)HESTON_NOALLOC_SCRATCH_BYTES)
        return HESTON_ERR_WORKSPACE;
    DeviceGuard g(pp.opt.device);
    if (g.err != cudaSuccess) return HESTON_ERR_CUDA;
    void *scratch = nullptr;
    rc = noalloc_scratch(&scratch);
    if (rc < 0) return rc;
    const int e = enqueue(pp, n_paths, rng_seed, scratch, HESTON_NOALLOC_SCRATCH_BYTES, d_out,
                          (cudaStream_t)pp.opt.cuda_stream);
    if (e < 0) return e;
    return pp.gamma_nan ? HESTON_WARN_GAMMA_UNDEFINED : HESTON_OK;
}

int heston_mc_price_greeks_ex(const heston_params *params, const heston_contract *contracts,
                              uint32_t n_contracts, uint64_t n_paths, uint32_t n_steps,
                              uint64_t rng_seed, const heston_options *opts, heston_result *out)
{
    if (!out) return HESTON_ERR_INVALID_ARG;
    Prepared pp;
    int rc = validate_and_prepare(params, contracts, n_contracts, n_paths, n_steps, opts, pp);
    if (rc < 0) {
        for (uint32_t c = 0; c < n_contracts && c < (uint32_t)kMaxC; ++c) out[c].status = rc;
        return rc;
    }
    if (pp.opt.rng == HESTON_RNG_SOBOL_BB) {
        rc = qmc_price_sync(pp, n_paths, rng_seed, out);
        if (rc < 0)
            for (uint32_t c = 0; c < n_contracts; ++c) out[c].status = rc;
        return rc;
    }
    DeviceGuard g(pp.opt.device);
    if (g.err != cudaSuccess) return HESTON_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)pp.opt.cuda_stream;
    const size_t ws_bytes = workspace_bytes(n_contracts, n_paths);
    const size_t out_bytes = 12u * n_contracts * sizeof(double);
    void *ws = nullptr;
    if (scratch_alloc(&ws, ws_bytes + align256(out_bytes), st) != cudaSuccess) {
        cudaGetLastError();
        return HESTON_ERR_NOMEM;
    }
    double *d_out = (double *)((char *)ws + ws_bytes);
    double h[12 * kMaxC];
    int e = enqueue(pp, n_paths, rng_seed, ws, ws_bytes, d_out, st);
    if (e == HESTON_OK) {
        if (cudaMemcpyAsync(h, d_out, out_bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            e = HESTON_ERR_CUDA;
    }
    cudaFreeAsync(ws, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) e = HESTON_ERR_CUDA;
    if (e < 0) {
        for (uint32_t c = 0; c < n_contracts; ++c) out[c].status = e;
        return e;
    }
    const int status = pp.gamma_nan ? HESTON_WARN_GAMMA_UNDEFINED : HESTON_OK;
    return fill_results(h, n_contracts, n_paths, status, out);
}

int heston_mc_price_greeks(const heston_params *params, const heston_contract *contract,
                           uint64_t n_paths, uint32_t n_steps, uint64_t rng_seed,
                           heston_result *out)
{
    return heston_mc_price_greeks_ex(params, contract, 1, n_paths, n_steps, rng_seed, nullptr, out);
}

int heston_mc_launch_tiles(const heston_params *params, const heston_contract *contracts,
                           uint32_t n_contracts, uint64_t path_begin, uint64_t n_paths,
                           uint32_t n_steps, uint64_t rng_seed, const heston_options *opts,
                           double *d_tile_sums)
{
    Prepared pp;
    int rc = validate_and_prepare(params, contracts, n_contracts, n_paths < 2 ? 2 : n_paths,
                                  n_steps, opts, pp);
    if (rc < 0) return rc;
    if (pp.opt.rng != HESTON_RNG_PHILOX) return HESTON_ERR_UNSUPPORTED;
    if (n_paths == 0 || !d_tile_sums || (path_begin % kTile) != 0) return HESTON_ERR_INVALID_ARG;
    DeviceGuard g(pp.opt.device);
    if (g.err != cudaSuccess) return HESTON_ERR_CUDA;
    Launch a;
    a.key = key_of(rng_seed);
    a.path_begin = path_begin;
    a.n_paths = n_paths;
    a.n_tiles = tiles_for(n_paths);
    a.N = pp.N;
    a.tile_sums = d_tile_sums;
    if (launch_paths(pp, a, (cudaStream_t)pp.opt.cuda_stream) != cudaSuccess) return HESTON_ERR_CUDA;
    return pp.gamma_nan ? HESTON_WARN_GAMMA_UNDEFINED : HESTON_OK;
}

int heston_mc_reduce_tiles(const double *d_tile_sums, uint64_t n_tiles, uint32_t n_contracts,
                           uint64_t n_paths_total, void *d_workspace, size_t workspace_bytes_,
                           double *d_out, void *stream)
{
    if (!d_tile_sums || !d_out || !d_workspace || n_contracts == 0 ||
        n_contracts > (uint32_t)kMaxC || n_paths_total < 2 || n_tiles != tiles_for(n_paths_total))
        return HESTON_ERR_INVALID_ARG;
    if (((uintptr_t)d_workspace & 255u) || workspace_bytes_ < workspace_bytes(n_contracts, n_paths_total))
        return HESTON_ERR_WORKSPACE;
    const size_t w = 12u * n_contracts * sizeof(double);
    double *group_sums = (double *)((char *)d_workspace + align256(n_tiles * w));
    if (launch_reduce(d_tile_sums, n_tiles, (int)n_contracts, n_paths_total, group_sums, false, d_out,
                      (cudaStream_t)stream) != cudaSuccess)
        return HESTON_ERR_CUDA;
    return HESTON_OK;
}

int heston_mc_debug_paths(const heston_params *params, const heston_contract *contracts,
                          uint32_t n_contracts, uint32_t n_steps, uint64_t rng_seed,
                          const heston_options *opts, const uint64_t *paths, uint32_t count,
                          double *h_records, double *h_estimators)
{
    Prepared pp;
    int rc = validate_and_prepare(params, contracts, n_contracts, 2, n_steps, opts, pp);
    if (rc < 0) return rc;
    if (pp.opt.rng != HESTON_RNG_PHILOX) return HESTON_ERR_UNSUPPORTED;
    if (!paths || count == 0 || !h_records || !h_estimators) return HESTON_ERR_INVALID_ARG;
    DeviceGuard g(pp.opt.device);
    if (g.err != cudaSuccess) return HESTON_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)pp.opt.cuda_stream;
    const size_t pb = sizeof(uint64_t) * count;
    const size_t rb = sizeof(double) * kRecordDoubles * count;
    const size_t eb = sizeof(double) * 6 * n_contracts * (size_t)count;
    char *buf = nullptr;
    if (scratch_alloc((void **)&buf, align256(pb) + align256(rb) + align256(eb), st) != cudaSuccess) {
        cudaGetLastError();
        return HESTON_ERR_NOMEM;
    }
    uint64_t *dp = (uint64_t *)buf;
    double *dr = (double *)(buf + align256(pb));
    double *de = (double *)(buf + align256(pb) + align256(rb));
    int e = HESTON_OK;
    if (cudaMemcpyAsync(dp, paths, pb, cudaMemcpyHostToDevice, st) != cudaSuccess) e = HESTON_ERR_CUDA;
    if (e == HESTON_OK) {
        const unsigned grid = (count + 127) / 128;
        const PhiloxKey key = key_of(rng_seed);
        const int mon = mon_mode(pp.cs);
        const int step = step_of(pp.opt);
#define HESTON_DBG(R, SP, MO, K) heston_debug_kernel<R, SP, MO><<<grid, 128, 0, st>>>(K, cs_of<R>(pp), key, pp.N, dp, count, dr, de)
#define HESTON_DBG_M(R, SP, K) do { if (mon == MON_NONE) HESTON_DBG(R, SP, MON_NONE, K); \
                                    else if (mon == MON_EVERY) HESTON_DBG(R, SP, MON_EVERY, K); \
                                    else HESTON_DBG(R, SP, MON_STRIDE, K); } while (0)
#define HESTON_DBG_S(R, K) do { switch (step) { \
            case STEP_MIL_FULL: HESTON_DBG_M(R, STEP_MIL_FULL, K); break; \
            case STEP_MIL_FLOOR: HESTON_DBG_M(R, STEP_MIL_FLOOR, K); break; \
            case STEP_EUL_FULL: HESTON_DBG_M(R, STEP_EUL_FULL, K); break; \
            case STEP_EUL_FLOOR: HESTON_DBG_M(R, STEP_EUL_FLOOR, K); break; \
            default: HESTON_DBG_M(R, STEP_QE, K); } } while (0)
        if (pp.opt.prec == HESTON_FP32) HESTON_DBG_S(float, pp.kf);
        else HESTON_DBG_S(double, pp.kd);
#undef HESTON_DBG_S
#undef HESTON_DBG_M
#undef HESTON_DBG
        if (cudaGetLastError() != cudaSuccess) e = HESTON_ERR_CUDA;
    }
    if (e == HESTON_OK && (cudaMemcpyAsync(h_records, dr, rb, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                           cudaMemcpyAsync(h_estimators, de, eb, cudaMemcpyDeviceToHost, st) != cudaSuccess))
        e = HESTON_ERR_CUDA;
    cudaFreeAsync(buf, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) e = HESTON_ERR_CUDA;
    if (e < 0) return e;
    return pp.gamma_nan ? HESTON_WARN_GAMMA_UNDEFINED : HESTON_OK;
}

int heston_rng_debug(uint64_t rng_seed, const uint64_t *paths, const uint32_t *steps, uint32_t count,
                     int32_t prec, uint32_t *h_words, double *h_normals)
{
    if (!paths || !steps || !h_words || !h_normals || count == 0) return HESTON_ERR_INVALID_ARG;
    if (prec != HESTON_FP32 && prec != HESTON_FP64) return HESTON_ERR_INVALID_ARG;
    const size_t pb = sizeof(uint64_t) * count, sb = sizeof(uint32_t) * count;
    const size_t wb = 4 * sizeof(uint32_t) * count, nb = 2 * sizeof(double) * count;
    char *buf = nullptr;
    if (cudaMalloc((void **)&buf, align256(pb) + align256(sb) + align256(wb) + align256(nb)) != cudaSuccess) {
        cudaGetLastError();
        return HESTON_ERR_NOMEM;
    }
    uint64_t *dp = (uint64_t *)buf;
    uint32_t *ds = (uint32_t *)(buf + align256(pb));
    uint32_t *dw = (uint32_t *)(buf + align256(pb) + align256(sb));
    double *dn = (double *)(buf + align256(pb) + align256(sb) + align256(wb));
    int e = HESTON_OK;
    if (cudaMemcpy(dp, paths, pb, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ds, steps, sb, cudaMemcpyHostToDevice) != cudaSuccess)
        e = HESTON_ERR_CUDA;
    if (e == HESTON_OK) {
        const unsigned grid = (count + 127) / 128;
        if (prec == HESTON_FP32) rng_debug_kernel<float><<<grid, 128>>>(key_of(rng_seed), dp, ds, count, dw, dn);
        else                     rng_debug_kernel<double><<<grid, 128>>>(key_of(rng_seed), dp, ds, count, dw, dn);
        if (cudaGetLastError() != cudaSuccess) e = HESTON_ERR_CUDA;
    }
    if (e == HESTON_OK && (cudaMemcpy(h_words, dw, wb, cudaMemcpyDeviceToHost) != cudaSuccess ||
                           cudaMemcpy(h_normals, dn, nb, cudaMemcpyDeviceToHost) != cudaSuccess))
        e = HESTON_ERR_CUDA;
    cudaFree(buf);
    return e;
}

int heston_bm64_debug(uint32_t first, uint32_t count, double *h_out)
{
    if (!h_out || count == 0 || (uint64_t)first + count > (1ull << 24)) return HESTON_ERR_INVALID_ARG;
    const size_t bytes = 6 * sizeof(double) * (size_t)count;
    double *d = nullptr;
    if (cudaMalloc((void **)&d, bytes) != cudaSuccess) {
        cudaGetLastError();
        return HESTON_ERR_NOMEM;
    }
    int e = HESTON_OK;
    bm64_debug_kernel<<<(count + 255) / 256, 256>>>(first, count, d);
    if (cudaGetLastError() != cudaSuccess || cudaMemcpy(h_out, d, bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
        e = HESTON_ERR_CUDA;
    cudaFree(d);
    return e;
}

int heston_batch_plan_make(const heston_batch_item *items, uint32_t n_items,
                           const heston_options *opts, heston_batch_plan *plan)
{
    return batch_prepare_items(items, n_items, opts, nullptr, plan);
}

int heston_batch_prepare(const heston_batch_item *items, const heston_options *opts,
                         const heston_batch_plan *plan, void *d_desc)
{
    if (!plan) return HESTON_ERR_INVALID_ARG;
    DeviceGuard g(opts ? opts->device : -1);
    if (g.err != cudaSuccess) return HESTON_ERR_CUDA;
    return batch_prepare(items, opts, plan, d_desc);
}

int heston_mc_launch_batch(const heston_batch_plan *plan, const void *d_desc,
                           const heston_options *opts, void *d_workspace, double *d_out,
                           int32_t *d_status)
{
    return batch_launch(plan, d_desc, opts, d_workspace, d_out, d_status);
}

int heston_mc_price_greeks_batch(const heston_batch_item *items, uint32_t n_items,
                                 const heston_options *opts, heston_result *out)
{
    if (!out) return HESTON_ERR_INVALID_ARG;
    heston_batch_plan plan;
    int rc = batch_prepare_items(items, n_items, opts, nullptr, &plan);
    if (rc < 0) return rc;
    DeviceGuard g(opts ? opts->device : -1);
    if (g.err != cudaSuccess) return HESTON_ERR_CUDA;
    cudaStream_t st = opts ? (cudaStream_t)opts->cuda_stream : nullptr;
    const size_t ob = align256((size_t)n_items * 12u * sizeof(double));
    char *buf = nullptr;
    if (cudaMalloc((void **)&buf, plan.descriptor_bytes + plan.workspace_bytes + ob) != cudaSuccess) {
        cudaGetLastError();
        return HESTON_ERR_NOMEM;
    }
    double *d_out = (double *)(buf + plan.descriptor_bytes + plan.workspace_bytes);
    int e = batch_prepare(items, opts, &plan, buf);
    if (e == HESTON_OK) e = batch_launch(&plan, buf, opts, buf + plan.descriptor_bytes, d_out, nullptr);
    std::vector<double> h((size_t)n_items * 12u);
    if (e == HESTON_OK && cudaMemcpyAsync(h.data(), d_out, h.size() * sizeof(double),
                                          cudaMemcpyDeviceToHost, st) != cudaSuccess)
        e = HESTON_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) e = HESTON_ERR_CUDA;
    cudaFree(buf);
    if (e < 0) return e;
    int worst = HESTON_OK;
    for (uint32_t i = 0; i < n_items; ++i) {
        const bool gn = std::fabs(items[i].params.rho) == 1.0 || items[i].params.v0 == 0.0;
        const int status = fill_results(h.data() + (size_t)i * 12u, 1, items[i].n_paths,
                                        gn ? HESTON_WARN_GAMMA_UNDEFINED : HESTON_OK, out + i);
        if (status > worst) worst = status;
    }
    return worst;
}

int heston_adjoint_workspace_bytes(uint64_t n_paths, uint32_t n_steps, size_t *bytes)
{
    if (!bytes || n_paths < 2 || n_paths > (1ull << 40) || n_steps == 0) return HESTON_ERR_INVALID_ARG;
    if (n_steps > kAdjMaxSteps) return HESTON_ERR_UNSUPPORTED;
    const AdjLayout L = adj_layout(n_paths, n_steps);
    *bytes = L.total;
    return HESTON_OK;
}

int heston_mc_adjoint_forward(const heston_params *params, const heston_contract *contract,
                              uint64_t n_paths, uint32_t n_steps, uint64_t rng_seed,
                              const heston_options *opts, void *d_workspace, size_t workspace_bytes_,
                              double *d_price)
{
    return adjoint_enqueue(false, params, contract, n_paths, n_steps, rng_seed, opts, d_workspace,
                           workspace_bytes_, d_price);
}

int heston_mc_adjoint_backward(const heston_params *params, const heston_contract *contract,
                               uint64_t n_paths, uint32_t n_steps, uint64_t rng_seed,
                               const heston_options *opts, void *d_workspace, size_t workspace_bytes_,
                               double *d_grad)
{
    return adjoint_enqueue(true, params, contract, n_paths, n_steps, rng_seed, opts, d_workspace,
                           workspace_bytes_, d_grad);
}

int heston_mc_adjoint_debug_paths(const heston_params *params, const heston_contract *contract,
                                  uint64_t n_paths, uint32_t n_steps, uint64_t rng_seed,
                                  const heston_options *opts, void *d_workspace, size_t workspace_bytes_,
                                  double *d_per_path)
{
    if (!d_per_path) return HESTON_ERR_INVALID_ARG;
    Prepared pp;
    int rc = validate_and_prepare(params, contract, 1, n_paths, n_steps, opts, pp);
    if (rc < 0) return rc;
    // price (2 doubles) and gradient (14) past the workspace proper: at most 255
    // bytes of alignment + 256 + 112 <= 768
    if (!d_workspace || workspace_bytes_ < adj_layout(n_paths, n_steps).total + 768u)
        return HESTON_ERR_WORKSPACE;
    // the estimates go to the end of the workspace; only the per-path values are returned
    char *tail = (char *)d_workspace + adj_layout(n_paths, n_steps).total;
    double *d_price = (double *)(((uintptr_t)tail + 255u) & ~(uintptr_t)255u);
    double *d_grad = d_price + 32;
    const size_t ws = adj_layout(n_paths, n_steps).total;
    rc = adjoint_enqueue(false, params, contract, n_paths, n_steps, rng_seed, opts, d_workspace, ws, d_price);
    if (rc < 0) return rc;
    return adjoint_enqueue(true, params, contract, n_paths, n_steps, rng_seed, opts, d_workspace, ws, d_grad,
                           d_per_path);
}

int heston_release_cached_memory(int32_t device)
{
    int lo = device, hi = device + 1;
    if (device < 0) { lo = 0; hi = kMaxPoolDevices; }
    if (hi > kMaxPoolDevices) return HESTON_ERR_INVALID_ARG;
    for (int d = lo; d < hi; ++d) {
        cudaMemPool_t pool = scratch_pool(d, false);
        if (pool && cudaMemPoolTrimTo(pool, 0) != cudaSuccess) {
            cudaGetLastError();
            return HESTON_ERR_CUDA;
        }
    }
    return HESTON_OK;
}

int heston_server_create(const heston_server_config *cfg, heston_server **out)
{
    if (!cfg || !out || cfg->reserved != 0 || cfg->memory_bytes < 4096) return HESTON_ERR_INVALID_ARG;
    if (cfg->trunc != HESTON_TRUNC_FULL && cfg->trunc != HESTON_TRUNC_PAPER_FLOOR) return HESTON_ERR_INVALID_ARG;
    heston_server *s = new heston_server();
    s->cfg = *cfg;
    if (!s->cfg.max_active) s->cfg.max_active = 1024;
    if (!s->cfg.tiles_per_round) s->cfg.tiles_per_round = 65536;
    const uint32_t S = s->cfg.max_active;
    int e = 0;
    if (cfg->device >= 0) e |= (int)cudaSetDevice(cfg->device);
    e |= (int)cudaGetDevice(&s->device);
    e |= (int)cudaDeviceGetAttribute(&s->n_sm, cudaDevAttrMultiProcessorCount, s->device);
    e |= (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(&s->per_sm, heston_batch_kernel<0>, kPathBlock, 0);
    if (s->per_sm < 1) s->per_sm = 1;
    s->pool_bytes = cfg->memory_bytes / kPoolUnit * kPoolUnit;
    e |= (int)cudaMalloc((void **)&s->d_slots, S * sizeof(BatchItemDev));
    e |= (int)cudaMalloc((void **)&s->d_pool, s->pool_bytes);
    e |= (int)cudaHostAlloc((void **)&s->h_slots, S * sizeof(BatchItemDev), cudaHostAllocDefault);
    // group rows of one round's finishing requests: at most one partial group each beyond
    // the whole groups of the pool
    const size_t group_bytes = ((size_t)groups_for(s->pool_bytes / 96 + 1) + S) * 12 * sizeof(double);
    const size_t pack_bytes = round_layout(S, S).total;
    for (int b = 0; b < 2; ++b) {
        e |= (int)cudaStreamCreateWithFlags(&s->strm[b], cudaStreamNonBlocking);
        e |= (int)cudaMalloc((void **)&s->d_groups[b], group_bytes);
        e |= (int)cudaMalloc((void **)&s->d_pack[b], pack_bytes);
        e |= (int)cudaMalloc((void **)&s->d_res[b], (size_t)S * 12 * sizeof(double));
        e |= (int)cudaHostAlloc((void **)&s->h_pack[b], pack_bytes, cudaHostAllocDefault);
        e |= (int)cudaHostAlloc((void **)&s->h_res[b], (size_t)S * 12 * sizeof(double), cudaHostAllocDefault);
        e |= (int)cudaEventCreateWithFlags(&s->ev[b], cudaEventDisableTiming);
        e |= (int)cudaEventCreateWithFlags(&s->ev_copy[b], cudaEventDisableTiming);
        e |= (int)cudaEventCreateWithFlags(&s->ev_kern[b], cudaEventDisableTiming);
    }
    for (int b = 0; b < 2 && e == 0; ++b) {
        cudaEventRecord(s->ev[b], s->strm[b]);
        cudaEventRecord(s->ev_copy[b], s->strm[b]);
        cudaEventRecord(s->ev_kern[b], s->strm[b]);
    }
    if (e != 0) {
        cudaGetLastError();
        srv_free_buffers(s);
        delete s;
        return HESTON_ERR_NOMEM;
    }
    s->slots.resize(S);
    for (int i = (int)S - 1; i >= 0; --i) s->free_slots.push_back(i);
    s->free_blocks[0] = s->pool_bytes;
    s->th = std::thread(srv_loop, s);
    *out = s;
    return HESTON_OK;
}

int heston_server_submit(heston_server *s, const heston_batch_item *item, uint64_t *ticket)
{
    if (!s || !item || !ticket) return HESTON_ERR_INVALID_ARG;
    heston_options o;
    std::memset(&o, 0, sizeof(o));
    o.prec = HESTON_FP32;
    o.trunc = s->cfg.trunc;
    o.device = -1;
    std::vector<BatchItemDev> dev;
    heston_batch_plan plan;
    const int rc = batch_prepare_items(item, 1, &o, &dev, &plan);
    if (rc < 0) return rc;
    heston_server::Req r;
    r.dev = dev[0];
    r.tiles = dev[0].n_tiles;
    r.bytes = srv_req_bytes(r.tiles);
    if (r.bytes > s->pool_bytes) return HESTON_ERR_NOMEM;
    r.t_submit = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stop) return HESTON_ERR_CANCELLED;
        r.ticket = s->next_ticket++;
        *ticket = r.ticket;
        s->queue.push_back(r);
        s->st.submitted += 1;
        s->st.queued += 1;
    }
    s->cv_work.notify_one();
    return HESTON_OK;
}

int heston_server_wait(heston_server *s, uint64_t ticket, uint32_t timeout_ms, heston_result *out,
                       double *latency_s)
{
    if (!s || !out) return HESTON_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lock(s->mu);
    if (ticket == 0 || ticket >= s->next_ticket) return HESTON_ERR_INVALID_ARG;
    const bool ok = s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms),
                                        [&] { return s->done.count(ticket) > 0; });
    if (!ok) return 0;
    auto it = s->done.find(ticket);
    *out = it->second.res;
    if (latency_s) *latency_s = it->second.latency;
    s->done.erase(it);
    return 1;
}

int heston_server_poll(heston_server *s, uint64_t ticket, heston_result *out, double *latency_s)
{
    return heston_server_wait(s, ticket, 0, out, latency_s);
}

int heston_server_stats_get(heston_server *s, heston_server_stats *out)
{
    if (!s || !out) return HESTON_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    *out = s->st;
    return HESTON_OK;
}

int heston_server_destroy(heston_server *s)
{
    if (!s) return HESTON_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->th.joinable()) s->th.join();
    cudaStreamSynchronize(s->strm[0]);
    cudaStreamSynchronize(s->strm[1]);
    srv_free_buffers(s);
    delete s;
    return HESTON_OK;
}

int heston_sobol_directions(uint32_t n_dims, uint32_t *h_out)
{
    if (!h_out || n_dims == 0 || n_dims > 2 * kQmcMaxSteps) return HESTON_ERR_INVALID_ARG;
    sobol_directions_host(n_dims, h_out);
    return HESTON_OK;
}

int heston_qmc_tables_bytes(uint32_t n_steps, size_t *bytes)
{
    if (!bytes || n_steps == 0) return HESTON_ERR_INVALID_ARG;
    BridgePlanHost plan;
    if (!plan_bridge(n_steps, plan)) return HESTON_ERR_UNSUPPORTED;
    *bytes = qmc_layout(n_steps, plan.ev.size()).total;
    return HESTON_OK;
}

int heston_qmc_build_tables(uint32_t n_steps, void *d_tables, size_t bytes, int32_t device)
{
    if (n_steps == 0) return HESTON_ERR_INVALID_ARG;
    DeviceGuard g(device);
    if (g.err != cudaSuccess) return HESTON_ERR_CUDA;
    return build_qmc_tables(n_steps, d_tables, bytes);
}

int heston_mc_workspace_bytes_qmc(uint32_t n_contracts, uint64_t n_paths, uint32_t n_steps,
                                  uint32_t n_shifts, size_t *bytes)
{
    if (!bytes || n_contracts == 0 || n_contracts > (uint32_t)kMaxC || n_steps == 0 ||
        n_steps > kQmcMaxSteps || n_shifts < 2 || n_paths % n_shifts ||
        (n_paths / n_shifts) % kTile || n_paths / n_shifts > (1ull << 32))
        return HESTON_ERR_INVALID_ARG;
    *bytes = qmc_ws_layout(n_contracts, n_paths, n_steps, n_shifts).total;
    return HESTON_OK;
}

int heston_mc_launch_qmc(const heston_params *params, const heston_contract *contracts,
                         uint32_t n_contracts, uint64_t n_paths, uint32_t n_steps, uint64_t rng_seed,
                         const heston_options *opts, const void *d_tables, void *d_workspace,
                         size_t workspace_bytes_, double *d_out)
{
    Prepared pp;
    int rc = validate_and_prepare(params, contracts, n_contracts, n_paths, n_steps, opts, pp);
    if (rc < 0) return rc;
    if (pp.opt.rng != HESTON_RNG_SOBOL_BB) return HESTON_ERR_INVALID_ARG;
    rc = validate_qmc(n_paths, n_steps, pp);
    if (rc < 0) return rc;
    DeviceGuard g(pp.opt.device);
    if (g.err != cudaSuccess) return HESTON_ERR_CUDA;
    const int e = enqueue_qmc(pp, n_paths, rng_seed, d_tables, d_workspace, workspace_bytes_, d_out,
                              (cudaStream_t)pp.opt.cuda_stream);
    if (e < 0) return e;
    return pp.gamma_nan ? HESTON_WARN_GAMMA_UNDEFINED : HESTON_OK;
}

int heston_qmc_debug_paths(const heston_params *params, const heston_contract *contracts,
                           uint32_t n_contracts, uint32_t n_steps, uint64_t rng_seed,
                           const heston_options *opts, uint32_t replicate, const uint32_t *points,
                           uint32_t count, double *h_records, double *h_estimators)
{
    Prepared pp;
    int rc = validate_and_prepare(params, contracts, n_contracts, 2, n_steps, opts, pp);
    if (rc < 0) return rc;
    if (pp.opt.rng != HESTON_RNG_SOBOL_BB || !points || count == 0 || !h_records || !h_estimators ||
        replicate >= (1u << 16))
        return HESTON_ERR_INVALID_ARG;
    if (pp.opt.prec != HESTON_FP32 || n_steps > kQmcMaxSteps) return HESTON_ERR_UNSUPPORTED;
    BridgePlanHost plan;
    if (!plan_bridge(n_steps, plan)) return HESTON_ERR_UNSUPPORTED;
    DeviceGuard g(pp.opt.device);
    if (g.err != cudaSuccess) return HESTON_ERR_CUDA;
    const uint32_t D = 2u * n_steps;
    const QmcLayout TL = qmc_layout(n_steps, plan.ev.size());
    const size_t pb = align256(sizeof(uint32_t) * count);
    const size_t ub = align256(sizeof(uint32_t) * (size_t)count * D);
    const size_t sb = align256(sizeof(uint32_t) * (size_t)(replicate + 1) * D);
    const size_t rb = align256(sizeof(double) * kRecordDoubles * count);
    const size_t eb = align256(sizeof(double) * 6 * n_contracts * (size_t)count);
    char *buf = nullptr;
    if (cudaMalloc((void **)&buf, TL.total + pb + ub + sb + rb + eb) != cudaSuccess) {
        cudaGetLastError();
        return HESTON_ERR_NOMEM;
    }
    char *p = buf + TL.total;
    uint32_t *dp = (uint32_t *)p;         p += pb;
    uint32_t *dU = (uint32_t *)p;         p += ub;
    uint32_t *dS = (uint32_t *)p;         p += sb;
    double *dr = (double *)p;             p += rb;
    double *de = (double *)p;
    int e = build_qmc_tables(n_steps, buf, TL.total);
    if (e == HESTON_OK && cudaMemcpy(dp, points, sizeof(uint32_t) * count, cudaMemcpyHostToDevice) != cudaSuccess)
        e = HESTON_ERR_CUDA;
    if (e == HESTON_OK) {
        const QmcTables tb = qmc_tables_at(buf, TL);
        const uint64_t nu = (uint64_t)count * D;
        qmc_debug_high_bits_kernel<<<(unsigned)((nu + 255) / 256), 256>>>(tb.V, D, dp, count, dU);
        const uint64_t ns = (uint64_t)(replicate + 1) * D;
        qmc_setup_kernel<<<(unsigned)((ns + 255) / 256), 256>>>(tb.V, D, 0, replicate + 1,
                                                                 key_of(rng_seed), nullptr, dS);
        const uint32_t *srow = dS + (uint64_t)replicate * D;
        const unsigned grid = (count + 127) / 128;
        const int mon = mon_mode(pp.cs);
        const bool full = pp.opt.trunc == HESTON_TRUNC_FULL;
#define HESTON_QDBG(TR, MO) heston_qmc_debug_kernel<TR, MO><<<grid, 128>>>(pp.kf, pp.csf, tb, n_steps, dp, dU, srow, count, dr, de)
        if (full) { if (mon == MON_NONE) HESTON_QDBG(0, MON_NONE); else if (mon == MON_EVERY) HESTON_QDBG(0, MON_EVERY); else HESTON_QDBG(0, MON_STRIDE); }
        else      { if (mon == MON_NONE) HESTON_QDBG(1, MON_NONE); else if (mon == MON_EVERY) HESTON_QDBG(1, MON_EVERY); else HESTON_QDBG(1, MON_STRIDE); }
#undef HESTON_QDBG
        if (cudaGetLastError() != cudaSuccess) e = HESTON_ERR_CUDA;
    }
    if (e == HESTON_OK &&
        (cudaMemcpy(h_records, dr, sizeof(double) * kRecordDoubles * count, cudaMemcpyDeviceToHost) != cudaSuccess ||
         cudaMemcpy(h_estimators, de, sizeof(double) * 6 * n_contracts * (size_t)count, cudaMemcpyDeviceToHost) != cudaSuccess))
        e = HESTON_ERR_CUDA;
    cudaFree(buf);
    if (e < 0) return e;
    return pp.gamma_nan ? HESTON_WARN_GAMMA_UNDEFINED : HESTON_OK;
}

}  // extern "C"
