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
// Asian sums); a warp owns 64-path tiles and reduces each tile's estimators
// with shuffles; tile rows go to a workspace and two fixed-order kernels
// reduce them in FP64.  No per-path or per-step data touches memory.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "heston_mc.h"

namespace {

constexpr int kTile = HESTON_TILE_PATHS;   // paths per tile = 32 lanes x 2
constexpr int kMaxC = HESTON_MAX_CONTRACTS;
constexpr int kGroupTiles = 256;           // tiles per first-level reduction group
constexpr int kRecordDoubles = 15;
constexpr int kPathBlock = 128;            // default threads per path-kernel CTA

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies, the high halves xored with the other two words and
// the round key; the key advances by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
struct PhiloxKey {
    uint32_t k0, k1;
};

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, PhiloxKey key)
{
    uint32_t k0 = key.k0, k1 = key.k1;
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const unsigned long long p0 = (unsigned long long)c.x * 0xD2511F53u;
        const unsigned long long p1 = (unsigned long long)c.z * 0xCD9E8D57u;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// ---------------------------------------------------------------------------
// Box-Muller on 24-bit uniforms: u1 = (a>>8 + 1) 2^-24 in (0,1],
// u2 = (b>>8) 2^-24 in [0,1); Za = sqrt(-2 ln u1) cos 2 pi u2,
// Zb = sqrt(-2 ln u1) sin 2 pi u2.  The uniforms are exact in both precisions.
// ---------------------------------------------------------------------------
// FP32 special-function unit approximations (PTX .approx forms).  Documented
// bounds: sin/cos absolute error about 2^-20.9 on [-pi, pi]; lg2 absolute
// error about 2^-22; ex2, rsqrt, sqrt relative error about 2^-22.
__device__ __forceinline__ float sin_approx(float x) { float y; asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float cos_approx(float x) { float y; asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float ex2_approx(float x) { float y; asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float sqrt_approx(float x) { float y; asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float lg2_approx(float x) { float y; asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float rsqrt_approx(float x) { float y; asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }

__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float &za, float &zb)
{
    // u1 = (a>>8) 2^-24 + 2^-24: the top 24 bits convert exactly.
    const float u1 = fmaf((float)(a & 0xFFFFFF00u), 2.3283064365386963e-10f, 5.9604644775390625e-8f);
    // The top 24 bits of b read as a signed 32-bit integer are 2^32 (u2 - [u2 >= 1/2]),
    // so the angle 2 pi u2 lands in [-pi, pi) with the same sine and cosine.
    const float ang = (float)(int32_t)(b & 0xFFFFFF00u) * 1.4629180792671596e-9f;   // 2 pi / 2^32
    // r2 = -2 ln u1.  For u1 <= 0.9 from lg2.approx, whose absolute error
    // (2 ln2 2^-22 in r2) is below 1.6e-6 of r2 >= 0.21.  Near 1, where that
    // absolute error would swamp the small radius, from the series
    // -2 ln(1 - w) = 2 sum_k w^k / k in w = 1 - u1 (exact), truncated after
    // w^7 (relative error < 1.4e-8 at w = 0.1).  Both are evaluated and one
    // selected: lanes of a warp fall on both sides.
    const float w = 1.0f - u1;
    const float r2_far = -1.3862943611198906f * lg2_approx(u1);
    float p = fmaf(w, 0.2857142857f, 0.3333333333f);
    p = fmaf(w, p, 0.4f);
    p = fmaf(w, p, 0.5f);
    p = fmaf(w, p, 0.6666666667f);
    p = fmaf(w, p, 1.0f);
    p = fmaf(w, p, 2.0f);
    const float r2 = u1 > 0.9f ? w * p : r2_far;
    const float rad = sqrt_approx(r2);
    za = rad * cos_approx(ang);
    zb = rad * sin_approx(ang);
}

__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, double &za, double &zb)
{
    const double u1 = (double)((a >> 8) + 1u) * 5.9604644775390625e-8;
    const double u2 = (double)(b >> 8) * 5.9604644775390625e-8;
    const double rad = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    za = rad * c;
    zb = rad * s;
}

__device__ __forceinline__ float rsqrt_pos(float y) { return y > 0.0f ? rsqrt_approx(y) : 0.0f; }
__device__ __forceinline__ double rsqrt_pos(double y) { return y > 0.0 ? rsqrt(y) : 0.0; }
__device__ __forceinline__ float exp_r(float x) { return ex2_approx(x * 1.44269504f); }
__device__ __forceinline__ double exp_r(double x) { return exp(x); }

// ---------------------------------------------------------------------------
// Scheme coefficients, computed in FP64 on the host and rounded once.
// ---------------------------------------------------------------------------
template <typename R>
struct Coef {
    R v0;
    R dt, ddt, half_dt, r;        // dt = T/N, ddt = d(dt)/dT = 1/N
    R kdt, kth_dt, kth_ddt, kappa_ddt;
    R xi, c4, c4T;                // c4 = xi^2 dt / 4, c4T = xi^2 / (4N)
    R rho, sq;                    // sq = sqrt(1 - rho^2)
};

// Contracts priced on the shared paths (all with the same T and Asian M),
// with their constants rounded once on the host to the path precision.
template <typename R>
struct ContractSet {
    int32_t n;
    int32_t has_asian;
    uint32_t M, stride;           // Asian dates and steps between them
    int32_t payoff[kMaxC];
    int32_t is_put[kMaxC];
    R K[kMaxC];
    R T, D, r;                    // D = exp(-rT)
    R S0, inv_S0, inv_S0sq;
    R inv_sq;                     // 1 / sqrt(1 - rho^2)
    R S0_over_M;                  // S0 / M
    R dAr_scale;                  // S0 T / M^2: d Sbar / dr = dAr_scale ((M+1) sA - sC)
    R Mp1;                        // M + 1
};

struct Launch {
    PhiloxKey key;
    uint64_t path_begin;          // global index of local path 0
    uint64_t n_paths;             // local paths
    uint64_t n_tiles;
    uint32_t N;
    double *tile_sums;            // [n_tiles][12 * n]
};

// Registers of one path.  X = ln(S/S0); *_v = d/dv0, *_T = d/dT tangents.
// Over the dates i = 1..M: sA = sum_i e^{X(t_i)} (running), sC = sum of the
// running sA after each date, so that sum_i i e^{X(t_i)} = (M+1) sA - sC;
// sAv / sAT = sum_i e^{X(t_i)} X_v(t_i) / X_T(t_i).  GE/QE: Gamma weights
// sum_k u_k W_k and sum_k V_k+ dt over all steps; GA/QA: the same over the
// steps before the first monitoring date.
template <typename R>
struct PathState {
    R X, V, Xv, Vv, XT, VT;
    R sA, sC, sAv, sAT;
    R GE, QE, GA, QA;
};

template <typename R>
__device__ __forceinline__ void init_state(PathState<R> &s, R v0)
{
    s.X = R(0); s.V = v0; s.Xv = R(0); s.Vv = R(1); s.XT = R(0); s.VT = R(0);
    s.sA = R(0); s.sC = R(0); s.sAv = R(0); s.sAT = R(0);
    s.GE = R(0); s.QE = R(0); s.GA = R(0); s.QA = R(0);
}

// One Milstein step with its tangents, from independent normals (za, zb).
// FP32 full truncation: the same recursion with shared products hoisted
// (xi Z2 feeds V and both V tangents; the truncation mask scales 1/(2u)).
__device__ __forceinline__ void milstein_step_f32_full(PathState<float> &s, float za, float zb,
                                                       const Coef<float> &k)
{
    const float Z2 = fmaf(k.rho, za, k.sq * zb);
    const float W = fmaf(k.sq, za, -k.rho * zb);
    const float xZ2 = k.xi * Z2;
    const bool pos = s.V > 0.0f;
    const float Vp = fmaxf(s.V, 0.0f);
    const float Vpv = pos ? s.Vv : 0.0f;
    const float VpT = pos ? s.VT : 0.0f;
    const float y = Vp * k.dt;                                  // V+ dt
    const float rs = rsqrt_approx(fmaxf(y, 1e-30f));            // finite at y = 0
    const float u = y * rs;                                     // sqrt(V+ dt), 0 at 0
    const float hdt = 0.5f * k.dt * rs;                         // dt / (2u)
    const float uv = Vpv * hdt;                                 // du/dv0
    const float uT = fmaf(VpT, hdt, Vp * (0.5f * k.ddt * rs));  // du/dT
    s.GE = fmaf(u, W, s.GE);
    s.QE += y;
    const float drift = fmaf(-0.5f, Vp, k.r);
    s.X = fmaf(u, za, fmaf(drift, k.dt, s.X));
    s.Xv = fmaf(uv, za, fmaf(-k.half_dt, Vpv, s.Xv));
    s.XT = fmaf(uT, za, fmaf(-k.half_dt, VpT, fmaf(drift, k.ddt, s.XT)));
    const float z2m1 = fmaf(Z2, Z2, -1.0f);
    const float c4 = pos ? k.c4 : 0.0f, c4T = pos ? k.c4T : 0.0f;
    s.V = fmaf(c4, z2m1, fmaf(xZ2, u, fmaf(-k.kdt, Vp, s.V + k.kth_dt)));
    s.Vv = fmaf(xZ2, uv, fmaf(-k.kdt, Vpv, s.Vv));
    s.VT = fmaf(c4T, z2m1, fmaf(xZ2, uT, fmaf(-k.kdt, VpT, fmaf(-k.kappa_ddt, Vp, s.VT + k.kth_ddt))));
}

template <typename R, int TRUNC>
__device__ __forceinline__ void milstein_step_generic(PathState<R> &s, R za, R zb, const Coef<R> &k)
{
    const R Z1 = za;
    const R Z2 = k.rho * za + k.sq * zb;
    const R W = k.sq * za - k.rho * zb;             // Z1 = rho Z2 + sq W

    const bool pos = s.V > R(0);
    const R Vp = pos ? s.V : R(0);
    const R Vpv = pos ? s.Vv : R(0);
    const R VpT = pos ? s.VT : R(0);
    const R y = Vp * k.dt;                           // V+ dt
    const R rs = rsqrt_pos(y);                       // 1 / sqrt(V+ dt), 0 at 0
    const R u = y * rs;                              // sqrt(V+ dt)
    const R hr = R(0.5) * rs;
    const R uv = Vpv * k.dt * hr;                    // du/dv0
    const R uT = (VpT * k.dt + Vp * k.ddt) * hr;     // du/dT

    s.GE += u * W;
    s.QE += y;

    // ln S with the pre-update variance
    const R drift = k.r - R(0.5) * Vp;
    s.X += drift * k.dt + u * Z1;
    s.Xv += uv * Z1 - k.half_dt * Vpv;
    s.XT += drift * k.ddt - k.half_dt * VpT + uT * Z1;

    const R z2m1 = Z2 * Z2 - R(1);
    if (TRUNC == HESTON_TRUNC_FULL) {
        const R mil = pos ? k.c4 * z2m1 : R(0);
        const R milT = pos ? k.c4T * z2m1 : R(0);
        s.V += k.kth_dt - k.kdt * Vp + k.xi * u * Z2 + mil;
        s.Vv += k.xi * uv * Z2 - k.kdt * Vpv;
        s.VT += k.kth_ddt - k.kappa_ddt * Vp - k.kdt * VpT + k.xi * uT * Z2 + milT;
    } else {
        const R Vt = s.V + k.kth_dt - k.kdt * s.V + k.xi * u * Z2 + k.c4 * z2m1;
        const R Vtv = s.Vv - k.kdt * s.Vv + k.xi * uv * Z2;
        const R VtT = s.VT + k.kth_ddt - k.kappa_ddt * s.V - k.kdt * s.VT + k.xi * uT * Z2
                      + k.c4T * z2m1;
        const bool keep = Vt > R(0);
        s.V = keep ? Vt : R(0);
        s.Vv = keep ? Vtv : R(0);
        s.VT = keep ? VtT : R(0);
    }
}

template <typename R, int TRUNC>
__device__ __forceinline__ void milstein_step(PathState<R> &s, R za, R zb, const Coef<R> &k)
{
    if constexpr (sizeof(R) == 4 && TRUNC == HESTON_TRUNC_FULL)
        milstein_step_f32_full(s, za, zb, k);
    else
        milstein_step_generic<R, TRUNC>(s, za, zb, k);
}

// Asian monitoring date (first: the first date, which closes the Asian
// Gamma weight window).
template <typename R>
__device__ __forceinline__ void monitor(PathState<R> &s, bool first)
{
    const R e = exp_r(s.X);
    s.sA += e;
    s.sC += s.sA;
    s.sAv += e * s.Xv;
    s.sAT += e * s.XT;
    if (first) { s.GA = s.GE; s.QA = s.QE; }
}

// Per-path estimators of contract c: price, delta, gamma, vega, rho, theta.
// With A the payoff's underlying (S_T or Sbar), phi the payoff and phi' its
// slope (1{A>K} for calls, -1{A<K} for puts):
//   price = D phi(A); delta = D phi' A/S0; gamma = D phi' A/S0^2 (lr - 1);
//   vega = D phi' dA/dv0; rho = -T price + D phi' dA/dr; theta = r price - D phi' dA/dT.
// For the European call rho reduces to D K T 1{S_T > K} (Eq. euro_pw).
template <typename R>
__device__ __forceinline__ void estimators(const PathState<R> &s, const ContractSet<R> &cs, int c,
                                           R eT, R est[6])
{
    const R K = cs.K[c], D = cs.D, T = cs.T;
    const bool euro = cs.payoff[c] == HESTON_EUROPEAN;
    R A, dAv, dAT, dAr, lr;
    if (euro) {
        A = cs.S0 * eT;
        dAv = A * s.Xv;
        dAT = A * s.XT;
        dAr = T * A;
        lr = s.GE * cs.inv_sq / s.QE;
    } else {
        A = cs.S0_over_M * s.sA;
        dAv = cs.S0_over_M * s.sAv;
        dAT = cs.S0_over_M * s.sAT;
        dAr = cs.dAr_scale * (cs.Mp1 * s.sA - s.sC);
        lr = s.GA * cs.inv_sq / s.QA;
    }
    R pay, slope;
    if (!cs.is_put[c]) {
        slope = A > K ? R(1) : R(0);
        pay = A > K ? A - K : R(0);
    } else {
        slope = A < K ? R(-1) : R(0);
        pay = A < K ? K - A : R(0);
    }
    const R Dslope = D * slope;
    est[0] = D * pay;
    est[1] = Dslope * A * cs.inv_S0;
    est[2] = Dslope * A * cs.inv_S0sq * (lr - R(1));
    est[3] = Dslope * dAv;
    est[4] = euro ? Dslope * K * T : Dslope * dAr - T * est[0];
    est[5] = cs.r * est[0] - Dslope * dAT;
}

template <typename R>
__device__ __forceinline__ R warp_sum(R v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Asian monitoring layout: none, a date after every step, or every `stride` steps.
enum { MON_NONE = 0, MON_EVERY = 1, MON_STRIDE = 2 };

// Run NP paths (one lane) through all N steps.  Step k uses Philox counter
// (k/2, path_lo, path_hi, 0): words (x, y) for even k, (z, w) for odd k.
template <typename R, int TRUNC, int MON, int NP>
__device__ __forceinline__ void simulate(PathState<R> (&s)[NP], const uint32_t (&plo)[NP],
                                         const uint32_t (&phi)[NP], const Coef<R> &k,
                                         const ContractSet<R> &cs, PhiloxKey key, uint32_t N)
{
#pragma unroll
    for (int q = 0; q < NP; ++q) init_state(s[q], k.v0);
    const uint32_t stride = cs.stride;
    uint32_t next_mon = stride;
    const uint32_t n_pairs = N >> 1;
    for (uint32_t j = 0; j < n_pairs; ++j) {
        uint4 w[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) w[q] = philox4x32_10(make_uint4(j, plo[q], phi[q], 0u), key);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                R za, zb;
                if (h == 0) box_muller(w[q].x, w[q].y, za, zb);
                else        box_muller(w[q].z, w[q].w, za, zb);
                milstein_step<R, TRUNC>(s[q], za, zb, k);
            }
            const uint32_t kp1 = 2u * j + 1u + (uint32_t)h;
            if (MON == MON_EVERY) {
                const bool first = (h == 0) && (j == 0);
#pragma unroll
                for (int q = 0; q < NP; ++q) monitor(s[q], first);
            } else if (MON == MON_STRIDE) {
                if (kp1 == next_mon) {
#pragma unroll
                    for (int q = 0; q < NP; ++q) monitor(s[q], kp1 == stride);
                    next_mon += stride;
                }
            }
        }
    }
    if (N & 1u) {
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const uint4 w = philox4x32_10(make_uint4(n_pairs, plo[q], phi[q], 0u), key);
            R za, zb;
            box_muller(w.x, w.y, za, zb);
            milstein_step<R, TRUNC>(s[q], za, zb, k);
        }
        if (MON == MON_EVERY || (MON == MON_STRIDE && N == next_mon)) {
#pragma unroll
            for (int q = 0; q < NP; ++q) monitor(s[q], N == stride);
        }
    }
}

// ---------------------------------------------------------------------------
// K1: path kernel.  Warp w handles tiles w, w + n_warps, ...; lane l carries
// paths tile*64 + l and tile*64 + l + 32.  Per tile and estimator it writes
// sum_x and sum_x^2 (the lane's two paths added first, then a fixed xor
// butterfly), so tile rows do not depend on the launch shape.
// ---------------------------------------------------------------------------
template <typename R, int TRUNC, int MON>
__global__ void __launch_bounds__(kPathBlock) heston_paths_kernel(Coef<R> k, ContractSet<R> cs, Launch a)
{
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const int nc = cs.n;
    const int width = 12 * nc;

    for (uint64_t tile = warp; tile < a.n_tiles; tile += n_warps) {
        PathState<R> s[2];
        uint32_t plo[2], phi[2];
        bool keep[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const uint64_t local = tile * kTile + (uint64_t)lane + 32u * (uint64_t)q;
            keep[q] = local < a.n_paths;                      // ragged last tile
            const uint64_t g = a.path_begin + local;
            plo[q] = (uint32_t)g;
            phi[q] = (uint32_t)(g >> 32);
        }
        simulate<R, TRUNC, MON, 2>(s, plo, phi, k, cs, a.key, a.N);

        R eT[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) eT[q] = exp_r(s[q].X);
        double *row = a.tile_sums + tile * (uint64_t)width;
#pragma unroll
        for (int c = 0; c < kMaxC; ++c) {
            if (c >= nc) break;
            R e0[6], e1[6];
            estimators(s[0], cs, c, eT[0], e0);
            estimators(s[1], cs, c, eT[1], e1);
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                const R x0 = keep[0] ? e0[j] : R(0), x1 = keep[1] ? e1[j] : R(0);
                const R sx = warp_sum(x0 + x1);
                const R sxx = warp_sum(x0 * x0 + x1 * x1);
                if (lane == j) row[c * 6 + j] = (double)sx;
                if (lane == 6 + j) row[6 * nc + c * 6 + j] = (double)sxx;
            }
        }
    }
}

// Test kernel: one thread per requested path, the same step code, writes the
// per-path record and estimators.
template <typename R, int TRUNC, int MON>
__global__ void heston_debug_kernel(Coef<R> k, ContractSet<R> cs, PhiloxKey key, uint32_t N,
                                    const uint64_t *paths, uint32_t count, double *rec, double *est)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const uint64_t g = paths[i];
    PathState<R> s[1];
    const uint32_t plo[1] = {(uint32_t)g}, phi[1] = {(uint32_t)(g >> 32)};
    simulate<R, TRUNC, MON, 1>(s, plo, phi, k, cs, key, N);
    const R eT = exp_r(s[0].X);
    const double S0 = (double)cs.S0, M = (double)cs.M;
    double *o = rec + (uint64_t)i * kRecordDoubles;
    o[0] = (double)s[0].X;   o[1] = (double)s[0].V;
    o[2] = (double)s[0].Xv;  o[3] = (double)s[0].Vv;
    o[4] = (double)s[0].XT;  o[5] = (double)s[0].VT;
    o[6] = S0 * (double)s[0].sA;
    o[7] = S0 * ((double)cs.T / M) * ((M + 1.0) * (double)s[0].sA - (double)s[0].sC);
    o[8] = S0 * (double)s[0].sAv;
    o[9] = S0 * (double)s[0].sAT;
    o[10] = (double)s[0].GE; o[11] = (double)s[0].QE;
    o[12] = (double)s[0].GA; o[13] = (double)s[0].QA;
    o[14] = 0.0;
    for (int c = 0; c < cs.n; ++c) {
        R e[6];
        estimators(s[0], cs, c, eT, e);
        for (int j = 0; j < 6; ++j) est[((uint64_t)i * cs.n + c) * 6 + j] = (double)e[j];
    }
}

template <typename R>
__global__ void rng_debug_kernel(PhiloxKey key, const uint64_t *paths, const uint32_t *steps,
                                 uint32_t count, uint32_t *words, double *normals)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const uint64_t g = paths[i];
    const uint32_t st = steps[i];
    const uint4 w = philox4x32_10(make_uint4(st >> 1, (uint32_t)g, (uint32_t)(g >> 32), 0u), key);
    words[4 * i + 0] = w.x; words[4 * i + 1] = w.y;
    words[4 * i + 2] = w.z; words[4 * i + 3] = w.w;
    R za, zb;
    if (st & 1u) box_muller(w.z, w.w, za, zb);
    else         box_muller(w.x, w.y, za, zb);
    normals[2 * i] = (double)za;
    normals[2 * i + 1] = (double)zb;
}

// ---------------------------------------------------------------------------
// K2: fixed-order FP64 reduction.  Level 1: group g sums tiles
// [g*256, (g+1)*256) column by column in tile order.  Level 2: one CTA sums
// the groups in order and forms mean and standard error per estimator.
// ---------------------------------------------------------------------------
__global__ void reduce_groups_kernel(const double *tile_sums, uint64_t n_tiles, int width,
                                     double *group_sums)
{
    const uint64_t g = blockIdx.x;
    const uint64_t lo = g * kGroupTiles;
    const uint64_t hi = lo + kGroupTiles < n_tiles ? lo + kGroupTiles : n_tiles;
    for (int col = threadIdx.x; col < width; col += blockDim.x) {
        double acc = 0.0;
        for (uint64_t t = lo; t < hi; ++t) acc += tile_sums[t * width + col];
        group_sums[g * width + col] = acc;
    }
}

__global__ void reduce_final_kernel(const double *group_sums, uint64_t n_groups, int n_contracts,
                                    double n_paths, int gamma_nan, double *out)
{
    __shared__ double tot[12 * kMaxC];
    const int width = 12 * n_contracts;
    const int E = 6 * n_contracts;
    for (int col = threadIdx.x; col < width; col += blockDim.x) {
        double acc = 0.0;
        for (uint64_t g = 0; g < n_groups; ++g) acc += group_sums[g * width + col];
        tot[col] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const int c = e / 6, j = e % 6;
        const double mean = tot[e] / n_paths;
        const double var = (tot[E + e] - n_paths * mean * mean) / (n_paths - 1.0);
        double se = sqrt(var > 0.0 ? var / n_paths : 0.0);
        double m = mean;
        if (gamma_nan && j == 2) { m = nan(""); se = nan(""); }
        out[c * 12 + j] = m;
        out[c * 12 + 6 + j] = se;
    }
}

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

struct Prepared {
    ContractSet<double> cs;
    ContractSet<float> csf;
    Coef<float> kf;
    Coef<double> kd;
    heston_options opt;
    uint32_t N;
    bool gamma_nan;
};

template <typename R> const ContractSet<R> &cs_of(const Prepared &pp);
template <> const ContractSet<double> &cs_of<double>(const Prepared &pp) { return pp.cs; }
template <> const ContractSet<float> &cs_of<float>(const Prepared &pp) { return pp.csf; }

bool finite_nonneg(double x) { return std::isfinite(x) && x >= 0.0; }

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
    if (o.rng == HESTON_RNG_SOBOL_BB) return HESTON_ERR_UNSUPPORTED;
    if (o.reserved != 0) return HESTON_ERR_INVALID_ARG;
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
    Coef<float> kf;
    kf.v0 = (float)kd.v0; kf.dt = (float)kd.dt; kf.ddt = (float)kd.ddt;
    kf.half_dt = (float)kd.half_dt; kf.r = (float)kd.r; kf.kdt = (float)kd.kdt;
    kf.kth_dt = (float)kd.kth_dt; kf.kth_ddt = (float)kd.kth_ddt; kf.kappa_ddt = (float)kd.kappa_ddt;
    kf.xi = (float)kd.xi; kf.c4 = (float)kd.c4; kf.c4T = (float)kd.c4T;
    kf.rho = (float)kd.rho; kf.sq = (float)kd.sq;

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
uint64_t groups_for(uint64_t n_tiles) { return (n_tiles + kGroupTiles - 1) / kGroupTiles; }
size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t workspace_bytes(uint32_t nc, uint64_t n_paths)
{
    const uint64_t nt = tiles_for(n_paths);
    const size_t w = 12u * nc * sizeof(double);
    return align256(nt * w) + align256(groups_for(nt) * w);
}

template <typename R, int TRUNC, int MON>
cudaError_t launch_paths_t(const Prepared &pp, const Coef<R> &k, const Launch &a, cudaStream_t st)
{
    auto kern = heston_paths_kernel<R, TRUNC, MON>;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int n_sm = 0;
    e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int block = pp.opt.block_threads ? (int)pp.opt.block_threads : kPathBlock;
    uint64_t grid;
    if (pp.opt.grid_ctas) {
        grid = pp.opt.grid_ctas;
    } else {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, 0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        const uint64_t warps_per_cta = (uint64_t)block / 32;
        const uint64_t need = (a.n_tiles + warps_per_cta - 1) / warps_per_cta;
        const uint64_t full = (uint64_t)n_sm * (uint64_t)per_sm;
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

template <typename R>
cudaError_t launch_paths_r(const Prepared &pp, const Coef<R> &k, const Launch &a, cudaStream_t st)
{
    const int mon = mon_mode(pp.cs);
    if (pp.opt.trunc == HESTON_TRUNC_FULL) {
        if (mon == MON_NONE) return launch_paths_t<R, 0, MON_NONE>(pp, k, a, st);
        if (mon == MON_EVERY) return launch_paths_t<R, 0, MON_EVERY>(pp, k, a, st);
        return launch_paths_t<R, 0, MON_STRIDE>(pp, k, a, st);
    }
    if (mon == MON_NONE) return launch_paths_t<R, 1, MON_NONE>(pp, k, a, st);
    if (mon == MON_EVERY) return launch_paths_t<R, 1, MON_EVERY>(pp, k, a, st);
    return launch_paths_t<R, 1, MON_STRIDE>(pp, k, a, st);
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
    reduce_groups_kernel<<<(unsigned)ng, 128, 0, st>>>(tile_sums, n_tiles, width, group_sums);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_final_kernel<<<1, 128, 0, st>>>(group_sums, ng, nc, (double)n_paths, gamma_nan ? 1 : 0, out);
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

void fill_results(const double *h, uint32_t nc, uint64_t n_paths, int status, heston_result *out)
{
    for (uint32_t c = 0; c < nc; ++c) {
        heston_result &r = out[c];
        r.price = h[c * 12 + 0]; r.delta = h[c * 12 + 1]; r.gamma = h[c * 12 + 2];
        r.vega = h[c * 12 + 3];  r.rho = h[c * 12 + 4];   r.theta = h[c * 12 + 5];
        for (int j = 0; j < 6; ++j) r.se[j] = h[c * 12 + 6 + j];
        r.n_paths = n_paths;
        r.status = status;
        r.reserved = 0;
    }
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

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char *heston_status_string(int status)
{
    switch (status) {
    case HESTON_OK: return "ok";
    case HESTON_WARN_GAMMA_UNDEFINED: return "gamma undefined (|rho| == 1 or v0 == 0); set to NaN";
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
    DeviceGuard g(pp.opt.device);
    if (g.err != cudaSuccess) return HESTON_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)pp.opt.cuda_stream;
    const size_t ws_bytes = workspace_bytes(n_contracts, n_paths);
    const size_t out_bytes = 12u * n_contracts * sizeof(double);
    void *ws = nullptr;
    if (cudaMallocAsync(&ws, ws_bytes + align256(out_bytes), st) != cudaSuccess) {
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
    fill_results(h, n_contracts, n_paths, status, out);
    return status;
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
    if (!paths || count == 0 || !h_records || !h_estimators) return HESTON_ERR_INVALID_ARG;
    DeviceGuard g(pp.opt.device);
    if (g.err != cudaSuccess) return HESTON_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)pp.opt.cuda_stream;
    const size_t pb = sizeof(uint64_t) * count;
    const size_t rb = sizeof(double) * kRecordDoubles * count;
    const size_t eb = sizeof(double) * 6 * n_contracts * (size_t)count;
    char *buf = nullptr;
    if (cudaMallocAsync((void **)&buf, align256(pb) + align256(rb) + align256(eb), st) != cudaSuccess) {
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
        const bool full = pp.opt.trunc == HESTON_TRUNC_FULL;
#define HESTON_DBG(R, TR, MO, K) heston_debug_kernel<R, TR, MO><<<grid, 128, 0, st>>>(K, cs_of<R>(pp), key, pp.N, dp, count, dr, de)
#define HESTON_DBG_M(R, TR, K) do { if (mon == MON_NONE) HESTON_DBG(R, TR, MON_NONE, K); \
                                    else if (mon == MON_EVERY) HESTON_DBG(R, TR, MON_EVERY, K); \
                                    else HESTON_DBG(R, TR, MON_STRIDE, K); } while (0)
        if (pp.opt.prec == HESTON_FP32) {
            if (full) HESTON_DBG_M(float, 0, pp.kf); else HESTON_DBG_M(float, 1, pp.kf);
        } else {
            if (full) HESTON_DBG_M(double, 0, pp.kd); else HESTON_DBG_M(double, 1, pp.kd);
        }
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

}  // extern "C"
