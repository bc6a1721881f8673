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

__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, PhiloxKey key)
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
    R kappa, theta;               // for the adjoint
    // QE (E = e^{-kappa dt}, g = (1 - E)/kappa; *_T = d/dT at fixed N):
    // m = qmth + V qE, s^2 = qs0 + V qs1, ln S += qK0r + qK1 V + qK2 V' + sq ut Zb
    // with ut^2 = qhdt (V + V').
    R qE, qE_T, qmth, qmth_T;
    R qs1, qs1_T, qs0, qs0_T;
    R qK0r, qK0r_T, qK1, qK2, qK12_T;
    R qhdt, qhddt;
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

// One Milstein step with its tangents, from independent normals (za, zb);
// EULER drops the xi^2 dt (Z2^2 - 1) / 4 term (Sec. 2.4.1).
// FP32 full truncation: the same recursion with shared products hoisted
// (xi Z2 feeds V and both V tangents; the truncation mask scales 1/(2u)).
template <bool EULER>
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
    const float c4 = (pos && !EULER) ? k.c4 : 0.0f, c4T = (pos && !EULER) ? k.c4T : 0.0f;
    s.V = fmaf(c4, z2m1, fmaf(xZ2, u, fmaf(-k.kdt, Vp, s.V + k.kth_dt)));
    s.Vv = fmaf(xZ2, uv, fmaf(-k.kdt, Vpv, s.Vv));
    s.VT = fmaf(c4T, z2m1, fmaf(xZ2, uT, fmaf(-k.kdt, VpT, fmaf(-k.kappa_ddt, Vp, s.VT + k.kth_ddt))));
}

template <typename R, int TRUNC, bool EULER>
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

    const R z2m1 = EULER ? R(0) : Z2 * Z2 - R(1);
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

__device__ __forceinline__ float norm_cdf(float x) { return normcdff(x); }
__device__ __forceinline__ double norm_cdf(double x) { return normcdf(x); }
__device__ __forceinline__ float log_pos(float x) { return lg2_approx(x) * 0.69314718f; }
__device__ __forceinline__ double log_pos(double x) { return log(x); }

// One QE step (Andersen 2008) with its tangents.  The variance: exact
// conditional mean m and variance s^2 of the CIR transition, psi = s^2/m^2;
// psi <= 1.5: V' = a (b + Za)^2, b^2 = 2/psi - 1 + sqrt(2/psi (2/psi - 1)),
// a = m / (1 + b^2); psi > 1.5: V' = 0 when Phi(-Za) >= 1 - p, else
// m ln((1 - p)/Phi(-Za)) / (1 - p) with 1 - p = 2 / (psi + 1).  Then
// ln S' = ln S + r dt + K0 + K1 V + K2 V' + sq ut Zb, ut = sqrt(dt (V + V')/2);
// Zb does not move the variance, so the Gamma weights are ut Zb and ut^2.
template <typename R>
__device__ __forceinline__ void qe_step(PathState<R> &s, R za, R zb, const Coef<R> &k)
{
    const R m = k.qmth + s.V * k.qE;
    const R mv = s.Vv * k.qE;
    const R mT = k.qmth_T + s.V * k.qE_T + s.VT * k.qE;
    const R s2 = k.qs0 + s.V * k.qs1;
    const R s2v = s.Vv * k.qs1;
    const R s2T = k.qs0_T + s.V * k.qs1_T + s.VT * k.qs1;
    const R im = R(1) / m;                           // m >= theta (1 - E) > 0
    const R psi = s2 * im * im;
    const R psiv = (s2v - R(2) * s2 * mv * im) * im * im;
    const R psiT = (s2T - R(2) * s2 * mT * im) * im * im;
    R Vn, Vnv, VnT;
    if (psi <= R(1.5)) {
        const R y = R(2) / psi;
        const R hy2 = R(-0.5) * y * y;               // dy/dpsi
        const R root = sqrt(y * (y - R(1)));
        const R b2 = y - R(1) + root;
        const R db2 = (R(1) + (R(2) * y - R(1)) / (R(2) * root)) * hy2;   // db^2/dpsi
        const R b = sqrt(b2);
        const R ia = R(1) / (R(1) + b2);
        const R a = m * ia;
        const R b2v = db2 * psiv, b2T = db2 * psiT;
        const R hb = R(0.5) / b;
        const R av = (mv - a * b2v) * ia, aT = (mT - a * b2T) * ia;
        const R bz = b + za;
        Vn = a * bz * bz;
        Vnv = bz * (av * bz + R(2) * a * b2v * hb);
        VnT = bz * (aT * bz + R(2) * a * b2T * hb);
    } else {
        const R omp = R(2) / (psi + R(1));           // 1 - p
        const R q = norm_cdf(-za);                   // 1 - Uv
        if (q < omp) {
            const R L = log_pos(omp / q);
            const R iomp = R(1) / omp;
            Vn = m * L * iomp;
            Vnv = mv * L * iomp + R(0.5) * m * psiv * (L - R(1));
            VnT = mT * L * iomp + R(0.5) * m * psiT * (L - R(1));
        } else {
            Vn = R(0); Vnv = R(0); VnT = R(0);
        }
    }
    const R sum = s.V + Vn;
    const R y = k.qhdt * sum;                        // ut^2
    const R rs = rsqrt_pos(y);
    const R ut = y * rs;
    const R utv = R(0.5) * k.qhdt * (s.Vv + Vnv) * rs;
    const R utT = R(0.5) * (k.qhddt * sum + k.qhdt * (s.VT + VnT)) * rs;
    s.GE += ut * zb;
    s.QE += y;
    s.X += k.qK0r + k.qK1 * s.V + k.qK2 * Vn + k.sq * ut * zb;
    s.Xv += k.qK1 * s.Vv + k.qK2 * Vnv + k.sq * utv * zb;
    s.XT += k.qK0r_T + k.qK12_T * sum + k.qK1 * s.VT + k.qK2 * VnT + k.sq * utT * zb;
    s.V = Vn; s.Vv = Vnv; s.VT = VnT;
}

// Scheme of a kernel instantiation: Milstein or Euler with full truncation
// or the floor, or QE.  Values 0 and 1 are the Milstein truncations.
enum { STEP_MIL_FULL = 0, STEP_MIL_FLOOR = 1, STEP_EUL_FULL = 2, STEP_EUL_FLOOR = 3, STEP_QE = 4 };

template <typename R, int STEP>
__device__ __forceinline__ void scheme_step(PathState<R> &s, R za, R zb, const Coef<R> &k)
{
    if constexpr (STEP == STEP_QE)
        qe_step(s, za, zb, k);
    else if constexpr (sizeof(R) == 4 && (STEP & 1) == HESTON_TRUNC_FULL)
        milstein_step_f32_full<(STEP >= STEP_EUL_FULL)>(s, za, zb, k);
    else
        milstein_step_generic<R, STEP & 1, (STEP >= STEP_EUL_FULL)>(s, za, zb, k);
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
template <typename R, int STEP, int MON, int NP>
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
                scheme_step<R, STEP>(s[q], za, zb, k);
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
            scheme_step<R, STEP>(s[q], za, zb, k);
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
template <typename R, int STEP, int MON>
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
        simulate<R, STEP, MON, 2>(s, plo, phi, k, cs, a.key, a.N);

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

// Per-path record (see heston_mc_debug_paths) and estimators of one path.
template <typename R>
__device__ void write_debug_record(const PathState<R> &s, const ContractSet<R> &cs, double *o,
                                   double *est)
{
    const R eT = exp_r(s.X);
    const double S0 = (double)cs.S0, M = (double)cs.M;
    o[0] = (double)s.X;   o[1] = (double)s.V;
    o[2] = (double)s.Xv;  o[3] = (double)s.Vv;
    o[4] = (double)s.XT;  o[5] = (double)s.VT;
    o[6] = S0 * (double)s.sA;
    o[7] = S0 * ((double)cs.T / M) * ((M + 1.0) * (double)s.sA - (double)s.sC);
    o[8] = S0 * (double)s.sAv;
    o[9] = S0 * (double)s.sAT;
    o[10] = (double)s.GE; o[11] = (double)s.QE;
    o[12] = (double)s.GA; o[13] = (double)s.QA;
    o[14] = 0.0;
    for (int c = 0; c < cs.n; ++c) {
        R e[6];
        estimators(s, cs, c, eT, e);
        for (int j = 0; j < 6; ++j) est[c * 6 + j] = (double)e[j];
    }
}

// Test kernel: one thread per requested path, the same step code, writes the
// per-path record and estimators.
template <typename R, int STEP, int MON>
__global__ void heston_debug_kernel(Coef<R> k, ContractSet<R> cs, PhiloxKey key, uint32_t N,
                                    const uint64_t *paths, uint32_t count, double *rec, double *est)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const uint64_t g = paths[i];
    PathState<R> s[1];
    const uint32_t plo[1] = {(uint32_t)g}, phi[1] = {(uint32_t)(g >> 32)};
    simulate<R, STEP, MON, 1>(s, plo, phi, k, cs, key, N);
    write_debug_record(s[0], cs, rec + (uint64_t)i * kRecordDoubles, est + (uint64_t)i * cs.n * 6);
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
// Randomised quasi-Monte Carlo normals (Sec. 2.7): a Sobol sequence with
// digital shifts, fed through a Brownian bridge so that the first dimensions
// carry the coarse shape of both Brownian motions.  Definitions (the test
// oracle implements the same ones separately):
//   * dimension 0: v_k = 2^(32-k); dimension j >= 1: the j-th primitive
//     polynomial over GF(2) ordered by (degree, coefficient bits), initial
//     m_1..m_s from Philox (key 0x50B01, counter ((k-1)/4, j, c, 3), word
//     (k-1)%4, m_k = 2 (w mod 2^(k-1)) + 1); for j < 32 the first candidate c
//     that keeps the leading (j+1)x(j+1) first-digit matrix non-singular
//     over GF(2) (Property A), else c = 0; Bratley-Fox recurrence.
//   * replicate r's shift of dimension d: Philox (seed key) counter
//     (d/4, r, 0, 2), word d%4; y = x_d(point) XOR shift.
//   * u = ((y >> 8) + 1/2) 2^-24, z = Phi^-1(u).
//   * Brownian bridge on the step grid 0..N: node 0 = time N; then
//     breadth-first bisection m = l + (r-l)/2 of intervals with r - l >= 2.
//     Node j drives motion a with dimension 2j and motion b with 2j+1.
// In the kernel the bridge runs in time order: a per-thread stack holds W at
// the right ends of the open intervals.  Entering step k (W_k known), the
// plan pushes W_m = W_k + (m-k)/(r-k) (W_r - W_k) + sqrt((m-k)(r-m)/(r-k)) z
// for the nodes m of [k, r] down to [k, k+1] (r: the stack top), then pops
// W_{k+1}; the step normal is W_{k+1} - W_k.  Every W is interpolated from
// two stored values, so FP32 rounding does not accumulate along the path.
// ---------------------------------------------------------------------------
constexpr int kQmcMaxLevels = 14;           // stack slots (slot 0 = 0); n_steps <= 2048
constexpr uint32_t kQmcMaxSteps = 2048;
constexpr uint32_t kSobolKey0 = 0x50B01u, kSobolKey1 = 0u;
constexpr uint32_t kSobolInitTag = 3u, kSobolShiftTag = 2u;

struct BridgeOp {
    int32_t node;       // node j: normals from dimensions 2j and 2j+1
    float a;            // (m - k) / (r - k)
    float s;            // sqrt((m - k)(r - m) / (r - k)); node 0: a = 0, s = sqrt(N)
    int32_t pad;
};

struct QmcTables {
    const uint32_t *V;        // [D][32] direction integers
    const uint32_t *T;        // [D][64] x_d(p) for the 64 points p of a tile
    const BridgeOp *ev;       // stack pushes, step-major
    const int32_t *ev_off;    // [N + 1] first push of each step
};

struct QmcLaunch {
    QmcTables tb;
    const uint32_t *U;        // [tiles per replicate][D]: x_d(64 t), high bits of the point
    const uint32_t *shift;    // [replicates][D]
    uint32_t D, N, tpr;       // Sobol dims (2N), steps, tiles per replicate
    uint64_t n_tiles;
    double *tile_sums;
};

// Phi^-1 of the 24-bit uniform of y, taking the lower half by symmetry so that
// the FP32 uniform (2k + 1) 2^-25 is exact and never 1.
__device__ __forceinline__ float qmc_normal(uint32_t y)
{
    const uint32_t k = y >> 8;
    const bool upper = k >= 0x800000u;
    const uint32_t kk = upper ? 0xFFFFFFu - k : k;
    const float u = (float)(2u * kk + 1u) * 2.98023223876953125e-8f;
    const float z = normcdfinvf(u);
    return upper ? -z : z;
}

// NP paths of one lane through all N steps with bridge normals.  pos[q]: the
// path's position in its 64-point tile; U / Sh: the tile's high-bit Sobol
// integers and the replicate's shifts.
template <int TRUNC, int MON, int NP>
__device__ __forceinline__ void simulate_qmc(PathState<float> (&s)[NP], const uint32_t (&pos)[NP],
                                             const Coef<float> &k, const ContractSet<float> &cs,
                                             const QmcTables &tb, const uint32_t *U,
                                             const uint32_t *Sh, uint32_t N)
{
    float st[NP][2][kQmcMaxLevels];             // W at pending right ends; slot 0 = 0
    float Wk[NP][2];                            // W at the current time
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        init_state(s[q], k.v0);
        Wk[q][0] = 0.0f;
        Wk[q][1] = 0.0f;
        st[q][0][0] = 0.0f;
        st[q][1][0] = 0.0f;
    }
    int top = 0;
    const uint32_t stride = cs.stride;
    uint32_t next_mon = stride;
    for (uint32_t kk = 0; kk < N; ++kk) {
        const int e1 = tb.ev_off[kk + 1];
        for (int e = tb.ev_off[kk]; e < e1; ++e) {
            const BridgeOp op = tb.ev[e];
#pragma unroll
            for (int mu = 0; mu < 2; ++mu) {
                const uint32_t dim = 2u * (uint32_t)op.node + (uint32_t)mu;
                const uint32_t hi = U[dim] ^ Sh[dim];
#pragma unroll
                for (int q = 0; q < NP; ++q) {
                    const float z = qmc_normal(tb.T[dim * 64u + pos[q]] ^ hi);
                    const float Wr = st[q][mu][top];
                    st[q][mu][top + 1] = fmaf(op.s, z, fmaf(op.a, Wr - Wk[q][mu], Wk[q][mu]));
                }
            }
            ++top;
        }
        float za[NP], zb[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const float wa = st[q][0][top], wb = st[q][1][top];
            za[q] = wa - Wk[q][0];
            zb[q] = wb - Wk[q][1];
            Wk[q][0] = wa;
            Wk[q][1] = wb;
        }
        --top;
#pragma unroll
        for (int q = 0; q < NP; ++q) scheme_step<float, TRUNC>(s[q], za[q], zb[q], k);
        const uint32_t kp1 = kk + 1u;
        if (MON == MON_EVERY) {
#pragma unroll
            for (int q = 0; q < NP; ++q) monitor(s[q], kk == 0);
        } else if (MON == MON_STRIDE) {
            if (kp1 == next_mon) {
#pragma unroll
                for (int q = 0; q < NP; ++q) monitor(s[q], kp1 == stride);
                next_mon += stride;
            }
        }
    }
}

// QMC path kernel: same tile layout and epilogue as heston_paths_kernel.
// Tile t belongs to replicate t / tpr; every tile is full (points per
// replicate are a multiple of 64).
template <int TRUNC, int MON>
__global__ void __launch_bounds__(kPathBlock) heston_qmc_kernel(Coef<float> k, ContractSet<float> cs,
                                                                QmcLaunch a)
{
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const int nc = cs.n;
    const int width = 12 * nc;
    for (uint64_t tile = warp; tile < a.n_tiles; tile += n_warps) {
        const uint32_t rep = (uint32_t)(tile / a.tpr), tin = (uint32_t)(tile % a.tpr);
        PathState<float> s[2];
        const uint32_t pos[2] = {(uint32_t)lane, (uint32_t)lane + 32u};
        simulate_qmc<TRUNC, MON, 2>(s, pos, k, cs, a.tb, a.U + (uint64_t)tin * a.D,
                                    a.shift + (uint64_t)rep * a.D, a.N);
        float eT[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) eT[q] = exp_r(s[q].X);
        double *row = a.tile_sums + tile * (uint64_t)width;
#pragma unroll
        for (int c = 0; c < kMaxC; ++c) {
            if (c >= nc) break;
            float e0[6], e1[6];
            estimators(s[0], cs, c, eT[0], e0);
            estimators(s[1], cs, c, eT[1], e1);
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                const float sx = warp_sum(e0[j] + e1[j]);
                const float sxx = warp_sum(e0[j] * e0[j] + e1[j] * e1[j]);
                if (lane == j) row[c * 6 + j] = (double)sx;
                if (lane == 6 + j) row[6 * nc + c * 6 + j] = (double)sxx;
            }
        }
    }
}

// Per-launch tables: U[t][d] = x_d(64 t) and the replicates' digital shifts.
__global__ void qmc_setup_kernel(const uint32_t *V, uint32_t D, uint32_t tpr, uint32_t R,
                                 PhiloxKey key, uint32_t *U, uint32_t *shift)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nU = (uint64_t)tpr * D;
    if (i < nU) {
        const uint32_t t = (uint32_t)(i / D), d = (uint32_t)(i % D);
        const uint64_t n = (uint64_t)t * 64u;
        uint32_t x = 0;
        for (int b = 6; b < 32; ++b)
            if ((n >> b) & 1u) x ^= V[d * 32u + b];
        U[i] = x;
    } else if (i < nU + (uint64_t)R * D) {
        const uint64_t j = i - nU;
        const uint32_t r = (uint32_t)(j / D), d = (uint32_t)(j % D);
        const uint4 w = philox4x32_10(make_uint4(d >> 2, r, 0u, kSobolShiftTag), key);
        const uint32_t sel = d & 3u;
        shift[j] = sel == 0 ? w.x : sel == 1 ? w.y : sel == 2 ? w.z : w.w;
    }
}

// Test support: Udbg[i][d] = x_d(points[i] with its low 6 bits cleared).
__global__ void qmc_debug_high_bits_kernel(const uint32_t *V, uint32_t D, const uint32_t *points,
                                           uint32_t count, uint32_t *Udbg)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (uint64_t)count * D) return;
    const uint32_t p = (uint32_t)(i / D), d = (uint32_t)(i % D);
    const uint32_t n = points[p];
    uint32_t x = 0;
    for (int b = 6; b < 32; ++b)
        if ((n >> b) & 1u) x ^= V[d * 32u + b];
    Udbg[i] = x;
}

// Test kernel: one thread per requested point of one replicate, through the
// same simulate_qmc as the path kernel.
template <int TRUNC, int MON>
__global__ void heston_qmc_debug_kernel(Coef<float> k, ContractSet<float> cs, QmcTables tb,
                                        uint32_t N, const uint32_t *points, const uint32_t *Udbg,
                                        const uint32_t *shift_row, uint32_t count, double *rec,
                                        double *est)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    PathState<float> s[1];
    const uint32_t pos[1] = {points[i] & 63u};
    simulate_qmc<TRUNC, MON, 1>(s, pos, k, cs, tb, Udbg + (uint64_t)i * 2u * N, shift_row, N);
    write_debug_record(s[0], cs, rec + (uint64_t)i * kRecordDoubles, est + (uint64_t)i * cs.n * 6);
}

__global__ void reduce_replicates_kernel(const double *tile_sums, uint32_t tpr, int width,
                                         double *rep_sums)
{
    const uint64_t r = blockIdx.x;
    for (int col = threadIdx.x; col < width; col += blockDim.x) {
        double acc = 0.0;
        for (uint32_t t = 0; t < tpr; ++t) acc += tile_sums[(r * tpr + t) * (uint64_t)width + col];
        rep_sums[r * width + col] = acc;
    }
}

// Randomised-QMC estimate: mean over replicates of the replicate averages;
// SE = their sample stdev / sqrt(R).
__global__ void reduce_final_qmc_kernel(const double *rep_sums, uint32_t R, int n_contracts,
                                        double ppr, int gamma_nan, double *out)
{
    const int width = 12 * n_contracts;
    const int E = 6 * n_contracts;
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        double mean = 0.0;
        for (uint32_t r = 0; r < R; ++r) mean += rep_sums[(uint64_t)r * width + e] / ppr;
        mean /= (double)R;
        double var = 0.0;
        for (uint32_t r = 0; r < R; ++r) {
            const double d = rep_sums[(uint64_t)r * width + e] / ppr - mean;
            var += d * d;
        }
        var /= (double)(R - 1);
        double se = sqrt(var / (double)R);
        const int c = e / 6, j = e % 6;
        if (gamma_nan && j == 2) { mean = nan(""); se = nan(""); }
        out[c * 12 + j] = mean;
        out[c * 12 + 6 + j] = se;
    }
}

// ---------------------------------------------------------------------------
// K2: fixed-order FP64 reduction.  Level 1: group g sums tiles
// [g*256, (g+1)*256) column by column in tile order.  Level 2: one CTA sums
// the groups in order and forms mean and standard error per estimator.
// ---------------------------------------------------------------------------
// Column sums of tile rows [lo, hi) in row order (one group of <= 256 tiles).
__device__ __forceinline__ void sum_rows(const double *rows, uint64_t lo, uint64_t hi, int width,
                                         double *out_row)
{
    for (int col = threadIdx.x; col < width; col += blockDim.x) {
        double acc = 0.0;
        for (uint64_t t = lo; t < hi; ++t) acc += rows[t * width + col];
        out_row[col] = acc;
    }
}

// Sum n_groups group rows in order and write mean / SE per estimator.
__device__ __forceinline__ void finish_groups(const double *group_sums, uint64_t n_groups,
                                              int n_contracts, double n_paths, int gamma_nan,
                                              double *out)
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

__global__ void reduce_groups_kernel(const double *tile_sums, uint64_t n_tiles, int width,
                                     double *group_sums)
{
    const uint64_t g = blockIdx.x;
    const uint64_t lo = g * kGroupTiles;
    const uint64_t hi = lo + kGroupTiles < n_tiles ? lo + kGroupTiles : n_tiles;
    sum_rows(tile_sums, lo, hi, width, group_sums + g * width);
}

__global__ void reduce_final_kernel(const double *group_sums, uint64_t n_groups, int n_contracts,
                                    double n_paths, int gamma_nan, double *out)
{
    finish_groups(group_sums, n_groups, n_contracts, n_paths, gamma_nan, out);
}

// ---------------------------------------------------------------------------
// Batched persistent launch: many contracts, each with its own parameters,
// path count, step count and seed, in one launch.  Work items are
// (contract, 64-path tile) pairs handed out through an atomic counter,
// contracts with the most steps first; each contract's tile rows and their
// reduction (sum_rows / finish_groups) are those of its own launch, so every
// result equals the contract's own launch bit for bit.  A device status word
// lets a caller stop the launch between work items: 0 = run, 1 = cancel
// requested, 2 = the kernel saw the request and took no further work.
// ---------------------------------------------------------------------------
struct BatchItemDev {
    Coef<float> k;
    ContractSet<float> cs;        // one contract
    PhiloxKey key;
    uint64_t n_paths;
    uint64_t n_tiles;
    uint64_t row_begin;           // first tile row of this contract
    uint64_t group_begin;         // first group row of this contract
    uint32_t N;
    int32_t mon;
    int32_t gamma_nan;
    int32_t pad;
};

struct BatchLaunch {
    const BatchItemDev *items;    // caller order
    const uint64_t *work_begin;   // [n_items] first work index of the p-th contract in work order
    const uint32_t *work_item;    // [n_items] contract of the p-th position in work order
    const uint64_t *work_tile0;   // [n_items] first tile of the p-th position (NULL = 0)
    const uint64_t *group_begin;  // [n_items] (caller order) first group row, for the reductions
    uint32_t n_items;
    uint64_t total_work;
    unsigned long long *counter;
    int32_t *status;
    double *rows;
};

template <int TRUNC>
__global__ void __launch_bounds__(kPathBlock) heston_batch_kernel(BatchLaunch a)
{
    const int lane = threadIdx.x & 31;
    bool saw_cancel = false;
    while (true) {
        unsigned long long g = ~0ull;
        if (lane == 0) {
            const int32_t st = a.status ? *(volatile int32_t *)a.status : 0;
            if (st != 0) saw_cancel = true;
            else g = atomicAdd(a.counter, 1ull);
        }
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= a.total_work) break;
        uint32_t lo = 0, hi = a.n_items;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (a.work_begin[mid] <= g) lo = mid; else hi = mid;
        }
        const BatchItemDev &it = a.items[a.work_item[lo]];
        const uint64_t t = g - a.work_begin[lo] + (a.work_tile0 ? a.work_tile0[lo] : 0ull);
        const Coef<float> k = it.k;
        const PhiloxKey key = it.key;
        PathState<float> s[2];
        uint32_t plo[2], phi[2];
        bool keep[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const uint64_t local = t * kTile + (uint64_t)lane + 32u * (uint64_t)q;
            keep[q] = local < it.n_paths;
            plo[q] = (uint32_t)local;
            phi[q] = (uint32_t)(local >> 32);
        }
        if (it.mon == MON_NONE)       simulate<float, TRUNC, MON_NONE, 2>(s, plo, phi, k, it.cs, key, it.N);
        else if (it.mon == MON_EVERY) simulate<float, TRUNC, MON_EVERY, 2>(s, plo, phi, k, it.cs, key, it.N);
        else                          simulate<float, TRUNC, MON_STRIDE, 2>(s, plo, phi, k, it.cs, key, it.N);
        float e0[6], e1[6];
        estimators(s[0], it.cs, 0, exp_r(s[0].X), e0);
        estimators(s[1], it.cs, 0, exp_r(s[1].X), e1);
        double *row = a.rows + (it.row_begin + t) * 12u;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            const float x0 = keep[0] ? e0[j] : 0.0f, x1 = keep[1] ? e1[j] : 0.0f;
            const float sx = warp_sum(x0 + x1);
            const float sxx = warp_sum(x0 * x0 + x1 * x1);
            if (lane == j) row[j] = (double)sx;
            if (lane == 6 + j) row[6 + j] = (double)sxx;
        }
    }
    if (saw_cancel) atomicCAS(a.status, 1, 2);
}

// One block per group row of the whole batch: the contract is found from
// the flat group index.
__global__ void batch_reduce_groups_kernel(const BatchItemDev *items, const uint64_t *group_begin,
                                           uint32_t n_items, const double *rows, double *groups)
{
    const uint64_t g = blockIdx.x;
    uint32_t lo = 0, hi = n_items;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (group_begin[mid] <= g) lo = mid; else hi = mid;
    }
    const BatchItemDev &it = items[lo];
    const uint64_t j = g - it.group_begin;
    const uint64_t t0 = j * kGroupTiles;
    const uint64_t t1 = t0 + kGroupTiles < it.n_tiles ? t0 + kGroupTiles : it.n_tiles;
    sum_rows(rows + it.row_begin * 12u, t0, t1, 12, groups + g * 12u);
}

__global__ void batch_reduce_final_kernel(const BatchItemDev *items, const double *groups, double *out)
{
    const BatchItemDev &it = items[blockIdx.x];
    const uint64_t ng = (it.n_tiles + kGroupTiles - 1) / kGroupTiles;
    finish_groups(groups + it.group_begin * 12u, ng, 1, (double)it.n_paths, it.gamma_nan,
                  out + (uint64_t)blockIdx.x * 12u);
}


// ---------------------------------------------------------------------------
// Adjoint (reverse-mode pathwise) gradient of the price with respect to
// (S0, v0, kappa, theta, xi, rho, r), full truncation, FP32 paths, FP64 sums.
// The forward kernel prices and stores, per path, (X, V) every C = ceil(sqrt N)
// steps plus the payoff seed; the backward kernel rebuilds each C-step segment
// from its checkpoint (normals recomputed from the Philox counters) and sweeps
// the adjoints of the Milstein step (Sec. 2.4.2) in reverse:
//   X' = X + (r - V+/2) dt + u Za,   u = sqrt(V+ dt),   Z2 = rho Za + s Zb,
//   V' = V + kappa (theta - V+) dt + xi u Z2 + xi^2 dt (Z2^2 - 1) 1{V>0} / 4,
// with P = e^{-rT} phi(A), A = S0 e^{X_N} or (S0/M) sum_i e^{X(t_i)}.
// ---------------------------------------------------------------------------
constexpr int kAdjMaxSeg = 32;             // segment length C <= 32: n_steps <= 1024

struct AdjLaunch {
    PhiloxKey key;
    uint64_t n_paths, n_tiles;
    uint32_t N, C, n_seg;                   // steps, segment length, segments
    float2 *ckpt;                           // [n_seg][n_paths] (X, V) at each segment start
    float2 *seed;                           // [n_paths] (payoff, D phi'(A) / M or D phi'(S_T))
    double *rows;                           // tile rows
};

// Normals of step k of a path (words by parity, as in simulate()).
__device__ __forceinline__ void step_normals(PhiloxKey key, uint32_t plo, uint32_t phi, uint32_t k,
                                             float &za, float &zb)
{
    const uint4 w = philox4x32_10(make_uint4(k >> 1, plo, phi, 0u), key);
    if (k & 1u) box_muller(w.z, w.w, za, zb);
    else        box_muller(w.x, w.y, za, zb);
}

// One plain Milstein step (no tangents), full truncation: the forward of the adjoint.
__device__ __forceinline__ void plain_step(float &X, float &V, float za, float zb, const Coef<float> &k)
{
    const float Z2 = fmaf(k.rho, za, k.sq * zb);
    const bool pos = V > 0.0f;
    const float Vp = fmaxf(V, 0.0f);
    const float u = sqrt_approx(Vp * k.dt);
    X = fmaf(u, za, fmaf(fmaf(-0.5f, Vp, k.r), k.dt, X));
    const float z2m1 = fmaf(Z2, Z2, -1.0f);
    V = fmaf(pos ? k.c4 : 0.0f, z2m1, fmaf(k.xi * Z2, u, fmaf(-k.kdt, Vp, V + k.kth_dt)));
}

template <int MON>
__global__ void __launch_bounds__(kPathBlock) heston_adj_fwd_kernel(Coef<float> k, ContractSet<float> cs,
                                                                    AdjLaunch a)
{
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t tile = warp; tile < a.n_tiles; tile += n_warps) {
        float x[2];
#pragma unroll 1
        for (int q = 0; q < 2; ++q) {
            const uint64_t path = tile * kTile + (uint64_t)lane + 32u * (uint64_t)q;
            const bool keep = path < a.n_paths;
            const uint32_t plo = (uint32_t)path, phi = (uint32_t)(path >> 32);
            float X = 0.0f, V = k.v0, sA = 0.0f;
            for (uint32_t kk = 0; kk < a.N; ++kk) {
                if (keep && kk % a.C == 0) a.ckpt[(uint64_t)(kk / a.C) * a.n_paths + path] = make_float2(X, V);
                float za, zb;
                step_normals(a.key, plo, phi, kk, za, zb);
                plain_step(X, V, za, zb, k);
                if (MON != MON_NONE && (kk + 1) % cs.stride == 0) sA += exp_r(X);
            }
            const float A = MON == MON_NONE ? cs.S0 * exp_r(X) : cs.S0_over_M * sA;
            const float K = cs.K[0];
            float pay, slope;
            if (!cs.is_put[0]) { slope = A > K ? 1.0f : 0.0f; pay = A > K ? A - K : 0.0f; }
            else               { slope = A < K ? -1.0f : 0.0f; pay = A < K ? K - A : 0.0f; }
            const float scale = MON == MON_NONE ? 1.0f : 1.0f / (float)cs.M;
            if (keep) a.seed[path] = make_float2(cs.D * pay, cs.D * slope * scale);
            x[q] = keep ? cs.D * pay : 0.0f;
        }
        const float sx = warp_sum(x[0] + x[1]);
        const float sxx = warp_sum(x[0] * x[0] + x[1] * x[1]);
        if (lane == 0) { a.rows[tile * 2] = (double)sx; a.rows[tile * 2 + 1] = (double)sxx; }
    }
}

template <int MON>
__global__ void __launch_bounds__(kPathBlock) heston_adj_bwd_kernel(Coef<float> k, ContractSet<float> cs,
                                                                    AdjLaunch a, float T)
{
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const float inv_sq = 1.0f / k.sq;
    for (uint64_t tile = warp; tile < a.n_tiles; tile += n_warps) {
        float g[2][7];
#pragma unroll 1
        for (int q = 0; q < 2; ++q) {
            const uint64_t path = tile * kTile + (uint64_t)lane + 32u * (uint64_t)q;
            const bool keep = path < a.n_paths;
            const uint64_t pidx = keep ? path : 0;          // a valid index for the loads
            const uint32_t plo = (uint32_t)path, phi = (uint32_t)(path >> 32);
            const float2 sd = a.seed[pidx];
            const float aseed = sd.y;                       // dP/dS_i (Asian) or dP/dS_T
            float gS0 = 0.0f, gk = 0.0f, gth = 0.0f, gxi = 0.0f, grho = 0.0f, gr = 0.0f;
            float Xb = 0.0f, Vb = 0.0f;                     // adjoints of the state after the step
            float Xs[kAdjMaxSeg + 1], Vs[kAdjMaxSeg], Zas[kAdjMaxSeg], Zbs[kAdjMaxSeg];
            for (int seg = (int)a.n_seg - 1; seg >= 0; --seg) {
                const uint32_t k0 = (uint32_t)seg * a.C;
                const uint32_t k1 = min(a.N, k0 + a.C);
                const float2 c0 = a.ckpt[(uint64_t)seg * a.n_paths + pidx];
                float X = c0.x, V = c0.y;
                Xs[0] = X;
                for (uint32_t kk = k0; kk < k1; ++kk) {
                    float za, zb;
                    step_normals(a.key, plo, phi, kk, za, zb);
                    const uint32_t i = kk - k0;
                    Vs[i] = V; Zas[i] = za; Zbs[i] = zb;
                    plain_step(X, V, za, zb, k);
                    Xs[i + 1] = X;
                }
                for (int i = (int)(k1 - k0) - 1; i >= 0; --i) {
                    const uint32_t kp1 = k0 + (uint32_t)i + 1u;
                    // the payoff's dependence on X_{k+1}
                    const bool date = MON == MON_NONE ? kp1 == a.N : (kp1 % cs.stride == 0);
                    if (date) {
                        const float e = exp_r(Xs[i + 1]);
                        Xb = fmaf(aseed * cs.S0, e, Xb);
                        gS0 = fmaf(aseed, e, gS0);
                    }
                    const float za = Zas[i], zb = Zbs[i], Vk = Vs[i];
                    const float Z2 = fmaf(k.rho, za, k.sq * zb);
                    const bool pos = Vk > 0.0f;
                    const float Vp = fmaxf(Vk, 0.0f);
                    const float y = Vp * k.dt;
                    const float rs = rsqrt_approx(fmaxf(y, 1e-30f));
                    const float u = y * rs;
                    const float z2m1 = fmaf(Z2, Z2, -1.0f);
                    gr = fmaf(Xb, k.dt, gr);
                    float Vpb = fmaf(-0.5f * k.dt, Xb, -k.kdt * Vb);
                    const float ub = fmaf(za, Xb, k.xi * Z2 * Vb);
                    gk = fmaf(Vb, (k.theta - Vp) * k.dt, gk);
                    gth = fmaf(Vb, k.kdt, gth);
                    gxi = fmaf(Vb, fmaf(u, Z2, pos ? 0.5f * k.xi * k.dt * z2m1 : 0.0f), gxi);
                    const float Z2b = Vb * fmaf(k.xi, u, pos ? 0.5f * k.xi * k.xi * k.dt * Z2 : 0.0f);
                    grho = fmaf(Z2b, fmaf(-k.rho * inv_sq, zb, za), grho);
                    Vpb = fmaf(ub, 0.5f * k.dt * rs, Vpb);           // du/dV+ = dt / (2u); 0 where u = 0
                    Vb = pos ? Vb + Vpb : Vb;
                }
            }
            g[q][0] = gS0;
            g[q][1] = Vb;                                            // dP/dv0 = adjoint of V_0
            g[q][2] = gk;
            g[q][3] = gth;
            g[q][4] = gxi;
            g[q][5] = grho;
            g[q][6] = fmaf(-T, sd.x, gr);                            // plus the discount factor
            if (!keep) {
#pragma unroll
                for (int j = 0; j < 7; ++j) g[q][j] = 0.0f;
            }
        }
        double *row = a.rows + tile * 14u;
#pragma unroll
        for (int j = 0; j < 7; ++j) {
            const float sx = warp_sum(g[0][j] + g[1][j]);
            const float sxx = warp_sum(g[0][j] * g[0][j] + g[1][j] * g[1][j]);
            if (lane == j) row[j] = (double)sx;
            if (lane == 7 + j) row[7 + j] = (double)sxx;
        }
    }
}

// Reduce tile rows of `width` columns (sums then sums of squares, E = width/2
// estimators) in the fixed group order, writing mean[E] then se[E].
__global__ void reduce_generic_final_kernel(const double *group_sums, uint64_t n_groups, int E,
                                            double n_paths, double *out)
{
    __shared__ double tot[32];
    const int width = 2 * E;
    for (int col = threadIdx.x; col < width; col += blockDim.x) {
        double acc = 0.0;
        for (uint64_t g = 0; g < n_groups; ++g) acc += group_sums[g * width + col];
        tot[col] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const double mean = tot[e] / n_paths;
        const double var = (tot[E + e] - n_paths * mean * mean) / (n_paths - 1.0);
        out[e] = mean;
        out[E + e] = sqrt(var > 0.0 ? var / n_paths : 0.0);
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
    L.off_evoff = align256(L.off_T + D * 64 * sizeof(uint32_t));
    L.off_ev = align256(L.off_evoff + (N + 1) * sizeof(int32_t));
    L.total = align256(L.off_ev + n_ev * sizeof(BridgeOp));
    return L;
}

QmcTables qmc_tables_at(const void *base, const QmcLayout &L)
{
    const char *b = (const char *)base;
    return QmcTables{(const uint32_t *)(b + L.off_V), (const uint32_t *)(b + L.off_T),
                     (const BridgeOp *)(b + L.off_ev), (const int32_t *)(b + L.off_evoff)};
}

// QMC workspace: tile rows | replicate sums | U [tpr][D] | shifts [R][D].
struct QmcWs {
    size_t off_rows, off_rep, off_U, off_shift, total;
};

QmcWs qmc_ws_layout(uint32_t nc, uint64_t n_paths, uint32_t N, uint32_t R)
{
    const size_t w = 12u * nc * sizeof(double);
    const uint64_t tiles = tiles_for(n_paths);
    const uint64_t tpr = tiles / R;
    const size_t D = 2u * (size_t)N;
    QmcWs L;
    L.off_rows = 0;
    L.off_rep = align256(tiles * w);
    L.off_U = L.off_rep + align256((size_t)R * w);
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
    int dev = 0, n_sm = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPathBlock, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    uint64_t grid = pp.opt.grid_ctas ? pp.opt.grid_ctas
                                     : std::min<uint64_t>((a.n_tiles + 3) / 4, (uint64_t)n_sm * per_sm);
    if (grid < 1) grid = 1;
    const int block = pp.opt.block_threads ? (int)pp.opt.block_threads : kPathBlock;
    kern<<<(unsigned)grid, block, 0, st>>>(pp.kf, pp.csf, a);
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
    double *rep = (double *)(b + WL.off_rep);
    reduce_replicates_kernel<<<R, 128, 0, st>>>(a.tile_sums, a.tpr, width, rep);
    if (cudaGetLastError() != cudaSuccess) return HESTON_ERR_CUDA;
    reduce_final_qmc_kernel<<<1, 128, 0, st>>>(rep, R, pp.cs.n, (double)(n_paths / R),
                                               pp.gamma_nan ? 1 : 0, d_out);
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
    for (uint32_t d = 0; d < D; ++d)
        for (uint32_t p = 0; p < 64; ++p) {
            uint32_t x = 0;
            for (int b = 0; b < 6; ++b)
                if ((p >> b) & 1u) x ^= V[d * 32u + b];
            T[d * 64u + p] = x;
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
    batch_reduce_groups_kernel<<<(unsigned)plan->total_groups, 64, 0, st>>>(a.items, a.group_begin, n,
                                                                            a.rows, groups);
    if (cudaGetLastError() != cudaSuccess) return HESTON_ERR_CUDA;
    batch_reduce_final_kernel<<<n, 64, 0, st>>>(a.items, groups, d_out);
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
    L.C = (uint32_t)std::ceil(std::sqrt((double)N));
    if (L.C < 1) L.C = 1;
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
    if (backward) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, heston_adj_bwd_kernel<MON>, kPathBlock, 0);
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
                    void *ws, size_t ws_bytes, double *d_out)
{
    Prepared pp;
    int rc = validate_and_prepare(params, contract, 1, n_paths, N, opts, pp);
    if (rc < 0) return rc;
    if (pp.opt.prec != HESTON_FP32 || pp.opt.trunc != HESTON_TRUNC_FULL || pp.opt.rng != HESTON_RNG_PHILOX ||
        pp.opt.scheme != HESTON_SCHEME_MILSTEIN)
        return HESTON_ERR_UNSUPPORTED;
    const AdjLayout L = adj_layout(n_paths, N);
    if (L.C > (uint32_t)kAdjMaxSeg) return HESTON_ERR_UNSUPPORTED;
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
    cudaStream_t stream = nullptr;
    int n_sm = 0, per_sm = 0;
    // device buffers
    BatchItemDev *d_slots = nullptr;
    double *d_pool = nullptr, *d_groups = nullptr, *d_results = nullptr;
    uint64_t *d_wb[2] = {nullptr, nullptr}, *d_wt[2] = {nullptr, nullptr};
    uint32_t *d_wi[2] = {nullptr, nullptr};
    unsigned long long *d_counter = nullptr;
    // pinned host staging
    BatchItemDev *h_slots = nullptr;
    uint64_t *h_wb[2] = {nullptr, nullptr}, *h_wt[2] = {nullptr, nullptr};
    uint32_t *h_wi[2] = {nullptr, nullptr};
    double *h_results = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
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

// Retire the requests whose reduction ran in the round on buffer b.
void srv_retire(heston_server *s, int b)
{
    if (s->pending[b].empty()) return;
    const bool failed = cudaEventSynchronize(s->ev[b]) != cudaSuccess;
    const auto now = std::chrono::steady_clock::now();
    std::lock_guard<std::mutex> lock(s->mu);
    for (int slot : s->pending[b]) {
        heston_server::Req &r = s->slots[slot];
        heston_server::Done d;
        const bool gn = r.dev.gamma_nan != 0;
        fill_results(s->h_results + (size_t)slot * 12u, 1, r.dev.n_paths,
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
                                cudaMemcpyHostToDevice, s->stream);
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
            }
            const bool busy = !round_slots.empty() || !s->pending[0].empty() || !s->pending[1].empty();
            if (!busy) {
                if (s->stop && s->queue.empty() && s->order.empty()) break;
                s->cv_work.wait_for(lock, std::chrono::milliseconds(2));
                continue;
            }
        }
        if (!round_slots.empty()) {
            // buffer b was last used two rounds ago: its copies and kernels are done
            srv_retire(s, b);
            cudaEventSynchronize(s->ev[b]);
            const uint32_t n = (uint32_t)round_slots.size();
            uint64_t acc = 0;
            for (uint32_t p = 0; p < n; ++p) {
                heston_server::Req &r = s->slots[round_slots[p]];
                s->h_wb[b][p] = acc;
                s->h_wi[b][p] = (uint32_t)round_slots[p];
                s->h_wt[b][p] = r.next_tile;
                acc += round_tiles[p];
                r.next_tile += round_tiles[p];
                if (r.next_tile == r.tiles) finishing.push_back(round_slots[p]);
            }
            cudaMemcpyAsync(s->d_wb[b], s->h_wb[b], n * sizeof(uint64_t), cudaMemcpyHostToDevice, s->stream);
            cudaMemcpyAsync(s->d_wi[b], s->h_wi[b], n * sizeof(uint32_t), cudaMemcpyHostToDevice, s->stream);
            cudaMemcpyAsync(s->d_wt[b], s->h_wt[b], n * sizeof(uint64_t), cudaMemcpyHostToDevice, s->stream);
            cudaMemsetAsync(s->d_counter, 0, sizeof(unsigned long long), s->stream);
            BatchLaunch a;
            a.items = s->d_slots;
            a.work_begin = s->d_wb[b];
            a.work_item = s->d_wi[b];
            a.work_tile0 = s->d_wt[b];
            a.group_begin = nullptr;
            a.n_items = n;
            a.total_work = acc;
            a.counter = s->d_counter;
            a.status = nullptr;
            a.rows = s->d_pool;
            const uint64_t grid = std::min<uint64_t>((acc + 3) / 4, (uint64_t)s->n_sm * s->per_sm);
            if (s->cfg.trunc == HESTON_TRUNC_FULL)
                heston_batch_kernel<0><<<(unsigned)std::max<uint64_t>(grid, 1), kPathBlock, 0, s->stream>>>(a);
            else
                heston_batch_kernel<1><<<(unsigned)std::max<uint64_t>(grid, 1), kPathBlock, 0, s->stream>>>(a);
            for (int slot : finishing) {
                const heston_server::Req &r = s->slots[slot];
                const double *rows = s->d_pool + r.dev.row_begin * 12u;
                const uint64_t ng = groups_for(r.tiles);
                reduce_groups_kernel<<<(unsigned)ng, 64, 0, s->stream>>>(rows, r.tiles, 12, s->d_groups);
                reduce_final_kernel<<<1, 64, 0, s->stream>>>(s->d_groups, ng, 1, (double)r.dev.n_paths,
                                                             r.dev.gamma_nan, s->d_results + (size_t)slot * 12u);
                cudaMemcpyAsync(s->h_results + (size_t)slot * 12u, s->d_results + (size_t)slot * 12u,
                                12u * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
            }
            cudaEventRecord(s->ev[b], s->stream);
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
    cudaFree(s->d_slots); cudaFree(s->d_pool); cudaFree(s->d_groups); cudaFree(s->d_results);
    cudaFree(s->d_counter);
    for (int b = 0; b < 2; ++b) {
        cudaFree(s->d_wb[b]); cudaFree(s->d_wi[b]); cudaFree(s->d_wt[b]);
        cudaFreeHost(s->h_wb[b]); cudaFreeHost(s->h_wi[b]); cudaFreeHost(s->h_wt[b]);
        if (s->ev[b]) cudaEventDestroy(s->ev[b]);
    }
    cudaFreeHost(s->h_slots); cudaFreeHost(s->h_results);
    if (s->stream) cudaStreamDestroy(s->stream);
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
    if (cudaMallocAsync((void **)&buf, tb + wb + align256(ob), st) != cudaSuccess) {
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
    const AdjLayout L = adj_layout(n_paths, n_steps);
    if (L.C > (uint32_t)kAdjMaxSeg) return HESTON_ERR_UNSUPPORTED;
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
    e |= (int)cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    s->pool_bytes = cfg->memory_bytes / kPoolUnit * kPoolUnit;
    e |= (int)cudaMalloc((void **)&s->d_slots, S * sizeof(BatchItemDev));
    e |= (int)cudaMalloc((void **)&s->d_pool, s->pool_bytes);
    e |= (int)cudaMalloc((void **)&s->d_groups, (size_t)groups_for(s->pool_bytes / 96 + 1) * 12 * sizeof(double) + 256);
    e |= (int)cudaMalloc((void **)&s->d_results, (size_t)S * 12 * sizeof(double));
    e |= (int)cudaMalloc((void **)&s->d_counter, 256);
    e |= (int)cudaHostAlloc((void **)&s->h_slots, S * sizeof(BatchItemDev), cudaHostAllocDefault);
    e |= (int)cudaHostAlloc((void **)&s->h_results, (size_t)S * 12 * sizeof(double), cudaHostAllocDefault);
    for (int b = 0; b < 2; ++b) {
        e |= (int)cudaMalloc((void **)&s->d_wb[b], S * sizeof(uint64_t));
        e |= (int)cudaMalloc((void **)&s->d_wi[b], S * sizeof(uint32_t));
        e |= (int)cudaMalloc((void **)&s->d_wt[b], S * sizeof(uint64_t));
        e |= (int)cudaHostAlloc((void **)&s->h_wb[b], S * sizeof(uint64_t), cudaHostAllocDefault);
        e |= (int)cudaHostAlloc((void **)&s->h_wi[b], S * sizeof(uint32_t), cudaHostAllocDefault);
        e |= (int)cudaHostAlloc((void **)&s->h_wt[b], S * sizeof(uint64_t), cudaHostAllocDefault);
        e |= (int)cudaEventCreateWithFlags(&s->ev[b], cudaEventDisableTiming);
        cudaEventRecord(s->ev[b], s->stream);
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
    cudaStreamSynchronize(s->stream);
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
