/*
 * heston_oracle.c -- FP64 CPU oracle for Monte Carlo Heston pricing and
 * pathwise Greeks (arXiv 2309.10477).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file.  Only tests/, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or constant with
 * the CUDA path: the two sides are written independently and meet only on
 * the random-number contract (Philox4x32-10 + Box-Muller, implemented here
 * from their published definitions).
 *
 * What it computes, in the paper's order and notation:
 *   - Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers:
 *     As Easy as 1, 2, 3", SC'11), the counter-based generator standing in
 *     for the paper's in-kernel cuRAND draws (Sec. 3, "MGPU").
 *   - Box-Muller normals and the correlation step of the paper's Algorithm
 *     "Generation of two correlated Normal random variables" (Sec. 2.4.1).
 *   - The Milstein scheme for ln S and V under Heston (Sec. 2.4.2, the
 *     equations for ln S_{t+dt} and V_{t+dt}, and the Algorithm "Milstein
 *     approximation under Heston model"), with exactly N integer steps and
 *     either full truncation (Lord, Koekkoek, van Dijk 2010) or the paper's
 *     floor max(V, 0) after each update.
 *   - Two more schemes on the same normals: the Euler scheme of Sec. 2.4.1
 *     (the Milstein step without its xi^2 dt (Z^2 - 1) / 4 term; same
 *     truncation choices), and Andersen's quadratic-exponential (QE) scheme,
 *     which the paper names as the next method to try (Sec. 5), written from
 *     L. Andersen, "Simple and efficient simulation of the Heston stochastic
 *     volatility model", J. Comput. Finance 11(3), 2008 (Sec. 3.2.3 and the
 *     log-price step of its Sec. 4.2 with gamma1 = gamma2 = 1/2, no
 *     martingale correction).
 *   - The Monte Carlo estimator of the Algorithm "Monte Carlo option pricing
 *     estimation" (Sec. 2.5), extended to the pathwise Greeks of
 *     Eq. (euro_pw) and Eq. (asian_pw) (pathwise method, Sec. 2).  Asian Rho uses the
 *     derivative of the Asian payoff (the printed K*T prefactor is dropped;
 *     with one monitoring date it then reduces to the European Rho).
 *   - Gamma, Vega and Theta, which the paper only names (Sec. 2): Gamma by
 *     a pathwise / likelihood-ratio mix on the same paths, Vega = dV/dv0 and
 *     Theta = -dV/dT by pathwise tangent recursions.
 *
 * Parity pins for every function are in tests/test_oracle_*.py.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Inputs                                                              */
/* ------------------------------------------------------------------ */

/* Heston parameters, Eq. (heston_eq): dS = r S dt + sqrt(V) S dW1,
 * dV = kappa (theta - V) dt + xi sqrt(V) dW2, corr(dW1, dW2) = rho.
 * The paper writes sigma for the vol-of-vol; here it is xi. */
typedef struct {
    double S0, v0, kappa, theta, xi, rho, r;
} orc_params;

/* One contract.  payoff: 0 = European, 1 = arithmetic Asian.  is_put: 0/1.
 * n_monitor: Asian dates t_i = i*T/M, i = 1..M (0 means M = N). */
typedef struct {
    int32_t payoff;
    int32_t is_put;
    double K;
    double T;
    uint32_t n_monitor;
    uint32_t pad_;
} orc_contract;

enum { ORC_TRUNC_FULL = 0, ORC_TRUNC_FLOOR = 1 };
enum { ORC_SCHEME_MILSTEIN = 0, ORC_SCHEME_EULER = 1, ORC_SCHEME_QE = 2 };
/* QE switching level of psi = s^2 / m^2 (Andersen's suggested value). */
static const double ORC_QE_PSI_C = 1.5;

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11 paper, Sec. 4 "Philox")                        */
/* ------------------------------------------------------------------ */

/* Round multipliers and Weyl key increments of Philox4x32. */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {            /* key schedule: k_i = k_0 + i * W */
            k0 += ORC_PHILOX_W0;
            k1 += ORC_PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------ */
/* Random-number contract                                              */
/* ------------------------------------------------------------------ */
/* Path `path`, time step `step`: counter = (step / 2, path_lo, path_hi,
 * stream_tag), key = (seed_lo, seed_hi).  Words (x0, x1) feed the even step
 * and (x2, x3) the odd step.  Uniforms keep the top 24 bits:
 *   u1 = ((x >> 8) + 1) * 2^-24 in (0, 1],   u2 = (x >> 8) * 2^-24 in [0, 1).
 * Box-Muller: Za = sqrt(-2 ln u1) cos(2 pi u2), Zb = sqrt(-2 ln u1) sin(2 pi u2). */

static const double ORC_TWO_PI = 6.283185307179586476925286766559;

void orc_uniform_pair(uint64_t seed, uint64_t path, uint32_t step, uint32_t stream_tag,
                      double *u1, double *u2)
{
    uint32_t ctr[4] = { step / 2u, (uint32_t)path, (uint32_t)(path >> 32), stream_tag };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    uint32_t a = (step & 1u) ? x[2] : x[0];
    uint32_t b = (step & 1u) ? x[3] : x[1];
    *u1 = ldexp((double)((a >> 8) + 1u), -24);
    *u2 = ldexp((double)(b >> 8), -24);
}

void orc_normal_pair(uint64_t seed, uint64_t path, uint32_t step, uint32_t stream_tag,
                     double *za, double *zb)
{
    double u1, u2;
    orc_uniform_pair(seed, path, step, stream_tag, &u1, &u2);
    double rad = sqrt(-2.0 * log(u1));
    *za = rad * cos(ORC_TWO_PI * u2);
    *zb = rad * sin(ORC_TWO_PI * u2);
}

/* Fill Za[0..N), Zb[0..N) for one path. */
void orc_path_normals(uint64_t seed, uint64_t path, uint32_t n_steps, uint32_t stream_tag,
                      double *Za, double *Zb)
{
    for (uint32_t k = 0; k < n_steps; ++k)
        orc_normal_pair(seed, path, k, stream_tag, &Za[k], &Zb[k]);
}

/* ------------------------------------------------------------------ */
/* One path with tangents: Milstein (Sec. 2.4.2), Euler (Sec. 2.4.1), QE */
/* ------------------------------------------------------------------ */

/* Per-path record.  X = ln(S/S0); V = variance state; *_v = d/dv0 and
 * *_T = d/dT tangents (normals held fixed, N and M held fixed so that
 * dt = T/N and t_i = i*T/M move with T).  Asian sums run over the M
 * monitoring dates.  GE/QE: Gamma weights over all N steps; GA/QA: over
 * the steps before the first monitoring date. */
typedef struct {
    double X, V, X_v, V_v, X_T, V_T;
    double sumS, sumtS, sumS_Xv, sumS_XT;   /* sum S_ti, sum t_i S_ti, sum S_ti X_v(t_i), sum S_ti X_T(t_i) */
    double GE, QE, GA, QA;
    double minabsV;                         /* smallest distance to a branch decision (flip classification) */
} orc_path;

/* Number of doubles in orc_path, for the flat per-path dump. */
#define ORC_PATH_DOUBLES 15

/* Standard normal lower tail Phi(x), from the C library's erfc. */
static double orc_norm_cdf(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

/* One QE step of the variance (Andersen 2008, Sec. 3.2.3) with its v0- and
 * T-tangents.  Given V = V(t) >= 0, the exact conditional mean and variance
 * of the CIR process over dt are
 *   m  = theta + (V - theta) e^{-kappa dt},
 *   s2 = V xi^2 e^{-kappa dt} (1 - e^{-kappa dt}) / kappa
 *        + theta xi^2 (1 - e^{-kappa dt})^2 / (2 kappa),
 * and psi = s2 / m^2.  For psi <= psi_c the next value is a (b + Zv)^2 with
 *   b^2 = 2/psi - 1 + sqrt(2/psi) sqrt(2/psi - 1),  a = m / (1 + b^2);
 * otherwise it is 0 when Uv <= p and ln((1 - p) / (1 - Uv)) / beta above,
 *   p = (psi - 1) / (psi + 1),  beta = (1 - p) / m.
 * Zv = Za and Uv = Phi(Za): one uniform drives both branches (only one is
 * used per step).  *margin receives the distance, in variance units, of
 * this step from its branch decisions. */
static void orc_qe_variance(const orc_params *p, double dt, double ddt, double V, double V_v,
                            double V_T, double Za, double *Vn, double *Vn_v, double *Vn_T,
                            double *margin)
{
    const double kap = p->kappa, th = p->theta, xi2 = p->xi * p->xi;
    const double E = exp(-kap * dt);
    const double E_T = -kap * E * ddt;                         /* dE/dT */
    /* g = (1 - E) / kappa, with its kappa -> 0 limit dt; dg/dT = E / N. */
    const double g = kap > 0.0 ? -expm1(-kap * dt) / kap : dt;
    const double g_T = E * ddt;
    const double omE = kap > 0.0 ? -expm1(-kap * dt) : 0.0;    /* 1 - E */

    const double m = th + (V - th) * E;
    const double m_v = V_v * E;
    const double m_T = V_T * E + (V - th) * E_T;
    const double s2 = V * xi2 * E * g + 0.5 * th * xi2 * omE * g;
    const double s2_v = V_v * xi2 * E * g;
    const double s2_T = xi2 * (V_T * E * g + V * (E_T * g + E * g_T))
                        + 0.5 * th * xi2 * (-E_T * g + omE * g_T);
    const double psi = s2 / (m * m);
    const double psi_v = s2_v / (m * m) - 2.0 * s2 * m_v / (m * m * m);
    const double psi_T = s2_T / (m * m) - 2.0 * s2 * m_T / (m * m * m);
    double mg = m * fabs(psi - ORC_QE_PSI_C) / ORC_QE_PSI_C;

    if (psi <= ORC_QE_PSI_C) {
        /* quadratic branch */
        const double y = 2.0 / psi;
        const double y_v = -2.0 * psi_v / (psi * psi);
        const double y_T = -2.0 * psi_T / (psi * psi);
        const double root = sqrt(y) * sqrt(y - 1.0);
        const double b2 = y - 1.0 + root;
        const double db2_dy = 1.0 + (2.0 * y - 1.0) / (2.0 * root);
        const double b = sqrt(b2);
        const double a = m / (1.0 + b2);
        const double b2_v = db2_dy * y_v, b2_T = db2_dy * y_T;
        const double b_v = b2_v / (2.0 * b), b_T = b2_T / (2.0 * b);
        const double a_v = m_v / (1.0 + b2) - m * b2_v / ((1.0 + b2) * (1.0 + b2));
        const double a_T = m_T / (1.0 + b2) - m * b2_T / ((1.0 + b2) * (1.0 + b2));
        *Vn = a * (b + Za) * (b + Za);
        *Vn_v = a_v * (b + Za) * (b + Za) + 2.0 * a * (b + Za) * b_v;
        *Vn_T = a_T * (b + Za) * (b + Za) + 2.0 * a * (b + Za) * b_T;
    } else {
        /* exponential branch: Psi^{-1}(Uv) with the mass p at zero */
        const double pr = (psi - 1.0) / (psi + 1.0);
        const double pr_v = 2.0 * psi_v / ((psi + 1.0) * (psi + 1.0));
        const double pr_T = 2.0 * psi_T / ((psi + 1.0) * (psi + 1.0));
        const double beta = (1.0 - pr) / m;
        const double Uv = orc_norm_cdf(Za);
        const double one_m_U = orc_norm_cdf(-Za);              /* 1 - Uv without cancellation */
        const double dm = m * fabs(one_m_U - (1.0 - pr)) / (1.0 - pr);
        if (dm < mg) mg = dm;
        if (Uv <= pr) {
            *Vn = 0.0; *Vn_v = 0.0; *Vn_T = 0.0;
        } else {
            const double L = log((1.0 - pr) / one_m_U);
            *Vn = L / beta;
            /* V' = m L / (1 - p), L = ln(1 - p) - ln(1 - Uv) */
            *Vn_v = m_v * L / (1.0 - pr) + m * pr_v * (L - 1.0) / ((1.0 - pr) * (1.0 - pr));
            *Vn_T = m_T * L / (1.0 - pr) + m * pr_T * (L - 1.0) / ((1.0 - pr) * (1.0 - pr));
        }
    }
    *margin = mg;
}

/* Simulate one path from the given normals.  Za, Zb: independent N(0,1)
 * draws per step (Algorithm "Generation of two correlated Normal random
 * variables", step 1).  M = number of Asian dates (N % M == 0).
 * scheme: Milstein, Euler (trunc applies to both) or QE (trunc ignored:
 * its variance is never negative).  traj_X / traj_V, when non-NULL,
 * receive X_k, V_k for k = 0..N. */
void orc_scheme_path(const orc_params *p, double T, uint32_t N, uint32_t M, int trunc, int scheme,
                     const double *Za, const double *Zb, orc_path *out,
                     double *traj_X, double *traj_V)
{
    const double dt = T / (double)N;
    const double ddt = 1.0 / (double)N;            /* d(dt)/dT */
    const double sq = sqrt(1.0 - p->rho * p->rho);
    const uint32_t stride = N / M;                  /* steps between monitoring dates */
    /* the Milstein term xi^2 dt (Z2^2 - 1) / 4 is what Euler leaves out */
    const double mil_on = scheme == ORC_SCHEME_MILSTEIN ? 1.0 : 0.0;

    double X = 0.0, V = p->v0;
    double X_v = 0.0, V_v = 1.0;                    /* dX/dv0, dV/dv0 at t = 0 */
    double X_T = 0.0, V_T = 0.0;                    /* dX/dT,  dV/dT  at t = 0 */
    double sumS = 0.0, sumtS = 0.0, sumS_Xv = 0.0, sumS_XT = 0.0;
    double GE = 0.0, QE = 0.0, GA = 0.0, QA = 0.0;
    double minabsV = scheme == ORC_SCHEME_QE ? INFINITY : fabs(V);

    if (traj_X) { traj_X[0] = X; traj_V[0] = V; }

    for (uint32_t k = 0; k < N; ++k) {
        double Xn, Xn_v, Xn_T, Vn, Vn_v, Vn_T;
        double branch;              /* distance from the branch decision of this step */
        if (scheme == ORC_SCHEME_QE) {
            /* Variance first (Zv = Za), then ln S from both variances with
             * the independent normal Zb (Andersen 2008, Sec. 4.2):
             * ln S' = ln S + r dt + K0 + K1 V + K2 V' + sqrt(K3 V + K4 V') Zb,
             * K0 = -rho kappa theta dt / xi, K1 = dt/2 (kappa rho / xi - 1/2) - rho / xi,
             * K2 = dt/2 (kappa rho / xi - 1/2) + rho / xi, K3 = K4 = dt/2 (1 - rho^2). */
            orc_qe_variance(p, dt, ddt, V, V_v, V_T, Za[k], &Vn, &Vn_v, &Vn_T, &branch);
            const double K0 = -p->rho * p->kappa * p->theta * dt / p->xi;
            const double K0_T = -p->rho * p->kappa * p->theta * ddt / p->xi;
            const double K1 = 0.5 * dt * (p->kappa * p->rho / p->xi - 0.5) - p->rho / p->xi;
            const double K2 = 0.5 * dt * (p->kappa * p->rho / p->xi - 0.5) + p->rho / p->xi;
            const double K12_T = 0.5 * ddt * (p->kappa * p->rho / p->xi - 0.5);
            const double K3 = 0.5 * dt * (1.0 - p->rho * p->rho);
            const double K3_T = 0.5 * ddt * (1.0 - p->rho * p->rho);
            const double sig = sqrt(K3 * (V + Vn));
            Xn = X + p->r * dt + K0 + K1 * V + K2 * Vn + sig * Zb[k];
            Xn_v = X_v + K1 * V_v + K2 * Vn_v
                   + (sig > 0.0 ? K3 * (V_v + Vn_v) / (2.0 * sig) : 0.0) * Zb[k];
            Xn_T = X_T + p->r * ddt + K0_T + K12_T * V + K1 * V_T + K12_T * Vn + K2 * Vn_T
                   + (sig > 0.0 ? (K3_T * (V + Vn) + K3 * (V_T + Vn_T)) / (2.0 * sig) : 0.0) * Zb[k];
            /* Gamma weights: given the variance path, the ln S noise of the
             * step is sq * ut * Zb with ut = sqrt(dt (V + V') / 2), and Zb
             * does not move the variance. */
            const double ut = sqrt(0.5 * dt * (V + Vn));
            GE += ut * Zb[k];
            QE += 0.5 * dt * (V + Vn);
            if (k < stride) { GA += ut * Zb[k]; QA += 0.5 * dt * (V + Vn); }
        } else {
            /* Correlation step: Z1 = Za, Z2 = rho Z1 + sqrt(1 - rho^2) Zb.
             * W is the component of Z1 orthogonal to Z2 (used by Gamma):
             * Z1 = rho Z2 + sqrt(1 - rho^2) W. */
            const double Z1 = Za[k];
            const double Z2 = p->rho * Z1 + sq * Zb[k];
            const double W = sq * Za[k] - p->rho * Zb[k];

            /* Positive part used by drift and diffusion.  Under the paper's
             * floor V is never negative, so Vp == V there. */
            const int pos = V > 0.0;
            const double Vp = pos ? V : 0.0;
            const double Vp_v = pos ? V_v : 0.0;
            const double Vp_T = pos ? V_T : 0.0;
            const double u = sqrt(Vp * dt);              /* sqrt(V dt) */
            /* d u = d(Vp dt) / (2 u); zero where u == 0. */
            const double u_v = (u > 0.0) ? (Vp_v * dt) / (2.0 * u) : 0.0;
            const double u_T = (u > 0.0) ? (Vp_T * dt + Vp * ddt) / (2.0 * u) : 0.0;

            /* Gamma weights accumulate before this step's update. */
            GE += u * W;
            QE += Vp * dt;
            if (k < stride) { GA += u * W; QA += Vp * dt; }

            /* ln S step with the pre-update variance:
             * ln S_{t+dt} = ln S_t + (r - V/2) dt + sqrt(V dt) Z1. */
            Xn = X + (p->r - 0.5 * Vp) * dt + u * Z1;
            Xn_v = X_v - 0.5 * Vp_v * dt + u_v * Z1;
            Xn_T = X_T + (p->r - 0.5 * Vp) * ddt - 0.5 * Vp_T * dt + u_T * Z1;

            /* V step: V + kappa (theta - V) dt + xi sqrt(V dt) Z2 [+ xi^2 dt (Z2^2 - 1) / 4]. */
            if (trunc == ORC_TRUNC_FULL) {
                /* Full truncation: the state keeps its sign; drift, diffusion and
                 * the Milstein term (which comes from the diffusion) see V+. */
                const double mil = pos ? mil_on : 0.0;
                Vn = V + p->kappa * (p->theta - Vp) * dt + p->xi * u * Z2
                     + 0.25 * p->xi * p->xi * dt * (Z2 * Z2 - 1.0) * mil;
                Vn_v = V_v - p->kappa * Vp_v * dt + p->xi * u_v * Z2;
                Vn_T = V_T + p->kappa * (p->theta - Vp) * ddt - p->kappa * Vp_T * dt
                       + p->xi * u_T * Z2 + 0.25 * p->xi * p->xi * ddt * (Z2 * Z2 - 1.0) * mil;
                branch = fabs(Vn);
            } else {
                /* The paper's scheme as printed: update with V, then V = max(V, 0). */
                const double Vt = V + p->kappa * (p->theta - V) * dt + p->xi * u * Z2
                                  + 0.25 * p->xi * p->xi * dt * (Z2 * Z2 - 1.0) * mil_on;
                const double Vt_v = V_v - p->kappa * V_v * dt + p->xi * u_v * Z2;
                const double Vt_T = V_T + p->kappa * (p->theta - V) * ddt - p->kappa * V_T * dt
                                    + p->xi * u_T * Z2
                                    + 0.25 * p->xi * p->xi * ddt * (Z2 * Z2 - 1.0) * mil_on;
                const int keep = Vt > 0.0;
                Vn = keep ? Vt : 0.0;
                Vn_v = keep ? Vt_v : 0.0;
                Vn_T = keep ? Vt_T : 0.0;
                branch = fabs(Vt);
            }
        }

        X = Xn; X_v = Xn_v; X_T = Xn_T;
        V = Vn; V_v = Vn_v; V_T = Vn_T;
        if (branch < minabsV) minabsV = branch;
        if (traj_X) { traj_X[k + 1] = X; traj_V[k + 1] = V; }

        /* Asian monitoring date t_i = (k+1) dt when (k+1) is a multiple of the stride. */
        if ((k + 1) % stride == 0) {
            const double S = p->S0 * exp(X);
            const double t = (double)(k + 1) * dt;
            sumS += S;
            sumtS += t * S;
            sumS_Xv += S * X_v;
            sumS_XT += S * X_T;
        }
    }

    out->X = X; out->V = V; out->X_v = X_v; out->V_v = V_v; out->X_T = X_T; out->V_T = V_T;
    out->sumS = sumS; out->sumtS = sumtS; out->sumS_Xv = sumS_Xv; out->sumS_XT = sumS_XT;
    out->GE = GE; out->QE = QE; out->GA = GA; out->QA = QA;
    out->minabsV = minabsV;
}

/* Scheme arguments a driver accepts: QE needs kappa, theta, xi > 0 (its
 * moments divide by kappa and xi, and m = 0 would make psi undefined). */
static int orc_scheme_ok(const orc_params *p, int trunc, int scheme)
{
    if (trunc != ORC_TRUNC_FULL && trunc != ORC_TRUNC_FLOOR) return 0;
    if (scheme == ORC_SCHEME_MILSTEIN || scheme == ORC_SCHEME_EULER) return 1;
    if (scheme != ORC_SCHEME_QE) return 0;
    return p->kappa > 0.0 && p->theta > 0.0 && p->xi > 0.0;
}

/* ------------------------------------------------------------------ */
/* Per-path estimators (Eq. euro_pw, Eq. asian_pw, plus Gamma/Vega/Theta) */
/* ------------------------------------------------------------------ */

/* est[0..5] = price, delta, gamma, vega (d/dv0), rho, theta (-d/dT), all
 * discounted, for one path.  Call formulas follow the paper; puts mirror
 * the indicator (d (K - A)+ / dA = -1{A < K}). */
void orc_estimators(const orc_params *p, const orc_contract *c, uint32_t N,
                    const orc_path *w, double est[6])
{
    const double T = c->T, K = c->K, S0 = p->S0, r = p->r;
    const double D = exp(-r * T);
    const double sq = sqrt(1.0 - p->rho * p->rho);
    const uint32_t M = c->n_monitor ? c->n_monitor : N;

    if (c->payoff == 0) {
        /* European: A = S_T; Gamma weight over all N steps. */
        const double ST = S0 * exp(w->X);
        const double lr = w->GE / (sq * w->QE);          /* S0 * d ln p / d S0 */
        if (!c->is_put) {
            const double ind = ST > K ? 1.0 : 0.0;
            est[0] = D * (ST > K ? ST - K : 0.0);
            est[1] = D * (ST / S0) * ind;                               /* Eq. euro_pw, Delta */
            est[2] = D * ind * (ST / (S0 * S0)) * (lr - 1.0);
            est[3] = D * ind * ST * w->X_v;
            est[4] = D * K * T * ind;                                   /* Eq. euro_pw, Rho */
            est[5] = r * est[0] - D * ind * ST * w->X_T;
        } else {
            const double ind = ST < K ? 1.0 : 0.0;
            est[0] = D * (ST < K ? K - ST : 0.0);
            est[1] = -D * (ST / S0) * ind;
            est[2] = -D * ind * (ST / (S0 * S0)) * (lr - 1.0);
            est[3] = -D * ind * ST * w->X_v;
            est[4] = -D * K * T * ind;
            est[5] = r * est[0] + D * ind * ST * w->X_T;
        }
    } else {
        /* Arithmetic Asian: Sbar = (1/M) sum S_ti; Gamma weight over the
         * steps before the first date. */
        const double Sbar = w->sumS / (double)M;
        const double tSbar = w->sumtS / (double)M;       /* (1/M) sum t_i S_ti = d Sbar / dr */
        const double dSbar_v = w->sumS_Xv / (double)M;
        const double dSbar_T = w->sumS_XT / (double)M;
        const double lr = w->GA / (sq * w->QA);
        if (!c->is_put) {
            const double ind = Sbar > K ? 1.0 : 0.0;
            est[0] = D * (Sbar > K ? Sbar - K : 0.0);
            est[1] = D * (Sbar / S0) * ind;                             /* Eq. asian_pw, Delta */
            est[2] = D * ind * (Sbar / (S0 * S0)) * (lr - 1.0);
            est[3] = D * ind * dSbar_v;
            est[4] = D * ind * (tSbar - T * (Sbar - K));                /* Eq. asian_pw, Rho (corrected) */
            est[5] = r * est[0] - D * ind * dSbar_T;
        } else {
            const double ind = Sbar < K ? 1.0 : 0.0;
            est[0] = D * (Sbar < K ? K - Sbar : 0.0);
            est[1] = -D * (Sbar / S0) * ind;
            est[2] = -D * ind * (Sbar / (S0 * S0)) * (lr - 1.0);
            est[3] = -D * ind * dSbar_v;
            est[4] = -D * ind * (tSbar + T * (K - Sbar));
            est[5] = r * est[0] + D * ind * dSbar_T;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Monte Carlo driver (Algorithm "Monte Carlo option pricing estimation") */
/* ------------------------------------------------------------------ */

/* Paths are grouped in chunks of ORC_CHUNK consecutive indices.  Each chunk
 * sums its paths in index order; chunk sums are added in chunk order.  The
 * result is therefore the same for any thread count. */
#define ORC_CHUNK 4096

/* Simulate paths [path_begin, path_begin + n_paths) with Philox normals and
 * return, for every contract c and estimator e, sum[c*6+e] = sum_x and
 * sumsq[c*6+e] = sum_x^2 over the paths.  All contracts must share T (they
 * share the paths) and all Asian contracts must share M.
 * Returns 0, or -1 on invalid input. */
/* Sensitivity probe support: move each normal of step k of a path by
 * (eps_abs + eps_rel R) (2U - 1), R = sqrt(Za^2 + Zb^2), with U uniform on
 * [0, 1) from Philox4x32-10 (key pert_seed, counter (k / 2, path_lo,
 * path_hi, 7); words 0-1 for even k, 2-3 for odd k; U = (w >> 8) 2^-24). */
static void orc_perturb_normals(uint64_t pert_seed, uint64_t path, uint32_t N, double eps_abs,
                                double eps_rel, double *Za, double *Zb)
{
    const uint32_t key[2] = { (uint32_t)pert_seed, (uint32_t)(pert_seed >> 32) };
    uint32_t x[4] = { 0, 0, 0, 0 };
    for (uint32_t k = 0; k < N; ++k) {
        if ((k & 1u) == 0) {
            const uint32_t ctr[4] = { k / 2u, (uint32_t)path, (uint32_t)(path >> 32), 7u };
            orc_philox4x32_10(ctr, key, x);
        }
        const uint32_t wa = (k & 1u) ? x[2] : x[0], wb = (k & 1u) ? x[3] : x[1];
        const double bound = eps_abs + eps_rel * sqrt(Za[k] * Za[k] + Zb[k] * Zb[k]);
        Za[k] += bound * (2.0 * ldexp((double)(wa >> 8), -24) - 1.0);
        Zb[k] += bound * (2.0 * ldexp((double)(wb >> 8), -24) - 1.0);
    }
}

static int orc_mc_sums_impl(const orc_params *p, const orc_contract *contracts, uint32_t n_contracts,
                            uint64_t path_begin, uint64_t n_paths, uint32_t N, uint64_t seed, int trunc,
                            int scheme, int n_threads, double eps_abs, double eps_rel,
                            uint64_t pert_seed, double *sum, double *sumsq);

int orc_mc_sums(const orc_params *p, const orc_contract *contracts, uint32_t n_contracts,
                uint64_t path_begin, uint64_t n_paths, uint32_t N, uint64_t seed, int trunc,
                int scheme, int n_threads, double *sum, double *sumsq)
{
    return orc_mc_sums_impl(p, contracts, n_contracts, path_begin, n_paths, N, seed, trunc, scheme,
                            n_threads, 0.0, 0.0, 0u, sum, sumsq);
}

/* orc_mc_sums with every normal perturbed as in orc_perturb_normals: how far
 * the estimates move under perturbations of a given size (the conditioning
 * of an estimate for a path computed at lower precision).  Test support. */
int orc_mc_sums_perturbed(const orc_params *p, const orc_contract *contracts, uint32_t n_contracts,
                          uint64_t path_begin, uint64_t n_paths, uint32_t N, uint64_t seed, int trunc,
                          int scheme, int n_threads, double eps_abs, double eps_rel,
                          uint64_t pert_seed, double *sum, double *sumsq)
{
    if (!(eps_abs >= 0.0) || !(eps_rel >= 0.0)) return -1;
    return orc_mc_sums_impl(p, contracts, n_contracts, path_begin, n_paths, N, seed, trunc, scheme,
                            n_threads, eps_abs, eps_rel, pert_seed, sum, sumsq);
}

static int orc_mc_sums_impl(const orc_params *p, const orc_contract *contracts, uint32_t n_contracts,
                            uint64_t path_begin, uint64_t n_paths, uint32_t N, uint64_t seed, int trunc,
                            int scheme, int n_threads, double eps_abs, double eps_rel,
                            uint64_t pert_seed, double *sum, double *sumsq)
{
    if (n_contracts == 0 || N == 0 || !orc_scheme_ok(p, trunc, scheme)) return -1;
    const double T = contracts[0].T;
    uint32_t M = N;
    for (uint32_t c = 0; c < n_contracts; ++c) {
        if (contracts[c].T != T) return -1;
        if (contracts[c].payoff == 1) {
            uint32_t Mc = contracts[c].n_monitor ? contracts[c].n_monitor : N;
            if (N % Mc != 0) return -1;
            M = Mc;
        }
    }
    const uint32_t E = 6u * n_contracts;
    const uint64_t n_chunks = (n_paths + ORC_CHUNK - 1) / ORC_CHUNK;
    double *csum = (double *)calloc((size_t)n_chunks * E * 2, sizeof(double));
    if (!csum) return -1;

#ifdef _OPENMP
    const int threads_before = omp_get_max_threads();
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel
#endif
    {
        double *Za = (double *)malloc(sizeof(double) * N);
        double *Zb = (double *)malloc(sizeof(double) * N);
        double est[6];
        orc_path w;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t ch = 0; ch < (int64_t)n_chunks; ++ch) {
            double *s = csum + (size_t)ch * E * 2;
            uint64_t lo = (uint64_t)ch * ORC_CHUNK;
            uint64_t hi = lo + ORC_CHUNK < n_paths ? lo + ORC_CHUNK : n_paths;
            for (uint64_t i = lo; i < hi; ++i) {
                orc_path_normals(seed, path_begin + i, N, 0u, Za, Zb);
                if (eps_abs > 0.0 || eps_rel > 0.0)
                    orc_perturb_normals(pert_seed, path_begin + i, N, eps_abs, eps_rel, Za, Zb);
                orc_scheme_path(p, T, N, M, trunc, scheme, Za, Zb, &w, NULL, NULL);
                for (uint32_t c = 0; c < n_contracts; ++c) {
                    orc_estimators(p, &contracts[c], N, &w, est);
                    for (int e = 0; e < 6; ++e) {
                        s[c * 6 + e] += est[e];
                        s[E + c * 6 + e] += est[e] * est[e];
                    }
                }
            }
        }
        free(Za);
        free(Zb);
    }

#ifdef _OPENMP
    omp_set_num_threads(threads_before);      /* n_threads applies to this call only */
#endif
    for (uint32_t e = 0; e < E; ++e) { sum[e] = 0.0; sumsq[e] = 0.0; }
    for (uint64_t ch = 0; ch < n_chunks; ++ch) {
        const double *s = csum + (size_t)ch * E * 2;
        for (uint32_t e = 0; e < E; ++e) { sum[e] += s[e]; sumsq[e] += s[E + e]; }
    }
    free(csum);
    return 0;
}

/* Per-path dump for a list of path indices: rec[i*ORC_PATH_DOUBLES ...] is
 * the orc_path record and est[i*6*n_contracts ...] the estimators. */
int orc_debug_paths(const orc_params *p, const orc_contract *contracts, uint32_t n_contracts,
                    const uint64_t *paths, uint64_t count, uint32_t N, uint64_t seed, int trunc,
                    int scheme, double *rec, double *est)
{
    if (n_contracts == 0 || N == 0 || !orc_scheme_ok(p, trunc, scheme)) return -1;
    const double T = contracts[0].T;
    uint32_t M = N;
    for (uint32_t c = 0; c < n_contracts; ++c) {
        if (contracts[c].T != T) return -1;
        if (contracts[c].payoff == 1) {
            uint32_t Mc = contracts[c].n_monitor ? contracts[c].n_monitor : N;
            if (N % Mc != 0) return -1;
            M = Mc;
        }
    }
    double *Za = (double *)malloc(sizeof(double) * N);
    double *Zb = (double *)malloc(sizeof(double) * N);
    for (uint64_t i = 0; i < count; ++i) {
        orc_path w;
        orc_path_normals(seed, paths[i], N, 0u, Za, Zb);
        orc_scheme_path(p, T, N, M, trunc, scheme, Za, Zb, &w, NULL, NULL);
        memcpy(rec + i * ORC_PATH_DOUBLES, &w, sizeof(double) * ORC_PATH_DOUBLES);
        for (uint32_t c = 0; c < n_contracts; ++c)
            orc_estimators(p, &contracts[c], N, &w, est + (i * n_contracts + c) * 6);
    }
    free(Za);
    free(Zb);
    return 0;
}

/* Single path from caller-supplied normals, with the full trajectory. */
int orc_path_from_normals(const orc_params *p, const orc_contract *contracts, uint32_t n_contracts,
                          uint32_t N, int trunc, int scheme, const double *Za, const double *Zb,
                          double *rec, double *est, double *traj_X, double *traj_V)
{
    if (n_contracts == 0 || N == 0 || !orc_scheme_ok(p, trunc, scheme)) return -1;
    uint32_t M = N;
    for (uint32_t c = 0; c < n_contracts; ++c)
        if (contracts[c].payoff == 1 && contracts[c].n_monitor) M = contracts[c].n_monitor;
    if (N % M != 0) return -1;
    orc_path w;
    orc_scheme_path(p, contracts[0].T, N, M, trunc, scheme, Za, Zb, &w, traj_X, traj_V);
    memcpy(rec, &w, sizeof(double) * ORC_PATH_DOUBLES);
    for (uint32_t c = 0; c < n_contracts; ++c)
        orc_estimators(p, &contracts[c], N, &w, est + c * 6);
    return 0;
}

/* Many paths from caller-supplied normals: Za, Zb are (n_paths x N) row-major;
 * rec receives n_paths x ORC_PATH_DOUBLES and est n_paths x n_contracts x 6. */
int orc_paths_from_normals(const orc_params *p, const orc_contract *contracts, uint32_t n_contracts,
                           uint32_t N, int trunc, int scheme, uint64_t n_paths, const double *Za,
                           const double *Zb, double *rec, double *est)
{
    if (n_contracts == 0 || N == 0 || !orc_scheme_ok(p, trunc, scheme)) return -1;
    uint32_t M = N;
    for (uint32_t c = 0; c < n_contracts; ++c) {
        if (contracts[c].T != contracts[0].T) return -1;
        if (contracts[c].payoff == 1 && contracts[c].n_monitor) M = contracts[c].n_monitor;
    }
    if (N % M != 0) return -1;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < (int64_t)n_paths; ++i) {
        orc_path w;
        orc_scheme_path(p, contracts[0].T, N, M, trunc, scheme, Za + (size_t)i * N,
                        Zb + (size_t)i * N, &w, NULL, NULL);
        memcpy(rec + (size_t)i * ORC_PATH_DOUBLES, &w, sizeof(double) * ORC_PATH_DOUBLES);
        for (uint32_t c = 0; c < n_contracts; ++c)
            orc_estimators(p, &contracts[c], N, &w, est + ((size_t)i * n_contracts + c) * 6);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Parameter gradient of the discounted payoff (forward-mode tangents)  */
/* ------------------------------------------------------------------ */

/* For one path from given normals: the discounted payoff P and its
 * derivatives with respect to (S0, v0, kappa, theta, xi, rho, r), full
 * truncation.  Each parameter carries its own tangent (dX, dV) through the
 * Milstein recursion of Sec. 2.4.2; the payoff (Eq. euro_pw / asian_pw
 * setting) is D phi(A) with A = S_T or Sbar and D = e^{-rT}. */
void orc_path_gradient(const orc_params *p, const orc_contract *c, uint32_t N,
                       const double *Za, const double *Zb, double *pay, double grad[7])
{
    const double T = c->T, dt = T / (double)N;
    const double sq = sqrt(1.0 - p->rho * p->rho);
    const uint32_t M = c->n_monitor ? c->n_monitor : N;
    const uint32_t stride = N / M;
    /* tangent index: 0 S0, 1 v0, 2 kappa, 3 theta, 4 xi, 5 rho, 6 r */
    double X = 0.0, V = p->v0, dX[7] = {0}, dV[7] = {0};
    dV[1] = 1.0;
    double A = 0.0, dA[7] = {0};          /* sum of e^{X} over the dates and its tangents */
    for (uint32_t k = 0; k < N; ++k) {
        const double za = Za[k], zb = Zb[k];
        const double Z2 = p->rho * za + sq * zb;
        const int pos = V > 0.0;
        const double Vp = pos ? V : 0.0;
        const double u = sqrt(Vp * dt);
        const double mil = pos ? 1.0 : 0.0;
        double nX[7], nV[7];
        for (int i = 0; i < 7; ++i) {
            const double dZ2 = (i == 5) ? za - (p->rho / sq) * zb : 0.0;
            const double dVp = pos ? dV[i] : 0.0;
            const double du = (u > 0.0) ? dVp * dt / (2.0 * u) : 0.0;
            const double dr = (i == 6) ? 1.0 : 0.0, dk = (i == 2) ? 1.0 : 0.0;
            const double dth = (i == 3) ? 1.0 : 0.0, dxi = (i == 4) ? 1.0 : 0.0;
            nX[i] = dX[i] + dr * dt - 0.5 * dVp * dt + du * za;
            nV[i] = dV[i] + dk * (p->theta - Vp) * dt + p->kappa * (dth - dVp) * dt
                    + dxi * u * Z2 + p->xi * du * Z2 + p->xi * u * dZ2
                    + (0.5 * p->xi * dxi * dt * (Z2 * Z2 - 1.0) + 0.5 * p->xi * p->xi * dt * Z2 * dZ2) * mil;
        }
        X = X + (p->r - 0.5 * Vp) * dt + u * za;
        V = V + p->kappa * (p->theta - Vp) * dt + p->xi * u * Z2
            + 0.25 * p->xi * p->xi * dt * (Z2 * Z2 - 1.0) * mil;
        for (int i = 0; i < 7; ++i) { dX[i] = nX[i]; dV[i] = nV[i]; }
        if (c->payoff == 1 && (k + 1) % stride == 0) {
            const double e = exp(X);
            A += e;
            for (int i = 0; i < 7; ++i) dA[i] += e * dX[i];
        }
    }
    const double D = exp(-p->r * T);
    double Aval, dAval[7];
    if (c->payoff == 0) {
        const double e = exp(X);
        Aval = p->S0 * e;
        for (int i = 0; i < 7; ++i) dAval[i] = p->S0 * e * dX[i];
    } else {
        Aval = p->S0 * A / (double)M;
        for (int i = 0; i < 7; ++i) dAval[i] = p->S0 * dA[i] / (double)M;
    }
    dAval[0] += Aval / p->S0;            /* A is proportional to S0 */
    double phi, slope;
    if (!c->is_put) { phi = Aval > c->K ? Aval - c->K : 0.0; slope = Aval > c->K ? 1.0 : 0.0; }
    else            { phi = Aval < c->K ? c->K - Aval : 0.0; slope = Aval < c->K ? -1.0 : 0.0; }
    *pay = D * phi;
    for (int i = 0; i < 7; ++i) grad[i] = D * slope * dAval[i];
    grad[6] += -T * D * phi;             /* discount factor */
}

/* Price and gradient estimates over paths [0, n) with Philox normals:
 * mean[8] (price, then the 7 derivatives) and se[8]. */
int orc_mc_gradient(const orc_params *p, const orc_contract *c, uint64_t n_paths, uint32_t N,
                    uint64_t seed, double *mean, double *se)
{
    if (N == 0 || n_paths < 2) return -1;
    const uint32_t M = c->n_monitor ? c->n_monitor : N;
    if (N % M) return -1;
    const uint64_t n_chunks = (n_paths + ORC_CHUNK - 1) / ORC_CHUNK;
    double *cs = (double *)calloc((size_t)n_chunks * 16, sizeof(double));
    if (!cs) return -1;
#ifdef _OPENMP
#pragma omp parallel
#endif
    {
        double *Za = (double *)malloc(sizeof(double) * N), *Zb = (double *)malloc(sizeof(double) * N);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t ch = 0; ch < (int64_t)n_chunks; ++ch) {
            double *s = cs + (size_t)ch * 16;
            const uint64_t lo = (uint64_t)ch * ORC_CHUNK;
            const uint64_t hi = lo + ORC_CHUNK < n_paths ? lo + ORC_CHUNK : n_paths;
            for (uint64_t i = lo; i < hi; ++i) {
                double pay, g[7];
                orc_path_normals(seed, i, N, 0u, Za, Zb);
                orc_path_gradient(p, c, N, Za, Zb, &pay, g);
                s[0] += pay; s[8] += pay * pay;
                for (int j = 0; j < 7; ++j) { s[1 + j] += g[j]; s[9 + j] += g[j] * g[j]; }
            }
        }
        free(Za);
        free(Zb);
    }
    double tot[16] = {0};
    for (uint64_t ch = 0; ch < n_chunks; ++ch)
        for (int j = 0; j < 16; ++j) tot[j] += cs[(size_t)ch * 16 + j];
    free(cs);
    const double n = (double)n_paths;
    for (int j = 0; j < 8; ++j) {
        mean[j] = tot[j] / n;
        const double var = (tot[8 + j] - n * mean[j] * mean[j]) / (n - 1.0);
        se[j] = sqrt(var > 0.0 ? var / n : 0.0);
    }
    return 0;
}

/* Per-path gradients from given normals (n_paths x N each, row-major),
 * test support: out[i*8 ...] = (payoff, 7 derivatives). */
int orc_gradients_from_normals(const orc_params *p, const orc_contract *c, uint32_t N,
                               uint64_t n_paths, const double *Za, const double *Zb, double *out)
{
    if (N == 0) return -1;
    const uint32_t M = c->n_monitor ? c->n_monitor : N;
    if (N % M) return -1;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < (int64_t)n_paths; ++i)
        orc_path_gradient(p, c, N, Za + (size_t)i * N, Zb + (size_t)i * N, out + (size_t)i * 8,
                          out + (size_t)i * 8 + 1);
    return 0;
}

/* Per-path gradients for a list of paths (test support): out[i*8 ...] =
 * (payoff, 7 derivatives). */
int orc_debug_gradients(const orc_params *p, const orc_contract *c, const uint64_t *paths,
                        uint64_t count, uint32_t N, uint64_t seed, double *out)
{
    double *Za = (double *)malloc(sizeof(double) * N), *Zb = (double *)malloc(sizeof(double) * N);
    for (uint64_t i = 0; i < count; ++i) {
        orc_path_normals(seed, paths[i], N, 0u, Za, Zb);
        orc_path_gradient(p, c, N, Za, Zb, out + i * 8, out + i * 8 + 1);
    }
    free(Za);
    free(Zb);
    return 0;
}

/* Threads of every later parallel call that does not set its own count
 * (n <= 0: one per core); the benchmark's one-core timings use it. */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
#else
    (void)n;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
