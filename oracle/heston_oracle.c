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
/* One Milstein path with tangents (Sec. 2.4.2)                        */
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
    double minabsV;                         /* min |value deciding a truncation branch| (flip classification) */
} orc_path;

/* Number of doubles in orc_path, for the flat per-path dump. */
#define ORC_PATH_DOUBLES 15

/* Simulate one path from the given normals.  Za, Zb: independent N(0,1)
 * draws per step (Algorithm "Generation of two correlated Normal random
 * variables", step 1).  M = number of Asian dates (N % M == 0).
 * traj_X / traj_V, when non-NULL, receive X_k, V_k for k = 0..N. */
void orc_milstein_path(const orc_params *p, double T, uint32_t N, uint32_t M, int trunc,
                       const double *Za, const double *Zb, orc_path *out,
                       double *traj_X, double *traj_V)
{
    const double dt = T / (double)N;
    const double ddt = 1.0 / (double)N;            /* d(dt)/dT */
    const double sq = sqrt(1.0 - p->rho * p->rho);
    const uint32_t stride = N / M;                  /* steps between monitoring dates */

    double X = 0.0, V = p->v0;
    double X_v = 0.0, V_v = 1.0;                    /* dX/dv0, dV/dv0 at t = 0 */
    double X_T = 0.0, V_T = 0.0;                    /* dX/dT,  dV/dT  at t = 0 */
    double sumS = 0.0, sumtS = 0.0, sumS_Xv = 0.0, sumS_XT = 0.0;
    double GE = 0.0, QE = 0.0, GA = 0.0, QA = 0.0;
    double minabsV = fabs(V);

    if (traj_X) { traj_X[0] = X; traj_V[0] = V; }

    for (uint32_t k = 0; k < N; ++k) {
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
        const double Xn = X + (p->r - 0.5 * Vp) * dt + u * Z1;
        const double Xn_v = X_v - 0.5 * Vp_v * dt + u_v * Z1;
        const double Xn_T = X_T + (p->r - 0.5 * Vp) * ddt - 0.5 * Vp_T * dt + u_T * Z1;

        /* V step: V + kappa (theta - V) dt + xi sqrt(V dt) Z2 + xi^2 dt (Z2^2 - 1) / 4. */
        double Vn, Vn_v, Vn_T;
        double branch;              /* the value whose sign picks the next branch */
        if (trunc == ORC_TRUNC_FULL) {
            /* Full truncation: the state keeps its sign; drift, diffusion and
             * the Milstein term (which comes from the diffusion) see V+. */
            const double mil = pos ? 1.0 : 0.0;
            Vn = V + p->kappa * (p->theta - Vp) * dt + p->xi * u * Z2
                 + 0.25 * p->xi * p->xi * dt * (Z2 * Z2 - 1.0) * mil;
            Vn_v = V_v - p->kappa * Vp_v * dt + p->xi * u_v * Z2;
            Vn_T = V_T + p->kappa * (p->theta - Vp) * ddt - p->kappa * Vp_T * dt
                   + p->xi * u_T * Z2 + 0.25 * p->xi * p->xi * ddt * (Z2 * Z2 - 1.0) * mil;
            branch = Vn;
        } else {
            /* The paper's scheme as printed: update with V, then V = max(V, 0). */
            const double Vt = V + p->kappa * (p->theta - V) * dt + p->xi * u * Z2
                              + 0.25 * p->xi * p->xi * dt * (Z2 * Z2 - 1.0);
            const double Vt_v = V_v - p->kappa * V_v * dt + p->xi * u_v * Z2;
            const double Vt_T = V_T + p->kappa * (p->theta - V) * ddt - p->kappa * V_T * dt
                                + p->xi * u_T * Z2 + 0.25 * p->xi * p->xi * ddt * (Z2 * Z2 - 1.0);
            const int keep = Vt > 0.0;
            Vn = keep ? Vt : 0.0;
            Vn_v = keep ? Vt_v : 0.0;
            Vn_T = keep ? Vt_T : 0.0;
            branch = Vt;
        }

        X = Xn; X_v = Xn_v; X_T = Xn_T;
        V = Vn; V_v = Vn_v; V_T = Vn_T;
        if (fabs(branch) < minabsV) minabsV = fabs(branch);
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
int orc_mc_sums(const orc_params *p, const orc_contract *contracts, uint32_t n_contracts,
                uint64_t path_begin, uint64_t n_paths, uint32_t N, uint64_t seed, int trunc,
                int n_threads, double *sum, double *sumsq)
{
    if (n_contracts == 0 || N == 0) return -1;
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
                orc_milstein_path(p, T, N, M, trunc, Za, Zb, &w, NULL, NULL);
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
                    double *rec, double *est)
{
    if (n_contracts == 0 || N == 0) return -1;
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
        orc_milstein_path(p, T, N, M, trunc, Za, Zb, &w, NULL, NULL);
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
                          uint32_t N, int trunc, const double *Za, const double *Zb,
                          double *rec, double *est, double *traj_X, double *traj_V)
{
    if (n_contracts == 0 || N == 0) return -1;
    uint32_t M = N;
    for (uint32_t c = 0; c < n_contracts; ++c)
        if (contracts[c].payoff == 1 && contracts[c].n_monitor) M = contracts[c].n_monitor;
    if (N % M != 0) return -1;
    orc_path w;
    orc_milstein_path(p, contracts[0].T, N, M, trunc, Za, Zb, &w, traj_X, traj_V);
    memcpy(rec, &w, sizeof(double) * ORC_PATH_DOUBLES);
    for (uint32_t c = 0; c < n_contracts; ++c)
        orc_estimators(p, &contracts[c], N, &w, est + c * 6);
    return 0;
}

/* Many paths from caller-supplied normals: Za, Zb are (n_paths x N) row-major;
 * rec receives n_paths x ORC_PATH_DOUBLES and est n_paths x n_contracts x 6. */
int orc_paths_from_normals(const orc_params *p, const orc_contract *contracts, uint32_t n_contracts,
                           uint32_t N, int trunc, uint64_t n_paths, const double *Za,
                           const double *Zb, double *rec, double *est)
{
    if (n_contracts == 0 || N == 0) return -1;
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
        orc_milstein_path(p, contracts[0].T, N, M, trunc, Za + (size_t)i * N, Zb + (size_t)i * N,
                          &w, NULL, NULL);
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

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
