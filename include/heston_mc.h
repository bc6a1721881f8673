/*
 * heston_mc.h -- C ABI of the GB300 Monte Carlo Heston pricer (arXiv 2309.10477).
 *
 * The library simulates Heston paths (Eq. heston_eq, Sec. 2.1) with the
 * Milstein scheme for ln S and V (Sec. 2.4.2, Algorithm "Milstein
 * approximation under Heston model"), driven by correlated normals
 * (Algorithm "Generation of two correlated Normal random variables"), and
 * returns Monte Carlo estimates (Algorithm "Monte Carlo option pricing
 * estimation", Sec. 2.5) of the discounted price and the Greeks Delta,
 * Gamma, Vega, Rho and Theta (named in Sec. 2; pathwise Delta and Rho of
 * Eq. euro_pw and Eq. asian_pw) with their standard errors, all from the
 * same paths.  Every path lives in registers on the GPU; nothing per path
 * is written to memory.
 *
 * Conventions for every entry point:
 *   - Pointers documented "host" point to caller-owned host memory; pointers
 *     documented "device" point to caller-owned memory on the selected CUDA
 *     device.  The library never retains a pointer after a call returns.
 *   - Return value: HESTON_OK (0) on success, a positive HESTON_WARN_* code
 *     when results are produced but some are undefined (set to NaN), or a
 *     negative HESTON_ERR_* code; on error nothing is launched and no output
 *     is written unless stated.  No C++ exception crosses this interface.
 *   - Calls on different streams may run concurrently from different host
 *     threads; the library holds no global mutable state apart from the
 *     static scratch array of heston_mc_launch_noalloc.
 *   - Per-device handles are cached for the life of the process: the
 *     scratch memory pool of the synchronous entry points and the device
 *     address of the static scratch array.  cudaDeviceReset invalidates
 *     them, so a process must not call the library on a device after
 *     resetting it.
 *
 * Random numbers (the contract both the GPU path and the test oracle
 * implement): Philox4x32-10 (Salmon et al., SC'11) with key = rng_seed
 * (low word first) and counter = (step / 2, path_lo, path_hi, 0) for path
 * index `path` and time step `step`; words 0-1 feed even steps and words
 * 2-3 odd steps as (u1, u2) with u1 = ((w >> 8) + 1) * 2^-24 and
 * u2 = (w >> 8) * 2^-24; Box-Muller Za = sqrt(-2 ln u1) cos(2 pi u2),
 * Zb = sqrt(-2 ln u1) sin(2 pi u2).  The FP32 path evaluates ln, sqrt, sin
 * and cos with the special-function unit's approximations (its normals lie
 * within 1e-7 + 1.5e-6 R of the exact ones, R = sqrt(Za^2 + Zb^2)); the FP64
 * path takes ln u1 and sin/cos(2 pi u2) from table-driven FP64 functions
 * (within about 2 ulp; see heston_bm64_debug).  Results are therefore a
 * function of (inputs, seed) only, independent of launch shape, device and
 * sharding.
 */
#ifndef HESTON_MC_H
#define HESTON_MC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ----------------------------------------------------- */
#define HESTON_OK                    0
#define HESTON_WARN_GAMMA_UNDEFINED  1  /* |rho| == 1 or v0 == 0: Gamma (and its SE) set to NaN */
#define HESTON_WARN_TANGENT_UNSTABLE 2  /* a Vega or Theta estimate or SE is not finite (see below) */
#define HESTON_ERR_INVALID_ARG      -1  /* a parameter is out of its domain (see heston_mc_price_greeks_ex) */
#define HESTON_ERR_CUDA             -2  /* a CUDA runtime call failed */
#define HESTON_ERR_NOMEM            -3  /* device allocation failed */
#define HESTON_ERR_TIMEOUT          -4  /* reserved: a bounded device wait expired */
#define HESTON_ERR_CANCELLED        -5  /* reserved: a cancel flag was raised */
#define HESTON_ERR_UNSUPPORTED      -6  /* option combination not built */
#define HESTON_ERR_WORKSPACE        -7  /* caller workspace missing, misaligned or too small */

#define HESTON_MAX_CONTRACTS 8          /* contracts priced on one set of paths */
#define HESTON_TILE_PATHS   64          /* paths per deterministic partial sum */

/* ---- inputs ------------------------------------------------------------ */

/* Heston parameters (Eq. heston_eq and Table "Heston model parameters"):
 * dS = r S dt + sqrt(V) S dW1, dV = kappa (theta - V) dt + xi sqrt(V) dW2,
 * corr(dW1, dW2) = rho.  The paper writes sigma for xi. */
typedef struct {
    double S0, v0, kappa, theta, xi, rho, r;
} heston_params;

typedef enum { HESTON_EUROPEAN = 0, HESTON_ASIAN_ARITH = 1 } heston_payoff;

/* One option.  European payoff max(S_T - K, 0) (put: max(K - S_T, 0));
 * arithmetic Asian payoff on Sbar = (1/M) sum_{i=1..M} S_{t_i} with equal
 * dates t_i = i T / M (Sec. 2).  n_monitor = M; 0 means M = n_steps;
 * n_steps must be a multiple of M. */
typedef struct {
    int32_t payoff;      /* heston_payoff */
    int32_t is_put;      /* 0 = call, 1 = put */
    double K;            /* strike, >= 0 */
    double T;            /* maturity in years, > 0 */
    uint32_t n_monitor;  /* Asian dates M (0 = every step) */
    uint32_t reserved;   /* must be 0 */
} heston_contract;

typedef enum { HESTON_TRUNC_FULL = 0, HESTON_TRUNC_PAPER_FLOOR = 1 } heston_trunc;
typedef enum { HESTON_RNG_PHILOX = 0, HESTON_RNG_SOBOL_BB = 1 } heston_rng;
typedef enum { HESTON_FP32 = 0, HESTON_FP64 = 1 } heston_prec;
/* Discretisation of one step (all on the same Philox normals Za, Zb):
 * MILSTEIN (Sec. 2.4.2, default); EULER (Sec. 2.4.1: the Milstein step
 * without the xi^2 dt (Z2^2 - 1) / 4 term, same truncation choices); QE,
 * Andersen's quadratic-exponential scheme (the method Sec. 5 names as the
 * next one to try; L. Andersen, J. Comput. Finance 11(3), 2008): the
 * variance from its exact conditional mean and variance, matched by
 * a (b + Za)^2 when psi = s^2/m^2 <= 1.5 and by a point mass at zero plus
 * an exponential tail driven by Uv = Phi(Za) above; ln S from both
 * variances with the independent normal Zb, gamma1 = gamma2 = 1/2, no
 * martingale correction.  QE ignores trunc (its variance is never
 * negative) and needs kappa, theta, xi > 0 (HESTON_ERR_INVALID_ARG
 * otherwise).  EULER and QE run with rng = PHILOX on the single-set entry
 * points (heston_mc_price_greeks[_ex], heston_mc_launch[_noalloc],
 * heston_mc_launch_tiles, heston_mc_debug_paths); the QMC, batched,
 * serving and adjoint entry points return HESTON_ERR_UNSUPPORTED for them. */
typedef enum { HESTON_SCHEME_MILSTEIN = 0, HESTON_SCHEME_EULER = 1, HESTON_SCHEME_QE = 2 } heston_scheme;

/* Options.  trunc: full truncation (the state keeps its sign; drift,
 * diffusion and the Milstein term see max(V, 0)) or the paper's floor
 * V = max(V, 0) after each update (Sec. 2.4.2).  prec: arithmetic of the
 * path recursion; sums are always FP64 above the 64-path tile.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).  device:
 * CUDA ordinal, or -1 for the calling thread's current device.
 * grid_ctas / block_threads: launch shape of the path kernel (0 = choose);
 * results do not depend on them.  rng: Philox (pseudo-random) or the
 * randomised-QMC variant below, with n_shifts replicates. */
typedef struct {
    int32_t trunc;
    int32_t rng;
    int32_t prec;
    uint32_t n_shifts;
    void *cuda_stream;
    int32_t device;
    uint32_t grid_ctas;
    uint32_t block_threads;
    int32_t scheme;            /* heston_scheme */
    uint32_t reserved;
} heston_options;

/* Vega and Theta are pathwise tangents through sqrt(V): each step scales the
 * v0- and T-tangents by about 1 + xi sqrt(dt) Z / (2 sqrt(V)).  When the
 * variance process comes close to zero (parameters far from the Feller
 * condition 2 kappa theta >= xi^2, many steps) the per-path tangents have
 * unbounded variance, the estimates are meaningless and in FP32 may
 * overflow; the synchronous entry points then return
 * HESTON_WARN_TANGENT_UNSTABLE (per result in heston_result.status).  Price,
 * Delta, Gamma and Rho do not use the tangents and are unaffected.
 *
 * Result for one contract: discounted price, Delta = dV/dS0,
 * Gamma = d2V/dS0^2, Vega = dV/dv0, Rho = dV/dr, Theta = -dV/dT, and the
 * standard error of each mean (sample stdev / sqrt(n)), se[] in the same
 * order.  The first 12 doubles match the device output layout below. */
typedef struct {
    double price, delta, gamma, vega, rho, theta;
    double se[6];
    uint64_t n_paths;
    int32_t status;
    int32_t reserved;
} heston_result;

/* ---- synchronous host API ------------------------------------------------ */

/* Price one contract with the defaults (full truncation, Philox, FP64 path,
 * legacy default stream, current device).  params, contract, out: host.
 * Blocks until the result is in *out.  out->status mirrors the return. */
int heston_mc_price_greeks(const heston_params *params, const heston_contract *contract,
                           uint64_t n_paths, uint32_t n_steps, uint64_t rng_seed,
                           heston_result *out);

/* Price n_contracts (1..HESTON_MAX_CONTRACTS) options on the same n_paths
 * paths of n_steps steps.  All contracts must share T; Asian contracts must
 * share M.  opts may be NULL (defaults).  out: host array of n_contracts.
 * Allocates its device workspace stream-ordered on opts->cuda_stream, from
 * a pool that keeps the memory for the next call (heston_release_cached_memory
 * returns it), and returns after that stream has produced the results.
 * HESTON_ERR_INVALID_ARG when: a pointer is NULL; S0 <= 0; K < 0; T <= 0;
 * v0, theta, kappa or xi < 0; |rho| > 1; any value not finite; n_steps == 0;
 * n_paths < 2 or > 2^40; N % M != 0; contracts disagree on T or on M;
 * payoff or is_put out of range; an enum or reserved field out of range. */
int heston_mc_price_greeks_ex(const heston_params *params, const heston_contract *contracts,
                              uint32_t n_contracts, uint64_t n_paths, uint32_t n_steps,
                              uint64_t rng_seed, const heston_options *opts,
                              heston_result *out);

/* ---- asynchronous device API (no allocation, no synchronisation) -------- */

/* Bytes of device workspace heston_mc_launch needs for these sizes. */
int heston_mc_workspace_bytes(uint32_t n_contracts, uint64_t n_paths, size_t *bytes);

/* Enqueue the whole estimate on opts->cuda_stream and return at once.
 * d_workspace: device, >= heston_mc_workspace_bytes() bytes, 256-byte
 * aligned, not used by another launch in flight.  d_out: device array of
 * n_contracts x 12 doubles: out[c*12 + j] = mean of estimator j and
 * out[c*12 + 6 + j] = its standard error, j in (price, delta, gamma, vega,
 * rho, theta).  Validation as in heston_mc_price_greeks_ex; a CUDA launch
 * failure returns HESTON_ERR_CUDA. */
int heston_mc_launch(const heston_params *params, const heston_contract *contracts,
                     uint32_t n_contracts, uint64_t n_paths, uint32_t n_steps,
                     uint64_t rng_seed, const heston_options *opts,
                     void *d_workspace, size_t workspace_bytes, double *d_out);

/* ---- allocation-free launch ---------------------------------------------- */

/* The paper has no counterpart to this entry point.  It exists for callers
 * that must not allocate device memory themselves or let a library do it:
 * a pricing engine embedded in a host application whose device memory is
 * owned by another allocator (a framework's caching allocator or a fixed
 * arena that a third-party cudaMalloc would fragment or overrun), and
 * latency-critical request loops, where cudaMalloc / cudaFree can
 * synchronise the device and stall work on other streams.
 *
 * HESTON_NOALLOC_SCRATCH_BYTES is the size of the library's static device
 * scratch array (16 MiB); every GPU that loads the library holds it until
 * the process exits.  A request fits when heston_mc_workspace_bytes() for
 * its (n_contracts, n_paths) is at most this size: e.g. up to about 1.8 M
 * paths for 6 contracts, or 11 M paths for 1 contract. */
#define HESTON_NOALLOC_SCRATCH_BYTES (16u << 20)

/* Same estimate, inputs and output as heston_mc_launch, with the workspace
 * taken from the static scratch array instead of the caller: enqueues on
 * opts->cuda_stream and returns at once; d_out: device array of
 * n_contracts x 12 doubles (layout as for heston_mc_launch).
 *   - Calls no cudaMalloc, cudaFree or other allocating routine.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current and caches it for the
 *     process; make that first call before any stream capture on the
 *     device, and make no call on a device after cudaDeviceReset on it (the
 *     cached address would be stale).
 *   - A request larger than HESTON_NOALLOC_SCRATCH_BYTES returns
 *     HESTON_ERR_WORKSPACE and launches nothing; other errors as for
 *     heston_mc_launch (HESTON_ERR_INVALID_ARG also for d_out == NULL).
 *   - All calls on a device share the one array, which keeps the last
 *     call's contents.  Every call writes the rows it reads before reading
 *     them, so nothing needs clearing; but calls whose kernels overlap on
 *     the GPU (different streams or host threads without ordering between
 *     them) race on the array and give wrong results: order them, e.g. on
 *     one stream. */
int heston_mc_launch_noalloc(const heston_params *params, const heston_contract *contracts,
                             uint32_t n_contracts, uint64_t n_paths, uint32_t n_steps,
                             uint64_t rng_seed, const heston_options *opts, double *d_out);

/* ---- sharding: path-range partial sums and their reduction -------------- */

/* Simulate global paths [path_begin, path_begin + n_paths) and write one
 * partial-sum row per 64-path tile: d_tile_sums (device) holds
 * ceil(n_paths / 64) rows of 12 * n_contracts doubles, row = (sum_x[6C],
 * sum_x^2[6C]) with contract-major order.  path_begin must be a multiple
 * of HESTON_TILE_PATHS.  Rows of consecutive shards concatenate into the
 * rows of the unsharded range, so the reduction below gives bit-identical
 * results for any split. */
int heston_mc_launch_tiles(const heston_params *params, const heston_contract *contracts,
                           uint32_t n_contracts, uint64_t path_begin, uint64_t n_paths,
                           uint32_t n_steps, uint64_t rng_seed, const heston_options *opts,
                           double *d_tile_sums);

/* Reduce n_tiles rows of tile sums (device) over n_paths_total paths into
 * d_out (device, n_contracts x 12 doubles as for heston_mc_launch), in a
 * fixed order.  d_workspace: device scratch of at least
 * heston_mc_workspace_bytes(n_contracts, n_paths_total) bytes (only its
 * group-sum part is used).  stream: cudaStream_t or NULL. */
int heston_mc_reduce_tiles(const double *d_tile_sums, uint64_t n_tiles, uint32_t n_contracts,
                           uint64_t n_paths_total, void *d_workspace, size_t workspace_bytes,
                           double *d_out, void *stream);

/* ---- randomised quasi-Monte Carlo variant ------------------------------- */

/* Normals from a Sobol sequence randomised by digital shifts and fed
 * through a Brownian bridge (Sobol sequences and Property A: Sec. 2.7; the
 * paper found plain QMC unsatisfactory for the discretised schemes, Sec. 3,
 * which the bridge addresses by putting the coarse shape of each Brownian
 * motion in the first dimensions).  Definitions shared with the test oracle:
 *   - 2 n_steps dimensions; dimension 0: v_k = 2^(32-k); dimension j >= 1:
 *     the j-th primitive polynomial over GF(2) by (degree, coefficient
 *     bits), initial numbers m_1..m_s from Philox4x32-10 with key
 *     (0x50B01, 0) and counter ((k-1)/4, j, c, 3), word (k-1)%4,
 *     m_k = 2 (w mod 2^(k-1)) + 1; for j < 32 the first candidate c that
 *     keeps the leading (j+1)x(j+1) matrix of first binary digits
 *     non-singular (Property A for the first j+1 dimensions), else c = 0;
 *     Bratley-Fox recurrence to 32-bit direction integers.
 *   - replicate r (of opts->n_shifts) XORs word d%4 of Philox block
 *     (d/4, r, 0, 2) under key rng_seed into dimension d; path index
 *     p = r * P + n with P = n_paths / n_shifts points per replicate.
 *   - u = ((y >> 8) + 1/2) 2^-24, z = Phi^-1(u).  The FP32 kernels evaluate
 *     Phi^-1 as v P(w), v = 2u - 1, w = -ln(1 - v^2), with polynomials
 *     fitted for this library: relative error below 3e-7 over all 2^24
 *     values of u (apart from the lg2 / sqrt approximations, ~2e-8).
 *   - Brownian bridge on the step grid 0..N: node 0 is time N; then
 *     intervals [l, r] with r - l >= 2 are bisected breadth-first at
 *     m = l + (r-l)/2.  Node j drives motion a (Za) with dimension 2j and
 *     motion b (Zb) with 2j+1; step normals are the bridge increments.
 *   - Estimates: mean over replicates of each replicate's average;
 *     SE = sample stdev of the replicate averages / sqrt(n_shifts).
 * Constraints: FP32 path only (HESTON_ERR_UNSUPPORTED otherwise);
 * n_steps <= 2048; n_shifts >= 2; P a multiple of 64 and <= 2^32.
 * heston_mc_price_greeks_ex runs this variant when opts->rng is
 * HESTON_RNG_SOBOL_BB; the other launch entry points accept only Philox. */

/* Host-built direction integers (test support): h_out, n_dims x 32 uint32,
 * row d holds v_{d,1..32}.  n_dims <= 4096. */
int heston_sobol_directions(uint32_t n_dims, uint32_t *h_out);

/* Bytes of the device table buffer for n_steps (direction integers, the
 * 64-point tile table and the bridge event plan). */
int heston_qmc_tables_bytes(uint32_t n_steps, size_t *bytes);

/* Build the tables for n_steps into d_tables (device, 256-byte aligned,
 * >= heston_qmc_tables_bytes).  Synchronous (host computation and a copy);
 * the buffer is then read-only and may serve any number of launches with
 * the same n_steps.  device: CUDA ordinal or -1 for the current device. */
int heston_qmc_build_tables(uint32_t n_steps, void *d_tables, size_t bytes, int32_t device);

/* Workspace bytes of heston_mc_launch_qmc. */
int heston_mc_workspace_bytes_qmc(uint32_t n_contracts, uint64_t n_paths, uint32_t n_steps,
                                  uint32_t n_shifts, size_t *bytes);

/* Enqueue a randomised-QMC estimate (opts->rng == HESTON_RNG_SOBOL_BB,
 * opts->n_shifts replicates) on opts->cuda_stream: no allocation, no
 * synchronisation.  d_tables: built by heston_qmc_build_tables for the same
 * n_steps.  d_workspace: device, 256-byte aligned, >=
 * heston_mc_workspace_bytes_qmc.  d_out: as for heston_mc_launch. */
int heston_mc_launch_qmc(const heston_params *params, const heston_contract *contracts,
                         uint32_t n_contracts, uint64_t n_paths, uint32_t n_steps,
                         uint64_t rng_seed, const heston_options *opts, const void *d_tables,
                         void *d_workspace, size_t workspace_bytes, double *d_out);

/* Per-path dump of the QMC variant (test support): `count` points (host
 * array, indices within replicate `replicate` < 2^16); records and
 * estimators as for heston_mc_debug_paths.  Synchronous; allocates. */
int heston_qmc_debug_paths(const heston_params *params, const heston_contract *contracts,
                           uint32_t n_contracts, uint32_t n_steps, uint64_t rng_seed,
                           const heston_options *opts, uint32_t replicate, const uint32_t *points,
                           uint32_t count, double *h_records, double *h_estimators);

/* ---- batched persistent launch -------------------------------------------- */

/* Many uneven contracts in one launch (the batched form of the paper's
 * Algorithm "Monte Carlo option pricing estimation", Sec. 2.5): each item
 * has its own parameters, path count, step count and seed, and its result
 * equals heston_mc_launch of that item alone (same seed) bit for bit.
 * Work items are (contract, 64-path tile) pairs taken from a device counter,
 * contracts with the most steps first, by persistent warps.  FP32 paths
 * only; trunc from the options, common to the batch. */
typedef struct {
    heston_params params;
    heston_contract contract;
    uint64_t n_paths;
    uint32_t n_steps;
    uint32_t reserved;          /* must be 0 */
    uint64_t rng_seed;
} heston_batch_item;

/* Host-side plan of a batch: sizes the caller allocates and the totals the
 * launch needs.  Filled by heston_batch_plan_make. */
typedef struct {
    uint64_t total_tiles;       /* work items */
    uint64_t total_groups;      /* first-level reduction rows */
    uint64_t total_path_steps;
    uint32_t n_items;
    int32_t trunc;
    size_t descriptor_bytes;    /* device buffer for heston_batch_prepare */
    size_t workspace_bytes;     /* device buffer for heston_mc_launch_batch */
} heston_batch_plan;

/* Validate every item (as heston_mc_price_greeks_ex would; FP32 only) and
 * size the buffers.  items: host array of n_items (>= 1). */
int heston_batch_plan_make(const heston_batch_item *items, uint32_t n_items,
                           const heston_options *opts, heston_batch_plan *plan);

/* Write the device descriptors of the batch (per-contract constants, work
 * order) into d_desc (device, 256-byte aligned, plan->descriptor_bytes).
 * Synchronous.  The descriptors are read-only afterwards and serve any
 * number of launches. */
int heston_batch_prepare(const heston_batch_item *items, const heston_options *opts,
                         const heston_batch_plan *plan, void *d_desc);

/* Enqueue the batch on opts->cuda_stream: one memset, the persistent path
 * kernel and two reduction kernels; no allocation, no synchronisation.
 * d_workspace: device, 256-byte aligned, plan->workspace_bytes.  d_out:
 * device, n_items x 12 doubles (layout as heston_mc_launch, one contract per
 * item).  d_status: optional device int32 (NULL = none): 0 runs the batch;
 * if it holds 1 the warps take no further work items and set it to 2
 * (the outputs are then incomplete); the launch never resets it. */
int heston_mc_launch_batch(const heston_batch_plan *plan, const void *d_desc,
                           const heston_options *opts, void *d_workspace, double *d_out,
                           int32_t *d_status);

/* Synchronous convenience: plan, allocate, prepare, launch, copy back.
 * out: host array of n_items results. */
int heston_mc_price_greeks_batch(const heston_batch_item *items, uint32_t n_items,
                                 const heston_options *opts, heston_result *out);

/* ---- cached scratch -------------------------------------------------------- */

/* The synchronous entry points (heston_mc_price_greeks[_ex] and
 * heston_mc_debug_paths) take their device scratch stream-ordered from a
 * memory pool per device owned by this library, which keeps freed blocks
 * mapped for the next call.  This returns the unused cached memory of one
 * device (device >= 0) or of every device (device = -1) to the driver;
 * memory still in use by a call in flight stays.  HESTON_ERR_INVALID_ARG
 * for device >= 64; HESTON_ERR_CUDA if the driver refuses. */
int heston_release_cached_memory(int32_t device);

/* ---- serving engine (continuous batching) ---------------------------------- */

/* A request loop over the batched kernel: requests (heston_batch_item, one
 * contract each) are submitted from any host thread at any time; a server
 * thread admits them to the device as slots and pool memory free up, and
 * runs rounds: each round hands every active request a share of
 * `tiles_per_round` 64-path tiles and launches them together (the
 * persistent batch kernel with per-request tile offsets), so the work of
 * requests that arrived at different times overlaps on the GPU.  A request
 * whose last tile ran is reduced (fixed order) and copied back while the next
 * round runs.  Every result equals heston_mc_price_greeks_ex of the same item
 * alone bit for bit (FP32 path; tile rows are fixed by the path index).
 * Admission is by device memory: a request needs ceil(n_paths/64) * 96 bytes
 * of the pool until it completes; requests that do not fit wait in FIFO
 * order; one larger than the whole pool is refused at submit
 * (HESTON_ERR_NOMEM).  No device code waits on the host: all waiting is on
 * host condition variables with bounded timeouts. */
typedef struct heston_server heston_server;

typedef struct {
    int32_t device;            /* CUDA ordinal, -1 = current */
    int32_t trunc;             /* heston_trunc for every request */
    size_t memory_bytes;       /* device pool for the tile rows of admitted requests */
    uint32_t max_active;       /* requests on the device at once (0 = 1024) */
    uint32_t reserved;         /* must be 0 */
    uint64_t tiles_per_round;  /* 64-path tiles per round (0 = 65536) */
} heston_server_config;

typedef struct {
    uint64_t submitted, completed, rounds, tiles_done;
    uint32_t queued, active;
    size_t memory_in_use, memory_peak;
} heston_server_stats;

/* Create a server (allocates its device buffers and starts its thread).
 * HESTON_ERR_INVALID_ARG for a NULL argument, nonzero reserved, unknown
 * trunc or memory_bytes < 4096; HESTON_ERR_NOMEM if a buffer cannot be
 * allocated (nothing is left allocated).  The caller owns the handle until
 * heston_server_destroy. */
int heston_server_create(const heston_server_config *cfg, heston_server **out);

/* Queue one request (host struct, copied); *ticket identifies it.
 * Validation as heston_mc_price_greeks_ex; FP32 Philox only. */
int heston_server_submit(heston_server *s, const heston_batch_item *item, uint64_t *ticket);

/* Non-blocking: returns 1 and fills *out (and *latency_s: submit to result on
 * the host, seconds; may be NULL) once the request is done, 0 while pending.
 * A ticket is reported once.  A ticket never issued by this server gives
 * HESTON_ERR_INVALID_ARG.  A CUDA failure in the request's rounds is
 * reported as out->status = HESTON_ERR_CUDA. */
int heston_server_poll(heston_server *s, uint64_t ticket, heston_result *out, double *latency_s);

/* As poll, waiting up to timeout_ms milliseconds. */
int heston_server_wait(heston_server *s, uint64_t ticket, uint32_t timeout_ms, heston_result *out,
                       double *latency_s);

int heston_server_stats_get(heston_server *s, heston_server_stats *out);

/* Finish every submitted request, stop the thread, free the device buffers.
 * Results not yet polled are discarded. */
int heston_server_destroy(heston_server *s);

/* ---- adjoint (reverse-mode pathwise) parameter gradient -------------------- */

/* Gradient of the discounted price of one contract with respect to
 * (S0, v0, kappa, theta, xi, rho, r): the pathwise method (Sec. 2, the
 * chain rule through the path, Eq. pw_est) applied in reverse mode to the
 * Milstein recursion with full truncation.  FP32 paths, FP64 sums, Philox
 * normals, n_steps <= 1024; other options return HESTON_ERR_UNSUPPORTED.
 * The forward call prices the contract and stores, per path, (X, V) every
 * 8 steps and the payoff slope; the backward call rebuilds each 8-step
 * segment from its checkpoint (normals recomputed from their Philox
 * counters) in registers and runs the adjoint sweep.  Both are asynchronous
 * on opts->cuda_stream, allocate nothing, and must use the same workspace,
 * inputs and seed, the backward after the forward.
 *   d_workspace: device, 256-byte aligned, >= heston_adjoint_workspace_bytes.
 *   d_price: device, 2 doubles (price, SE).
 *   d_grad:  device, 14 doubles (the 7 derivatives, then their SEs). */
int heston_adjoint_workspace_bytes(uint64_t n_paths, uint32_t n_steps, size_t *bytes);

int heston_mc_adjoint_forward(const heston_params *params, const heston_contract *contract,
                              uint64_t n_paths, uint32_t n_steps, uint64_t rng_seed,
                              const heston_options *opts, void *d_workspace, size_t workspace_bytes,
                              double *d_price);

int heston_mc_adjoint_backward(const heston_params *params, const heston_contract *contract,
                               uint64_t n_paths, uint32_t n_steps, uint64_t rng_seed,
                               const heston_options *opts, void *d_workspace, size_t workspace_bytes,
                               double *d_grad);

/* Test support: the per-path values of the adjoint kernels for paths
 * 0 .. n_paths-1 (forward and backward enqueued on opts->cuda_stream, as
 * above).  d_per_path: device, n_paths x 8 doubles per path: the discounted
 * payoff, then its derivatives with respect to (S0, v0, kappa, theta, xi,
 * rho, r) -- the FP32 values the estimates sum.  d_workspace must hold
 * heston_adjoint_workspace_bytes + 768 bytes (the estimates are written
 * past the workspace proper and not returned); HESTON_ERR_WORKSPACE if not. */
int heston_mc_adjoint_debug_paths(const heston_params *params, const heston_contract *contract,
                                  uint64_t n_paths, uint32_t n_steps, uint64_t rng_seed,
                                  const heston_options *opts, void *d_workspace, size_t workspace_bytes,
                                  double *d_per_path);

/* ---- test support --------------------------------------------------------- */

/* Per-path dump for `count` global path indices (host array `paths`):
 * h_records (host, count x 15 doubles) receives X_N = ln(S_T/S0), V_N,
 * dX_N/dv0, dV_N/dv0, dX_N/dT, dV_N/dT, sum S_ti, sum t_i S_ti,
 * sum S_ti dX_ti/dv0, sum S_ti dX_ti/dT, the Gamma weights over all steps
 * (sum u_k W_k, sum V_k+ dt) and over the steps before the first date,
 * and min |V_k|; h_estimators (host, count x n_contracts x 6 doubles) the
 * per-path estimators.  Synchronous; allocates device memory. */
int heston_mc_debug_paths(const heston_params *params, const heston_contract *contracts,
                          uint32_t n_contracts, uint32_t n_steps, uint64_t rng_seed,
                          const heston_options *opts, const uint64_t *paths, uint32_t count,
                          double *h_records, double *h_estimators);

/* Raw random-number contract on the device, for tests: for each of `count`
 * (path, step) pairs (host arrays) write the Philox words of the step's
 * pair (4 x uint32, host h_words) and the step's (Za, Zb) in the chosen
 * precision widened to double (host h_normals, 2 per entry). */
int heston_rng_debug(uint64_t rng_seed, const uint64_t *paths, const uint32_t *steps,
                     uint32_t count, int32_t prec, uint32_t *h_words, double *h_normals);

/* The FP64 Box-Muller's table-driven logarithm and sine/cosine beside
 * CUDA's, for tests (Sec. 2.4's normals; the uniforms are those of the
 * random-number contract above): for i in [0, count), with n = first + i + 1
 * and g = first + i, h_out (host, count x 6 doubles) receives ln(n 2^-24) by
 * the table method and by CUDA's log, then sin and cos of 2 pi g 2^-24 by
 * the table method and by CUDA's sincospi.  first + count <= 2^24, count >= 1
 * (HESTON_ERR_INVALID_ARG otherwise).  Synchronous; allocates device memory. */
int heston_bm64_debug(uint32_t first, uint32_t count, double *h_out);

/* Static description of a status code (never NULL). */
const char *heston_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* HESTON_MC_H */
