/*
 * pa.h -- C ABI of the GB300 population-annealing library (libpa.so).
 *
 * Population annealing (PA), Sec. 2 of Ebert, Gessert, Janke & Weigel,
 * "Optimized population Monte Carlo" (arXiv:2401.07965): a population of R
 * replicas of a periodic Ising / Edwards-Anderson +-J lattice is cooled from
 * beta_0 = 0 to beta_f in steps.  Each temperature step i
 *   (a) reweights replica j by exp(-(beta_i - beta_{i-1}) E_j), normalised by
 *       Q_i of Eq. (Q),
 *   (b) draws integer copy numbers r_j with <r_j> = tau_j (Sec. 3) by one of
 *       five rules and replicates the population accordingly (with families),
 *   (c) runs theta_i checkerboard Metropolis sweeps on every replica at beta_i,
 *   (d) measures population averages (step 4) and accumulates
 *       -beta_i F_i = ln Z_0 + sum_k ln Q_k (Eq. free-energy-estimator).
 * All of (a)-(d) run in CUDA kernels on the device that owns the stream.
 *
 * Conventions
 *  - Every call returns pa_status; nothing else crosses the ABI (no C++
 *    exceptions, no device traps).  Kernels report errors through a device
 *    status word that the next synchronising call (pa_sync, pa_observables,
 *    pa_free_energy, pa_get_array) returns.  After any error other than
 *    PA_ERR_ARG the context only accepts pa_destroy and the query calls.
 *  - Host arrays passed in are read during the call and copied; the caller
 *    keeps ownership.  Device memory is either a caller-provided workspace
 *    (pa_workspace_bytes tells its size; the library then allocates nothing
 *    on the device) or, if workspace == NULL, allocated by pa_init and freed
 *    by pa_destroy.
 *  - Work is enqueued on the caller's CUDA stream (NULL = legacy default).
 *    pa_step is asynchronous.  A context must not be used from two host
 *    threads at once.
 *  - Lattice: dim in {2,3}, L even, 2 <= L, N = L^dim <= 32768 sites,
 *    periodic; site s = x + L*y (+ L*L*z).  Spins are stored one bit per
 *    site, bit (s & 31) of word (s >> 5), bit value 1 meaning sigma = -1.
 */
#ifndef PA_H
#define PA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pa_ctx pa_ctx;

typedef enum {
    PA_OK = 0,
    PA_ERR_ARG = 1,           /* invalid argument; the context is unchanged            */
    PA_ERR_CUDA = 2,          /* a CUDA runtime call failed                             */
    PA_ERR_NOMEM = 3,         /* device allocation failed or workspace too small        */
    PA_ERR_CAPACITY = 4,      /* variable-size resampling produced R_i > R_cap          */
    PA_ERR_POISSON_KMAX = 5,  /* a Poisson inversion exceeded 256 per chunk (p < 1e-300)*/
    PA_ERR_TIMEOUT = 6,       /* a bounded device wait gave up                          */
    PA_ERR_STATE = 7,         /* the context holds an earlier device error              */
    PA_ERR_DONE = 8,          /* the schedule has no further temperature step           */
    PA_ERR_LIMIT = 9          /* a size exceeds a fixed limit: R or R_cap >= 2^24, or the */
                              /* scratch limit of pa_weights_static                     */
} pa_status;

/* Copy-count rules of Sec. 3.  Multinomial, systematic and residual keep
 * R_i = R; Poisson and nearest-integer let R_i fluctuate and use the rescaled
 * factors tau-hat = (R / R_{i-1}) tau of Eq. (taus). */
typedef enum {
    PA_MULTINOMIAL = 0,  /* R labels iid uniform on the weight axis (Fig. 2a)       */
    PA_SYSTEMATIC = 1,   /* one uniform offset, labels spaced by one (Fig. 2b)       */
    PA_RESIDUAL = 2,     /* floor(tau) copies + multinomial draws on the remainders  */
    PA_POISSON = 3,      /* r_j ~ Poisson(tau-hat_j)                                 */
    PA_NEAREST = 4       /* floor(tau-hat) copies + 1 with prob. tau-hat - floor     */
} pa_resampler;

typedef struct {
    int32_t dim; /* 2 or 3 */
    int32_t L;   /* even, >= 2 */
} pa_lattice;

typedef enum {
    PA_COUPLING_FERRO = 0,    /* J = +1 on every bond (Eq. Hamiltonian)               */
    PA_COUPLING_EA_PM = 1,    /* J = +-1 iid with p = 1/2 from (disorder_seed, realization) */
    PA_COUPLING_EXPLICIT = 2  /* J[a*N + s] in {+1,-1} for the bond (s, s + e_a)       */
} pa_coupling_kind;

typedef struct {
    int32_t kind;            /* pa_coupling_kind                                   */
    uint32_t realization;    /* EA: disorder realization index                     */
    uint64_t disorder_seed;  /* EA: Philox key of the couplings                     */
    const int8_t *J;         /* EXPLICIT: host array of dim*N values (+1 or -1)     */
} pa_couplings;

/* Annealing schedule (Sec. 2 steps 1-5): beta[0] = 0 (exact sampling of the
 * initial population), beta strictly increasing, theta[i-1] >= 0 sweeps at
 * beta[i].  Copied at pa_init. */
typedef struct {
    int32_t n_steps;        /* number of temperature steps n >= 1                 */
    const double *beta;     /* host, n_steps + 1 values                            */
    const uint32_t *theta;  /* host, n_steps values, each < 2^24                   */
} pa_schedule;

/* Population averages after the sweeps of the current step (Sec. 2 step 4).
 * Integer sums are exact; e = <E>/N, m = M/N.  Under partial resampling
 * (pa_set_partial_resampling) e, e2, absm, m2, c and chi are the weighted
 * averages sum_j w_j O_j / sum_j w_j; the integer sums stay unweighted. */
typedef struct {
    int32_t step;          /* completed temperature steps i                         */
    uint32_t R_i;          /* population size after step i                         */
    uint32_t R_prev;       /* population size before the resampling of step i      */
    uint32_t pad0;
    double beta;           /* beta_i                                                */
    double lnQ;            /* ln Q_i of Eq. (Q)                                     */
    double sum_lnQ;        /* sum_{k<=i} ln Q_k                                      */
    int64_t sumE, sumE2, sumAbsM, sumM2;
    int64_t sumC2;         /* sum over families k of c_k^2 (c_k = members)          */
    uint64_t accepts;      /* accepted Metropolis flips during step i               */
    double entropy;        /* -sum_k (c_k/R_i) ln(c_k/R_i)                           */
    double sv;             /* sampling variance, Eq. (sv), over the R_prev parents  */
    double e, e2, absm, m2;/* <E>/N, <E^2>/N^2, <|M|>/N, <M^2>/N^2                 */
    double c;              /* specific heat per spin beta^2 N (<e^2> - <e>^2)        */
    double chi;            /* susceptibility per spin beta N (<m^2> - <|m|>^2)        */
    double rho_t;          /* family statistic of Eq. (rho_t), sum c_k^2 / R_i       */
    double accept_rate;    /* accepts / (theta_i N R_i)                             */
    float features[8];     /* learned schedule: the controller's inputs after step i */
    int32_t u_next;        /* its choice for step i+1: grid points (0 = none) ...   */
    uint32_t theta_next;   /* ... and sweeps                                        */
    double ess;            /* partial resampling: (sum w)^2 / sum w^2 of the step's  */
                           /* reweighted population (R_i otherwise)                 */
    int32_t resampled;     /* partial resampling: 1 if step i resampled (always 1   */
    int32_t pad1;          /* otherwise)                                             */
} pa_obs;

/* One run of a batch (pa_batch_init).  All runs of a batch share the
 * dimension, the coupling kind (ferromagnet or not), the copy-count rule, the
 * schedule and the Philox key; lattice size, couplings, R and R_cap are per
 * run.  Runs with the same ensemble id must repeat one system (same lattice
 * and couplings): pa_weighted combines them (Sec. 4). */
typedef struct {
    pa_lattice lattice;
    pa_couplings couplings;
    uint32_t R;
    uint32_t R_cap;          /* 0 = default capacity                               */
    int32_t ensemble;        /* >= 0                                              */
} pa_run_spec;

/* Weighted average over the runs of one ensemble at one temperature step,
 * with omega^(m) = R_i^(m) exp(-beta_i F_i^(m)) / sum (Eq. weighted-averages). */
typedef struct {
    int32_t step;
    int32_t n_runs;
    double beta;
    double lnZ;           /* ln( sum_m R^(m) Zhat_m / sum_m R^(m) ) - ln Z_0          */
    double minus_beta_F;  /* N ln 2 + lnZ                                          */
    double w_max;         /* largest omega                                         */
    double eff_runs;      /* 1 / sum omega^2                                        */
    double e, e2, absm, m2;   /* W[e], W[e^2], W[|m|], W[m^2]                        */
    double c;             /* Wvar[c] = beta^2 N (W[e^2] - W[e]^2), Eq. (Wvar_C)     */
    double chi;           /* Wvar[chi] = beta N (W[m^2] - W[|m|]^2), Eq. (Wvar_Chi) */
    double c_naive;       /* sum_m omega c^(m) (the naive weighting)               */
    double chi_naive;     /* sum_m omega chi^(m)                                   */
    double e_plain, c_plain, chi_plain;  /* unweighted means over the runs          */
} pa_weighted_obs;

/* Arrays readable with pa_get_array. */
typedef enum {
    PA_ARRAY_SPINS = 0,      /* uint32 [R_i][ceil(N/32)] packed spins              */
    PA_ARRAY_ENERGY = 1,     /* int32  [R_i]                                       */
    PA_ARRAY_FAMILY = 2,     /* uint32 [R_i] index of the initial ancestor         */
    PA_ARRAY_COUNTS = 3,     /* uint32 [R_prev] copy numbers r_j of the last step  */
    PA_ARRAY_ANCESTOR = 4,   /* uint32 [R_i] parent slot j of each new slot        */
    PA_ARRAY_MAGNET = 5,     /* int32  [R_i] magnetisation M = sum sigma           */
    PA_ARRAY_WEIGHT = 6      /* double [R_i] replica weights (partial resampling;  */
                             /*        1 otherwise)                                */
} pa_array;

/* Bytes of device workspace a context needs (0 on invalid arguments).
 * R_cap = 0 selects the default capacity R + ceil(10 sqrt(R)) + 64 for the
 * variable-size rules and R for the fixed-size ones. */
size_t pa_workspace_bytes(const pa_lattice *lat, uint32_t R, uint32_t R_cap, int32_t n_steps,
                          pa_resampler resampler);

/* Create a context and draw the initial population at beta_0 = 0 (Sec. 2
 * step 1: every replica iid uniform, family_j = j, R_0 = R).
 * seed: 64-bit Philox key of every draw of the run.
 * cuda_stream: a cudaStream_t (may be NULL).
 * workspace / workspace_bytes: optional caller-owned device memory (256-byte
 * aligned, at least pa_workspace_bytes) or NULL / 0.
 * R and R_cap are below 2^24: the expected copy numbers are 2^-40 fixed-point
 * integers whose total, R 2^40, must fit in 64 bits.
 * Errors: PA_ERR_ARG (bad lattice, R == 0, R_cap < R, schedule not starting
 * at 0 or not increasing, theta too large), PA_ERR_LIMIT (R or R_cap >= 2^24),
 * PA_ERR_NOMEM, PA_ERR_CUDA. */
pa_status pa_init(pa_ctx **out, const pa_lattice *lat, const pa_couplings *cpl, uint32_t R,
                  uint32_t R_cap, const pa_schedule *sched, pa_resampler resampler,
                  uint64_t seed, void *cuda_stream, void *workspace, size_t workspace_bytes);

/* Enqueue n temperature steps (Sec. 2 steps 2-4 each).  Asynchronous.
 * Returns PA_ERR_DONE without enqueuing anything if fewer than n steps remain. */
pa_status pa_step(pa_ctx *ctx, int32_t n);

/* Wait for the stream and return the device status word. */
pa_status pa_sync(pa_ctx *ctx);

/* Synchronise and fill *out for the current step. */
pa_status pa_observables(pa_ctx *ctx, pa_obs *out);

/* Synchronise and fill rows[0..min(max_rows, step+1)) with the observables of
 * steps 0..step (step 0 = the initial population); *n_rows receives the count. */
pa_status pa_trace(pa_ctx *ctx, pa_obs *rows, int32_t max_rows, int32_t *n_rows);

/* Synchronise and return -beta_i F_i = N ln 2 + sum_k ln Q_k
 * (Eq. free-energy-estimator with ln Z_0 = N ln 2) and F_i / N
 * (NaN at beta = 0). */
pa_status pa_free_energy(pa_ctx *ctx, double *minus_beta_F, double *f_per_spin);

/* Synchronise and copy one state array to host memory.  capacity is in
 * elements (words for PA_ARRAY_SPINS); *n_out receives the element count
 * written.  PA_ERR_ARG if capacity is too small. */
pa_status pa_get_array(pa_ctx *ctx, pa_array which, void *host, size_t capacity, size_t *n_out);

/* Checkpoint restore: replace the population by R_i replicas of packed spins
 * (host, [R_i][ceil(N/32)] words) and families (host, may be NULL for j),
 * and set the completed step count and the running sum of ln Q.  Energies and
 * magnetisations are recomputed on the device.  Because every draw is keyed
 * by (seed, step, slot, site), a restored run continues bit for bit like the
 * uninterrupted one. */
pa_status pa_set_state(pa_ctx *ctx, const uint32_t *spins, const uint32_t *family, uint32_t R_i,
                       int32_t step, double sum_lnQ);

/* Kernel timing for roofline accounting.  When enabled, every following
 * sweep launch is bracketed by CUDA events on the context's stream.
 * pa_sweep_timing synchronises and returns the summed sweep-kernel time in
 * milliseconds, the number of timed launches and the spin updates they did. */
pa_status pa_enable_timing(pa_ctx *ctx, int32_t on);
pa_status pa_sweep_timing(pa_ctx *ctx, double *ms, int64_t *launches, double *updates);

/* Number of kernels this context has launched so far. */
int64_t pa_launch_count(const pa_ctx *ctx);

/* Launch configuration of the sweep kernel: threads per CTA (64, 128, 256, 384 or
 * 512; each CTA holds 32 replicas).  Results do not depend on it, only the
 * speed; the package's autotuner times the candidates and picks one.
 * PA_ERR_ARG for other values. */
pa_status pa_set_sweep_threads(pa_ctx *ctx, int32_t threads);
int32_t pa_get_sweep_threads(const pa_ctx *ctx);

/* Test hook of the sweep kernel (Sec. 2 step 3): per half-sweep the kernel
 * queues the sites whose Metropolis test is still undecided after the first
 * eight bits of the uniforms and finishes them in a second pass; sites that
 * find the queue full finish at once.  cap limits the queue to cap entries
 * (0: every site finishes at once; -1: the kernel's full queue, the default)
 * so that both paths can be checked.  Results do not depend on it.
 * PA_ERR_ARG for cap < -1. */
pa_status pa_set_sweep_queue(pa_ctx *ctx, int32_t cap);

/* Launch configuration of the grouped 3D sweep kernel (Sec. 2 step 3 for 3D
 * lattices of even side 4..16): a CTA holds a number of replica groups that
 * depends on the side; mult = 2 doubles it (fewer, larger CTAs), mult = 1 is
 * the default.  Results do not depend on it; the package's autotuner times both.
 * A context whose runs do not use the grouped kernel accepts mult = 1 only.
 * Synchronises the context's stream.  PA_ERR_ARG for other values,
 * PA_ERR_STATE after an earlier device error.  pa_get_sweep_groups returns the
 * multiple in use (1 without the grouped kernel). */
pa_status pa_set_sweep_groups(pa_ctx *ctx, int32_t mult);
int32_t pa_get_sweep_groups(const pa_ctx *ctx);

/* Test hook of the failure path (no counterpart in the paper).  The scans of the
 * copy numbers (Sec. 2 step 2) are single-pass: a block waits, by a bounded
 * spin, for the prefix its predecessor publishes.  With on = 1 the first block
 * of every run withholds its prefix, so the other blocks' waits run out after
 * their bound (about a second) and the step ends with PA_ERR_TIMEOUT: nothing
 * faults or hangs, and the context then accepts queries and pa_destroy only.
 * on = 0 (the default) restores normal operation before a failure.  PA_ERR_ARG
 * for a null context or another value of on. */
pa_status pa_set_wait_test(pa_ctx *ctx, int32_t on);

/* Reweighting of one temperature step without any device allocation.
 *
 * Some callers cannot call cudaMalloc: code embedded in a host framework that
 * owns all device memory through its own pool (a stray allocation would break
 * its accounting or exceed its budget), services that forbid allocation after
 * start-up because an allocation can block or fail under load, and callers
 * that want the weights of a population they already hold without creating a
 * context and its workspace.  This entry point serves them: it needs only the
 * caller's input and output buffers.  The paper has no counterpart; it is the
 * weights stage of pa_step offered on its own.
 *
 * From the energies E[0..R_prev) (device, int32, each a valid energy of the
 * dim-dimensional periodic L^dim lattice whose number of J = -1 bonds has the
 * given parity), for the step dbeta = beta_i - beta_{i-1} > 0 it writes
 *   *lnQ (device double)          ln Q_i, the same bits as pa_step computes,
 *   f[0..R_prev) (device uint64)  floor(2^40 R w_j / sum_k w_k), w_j the
 *                                 Boltzmann factor of E_j at dbeta: the
 *                                 fixed-point expected copy numbers of pa_step
 *                                 for nominal size R,
 * asynchronously on cuda_stream (NULL = legacy default stream).  If an energy
 * is not a valid one (outside [-dim N, dim N], or (E + dim N)/2 not an integer
 * of the given parity), *lnQ is set to NaN and f is not written.
 *
 * Scratch: one statically allocated device array (about 1.3 MB) that every
 * GPU loading the library holds until the process exits.  Every call shares
 * it and it keeps the last call's contents (the call clears what must start
 * at zero), so calls whose kernels overlap on the GPU -- on different streams,
 * or from several host threads -- race and must be serialised by the caller.
 * Each call looks up the array's device address with the caller's device
 * current; the first call on a device loads the library's device code there,
 * so make that first call before any stream capture begins.
 *
 * Limits: dim*N/2 + 1 <= 65536 energy levels, N <= 32768 sites and R < 2^24,
 * else PA_ERR_LIMIT; other bad arguments give PA_ERR_ARG.  No cudaMalloc,
 * cudaFree or allocating library routine is called. */
pa_status pa_weights_static(const int32_t *E, uint32_t R_prev, uint32_t R, int32_t dim, int32_t L,
                            int32_t parity, double dbeta, double *lnQ, uint64_t *f,
                            void *cuda_stream);

/* ---- batches of runs ------------------------------------------------------
 *
 * A batch advances M independent runs with the same kernels (one launch per
 * phase for all runs).  Run m's draws use the context's seed with run m's
 * identity in the counter: its sweep and initial draws use replica slots
 * offset by 32 x (the sweep CTAs of runs 0..m-1) and its resampling draws carry
 * m; a batch of one run is identical to pa_init.  The single-run calls above
 * act on run 0; pa_set_state needs M = 1. */
size_t pa_batch_workspace_bytes(const pa_run_spec *runs, int32_t M, int32_t n_steps,
                                pa_resampler resampler);
pa_status pa_batch_init(pa_ctx **out, const pa_run_spec *runs, int32_t M,
                        const pa_schedule *sched, pa_resampler resampler, uint64_t seed,
                        void *cuda_stream, void *workspace, size_t workspace_bytes);
int32_t pa_batch_size(const pa_ctx *ctx);
pa_status pa_run_observables(pa_ctx *ctx, int32_t run, pa_obs *out);
pa_status pa_run_trace(pa_ctx *ctx, int32_t run, pa_obs *rows, int32_t max_rows,
                       int32_t *n_rows);
pa_status pa_run_free_energy(pa_ctx *ctx, int32_t run, double *minus_beta_F, double *f_per_spin);
pa_status pa_run_get_array(pa_ctx *ctx, int32_t run, pa_array which, void *host, size_t capacity,
                           size_t *n_out);

/* Synchronise, reduce on the device and copy rows 0..step of the weighted
 * averages of the runs whose ensemble id is `ensemble` (Sec. 4).
 * PA_ERR_ARG if no run has that id. */
pa_status pa_weighted(pa_ctx *ctx, int32_t ensemble, pa_weighted_obs *rows, int32_t max_rows,
                      int32_t *n_rows);


/* One run's summary at one temperature step, for combining runs that were
 * computed anywhere (other GPUs, other processes, other times). */
typedef struct {
    uint32_t R_i;          /* population size at the step                          */
    uint32_t R;            /* nominal population size                              */
    double sum_lnQ;        /* sum_{k<=i} ln Q_k                                     */
    int64_t sumE, sumE2, sumAbsM, sumM2;  /* exact sums over the population         */
    double wsum, wE, wE2, wAM, wM2;  /* weighted sums (partial resampling); wsum = 0 */
                                     /* means: use the exact sums                   */
} pa_run_row;

/* Weighted average (Eq. weighted-averages, Eqs. Wvar_C, Wvar_Chi) of n_runs run
 * summaries of one system (lattice of N sites) at inverse temperature beta;
 * the same combination as pa_weighted, computed on the GPU.  rows: host array,
 * n_runs entries (copied); out: host.  step is copied into out->step.  The
 * call allocates and frees its device buffers and synchronises cuda_stream
 * (nullable).  PA_ERR_ARG for a run with R_i = 0 or R = 0. */
pa_status pa_weighted_rows(const pa_run_row *rows, int32_t n_runs, int32_t N, double beta,
                           int32_t step, pa_weighted_obs *out, void *cuda_stream);

/* Partial resampling (Sec. 3: resampling is needed only once the variance of
 * the importance weights grows too large).  Call after init, before the first
 * step.  Replicas then carry weights w_j (initially 1).  Each step multiplies
 * them by exp(-dbeta (E_j - E_min)) (the same q^l level factors), sets
 *   ln Q_i = ln(sum_j wn_j) - ln(sum_j w_j) - dbeta E_min
 * and resamples (expected copies R wn_j / sum wn, the context's rule) only if
 * the effective size (sum wn)^2 / sum wn^2 is below alpha R_{i-1}; otherwise
 * every replica is kept with its weight (rescaled by a power of two so the
 * largest is in [1/2, 1)).  Sums are balanced binary trees over the replica
 * index in FP64, so counts and decisions are reproducible.  alpha in [0, 1]:
 * 0 never resamples (annealed importance sampling), 1 resamples whenever the
 * weights differ.  Observables become weighted averages (pa_obs).  Every run
 * of the batch needs R_cap <= 16384 x 512; pa_set_state is then unavailable.
 * PA_ERR_ARG for bad arguments or a context that has stepped. */
pa_status pa_set_partial_resampling(pa_ctx *ctx, double alpha);

/* Overlap distribution of two independent populations of one disorder sample
 * (the spin-glass observable P(q) of Sec. 4, Figs. 6 and 7).  Pair p is
 * (run_a[p], run_b[p]), two different runs of this batch with the same lattice
 * and couplings (ideally different seeds, i.e. different run indices).  At the
 * current step, replica slot j of run a is paired with slot j of run b for
 * j < min(R_i^a, R_i^b); the pair's overlap is q = (1/N) sum_s s^a_s s^b_s =
 * 1 - 2k/N with k the number of sites where the two differ.
 *   hist_dev: device array of n_pairs x (N+1) uint32, caller-owned, row-major;
 *             overwritten with the number of replica pairs at each k (a row
 *             whose runs hold a device error is not written).
 *   P_out:    host array of N+1 doubles, or NULL.  When given, receives the
 *             weighted estimate P(k) = sum_p omega_p hist_p[k] / n_p with
 *             omega_p proportional to (R_i^a Zhat_a)(R_i^b Zhat_b), the product
 *             of the two populations' weights of Eq. (weighted-averages), and
 *             the call synchronises; with NULL the histogram kernel is only
 *             enqueued on the context's stream.
 * All runs of the pairs must have the same N; 1 <= n_pairs <= batch size.
 * PA_ERR_ARG otherwise. */
pa_status pa_overlap(pa_ctx *ctx, const int32_t *run_a, const int32_t *run_b, int32_t n_pairs,
                     uint32_t *hist_dev, double *P_out);
/* Replay each temperature step as one captured CUDA graph (default on; needs a
 * non-NULL stream; timing mode launches directly). */
pa_status pa_set_graph(pa_ctx *ctx, int32_t on);

/* ---- learned schedule -----------------------------------------------------
 *
 * Adaptive temperature steps and sweep numbers (cited in Sec. 5 of the paper as
 * established practice) chosen by a small network after every step.  The
 * schedule given to pa_init becomes a grid: beta may only take its values
 * beta[0..K] (K = n_steps), a step advances u = 1..u_max grid points, and the
 * sweeps of all steps together stay within `budget`.  After each step a kernel
 * reads the population statistics (beta, <E>/N, var(E)/N, ln Q, rho_t,
 * family entropy, acceptance rate, L), evaluates an 8 -> 64 -> 64 -> 2 ReLU
 * network with BF16 parameters and FP32 accumulation, and writes the next
 * step's entries into the step tables: outputs s (step relative to the
 * average remaining step) and t (sweeps relative to budget / planned steps).
 * Non-finite or out-of-range outputs, or use_mlp = 0, take the plain step
 * (plain_units, plain_theta).  When beta reaches beta[K] the run finishes:
 * later pa_step calls launch nothing useful and pa_sync reports PA_OK.
 * In a batch every run takes its own steps (one controller CTA per run, the
 * run's own step tables, the same network and settings); runs finish after
 * different step counts, the context once all have finished (PA_ERR_DONE from
 * pa_step), and the per-run calls report each run at its own step.  pa_weighted
 * then returns PA_ERR_ARG (the runs' temperatures differ at a step index).
 * Call before the first pa_step; not with partial resampling (PA_ERR_ARG). */
#define PA_MLP_IN 8
#define PA_MLP_HIDDEN 64
#define PA_MLP_OUT 2
/* parameters in this order: W1[64][8], b1[64], W2[64][64], b2[64], W3[2][64], b3[2] */
#define PA_MLP_NPARAM 4866

typedef struct {
    const uint16_t *params;   /* host, PA_MLP_NPARAM BF16 values; NULL with use_mlp = 0 */
    int32_t use_mlp;
    int32_t plain_units;      /* grid points per plain step                          */
    uint32_t plain_theta;     /* sweeps per plain step                               */
    uint32_t theta_min, theta_max;
    uint32_t budget;          /* total sweeps; 0 = plain_theta * K / plain_units     */
    int32_t u_max;            /* largest step in grid points, 1..8                   */
} pa_controller;

pa_status pa_set_controller(pa_ctx *ctx, const pa_controller *cfg);

/* Synchronise and copy the schedule taken so far: beta[0..step] (host, step+1
 * values) and theta[0..step-1]; *n receives step + 1. */
pa_status pa_schedule_taken(pa_ctx *ctx, double *beta, uint32_t *theta, int32_t max,
                            int32_t *n);
/* The same for run `run` of a batch. */
pa_status pa_run_schedule_taken(pa_ctx *ctx, int32_t run, double *beta, uint32_t *theta,
                                int32_t max, int32_t *n);

/* Training of the network on the device (stateless; all pointers device).
 * X [B][8] features, Yt [B][2] targets, mask [B][2] weights of the squared
 * errors; params [PA_MLP_NPARAM] FP32 master values (the forward pass rounds
 * them to BF16 as inference does).  pa_mlp_gradients writes d(loss)/d(params)
 * with loss = sum mask (y - yt)^2 / (2B); scratch holds pa_mlp_scratch_bytes(B)
 * bytes.  pa_mlp_adam applies one Adam step (step >= 1) and refreshes the BF16
 * copy when params_bf16 != NULL.  pa_mlp_forward evaluates BF16 parameters. */
size_t pa_mlp_scratch_bytes(int32_t B);
pa_status pa_mlp_forward(const uint16_t *params_bf16, const float *X, int32_t B, float *Y,
                         void *cuda_stream);
pa_status pa_mlp_gradients(const float *params, const float *X, const float *Yt,
                           const float *mask, int32_t B, float *grads, float *loss,
                           void *scratch, size_t scratch_bytes, void *cuda_stream);
pa_status pa_mlp_adam(float *params, const float *grads, float *m, float *v,
                      uint16_t *params_bf16, int32_t step, float lr, void *cuda_stream);

/* Release the context (and the device memory it allocated).  NULL is a no-op. */
pa_status pa_destroy(pa_ctx *ctx);

const char *pa_strerror(pa_status s);

#ifdef __cplusplus
}
#endif

#endif /* PA_H */
