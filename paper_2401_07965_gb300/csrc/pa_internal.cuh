// pa_internal.cuh -- device-side definitions shared by the library's kernels.
//
// A context advances a batch of M >= 1 independent runs (same dimension,
// coupling kind, rule and schedule; lattice size, population size, couplings
// and seed-independent identity per run) with the same kernels: one launch per
// phase covers every run.
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11), keyed
// by the 64-bit seed of the context; the counter (c0, c1, c2, c3) carries the
// draw's purpose in the top nibble of c1 and the run's identity:
//   sweep      c0 = global replica group (slot_base + slot) >> 5,
//              c1 = (sweep << 4) | (colour << 3) | plane block, c2 = step, c3 = site
//   init       c0 = word >> 2, c1 = 1 << 28, c2 = 0, c3 = slot_base + replica
//   resample   c0 = index, c1 = (2 << 28) | (run << 8) | rule, c2 = step, c3 = chunk
//   disorder   c0 = bond >> 7, c1 = 3 << 28, c2 = 0, c3 = realization
// slot_base of run m is 32 x (the sweep CTAs of runs 0..m-1); a batch of one
// run has slot_base 0 and run index 0.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pa {

constexpr uint32_t PHILOX_M0 = 0xD2511F53u;
constexpr uint32_t PHILOX_M1 = 0xCD9E8D57u;
constexpr uint32_t PHILOX_W0 = 0x9E3779B9u;
constexpr uint32_t PHILOX_W1 = 0xBB67AE85u;

constexpr uint32_t DOM_SWEEP = 0x00000000u;
constexpr uint32_t DOM_INIT = 0x10000000u;
constexpr uint32_t DOM_RESAMPLE = 0x20000000u;
constexpr uint32_t DOM_DISORDER = 0x30000000u;
constexpr uint32_t RULE_NEAREST = 0u, RULE_SYSTEMATIC = 1u, RULE_MULTINOMIAL = 2u,
                   RULE_RESIDUAL = 3u, RULE_POISSON = 4u;

constexpr int FRAC_BITS = 40;          // tau-hat is carried as a 2^-40 fixed-point integer
// tau-hat_j <= R, so f_j = floor(2^40 tau-hat_j) and T = sum_j f_j <= R 2^40 fit in
// 64 bits only for R < 2^24: the largest nominal population (and capacity)
constexpr uint32_t MAX_POPULATION = (1u << 24) - 1u;
constexpr uint32_t POISSON_KMAX = 256; // per chunk of mean <= 16

enum Method { M_MULTINOMIAL = 0, M_SYSTEMATIC = 1, M_RESIDUAL = 2, M_POISSON = 3, M_NEAREST = 4 };

enum DevStatus { S_OK = 0, S_CAPACITY = 4, S_KMAX = 5, S_TIMEOUT = 6, S_DONE = 8 };

// learned-schedule controller (MLP 8 -> 64 -> 64 -> 2, BF16 parameters)
constexpr int MLP_IN = 8, MLP_HID = 64, MLP_OUT = 2;
constexpr int MLP_NPARAM = MLP_HID * MLP_IN + MLP_HID + MLP_HID * MLP_HID + MLP_HID +
                           MLP_OUT * MLP_HID + MLP_OUT;
constexpr int CTL_UMAX = 8;  // largest step in grid units
constexpr int CLN_TAB = 64;  // family sizes c <= CLN_TAB take c ln c from a table

struct CtlDev {
    uint16_t w[MLP_NPARAM];      // BF16 parameters: W1, b1, W2, b2, W3, b3
    int32_t use_mlp;             // 0: plain steps of plain_units with plain_theta
    int32_t K;                   // grid index of beta_f
    int32_t plain_units;
    uint32_t plain_theta;
    uint32_t theta_min, theta_max;
    uint32_t budget;             // total sweeps
    int32_t u_max;               // <= CTL_UMAX
    float theta_c;               // sweeps per step of the planned step count
    int32_t pad[3];
    const double* beta_grid;     // K + 1
    const uint32_t* thr_grid;    // 4 per grid point
    const double* dbeta_tab;     // (K + 1) x CTL_UMAX: beta[k+u] - beta[k]
    const double* q_tab;         // exp(-4 dbeta_tab)
};

struct uint4x {
    uint32_t x, y, z, w;
};

// One Philox4x32-10 block.  Usable on host (couplings) and device.
__host__ __device__ __forceinline__ uint4x philox(uint32_t c0, uint32_t c1, uint32_t c2,
                                                  uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        c0 = n0;
        c2 = n2;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    return {c0, c1, c2, c3};
}

// 32x32 -> 64-bit product as one wide multiply
__device__ __forceinline__ void mulhilo(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo) {
    const uint64_t p = (uint64_t)a * (uint64_t)b;
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
}

// Device state shared by the kernels of a run (one per context).
struct DevState {
    int32_t step;      // completed temperature steps
    int32_t status;    // DevStatus
    uint32_t R_cur;    // current population size
    uint32_t R_prev;   // size that the last resampling started from
    double sum_lnQ;    // running sum of ln Q_k
    uint32_t lmin;     // lowest occupied energy level of the last resampling
    uint32_t K;        // number of levels spanned
    uint64_t T;        // sum of fixed-point weights f_j
    uint64_t Tres;     // sum of their fractional parts (residual rule)
    uint64_t Rres;     // residual draws
    int32_t kgrid;     // learned schedule: grid index of the current beta
    uint32_t sweeps;   // learned schedule: sweeps spent so far
    int32_t resample;  // partial resampling: this step resamples
    int32_t wexp;      // partial resampling: exponent of the largest new weight
    double S_new;      // partial resampling: sum of the new weights
    uint32_t epoch;    // resampling steps taken (tags the look-back descriptors)
    int32_t kmax;      // a Poisson inversion of this step hit its limit
    int32_t hlo, hhi;  // lowest / highest histogram level filled since the last reweighting
};

// Look-back descriptor of one scan block (single-pass scans of the resampling
// step): the block's aggregate, then its inclusive prefix, published with a
// flag tagged by the step's epoch (2e+1: aggregate, 2e+2: inclusive prefix).
struct LBDesc {
    uint32_t flag;
    uint32_t pad;
    unsigned long long agg[2];
    unsigned long long inc[2];
    unsigned long long pad2;
};

// Per-step accumulators, device-resident (row i = after temperature step i).
struct TraceRow {
    double lnQ;
    double sum_lnQ;
    double c_ln_c;   // sum_k c_k ln c_k over families
    double sv_sum;   // sum_j (r_j - f_j 2^-40)^2 over parents
    unsigned long long sumE, sumE2, sumAbsM, sumM2, sumC2, accepts;  // two's complement
    uint32_t R_i, R_prev;
    float x[8];       // learned schedule: features seen by the controller after this step
    int32_t u_next;   // its choice: grid units of the next step (0 = none)
    uint32_t theta_next;  // and the sweeps of the next step
    // partial resampling: effective size of the reweighted population, whether
    // the step resampled, and the weighted sums sum_j w_j O_j after the sweeps
    double ess;
    int32_t resampled, pad;
    double wsum, wE, wE2, wAM, wM2;
};

// Per-run description, in device memory (one per run of the batch).
struct RunDesc {
    int L, N, W, Wp;         // lattice; W words per replica, Wp padded to 4
    int nlev;                // d*N/2 + 1 histogram levels (level = U >> 1)
    int parity;              // U mod 2, the same for every configuration
    uint32_t R, Rcap;
    uint32_t magicL, shiftL; // fast division by L
    int nblk;                // scan blocks of this run
    uint32_t blk0;           // its first block in the flattened scan grids
    uint32_t grp0;           // its first CTA in the flattened sweep grid (= slot_base / 32)
    uint32_t run;            // run index
    uint32_t cta0;           // 3D kernel: its first CTA in the launch for its side
    double lnR;              // ln max(R, 2), from the host's log (the controller's entropy scale)
    uint32_t* spins[2];
    int32_t* E[2];
    uint32_t* fam[2];
    int32_t* M;
    uint32_t* anc;
    uint32_t* counts;
    uint64_t* C;             // inclusive prefix of f
    uint64_t* G;             // inclusive prefix of the remainders (residual rule)
    uint32_t* hist;          // level histogram of the current population
    uint64_t* flev;          // fixed-point tau-hat per level
    double* tree;            // pairwise-sum scratch (power of two >= nlev)
    uint64_t* partA;         // per-block partial sums
    uint64_t* partB;
    uint64_t* offA;          // per-block exclusive offsets
    uint64_t* offB;
    double* partD;
    double* partCL;
    double* w;               // partial resampling: replica weights
    double* wpart;           // per-block tree sums of the weights (4 per block)
    double* opart;           // per-block tree sums of the weighted observables (5 per block)
    const uint8_t* jbits;    // bit a of byte s: bond (s, s+e_a) has J = -1
    DevState* st;
    TraceRow* trace;         // n_steps + 1 rows
    // the run's step tables (beta_i, dbeta_i, q_i, thresholds, theta_i): the batch's
    // shared tables, or the run's own under the learned schedule
    double* sbeta;
    double* sdbeta;
    double* sq;
    uint32_t* sthr;
    uint32_t* stheta;
    LBDesc* lb1;             // look-back descriptors: prefix of the expected copies
    LBDesc* lb2;             // and of the copy numbers
    uint32_t* tick;          // [0] scan-block tickets, [1] family-block tickets
};

// Batch-wide parameters, passed by value to every kernel.
struct KParams {
    int d, ea, method, n_steps, M;
    int maxN;                // largest lattice of the batch
    uint32_t k0, k1;         // Philox key = seed
    uint32_t rk0[10], rk1[10];  // its round keys k + r*W (round r = 0..9)
    uint32_t nblk_total;     // flattened scan grid
    uint32_t ngrp_total;     // flattened sweep grid
    const RunDesc* runs;
    const uint32_t* blk2run; // scan block -> run
    const uint32_t* grp2run; // sweep CTA -> run
    const double* beta;      // n_steps + 1
    const double* dbeta;     // n_steps
    const double* q;         // exp(-4 dbeta), n_steps
    const uint32_t* thr;     // 4 per step (index 1..d used)
    const uint32_t* theta;   // n_steps
    const CtlDev* ctl;       // null without a controller
    double alpha;            // partial resampling threshold (< 0: resample every step)
    int qcap_limit;          // sweep: cap on the undecided-site queue (< 0: its full size)
    int lb_hold;             // test: scan block 0 withholds its prefix (the waits run out)
    const double* clnc;      // c ln c for c = 0 .. CLN_TAB (0 for c < 2), from the host's log
    int L_all;               // the side L shared by every run of the batch (0 if they differ)
    // 3D kernel plan: one launch per distinct side (n3 = 0: the general kernel)
    int n3;
    int L3[4];
    int g3mul;               // groups per CTA: the side's base count times this (1 or 2)
    const uint32_t* c3map[4];  // CTA -> run of each launch
    uint32_t n3cta[4];
};

// partial resampling: blocks of a run whose tree sums one CTA can finish
constexpr int PARTIAL_MAX_BLOCKS = 16384;
static_assert(PARTIAL_MAX_BLOCKS % 1024 == 0, "leaves per thread of the final trees");

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 2;
constexpr int SCAN_CHUNK = SCAN_THREADS * SCAN_ITEMS;

}  // namespace pa

// kernel launchers (defined in the .cu files)
namespace pa {
cudaError_t launch_init_spins(const KParams& p, const RunDesc* host_runs, cudaStream_t s);
cudaError_t launch_measure(const KParams& p, int threads, cudaStream_t s);
cudaError_t launch_resample(const KParams& p, cudaStream_t s, int64_t* launches);
cudaError_t launch_partial_init(const KParams& p, cudaStream_t s);
cudaError_t launch_sweep(const KParams& p, int threads, cudaStream_t s);
cudaError_t launch_family_finish(const KParams& p, int mode, cudaStream_t s, int64_t* launches);
cudaError_t prepare_sweep(const KParams& p, int threads);
cudaError_t launch_sweep2d(const KParams& p, int threads, cudaStream_t s, bool attr_only,
                           bool* done);
int sweep3d_groups(int L, int gm);
cudaError_t launch_sweep3d(const KParams& p, int L, const uint32_t* cta2run, uint32_t ncta,
                           cudaStream_t s, bool attr_only);
cudaError_t launch_control(const KParams& p, cudaStream_t s);
int sweep_threads(int N);
bool sweep_threads_supported(int t);
}  // namespace pa
