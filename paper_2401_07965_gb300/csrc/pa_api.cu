// pa_api.cu -- the C ABI of include/pa.h: contexts (batches of runs), device
// workspace, host precomputation of the per-step tables, and the launch
// sequence of a temperature step (Sec. 2 steps 2-4), replayed as a CUDA graph.
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <algorithm>

#include "../../include/pa.h"
#include "pa_internal.cuh"

namespace pa {
cudaError_t launch_weighted(const KParams& p, const int32_t* run_ids, int n_runs, int n_rows,
                            pa_weighted_obs* out, cudaStream_t s);
cudaError_t launch_overlap(const KParams& p, const int32_t* pairs, int n_pairs, int Wp,
                           uint32_t max_rows, int bins, uint32_t* hist, double* P,
                           uint32_t* acc, uint32_t* tickets, cudaStream_t s);
}

using namespace pa;

namespace {

struct RunHost {
    int L, N, W, Wp, nlev, P;
    uint32_t R, Rcap;
    int nblk, ngrp;
    int g3, nct3;            // 3D kernel: replica groups per CTA, CTAs (0: not eligible)
    int ensemble;
    std::vector<uint8_t> jb;
    int parity;
};

enum Region {
    R_SPIN0, R_SPIN1, R_E0, R_E1, R_F0, R_F1, R_M, R_ANC, R_CNT, R_C, R_G, R_HIST, R_FLEV, R_TREE,
    R_PA, R_PB, R_OA, R_OB, R_PD, R_PCL, R_W, R_WP, R_OP, R_JB, R_ST, R_TRACE, R_LB1, R_LB2,
    R_TICK, R_SB, R_SDB, R_SQ, R_STHR, R_STH, R_COUNT
};

enum Shared {
    S_RUNS, S_B2R, S_G2R, S_BETA, S_DBETA, S_Q, S_THR, S_THETA, S_IDS, S_WOUT,
    S_CTL, S_GBETA, S_GTHR, S_GDB, S_GQ, S_PAIRS, S_POV, S_OVACC, S_OVTICK, S_C3, S_CLNC,
    S_COUNT
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t shared_off[S_COUNT];
    std::vector<std::array<size_t, R_COUNT>> run_off;
    size_t total = 0;
};

}  // namespace

struct pa_ctx {
    KParams kp;
    std::vector<RunHost> runs;
    std::vector<RunDesc> desc;
    int d = 0, n_steps = 0, method = 0, M = 0;
    uint64_t seed = 0;
    cudaStream_t stream = nullptr;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    bool owns = false;
    int host_step = 0;
    int threads = 64;
    int64_t launches = 0;
    pa_status sticky = PA_OK;
    bool timing = false;
    bool use_graph = true;
    cudaGraphExec_t graph = nullptr;
    int graph_threads = 0;
    int64_t graph_kernels = 0;
    std::vector<cudaEvent_t> ev_start, ev_stop;  // pool of timing events, reused
    size_t ev_used = 0;
    std::vector<int> timed_steps;
    std::vector<double> beta;
    std::vector<uint32_t> theta;
    int32_t* d_ids = nullptr;               // run index list for pa_weighted (device)
    pa_weighted_obs* d_wout = nullptr;      // its output rows (device)
    int32_t* d_pairs = nullptr;             // run pairs for pa_overlap (device)
    double* d_pov = nullptr;                // its weighted P(q) (device)
    uint32_t* d_ovacc = nullptr;            // its per-pair accumulators (zero between calls)
    uint32_t* d_ovtick = nullptr;           // and per-pair CTA tickets (zero between calls)
    std::vector<int32_t> pairs_cached;      // the pair list currently in d_pairs
    bool controlled = false;                // learned schedule active
    std::vector<std::vector<double>> rbeta;     // learned schedule: each run's betas and
    std::vector<std::vector<uint32_t>> rtheta;  // sweeps so far (host copies)
    std::vector<int> rstep;                     // and its completed steps
    std::vector<char> rdone;                    // beta_f reached
    std::vector<std::array<size_t, 5>> rtab_off;  // offsets of its own step tables
    bool finished = false;                  // beta_f reached under the controller
    CtlDev* d_ctl = nullptr;
    double* d_gbeta = nullptr;
    uint32_t* d_gthr = nullptr;
    double* d_gdb = nullptr;
    double* d_gq = nullptr;
};

namespace {

bool check_lattice(const pa_lattice* lat, long long* N) {
    if (!lat || lat->dim < 2 || lat->dim > 3 || lat->L < 2 || (lat->L & 1)) return false;
    long long n = 1;
    for (int a = 0; a < lat->dim; ++a) n *= lat->L;
    if (n > 32768) return false;  // the sweep keeps a lattice of 32 replicas in shared memory
    *N = n;
    return true;
}

uint32_t default_cap(uint32_t R, int method) {
    if (method == PA_POISSON || method == PA_NEAREST)
        return R + (uint32_t)std::ceil(10.0 * std::sqrt((double)R)) + 64u;
    return R;
}

// geometry and sizes of each run; couplings are filled by fill_couplings.
// PA_ERR_LIMIT for a population or capacity of 2^24 or more, PA_ERR_ARG for
// other invalid specifications.
pa_status make_runs(const pa_run_spec* specs, int M, int method, std::vector<RunHost>* out,
                    int* d) {
    if (!specs || M < 1 || M > (1 << 20) || method < 0 || method > 4) return PA_ERR_ARG;
    out->clear();
    for (int m = 0; m < M; ++m) {
        const pa_run_spec& s = specs[m];
        long long N;
        if (!check_lattice(&s.lattice, &N)) return PA_ERR_ARG;
        if (m == 0) *d = s.lattice.dim;
        if (s.lattice.dim != *d) return PA_ERR_ARG;
        if (s.R == 0 || s.ensemble < 0) return PA_ERR_ARG;
        if (s.couplings.kind < 0 || s.couplings.kind > 2) return PA_ERR_ARG;
        if ((s.couplings.kind == PA_COUPLING_FERRO) !=
            (specs[0].couplings.kind == PA_COUPLING_FERRO))
            return PA_ERR_ARG;
        if (s.couplings.kind == PA_COUPLING_EXPLICIT && !s.couplings.J) return PA_ERR_ARG;
        if (s.R > MAX_POPULATION || s.R_cap > MAX_POPULATION) return PA_ERR_LIMIT;
        RunHost h;
        h.L = s.lattice.L;
        h.N = (int)N;
        h.W = (int)((N + 31) / 32);
        h.Wp = (h.W + 3) & ~3;
        h.nlev = (int)(*d * N / 2 + 1);
        h.P = 1;
        while (h.P < h.nlev) h.P <<= 1;
        h.R = s.R;
        h.Rcap = s.R_cap ? s.R_cap : default_cap(s.R, method);
        if (h.Rcap < h.R) return PA_ERR_ARG;
        if (h.Rcap > MAX_POPULATION) return PA_ERR_LIMIT;
        h.nblk = (int)((h.Rcap + SCAN_CHUNK - 1) / SCAN_CHUNK);
        h.ngrp = (int)((h.Rcap + 31) / 32);
        h.g3 = (*d == 3) ? sweep3d_groups(h.L, 1) : 0;
        h.nct3 = h.g3 ? (h.ngrp + h.g3 - 1) / h.g3 : 0;
        h.ensemble = s.ensemble;
        h.parity = 0;
        out->push_back(std::move(h));
    }
    return PA_OK;
}

Layout make_layout(const std::vector<RunHost>& runs, int n_steps) {
    Layout L;
    size_t nblk = 0, ngrp = 0;
    for (const RunHost& h : runs) {
        nblk += h.nblk;
        ngrp += h.ngrp;
    }
    const size_t M = runs.size();
    size_t sz[S_COUNT];
    sz[S_RUNS] = M * sizeof(RunDesc);
    sz[S_B2R] = nblk * 4;
    sz[S_G2R] = ngrp * 4;
    sz[S_BETA] = (size_t)(n_steps + 1) * 8;
    sz[S_DBETA] = sz[S_Q] = (size_t)n_steps * 8;
    sz[S_THR] = (size_t)n_steps * 16;
    sz[S_THETA] = (size_t)n_steps * 4;
    sz[S_IDS] = M * 4;
    sz[S_WOUT] = (size_t)(n_steps + 1) * sizeof(pa_weighted_obs);
    sz[S_CTL] = sizeof(CtlDev);
    sz[S_GBETA] = (size_t)(n_steps + 1) * 8;
    sz[S_GTHR] = (size_t)(n_steps + 1) * 16;
    sz[S_GDB] = sz[S_GQ] = (size_t)(n_steps + 1) * CTL_UMAX * 8;
    int maxN = 0;
    for (const RunHost& h : runs) maxN = h.N > maxN ? h.N : maxN;
    sz[S_PAIRS] = M * 2 * 4;
    sz[S_POV] = (size_t)(maxN + 1) * 8;
    sz[S_OVACC] = M * (size_t)(maxN + 1) * 4;  // overlap accumulators, zero between calls
    sz[S_OVTICK] = M * 4;
    size_t nct3 = 0;
    for (const RunHost& h : runs) nct3 += (size_t)h.nct3;
    sz[S_C3] = nct3 * 4;
    sz[S_CLNC] = (CLN_TAB + 1) * 8;
    size_t o = 0;
    for (int r = 0; r < S_COUNT; ++r) {
        L.shared_off[r] = o;
        o += align256(sz[r]);
    }
    for (const RunHost& h : runs) {
        std::array<size_t, R_COUNT> off;
        size_t rs[R_COUNT];
        const size_t rows = h.Rcap;
        rs[R_SPIN0] = rs[R_SPIN1] = rows * h.Wp * 4;
        rs[R_E0] = rs[R_E1] = rs[R_F0] = rs[R_F1] = rs[R_M] = rs[R_ANC] = rs[R_CNT] = rows * 4;
        rs[R_C] = rs[R_G] = rows * 8;
        rs[R_HIST] = (size_t)h.nlev * 4;
        rs[R_FLEV] = (size_t)h.nlev * 8;
        rs[R_TREE] = (size_t)h.P * 8;
        rs[R_PA] = rs[R_PB] = rs[R_OA] = rs[R_OB] = rs[R_PD] = rs[R_PCL] = (size_t)h.nblk * 8;
        rs[R_W] = rows * 8;
        rs[R_WP] = (size_t)h.nblk * 4 * 8;
        rs[R_OP] = (size_t)h.nblk * 5 * 8;
        rs[R_JB] = (size_t)h.N;
        rs[R_ST] = sizeof(DevState);
        rs[R_TRACE] = (size_t)(n_steps + 1) * sizeof(TraceRow);
        rs[R_LB1] = rs[R_LB2] = (size_t)h.nblk * sizeof(LBDesc);
        rs[R_TICK] = 2 * sizeof(uint32_t);
        // the run's own step tables (used under the learned schedule)
        rs[R_SB] = (size_t)(n_steps + 1) * 8;
        rs[R_SDB] = rs[R_SQ] = (size_t)n_steps * 8;
        rs[R_STHR] = (size_t)n_steps * 16;
        rs[R_STH] = (size_t)n_steps * 4;
        for (int r = 0; r < R_COUNT; ++r) {
            off[r] = o;
            o += align256(rs[r]);
        }
        L.run_off.push_back(off);
    }
    L.total = o;
    return L;
}

// magic multiplier for s / L with s < 2^21: (s * m) >> sh
bool make_magic(int L, int N, uint32_t* m_out, uint32_t* sh_out) {
    int lg = 0;
    while ((1 << lg) < L) ++lg;
    for (int sh = 21 + lg; sh < 40; ++sh) {
        const uint64_t m = ((uint64_t)1 << sh) / (uint64_t)L + 1;
        if (m >= ((uint64_t)1 << 32)) break;
        bool ok = true;
        for (int s = 0; s < N && ok; ++s)
            if ((int)(((uint64_t)s * m) >> sh) != s / L) ok = false;
        if (ok) {
            *m_out = (uint32_t)m;
            *sh_out = (uint32_t)sh;
            return true;
        }
    }
    return false;
}

// couplings: bit a of byte s is set when the bond (s, s + e_a) has J = -1
bool fill_couplings(RunHost& h, int d, const pa_couplings& cpl) {
    h.jb.assign((size_t)h.N, 0);
    int nneg = 0;
    if (cpl.kind == PA_COUPLING_EA_PM) {
        const uint32_t dk0 = (uint32_t)(cpl.disorder_seed & 0xFFFFFFFFu);
        const uint32_t dk1 = (uint32_t)(cpl.disorder_seed >> 32);
        for (int b = 0; b < d * h.N; ++b) {
            const uint4x x =
                philox((uint32_t)(b >> 7), DOM_DISORDER, 0u, cpl.realization, dk0, dk1);
            const uint32_t lanes[4] = {x.x, x.y, x.z, x.w};
            if ((lanes[(b >> 5) & 3] >> (b & 31)) & 1u) {
                h.jb[b % h.N] |= (uint8_t)(1u << (b / h.N));
                ++nneg;
            }
        }
    } else if (cpl.kind == PA_COUPLING_EXPLICIT) {
        for (int b = 0; b < d * h.N; ++b) {
            const int8_t j = cpl.J[b];
            if (j != 1 && j != -1) return false;
            if (j == -1) {
                h.jb[b % h.N] |= (uint8_t)(1u << (b / h.N));
                ++nneg;
            }
        }
    }
    h.parity = nneg & 1;
    return true;
}

pa_status map_dev_status(int s) {
    switch (s) {
        case S_OK: return PA_OK;
        case S_CAPACITY: return PA_ERR_CAPACITY;
        case S_KMAX: return PA_ERR_POISSON_KMAX;
        case S_TIMEOUT: return PA_ERR_TIMEOUT;
        default: return PA_ERR_STATE;
    }
}

#define PA_CUDA(call)                  \
    do {                               \
        cudaError_t e_ = (call);       \
        if (e_ != cudaSuccess) {       \
            ctx->sticky = PA_ERR_CUDA; \
            return PA_ERR_CUDA;        \
        }                              \
    } while (0)

// look-back descriptors and block tickets start at zero (epoch 0 tags nothing)
cudaError_t clear_lookback(const RunDesc& r, const RunHost& h, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(r.lb1, 0, (size_t)h.nblk * sizeof(LBDesc), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(r.lb2, 0, (size_t)h.nblk * sizeof(LBDesc), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(r.tick, 0, 2 * sizeof(uint32_t), s);
    return e;
}

pa_status read_state(pa_ctx* ctx, int run, DevState* st) {
    PA_CUDA(cudaStreamSynchronize(ctx->stream));
    PA_CUDA(cudaMemcpy(st, ctx->desc[run].st, sizeof(DevState), cudaMemcpyDeviceToHost));
    return PA_OK;
}

pa_status enqueue_measure(pa_ctx* ctx) {
    PA_CUDA(launch_measure(ctx->kp, ctx->threads, ctx->stream));
    ctx->launches += 1;
    PA_CUDA(launch_family_finish(ctx->kp, 1, ctx->stream, &ctx->launches));
    return PA_OK;
}

void fill_obs(const pa_ctx* ctx, int run, const TraceRow& t, int step, pa_obs* o) {
    std::memset(o, 0, sizeof(*o));
    const double N = ctx->runs[run].N;
    o->step = step;
    o->R_i = t.R_i;
    o->R_prev = t.R_prev;
    o->beta = ctx->controlled ? ctx->rbeta[run][step] : ctx->beta[step];
    o->lnQ = t.lnQ;
    o->sum_lnQ = t.sum_lnQ;
    o->sumE = (int64_t)t.sumE;
    o->sumE2 = (int64_t)t.sumE2;
    o->sumAbsM = (int64_t)t.sumAbsM;
    o->sumM2 = (int64_t)t.sumM2;
    o->sumC2 = (int64_t)t.sumC2;
    o->accepts = t.accepts;
    const double R = t.R_i ? (double)t.R_i : 1.0;
    o->entropy = std::log(R) - t.c_ln_c / R;
    o->sv = (step > 0 && t.R_prev) ? t.sv_sum / (double)t.R_prev : 0.0;
    if (ctx->kp.alpha >= 0.0 && t.wsum > 0.0) {
        // partial resampling: weighted averages
        o->e = t.wE / (t.wsum * N);
        o->e2 = t.wE2 / (t.wsum * N * N);
        o->absm = t.wAM / (t.wsum * N);
        o->m2 = t.wM2 / (t.wsum * N * N);
        o->ess = t.ess;
        o->resampled = t.resampled;
    } else {
        o->e = (double)o->sumE / (R * N);
        o->e2 = (double)o->sumE2 / (R * N * N);
        o->absm = (double)o->sumAbsM / (R * N);
        o->m2 = (double)o->sumM2 / (R * N * N);
        o->ess = (double)t.R_i;
        o->resampled = 1;
    }
    o->c = o->beta * o->beta * N * (o->e2 - o->e * o->e);
    o->chi = o->beta * N * (o->m2 - o->absm * o->absm);
    o->rho_t = (double)o->sumC2 / R;
    const double th =
        step > 0 ? (double)(ctx->controlled ? ctx->rtheta[run][step - 1] : ctx->theta[step - 1])
                 : 0.0;
    o->accept_rate = th > 0 ? (double)o->accepts / (th * N * R) : 0.0;
    for (int k = 0; k < 8; ++k) o->features[k] = t.x[k];
    o->u_next = t.u_next;
    o->theta_next = t.theta_next;
}

// The grouped 3D kernel's CTA plan for group multiple gm: for each distinct side,
// the CTAs of its runs in run order (the CTA -> run map, from p.c3map[0] on, and
// each run's first CTA); the side's groups per CTA are its base count times gm.
void plan3d(pa_ctx* ctx, int gm, std::vector<uint32_t>& c3) {
    KParams& p = ctx->kp;
    c3.clear();
    uint32_t* base3 = const_cast<uint32_t*>(p.c3map[0]);
    for (int k = 0; k < p.n3; ++k) {
        p.c3map[k] = base3 + c3.size();
        const int G = sweep3d_groups(p.L3[k], gm);
        uint32_t n = 0;
        for (int m = 0; m < (int)ctx->runs.size(); ++m) {
            RunHost& h = ctx->runs[m];
            if (h.L != p.L3[k]) continue;
            h.nct3 = (h.ngrp + G - 1) / G;
            ctx->desc[m].cta0 = n;
            for (int c = 0; c < h.nct3; ++c) c3.push_back((uint32_t)m);
            n += (uint32_t)h.nct3;
        }
        p.n3cta[k] = n;
    }
    p.g3mul = gm;
}

// all kernels of one temperature step (and the controller's choice of the next)
pa_status enqueue_step(pa_ctx* ctx, int64_t* launches) {
    PA_CUDA(launch_resample(ctx->kp, ctx->stream, launches));
    PA_CUDA(launch_sweep(ctx->kp, ctx->threads, ctx->stream));
    if (launches) *launches += 1;
    // the family kernel's last CTA of each run also takes the controller's decision
    PA_CUDA(launch_family_finish(ctx->kp, 0, ctx->stream, launches));
    return PA_OK;
}

// Metropolis thresholds at beta: floor(2^32 exp(-4 k beta)), k = 1..3
void thresholds_at(double beta, uint32_t out[4]) {
    out[0] = 0xFFFFFFFFu;
    for (int k = 1; k < 4; ++k) {
        const double x = beta * (double)(4 * k);
        const double t = std::ldexp(std::exp(-x), 32);
        out[k] = (t >= 4294967295.0) ? 0xFFFFFFFFu : (uint32_t)std::floor(t);
    }
}

// copy the step tables written by the controller back to the host
pa_status refresh_schedule(pa_ctx* ctx) {
    const int n = ctx->n_steps;
    for (int m = 0; m < ctx->M; ++m) {
        PA_CUDA(cudaMemcpy(ctx->rbeta[m].data(), ctx->desc[m].sbeta, sizeof(double) * (n + 1),
                           cudaMemcpyDeviceToHost));
        PA_CUDA(cudaMemcpy(ctx->rtheta[m].data(), ctx->desc[m].stheta, sizeof(uint32_t) * n,
                           cudaMemcpyDeviceToHost));
    }
    return PA_OK;
}

// completed steps of one run (runs of a controlled batch advance separately)
int run_step(const pa_ctx* ctx, int run) {
    return ctx->controlled ? ctx->rstep[run] : ctx->host_step;
}
double run_beta(const pa_ctx* ctx, int run, int i) {
    return ctx->controlled ? ctx->rbeta[run][i] : ctx->beta[i];
}
uint32_t run_theta(const pa_ctx* ctx, int run, int i) {
    return ctx->controlled ? ctx->rtheta[run][i] : ctx->theta[i];
}

// capture one temperature step; every kernel reads the step index and the
// population sizes from device memory, so the same graph serves every step
pa_status build_graph(pa_ctx* ctx) {
    if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    PA_CUDA(prepare_sweep(ctx->kp, ctx->threads));
    cudaGraph_t g = nullptr;
    PA_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    int64_t n = 0;
    const pa_status s = enqueue_step(ctx, &n);
    const cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    if (s != PA_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) {
        ctx->sticky = PA_ERR_CUDA;
        return PA_ERR_CUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&ctx->graph, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        ctx->graph = nullptr;
        ctx->sticky = PA_ERR_CUDA;
        return PA_ERR_CUDA;
    }
    ctx->graph_threads = ctx->threads;
    ctx->graph_kernels = n;
    return PA_OK;
}

bool valid_schedule(const pa_schedule* sched) {
    if (!sched || !sched->beta || !sched->theta || sched->n_steps < 1) return false;
    const int n = sched->n_steps;
    if (sched->beta[0] != 0.0) return false;
    for (int i = 1; i <= n; ++i)
        if (!(sched->beta[i] > sched->beta[i - 1]) || !std::isfinite(sched->beta[i])) return false;
    for (int i = 0; i < n; ++i)
        if (sched->theta[i] >= (1u << 24)) return false;
    return true;
}

bool valid_run(const pa_ctx* ctx, int run) { return ctx && run >= 0 && run < ctx->M; }

// n more start/stop event pairs for timing mode (created outside the timed steps)
pa_status grow_event_pool(pa_ctx* ctx, size_t n) {
    for (size_t k = 0; k < n; ++k) {
        cudaEvent_t a = nullptr, b = nullptr;
        PA_CUDA(cudaEventCreate(&a));
        if (cudaEventCreate(&b) != cudaSuccess) {
            cudaEventDestroy(a);
            ctx->sticky = PA_ERR_CUDA;
            return PA_ERR_CUDA;
        }
        ctx->ev_start.push_back(a);
        ctx->ev_stop.push_back(b);
    }
    return PA_OK;
}

}  // namespace

extern "C" {

size_t pa_batch_workspace_bytes(const pa_run_spec* runs, int32_t M, int32_t n_steps,
                                pa_resampler resampler) {
    std::vector<RunHost> rh;
    int d = 0;
    if (n_steps < 1 || make_runs(runs, M, (int)resampler, &rh, &d) != PA_OK) return 0;
    return make_layout(rh, n_steps).total;
}

size_t pa_workspace_bytes(const pa_lattice* lat, uint32_t R, uint32_t R_cap, int32_t n_steps,
                          pa_resampler resampler) {
    if (!lat) return 0;
    pa_run_spec s;
    std::memset(&s, 0, sizeof(s));
    s.lattice = *lat;
    s.couplings.kind = PA_COUPLING_FERRO;
    s.R = R;
    s.R_cap = R_cap;
    return pa_batch_workspace_bytes(&s, 1, n_steps, resampler);
}

pa_status pa_batch_init(pa_ctx** out, const pa_run_spec* specs, int32_t M,
                        const pa_schedule* sched, pa_resampler resampler, uint64_t seed,
                        void* cuda_stream, void* workspace, size_t workspace_bytes) {
    if (!out) return PA_ERR_ARG;
    *out = nullptr;
    if (!valid_schedule(sched)) return PA_ERR_ARG;
    std::vector<RunHost> rh;
    int d = 0;
    const pa_status ms = make_runs(specs, M, (int)resampler, &rh, &d);
    if (ms != PA_OK) return ms;
    for (int m = 0; m < M; ++m)
        if (!fill_couplings(rh[m], d, specs[m].couplings)) return PA_ERR_ARG;
    const int n = sched->n_steps;

    pa_ctx* ctx = new (std::nothrow) pa_ctx();
    if (!ctx) return PA_ERR_NOMEM;
    ctx->d = d;
    ctx->M = M;
    ctx->n_steps = n;
    ctx->method = (int)resampler;
    ctx->seed = seed;
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->beta.assign(sched->beta, sched->beta + n + 1);
    ctx->theta.assign(sched->theta, sched->theta + n);
    int maxN = 0;
    for (const RunHost& h : rh) maxN = h.N > maxN ? h.N : maxN;
    ctx->threads = sweep_threads(maxN);
    ctx->runs = std::move(rh);

    const Layout lay = make_layout(ctx->runs, n);
    if (workspace) {
        if (workspace_bytes < lay.total || ((uintptr_t)workspace & 255u)) {
            delete ctx;
            return PA_ERR_NOMEM;
        }
        ctx->ws = workspace;
        ctx->ws_bytes = workspace_bytes;
        ctx->owns = false;
    } else {
        if (cudaMalloc(&ctx->ws, lay.total) != cudaSuccess) {
            delete ctx;
            return PA_ERR_NOMEM;
        }
        ctx->ws_bytes = lay.total;
        ctx->owns = true;
    }
    char* base = (char*)ctx->ws;

    // batch-wide parameters
    KParams& p = ctx->kp;
    std::memset(&p, 0, sizeof(p));
    p.d = d;
    p.ea = specs[0].couplings.kind != PA_COUPLING_FERRO;
    p.method = (int)resampler;
    p.n_steps = n;
    p.M = M;
    p.maxN = maxN;
    p.k0 = (uint32_t)(seed & 0xFFFFFFFFu);
    p.k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        p.rk0[r] = p.k0 + (uint32_t)r * PHILOX_W0;
        p.rk1[r] = p.k1 + (uint32_t)r * PHILOX_W1;
    }
    p.runs = (const RunDesc*)(base + lay.shared_off[S_RUNS]);
    p.blk2run = (const uint32_t*)(base + lay.shared_off[S_B2R]);
    p.grp2run = (const uint32_t*)(base + lay.shared_off[S_G2R]);
    p.beta = (const double*)(base + lay.shared_off[S_BETA]);
    p.dbeta = (const double*)(base + lay.shared_off[S_DBETA]);
    p.q = (const double*)(base + lay.shared_off[S_Q]);
    p.thr = (const uint32_t*)(base + lay.shared_off[S_THR]);
    p.theta = (const uint32_t*)(base + lay.shared_off[S_THETA]);
    p.clnc = (const double*)(base + lay.shared_off[S_CLNC]);
    ctx->d_ids = (int32_t*)(base + lay.shared_off[S_IDS]);
    ctx->d_wout = (pa_weighted_obs*)(base + lay.shared_off[S_WOUT]);
    ctx->d_pairs = (int32_t*)(base + lay.shared_off[S_PAIRS]);
    ctx->d_pov = (double*)(base + lay.shared_off[S_POV]);
    ctx->d_ovacc = (uint32_t*)(base + lay.shared_off[S_OVACC]);
    ctx->d_ovtick = (uint32_t*)(base + lay.shared_off[S_OVTICK]);
    p.ctl = nullptr;
    p.alpha = -1.0;
    p.qcap_limit = -1;
    p.lb_hold = 0;
    p.n3 = 0;
    p.g3mul = 1;
    p.L_all = ctx->runs[0].L;
    for (const RunHost& h : ctx->runs)
        if (h.L != p.L_all) p.L_all = 0;
    ctx->d_ctl = (CtlDev*)(base + lay.shared_off[S_CTL]);
    ctx->d_gbeta = (double*)(base + lay.shared_off[S_GBETA]);
    ctx->d_gthr = (uint32_t*)(base + lay.shared_off[S_GTHR]);
    ctx->d_gdb = (double*)(base + lay.shared_off[S_GDB]);
    ctx->d_gq = (double*)(base + lay.shared_off[S_GQ]);

    // per-run descriptors and block -> run maps
    std::vector<uint32_t> b2r, g2r;
    ctx->desc.resize(M);
    uint32_t blk0 = 0, grp0 = 0;
    for (int m = 0; m < M; ++m) {
        const RunHost& h = ctx->runs[m];
        const auto& off = lay.run_off[m];
        RunDesc& r = ctx->desc[m];
        std::memset(&r, 0, sizeof(r));
        r.L = h.L;
        r.N = h.N;
        r.W = h.W;
        r.Wp = h.Wp;
        r.nlev = h.nlev;
        r.parity = h.parity;
        r.R = h.R;
        r.lnR = std::log(std::max((double)h.R, 2.0));
        r.Rcap = h.Rcap;
        if (!make_magic(h.L, h.N, &r.magicL, &r.shiftL)) {
            pa_destroy(ctx);
            return PA_ERR_ARG;
        }
        r.nblk = h.nblk;
        r.blk0 = blk0;
        r.grp0 = grp0;
        r.run = (uint32_t)m;
        for (int b = 0; b < h.nblk; ++b) b2r.push_back((uint32_t)m);
        for (int g = 0; g < h.ngrp; ++g) g2r.push_back((uint32_t)m);
        blk0 += h.nblk;
        grp0 += h.ngrp;
        r.spins[0] = (uint32_t*)(base + off[R_SPIN0]);
        r.spins[1] = (uint32_t*)(base + off[R_SPIN1]);
        r.E[0] = (int32_t*)(base + off[R_E0]);
        r.E[1] = (int32_t*)(base + off[R_E1]);
        r.fam[0] = (uint32_t*)(base + off[R_F0]);
        r.fam[1] = (uint32_t*)(base + off[R_F1]);
        r.M = (int32_t*)(base + off[R_M]);
        r.anc = (uint32_t*)(base + off[R_ANC]);
        r.counts = (uint32_t*)(base + off[R_CNT]);
        r.C = (uint64_t*)(base + off[R_C]);
        r.G = (uint64_t*)(base + off[R_G]);
        r.hist = (uint32_t*)(base + off[R_HIST]);
        r.flev = (uint64_t*)(base + off[R_FLEV]);
        r.tree = (double*)(base + off[R_TREE]);
        r.partA = (uint64_t*)(base + off[R_PA]);
        r.partB = (uint64_t*)(base + off[R_PB]);
        r.offA = (uint64_t*)(base + off[R_OA]);
        r.offB = (uint64_t*)(base + off[R_OB]);
        r.partD = (double*)(base + off[R_PD]);
        r.partCL = (double*)(base + off[R_PCL]);
        r.w = (double*)(base + off[R_W]);
        r.wpart = (double*)(base + off[R_WP]);
        r.opart = (double*)(base + off[R_OP]);
        r.jbits = (const uint8_t*)(base + off[R_JB]);
        r.st = (DevState*)(base + off[R_ST]);
        r.trace = (TraceRow*)(base + off[R_TRACE]);
        r.sbeta = (double*)(base + lay.shared_off[S_BETA]);
        r.sdbeta = (double*)(base + lay.shared_off[S_DBETA]);
        r.sq = (double*)(base + lay.shared_off[S_Q]);
        r.sthr = (uint32_t*)(base + lay.shared_off[S_THR]);
        r.stheta = (uint32_t*)(base + lay.shared_off[S_THETA]);
        ctx->rtab_off.push_back({off[R_SB], off[R_SDB], off[R_SQ], off[R_STHR], off[R_STH]});
        r.lb1 = (LBDesc*)(base + off[R_LB1]);
        r.lb2 = (LBDesc*)(base + off[R_LB2]);
        r.tick = (uint32_t*)(base + off[R_TICK]);
    }
    p.nblk_total = blk0;
    p.ngrp_total = grp0;

    // 3D runs of sides 4..16: the grouped 3D kernel, one launch per distinct side
    // (at most four), each over the CTAs of the runs of that side in run order
    std::vector<uint32_t> c3;
    {
        std::vector<int> Ls;
        bool ok = d == 3;
        for (const RunHost& h : ctx->runs) {
            if (!h.g3) ok = false;
            if (std::find(Ls.begin(), Ls.end(), h.L) == Ls.end()) Ls.push_back(h.L);
        }
        if (ok && Ls.size() <= 4) {
            p.n3 = (int)Ls.size();
            for (int k = 0; k < p.n3; ++k) p.L3[k] = Ls[k];
            p.c3map[0] = (uint32_t*)(base + lay.shared_off[S_C3]);
            plan3d(ctx, 1, c3);
        }
    }

    // per-step tables: dbeta, q = exp(-4 dbeta), Metropolis thresholds at beta_i
    std::vector<double> dbeta(n), q(n);
    std::vector<uint32_t> thr((size_t)4 * n);
    for (int i = 1; i <= n; ++i) {
        dbeta[i - 1] = ctx->beta[i] - ctx->beta[i - 1];
        q[i - 1] = std::exp(-(4.0 * dbeta[i - 1]));
        thresholds_at(ctx->beta[i], &thr[4 * (i - 1)]);
    }

    cudaError_t e = cudaSuccess;
    auto up = [&](const void* dev, const void* host, size_t bytes) {
        if (e == cudaSuccess && bytes)
            e = cudaMemcpy((void*)dev, host, bytes, cudaMemcpyHostToDevice);
    };
    up(p.runs, ctx->desc.data(), sizeof(RunDesc) * M);
    up(p.blk2run, b2r.data(), b2r.size() * 4);
    up(p.grp2run, g2r.data(), g2r.size() * 4);
    if (!c3.empty()) up(p.c3map[0], c3.data(), c3.size() * 4);
    up(p.beta, ctx->beta.data(), sizeof(double) * (n + 1));
    up(p.dbeta, dbeta.data(), sizeof(double) * n);
    up(p.q, q.data(), sizeof(double) * n);
    up(p.thr, thr.data(), sizeof(uint32_t) * 4 * n);
    up(p.theta, ctx->theta.data(), sizeof(uint32_t) * n);
    double clnc[CLN_TAB + 1];
    for (int c = 0; c <= CLN_TAB; ++c) clnc[c] = c > 1 ? (double)c * std::log((double)c) : 0.0;
    up(p.clnc, clnc, sizeof(clnc));
    for (int m = 0; m < M && e == cudaSuccess; ++m) {
        const RunHost& h = ctx->runs[m];
        const RunDesc& r = ctx->desc[m];
        DevState st0;
        std::memset(&st0, 0, sizeof(st0));
        st0.R_cur = h.R;
        st0.R_prev = h.R;
        st0.hlo = 0x7FFFFFFF;
        st0.hhi = -1;
        up(r.jbits, h.jb.data(), h.jb.size());
        up(r.st, &st0, sizeof(st0));
        if (e == cudaSuccess) e = cudaMemsetAsync(r.hist, 0, (size_t)h.nlev * 4, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(r.trace, 0, (size_t)(n + 1) * sizeof(TraceRow), ctx->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(r.counts, 0, (size_t)h.Rcap * 4, ctx->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(r.anc, 0, (size_t)h.Rcap * 4, ctx->stream);
        if (e == cudaSuccess) e = clear_lookback(r, h, ctx->stream);
    }
    if (e == cudaSuccess)
        e = cudaMemsetAsync(ctx->d_ovacc, 0, (size_t)M * (maxN + 1) * 4, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_ovtick, 0, (size_t)M * 4, ctx->stream);
    if (e == cudaSuccess) e = launch_init_spins(p, ctx->desc.data(), ctx->stream);
    if (e != cudaSuccess) {
        pa_destroy(ctx);
        return PA_ERR_CUDA;
    }
    ctx->launches += 1;
    pa_status s = enqueue_measure(ctx);
    if (s == PA_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) s = PA_ERR_CUDA;
    if (s != PA_OK) {
        pa_destroy(ctx);
        return s;
    }
    *out = ctx;
    return PA_OK;
}

pa_status pa_init(pa_ctx** out, const pa_lattice* lat, const pa_couplings* cpl, uint32_t R,
                  uint32_t R_cap, const pa_schedule* sched, pa_resampler resampler, uint64_t seed,
                  void* cuda_stream, void* workspace, size_t workspace_bytes) {
    if (!out || !lat || !cpl) return PA_ERR_ARG;
    pa_run_spec s;
    std::memset(&s, 0, sizeof(s));
    s.lattice = *lat;
    s.couplings = *cpl;
    s.R = R;
    s.R_cap = R_cap;
    s.ensemble = 0;
    return pa_batch_init(out, &s, 1, sched, resampler, seed, cuda_stream, workspace,
                         workspace_bytes);
}

int32_t pa_batch_size(const pa_ctx* ctx) { return ctx ? ctx->M : 0; }

pa_status pa_step(pa_ctx* ctx, int32_t n) {
    if (!ctx || n < 0) return PA_ERR_ARG;
    if (ctx->sticky != PA_OK) return PA_ERR_STATE;
    if (ctx->controlled) {
        // the number of steps to beta_f is chosen on the device; steps launched
        // after it is reached return at once
        if (ctx->finished) return PA_ERR_DONE;
        if (ctx->host_step + n > ctx->n_steps) n = ctx->n_steps - ctx->host_step;
    }
    if (ctx->host_step + n > ctx->n_steps) return PA_ERR_DONE;
    const bool graph = ctx->use_graph && !ctx->timing && ctx->stream != nullptr;
    if (graph && n > 0 && (!ctx->graph || ctx->graph_threads != ctx->threads)) {
        const pa_status s = build_graph(ctx);
        if (s != PA_OK) return s;
    }
    for (int k = 0; k < n; ++k) {
        const int i = ctx->host_step + 1;
        if (graph) {
            PA_CUDA(cudaGraphLaunch(ctx->graph, ctx->stream));
            ctx->launches += ctx->graph_kernels;
        } else if (ctx->timing) {
            PA_CUDA(launch_resample(ctx->kp, ctx->stream, &ctx->launches));
            if (ctx->ev_used == ctx->ev_start.size()) {
                const pa_status ps = grow_event_pool(ctx, 1);
                if (ps != PA_OK) return ps;
            }
            cudaEvent_t a = ctx->ev_start[ctx->ev_used], b = ctx->ev_stop[ctx->ev_used];
            ctx->ev_used += 1;
            ctx->timed_steps.push_back(i);
            PA_CUDA(cudaEventRecord(a, ctx->stream));
            PA_CUDA(launch_sweep(ctx->kp, ctx->threads, ctx->stream));
            ctx->launches += 1;
            PA_CUDA(cudaEventRecord(b, ctx->stream));
            PA_CUDA(launch_family_finish(ctx->kp, 0, ctx->stream, &ctx->launches));
        } else {
            const pa_status s = enqueue_step(ctx, &ctx->launches);
            if (s != PA_OK) return s;
        }
        ctx->host_step = i;
    }
    return PA_OK;
}

pa_status pa_sync(pa_ctx* ctx) {
    if (!ctx) return PA_ERR_ARG;
    if (ctx->sticky != PA_OK) return ctx->sticky;
    PA_CUDA(cudaStreamSynchronize(ctx->stream));
    bool all_done = true;
    int most = 0;
    for (int m = 0; m < ctx->M; ++m) {
        DevState st;
        PA_CUDA(cudaMemcpy(&st, ctx->desc[m].st, sizeof(DevState), cudaMemcpyDeviceToHost));
        if (ctx->controlled) {
            // runs of a controlled batch reach beta_f after different step counts
            ctx->rstep[m] = st.step;
            most = std::max(most, st.step);
            if (st.status == S_DONE) {
                ctx->rdone[m] = 1;
                st.status = S_OK;
            }
            all_done = all_done && ctx->rdone[m];
        }
        const pa_status s = map_dev_status(st.status);
        if (s != PA_OK) {
            ctx->sticky = s;
            return s;
        }
    }
    if (ctx->controlled) {
        ctx->host_step = most;
        ctx->finished = all_done;
        return refresh_schedule(ctx);
    }
    return PA_OK;
}

pa_status pa_run_observables(pa_ctx* ctx, int32_t run, pa_obs* out) {
    if (!valid_run(ctx, run) || !out) return PA_ERR_ARG;
    pa_status s = pa_sync(ctx);
    if (s != PA_OK) return s;
    TraceRow t;
    const int step = run_step(ctx, run);
    PA_CUDA(cudaMemcpy(&t, ctx->desc[run].trace + step, sizeof(t), cudaMemcpyDeviceToHost));
    fill_obs(ctx, run, t, step, out);
    return PA_OK;
}

pa_status pa_observables(pa_ctx* ctx, pa_obs* out) { return pa_run_observables(ctx, 0, out); }

pa_status pa_run_trace(pa_ctx* ctx, int32_t run, pa_obs* rows, int32_t max_rows,
                       int32_t* n_rows) {
    if (!valid_run(ctx, run) || !rows || max_rows < 0) return PA_ERR_ARG;
    pa_status s = pa_sync(ctx);
    if (s != PA_OK) return s;
    int n = run_step(ctx, run) + 1;
    if (n > max_rows) n = max_rows;
    std::vector<TraceRow> t((size_t)n);
    if (n > 0)
        PA_CUDA(cudaMemcpy(t.data(), ctx->desc[run].trace, sizeof(TraceRow) * n,
                           cudaMemcpyDeviceToHost));
    for (int i = 0; i < n; ++i) fill_obs(ctx, run, t[i], i, rows + i);
    if (n_rows) *n_rows = n;
    return PA_OK;
}

pa_status pa_trace(pa_ctx* ctx, pa_obs* rows, int32_t max_rows, int32_t* n_rows) {
    return pa_run_trace(ctx, 0, rows, max_rows, n_rows);
}

pa_status pa_run_free_energy(pa_ctx* ctx, int32_t run, double* minus_beta_F, double* f_per_spin) {
    if (!valid_run(ctx, run)) return PA_ERR_ARG;
    pa_status s = pa_sync(ctx);
    if (s != PA_OK) return s;
    DevState st;
    s = read_state(ctx, run, &st);
    if (s != PA_OK) return s;
    const double N = ctx->runs[run].N;
    const double mbf = N * std::log(2.0) + st.sum_lnQ;
    const double b = run_beta(ctx, run, run_step(ctx, run));
    if (minus_beta_F) *minus_beta_F = mbf;
    if (f_per_spin) *f_per_spin = b > 0 ? -mbf / (b * N) : NAN;
    return PA_OK;
}

pa_status pa_free_energy(pa_ctx* ctx, double* minus_beta_F, double* f_per_spin) {
    return pa_run_free_energy(ctx, 0, minus_beta_F, f_per_spin);
}

pa_status pa_run_get_array(pa_ctx* ctx, int32_t run, pa_array which, void* host, size_t capacity,
                           size_t* n_out) {
    if (!valid_run(ctx, run) || !host) return PA_ERR_ARG;
    pa_status s = pa_sync(ctx);
    if (s != PA_OK) return s;
    DevState st;
    s = read_state(ctx, run, &st);
    if (s != PA_OK) return s;
    const int par = run_step(ctx, run) & 1;
    const RunDesc& r = ctx->desc[run];
    const RunHost& h = ctx->runs[run];
    size_t n = 0;
    switch (which) {
        case PA_ARRAY_SPINS:
            n = (size_t)st.R_cur * h.W;
            if (capacity < n) return PA_ERR_ARG;
            if (st.R_cur)
                PA_CUDA(cudaMemcpy2D(host, (size_t)h.W * 4, r.spins[par], (size_t)h.Wp * 4,
                                     (size_t)h.W * 4, st.R_cur, cudaMemcpyDeviceToHost));
            break;
        case PA_ARRAY_ENERGY:
        case PA_ARRAY_FAMILY:
        case PA_ARRAY_ANCESTOR:
        case PA_ARRAY_MAGNET: {
            n = st.R_cur;
            if (capacity < n) return PA_ERR_ARG;
            const void* src = which == PA_ARRAY_ENERGY   ? (const void*)r.E[par]
                              : which == PA_ARRAY_FAMILY ? (const void*)r.fam[par]
                              : which == PA_ARRAY_MAGNET ? (const void*)r.M
                                                         : (const void*)r.anc;
            if (n) PA_CUDA(cudaMemcpy(host, src, n * 4, cudaMemcpyDeviceToHost));
            break;
        }
        case PA_ARRAY_COUNTS:
            n = run_step(ctx, run) > 0 ? st.R_prev : 0;
            if (capacity < n) return PA_ERR_ARG;
            if (n) PA_CUDA(cudaMemcpy(host, r.counts, n * 4, cudaMemcpyDeviceToHost));
            break;
        case PA_ARRAY_WEIGHT:
            n = st.R_cur;
            if (capacity < n) return PA_ERR_ARG;
            if (ctx->kp.alpha >= 0.0) {
                if (n) PA_CUDA(cudaMemcpy(host, r.w, n * 8, cudaMemcpyDeviceToHost));
            } else {
                for (size_t j = 0; j < n; ++j) ((double*)host)[j] = 1.0;
            }
            break;
        default:
            return PA_ERR_ARG;
    }
    if (n_out) *n_out = n;
    return PA_OK;
}

pa_status pa_get_array(pa_ctx* ctx, pa_array which, void* host, size_t capacity, size_t* n_out) {
    return pa_run_get_array(ctx, 0, which, host, capacity, n_out);
}

pa_status pa_set_state(pa_ctx* ctx, const uint32_t* spins, const uint32_t* family, uint32_t R_i,
                       int32_t step, double sum_lnQ) {
    if (!ctx || ctx->M != 1 || !spins || R_i == 0 || R_i > ctx->runs[0].Rcap || step < 0 ||
        step > ctx->n_steps || ctx->kp.alpha >= 0.0)
        return PA_ERR_ARG;
    if (ctx->sticky != PA_OK) return PA_ERR_STATE;
    const RunDesc& r = ctx->desc[0];
    const RunHost& h = ctx->runs[0];
    const int par = step & 1;
    std::vector<uint32_t> fam((size_t)R_i);
    for (uint32_t j = 0; j < R_i; ++j) {
        fam[j] = family ? family[j] : j;
        if (fam[j] >= h.R) return PA_ERR_ARG;
        if (j > 0 && fam[j] < fam[j - 1]) return PA_ERR_ARG;  // families stay sorted by slot
    }
    PA_CUDA(cudaStreamSynchronize(ctx->stream));
    PA_CUDA(cudaMemset(r.spins[par], 0, (size_t)R_i * h.Wp * 4));
    PA_CUDA(cudaMemcpy2D(r.spins[par], (size_t)h.Wp * 4, spins, (size_t)h.W * 4, (size_t)h.W * 4,
                         R_i, cudaMemcpyHostToDevice));
    PA_CUDA(cudaMemcpy(r.fam[par], fam.data(), (size_t)R_i * 4, cudaMemcpyHostToDevice));
    DevState st;
    std::memset(&st, 0, sizeof(st));
    st.step = step;
    st.R_cur = R_i;
    st.R_prev = R_i;
    st.hlo = 0x7FFFFFFF;
    st.hhi = -1;
    st.sum_lnQ = sum_lnQ;
    PA_CUDA(cudaMemcpy(r.st, &st, sizeof(st), cudaMemcpyHostToDevice));
    PA_CUDA(cudaMemset(r.hist, 0, (size_t)h.nlev * 4));
    PA_CUDA(clear_lookback(r, h, ctx->stream));
    PA_CUDA(cudaStreamSynchronize(ctx->stream));
    TraceRow t;
    std::memset(&t, 0, sizeof(t));
    t.sum_lnQ = sum_lnQ;
    t.R_prev = R_i;
    PA_CUDA(cudaMemcpy(r.trace + step, &t, sizeof(t), cudaMemcpyHostToDevice));
    ctx->host_step = step;
    const pa_status s = enqueue_measure(ctx);
    if (s != PA_OK) return s;
    return pa_sync(ctx);
}

pa_status pa_weighted(pa_ctx* ctx, int32_t ensemble, pa_weighted_obs* rows, int32_t max_rows,
                      int32_t* n_rows) {
    if (!ctx || !rows || max_rows < 0) return PA_ERR_ARG;
    // under the learned schedule the runs' temperatures differ at a step index
    if (ctx->controlled && ctx->M > 1) return PA_ERR_ARG;
    std::vector<int32_t> ids;
    for (int m = 0; m < ctx->M; ++m)
        if (ctx->runs[m].ensemble == ensemble) ids.push_back(m);
    if (ids.empty()) return PA_ERR_ARG;
    for (int32_t m : ids)
        if (ctx->runs[m].N != ctx->runs[ids[0]].N) return PA_ERR_ARG;
    pa_status s = pa_sync(ctx);
    if (s != PA_OK) return s;
    int n = ctx->host_step + 1;
    if (n > max_rows) n = max_rows;
    if (n > 0) {
        PA_CUDA(cudaMemcpy(ctx->d_ids, ids.data(), ids.size() * 4, cudaMemcpyHostToDevice));
        PA_CUDA(launch_weighted(ctx->kp, ctx->d_ids, (int)ids.size(), n, ctx->d_wout,
                                ctx->stream));
        ctx->launches += 1;
        PA_CUDA(cudaStreamSynchronize(ctx->stream));
        PA_CUDA(cudaMemcpy(rows, ctx->d_wout, sizeof(pa_weighted_obs) * n,
                           cudaMemcpyDeviceToHost));
    }
    if (n_rows) *n_rows = n;
    return PA_OK;
}

pa_status pa_overlap(pa_ctx* ctx, const int32_t* run_a, const int32_t* run_b, int32_t n_pairs,
                     uint32_t* hist_dev, double* P_out) {
    if (!ctx || !run_a || !run_b || !hist_dev || n_pairs < 1 || n_pairs > ctx->M)
        return PA_ERR_ARG;
    if (ctx->sticky != PA_OK) return PA_ERR_STATE;
    std::vector<int32_t> pairs((size_t)2 * n_pairs);
    uint32_t rows = 0;
    const int N = valid_run(ctx, run_a[0]) ? ctx->runs[run_a[0]].N : -1;
    for (int q = 0; q < n_pairs; ++q) {
        const int a = run_a[q], b = run_b[q];
        if (!valid_run(ctx, a) || !valid_run(ctx, b) || a == b) return PA_ERR_ARG;
        if (ctx->runs[a].N != N || ctx->runs[b].N != N) return PA_ERR_ARG;
        pairs[2 * q] = a;
        pairs[2 * q + 1] = b;
        rows = std::max(rows, std::min(ctx->runs[a].Rcap, ctx->runs[b].Rcap));
    }
    if (pairs != ctx->pairs_cached) {  // the device copy of the pair list is kept
        PA_CUDA(cudaMemcpyAsync(ctx->d_pairs, pairs.data(), pairs.size() * 4,
                                cudaMemcpyHostToDevice, ctx->stream));
        PA_CUDA(cudaStreamSynchronize(ctx->stream));  // the host vector is temporary
        ctx->pairs_cached = pairs;
    }
    PA_CUDA(launch_overlap(ctx->kp, ctx->d_pairs, n_pairs, ctx->runs[run_a[0]].Wp, rows, N + 1,
                           hist_dev, P_out ? ctx->d_pov : nullptr, ctx->d_ovacc, ctx->d_ovtick,
                           ctx->stream));
    ctx->launches += P_out ? 2 : 1;
    if (!P_out) return PA_OK;  // asynchronous on the context's stream
    pa_status st = pa_sync(ctx);
    if (st != PA_OK) return st;
    PA_CUDA(cudaMemcpy(P_out, ctx->d_pov, sizeof(double) * (N + 1), cudaMemcpyDeviceToHost));
    return PA_OK;
}

pa_status pa_set_partial_resampling(pa_ctx* ctx, double alpha) {
    if (!ctx || ctx->host_step != 0 || ctx->kp.alpha >= 0.0 || ctx->controlled ||
        !(alpha >= 0.0 && alpha <= 1.0))
        return PA_ERR_ARG;
    if (ctx->sticky != PA_OK) return PA_ERR_STATE;
    for (const RunHost& h : ctx->runs)
        if (h.nblk > PARTIAL_MAX_BLOCKS) return PA_ERR_ARG;
    PA_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->kp.alpha = alpha;
    PA_CUDA(launch_partial_init(ctx->kp, ctx->stream));
    ctx->launches += 1;
    // row 0: all weights are 1, so the weighted sums are the exact sums
    for (int m = 0; m < ctx->M; ++m) {
        TraceRow t;
        PA_CUDA(cudaMemcpy(&t, ctx->desc[m].trace, sizeof(t), cudaMemcpyDeviceToHost));
        t.ess = (double)t.R_i;
        t.resampled = 1;
        t.wsum = (double)t.R_i;
        t.wE = (double)(long long)t.sumE;
        t.wE2 = (double)(long long)t.sumE2;
        t.wAM = (double)(long long)t.sumAbsM;
        t.wM2 = (double)(long long)t.sumM2;
        PA_CUDA(cudaMemcpy(ctx->desc[m].trace, &t, sizeof(t), cudaMemcpyHostToDevice));
    }
    if (ctx->graph) {  // the step graph must now include the weight kernels
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    return pa_sync(ctx);
}

pa_status pa_set_controller(pa_ctx* ctx, const pa_controller* cfg) {
    if (!ctx || !cfg || ctx->host_step != 0 || ctx->controlled || ctx->kp.alpha >= 0.0)
        return PA_ERR_ARG;
    if (ctx->sticky != PA_OK) return PA_ERR_STATE;
    const int K = ctx->n_steps;
    if (cfg->u_max < 1 || cfg->u_max > CTL_UMAX || cfg->plain_units < 1 ||
        cfg->plain_units > cfg->u_max || cfg->theta_min > cfg->theta_max ||
        cfg->theta_max >= (1u << 24) || cfg->plain_theta >= (1u << 24) ||
        (cfg->use_mlp && !cfg->params))
        return PA_ERR_ARG;
    CtlDev c;
    std::memset(&c, 0, sizeof(c));
    if (cfg->params) std::memcpy(c.w, cfg->params, sizeof(c.w));
    c.use_mlp = cfg->use_mlp ? 1 : 0;
    c.K = K;
    c.plain_units = cfg->plain_units;
    c.plain_theta = cfg->plain_theta;
    c.theta_min = cfg->theta_min;
    c.theta_max = cfg->theta_max;
    const int planned = (K + cfg->plain_units - 1) / cfg->plain_units;
    c.budget = cfg->budget ? cfg->budget : cfg->plain_theta * (uint32_t)planned;
    c.u_max = cfg->u_max;
    c.theta_c = (float)c.budget / (float)planned;
    c.beta_grid = ctx->d_gbeta;
    c.thr_grid = ctx->d_gthr;
    c.dbeta_tab = ctx->d_gdb;
    c.q_tab = ctx->d_gq;
    // grid tables: beta_k, thresholds at beta_k, and for each step of u points
    // dbeta = beta_{k+u} - beta_k with q = exp(-4 dbeta)
    std::vector<uint32_t> gthr((size_t)4 * (K + 1));
    std::vector<double> gdb((size_t)(K + 1) * CTL_UMAX, 0.0), gq((size_t)(K + 1) * CTL_UMAX, 1.0);
    for (int k = 0; k <= K; ++k) {
        thresholds_at(ctx->beta[k], &gthr[4 * k]);
        for (int u = 1; u <= CTL_UMAX && k + u <= K; ++u) {
            const double db = ctx->beta[k + u] - ctx->beta[k];
            gdb[(size_t)k * CTL_UMAX + u - 1] = db;
            gq[(size_t)k * CTL_UMAX + u - 1] = std::exp(-(4.0 * db));
        }
    }
    PA_CUDA(cudaStreamSynchronize(ctx->stream));
    PA_CUDA(cudaMemcpy(ctx->d_ctl, &c, sizeof(c), cudaMemcpyHostToDevice));
    PA_CUDA(cudaMemcpy(ctx->d_gbeta, ctx->beta.data(), sizeof(double) * (K + 1),
                       cudaMemcpyHostToDevice));
    PA_CUDA(cudaMemcpy(ctx->d_gthr, gthr.data(), gthr.size() * 4, cudaMemcpyHostToDevice));
    PA_CUDA(cudaMemcpy(ctx->d_gdb, gdb.data(), gdb.size() * 8, cudaMemcpyHostToDevice));
    PA_CUDA(cudaMemcpy(ctx->d_gq, gq.data(), gq.size() * 8, cudaMemcpyHostToDevice));
    // every run gets its own step tables, initialised from the shared ones, which the
    // controller then writes step by step
    char* base = (char*)ctx->ws;
    for (int m = 0; m < ctx->M; ++m) {
        RunDesc& r = ctx->desc[m];
        const auto& o = ctx->rtab_off[m];
        double* sb = (double*)(base + o[0]);
        double* sdb = (double*)(base + o[1]);
        double* sq = (double*)(base + o[2]);
        uint32_t* sthr = (uint32_t*)(base + o[3]);
        uint32_t* sth = (uint32_t*)(base + o[4]);
        PA_CUDA(cudaMemcpy(sb, ctx->kp.beta, sizeof(double) * (K + 1), cudaMemcpyDeviceToDevice));
        PA_CUDA(cudaMemcpy(sdb, ctx->kp.dbeta, sizeof(double) * K, cudaMemcpyDeviceToDevice));
        PA_CUDA(cudaMemcpy(sq, ctx->kp.q, sizeof(double) * K, cudaMemcpyDeviceToDevice));
        PA_CUDA(cudaMemcpy(sthr, ctx->kp.thr, sizeof(uint32_t) * 4 * K, cudaMemcpyDeviceToDevice));
        PA_CUDA(cudaMemcpy(sth, ctx->kp.theta, sizeof(uint32_t) * K, cudaMemcpyDeviceToDevice));
        r.sbeta = sb;
        r.sdbeta = sdb;
        r.sq = sq;
        r.sthr = sthr;
        r.stheta = sth;
    }
    PA_CUDA(cudaMemcpy((void*)ctx->kp.runs, ctx->desc.data(), sizeof(RunDesc) * ctx->M,
                       cudaMemcpyHostToDevice));
    ctx->rbeta.assign(ctx->M, ctx->beta);
    ctx->rtheta.assign(ctx->M, ctx->theta);
    ctx->rstep.assign(ctx->M, 0);
    ctx->rdone.assign(ctx->M, 0);
    ctx->kp.ctl = ctx->d_ctl;
    ctx->controlled = true;
    if (ctx->graph) {  // the step graph must now include the controller
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    // choose the first step from the initial population
    PA_CUDA(launch_control(ctx->kp, ctx->stream));
    ctx->launches += 1;
    return pa_sync(ctx);
}

pa_status pa_run_schedule_taken(pa_ctx* ctx, int32_t run, double* beta, uint32_t* theta,
                                int32_t max, int32_t* n) {
    if (!valid_run(ctx, run) || max < 0) return PA_ERR_ARG;
    pa_status s = pa_sync(ctx);
    if (s != PA_OK) return s;
    int cnt = run_step(ctx, run) + 1;
    if (cnt > max) cnt = max;
    for (int i = 0; i < cnt; ++i) {
        if (beta) beta[i] = run_beta(ctx, run, i);
        if (theta && i > 0) theta[i - 1] = run_theta(ctx, run, i - 1);
    }
    if (n) *n = cnt;
    return PA_OK;
}

pa_status pa_schedule_taken(pa_ctx* ctx, double* beta, uint32_t* theta, int32_t max,
                            int32_t* n) {
    return pa_run_schedule_taken(ctx, 0, beta, theta, max, n);
}

pa_status pa_set_graph(pa_ctx* ctx, int32_t on) {
    if (!ctx) return PA_ERR_ARG;
    ctx->use_graph = on != 0;
    return PA_OK;
}

pa_status pa_enable_timing(pa_ctx* ctx, int32_t on) {
    if (!ctx) return PA_ERR_ARG;
    ctx->timing = on != 0;
    if (ctx->timing) {
        // one event pair per remaining step, created now rather than inside pa_step
        const size_t want = ctx->ev_used + (size_t)(ctx->n_steps - ctx->host_step);
        if (want > ctx->ev_start.size()) return grow_event_pool(ctx, want - ctx->ev_start.size());
    }
    return PA_OK;
}

pa_status pa_sweep_timing(pa_ctx* ctx, double* ms, int64_t* launches, double* updates) {
    if (!ctx) return PA_ERR_ARG;
    pa_status s = pa_sync(ctx);
    if (s != PA_OK) return s;
    double total = 0.0, upd = 0.0;
    std::vector<std::vector<TraceRow>> t((size_t)ctx->M);
    for (int m = 0; m < ctx->M; ++m) {
        t[m].resize((size_t)ctx->n_steps + 1);
        PA_CUDA(cudaMemcpy(t[m].data(), ctx->desc[m].trace, sizeof(TraceRow) * t[m].size(),
                           cudaMemcpyDeviceToHost));
    }
    for (size_t k = 0; k < ctx->ev_used; ++k) {
        float f = 0.f;
        PA_CUDA(cudaEventElapsedTime(&f, ctx->ev_start[k], ctx->ev_stop[k]));
        total += f;
        const int i = ctx->timed_steps[k];
        for (int m = 0; m < ctx->M; ++m)
            upd += (double)run_theta(ctx, m, i - 1) * (double)ctx->runs[m].N * (double)t[m][i].R_i;
    }
    if (ms) *ms = total;
    if (launches) *launches = (int64_t)ctx->ev_used;
    if (updates) *updates = upd;
    ctx->ev_used = 0;  // the pool is kept for the next timed steps
    ctx->timed_steps.clear();
    return PA_OK;
}

int64_t pa_launch_count(const pa_ctx* ctx) { return ctx ? ctx->launches : 0; }

pa_status pa_set_sweep_threads(pa_ctx* ctx, int32_t threads) {
    if (!ctx || !sweep_threads_supported(threads)) return PA_ERR_ARG;
    ctx->threads = threads;
    if (ctx->graph) {  // the captured step holds the old launch configuration
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    return PA_OK;
}

pa_status pa_set_sweep_groups(pa_ctx* ctx, int32_t mult) {
    if (!ctx || (mult != 1 && mult != 2)) return PA_ERR_ARG;
    if (ctx->kp.n3 == 0) return mult == 1 ? PA_OK : PA_ERR_ARG;  // no grouped 3D kernel
    if (ctx->sticky != PA_OK) return PA_ERR_STATE;
    if (mult == ctx->kp.g3mul) return PA_OK;
    // no step in flight may read the old plan
    PA_CUDA(cudaStreamSynchronize(ctx->stream));
    std::vector<uint32_t> c3;
    plan3d(ctx, mult, c3);
    PA_CUDA(cudaMemcpy((void*)ctx->kp.c3map[0], c3.data(), c3.size() * 4, cudaMemcpyHostToDevice));
    PA_CUDA(cudaMemcpy((void*)ctx->kp.runs, ctx->desc.data(), sizeof(RunDesc) * ctx->desc.size(),
                       cudaMemcpyHostToDevice));
    if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    return PA_OK;
}

int32_t pa_get_sweep_groups(const pa_ctx* ctx) {
    return ctx ? (ctx->kp.n3 ? ctx->kp.g3mul : 1) : 0;
}

int32_t pa_get_sweep_threads(const pa_ctx* ctx) { return ctx ? ctx->threads : 0; }

pa_status pa_set_sweep_queue(pa_ctx* ctx, int32_t cap) {
    if (!ctx || cap < -1) return PA_ERR_ARG;
    ctx->kp.qcap_limit = cap;
    if (ctx->graph) {  // the captured step holds the old kernel parameters
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    return PA_OK;
}

pa_status pa_set_wait_test(pa_ctx* ctx, int32_t on) {
    if (!ctx || (on != 0 && on != 1)) return PA_ERR_ARG;
    ctx->kp.lb_hold = on;
    if (ctx->graph) {  // the captured step holds the old kernel parameters
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    return PA_OK;
}

pa_status pa_destroy(pa_ctx* ctx) {
    if (!ctx) return PA_OK;
    for (size_t k = 0; k < ctx->ev_start.size(); ++k) {
        cudaEventDestroy(ctx->ev_start[k]);
        cudaEventDestroy(ctx->ev_stop[k]);
    }
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    if (ctx->owns && ctx->ws) cudaFree(ctx->ws);
    delete ctx;
    return PA_OK;
}

const char* pa_strerror(pa_status s) {
    switch (s) {
        case PA_OK: return "ok";
        case PA_ERR_ARG: return "invalid argument";
        case PA_ERR_CUDA: return "CUDA runtime error";
        case PA_ERR_NOMEM: return "out of device memory or workspace too small";
        case PA_ERR_CAPACITY: return "population exceeded its capacity or died out";
        case PA_ERR_POISSON_KMAX: return "Poisson inversion exceeded its iteration limit";
        case PA_ERR_TIMEOUT: return "a bounded device wait timed out";
        case PA_ERR_STATE: return "context holds an earlier error";
        case PA_ERR_DONE: return "schedule exhausted";
        case PA_ERR_LIMIT: return "size exceeds a fixed limit of the library";
        default: return "unknown status";
    }
}

}  // extern "C"
