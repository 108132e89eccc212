// pa_api.cu -- the C ABI of include/pa.h: context, device workspace, host
// precomputation of the per-step tables, and the launch sequence of a
// temperature step (Sec. 2 steps 2-4).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/pa.h"
#include "pa_internal.cuh"

using namespace pa;

struct pa_ctx {
    KParams kp;
    int d = 0, L = 0, N = 0, W = 0, Wp = 0;
    uint32_t R = 0, Rcap = 0;
    int n_steps = 0, method = 0;
    uint64_t seed = 0;
    cudaStream_t stream = nullptr;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    bool owns = false;
    int host_step = 0;
    int threads = 32;
    int64_t launches = 0;
    pa_status sticky = PA_OK;
    bool timing = false;
    std::vector<cudaEvent_t> ev_start, ev_stop;
    std::vector<int> timed_steps;
    std::vector<double> beta;
    std::vector<uint32_t> theta;
};

namespace {

struct Layout {
    size_t off[40];
    size_t total;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Dims {
    int d, L, N, W, Wp, nlev, P, nblk;
    uint32_t R, Rcap;
    int n_steps;
};

bool make_dims(const pa_lattice* lat, uint32_t R, uint32_t R_cap, int32_t n_steps, int method,
               Dims* o) {
    if (!lat || lat->dim < 2 || lat->dim > 3 || lat->L < 2 || (lat->L & 1)) return false;
    if (R == 0 || n_steps < 1 || method < 0 || method > 4) return false;
    long long N = 1;
    for (int a = 0; a < lat->dim; ++a) N *= lat->L;
    if (N > 32768) return false;  // the sweep keeps a lattice of 32 replicas in shared memory
    o->d = lat->dim;
    o->L = lat->L;
    o->N = (int)N;
    o->W = (int)((N + 31) / 32);
    o->Wp = (o->W + 3) & ~3;
    o->nlev = (int)(o->d * N / 2 + 1);
    o->P = 1;
    while (o->P < o->nlev) o->P <<= 1;
    uint32_t cap = R_cap;
    if (cap == 0) {
        if (method == PA_POISSON || method == PA_NEAREST)
            cap = R + (uint32_t)std::ceil(10.0 * std::sqrt((double)R)) + 64u;
        else
            cap = R;
    }
    if (cap < R || cap > (1u << 30)) return false;
    o->R = R;
    o->Rcap = cap;
    o->nblk = (int)((cap + SCAN_CHUNK - 1) / SCAN_CHUNK);
    o->n_steps = n_steps;
    return true;
}

enum Region {
    R_SPIN0, R_SPIN1, R_E0, R_E1, R_F0, R_F1, R_M, R_ANC, R_CNT, R_C, R_G, R_HIST, R_FLEV, R_TREE,
    R_PA, R_PB, R_OA, R_OB, R_PD, R_PC2, R_PCL, R_JB, R_BETA, R_DBETA, R_Q, R_THR, R_THETA, R_ST,
    R_TRACE, R_COUNT
};

Layout make_layout(const Dims& m) {
    size_t sz[R_COUNT];
    const size_t rows = (size_t)m.Rcap;
    sz[R_SPIN0] = sz[R_SPIN1] = rows * m.Wp * 4;
    sz[R_E0] = sz[R_E1] = sz[R_F0] = sz[R_F1] = sz[R_M] = sz[R_ANC] = sz[R_CNT] = rows * 4;
    sz[R_C] = sz[R_G] = rows * 8;
    sz[R_HIST] = (size_t)m.nlev * 4;
    sz[R_FLEV] = (size_t)m.nlev * 8;
    sz[R_TREE] = (size_t)m.P * 8;
    sz[R_PA] = sz[R_PB] = sz[R_OA] = sz[R_OB] = sz[R_PD] = sz[R_PC2] = sz[R_PCL] =
        (size_t)m.nblk * 8;
    sz[R_JB] = (size_t)m.N;
    sz[R_BETA] = (size_t)(m.n_steps + 1) * 8;
    sz[R_DBETA] = sz[R_Q] = (size_t)m.n_steps * 8;
    sz[R_THR] = (size_t)m.n_steps * 16;
    sz[R_THETA] = (size_t)m.n_steps * 4;
    sz[R_ST] = sizeof(DevState);
    sz[R_TRACE] = (size_t)(m.n_steps + 1) * sizeof(TraceRow);
    Layout L;
    size_t o = 0;
    for (int r = 0; r < R_COUNT; ++r) {
        L.off[r] = o;
        o += align256(sz[r]);
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

pa_status map_dev_status(int s) {
    switch (s) {
        case S_OK: return PA_OK;
        case S_CAPACITY: return PA_ERR_CAPACITY;
        case S_KMAX: return PA_ERR_POISSON_KMAX;
        case S_TIMEOUT: return PA_ERR_TIMEOUT;
        default: return PA_ERR_STATE;
    }
}

#define PA_CUDA(call)                                  \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) {                       \
            ctx->sticky = PA_ERR_CUDA;                 \
            return PA_ERR_CUDA;                        \
        }                                              \
    } while (0)

pa_status read_state(pa_ctx* ctx, DevState* st) {
    PA_CUDA(cudaStreamSynchronize(ctx->stream));
    PA_CUDA(cudaMemcpy(st, ctx->kp.st, sizeof(DevState), cudaMemcpyDeviceToHost));
    return PA_OK;
}

pa_status enqueue_measure(pa_ctx* ctx) {
    PA_CUDA(launch_measure(ctx->kp, 1, ctx->threads, ctx->stream));
    ctx->launches += 1;
    PA_CUDA(launch_family_finish(ctx->kp, 1, ctx->stream, &ctx->launches));
    return PA_OK;
}

void fill_obs(const pa_ctx* ctx, const TraceRow& t, int step, pa_obs* o) {
    std::memset(o, 0, sizeof(*o));
    const double N = ctx->N;
    o->step = step;
    o->R_i = t.R_i;
    o->R_prev = t.R_prev;
    o->beta = ctx->beta[step];
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
    o->e = (double)o->sumE / (R * N);
    o->e2 = (double)o->sumE2 / (R * N * N);
    o->absm = (double)o->sumAbsM / (R * N);
    o->m2 = (double)o->sumM2 / (R * N * N);
    o->c = o->beta * o->beta * N * (o->e2 - o->e * o->e);
    o->chi = o->beta * N * (o->m2 - o->absm * o->absm);
    o->rho_t = (double)o->sumC2 / R;
    const double th = step > 0 ? (double)ctx->theta[step - 1] : 0.0;
    o->accept_rate = th > 0 ? (double)o->accepts / (th * N * R) : 0.0;
}

}  // namespace

extern "C" {

size_t pa_workspace_bytes(const pa_lattice* lat, uint32_t R, uint32_t R_cap, int32_t n_steps,
                          pa_resampler resampler) {
    Dims m;
    if (!make_dims(lat, R, R_cap, n_steps, (int)resampler, &m)) return 0;
    return make_layout(m).total;
}

pa_status pa_init(pa_ctx** out, const pa_lattice* lat, const pa_couplings* cpl, uint32_t R,
                  uint32_t R_cap, const pa_schedule* sched, pa_resampler resampler, uint64_t seed,
                  void* cuda_stream, void* workspace, size_t workspace_bytes) {
    if (!out || !cpl || !sched || !sched->beta || !sched->theta) return PA_ERR_ARG;
    *out = nullptr;
    Dims m;
    if (!make_dims(lat, R, R_cap, sched->n_steps, (int)resampler, &m)) return PA_ERR_ARG;
    const int n = sched->n_steps;
    if (sched->beta[0] != 0.0) return PA_ERR_ARG;
    for (int i = 1; i <= n; ++i)
        if (!(sched->beta[i] > sched->beta[i - 1]) || !std::isfinite(sched->beta[i]))
            return PA_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (sched->theta[i] >= (1u << 24)) return PA_ERR_ARG;
    if (cpl->kind < 0 || cpl->kind > 2) return PA_ERR_ARG;
    if (cpl->kind == PA_COUPLING_EXPLICIT && !cpl->J) return PA_ERR_ARG;

    // couplings: bit a of byte s is set when the bond (s, s + e_a) has J = -1
    std::vector<uint8_t> jb((size_t)m.N, 0);
    int nneg = 0;
    if (cpl->kind == PA_COUPLING_EA_PM) {
        const uint32_t dk0 = (uint32_t)(cpl->disorder_seed & 0xFFFFFFFFu);
        const uint32_t dk1 = (uint32_t)(cpl->disorder_seed >> 32);
        for (int b = 0; b < m.d * m.N; ++b) {
            const uint4x x = philox((uint32_t)(b >> 7), DOM_DISORDER, 0u, cpl->realization, dk0, dk1);
            const uint32_t lanes[4] = {x.x, x.y, x.z, x.w};
            const uint32_t bit = (lanes[(b >> 5) & 3] >> (b & 31)) & 1u;
            if (bit) {
                jb[b % m.N] |= (uint8_t)(1u << (b / m.N));
                ++nneg;
            }
        }
    } else if (cpl->kind == PA_COUPLING_EXPLICIT) {
        for (int b = 0; b < m.d * m.N; ++b) {
            const int8_t j = cpl->J[b];
            if (j != 1 && j != -1) return PA_ERR_ARG;
            if (j == -1) {
                jb[b % m.N] |= (uint8_t)(1u << (b / m.N));
                ++nneg;
            }
        }
    }

    pa_ctx* ctx = new (std::nothrow) pa_ctx();
    if (!ctx) return PA_ERR_NOMEM;
    ctx->d = m.d;
    ctx->L = m.L;
    ctx->N = m.N;
    ctx->W = m.W;
    ctx->Wp = m.Wp;
    ctx->R = m.R;
    ctx->Rcap = m.Rcap;
    ctx->n_steps = n;
    ctx->method = (int)resampler;
    ctx->seed = seed;
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->beta.assign(sched->beta, sched->beta + n + 1);
    ctx->theta.assign(sched->theta, sched->theta + n);
    ctx->threads = sweep_threads(m.N);

    const Layout lay = make_layout(m);
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
    KParams& p = ctx->kp;
    std::memset(&p, 0, sizeof(p));
    p.d = m.d;
    p.L = m.L;
    p.N = m.N;
    p.W = m.W;
    p.Wp = m.Wp;
    p.nlev = m.nlev;
    p.parity = nneg & 1;
    p.ea = cpl->kind != PA_COUPLING_FERRO;
    p.R = m.R;
    p.Rcap = m.Rcap;
    p.n_steps = n;
    p.method = (int)resampler;
    p.k0 = (uint32_t)(seed & 0xFFFFFFFFu);
    p.k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        p.rk0[r] = p.k0 + (uint32_t)r * PHILOX_W0;
        p.rk1[r] = p.k1 + (uint32_t)r * PHILOX_W1;
    }
    if (!make_magic(m.L, m.N, &p.magicL, &p.shiftL)) {
        pa_destroy(ctx);
        return PA_ERR_ARG;
    }
    p.nblk = m.nblk;
    p.spins[0] = (uint32_t*)(base + lay.off[R_SPIN0]);
    p.spins[1] = (uint32_t*)(base + lay.off[R_SPIN1]);
    p.E[0] = (int32_t*)(base + lay.off[R_E0]);
    p.E[1] = (int32_t*)(base + lay.off[R_E1]);
    p.fam[0] = (uint32_t*)(base + lay.off[R_F0]);
    p.fam[1] = (uint32_t*)(base + lay.off[R_F1]);
    p.M = (int32_t*)(base + lay.off[R_M]);
    p.anc = (uint32_t*)(base + lay.off[R_ANC]);
    p.counts = (uint32_t*)(base + lay.off[R_CNT]);
    p.C = (uint64_t*)(base + lay.off[R_C]);
    p.G = (uint64_t*)(base + lay.off[R_G]);
    p.hist = (uint32_t*)(base + lay.off[R_HIST]);
    p.flev = (uint64_t*)(base + lay.off[R_FLEV]);
    p.tree = (double*)(base + lay.off[R_TREE]);
    p.partA = (uint64_t*)(base + lay.off[R_PA]);
    p.partB = (uint64_t*)(base + lay.off[R_PB]);
    p.offA = (uint64_t*)(base + lay.off[R_OA]);
    p.offB = (uint64_t*)(base + lay.off[R_OB]);
    p.partD = (double*)(base + lay.off[R_PD]);
    p.partC2 = (unsigned long long*)(base + lay.off[R_PC2]);
    p.partCL = (double*)(base + lay.off[R_PCL]);
    p.jbits = (const uint8_t*)(base + lay.off[R_JB]);
    p.beta = (const double*)(base + lay.off[R_BETA]);
    p.dbeta = (const double*)(base + lay.off[R_DBETA]);
    p.q = (const double*)(base + lay.off[R_Q]);
    p.thr = (const uint32_t*)(base + lay.off[R_THR]);
    p.theta = (const uint32_t*)(base + lay.off[R_THETA]);
    p.st = (DevState*)(base + lay.off[R_ST]);
    p.trace = (TraceRow*)(base + lay.off[R_TRACE]);

    // per-step tables: dbeta, q = exp(-4 dbeta), Metropolis thresholds at beta_i
    std::vector<double> dbeta(n), q(n);
    std::vector<uint32_t> thr((size_t)4 * n);
    for (int i = 1; i <= n; ++i) {
        dbeta[i - 1] = ctx->beta[i] - ctx->beta[i - 1];
        q[i - 1] = std::exp(-(4.0 * dbeta[i - 1]));
        thr[4 * (i - 1)] = 0xFFFFFFFFu;
        for (int k = 1; k < 4; ++k) {
            const double x = ctx->beta[i] * (double)(4 * k);
            const double t = std::ldexp(std::exp(-x), 32);
            thr[4 * (i - 1) + k] = (t >= 4294967295.0) ? 0xFFFFFFFFu : (uint32_t)std::floor(t);
        }
    }
    DevState st0;
    std::memset(&st0, 0, sizeof(st0));
    st0.R_cur = m.R;
    st0.R_prev = m.R;

    cudaError_t e = cudaSuccess;
    auto up = [&](const void* dev, const void* host, size_t bytes) {
        if (e == cudaSuccess) e = cudaMemcpy((void*)dev, host, bytes, cudaMemcpyHostToDevice);
    };
    up(p.jbits, jb.data(), jb.size());
    up(p.beta, ctx->beta.data(), sizeof(double) * (n + 1));
    up(p.dbeta, dbeta.data(), sizeof(double) * n);
    up(p.q, q.data(), sizeof(double) * n);
    up(p.thr, thr.data(), sizeof(uint32_t) * 4 * n);
    up(p.theta, ctx->theta.data(), sizeof(uint32_t) * n);
    up(p.st, &st0, sizeof(st0));
    if (e == cudaSuccess) e = cudaMemsetAsync(p.hist, 0, (size_t)m.nlev * 4, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(p.trace, 0, (size_t)(n + 1) * sizeof(TraceRow), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p.counts, 0, (size_t)m.Rcap * 4, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p.anc, 0, (size_t)m.Rcap * 4, ctx->stream);
    if (e == cudaSuccess) e = launch_init_spins(p, ctx->stream);
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

pa_status pa_step(pa_ctx* ctx, int32_t n) {
    if (!ctx || n < 0) return PA_ERR_ARG;
    if (ctx->sticky != PA_OK) return PA_ERR_STATE;
    if (ctx->host_step + n > ctx->n_steps) return PA_ERR_DONE;
    for (int k = 0; k < n; ++k) {
        PA_CUDA(launch_resample(ctx->kp, ctx->stream, &ctx->launches));
        const int i = ctx->host_step + 1;
        if (ctx->timing) {
            cudaEvent_t a, b;
            PA_CUDA(cudaEventCreate(&a));
            PA_CUDA(cudaEventCreate(&b));
            ctx->ev_start.push_back(a);
            ctx->ev_stop.push_back(b);
            ctx->timed_steps.push_back(i);
            PA_CUDA(cudaEventRecord(a, ctx->stream));
        }
        PA_CUDA(launch_sweep(ctx->kp, ctx->threads, ctx->stream));
        ctx->launches += 1;
        if (ctx->timing) PA_CUDA(cudaEventRecord(ctx->ev_stop.back(), ctx->stream));
        PA_CUDA(launch_family_finish(ctx->kp, 0, ctx->stream, &ctx->launches));
        ctx->host_step = i;
    }
    return PA_OK;
}

pa_status pa_sync(pa_ctx* ctx) {
    if (!ctx) return PA_ERR_ARG;
    if (ctx->sticky != PA_OK) return ctx->sticky;
    DevState st;
    pa_status s = read_state(ctx, &st);
    if (s != PA_OK) return s;
    s = map_dev_status(st.status);
    if (s != PA_OK) ctx->sticky = s;
    return s;
}

pa_status pa_observables(pa_ctx* ctx, pa_obs* out) {
    if (!ctx || !out) return PA_ERR_ARG;
    pa_status s = pa_sync(ctx);
    if (s != PA_OK) return s;
    TraceRow t;
    PA_CUDA(cudaMemcpy(&t, ctx->kp.trace + ctx->host_step, sizeof(t), cudaMemcpyDeviceToHost));
    fill_obs(ctx, t, ctx->host_step, out);
    return PA_OK;
}

pa_status pa_trace(pa_ctx* ctx, pa_obs* rows, int32_t max_rows, int32_t* n_rows) {
    if (!ctx || !rows || max_rows < 0) return PA_ERR_ARG;
    pa_status s = pa_sync(ctx);
    if (s != PA_OK) return s;
    int n = ctx->host_step + 1;
    if (n > max_rows) n = max_rows;
    std::vector<TraceRow> t((size_t)n);
    if (n > 0)
        PA_CUDA(cudaMemcpy(t.data(), ctx->kp.trace, sizeof(TraceRow) * n, cudaMemcpyDeviceToHost));
    for (int i = 0; i < n; ++i) fill_obs(ctx, t[i], i, rows + i);
    if (n_rows) *n_rows = n;
    return PA_OK;
}

pa_status pa_free_energy(pa_ctx* ctx, double* minus_beta_F, double* f_per_spin) {
    if (!ctx) return PA_ERR_ARG;
    DevState st;
    pa_status s = pa_sync(ctx);
    if (s != PA_OK) return s;
    s = read_state(ctx, &st);
    if (s != PA_OK) return s;
    const double mbf = (double)ctx->N * std::log(2.0) + st.sum_lnQ;
    const double b = ctx->beta[ctx->host_step];
    if (minus_beta_F) *minus_beta_F = mbf;
    if (f_per_spin) *f_per_spin = b > 0 ? -mbf / (b * ctx->N) : NAN;
    return PA_OK;
}

pa_status pa_get_array(pa_ctx* ctx, pa_array which, void* host, size_t capacity, size_t* n_out) {
    if (!ctx || !host) return PA_ERR_ARG;
    pa_status s = pa_sync(ctx);
    if (s != PA_OK) return s;
    DevState st;
    s = read_state(ctx, &st);
    if (s != PA_OK) return s;
    const int par = ctx->host_step & 1;
    const KParams& p = ctx->kp;
    size_t n = 0;
    switch (which) {
        case PA_ARRAY_SPINS:
            n = (size_t)st.R_cur * ctx->W;
            if (capacity < n) return PA_ERR_ARG;
            if (st.R_cur)
                PA_CUDA(cudaMemcpy2D(host, (size_t)ctx->W * 4, p.spins[par], (size_t)ctx->Wp * 4,
                                     (size_t)ctx->W * 4, st.R_cur, cudaMemcpyDeviceToHost));
            break;
        case PA_ARRAY_ENERGY:
        case PA_ARRAY_FAMILY:
        case PA_ARRAY_ANCESTOR:
        case PA_ARRAY_MAGNET: {
            n = st.R_cur;
            if (capacity < n) return PA_ERR_ARG;
            const void* src = which == PA_ARRAY_ENERGY   ? (const void*)p.E[par]
                              : which == PA_ARRAY_FAMILY ? (const void*)p.fam[par]
                              : which == PA_ARRAY_MAGNET ? (const void*)p.M
                                                         : (const void*)p.anc;
            if (n) PA_CUDA(cudaMemcpy(host, src, n * 4, cudaMemcpyDeviceToHost));
            break;
        }
        case PA_ARRAY_COUNTS:
            n = ctx->host_step > 0 ? st.R_prev : 0;
            if (capacity < n) return PA_ERR_ARG;
            if (n) PA_CUDA(cudaMemcpy(host, p.counts, n * 4, cudaMemcpyDeviceToHost));
            break;
        default:
            return PA_ERR_ARG;
    }
    if (n_out) *n_out = n;
    return PA_OK;
}

pa_status pa_set_state(pa_ctx* ctx, const uint32_t* spins, const uint32_t* family, uint32_t R_i,
                       int32_t step, double sum_lnQ) {
    if (!ctx || !spins || R_i == 0 || R_i > ctx->Rcap || step < 0 || step > ctx->n_steps)
        return PA_ERR_ARG;
    if (ctx->sticky != PA_OK) return PA_ERR_STATE;
    const KParams& p = ctx->kp;
    const int par = step & 1;
    std::vector<uint32_t> fam((size_t)R_i);
    for (uint32_t j = 0; j < R_i; ++j) {
        fam[j] = family ? family[j] : j;
        if (fam[j] >= ctx->R) return PA_ERR_ARG;
        if (j > 0 && fam[j] < fam[j - 1]) return PA_ERR_ARG;  // families stay sorted by slot
    }
    PA_CUDA(cudaStreamSynchronize(ctx->stream));
    PA_CUDA(cudaMemset(p.spins[par], 0, (size_t)R_i * ctx->Wp * 4));
    PA_CUDA(cudaMemcpy2D(p.spins[par], (size_t)ctx->Wp * 4, spins, (size_t)ctx->W * 4,
                         (size_t)ctx->W * 4, R_i, cudaMemcpyHostToDevice));
    PA_CUDA(cudaMemcpy(p.fam[par], fam.data(), (size_t)R_i * 4, cudaMemcpyHostToDevice));
    DevState st;
    std::memset(&st, 0, sizeof(st));
    st.step = step;
    st.R_cur = R_i;
    st.R_prev = R_i;
    st.sum_lnQ = sum_lnQ;
    PA_CUDA(cudaMemcpy(p.st, &st, sizeof(st), cudaMemcpyHostToDevice));
    PA_CUDA(cudaMemset(p.hist, 0, (size_t)p.nlev * 4));
    TraceRow t;
    std::memset(&t, 0, sizeof(t));
    t.sum_lnQ = sum_lnQ;
    t.R_prev = R_i;
    PA_CUDA(cudaMemcpy(p.trace + step, &t, sizeof(t), cudaMemcpyHostToDevice));
    ctx->host_step = step;
    pa_status s = enqueue_measure(ctx);
    if (s != PA_OK) return s;
    return pa_sync(ctx);
}

pa_status pa_enable_timing(pa_ctx* ctx, int32_t on) {
    if (!ctx) return PA_ERR_ARG;
    ctx->timing = on != 0;
    return PA_OK;
}

pa_status pa_sweep_timing(pa_ctx* ctx, double* ms, int64_t* launches, double* updates) {
    if (!ctx) return PA_ERR_ARG;
    pa_status s = pa_sync(ctx);
    if (s != PA_OK) return s;
    double total = 0.0, upd = 0.0;
    std::vector<TraceRow> t((size_t)ctx->n_steps + 1);
    PA_CUDA(cudaMemcpy(t.data(), ctx->kp.trace, sizeof(TraceRow) * t.size(),
                       cudaMemcpyDeviceToHost));
    for (size_t k = 0; k < ctx->ev_start.size(); ++k) {
        float f = 0.f;
        PA_CUDA(cudaEventElapsedTime(&f, ctx->ev_start[k], ctx->ev_stop[k]));
        total += f;
        const int i = ctx->timed_steps[k];
        upd += (double)ctx->theta[i - 1] * (double)ctx->N * (double)t[i].R_i;
        cudaEventDestroy(ctx->ev_start[k]);
        cudaEventDestroy(ctx->ev_stop[k]);
    }
    if (ms) *ms = total;
    if (launches) *launches = (int64_t)ctx->ev_start.size();
    if (updates) *updates = upd;
    ctx->ev_start.clear();
    ctx->ev_stop.clear();
    ctx->timed_steps.clear();
    return PA_OK;
}

int64_t pa_launch_count(const pa_ctx* ctx) { return ctx ? ctx->launches : 0; }

pa_status pa_set_sweep_threads(pa_ctx* ctx, int32_t threads) {
    if (!ctx || !sweep_threads_supported(threads)) return PA_ERR_ARG;
    ctx->threads = threads;
    return PA_OK;
}

int32_t pa_get_sweep_threads(const pa_ctx* ctx) { return ctx ? ctx->threads : 0; }

pa_status pa_destroy(pa_ctx* ctx) {
    if (!ctx) return PA_OK;
    for (size_t k = 0; k < ctx->ev_start.size(); ++k) {
        cudaEventDestroy(ctx->ev_start[k]);
        cudaEventDestroy(ctx->ev_stop[k]);
    }
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
        case PA_ERR_LIMIT: return "size exceeds the static scratch limit of pa_weights_static";
        default: return "unknown status";
    }
}

}  // extern "C"
