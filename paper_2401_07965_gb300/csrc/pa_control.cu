// pa_control.cu -- the learned schedule controller (adaptive temperature steps
// and sweep numbers, cited as established practice in Sec. 5 of the paper) and
// the kernels that train its network.
//
// Network: 8 population statistics -> 64 -> 64 -> 2 (ReLU), BF16 parameters,
// FP32 accumulation in a fixed order (bias added last), no fused multiply-add.
// Outputs: s, the step size relative to the average remaining step, and t,
// the sweeps relative to the planned sweeps per step.
//
// Inference runs after every temperature step in one CTA (k_control): it
// reads the step's population sums, forms the features, evaluates the
// network, and writes the next step's entries of the step tables (beta on the
// schedule grid, dbeta, q = exp(-4 dbeta), Metropolis thresholds, theta) from
// tables precomputed on the host, so the PA step itself is unchanged and stays
// bit-exact.  With a non-finite or out-of-range output, or with the network
// switched off, the plain step (plain_units, plain_theta) is taken.
#include <cmath>
#include <cuda_bf16.h>

#include "../../include/pa.h"
#include "pa_internal.cuh"

namespace pa {

namespace {
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + MLP_HID * MLP_IN;
constexpr int OFF_W2 = OFF_B1 + MLP_HID;
constexpr int OFF_B2 = OFF_W2 + MLP_HID * MLP_HID;
constexpr int OFF_W3 = OFF_B2 + MLP_HID;
constexpr int OFF_B3 = OFF_W3 + MLP_OUT * MLP_HID;
constexpr int ROWS = 32;  // rows per CTA of the training kernels
}  // namespace

__device__ __forceinline__ float bf(uint16_t v) {
    return __uint_as_float(((uint32_t)v) << 16);
}

__device__ __forceinline__ float bf_round(float v) {
    return __bfloat162float(__float2bfloat16_rn(v));
}

// --------------------------------------------------------------------------
// controller step
//
// One CTA of 64 threads per run; its time is latency (one thread's FP64
// division or logarithm costs hundreds of cycles on this part), so the work is
// spread: each weight row is loaded into the registers of the thread that
// uses it at entry, the features are formed by threads 0-8 at once, and the
// step-table entries of every admissible step size are prefetched while the
// network runs.  Every value is formed by the same operations in the same
// order as a single thread would, so the results do not change.
// --------------------------------------------------------------------------
__device__ __forceinline__ float bf_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf_hi(uint32_t v) { return __uint_as_float(v & 0xFFFF0000u); }

// sum_k w[k] x[k] over a row of 64 BF16 weights held as 8 uint4, in order, then + bias
__device__ __forceinline__ float row64(const uint4 (&wr)[8], const float* xv, float bias) {
    float acc = 0.0f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const uint32_t v[4] = {wr[q].x, wr[q].y, wr[q].z, wr[q].w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            acc = __fadd_rn(acc, __fmul_rn(bf_lo(v[h]), xv[8 * q + 2 * h]));
            acc = __fadd_rn(acc, __fmul_rn(bf_hi(v[h]), xv[8 * q + 2 * h + 1]));
        }
    }
    return __fadd_rn(acc, bias);
}

__global__ void __launch_bounds__(64) k_control(KParams p) {
    static_assert(MLP_HID == 64 && MLP_IN == 8 && MLP_OUT == 2, "row layout of k_control");
    const RunDesc& r = p.runs[blockIdx.x];  // one CTA per run of the batch
    DevState* st = r.st;
    if (st->status != S_OK) return;
    const CtlDev& c = *p.ctl;
    const int i = st->step;
    const int kg = st->kgrid;
    TraceRow* tr = r.trace + i;
    __shared__ float x[MLP_IN], h1[MLP_HID], h2[MLP_HID], out[MLP_OUT];
    __shared__ double a5, lnR0;
    __shared__ double pbeta[CTL_UMAX], pdb[CTL_UMAX], pq[CTL_UMAX];
    __shared__ uint32_t pthr[CTL_UMAX][4];
    const int t = threadIdx.x;
    // the thread's weight rows (rows of 8 and 64 BF16 values are 16-byte aligned)
    const uint16_t* w = c.w;
    const uint4 w1 = *reinterpret_cast<const uint4*>(w + OFF_W1 + t * MLP_IN);
    uint4 w2[8], w3[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) w2[q] = reinterpret_cast<const uint4*>(w + OFF_W2 + t * MLP_HID)[q];
    if (t < MLP_OUT) {
#pragma unroll
        for (int q = 0; q < 8; ++q) w3[q] = reinterpret_cast<const uint4*>(w + OFF_W3 + t * MLP_HID)[q];
    }
    const float b1 = bf(w[OFF_B1 + t]), b2 = bf(w[OFF_B2 + t]);
    const float b3 = t < MLP_OUT ? bf(w[OFF_B3 + t]) : 0.0f;

    // features (R22), one per thread; thread 5's needs ln R_i and ln R (thread 8)
    {
        const double R = (double)tr->R_i, N = (double)r.N;
        if (t == 0) x[0] = (float)r.sbeta[i];
        if (t == 1 || t == 2) {
            const double mE = (double)(long long)tr->sumE / R;
            if (t == 1) {
                x[1] = (float)(mE / N);
            } else {
                const double var = ((double)(long long)tr->sumE2 / R - mE * mE) / N;
                x[2] = (float)(var / 10.0);
            }
        }
        if (t == 3) x[3] = (float)(tr->lnQ / N * 10.0);
        if (t == 4) x[4] = (float)((double)(long long)tr->sumC2 / (R * R));
        if (t == 5) a5 = log(R) - tr->c_ln_c / R;
        if (t == 6) {
            const double th = i > 0 ? (double)r.stheta[i - 1] : 0.0;
            x[6] = th > 0 ? (float)((double)tr->accepts / (th * N * R)) : 0.0f;
        }
        if (t == 7) x[7] = (float)r.L / 64.0f;
        if (t == 8) lnR0 = log(fmax((double)r.R, 2.0));
    }
    // the step tables of the admissible next steps u = 1 .. CTL_UMAX (k + u <= K)
    if (t >= 16 && t < 16 + CTL_UMAX) {
        const int u = t - 15;
        if (kg + u <= c.K) {
            const int kn = kg + u;
            pbeta[u - 1] = c.beta_grid[kn];
            pdb[u - 1] = c.dbeta_tab[(size_t)kg * CTL_UMAX + (u - 1)];
            pq[u - 1] = c.q_tab[(size_t)kg * CTL_UMAX + (u - 1)];
            for (int m = 0; m < 4; ++m) pthr[u - 1][m] = c.thr_grid[4 * kn + m];
        }
    }
    __syncthreads();
    if (t == 5) x[5] = (float)(a5 / lnR0);
    __syncthreads();
    if (t < MLP_IN) tr->x[t] = x[t];
    {
        const uint32_t v[4] = {w1.x, w1.y, w1.z, w1.w};
        float acc = 0.0f;
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            acc = __fadd_rn(acc, __fmul_rn(bf_lo(v[h]), x[2 * h]));
            acc = __fadd_rn(acc, __fmul_rn(bf_hi(v[h]), x[2 * h + 1]));
        }
        acc = __fadd_rn(acc, b1);
        h1[t] = acc > 0.0f ? acc : 0.0f;
    }
    __syncthreads();
    {
        const float acc = row64(w2, h1, b2);
        h2[t] = acc > 0.0f ? acc : 0.0f;
    }
    __syncthreads();
    if (t < MLP_OUT) out[t] = row64(w3, h2, b3);
    __syncthreads();
    if (t != 0) return;

    const int k = kg;
    const int D = c.K - k;
    if (D <= 0) {
        st->status = S_DONE;  // beta_f reached: the run is complete
        return;
    }
    const uint32_t used = st->sweeps;
    const uint32_t Brem = c.budget > used ? c.budget - used : 0u;
    const float s = out[0], tt = out[1];
    const bool ok = c.use_mlp && s == s && tt == tt && s >= 0.05f && s <= 20.0f && tt >= 0.05f &&
                    tt <= 20.0f;
    int u;
    uint32_t th;
    if (ok) {
        const float nrem = __fdiv_rn((float)Brem, c.theta_c);       // planned remaining steps
        const float ubar = __fdiv_rn((float)D, fmaxf(nrem, 1.0f));  // their average size
        const float uf = rintf(__fmul_rn(s, ubar));
        u = (int)fminf(fmaxf(uf, 1.0f), (float)c.u_max);
        const float tf = rintf(__fmul_rn(tt, c.theta_c));
        th = (uint32_t)fminf(fmaxf(tf, (float)c.theta_min), (float)c.theta_max);
    } else {
        u = c.plain_units;
        th = c.plain_theta;
    }
    if (u > D) u = D;
    if (ok) {
        // keep theta_min sweeps for each of the fewest steps that still reach beta_f
        const int need = (D - u + c.u_max - 1) / c.u_max;
        const long long cap = (long long)Brem - (long long)c.theta_min * need;
        if ((long long)th > cap) th = cap > (long long)c.theta_min ? (uint32_t)cap : c.theta_min;
    }
    const int kn = k + u;
    r.sbeta[i + 1] = pbeta[u - 1];
    r.sdbeta[i] = pdb[u - 1];
    r.sq[i] = pq[u - 1];
    for (int m = 0; m < 4; ++m) r.sthr[4 * i + m] = pthr[u - 1][m];
    r.stheta[i] = th;
    st->kgrid = kn;
    st->sweeps = used + th;
    tr->u_next = u;
    tr->theta_next = th;
}

cudaError_t launch_control(const KParams& p, cudaStream_t s) {
    k_control<<<p.M, 64, 0, s>>>(p);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// training: forward over a batch (parameters rounded to BF16 as in inference)
// --------------------------------------------------------------------------
template <bool MASTER>
__global__ void __launch_bounds__(64) k_mlp_fwd(const void* params, const float* __restrict__ X,
                                                int B, float* __restrict__ H1,
                                                float* __restrict__ H2, float* __restrict__ Y) {
    __shared__ float xs[ROWS][MLP_IN], a1[ROWS][MLP_HID], a2[ROWS][MLP_HID];
    __shared__ float W2s[MLP_HID * MLP_HID];
    const int t = threadIdx.x, r0 = blockIdx.x * ROWS;
    auto P = [&](int idx) -> float {
        return MASTER ? bf_round(((const float*)params)[idx]) : bf(((const uint16_t*)params)[idx]);
    };
    for (int e = t; e < ROWS * MLP_IN; e += 64) {
        const int rr = e / MLP_IN, k = e % MLP_IN;
        xs[rr][k] = (r0 + rr < B) ? X[(size_t)(r0 + rr) * MLP_IN + k] : 0.0f;
    }
    for (int e = t; e < MLP_HID * MLP_HID; e += 64) W2s[e] = P(OFF_W2 + e);
    __syncthreads();
    float w1[MLP_IN];
    for (int k = 0; k < MLP_IN; ++k) w1[k] = P(OFF_W1 + t * MLP_IN + k);
    const float b1 = P(OFF_B1 + t), b2 = P(OFF_B2 + t);
    for (int rr = 0; rr < ROWS; ++rr) {
        float acc = 0.0f;
        for (int k = 0; k < MLP_IN; ++k) acc = __fadd_rn(acc, __fmul_rn(w1[k], xs[rr][k]));
        acc = __fadd_rn(acc, b1);
        a1[rr][t] = acc > 0.0f ? acc : 0.0f;
    }
    __syncthreads();
    for (int rr = 0; rr < ROWS; ++rr) {
        float acc = 0.0f;
        for (int k = 0; k < MLP_HID; ++k) acc = __fadd_rn(acc, __fmul_rn(W2s[t * MLP_HID + k], a1[rr][k]));
        acc = __fadd_rn(acc, b2);
        a2[rr][t] = acc > 0.0f ? acc : 0.0f;
    }
    __syncthreads();
    const int rr = t >> 1, o = t & 1;
    float acc = 0.0f;
    for (int k = 0; k < MLP_HID; ++k) acc = __fadd_rn(acc, __fmul_rn(P(OFF_W3 + o * MLP_HID + k), a2[rr][k]));
    acc = __fadd_rn(acc, P(OFF_B3 + o));
    if (r0 + rr < B) Y[(size_t)(r0 + rr) * MLP_OUT + o] = acc;
    if (H1)
        for (int q = 0; q < ROWS; ++q)
            if (r0 + q < B) {
                H1[(size_t)(r0 + q) * MLP_HID + t] = a1[q][t];
                H2[(size_t)(r0 + q) * MLP_HID + t] = a2[q][t];
            }
}

// backward of the mean squared error over masked outputs; per-CTA partial
// gradients (row order fixed) in part[block][MLP_NPARAM + 1] (last: loss)
__global__ void __launch_bounds__(64) k_mlp_bwd(const float* __restrict__ params,
                                                const float* __restrict__ X,
                                                const float* __restrict__ Yt,
                                                const float* __restrict__ mask, int B,
                                                float norm, const float* __restrict__ H1,
                                                const float* __restrict__ H2,
                                                const float* __restrict__ Y,
                                                float* __restrict__ part) {
    __shared__ float dY[ROWS][MLP_OUT], d2[ROWS][MLP_HID], d1[ROWS][MLP_HID];
    __shared__ float a1[ROWS][MLP_HID], a2[ROWS][MLP_HID], xs[ROWS][MLP_IN];
    __shared__ float lossv[64];
    const int t = threadIdx.x, r0 = blockIdx.x * ROWS;
    for (int e = t; e < ROWS * MLP_HID; e += 64) {
        const int rr = e / MLP_HID, j = e % MLP_HID;
        const bool in = r0 + rr < B;
        a1[rr][j] = in ? H1[(size_t)(r0 + rr) * MLP_HID + j] : 0.0f;
        a2[rr][j] = in ? H2[(size_t)(r0 + rr) * MLP_HID + j] : 0.0f;
    }
    for (int e = t; e < ROWS * MLP_IN; e += 64) {
        const int rr = e / MLP_IN, k = e % MLP_IN;
        xs[rr][k] = (r0 + rr < B) ? X[(size_t)(r0 + rr) * MLP_IN + k] : 0.0f;
    }
    {
        const int rr = t >> 1, o = t & 1;
        float g = 0.0f, l = 0.0f;
        if (r0 + rr < B) {
            const size_t id = (size_t)(r0 + rr) * MLP_OUT + o;
            const float diff = __fsub_rn(Y[id], Yt[id]);
            const float mk = mask[id];
            g = __fmul_rn(__fmul_rn(2.0f, mk), __fmul_rn(diff, norm));
            l = __fmul_rn(mk, __fmul_rn(diff, diff));
        }
        dY[rr][o] = g;
        lossv[t] = l;
    }
    __syncthreads();
    // dH2 (thread t = hidden unit j)
    for (int rr = 0; rr < ROWS; ++rr) {
        float acc = 0.0f;
        for (int o = 0; o < MLP_OUT; ++o)
            acc = __fadd_rn(acc, __fmul_rn(dY[rr][o], bf_round(params[OFF_W3 + o * MLP_HID + t])));
        d2[rr][t] = a2[rr][t] > 0.0f ? acc : 0.0f;
    }
    __syncthreads();
    // dH1 (thread t = hidden unit i)
    for (int rr = 0; rr < ROWS; ++rr) {
        float acc = 0.0f;
        for (int j = 0; j < MLP_HID; ++j)
            acc = __fadd_rn(acc, __fmul_rn(d2[rr][j], bf_round(params[OFF_W2 + j * MLP_HID + t])));
        d1[rr][t] = a1[rr][t] > 0.0f ? acc : 0.0f;
    }
    __syncthreads();
    float* g = part + (size_t)blockIdx.x * (MLP_NPARAM + 1);
    // W1 row t, b1[t]
    for (int k = 0; k < MLP_IN; ++k) {
        float acc = 0.0f;
        for (int rr = 0; rr < ROWS; ++rr) acc = __fadd_rn(acc, __fmul_rn(d1[rr][t], xs[rr][k]));
        g[OFF_W1 + t * MLP_IN + k] = acc;
    }
    {
        float acc = 0.0f;
        for (int rr = 0; rr < ROWS; ++rr) acc = __fadd_rn(acc, d1[rr][t]);
        g[OFF_B1 + t] = acc;
    }
    // W2 row t (output unit t), b2[t]
    for (int k = 0; k < MLP_HID; ++k) {
        float acc = 0.0f;
        for (int rr = 0; rr < ROWS; ++rr) acc = __fadd_rn(acc, __fmul_rn(d2[rr][t], a1[rr][k]));
        g[OFF_W2 + t * MLP_HID + k] = acc;
    }
    {
        float acc = 0.0f;
        for (int rr = 0; rr < ROWS; ++rr) acc = __fadd_rn(acc, d2[rr][t]);
        g[OFF_B2 + t] = acc;
    }
    // W3 column t, b3
    for (int o = 0; o < MLP_OUT; ++o) {
        float acc = 0.0f;
        for (int rr = 0; rr < ROWS; ++rr) acc = __fadd_rn(acc, __fmul_rn(dY[rr][o], a2[rr][t]));
        g[OFF_W3 + o * MLP_HID + t] = acc;
    }
    if (t < MLP_OUT) {
        float acc = 0.0f;
        for (int rr = 0; rr < ROWS; ++rr) acc = __fadd_rn(acc, dY[rr][t]);
        g[OFF_B3 + t] = acc;
    }
    if (t == 0) {
        float acc = 0.0f;
        for (int q = 0; q < 64; ++q) acc = __fadd_rn(acc, lossv[q]);
        g[MLP_NPARAM] = __fmul_rn(acc, norm);
    }
}

// fixed-order sum of the per-CTA partials
__global__ void k_mlp_reduce(const float* __restrict__ part, int nb, float* __restrict__ grads,
                             float* __restrict__ loss) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > MLP_NPARAM) return;
    float acc = 0.0f;
    for (int b = 0; b < nb; ++b) acc = __fadd_rn(acc, part[(size_t)b * (MLP_NPARAM + 1) + k]);
    if (k < MLP_NPARAM) grads[k] = acc;
    else if (loss) *loss = acc;
}

// Adam (Kingma & Ba) on the FP32 master parameters; writes the BF16 copy
__global__ void k_mlp_adam(float* __restrict__ w, const float* __restrict__ g,
                           float* __restrict__ m, float* __restrict__ v,
                           uint16_t* __restrict__ wbf, float lr, float c1, float c2) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= MLP_NPARAM) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.0f - b1) * gk;
    const float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    const float wk = w[k] - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    w[k] = wk;
    if (wbf) wbf[k] = __bfloat16_as_ushort(__float2bfloat16_rn(wk));
}

}  // namespace pa

using namespace pa;

namespace {
size_t mlp_blocks(int B) { return (size_t)(B + ROWS - 1) / ROWS; }
}  // namespace

extern "C" {

size_t pa_mlp_scratch_bytes(int32_t B) {
    if (B <= 0) return 0;
    const size_t nb = mlp_blocks(B);
    return sizeof(float) * ((size_t)B * (2 * MLP_HID + MLP_OUT) + nb * (MLP_NPARAM + 1));
}

pa_status pa_mlp_forward(const uint16_t* params_bf16, const float* X, int32_t B, float* Y,
                         void* cuda_stream) {
    if (!params_bf16 || !X || !Y || B <= 0) return PA_ERR_ARG;
    k_mlp_fwd<false><<<(unsigned)mlp_blocks(B), 64, 0, (cudaStream_t)cuda_stream>>>(
        params_bf16, X, B, nullptr, nullptr, Y);
    return cudaGetLastError() == cudaSuccess ? PA_OK : PA_ERR_CUDA;
}

pa_status pa_mlp_gradients(const float* params, const float* X, const float* Yt,
                           const float* mask, int32_t B, float* grads, float* loss,
                           void* scratch, size_t scratch_bytes, void* cuda_stream) {
    if (!params || !X || !Yt || !mask || !grads || B <= 0 || !scratch) return PA_ERR_ARG;
    if (scratch_bytes < pa_mlp_scratch_bytes(B)) return PA_ERR_NOMEM;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    float* H1 = (float*)scratch;
    float* H2 = H1 + (size_t)B * MLP_HID;
    float* Y = H2 + (size_t)B * MLP_HID;
    float* part = Y + (size_t)B * MLP_OUT;
    const unsigned nb = (unsigned)mlp_blocks(B);
    const float norm = 1.0f / (float)(B * MLP_OUT);
    k_mlp_fwd<true><<<nb, 64, 0, s>>>(params, X, B, H1, H2, Y);
    k_mlp_bwd<<<nb, 64, 0, s>>>(params, X, Yt, mask, B, norm, H1, H2, Y, part);
    k_mlp_reduce<<<(MLP_NPARAM + 256) / 256, 256, 0, s>>>(part, (int)nb, grads, loss);
    return cudaGetLastError() == cudaSuccess ? PA_OK : PA_ERR_CUDA;
}

pa_status pa_mlp_adam(float* params, const float* grads, float* m, float* v, uint16_t* params_bf16,
                      int32_t step, float lr, void* cuda_stream) {
    if (!params || !grads || !m || !v || step < 1 || !(lr > 0.0f)) return PA_ERR_ARG;
    const float c1 = 1.0f - powf(0.9f, (float)step), c2 = 1.0f - powf(0.999f, (float)step);
    k_mlp_adam<<<(MLP_NPARAM + 255) / 256, 256, 0, (cudaStream_t)cuda_stream>>>(
        params, grads, m, v, params_bf16, lr, c1, c2);
    return cudaGetLastError() == cudaSuccess ? PA_OK : PA_ERR_CUDA;
}

}  // extern "C"
