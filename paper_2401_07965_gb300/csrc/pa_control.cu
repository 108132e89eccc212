// pa_control.cu -- the learned schedule controller (adaptive temperature steps
// and sweep numbers, cited as established practice in Sec. 5 of the paper) and
// the kernels that train its network.
//
// Network: 8 population statistics -> 64 -> 64 -> 2 (ReLU), BF16 parameters,
// FP32 accumulation in a fixed order (bias added last), no fused multiply-add.
// Outputs: s, the step size relative to the average remaining step, and t,
// the sweeps relative to the planned sweeps per step.
//
// Inference (pa_control.cuh) runs once per run when the controller is switched
// on (k_control) and then after every temperature step in the family kernel's
// last CTA of the run: it writes the next step's entries of the step tables
// from tables precomputed on the host, so the PA step itself is unchanged and
// stays bit-exact.
#include <cmath>
#include <cuda_bf16.h>

#include "../../include/pa.h"
#include "pa_control.cuh"

namespace pa {

namespace {
constexpr int ROWS = 32;  // rows per CTA of the training kernels
}  // namespace

__device__ __forceinline__ float bf_round(float v) {
    return __bfloat162float(__float2bfloat16_rn(v));
}

// --------------------------------------------------------------------------
// controller step: the first decision of a run (at pa_set_controller); after
// every step the family kernel's last CTA of the run makes it
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(64) k_control(KParams p) {
    const RunDesc& r = p.runs[blockIdx.x];  // one CTA per run of the batch
    control_after_step(p, r, r.st);
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
