// pa_control.cuh -- the learned schedule controller's step (adaptive temperature
// steps and sweep numbers, cited as established practice in Sec. 5 of the
// paper), shared by the kernel that makes the first decision of a run and by
// the family kernel, whose last CTA of a run makes the decision after every
// step (one kernel boundary less per step).
//
// Network: 8 population statistics -> 64 -> 64 -> 2 (ReLU), BF16 parameters,
// FP32 accumulation in a fixed order (bias added last), no fused multiply-add.
#pragma once

#include "pa_internal.cuh"

namespace pa {

namespace {
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + MLP_HID * MLP_IN;
constexpr int OFF_W2 = OFF_B1 + MLP_HID;
constexpr int OFF_B2 = OFF_W2 + MLP_HID * MLP_HID;
constexpr int OFF_W3 = OFF_B2 + MLP_HID;
constexpr int OFF_B3 = OFF_W3 + MLP_OUT * MLP_HID;
}  // namespace

__device__ __forceinline__ float bf(uint16_t v) {
    return __uint_as_float(((uint32_t)v) << 16);
}

// --------------------------------------------------------------------------
// controller step
//
// Called by every thread of one CTA of at least 64 threads per run (threads
// 0-63 work, the others only take part in the barriers).  Its time is latency:
// a dependent FP64 operation costs tens of cycles on this part and a logarithm
// about 2000, so the work is spread and the chains kept short.  Each weight
// row is loaded into the registers of the thread that uses it at entry; the
// features are formed by threads 0-7 at once, with products by 1/R_i in place
// of divisions and ln R_i from the host's ln R (equal to the direct formulas to
// an FP64 rounding or two, below the FP32 rounding of the features); the
// step-table entries of every admissible step size are prefetched while the
// network runs, whose sums keep the fixed order.  It writes the next step's
// entries of the step tables (beta on the schedule grid, dbeta, q, thresholds,
// theta) from tables precomputed on the host; a non-finite or out-of-range
// output, or the network switched off, takes the plain step (plain_units,
// plain_theta).
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

__device__ __forceinline__ void control_after_step(const KParams& p, const RunDesc& r,
                                                   DevState* st) {
    static_assert(MLP_HID == 64 && MLP_IN == 8 && MLP_OUT == 2, "row layout of the controller");
    if (st->status != S_OK) return;
    const CtlDev& c = *p.ctl;
    const int i = st->step;
    const int kg = st->kgrid;
    TraceRow* tr = r.trace + i;
    __shared__ float x[MLP_IN], h1[MLP_HID], h2[MLP_HID], out[MLP_OUT];
    __shared__ double pbeta[CTL_UMAX], pdb[CTL_UMAX], pq[CTL_UMAX];
    __shared__ uint32_t pthr[CTL_UMAX][4];
    const int t = threadIdx.x < 64 ? (int)threadIdx.x : 0;  // threads past 64 only wait
    const bool act = threadIdx.x < 64;
    // the thread's weight rows (rows of 8 and 64 BF16 values are 16-byte aligned)
    const uint16_t* w = c.w;
    const uint4 w1 = *reinterpret_cast<const uint4*>(w + OFF_W1 + t * MLP_IN);
    uint4 w2[8], w3[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) w2[q] = reinterpret_cast<const uint4*>(w + OFF_W2 + t * MLP_HID)[q];
    if (act && t < MLP_OUT) {
#pragma unroll
        for (int q = 0; q < 8; ++q) w3[q] = reinterpret_cast<const uint4*>(w + OFF_W3 + t * MLP_HID)[q];
    }
    const float b1 = bf(w[OFF_B1 + t]), b2 = bf(w[OFF_B2 + t]);
    const float b3 = t < MLP_OUT ? bf(w[OFF_B3 + t]) : 0.0f;

    // features (R22), one per thread (threads 0-7).  The FP64 divisions and
    // logarithms of this part have long dependent chains (a logarithm takes about
    // 2000 cycles), so each thread's chain is kept short: 1/R_i once, products
    // after it, and ln R_i = ln R + log1p((R_i - R) / R) from the host's ln R
    // (R_i = R for the fixed-size rules) with the small correction in FP32.
    if (act && t < MLP_IN) {
        const double Ri = (double)tr->R_i, N = (double)r.N;
        const double invR = 1.0 / Ri;
        float v;
        if (t == 0) {
            v = (float)r.sbeta[i];
        } else if (t == 1 || t == 2) {
            const double mE = (double)(long long)tr->sumE * invR;
            if (t == 1) {
                v = (float)(mE / N);
            } else {
                const double var = ((double)(long long)tr->sumE2 * invR - mE * mE) / N;
                v = (float)(var * 0.1);
            }
        } else if (t == 3) {
            v = (float)(tr->lnQ / N * 10.0);
        } else if (t == 4) {
            v = (float)((double)(long long)tr->sumC2 * invR * invR);
        } else if (t == 5) {
            const float dR = __fdiv_rn((float)((long long)tr->R_i - (long long)r.R), (float)r.R);
            const double lnRi = r.lnR + (double)log1pf(dR);
            v = (float)((lnRi - tr->c_ln_c * invR) / r.lnR);
        } else if (t == 6) {
            const double th = i > 0 ? (double)r.stheta[i - 1] : 0.0;
            v = th > 0 ? (float)((double)tr->accepts * invR / (th * N)) : 0.0f;
        } else {
            v = (float)r.L / 64.0f;
        }
        x[t] = v;
    }
    // the step tables of the admissible next steps u = 1 .. CTL_UMAX (k + u <= K)
    if (act && t >= 16 && t < 16 + CTL_UMAX) {
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
    if (act && t < MLP_IN) tr->x[t] = x[t];
    {
        const uint32_t v[4] = {w1.x, w1.y, w1.z, w1.w};
        float acc = 0.0f;
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            acc = __fadd_rn(acc, __fmul_rn(bf_lo(v[h]), x[2 * h]));
            acc = __fadd_rn(acc, __fmul_rn(bf_hi(v[h]), x[2 * h + 1]));
        }
        acc = __fadd_rn(acc, b1);
        if (act) h1[t] = acc > 0.0f ? acc : 0.0f;
    }
    __syncthreads();
    {
        const float acc = row64(w2, h1, b2);
        if (act) h2[t] = acc > 0.0f ? acc : 0.0f;
    }
    __syncthreads();
    if (act && t < MLP_OUT) out[t] = row64(w3, h2, b3);
    __syncthreads();
    if (threadIdx.x != 0) return;

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

}  // namespace pa
