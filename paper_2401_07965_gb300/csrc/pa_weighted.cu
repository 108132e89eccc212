// pa_weighted.cu -- weighted averages of repeated runs (Sec. 4 of the paper).
//
// Runs that repeat one system (same lattice and couplings, any population
// size) carry weights omega_i^(m) proportional to R_i^(m) exp(-beta_i F_i^(m))
// (Eq. weighted-averages), where -beta_i F_i^(m) = ln Z_0 + sum_k ln Q_k^(m)
// (Eq. free-energy-estimator); ln Z_0 is common to the runs and cancels.
// From each run's exact per-step sums the kernel forms, per temperature step,
//   W[e], W[e^2], W[|m|], W[m^2]                      (Eq. weighted-averages)
//   Wvar[c] = beta^2 N (W[e^2] - W[e]^2)              (Eq. Wvar_C)
//   Wvar[chi] = beta N (W[m^2] - W[|m|]^2)            (Eq. Wvar_Chi)
//   the naive weighting sum_m omega c^(m), sum_m omega chi^(m), the plain
//   means over runs, and the combined estimate of ln(Z_i / Z_0) as
//   ln( sum_m R^(m) Zhat_m / sum_m R^(m) ).
// One thread per step; runs are summed in index order (fixed order).  The
// same combination serves the runs of one batch (k_weighted, from the trace
// rows) and runs summarised anywhere else, e.g. on other GPUs
// (k_weighted_rows, from rows the caller passes in).
#include <cmath>

#include "../../include/pa.h"
#include "pa_internal.cuh"

namespace pa {

// what the combination needs of one run at one step
struct RunMoments {
    double Ri, Rnom, slnq;  // R_i, nominal R, sum of ln Q
    double e, e2, am, m2;   // per-run averages (weighted under partial resampling)
};

template <class Get>
__device__ pa_weighted_obs combine_runs(int n_runs, double N, double beta, int step, Get get) {
    double amax = -INFINITY, bmax = -INFINITY, Rnom = 0.0;
    for (int k = 0; k < n_runs; ++k) {
        const RunMoments r = get(k);
        amax = fmax(amax, log(r.Ri) + r.slnq);
        bmax = fmax(bmax, log(r.Rnom) + r.slnq);
        Rnom += r.Rnom;
    }
    double S = 0.0, Sb = 0.0;
    for (int k = 0; k < n_runs; ++k) {
        const RunMoments r = get(k);
        S += exp(log(r.Ri) + r.slnq - amax);
        Sb += exp(log(r.Rnom) + r.slnq - bmax);
    }
    double We = 0, We2 = 0, Wam = 0, Wm2 = 0, cn = 0, xn = 0, w2 = 0, wmax = 0;
    double pe = 0, pc = 0, px = 0;
    for (int k = 0; k < n_runs; ++k) {
        const RunMoments r = get(k);
        const double w = exp(log(r.Ri) + r.slnq - amax) / S;
        const double c = beta * beta * N * (r.e2 - r.e * r.e);
        const double x = beta * N * (r.m2 - r.am * r.am);
        We += w * r.e;
        We2 += w * r.e2;
        Wam += w * r.am;
        Wm2 += w * r.m2;
        cn += w * c;
        xn += w * x;
        w2 += w * w;
        wmax = fmax(wmax, w);
        pe += r.e;
        pc += c;
        px += x;
    }
    pa_weighted_obs o;
    o.step = step;
    o.n_runs = n_runs;
    o.beta = beta;
    o.lnZ = bmax + log(Sb) - log(Rnom);
    o.minus_beta_F = N * log(2.0) + o.lnZ;
    o.w_max = wmax;
    o.eff_runs = 1.0 / w2;
    o.e = We;
    o.e2 = We2;
    o.absm = Wam;
    o.m2 = Wm2;
    o.c = beta * beta * N * (We2 - We * We);
    o.chi = beta * N * (Wm2 - Wam * Wam);
    o.c_naive = cn;
    o.chi_naive = xn;
    o.e_plain = pe / n_runs;
    o.c_plain = pc / n_runs;
    o.chi_plain = px / n_runs;
    return o;
}

// per-run averages from the exact sums, or from the weighted sums if wsum > 0
__device__ __forceinline__ RunMoments moments(double Ri, double Rnom, double slnq, double N,
                                              long long sE, long long sE2, long long sAM,
                                              long long sM2, double wsum, double wE,
                                              double wE2, double wAM, double wM2) {
    RunMoments m;
    m.Ri = Ri;
    m.Rnom = Rnom;
    m.slnq = slnq;
    const bool wtd = wsum > 0.0;
    m.e = wtd ? wE / (wsum * N) : (double)sE / (Ri * N);
    m.e2 = wtd ? wE2 / (wsum * N * N) : (double)sE2 / (Ri * N * N);
    m.am = wtd ? wAM / (wsum * N) : (double)sAM / (Ri * N);
    m.m2 = wtd ? wM2 / (wsum * N * N) : (double)sM2 / (Ri * N * N);
    return m;
}

__global__ void k_weighted(KParams p, const int32_t* run_ids, int n_runs, int n_rows,
                           pa_weighted_obs* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_rows) return;
    const double N = (double)p.runs[run_ids[0]].N;
    const bool partial = p.alpha >= 0.0;
    out[i] = combine_runs(n_runs, N, p.beta[i], i, [&](int k) {
        const RunDesc& r = p.runs[run_ids[k]];
        const TraceRow& t = r.trace[i];
        return moments((double)t.R_i, (double)r.R, t.sum_lnQ, N, (long long)t.sumE,
                       (long long)t.sumE2, (long long)t.sumAbsM, (long long)t.sumM2,
                       partial ? t.wsum : 0.0, t.wE, t.wE2, t.wAM, t.wM2);
    });
}

__global__ void k_weighted_rows(const pa_run_row* rows, int n_runs, int N, double beta,
                                int32_t step, pa_weighted_obs* out) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const double Nd = (double)N;
    out[0] = combine_runs(n_runs, Nd, beta, step, [&](int k) {
        const pa_run_row& r = rows[k];
        return moments((double)r.R_i, (double)r.R, r.sum_lnQ, Nd, (long long)r.sumE,
                       (long long)r.sumE2, (long long)r.sumAbsM, (long long)r.sumM2, r.wsum,
                       r.wE, r.wE2, r.wAM, r.wM2);
    });
}

cudaError_t launch_weighted(const KParams& p, const int32_t* run_ids, int n_runs, int n_rows,
                            pa_weighted_obs* out, cudaStream_t s) {
    k_weighted<<<(n_rows + 127) / 128, 128, 0, s>>>(p, run_ids, n_runs, n_rows, out);
    return cudaGetLastError();
}

}  // namespace pa

using namespace pa;

extern "C" pa_status pa_weighted_rows(const pa_run_row* rows, int32_t n_runs, int32_t N,
                                      double beta, int32_t step, pa_weighted_obs* out,
                                      void* cuda_stream) {
    if (!rows || !out || n_runs < 1 || N < 1) return PA_ERR_ARG;
    for (int k = 0; k < n_runs; ++k)
        if (rows[k].R_i == 0 || rows[k].R == 0) return PA_ERR_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    pa_run_row* d_rows = nullptr;
    pa_weighted_obs* d_out = nullptr;
    if (cudaMalloc(&d_rows, sizeof(pa_run_row) * n_runs) != cudaSuccess) return PA_ERR_NOMEM;
    if (cudaMalloc(&d_out, sizeof(pa_weighted_obs)) != cudaSuccess) {
        cudaFree(d_rows);
        return PA_ERR_NOMEM;
    }
    cudaError_t e = cudaMemcpyAsync(d_rows, rows, sizeof(pa_run_row) * n_runs,
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        k_weighted_rows<<<1, 32, 0, s>>>(d_rows, n_runs, N, beta, step, d_out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, d_out, sizeof(pa_weighted_obs), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_rows);
    cudaFree(d_out);
    return e == cudaSuccess ? PA_OK : PA_ERR_CUDA;
}
