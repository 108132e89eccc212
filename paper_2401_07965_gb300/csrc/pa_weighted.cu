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
// One thread per step; runs are summed in index order (fixed order).
#include <cmath>

#include "../../include/pa.h"
#include "pa_internal.cuh"

namespace pa {

__global__ void k_weighted(KParams p, const int32_t* run_ids, int n_runs, int n_rows,
                           pa_weighted_obs* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_rows) return;
    const RunDesc& r0 = p.runs[run_ids[0]];
    const double N = (double)r0.N;
    const double beta = p.beta[i];
    double amax = -INFINITY, bmax = -INFINITY, Rnom = 0.0;
    for (int k = 0; k < n_runs; ++k) {
        const RunDesc& r = p.runs[run_ids[k]];
        const TraceRow& t = r.trace[i];
        amax = fmax(amax, log((double)t.R_i) + t.sum_lnQ);
        bmax = fmax(bmax, log((double)r.R) + t.sum_lnQ);
        Rnom += (double)r.R;
    }
    double S = 0.0, Sb = 0.0;
    for (int k = 0; k < n_runs; ++k) {
        const RunDesc& r = p.runs[run_ids[k]];
        const TraceRow& t = r.trace[i];
        S += exp(log((double)t.R_i) + t.sum_lnQ - amax);
        Sb += exp(log((double)r.R) + t.sum_lnQ - bmax);
    }
    double We = 0, We2 = 0, Wam = 0, Wm2 = 0, cn = 0, xn = 0, w2 = 0, wmax = 0;
    double pe = 0, pc = 0, px = 0;
    for (int k = 0; k < n_runs; ++k) {
        const RunDesc& r = p.runs[run_ids[k]];
        const TraceRow& t = r.trace[i];
        const double w = exp(log((double)t.R_i) + t.sum_lnQ - amax) / S;
        const double Ri = (double)t.R_i;
        // per-run averages: plain, or weighted under partial resampling
        const bool wtd = p.alpha >= 0.0 && t.wsum > 0.0;
        const double e = wtd ? t.wE / (t.wsum * N) : (double)(long long)t.sumE / (Ri * N);
        const double e2 =
            wtd ? t.wE2 / (t.wsum * N * N) : (double)(long long)t.sumE2 / (Ri * N * N);
        const double am = wtd ? t.wAM / (t.wsum * N) : (double)(long long)t.sumAbsM / (Ri * N);
        const double m2 =
            wtd ? t.wM2 / (t.wsum * N * N) : (double)(long long)t.sumM2 / (Ri * N * N);
        const double c = beta * beta * N * (e2 - e * e);
        const double x = beta * N * (m2 - am * am);
        We += w * e;
        We2 += w * e2;
        Wam += w * am;
        Wm2 += w * m2;
        cn += w * c;
        xn += w * x;
        w2 += w * w;
        wmax = fmax(wmax, w);
        pe += e;
        pc += c;
        px += x;
    }
    pa_weighted_obs o;
    o.step = i;
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
    out[i] = o;
}

cudaError_t launch_weighted(const KParams& p, const int32_t* run_ids, int n_runs, int n_rows,
                            pa_weighted_obs* out, cudaStream_t s) {
    k_weighted<<<(n_rows + 127) / 128, 128, 0, s>>>(p, run_ids, n_runs, n_rows, out);
    return cudaGetLastError();
}

}  // namespace pa
