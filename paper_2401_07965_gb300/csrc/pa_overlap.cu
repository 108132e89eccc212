// pa_overlap.cu -- overlap distribution of two independent populations of one
// disorder sample (the spin-glass observable of Sec. 4, Figs. 6 and 7).
//
// Runs a and b of a batch simulate the same lattice and couplings with
// independent draws.  At the current step, replica slot j of a is paired with
// slot j of b (j < min(R_i^a, R_i^b)); the pair's overlap is
// q = (1/N) sum_s sigma^a_s sigma^b_s = 1 - 2k/N, k = the number of sites where
// the two differ = popcount(row_a XOR row_b) (padding bits are zero in both).
//
// k_overlap_hist: G lanes per replica pair read the two rows with coalesced
// 128-bit loads, add the popcounts, reduce with shuffles, and one lane counts
// the pair in the CTA's shared-memory histogram, which is added to the pair's
// accumulator in the context's workspace at the end (counts are exact
// integers).  The last CTA of a pair to finish (a ticket counter) moves the
// accumulator into the caller's hist[p][k] with plain stores and leaves the
// accumulator and the ticket at zero for the next call, so no separate zeroing
// pass is needed.  The kernel is bound by HBM: 2 Wp words per replica pair are
// read once.
//
// k_overlap_P: one thread per k; the weighted estimate over pairs,
//   P(k) = sum_p omega_p hist_p[k] / n_p,  omega_p ∝ (R_i^a Zhat_a)(R_i^b Zhat_b),
// the product of the two populations' weights of Eq. (weighted-averages)
// (independent populations: the joint weight factorises), pairs summed in
// index order in FP64.
#include <algorithm>
#include <cmath>

#include "../../include/pa.h"
#include "pa_internal.cuh"

namespace pa {

// SMEM_HIST: counts go to a per-CTA shared-memory histogram first (one global
// atomic per non-empty bin per CTA); large lattices count in global memory.
template <bool SMEM_HIST>
__global__ void __launch_bounds__(256) k_overlap_hist(KParams p, const int32_t* pairs,
                                                      int lanes_per_pair, int bins,
                                                      uint32_t* hist, uint32_t* acc_all,
                                                      uint32_t* tickets) {
    extern __shared__ uint32_t sh[];
    __shared__ int last_cta;
    const int pair = blockIdx.y;
    const RunDesc& ra = p.runs[pairs[2 * pair]];
    const RunDesc& rb = p.runs[pairs[2 * pair + 1]];
    if (ra.st->status != S_OK || rb.st->status != S_OK) return;
    const int step = ra.st->step;
    const uint32_t n = min(ra.st->R_cur, rb.st->R_cur);
    const int G = lanes_per_pair;
    const int li = threadIdx.x % G;
    const int Wq = ra.Wp >> 2;  // 128-bit words per row
    uint32_t* out = hist + (size_t)pair * bins;
    uint32_t* acc = acc_all + (size_t)pair * bins;  // zero between calls
    if (SMEM_HIST) {
        for (int k = threadIdx.x; k < bins; k += blockDim.x) sh[k] = 0u;
        __syncthreads();
    }
    const uint32_t per_pass = (uint32_t)(gridDim.x * (blockDim.x / G));
    const uint4* A0 = reinterpret_cast<const uint4*>(ra.spins[step & 1]);
    const uint4* B0 = reinterpret_cast<const uint4*>(rb.spins[step & 1]);
    for (uint32_t j0 = blockIdx.x * (blockDim.x / G); j0 < n; j0 += per_pass) {
        const uint32_t j = j0 + threadIdx.x / G;
        uint32_t k = 0;
        if (j < n) {
            const uint4* A = A0 + (size_t)j * Wq;
            const uint4* B = B0 + (size_t)j * Wq;
            for (int c = li; c < Wq; c += G) {
                const uint4 x = A[c], y = B[c];
                k += __popc(x.x ^ y.x) + __popc(x.y ^ y.y) + __popc(x.z ^ y.z) +
                     __popc(x.w ^ y.w);
            }
        }
        // groups of G lanes are aligned within the warp (G divides 32)
        for (int o = G >> 1; o > 0; o >>= 1) k += __shfl_down_sync(0xffffffffu, k, o, G);
        if (li == 0 && j < n) {
            if (SMEM_HIST) atomicAdd(&sh[k], 1u);
            else atomicAdd(&acc[k], 1u);
        }
    }
    if (SMEM_HIST) {
        __syncthreads();
        for (int k = threadIdx.x; k < bins; k += blockDim.x)
            if (sh[k]) atomicAdd(&acc[k], sh[k]);
    }
    // make this CTA's additions visible, then take a ticket; the last CTA of the
    // pair sees every other CTA's additions
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last_cta = (atomicAdd(&tickets[pair], 1u) == gridDim.x - 1);
    __syncthreads();
    if (last_cta) {
        __threadfence();
        for (int k = threadIdx.x; k < bins; k += blockDim.x) out[k] = atomicExch(&acc[k], 0u);
        if (threadIdx.x == 0) tickets[pair] = 0u;
    }
}

__global__ void k_overlap_P(KParams p, const int32_t* pairs, int n_pairs, int bins,
                            const uint32_t* hist, double* P) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= bins) return;
    double lmax = -INFINITY;
    for (int q = 0; q < n_pairs; ++q) {
        const RunDesc& ra = p.runs[pairs[2 * q]];
        const RunDesc& rb = p.runs[pairs[2 * q + 1]];
        const TraceRow& ta = ra.trace[ra.st->step];
        const TraceRow& tb = rb.trace[rb.st->step];
        const double l = log((double)ta.R_i) + ta.sum_lnQ + log((double)tb.R_i) + tb.sum_lnQ;
        lmax = fmax(lmax, l);
    }
    double S = 0.0, acc = 0.0;
    for (int q = 0; q < n_pairs; ++q) {
        const RunDesc& ra = p.runs[pairs[2 * q]];
        const RunDesc& rb = p.runs[pairs[2 * q + 1]];
        const TraceRow& ta = ra.trace[ra.st->step];
        const TraceRow& tb = rb.trace[rb.st->step];
        const double w =
            exp(log((double)ta.R_i) + ta.sum_lnQ + log((double)tb.R_i) + tb.sum_lnQ - lmax);
        const double np = (double)min(ta.R_i, tb.R_i);
        S += w;
        acc += w * ((double)hist[(size_t)q * bins + k] / np);
    }
    P[k] = acc / S;
}

int overlap_lanes(int Wp) {
    int g = 1;
    while (g < 32 && 2 * g <= Wp / 4) g <<= 1;
    return g;
}

cudaError_t launch_overlap(const KParams& p, const int32_t* pairs, int n_pairs, int Wp,
                           uint32_t max_rows, int bins, uint32_t* hist, double* P,
                           uint32_t* acc, uint32_t* tickets, cudaStream_t s) {
    const int G = overlap_lanes(Wp);
    // CTAs per pair: about eight CTAs per SM over all pairs, each looping over
    // its share of the replica pairs
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const uint64_t passes = ((uint64_t)max_rows * G + 255) / 256;
    const uint64_t want = ((uint64_t)8 * nsm + n_pairs - 1) / n_pairs;
    const int per_pair = (int)std::max<uint64_t>(1, std::min<uint64_t>(passes, want));
    const dim3 grid((unsigned)per_pair, (unsigned)n_pairs);
    if (bins <= 12288)
        k_overlap_hist<true><<<grid, 256, (size_t)bins * 4, s>>>(p, pairs, G, bins, hist, acc,
                                                                 tickets);
    else
        k_overlap_hist<false><<<grid, 256, 0, s>>>(p, pairs, G, bins, hist, acc, tickets);
    e = cudaGetLastError();
    if (e != cudaSuccess || !P) return e;
    k_overlap_P<<<(bins + 127) / 128, 128, 0, s>>>(p, pairs, n_pairs, bins, hist, P);
    return cudaGetLastError();
}

}  // namespace pa
