// pa_resample.cu -- reweighting, Q and copy counts (Sec. 2 step 2, Sec. 3),
// the scan-plus-scatter that builds the ancestor array of the new population,
// and the family / sampling-variance measurements (Eqs. rho_t, sv).
//
// All floating-point work uses explicitly rounded IEEE double operations
// (no fused multiply-add) in a fixed order, so that the fixed-point weights
// and therefore every count are reproducible bit for bit:
//   level l = U >> 1 of a replica (U unsatisfied bonds), E = 2U - dN,
//   w_k = q^k (q = exp(-4 dbeta), binary powering), k = l - l_min,
//   S = fixed pairwise tree sum of n_k w_k over a power-of-two array,
//   ln Q = (ln S - ln R_{i-1}) - dbeta E_min,
//   f_k = floor(2^40 * ((R w_k) / S))  (tau-hat of Eq. taus in 2^-40 units).
// The copy counts are exact integer functions of f and of Philox draws.
//
// Partial resampling (alpha >= 0): replicas carry weights w_j.  The step
// multiplies them by the level factors q^(l_j - l_min) (k_pw_update), sums
// old and new weights and the squares in balanced binary trees over the
// replica index (blocks of SCAN_CHUNK aligned replicas, then the blocks:
// k_pw_final), and resamples with f_j = floor(2^40 (R wn_j) / S_new) only if
// (sum wn)^2 / sum wn^2 < alpha R_{i-1}; otherwise every replica is kept once
// and its weight is rescaled by a power of two (k_family).
#include <climits>

#include "pa_control.cuh"

namespace pa {

// q^k by binary powering from a table of the squares qsq[m] = q^(2^m), each the
// rounded square of the one before (qsq[0] = q): the product of the squares of
// the set bits of k, least significant first, every multiply rounded -- the
// same value as squaring and multiplying in one loop, with popc(k) multiplies
// on the dependent chain.
__device__ __forceinline__ double pow_tab(const double* qsq, uint32_t k) {
    double r = 1.0;
    for (int m = 0; k; ++m, k >>= 1)
        if (k & 1u) r = __dmul_rn(r, qsq[m]);
    return r;
}

// exp(x) = 2^n sum_{k<=13} r^k / k!, x = n ln2 + r (Cody-Waite reduction),
// every operation explicitly rounded.  Used for the Poisson rule, x in [-16, 0].
__device__ __forceinline__ double exp_taylor(double x) {
    const double INV_LN2 = 0x1.71547652b82fep+0;
    const double LN2_HI = 0x1.62e42fefa3800p-1;
    const double LN2_LO = 0x1.ef35793c76730p-45;
    const double c[14] = {0x1.0000000000000p+0,  0x1.0000000000000p+0,  0x1.0000000000000p-1,
                          0x1.5555555555555p-3,  0x1.5555555555555p-5,  0x1.1111111111111p-7,
                          0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-13, 0x1.a01a01a01a01ap-16,
                          0x1.71de3a556c734p-19, 0x1.27e4fb7789f5cp-22, 0x1.ae64567f544e4p-26,
                          0x1.1eed8eff8d898p-29, 0x1.6124613a86d09p-33};
    const double nd = floor(__dadd_rn(__dmul_rn(x, INV_LN2), 0.5));
    const double r = __dsub_rn(__dsub_rn(x, __dmul_rn(nd, LN2_HI)), __dmul_rn(nd, LN2_LO));
    double pp = c[13];
#pragma unroll
    for (int k = 12; k >= 0; --k) pp = __dadd_rn(__dmul_rn(pp, r), c[k]);
    return scalbn(pp, (int)nd);
}

struct U128 {
    uint64_t hi, lo;
};
__device__ __forceinline__ U128 mul128(uint64_t a, uint64_t b) { return {__umul64hi(a, b), a * b}; }
__device__ __forceinline__ bool lt128(U128 a, U128 b) {
    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__device__ __forceinline__ bool le128(U128 a, U128 b) { return !lt128(b, a); }

// Systematic rule: number of labels (k + u/2^32) T/R, k in [0,R), below x:
// with xR = aT + b, that is a + [b 2^32 > u T], at most R.
__device__ uint64_t sys_below(uint64_t x, uint64_t R, uint64_t T, uint32_t u) {
    const U128 P = mul128(x, R);
    // a = floor(xR / T) <= R < 2^24: an FP32 estimate is within a few units (FP64 is
    // slow on this part), and the 128-bit corrections below make it exact
    uint64_t a = (uint64_t)__fdiv_rn(__fmul_rn((float)x, (float)R), (float)T);
    for (int it = 0; it < 8 && lt128(P, mul128(a, T)); ++it) --a;
    for (int it = 0; it < 8 && le128(mul128(a + 1, T), P); ++it) ++a;
    const uint64_t b = P.lo - a * T;  // < T, exact in the low 64 bits
    const U128 lhs = {b >> 32, b << 32};
    const U128 rhs = mul128((uint64_t)u, T);
    const uint64_t n = a + (lt128(rhs, lhs) ? 1u : 0u);
    return n < R ? n : R;
}

__device__ __forceinline__ int level_of(int32_t E, int dN) {
    return ((E + dN) >> 1) >> 1;  // U = (E + dN)/2, level = U >> 1
}

// --------------------------------------------------------------------------
// block helpers
// --------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

// exclusive block scan of one value per thread (blockDim == SCAN_THREADS)
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* sh, T* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T incl = warp_incl_scan(v, lane);
    if (lane == 31) sh[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T w = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : (T)0;
        T wi = warp_incl_scan(w, lane);
        sh[lane] = wi - w;
        if (lane == 31) sh[32] = wi;
    }
    __syncthreads();
    T res = sh[warp] + incl - v;
    *total = sh[32];
    __syncthreads();
    return res;
}

// balanced binary tree sums (adjacent pairs first) in explicitly rounded FP64:
// over 8 or 16 consecutive values, and over the threads of a CTA (thread t =
// leaf t, blockDim a power of two); the root ends in every thread
template <int NL>
__device__ __forceinline__ double tree_regs(const double* a) {
    double t[NL];
#pragma unroll
    for (int k = 0; k < NL; ++k) t[k] = a[k];
#pragma unroll
    for (int w = 1; w < NL; w <<= 1)
#pragma unroll
        for (int k = 0; k + w < NL; k += 2 * w) t[k] = __dadd_rn(t[k], t[k + w]);
    return t[0];
}

__device__ double tree_threads(double v, double* sh) {
    // levels inside a warp by shuffles (lane t adds lane t + w for t a multiple
    // of 2w: the same pairs as the tree), then the same over the warps' sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int w = 1; w < 32; w <<= 1) v = __dadd_rn(v, __shfl_down_sync(0xffffffffu, v, w));
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double u = lane < nw ? sh[lane] : 0.0;
        for (int w = 1; w < nw; w <<= 1) u = __dadd_rn(u, __shfl_down_sync(0xffffffffu, u, w));
        if (lane == 0) sh[32] = u;
    }
    __syncthreads();
    const double root = sh[32];
    __syncthreads();
    return root;
}

__device__ double max_threads(double v, double* sh) {
    const int t = threadIdx.x, n = blockDim.x;
    sh[t] = v;
    __syncthreads();
    for (int w = n >> 1; w >= 1; w >>= 1) {
        if (t < w) sh[t] = fmax(sh[t], sh[t + w]);
        __syncthreads();
    }
    const double root = sh[0];
    __syncthreads();
    return root;
}

// --------------------------------------------------------------------------
// K3: weights, S, ln Q, f table (one CTA)
//
// One CTA of 1024 threads; its time is latency, not work, so the phases are
// kept few: the level counts are read from global memory once (into shared
// memory, while the occupied range is found), the logarithms of ln Q run on a
// warp that has no level of its own while the others compute f.
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_weights(KParams p) {
    const RunDesc& r = p.runs[blockIdx.x];
    DevState* st = r.st;
    if (st->status != S_OK) return;
    constexpr int TREE_SMEM = 2048;
    // tree and weights; before the tree is built, the counts of the K occupied
    // levels (cached when they fit in its 4 TREE_SMEM words)
    __shared__ double tw[2 * TREE_SMEM];
    double* tsm = tw;
    double* wsm = tw + TREE_SMEM;
    uint32_t* hc = reinterpret_cast<uint32_t*>(tw);
    __shared__ double qsq[32], S_sh, lnS_sh, lnR_sh;
    const int i = st->step + 1;
    const uint32_t Rprev = st->R_cur;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (int)(blockDim.x >> 5);
    // the occupied level range, recorded by the kernels that filled the histogram
    // (the lowest and highest level any replica took)
    const int lo = st->hlo, hi = st->hhi;
    const int lmin = lo;
    const int K = hi >= lo ? hi - lo + 1 : 0;
    const bool cached = K <= 4 * TREE_SMEM;
    if (cached)
        for (int k = threadIdx.x; k < K; k += blockDim.x) hc[k] = r.hist[lmin + k];
    __syncthreads();
    int P = 1;
    while (P < K) P <<= 1;
    const double q = r.sq[i - 1];
    // the squares q^(2^m) for the bits of k < K
    if (threadIdx.x == 0) {
        const int nb = K > 1 ? 32 - __clz(K - 1) : 0;
        double b = q;
        for (int m = 0; m < nb; ++m) {
            qsq[m] = b;
            b = __dmul_rn(b, b);
        }
    }
    const bool in_smem = P <= TREE_SMEM;
    // the counts of the thread's levels k = threadIdx.x + j blockDim.x, j < 2 (all
    // of them when the tree is in shared memory)
    uint32_t n0 = 0u, n1 = 0u;
    if (in_smem) {
        const int k0 = threadIdx.x, k1 = threadIdx.x + blockDim.x;
        if (k0 < K) n0 = cached ? hc[k0] : r.hist[lmin + k0];
        if (k1 < K) n1 = cached ? hc[k1] : r.hist[lmin + k1];
    }
    __syncthreads();  // qsq written; the count cache is free for the tree
    if (p.alpha >= 0.0) {
        // partial resampling: the level factors q^k; k_pw_final closes the step
        double* wl = reinterpret_cast<double*>(r.flev);
        for (int k = threadIdx.x; k < K; k += blockDim.x) wl[k] = pow_tab(qsq, (uint32_t)k);
        __syncthreads();
        for (int k = threadIdx.x; k < K; k += blockDim.x) r.hist[lmin + k] = 0u;
        if (threadIdx.x == 0) {
            st->R_prev = Rprev;
            st->lmin = (uint32_t)lmin;
            st->K = (uint32_t)K;
            st->hlo = 0x7FFFFFFF;  // the histogram is empty again
            st->hhi = -1;
            TraceRow* tr = r.trace + i;
            tr->c_ln_c = 0.0;
            tr->sv_sum = 0.0;
            tr->sumE = tr->sumE2 = tr->sumAbsM = tr->sumM2 = tr->sumC2 = tr->accepts = 0ull;
            tr->R_prev = Rprev;
            tr->R_i = 0;
        }
        return;
    }
    // S = sum_k n_k w_k as the fixed pairwise tree (t_k += t_{k+h}, h = P/2 ... 1) over
    // the zero-padded array: in shared memory when it fits (the usual case: the
    // occupied levels span a few hundred), else in the run's global scratch; the
    // last five levels by warp shuffles with the same pairs
    int h = P >> 1;
    if (in_smem) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int k = threadIdx.x + j * blockDim.x;
            if (k < P) {
                double v = 0.0;
                if (k < K) {
                    const double wk = pow_tab(qsq, (uint32_t)k);
                    wsm[k] = wk;
                    v = __dmul_rn((double)(j == 0 ? n0 : n1), wk);
                }
                tsm[k] = v;
            }
        }
        __syncthreads();
        for (; h >= 32; h >>= 1) {
            for (int k = threadIdx.x; k < h; k += blockDim.x)
                tsm[k] = __dadd_rn(tsm[k], tsm[k + h]);
            __syncthreads();
        }
    } else {
        volatile double* t = r.tree;
        for (int k = threadIdx.x; k < P; k += blockDim.x)
            t[k] = k < K ? __dmul_rn((double)r.hist[lmin + k], pow_tab(qsq, (uint32_t)k)) : 0.0;
        __threadfence_block();
        __syncthreads();
        for (; h >= 32; h >>= 1) {
            for (int k = threadIdx.x; k < h; k += blockDim.x) t[k] = __dadd_rn(t[k], t[k + h]);
            __threadfence_block();
            __syncthreads();
        }
    }
    if (warp == 0) {
        const int live = h > 0 ? 2 * h : 1;  // entries left after the shared-memory levels
        const volatile double* t = in_smem ? tsm : r.tree;
        double v = lane < live ? t[lane] : 0.0;
        for (; h >= 1; h >>= 1) v = __dadd_rn(v, __shfl_down_sync(0xffffffffu, v, h));
        if (lane == 0) S_sh = v;
    }
    __syncthreads();
    const double S = S_sh;
    // ln S and ln R_{i-1} on the last warp (lanes 0 and 1, one pass), before its levels
    if (warp == nwarps - 1) {
        const double lx = log(lane == 0 ? S : (double)Rprev);
        if (lane == 0) lnS_sh = lx;
        if (lane == 1) lnR_sh = lx;
    }
    const double Rd = (double)r.R;
    // f_k, and the totals T = sum_j f_j = sum_k n_k f_k and of the fractional parts
    // (exact integer sums; the copy-count kernels need them before any scan)
    unsigned long long sT = 0, sTr = 0;
    for (int k = threadIdx.x, j = 0; k < K; k += blockDim.x, ++j) {
        double a = __dmul_rn(Rd, in_smem ? wsm[k] : pow_tab(qsq, (uint32_t)k));
        a = __ddiv_rn(a, S);
        a = scalbn(a, FRAC_BITS);
        const uint64_t f = (uint64_t)floor(a);
        r.flev[k] = f;
        const uint64_t n = in_smem ? (j == 0 ? n0 : n1) : r.hist[lmin + k];
        sT += n * f;
        sTr += n * (f & ((1ull << FRAC_BITS) - 1));
    }
    for (int o = 16; o > 0; o >>= 1) {
        sT += __shfl_xor_sync(0xffffffffu, sT, o);
        sTr += __shfl_xor_sync(0xffffffffu, sTr, o);
    }
    __shared__ unsigned long long tsum[2];
    if (threadIdx.x == 0) tsum[0] = tsum[1] = 0ull;
    __syncthreads();
    if (lane == 0) {
        atomicAdd(&tsum[0], sT);
        atomicAdd(&tsum[1], sTr);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) r.hist[lmin + k] = 0u;
    if (threadIdx.x == 0) {
        st->T = tsum[0];
        st->Tres = tsum[1];
        st->Rres = (uint64_t)r.R - ((tsum[0] - tsum[1]) >> FRAC_BITS);
        st->epoch += 1u;
        st->kmax = 0;
        const int32_t Umin = 2 * lmin + r.parity;
        const int32_t Emin = 2 * Umin - p.d * r.N;
        const double lnQ = __dsub_rn(__dsub_rn(lnS_sh, lnR_sh),
                                     __dmul_rn(r.sdbeta[i - 1], (double)Emin));
        st->R_prev = Rprev;
        st->lmin = (uint32_t)lmin;
        st->K = (uint32_t)K;
        st->hlo = 0x7FFFFFFF;  // the histogram is empty again
        st->hhi = -1;
        st->sum_lnQ = __dadd_rn(st->sum_lnQ, lnQ);
        TraceRow* tr = r.trace + i;
        tr->lnQ = lnQ;
        tr->sum_lnQ = st->sum_lnQ;
        tr->c_ln_c = 0.0;
        tr->sv_sum = 0.0;
        tr->sumE = tr->sumE2 = tr->sumAbsM = tr->sumM2 = tr->sumC2 = tr->accepts = 0ull;
        tr->R_prev = Rprev;
        tr->R_i = 0;
    }
}

// --------------------------------------------------------------------------
// partial resampling: new weights and their per-block tree sums
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(SCAN_THREADS) k_pw_update(KParams p) {
    const RunDesc& r = p.runs[p.blk2run[blockIdx.x]];
    const uint32_t b = blockIdx.x - r.blk0;
    const DevState* st = r.st;
    if (st->status != S_OK) return;
    __shared__ double sh[SCAN_THREADS];
    const int i = st->step + 1;
    const int32_t* E = r.E[(i - 1) & 1];
    const uint32_t Rprev = st->R_prev, lmin = st->lmin;
    const int dN = p.d * r.N;
    const double* wl = reinterpret_cast<const double*>(r.flev);
    const int j0 = b * SCAN_CHUNK + threadIdx.x * SCAN_ITEMS;
    double wo[SCAN_ITEMS], wn[SCAN_ITEMS], w2[SCAN_ITEMS];
    double mx = 0.0;
#pragma unroll
    for (int e = 0; e < SCAN_ITEMS; ++e) {
        const int j = j0 + e;
        wo[e] = wn[e] = w2[e] = 0.0;
        if ((uint32_t)j < Rprev) {
            wo[e] = r.w[j];
            wn[e] = __dmul_rn(wo[e], wl[level_of(E[j], dN) - (int)lmin]);
            w2[e] = __dmul_rn(wn[e], wn[e]);
            r.w[j] = wn[e];
            mx = fmax(mx, wn[e]);
        }
    }
    const double s_old = tree_threads(tree_regs<SCAN_ITEMS>(wo), sh);
    const double s_new = tree_threads(tree_regs<SCAN_ITEMS>(wn), sh);
    const double s2 = tree_threads(tree_regs<SCAN_ITEMS>(w2), sh);
    mx = max_threads(mx, sh);
    if (threadIdx.x == 0) {
        r.wpart[4 * b + 0] = s_old;
        r.wpart[4 * b + 1] = s_new;
        r.wpart[4 * b + 2] = s2;
        r.wpart[4 * b + 3] = mx;
    }
}

// one CTA per run: tree over the blocks, ln Q, effective size, decision
__global__ void __launch_bounds__(1024) k_pw_final(KParams p) {
    const RunDesc& r = p.runs[blockIdx.x];
    DevState* st = r.st;
    if (st->status != S_OK) return;
    __shared__ double sh[1024];
    const int i = st->step + 1;
    const int nb = r.nblk;  // <= PARTIAL_MAX_BLOCKS = LEAVES leaves x 1024 threads
    constexpr int LEAVES = PARTIAL_MAX_BLOCKS / 1024;
    double S[3];
    for (int q = 0; q < 3; ++q) {
        double x[LEAVES];
#pragma unroll
        for (int k = 0; k < LEAVES; ++k) {
            const int bb = LEAVES * threadIdx.x + k;
            x[k] = bb < nb ? r.wpart[4 * bb + q] : 0.0;
        }
        S[q] = tree_threads(tree_regs<LEAVES>(x), sh);
    }
    double mx = 0.0;
    for (int bb = threadIdx.x; bb < nb; bb += blockDim.x) mx = fmax(mx, r.wpart[4 * bb + 3]);
    mx = max_threads(mx, sh);
    if (threadIdx.x == 0) {
        const uint32_t Rprev = st->R_prev;
        const int32_t Umin = 2 * (int32_t)st->lmin + r.parity;
        const int32_t Emin = 2 * Umin - p.d * r.N;
        const double lnQ = __dsub_rn(__dsub_rn(log(S[1]), log(S[0])),
                                     __dmul_rn(r.sdbeta[i - 1], (double)Emin));
        const double ess = __ddiv_rn(__dmul_rn(S[1], S[1]), S[2]);
        const int res = ess < __dmul_rn(p.alpha, (double)Rprev) ? 1 : 0;
        int e = 0;
        frexp(mx, &e);
        st->resample = res;
        st->wexp = e;
        st->S_new = S[1];
        st->sum_lnQ = __dadd_rn(st->sum_lnQ, lnQ);
        TraceRow* tr = r.trace + i;
        tr->lnQ = lnQ;
        tr->sum_lnQ = st->sum_lnQ;
        tr->ess = ess;
        tr->resampled = res;
    }
}

// weights of a new run: 1
__global__ void k_pw_init(KParams p) {
    const RunDesc& r = p.runs[blockIdx.y];
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < r.Rcap; j += gridDim.x * blockDim.x)
        r.w[j] = 1.0;
}

// --------------------------------------------------------------------------
// per-block sums of f (and of its 2^-40 fractional part)
// --------------------------------------------------------------------------
// expected copies of parent j in 2^-40 units: the level table, or under
// partial resampling floor(2^40 (R wn_j) / S_new) when the step resamples and
// exactly one copy when it does not
__device__ __forceinline__ uint64_t f_of(int j, const KParams& p, const RunDesc& r,
                                         const DevState* st, int dN, const int32_t* E,
                                         uint32_t lmin) {
    if (p.alpha >= 0.0) {
        if (!st->resample) return 1ull << FRAC_BITS;
        double a = __dmul_rn((double)r.R, r.w[j]);
        a = __ddiv_rn(a, st->S_new);
        a = scalbn(a, FRAC_BITS);
        return (uint64_t)floor(a);
    }
    return r.flev[level_of(E[j], dN) - (int)lmin];
}

__global__ void __launch_bounds__(SCAN_THREADS) k_fsum(KParams p) {
    const RunDesc& r = p.runs[p.blk2run[blockIdx.x]];
    const uint32_t b = blockIdx.x - r.blk0;
    const DevState* st = r.st;
    if (st->status != S_OK) return;
    if (p.alpha >= 0.0 && !st->resample) return;  // partial: population kept
    __shared__ uint64_t sh[33];
    const int i = st->step + 1;
    const int32_t* E = r.E[(i - 1) & 1];
    const uint32_t Rprev = st->R_prev, lmin = st->lmin;
    const int dN = p.d * r.N;
    const int j0 = b * SCAN_CHUNK + threadIdx.x * SCAN_ITEMS;
    uint64_t sf = 0, sg = 0;
    for (int e = 0; e < SCAN_ITEMS; ++e) {
        const int j = j0 + e;
        if ((uint32_t)j < Rprev) {
            const uint64_t f = f_of(j, p, r, st, dN, E, lmin);
            sf += f;
            sg += f & ((1ull << FRAC_BITS) - 1);
        }
    }
    uint64_t tot;
    block_excl_scan(sf, sh, &tot);
    if (threadIdx.x == 0) r.partA[b] = tot;
    block_excl_scan(sg, sh, &tot);
    if (threadIdx.x == 0) r.partB[b] = tot;
}

// exclusive scan of the per-block partials (one CTA of 1024 threads)
__device__ void scan_partials(const uint64_t* part, uint64_t* off, int n, uint64_t* total_out) {
    __shared__ uint64_t sh[33];
    __shared__ uint64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < n; b0 += blockDim.x) {
        const int b = b0 + threadIdx.x;
        const uint64_t v = (b < n) ? part[b] : 0ull;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        uint64_t incl = warp_incl_scan(v, lane);
        if (lane == 31) sh[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint64_t w = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0ull;
            uint64_t wi = warp_incl_scan(w, lane);
            sh[lane] = wi - w;
            if (lane == 31) sh[32] = wi;
        }
        __syncthreads();
        if (b < n) off[b] = carry + sh[warp] + incl - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += sh[32];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total_out = carry;
}

__global__ void __launch_bounds__(1024) k_fscan(KParams p) {
    const RunDesc& r = p.runs[blockIdx.x];
    DevState* st = r.st;
    if (st->status != S_OK) return;
    if (p.alpha >= 0.0 && !st->resample) return;
    __shared__ uint64_t tA, tB;
    scan_partials(r.partA, r.offA, r.nblk, &tA);
    scan_partials(r.partB, r.offB, r.nblk, &tB);
    __syncthreads();
    if (threadIdx.x == 0) {
        st->T = tA;
        st->Tres = tB;
        const uint64_t A = (tA - tB) >> FRAC_BITS;  // sum of floor(f / 2^40)
        st->Rres = (uint64_t)r.R - A;
    }
}

// --------------------------------------------------------------------------
// prefix sums C (and G) and the copy counts of the rules that need no search
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(SCAN_THREADS) k_counts(KParams p) {
    const RunDesc& r = p.runs[p.blk2run[blockIdx.x]];
    const uint32_t b = blockIdx.x - r.blk0;
    DevState* st = r.st;
    if (st->status != S_OK) return;
    __shared__ uint64_t sh[33];
    const int i = st->step + 1;
    const int32_t* E = r.E[(i - 1) & 1];
    const int dN = p.d * r.N;
    const uint32_t Rprev = st->R_prev, lmin = st->lmin;
    const uint64_t T = st->T;
    const int j0 = b * SCAN_CHUNK + threadIdx.x * SCAN_ITEMS;
    if (p.alpha >= 0.0 && !st->resample) {
        // partial resampling keeps every replica once: identity counts and
        // ancestors, no sampling variance (the scan kernels return at once)
        for (int e = 0; e < SCAN_ITEMS; ++e) {
            const int j = j0 + e;
            if ((uint32_t)j < Rprev) {
                r.counts[j] = 1u;
                r.anc[j] = (uint32_t)j;
            }
        }
        if (threadIdx.x == 0) r.partD[b] = 0.0;
        return;
    }
    uint64_t f[SCAN_ITEMS];
    uint64_t sf = 0, sg = 0;
#pragma unroll
    for (int e = 0; e < SCAN_ITEMS; ++e) {
        const int j = j0 + e;
        f[e] = ((uint32_t)j < Rprev) ? f_of(j, p, r, st, dN, E, lmin) : 0ull;
        sf += f[e];
        sg += f[e] & ((1ull << FRAC_BITS) - 1);
    }
    uint64_t tot;
    uint64_t cf = block_excl_scan(sf, sh, &tot) + r.offA[b];
    uint64_t cg = block_excl_scan(sg, sh, &tot) + r.offB[b];
    const int method = p.method;
    uint32_t usys = 0;
    if (method == M_SYSTEMATIC)
        usys = philox(0u, DOM_RESAMPLE | (r.run << 8) | RULE_SYSTEMATIC, (uint32_t)i, 0u, p.k0, p.k1).x;
    bool kmax = false;
#pragma unroll 1
    for (int e = 0; e < SCAN_ITEMS; ++e) {
        const int j = j0 + e;
        if ((uint32_t)j >= Rprev) break;
        const uint64_t prevC = cf;
        cf += f[e];
        cg += f[e] & ((1ull << FRAC_BITS) - 1);
        r.C[j] = cf;
        if (method == M_RESIDUAL) r.G[j] = cg;
        uint32_t cnt = 0;
        if (method == M_NEAREST) {
            const uint4x x = philox((uint32_t)j, DOM_RESAMPLE | (r.run << 8) | RULE_NEAREST, (uint32_t)i, 0u,
                                    p.k0, p.k1);
            const uint64_t u40 = (((uint64_t)x.y << 32) | x.x) >> 24;
            cnt = (uint32_t)(f[e] >> FRAC_BITS) +
                  (u40 < (f[e] & ((1ull << FRAC_BITS) - 1)) ? 1u : 0u);
        } else if (method == M_SYSTEMATIC) {
            cnt = (uint32_t)(sys_below(cf, r.R, T, usys) - sys_below(prevC, r.R, T, usys));
        } else if (method == M_RESIDUAL) {
            cnt = (uint32_t)(f[e] >> FRAC_BITS);
        } else if (method == M_POISSON) {
            const double lam = scalbn((double)f[e], -FRAC_BITS);
            const uint32_t M = (uint32_t)(f[e] >> 44) + 1u;
            const double lc = __ddiv_rn(lam, (double)M);
            uint32_t total = 0;
            for (uint32_t m = 0; m < M; ++m) {
                const uint4x x = philox((uint32_t)j, DOM_RESAMPLE | (r.run << 8) | RULE_POISSON, (uint32_t)i, m,
                                        p.k0, p.k1);
                const double u = scalbn((double)((((uint64_t)x.y << 32) | x.x) >> 11), -53);
                double pr = exp_taylor(-lc);
                double Pc = pr;
                uint32_t k = 0;
                while (u >= Pc) {
                    k += 1;
                    if (k > POISSON_KMAX) {
                        kmax = true;
                        break;
                    }
                    pr = __ddiv_rn(__dmul_rn(pr, lc), (double)k);
                    Pc = __dadd_rn(Pc, pr);
                }
                total += k;
            }
            cnt = total;
        }
        r.counts[j] = cnt;
    }
    if (kmax) atomicCAS(&st->status, S_OK, S_KMAX);
}

// multinomial draws (multinomial rule: R draws over C; residual rule: R_res
// draws over the remainders G, or over C if every remainder is zero)
__global__ void __launch_bounds__(SCAN_THREADS) k_draws(KParams p) {
    const RunDesc& r = p.runs[p.blk2run[blockIdx.x]];
    const uint32_t b = blockIdx.x - r.blk0;
    const DevState* st = r.st;
    if (st->status != S_OK) return;
    if (p.alpha >= 0.0 && !st->resample) return;  // partial: no resampling this step
    const int i = st->step + 1;
    const uint32_t Rprev = st->R_prev;
    uint64_t n;
    const uint64_t* box;
    uint64_t total;
    uint32_t rule;
    if (p.method == M_MULTINOMIAL) {
        n = r.R;
        box = r.C;
        total = st->T;
        rule = RULE_MULTINOMIAL;
    } else {
        n = st->Rres;
        const bool use_g = st->Tres > 0;
        box = use_g ? r.G : r.C;
        total = use_g ? st->Tres : st->T;
        rule = RULE_RESIDUAL;
    }
    const uint64_t stride = (uint64_t)r.nblk * SCAN_THREADS;
    for (uint64_t k = (uint64_t)b * SCAN_THREADS + threadIdx.x; k < n; k += stride) {
        const uint4x x = philox((uint32_t)(k >> 1), DOM_RESAMPLE | (r.run << 8) | rule, (uint32_t)i,
                                0u, p.k0, p.k1);
        const uint64_t u = (k & 1) ? (((uint64_t)x.w << 32) | x.z) : (((uint64_t)x.y << 32) | x.x);
        const uint64_t pos = __umul64hi(u, total);
        uint32_t lo = 0, hi = Rprev;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (pos < box[mid]) hi = mid;
            else lo = mid + 1;
        }
        atomicAdd(&r.counts[lo], 1u);
    }
}

// --------------------------------------------------------------------------
// scan of the counts and scatter of the ancestor array
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(SCAN_THREADS) k_rsum(KParams p) {
    const RunDesc& r = p.runs[p.blk2run[blockIdx.x]];
    const uint32_t b = blockIdx.x - r.blk0;
    const DevState* st = r.st;
    if (st->status != S_OK) return;
    if (p.alpha >= 0.0 && !st->resample) return;
    __shared__ uint64_t sh[33];
    const uint32_t Rprev = st->R_prev;
    const int j0 = b * SCAN_CHUNK + threadIdx.x * SCAN_ITEMS;
    uint64_t s = 0;
    for (int e = 0; e < SCAN_ITEMS; ++e) {
        const int j = j0 + e;
        if ((uint32_t)j < Rprev) s += r.counts[j];
    }
    uint64_t tot;
    block_excl_scan(s, sh, &tot);
    if (threadIdx.x == 0) r.partA[b] = tot;
}

__global__ void __launch_bounds__(1024) k_rscan(KParams p) {
    const RunDesc& r = p.runs[blockIdx.x];
    DevState* st = r.st;
    if (st->status != S_OK) return;
    if (p.alpha >= 0.0 && !st->resample) return;  // R_i = R_{i-1}
    __shared__ uint64_t tA;
    scan_partials(r.partA, r.offA, r.nblk, &tA);
    __syncthreads();
    if (threadIdx.x == 0) {
        // a population that outgrows its capacity, or dies out, stops the run
        if (tA > (uint64_t)r.Rcap || tA == 0) st->status = S_CAPACITY;
        else st->R_cur = (uint32_t)tA;
    }
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scatter(KParams p) {
    const RunDesc& r = p.runs[p.blk2run[blockIdx.x]];
    const uint32_t b = blockIdx.x - r.blk0;
    const DevState* st = r.st;
    if (st->status != S_OK) return;
    if (p.alpha >= 0.0 && !st->resample) return;  // identity written by k_counts
    __shared__ uint64_t sh[33];
    __shared__ double sd[SCAN_THREADS];
    const int i = st->step + 1;
    const int32_t* E = r.E[(i - 1) & 1];
    const int dN = p.d * r.N;
    const uint32_t Rprev = st->R_prev, lmin = st->lmin;
    const int j0 = b * SCAN_CHUNK + threadIdx.x * SCAN_ITEMS;
    uint32_t rc[SCAN_ITEMS];
    uint64_t s = 0;
#pragma unroll
    for (int e = 0; e < SCAN_ITEMS; ++e) {
        const int j = j0 + e;
        rc[e] = ((uint32_t)j < Rprev) ? r.counts[j] : 0u;
        s += rc[e];
    }
    uint64_t tot;
    uint64_t o = block_excl_scan(s, sh, &tot) + r.offA[b];
    double sv = 0.0;
    for (int e = 0; e < SCAN_ITEMS; ++e) {
        const int j = j0 + e;
        if ((uint32_t)j >= Rprev) break;
        for (uint32_t c = 0; c < rc[e]; ++c) r.anc[o + c] = (uint32_t)j;
        o += rc[e];
        const double tau = scalbn((double)f_of(j, p, r, st, dN, E, lmin), -FRAC_BITS);
        const double dl = __dsub_rn((double)rc[e], tau);
        sv = __dadd_rn(sv, __dmul_rn(dl, dl));
    }
    // fixed-order tree reduction of the block's sampling-variance terms
    sd[threadIdx.x] = sv;
    __syncthreads();
    for (int h = SCAN_THREADS / 2; h >= 1; h >>= 1) {
        if ((int)threadIdx.x < h) sd[threadIdx.x] = __dadd_rn(sd[threadIdx.x], sd[threadIdx.x + h]);
        __syncthreads();
    }
    if (threadIdx.x == 0) r.partD[b] = sd[0];
}

// --------------------------------------------------------------------------
// family statistics of the new population (families stay sorted by slot)
// --------------------------------------------------------------------------
template <bool PARTIAL>
__device__ void finish_run(const KParams& p, const RunDesc& r, DevState* st, int mode, double* a,
                           double* b, double* ws);

// PARTIAL: partial resampling (weighted sums); CTL: the run's last CTA then
// takes the learned controller's decision for the next step.  Separate
// instances keep the registers of the plain step's kernel low.
template <bool PARTIAL, bool CTL>
__global__ void __launch_bounds__(SCAN_THREADS) k_family(KParams p, int mode) {
    const RunDesc& r = p.runs[p.blk2run[blockIdx.x]];
    const uint32_t b = blockIdx.x - r.blk0;
    DevState* st = r.st;
    if (st->status != S_OK) return;
    __shared__ double sd[SCAN_THREADS], fa[SCAN_THREADS], fb[SCAN_THREADS];
    __shared__ unsigned long long sc2;
    __shared__ int last;
    const int i = (mode == 0) ? st->step + 1 : st->step;
    const uint32_t Ri = st->R_cur;
    const uint32_t* fam = r.fam[i & 1];
    const int j0 = b * SCAN_CHUNK + threadIdx.x * SCAN_ITEMS;
    // Families stay sorted by slot, so a family is a run of equal values.  The
    // block's slots go to shared memory; each run start finds its end from the
    // 32-slot masks of run starts, and warp 0 searches the array beyond the block
    // for the end of the block's last run, which may go on past it.  c ln c of
    // small families comes from a table the host computes once.
    constexpr int FTAB = CLN_TAB;
    __shared__ uint32_t sf[SCAN_CHUNK];
    __shared__ uint32_t smask[SCAN_CHUNK / 32];
    __shared__ double clt[FTAB + 1];
    const uint32_t B0 = b * SCAN_CHUNK;
    const uint32_t nin = B0 < Ri ? min((uint32_t)SCAN_CHUNK, Ri - B0) : 0u;
    if (threadIdx.x == 0) sc2 = 0ull;
    for (int c = threadIdx.x; c <= FTAB; c += blockDim.x) clt[c] = p.clnc[c];
    for (int l = threadIdx.x; l < SCAN_CHUNK; l += blockDim.x)
        sf[l] = (uint32_t)l < nin ? fam[B0 + l] : 0xFFFFFFFFu;
    __syncthreads();
    const uint32_t before = (B0 > 0 && nin) ? fam[B0 - 1] : 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int rnd = 0; rnd < SCAN_CHUNK / SCAN_THREADS; ++rnd) {
        const int l = rnd * SCAN_THREADS + warp * 32 + lane;
        const bool st_l = (uint32_t)l < nin && (l == 0 ? (B0 == 0 || before != sf[0])
                                                       : sf[l - 1] != sf[l]);
        const uint32_t m = __ballot_sync(0xffffffffu, st_l);
        if (lane == 0) smask[rnd * (SCAN_THREADS / 32) + warp] = m;
    }
    __syncthreads();
    double cl = 0.0;
    unsigned long long c2 = 0;
    __shared__ int slast;  // the block's last run start (-1: no slot in the block)
    if (threadIdx.x == 0) slast = -1;
    __syncthreads();
    for (int rnd = 0; rnd < SCAN_CHUNK / SCAN_THREADS; ++rnd) {
        const int l = rnd * SCAN_THREADS + warp * 32 + lane;
        int q = l >> 5;
        const int bit = l & 31;
        if (!((smask[q] >> bit) & 1u)) continue;  // not a run start (or past R_i)
        uint32_t m = bit == 31 ? 0u : (smask[q] & (0xFFFFFFFFu << (bit + 1)));
        while (m == 0u && q + 1 < SCAN_CHUNK / 32) m = smask[++q];
        if (!m) {  // the block's last run: it may continue past the block (below)
            slast = l;
            continue;
        }
        const uint64_t c = (uint64_t)(q * 32 + __ffs(m) - 1 - l);
        c2 += c * c;
        if (c > 1) cl = __dadd_rn(cl, c <= FTAB ? clt[c] : __dmul_rn((double)c, log((double)c)));
    }
    __syncthreads();
    // The last run ends at the first slot from B0 + nin on whose family differs
    // (families are sorted, so "differs" holds from there on): warp 0 finds it by
    // a 32-way search, each round sampling 32 evenly spaced slots of the interval
    // that holds the end (at most five rounds below 2^24 slots).
    if (warp == 0 && slast >= 0) {
        const uint32_t f = sf[slast];
        uint32_t lo = B0 + nin, hi = Ri;  // the end lies in [lo, hi]
        while (hi - lo > 32u) {
            const uint32_t step = (hi - lo + 31u) / 32u;
            const uint32_t pos = lo + (uint32_t)lane * step;
            const bool ne = pos >= hi || fam[pos] != f;
            const uint32_t bal = __ballot_sync(0xffffffffu, ne);
            const int k = bal ? __ffs(bal) - 1 : 32;
            if (k == 0) {
                hi = lo;
                break;
            }
            const uint32_t nlo = lo + (uint32_t)(k - 1) * step + 1u;
            if (k < 32) hi = min(hi, lo + (uint32_t)k * step);
            lo = nlo;
        }
        if (lo < hi) {
            const uint32_t pos = lo + (uint32_t)lane;
            const bool ne = pos >= hi || fam[pos] != f;
            const uint32_t bal = __ballot_sync(0xffffffffu, ne);
            lo = bal ? min(hi, lo + (uint32_t)(__ffs(bal) - 1)) : hi;
        }
        if (lane == 0) {
            const uint64_t c = (uint64_t)(lo - (B0 + (uint32_t)slast));
            c2 += c * c;
            if (c > 1) cl = __dadd_rn(cl, c <= FTAB ? clt[c] : __dmul_rn((double)c, log((double)c)));
        }
    }
    for (int o = 16; o > 0; o >>= 1) c2 += __shfl_xor_sync(0xffffffffu, c2, o);
    if ((threadIdx.x & 31) == 0 && c2) atomicAdd(&sc2, c2);
    sd[threadIdx.x] = cl;
    __syncthreads();
    for (int h = SCAN_THREADS / 2; h >= 1; h >>= 1) {
        if ((int)threadIdx.x < h) sd[threadIdx.x] = __dadd_rn(sd[threadIdx.x], sd[threadIdx.x + h]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        r.partCL[b] = sd[0];
        if (sc2) atomicAdd(&r.trace[i].sumC2, sc2);
    }
    if (PARTIAL) {
        // partial resampling: the new population's weights (1 after a
        // resampling, else the kept weight rescaled by 2^-wexp), then the
        // block's tree sums of w, w E, w E^2, w |M|, w M^2
        __syncthreads();
        const int32_t* Ec = r.E[i & 1];
        double v[5][SCAN_ITEMS];
#pragma unroll
        for (int e = 0; e < SCAN_ITEMS; ++e) {
            const uint32_t d = (uint32_t)(j0 + e);
            double w = 0.0, E = 0.0, M = 0.0;
            if (d < Ri) {
                w = r.w[d];
                if (mode == 0) {
                    w = st->resample ? 1.0 : scalbn(w, -st->wexp);
                    r.w[d] = w;
                }
                E = (double)Ec[d];
                M = (double)r.M[d];
            }
            v[0][e] = w;
            v[1][e] = __dmul_rn(w, E);
            v[2][e] = __dmul_rn(w, __dmul_rn(E, E));
            v[3][e] = __dmul_rn(w, fabs(M));
            v[4][e] = __dmul_rn(w, __dmul_rn(M, M));
        }
        for (int q = 0; q < 5; ++q) {
            const double root = tree_threads(tree_regs<SCAN_ITEMS>(v[q]), sd);
            if (threadIdx.x == 0) r.opart[5 * b + q] = root;
        }
    }
    // the run's last family block to finish closes the step: its ticket says every
    // other block's partials are written (each fenced them before its ticket)
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(&r.tick[1], 1u) == (uint32_t)r.nblk - 1u);
    __syncthreads();
    if (!last) return;
    if (threadIdx.x == 0) r.tick[1] = 0u;
    __threadfence();
    finish_run<PARTIAL>(p, r, st, mode, fa, fb, sd);
    if (CTL && mode == 0) {
        __syncthreads();  // the trace row and the step count are written
        control_after_step(p, r, st);
    }
}

// fixed-order sums of the run's per-block partials, close the step (one CTA of
// SCAN_THREADS threads; a, b, ws: shared arrays of SCAN_THREADS doubles)
template <bool PARTIAL>
__device__ void finish_run(const KParams& p, const RunDesc& r, DevState* st, int mode, double* a,
                           double* b, double* ws) {
    const int i = (mode == 0) ? st->step + 1 : st->step;
    const int nb_sv = (mode == 0) ? (int)((st->R_prev + SCAN_CHUNK - 1) / SCAN_CHUNK) : 0;
    const int nb_f = (int)((st->R_cur + SCAN_CHUNK - 1) / SCAN_CHUNK);
    double sa = 0.0, sb = 0.0;
    for (int k = threadIdx.x; k < nb_sv; k += blockDim.x) sa = __dadd_rn(sa, __ldcg(&r.partD[k]));
    for (int k = threadIdx.x; k < nb_f; k += blockDim.x) sb = __dadd_rn(sb, __ldcg(&r.partCL[k]));
    a[threadIdx.x] = sa;
    b[threadIdx.x] = sb;
    __syncthreads();
    for (int h = 128; h >= 1; h >>= 1) {
        if ((int)threadIdx.x < h) {
            a[threadIdx.x] = __dadd_rn(a[threadIdx.x], a[threadIdx.x + h]);
            b[threadIdx.x] = __dadd_rn(b[threadIdx.x], b[threadIdx.x + h]);
        }
        __syncthreads();
    }
    if (PARTIAL) {
        // partial resampling: tree over the blocks' weighted sums
        // (PARTIAL_MAX_BLOCKS leaves in all, zero past the run's blocks)
        const int nb = r.nblk;
        constexpr int LEAVES = PARTIAL_MAX_BLOCKS / 256;
        for (int q = 0; q < 5; ++q) {
            double x[LEAVES];
#pragma unroll
            for (int k = 0; k < LEAVES; ++k) {
                const int bb = LEAVES * threadIdx.x + k;
                x[k] = bb < nb ? __ldcg(&r.opart[5 * bb + q]) : 0.0;
            }
            const double root = tree_threads(tree_regs<LEAVES>(x), ws);
            if (threadIdx.x == 0) {
                TraceRow* tr = r.trace + i;
                double* dst[5] = {&tr->wsum, &tr->wE, &tr->wE2, &tr->wAM, &tr->wM2};
                *dst[q] = root;
            }
        }
    }
    if (threadIdx.x == 0) {
        TraceRow* tr = r.trace + i;
        tr->sv_sum = a[0];
        tr->c_ln_c = b[0];
        tr->R_i = st->R_cur;
        if (mode == 0) st->step = i;
        else tr->R_prev = st->R_cur;
    }
}

// --------------------------------------------------------------------------
// Single-pass scans (look-back).  A scan block takes a ticket for its logical
// index b within its run, computes its block sums, publishes them, and obtains
// the sum over blocks 0..b-1 from its predecessors' descriptors: the nearest
// inclusive prefix plus the aggregates after it.  Blocks only wait on blocks
// with earlier tickets, which are already running, so the waits end; each wait
// is bounded all the same (a run that exceeds it reports PA_ERR_TIMEOUT).
// --------------------------------------------------------------------------
constexpr uint32_t LB_SPIN_LIMIT = 1u << 22;

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* a) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint32_t* a, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Called by the 32 lanes of warp 0.  Publishes (a0, a1) of block b and returns in
// (p0, p1) the sums over blocks 0..b-1 (every lane); false if a wait gave up.
// publish = false (a test of the bounded waits) leaves block b's descriptor unset.
__device__ bool look_back(LBDesc* d, int b, unsigned long long a0, unsigned long long a1,
                          uint32_t ep, unsigned long long& p0, unsigned long long& p1,
                          bool publish = true) {
    const int lane = threadIdx.x & 31;
    const uint32_t FA = 2u * ep + 1u, FI = 2u * ep + 2u;
    if (lane == 0 && publish) {
        d[b].agg[0] = a0;
        d[b].agg[1] = a1;
        if (b == 0) {
            d[0].inc[0] = a0;
            d[0].inc[1] = a1;
        }
        st_release(&d[b].flag, b == 0 ? FI : FA);
    }
    p0 = p1 = 0ull;
    bool ok = true;
    if (b > 0) {
        int j0 = b - 1;
        uint32_t spins = 0;
        while (true) {
            const int j = j0 - lane;
            const uint32_t f = (j >= 0) ? ld_acquire(&d[j].flag) : FI;
            const uint32_t valid = __ballot_sync(0xffffffffu, f == FA || f == FI);
            const uint32_t incl = __ballot_sync(0xffffffffu, f == FI);
            // lanes 0..m-1 (blocks j0, j0-1, ...) have published
            const int m = (valid == 0xffffffffu) ? 32 : __ffs(~valid) - 1;
            const uint32_t usable = incl & (m == 32 ? 0xffffffffu : ((1u << m) - 1u));
            if (usable) {
                const int k = __ffs(usable) - 1;
                unsigned long long v0 = 0ull, v1 = 0ull;
                if (lane < k) {
                    v0 = __ldcg(&d[j].agg[0]);
                    v1 = __ldcg(&d[j].agg[1]);
                } else if (lane == k && j >= 0) {
                    v0 = __ldcg(&d[j].inc[0]);
                    v1 = __ldcg(&d[j].inc[1]);
                }
                p0 += warp_sum_u64(v0);
                p1 += warp_sum_u64(v1);
                break;
            }
            if (m == 32) {  // 32 aggregates, none inclusive: take them and look further
                p0 += warp_sum_u64(__ldcg(&d[j].agg[0]));
                p1 += warp_sum_u64(__ldcg(&d[j].agg[1]));
                j0 -= 32;
                continue;
            }
            if (++spins > LB_SPIN_LIMIT) {
                ok = false;
                break;
            }
            __nanosleep(64);
        }
        if (lane == 0 && ok && publish) {
            d[b].inc[0] = p0 + a0;
            d[b].inc[1] = p1 + a1;
            st_release(&d[b].flag, FI);
        }
    }
    return __all_sync(0xffffffffu, ok);
}

// the block's ticket: its logical index within the run
__device__ __forceinline__ int take_ticket(uint32_t* tick, int* sb) {
    if (threadIdx.x == 0) *sb = (int)atomicAdd(tick, 1u);
    __syncthreads();
    return *sb;
}

// Copy numbers' exclusive scan (look-back over lb2), the ancestor scatter and the
// block's sampling-variance partial; the last block sets the new population size
// (or the capacity error) and resets the tickets.
__device__ __forceinline__ void count_scan_scatter(const KParams& p, const RunDesc& r,
                                                   DevState* st, int b,
                                                   const uint32_t (&rc)[SCAN_ITEMS], uint64_t* sh,
                                                   double* sd, int* flag_sh,
                                                   const uint64_t (&fv)[SCAN_ITEMS], bool have_f) {
    const int i = st->step + 1;
    const int32_t* E = r.E[(i - 1) & 1];
    const int dN = p.d * r.N;
    const uint32_t Rprev = st->R_prev, lmin = st->lmin;
    const int j0 = b * SCAN_CHUNK + threadIdx.x * SCAN_ITEMS;
    uint64_t sum = 0;
#pragma unroll
    for (int e = 0; e < SCAN_ITEMS; ++e) sum += rc[e];
    uint64_t tot;
    const uint64_t ex = block_excl_scan(sum, sh, &tot);
    __shared__ unsigned long long pre;
    if (threadIdx.x < 32) {
        unsigned long long p0, p1;
        const bool ok = look_back(r.lb2, b, tot, 0ull, st->epoch, p0, p1);
        if (threadIdx.x == 0) {
            pre = p0;
            *flag_sh = ok;
        }
    }
    __syncthreads();
    if (!*flag_sh) {
        if (threadIdx.x == 0) atomicCAS(&st->status, S_OK, S_TIMEOUT);
        return;
    }
    uint64_t o = pre + ex;
    double sv = 0.0;
#pragma unroll
    for (int e = 0; e < SCAN_ITEMS; ++e) {
        const int j = j0 + e;
        if ((uint32_t)j >= Rprev) break;
        // the total is known only to the last block: slots past the capacity are
        // not written (the last block then stops the run with the capacity error)
        for (uint32_t c = 0; c < rc[e]; ++c)
            if (o + c < (uint64_t)r.Rcap) r.anc[o + c] = (uint32_t)j;
        o += rc[e];
        const double tau =
            scalbn((double)(have_f ? fv[e] : f_of(j, p, r, st, dN, E, lmin)), -FRAC_BITS);
        const double dl = __dsub_rn((double)rc[e], tau);
        sv = __dadd_rn(sv, __dmul_rn(dl, dl));
    }
    // fixed-order tree reduction of the block's sampling-variance terms
    sd[threadIdx.x] = sv;
    __syncthreads();
    for (int h = SCAN_THREADS / 2; h >= 1; h >>= 1) {
        if ((int)threadIdx.x < h) sd[threadIdx.x] = __dadd_rn(sd[threadIdx.x], sd[threadIdx.x + h]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        r.partD[b] = sd[0];
        if (b == r.nblk - 1) {
            const uint64_t Ri = pre + tot;
            // a population that outgrows its capacity, or dies out, stops the run
            if (st->kmax) st->status = S_KMAX;
            else if (Ri > (uint64_t)r.Rcap || Ri == 0) st->status = S_CAPACITY;
            else st->R_cur = (uint32_t)Ri;
            r.tick[0] = 0u;
        }
    }
}

// Expected copies f_j, their prefix C (and that of the fractional parts, G) by
// look-back over lb1, and the copy numbers of the rules that need no search.
// FULL (nearest, systematic, Poisson): then the count scan and the scatter too.
template <bool FULL>
__global__ void __launch_bounds__(SCAN_THREADS, 4) k_resample(KParams p) {
    const RunDesc& r = p.runs[p.blk2run[blockIdx.x]];
    DevState* st = r.st;
    if (st->status != S_OK) return;
    __shared__ uint64_t sh[33];
    __shared__ double sd[SCAN_THREADS];
    __shared__ int sb, okf;
    __shared__ unsigned long long pre[2];
    const int b = take_ticket(&r.tick[0], &sb);
    const int i = st->step + 1;
    const int32_t* E = r.E[(i - 1) & 1];
    const int dN = p.d * r.N;
    const uint32_t Rprev = st->R_prev, lmin = st->lmin;
    const uint64_t T = st->T;
    const int j0 = b * SCAN_CHUNK + threadIdx.x * SCAN_ITEMS;
    uint64_t f[SCAN_ITEMS];
    uint64_t sf = 0, sg = 0;
#pragma unroll
    for (int e = 0; e < SCAN_ITEMS; ++e) {
        const int j = j0 + e;
        f[e] = ((uint32_t)j < Rprev) ? f_of(j, p, r, st, dN, E, lmin) : 0ull;
        sf += f[e];
        sg += f[e] & ((1ull << FRAC_BITS) - 1);
    }
    uint64_t tf, tg;
    const uint64_t ef = block_excl_scan(sf, sh, &tf);
    const uint64_t eg = block_excl_scan(sg, sh, &tg);
    if (threadIdx.x < 32) {
        unsigned long long p0, p1;
        const bool ok = look_back(r.lb1, b, tf, tg, st->epoch, p0, p1, !(p.lb_hold && b == 0));
        if (threadIdx.x == 0) {
            pre[0] = p0;
            pre[1] = p1;
            okf = ok;
        }
    }
    __syncthreads();
    if (!okf) {
        if (threadIdx.x == 0) atomicCAS(&st->status, S_OK, S_TIMEOUT);
        return;
    }
    uint64_t cf = pre[0] + ef, cg = pre[1] + eg;
    const int method = p.method;
    uint32_t usys = 0;
    if (method == M_SYSTEMATIC)
        usys = philox(0u, DOM_RESAMPLE | (r.run << 8) | RULE_SYSTEMATIC, (uint32_t)i, 0u, p.k0, p.k1).x;
    bool kmax = false;
    uint32_t rc[SCAN_ITEMS];
    // systematic: labels below the running boundary, carried from item to item
    uint64_t below = method == M_SYSTEMATIC ? sys_below(cf, r.R, T, usys) : 0ull;
#pragma unroll 1
    for (int e = 0; e < SCAN_ITEMS; ++e) {
        const int j = j0 + e;
        rc[e] = 0u;
        if ((uint32_t)j >= Rprev) continue;
        cf += f[e];
        cg += f[e] & ((1ull << FRAC_BITS) - 1);
        uint32_t cnt = 0;
        if (method == M_NEAREST) {
            const uint4x x = philox((uint32_t)j, DOM_RESAMPLE | (r.run << 8) | RULE_NEAREST, (uint32_t)i, 0u,
                                    p.k0, p.k1);
            const uint64_t u40 = (((uint64_t)x.y << 32) | x.x) >> 24;
            cnt = (uint32_t)(f[e] >> FRAC_BITS) +
                  (u40 < (f[e] & ((1ull << FRAC_BITS) - 1)) ? 1u : 0u);
        } else if (method == M_SYSTEMATIC) {
            const uint64_t bn = sys_below(cf, r.R, T, usys);
            cnt = (uint32_t)(bn - below);
            below = bn;
        } else if (method == M_RESIDUAL) {
            r.C[j] = cf;
            r.G[j] = cg;
            cnt = (uint32_t)(f[e] >> FRAC_BITS);
        } else if (method == M_MULTINOMIAL) {
            r.C[j] = cf;
        } else {  // Poisson
            const double lam = scalbn((double)f[e], -FRAC_BITS);
            const uint32_t M = (uint32_t)(f[e] >> 44) + 1u;
            const double lc = __ddiv_rn(lam, (double)M);
            uint32_t total = 0;
            for (uint32_t m = 0; m < M; ++m) {
                const uint4x x = philox((uint32_t)j, DOM_RESAMPLE | (r.run << 8) | RULE_POISSON, (uint32_t)i, m,
                                        p.k0, p.k1);
                const double u = scalbn((double)((((uint64_t)x.y << 32) | x.x) >> 11), -53);
                double pr = exp_taylor(-lc);
                double Pc = pr;
                uint32_t k = 0;
                while (u >= Pc) {
                    k += 1;
                    if (k > POISSON_KMAX) {
                        kmax = true;
                        break;
                    }
                    pr = __ddiv_rn(__dmul_rn(pr, lc), (double)k);
                    Pc = __dadd_rn(Pc, pr);
                }
                total += k;
            }
            cnt = total;
        }
        rc[e] = cnt;
        r.counts[j] = cnt;
    }
    if (kmax) {  // promoted to the status word by the scan's last block
        atomicOr(&st->kmax, 1);
        __threadfence();
    }
    if (!FULL) {
        if (threadIdx.x == 0 && b == r.nblk - 1) r.tick[0] = 0u;
        return;
    }
    count_scan_scatter(p, r, st, b, rc, sh, sd, &okf, f, true);
}

// multinomial / residual: the copy numbers are complete after k_draws
__global__ void __launch_bounds__(SCAN_THREADS) k_cscan(KParams p) {
    const RunDesc& r = p.runs[p.blk2run[blockIdx.x]];
    DevState* st = r.st;
    if (st->status != S_OK) return;
    __shared__ uint64_t sh[33];
    __shared__ double sd[SCAN_THREADS];
    __shared__ int sb, okf;
    const int b = take_ticket(&r.tick[0], &sb);
    const uint32_t Rprev = st->R_prev;
    const int j0 = b * SCAN_CHUNK + threadIdx.x * SCAN_ITEMS;
    uint32_t rc[SCAN_ITEMS];
#pragma unroll
    for (int e = 0; e < SCAN_ITEMS; ++e) {
        const int j = j0 + e;
        rc[e] = ((uint32_t)j < Rprev) ? r.counts[j] : 0u;
    }
    const uint64_t nof[SCAN_ITEMS] = {};
    count_scan_scatter(p, r, st, b, rc, sh, sd, &okf, nof, false);
}

// --------------------------------------------------------------------------
cudaError_t launch_resample(const KParams& p, cudaStream_t s, int64_t* launches) {
    k_weights<<<p.M, 1024, 0, s>>>(p);
    int n = 1;
    if (p.alpha >= 0.0) {
        // partial resampling: the expected copies depend on per-replica weights, so
        // their total comes from a scan over the replicas
        k_pw_update<<<p.nblk_total, SCAN_THREADS, 0, s>>>(p);
        k_pw_final<<<p.M, 1024, 0, s>>>(p);
        k_fsum<<<p.nblk_total, SCAN_THREADS, 0, s>>>(p);
        k_fscan<<<p.M, 1024, 0, s>>>(p);
        k_counts<<<p.nblk_total, SCAN_THREADS, 0, s>>>(p);
        n += 5;
        if (p.method == M_MULTINOMIAL || p.method == M_RESIDUAL) {
            k_draws<<<p.nblk_total, SCAN_THREADS, 0, s>>>(p);
            ++n;
        }
        k_rsum<<<p.nblk_total, SCAN_THREADS, 0, s>>>(p);
        k_rscan<<<p.M, 1024, 0, s>>>(p);
        k_scatter<<<p.nblk_total, SCAN_THREADS, 0, s>>>(p);
        n += 3;
    } else if (p.method == M_MULTINOMIAL || p.method == M_RESIDUAL) {
        k_resample<false><<<p.nblk_total, SCAN_THREADS, 0, s>>>(p);
        k_draws<<<p.nblk_total, SCAN_THREADS, 0, s>>>(p);
        k_cscan<<<p.nblk_total, SCAN_THREADS, 0, s>>>(p);
        n += 3;
    } else {
        k_resample<true><<<p.nblk_total, SCAN_THREADS, 0, s>>>(p);
        n += 1;
    }
    if (launches) *launches += n;
    return cudaGetLastError();
}

cudaError_t launch_partial_init(const KParams& p, cudaStream_t s) {
    k_pw_init<<<dim3(64, (unsigned)p.M), 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_family_finish(const KParams& p, int mode, cudaStream_t s, int64_t* launches) {
    if (p.alpha >= 0.0) k_family<true, false><<<p.nblk_total, SCAN_THREADS, 0, s>>>(p, mode);
    else if (p.ctl) k_family<false, true><<<p.nblk_total, SCAN_THREADS, 0, s>>>(p, mode);
    else k_family<false, false><<<p.nblk_total, SCAN_THREADS, 0, s>>>(p, mode);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

}  // namespace pa
