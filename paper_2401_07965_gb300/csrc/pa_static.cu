// pa_static.cu -- pa_weights_static: the reweighting of one temperature step
// (energy-level histogram, Boltzmann weights, Q and the fixed-point expected
// copy numbers) for callers that cannot allocate device memory.
//
// Its scratch (the level histogram, the per-level weights and the pairwise-sum
// tree) lives in one file-scope __device__ array, so the call allocates
// nothing.  The arithmetic is the one of the context path's weights kernel,
// operation for operation, so both give the same bits.
#include <cmath>

#include "../../include/pa.h"
#include "pa_internal.cuh"

namespace {

constexpr int STATIC_MAX_LEVELS = 65536;  // d*N/2 + 1 <= 65536 energy levels
constexpr int STATIC_THREADS = 1024;

struct StaticScratch {
    uint32_t hist[STATIC_MAX_LEVELS];
    uint64_t flev[STATIC_MAX_LEVELS];
    double tree[STATIC_MAX_LEVELS];
    int32_t bad;  // set when an energy lies outside the lattice's range
};

// One copy per device that loads the library (about 1.3 MB), kept until exit.
static __device__ __align__(256) StaticScratch g_scratch;

__device__ __forceinline__ double pow_bin_s(double q, uint32_t k) {
    double r = 1.0, b = q;
    while (k) {
        if (k & 1u) r = __dmul_rn(r, b);
        b = __dmul_rn(b, b);
        k >>= 1;
    }
    return r;
}

__global__ void __launch_bounds__(STATIC_THREADS)
k_weights_static(StaticScratch* sc, const int32_t* __restrict__ E, uint32_t R_prev, uint32_t R,
                 int d, int N, int parity, double dbeta, double q, double* lnQ_out,
                 uint64_t* f_out) {
    __shared__ int smin[32], smax[32];
    const int nlev = d * N / 2 + 1;
    // the array keeps the previous call's contents: clear what must start at zero
    for (int l = threadIdx.x; l < nlev; l += blockDim.x) sc->hist[l] = 0u;
    if (threadIdx.x == 0) sc->bad = 0;
    __threadfence_block();
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < R_prev; j += blockDim.x) {
        // 2U = E + dN (U unsatisfied bonds) in 64 bits: no overflow for any int32 E.
        // A valid energy has 0 <= U <= dN and U = parity (mod 2).
        const long long twoU = (long long)E[j] + (long long)d * N;
        if (twoU < 0 || twoU > 2LL * d * N || (twoU & 1) || (((twoU >> 1) & 1) != parity)) {
            atomicExch(&sc->bad, 1);
            continue;
        }
        atomicAdd(&sc->hist[(int)(twoU >> 2)], 1u);
    }
    __threadfence_block();
    __syncthreads();
    volatile uint32_t* hist = sc->hist;
    int lo = 0x7fffffff, hi = -1;
    for (int l = threadIdx.x; l < nlev; l += blockDim.x)
        if (hist[l]) {
            lo = min(lo, l);
            hi = max(hi, l);
        }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        smin[warp] = lo;
        smax[warp] = hi;
    }
    __syncthreads();
    lo = 0x7fffffff;
    hi = -1;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        lo = min(lo, smin[w]);
        hi = max(hi, smax[w]);
    }
    volatile int32_t* bad = &sc->bad;
    if (hi < 0 || *bad) {  // no valid energy: report NaN, write no weights
        if (threadIdx.x == 0) *lnQ_out = NAN;
        return;
    }
    const int lmin = lo, K = hi - lo + 1;
    int P = 1;
    while (P < K) P <<= 1;
    volatile double* t = sc->tree;
    for (int k = threadIdx.x; k < P; k += blockDim.x)
        t[k] = (k < K) ? __dmul_rn((double)hist[lmin + k], pow_bin_s(q, (uint32_t)k)) : 0.0;
    __threadfence_block();
    __syncthreads();
    for (int h = P >> 1; h >= 1; h >>= 1) {
        for (int k = threadIdx.x; k < h; k += blockDim.x) t[k] = __dadd_rn(t[k], t[k + h]);
        __threadfence_block();
        __syncthreads();
    }
    const double S = t[0];
    const double Rd = (double)R;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        double a = __dmul_rn(Rd, pow_bin_s(q, (uint32_t)k));
        a = __ddiv_rn(a, S);
        a = scalbn(a, pa::FRAC_BITS);
        sc->flev[k] = (uint64_t)floor(a);
    }
    __threadfence_block();
    __syncthreads();
    volatile uint64_t* flev = sc->flev;
    for (uint32_t j = threadIdx.x; j < R_prev; j += blockDim.x)
        f_out[j] = flev[(((E[j] + d * N) >> 1) >> 1) - lmin];
    if (threadIdx.x == 0) {
        const int32_t Umin = 2 * lmin + parity;
        const int32_t Emin = 2 * Umin - d * N;
        *lnQ_out = __dsub_rn(__dsub_rn(log(S), log((double)R_prev)), __dmul_rn(dbeta, (double)Emin));
    }
}

}  // namespace

extern "C" pa_status pa_weights_static(const int32_t* E, uint32_t R_prev, uint32_t R, int32_t dim,
                                       int32_t L, int32_t parity, double dbeta, double* lnQ,
                                       uint64_t* f, void* cuda_stream) {
    if (!E || !lnQ || !f || R_prev == 0 || R == 0 || (parity & ~1)) return PA_ERR_ARG;
    if (dim < 2 || dim > 3 || L < 2 || (L & 1)) return PA_ERR_ARG;
    if (!(dbeta > 0.0) || !std::isfinite(dbeta)) return PA_ERR_ARG;
    long long N = 1;
    for (int a = 0; a < dim && N <= 32768; ++a) N *= L;
    if (N > 32768 || dim * N / 2 + 1 > STATIC_MAX_LEVELS) return PA_ERR_LIMIT;
    if (R > pa::MAX_POPULATION) return PA_ERR_LIMIT;  // 2^40 R must fit in 64 bits
    // The array's device address, looked up with the caller's device current on
    // every call: a cached pointer would outlive a reset of the device's context
    // (the module, and the array with it, is then loaded again elsewhere).  The
    // lookup is a host-side table query; only the first one on a device loads the
    // module.
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) return PA_ERR_CUDA;
    StaticScratch* sc = (StaticScratch*)ptr;
    const double q = std::exp(-(4.0 * dbeta));
    k_weights_static<<<1, STATIC_THREADS, 0, (cudaStream_t)cuda_stream>>>(
        sc, E, R_prev, R, dim, (int)N, parity, dbeta, q, lnQ, f);
    return cudaGetLastError() == cudaSuccess ? PA_OK : PA_ERR_CUDA;
}
