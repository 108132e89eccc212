// pa_sweep.cu -- initial population and the theta checkerboard Metropolis
// sweeps of Sec. 2 step 3, fused with the replica copy of step 2 and the
// measurements of step 4.
//
// Layout.  In HBM a replica is a row of Wp uint32 words (bit s&31 of word
// s>>5 = site s; Wp = ceil(N/32) rounded up to 4 so rows are 16-byte
// aligned).  A CTA owns 32 consecutive destination slots.  It reads the 32
// parent rows named by the ancestor array (the gather of the resampling
// step), transposes each 32x32 bit block with warp shuffles into one word per
// site whose bit r is replica r ("multi-spin" layout), and keeps the whole
// lattice of its 32 replicas in shared memory for all theta sweeps.  Neighbour
// sums and acceptance masks are then bit-parallel over the 32 replicas; only
// the uniform draw and its threshold compare are per (replica, site).
//
// Metropolis at beta_i: for site s with n unsatisfied bonds out of 2d,
// dE = 4 (d - n).  dE <= 0 flips; dE = 4k > 0 flips iff u < thr[k] with u a
// uint32 uniform whose bits are bit planes shared by the CTA's 32 replicas
// (see below).  Colour 0 (x+y+z even) is updated before colour 1 in every
// sweep; thread k of a half-sweep updates the k-th site of the colour.
//
// After the sweeps the CTA recomputes E = 2U - dN (U = unsatisfied bonds)
// and M, writes the 32 rows back, adds each replica to the energy-level
// histogram used by the next reweighting, and adds the population sums of
// E, E^2, |M|, M^2 and the accepted flips to the step's trace row.
#include "pa_sweep_common.cuh"

namespace pa {

// lattice geometry of the CTA's run
struct Geo {
    int L, N;
    uint32_t magicL, shiftL;
};

__device__ __forceinline__ int div_L(int s, const Geo& g) {
    return (int)(((uint64_t)(uint32_t)s * g.magicL) >> g.shiftL);
}

// ---------------------------------------------------------------------------
// Initial population (Sec. 2 step 1): every site an independent fair bit.
// Thread (j, g) writes words 4g..4g+3 of replica j from one INIT draw.
// ---------------------------------------------------------------------------
__global__ void k_init_spins(KParams p) {
    const RunDesc& r = p.runs[blockIdx.y];
    const uint32_t nq = (uint32_t)(r.Wp >> 2);
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t total = (uint64_t)r.R * nq;
    if (tid >= total) return;
    const uint32_t j = (uint32_t)(tid / nq);
    const uint32_t g = (uint32_t)(tid - (uint64_t)j * nq);
    uint4x x = philox(g, DOM_INIT, 0u, 32u * r.grp0 + j, p.k0, p.k1);
    uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int word = 4 * (int)g + m;
        const int lo = 32 * word;
        if (lo >= r.N) w[m] = 0u;
        else if (r.N - lo < 32) w[m] &= (1u << (r.N - lo)) - 1u;
    }
    uint4* dst = reinterpret_cast<uint4*>(r.spins[0] + (size_t)j * r.Wp) + g;
    *dst = make_uint4(w[0], w[1], w[2], w[3]);
    if (g == 0) r.fam[0][j] = j;
}

// the site of a half-sweep and its neighbours (periodic)
struct Nbr {
    int s, xp, xm, yp, ym, zp, zm;
};

// generic: the k-th site of the colour, any even L (x fastest)
template <int D>
__device__ __forceinline__ Nbr site_index(const Geo& geo, int k, int colour) {
    const int L = geo.L;
    const int LL = L * L;
    const int s0 = 2 * k;
    int q1 = div_L(s0, geo);
    int x = s0 - q1 * L, y, z = 0;
    if (D == 3) {
        z = div_L(q1, geo);
        y = q1 - z * L;
    } else {
        y = q1;
    }
    const int off = ((y + z) & 1) != colour;
    Nbr n;
    n.s = s0 + off;
    x += off;
    n.xp = (x == L - 1) ? n.s - (L - 1) : n.s + 1;
    n.xm = (x == 0) ? n.s + (L - 1) : n.s - 1;
    n.yp = (y == L - 1) ? n.s - (L - 1) * L : n.s + L;
    n.ym = (y == 0) ? n.s + (L - 1) * L : n.s - L;
    n.zp = n.zm = 0;
    if (D == 3) {
        n.zp = (z == L - 1) ? n.s - (L - 1) * LL : n.s + LL;
        n.zm = (z == 0) ? n.s + (L - 1) * LL : n.s - LL;
    }
    return n;
}

// classes of the site's replicas and the site-dependent Philox rounds 2 and 3
template <int D, bool EA>
__device__ __forceinline__ void site_prepare(SiteCmp<D>& c, const uint32_t* ms, const uint8_t* jb,
                                             const Nbr& n, uint32_t A2x, uint32_t B1k,
                                             uint32_t vmask) {
    const int s = n.s;
    const uint32_t w = ms[s];
    uint32_t P0 = w ^ ms[n.xp], P1 = w ^ ms[n.xm], P2 = w ^ ms[n.yp], P3 = w ^ ms[n.ym];
    uint32_t P4 = 0, P5 = 0;
    if (D == 3) {
        P4 = w ^ ms[n.zp];
        P5 = w ^ ms[n.zm];
    }
    if (EA) {
        const uint32_t js = jb[s];
        P0 ^= 0u - (js & 1u);
        P1 ^= 0u - (uint32_t)(jb[n.xm] & 1u);
        P2 ^= 0u - ((js >> 1) & 1u);
        P3 ^= 0u - (uint32_t)((jb[n.ym] >> 1) & 1u);
        if (D == 3) {
            P4 ^= 0u - ((js >> 2) & 1u);
            P5 ^= 0u - (uint32_t)((jb[n.zm] >> 2) & 1u);
        }
    }
    // classes of dE = 4 (d - n), n unsatisfied bonds
    uint32_t need;
    if (D == 2) {
        const uint32_t any = P0 | P1 | P2 | P3;
        const uint32_t two = (P0 & P1) | (P2 & P3) | ((P0 | P1) & (P2 | P3));
        need = ~two;                 // n <= 1: dE > 0
        c.cls[D - 1] = ~any;         // n == 0: dE = 8
        c.cls[0] = need & any;       // n == 1: dE = 4
    } else {
        const uint32_t sa = P0 ^ P1 ^ P2, ca = (P0 & P1) | (P2 & (P0 ^ P1));
        const uint32_t sb = P3 ^ P4 ^ P5, cb = (P3 & P4) | (P5 & (P3 ^ P4));
        const uint32_t n0 = sa ^ sb, kc = sa & sb;
        const uint32_t n1 = ca ^ cb ^ kc, n2 = (ca & cb) | (kc & (ca ^ cb));
        need = ~n2 & ~(n1 & n0);         // n <= 2
        c.cls[D - 1] = ~(n0 | n1 | n2);  // n == 0: dE = 12
        c.cls[1] = ~n2 & ~n1 & n0;       // n == 1: dE = 8
        c.cls[0] = ~n2 & n1 & ~n0;       // n == 2: dE = 4
    }
    c.s = s;
    c.need = need & vmask;
    c.und = c.need;
    c.lt = 0u;
    // rounds 2 and 3: the site-dependent halves
    const uint32_t A2 = A2x ^ (uint32_t)s;
    uint32_t h1b, l1b;
    mulhilo(PHILOX_M1, A2, h1b, l1b);
    c.B1 = l1b;
    mulhilo(PHILOX_M0, h1b ^ B1k, c.h0c, c.l0c);
}

template <int D>
__device__ __forceinline__ uint32_t site_flip(const SiteCmp<D>& c, uint32_t* ms, uint32_t vmask) {
    const uint32_t f = (~c.need | c.lt) & vmask;
    ms[c.s] ^= f;
    return (uint32_t)__popc(f);
}

// queue of sites still undecided after the first two plane blocks (one per
// CTA, struct of arrays in dynamic shared memory)
template <int D>
struct SiteQueue {
    uint32_t* w;  // (7 + D) arrays of cap words
    int cap;
    __device__ void put(int e, const SiteCmp<D>& c) {
        w[0 * cap + e] = (uint32_t)c.s;
        w[1 * cap + e] = c.need;
        w[2 * cap + e] = c.und;
        w[3 * cap + e] = c.lt;
        w[4 * cap + e] = c.B1;
        w[5 * cap + e] = c.h0c;
        w[6 * cap + e] = c.l0c;
#pragma unroll
        for (int a = 0; a < D; ++a) w[(7 + a) * cap + e] = c.cls[a];
    }
    __device__ void get(int e, SiteCmp<D>& c) const {
        c.s = (int)w[0 * cap + e];
        c.need = w[1 * cap + e];
        c.und = w[2 * cap + e];
        c.lt = w[3 * cap + e];
        c.B1 = w[4 * cap + e];
        c.h0c = w[5 * cap + e];
        c.l0c = w[6 * cap + e];
#pragma unroll
        for (int a = 0; a < D; ++a) c.cls[a] = w[(7 + a) * cap + e];
    }
};

// sites queued per half-sweep.  A site is still undecided after two plane
// blocks (8 bits of u) with probability 1 - (1 - 2^-8)^32 = 11.8% at most, so
// 5/32 of the sites of a colour plus 32 leaves the queue full only in rare
// fluctuations (those sites finish inline); the small queue lets seven CTAs
// of a 64 x 64 lattice share an SM.
__host__ __device__ __forceinline__ int queue_capacity(int N) {
    return (((N / 2) * 5 / 32 + 32) + 31) / 32 * 32;
}

// ---------------------------------------------------------------------------
// mode 0: one temperature step's copy + sweeps + measurement (slots of the
//         new population, parents from the ancestor array).
// mode 1: measurement of the current population only (init / restore).
// ---------------------------------------------------------------------------
template <int D, bool EA, int NT>
__global__ void __launch_bounds__(NT) k_group(KParams p, int mode) {
    extern __shared__ __align__(16) uint32_t smem[];
    // the CTA's run and its replica group within the run; the flattened CTA
    // index is the global replica group of the sweep draws
    const RunDesc& r = p.runs[p.grp2run[blockIdx.x]];
    const Geo geo = {r.L, r.N, r.magicL, r.shiftL};
    uint32_t* ms = smem;
    uint8_t* jb = reinterpret_cast<uint8_t*>(smem + r.N);
    const int qcap = (p.qcap_limit >= 0 && p.qcap_limit < queue_capacity(r.N))
                         ? p.qcap_limit : queue_capacity(r.N);
    uint32_t* qwords = smem + r.N + (EA ? (r.N + 15) / 16 * 4 : 0);
    __shared__ int32_t sU[32];
    __shared__ int32_t sNup[32];
    __shared__ unsigned long long sAcc;
    __shared__ PlaneTab tabs[2][8];
    __shared__ int qn[2];

    const DevState* st = r.st;
    if (st->status != S_OK) return;
    const int i = (mode == 0) ? st->step + 1 : st->step;
    const uint32_t R = st->R_cur;
    const uint32_t base = (blockIdx.x - r.grp0) * 32u;
    if (base >= R) return;
    const uint32_t nval = min(32u, R - base);
    const uint32_t vmask = (nval == 32u) ? 0xFFFFFFFFu : ((1u << nval) - 1u);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int N = r.N, W = r.W, Wp = r.Wp;
    const uint32_t* src = r.spins[mode == 0 ? ((i - 1) & 1) : (i & 1)];
    uint32_t* dst = r.spins[i & 1];

    if (threadIdx.x < 32) {
        sU[threadIdx.x] = 0;
        sNup[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) sAcc = 0ull;

    const bool valid = (uint32_t)lane < nval;
    uint32_t my_src = base + lane;
    if (mode == 0 && valid) my_src = r.anc[base + lane];
    if (mode == 0 && warp == 0 && valid) r.fam[i & 1][base + lane] = r.fam[(i - 1) & 1][my_src];

    // gather the 32 parent rows and transpose them into the multi-spin layout
    for (int c4 = warp; 4 * c4 < W; c4 += nwarp) {
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (valid) v = reinterpret_cast<const uint4*>(src + (size_t)my_src * Wp)[c4];
        const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int b = 4 * c4 + k;
            if (b < W) {
                const uint32_t t = transpose32(w4[k], lane);
                const int s = 32 * b + lane;
                if (s < N) ms[s] = t;
            }
        }
    }
    if (EA)
        for (int s = threadIdx.x; s < N; s += blockDim.x) jb[s] = r.jbits[s];
    __syncthreads();

    uint32_t acc = 0;
    if (mode == 0) {
        const uint32_t theta = r.stheta[i - 1];
        uint32_t thr[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) thr[k] = r.sthr[4 * (i - 1) + k];
        const uint32_t grp = blockIdx.x;         // global replica group
        uint32_t h0a, l0a, h1a, l1a;
        mulhilo(PHILOX_M0, grp, h0a, l0a);
        mulhilo(PHILOX_M1, (uint32_t)i, h1a, l1a);
        const uint32_t A2x = h0a ^ p.rk1[0];     // round-1 lane 2 without the site
        const uint32_t B1k = l1a ^ p.rk0[1];     // round-2 lane 0 key part
        const int nhalf = N / 2;
        // row-wise walk of the sites (2D, L a power of two dividing the CTA size)
        const int lgL = __ffs(geo.L) - 1;
        const int rows2 = (D == 2 && (geo.L & (geo.L - 1)) == 0 && NT % geo.L == 0)
                              ? 2 * NT / geo.L : 0;
        const uint32_t nh = 2u * theta;          // half-sweeps
        SiteQueue<D> queue;
        queue.w = qwords;
        queue.cap = qcap;
        if (nh > 0 && threadIdx.x < 8)
            build_plane_tab(tabs[0], threadIdx.x, p, grp, (uint32_t)i, 0u, 0, thr);
        if (threadIdx.x == 0) {
            qn[0] = 0;
            qn[1] = 0;
        }
        __syncthreads();
        for (uint32_t h = 0; h < nh; ++h) {
            const int colour = (int)(h & 1u);
            // the table of the next half-sweep goes to the other buffer
            if (h + 1 < nh && threadIdx.x < 8)
                build_plane_tab(tabs[(h + 1) & 1u], threadIdx.x, p, grp, (uint32_t)i,
                                (h + 1) >> 1, (int)((h + 1) & 1u), thr);
            if (threadIdx.x == 0) qn[(h + 1) & 1u] = 0;
            const PlaneTab* tab = tabs[h & 1u];
            // pass 1: every site runs plane blocks 0 and 1 (decides ~88% of sites)
            auto pass1 = [&](const Nbr& n) {
                SiteCmp<D> c;
                site_prepare<D, EA>(c, ms, jb, n, A2x, B1k, vmask);
                if (c.need) {
                    uint32_t W[4], V[4];
                    block_draw2<D>(c, tab[0], tab[1], p, W, V);
                    compare8<D>(c, tab[0], tab[1], W, V);
                }
                if (c.und) {
                    const int e = atomicAdd(&qn[h & 1u], 1);
                    if (e < qcap) {
                        queue.put(e, c);
                        return;
                    }
                    for (int g = 2; g < 8 && c.und; ++g) plane_block<D>(c, tab[g], p);
                }
                acc += site_flip<D>(c, ms, vmask);
            };
            if (rows2) {
                // 2D, L = 2^lgL, 2 NT / L rows per pass (even): the thread's x is
                // the same in every row it visits, and the row wrap is a mask
                const int L = geo.L;
                const int x = 2 * (int)(threadIdx.x & ((L >> 1) - 1)) +
                              (((int)(threadIdx.x >> (lgL - 1)) + colour) & 1);
                const int dxp = (x == L - 1) ? -(L - 1) : 1;
                const int dxm = (x == 0) ? (L - 1) : -1;
                for (int y = (int)(threadIdx.x >> (lgL - 1)); y < L; y += rows2) {
                    Nbr n;
                    n.s = (y << lgL) + x;
                    n.xp = n.s + dxp;
                    n.xm = n.s + dxm;
                    n.yp = (n.s + L) & (N - 1);
                    n.ym = (n.s - L) & (N - 1);
                    n.zp = n.zm = 0;
                    pass1(n);
                }
            } else {
                for (int k = threadIdx.x; k < nhalf; k += blockDim.x)
                    pass1(site_index<D>(geo, k, colour));
            }
            __syncthreads();
            // pass 2: the undecided sites, one per thread, from plane block 2 on
            const int nq = min(qn[h & 1u], qcap);
            for (int e = threadIdx.x; e < nq; e += blockDim.x) {
                SiteCmp<D> c;
                queue.get(e, c);
#pragma unroll 1
                for (int g = 2; g < 8; ++g) {
                    plane_block<D>(c, tab[g], p);
                    if (!c.und) break;
                }
                acc += site_flip<D>(c, ms, vmask);
            }
            __syncthreads();
        }
    }

    // measurement: unsatisfied bonds U and up-count per replica, write back
    int32_t U = 0, nup = 0;
    for (int c4 = warp; 4 * c4 < Wp; c4 += nwarp) {
        uint32_t out[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int b = 4 * c4 + k;
            out[k] = 0u;
            if (b < W) {  // warp-uniform
                const int s = 32 * b + lane;
                const bool in = s < N;
                const uint32_t w = in ? ms[s] : 0u;
                const uint32_t tw = transpose32(w, lane);
                out[k] = tw;
                nup += __popc(tw);
                // unsatisfied-bond planes of the + bonds of s (0 past the last site)
                uint32_t P0 = 0u, P1 = 0u, P2 = 0u;
                if (in) {
                    int q1 = div_L(s, geo);
                    int x = s - q1 * geo.L, y, z = 0;
                    if (D == 3) {
                        z = div_L(q1, geo);
                        y = q1 - z * geo.L;
                    } else {
                        y = q1;
                    }
                    const int L = geo.L;
                    const int xp = (x == L - 1) ? s - (L - 1) : s + 1;
                    const int yp = (y == L - 1) ? s - (L - 1) * L : s + L;
                    const uint32_t js = EA ? (uint32_t)jb[s] : 0u;
                    P0 = w ^ ms[xp] ^ (0u - (js & 1u));
                    P1 = w ^ ms[yp] ^ (0u - ((js >> 1) & 1u));
                    if (D == 3) {
                        const int zp = (z == L - 1) ? s - (L - 1) * L * L : s + L * L;
                        P2 = w ^ ms[zp] ^ (0u - ((js >> 2) & 1u));
                    }
                }
                // all lanes take part in the transposes
                U += __popc(transpose32(P0, lane));
                U += __popc(transpose32(P1, lane));
                if (D == 3) U += __popc(transpose32(P2, lane));
            }
        }
        if (valid)
            reinterpret_cast<uint4*>(dst + (size_t)(base + lane) * Wp)[c4] =
                make_uint4(out[0], out[1], out[2], out[3]);
    }
    atomicAdd(&sU[lane], U);
    atomicAdd(&sNup[lane], nup);
    // accepted flips of the CTA
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0 && acc) atomicAdd(&sAcc, (unsigned long long)acc);
    __syncthreads();

    if (warp == 0) {
        long long e = 0, e2 = 0, am = 0, m2 = 0;
        int lvmin = 0x7FFFFFFF, lvmax = -1;  // the warp's histogram levels
        if (valid) {
            const int32_t Uv = sU[lane];
            const int32_t E = 2 * Uv - D * N;
            const int32_t M = N - 2 * sNup[lane];
            r.E[i & 1][base + lane] = E;
            r.M[base + lane] = M;
            atomicAdd(&r.hist[Uv >> 1], 1u);
            lvmin = lvmax = Uv >> 1;
            e = E;
            e2 = (long long)E * E;
            am = M < 0 ? -M : M;
            m2 = (long long)M * M;
        }
        for (int o = 16; o > 0; o >>= 1) {
            e += __shfl_xor_sync(0xffffffffu, e, o);
            e2 += __shfl_xor_sync(0xffffffffu, e2, o);
            am += __shfl_xor_sync(0xffffffffu, am, o);
            m2 += __shfl_xor_sync(0xffffffffu, m2, o);
        }
        lvmin = __reduce_min_sync(0xffffffffu, lvmin);
        lvmax = __reduce_max_sync(0xffffffffu, lvmax);
        if (lane == 0 && lvmax >= 0) {  // the occupied level range for the reweighting
            atomicMin(&r.st->hlo, lvmin);
            atomicMax(&r.st->hhi, lvmax);
        }
        if (lane == 0) {
            TraceRow* tr = r.trace + i;
            atomicAdd(&tr->sumE, (unsigned long long)e);
            atomicAdd(&tr->sumE2, (unsigned long long)e2);
            atomicAdd(&tr->sumAbsM, (unsigned long long)am);
            atomicAdd(&tr->sumM2, (unsigned long long)m2);
            if (sAcc) atomicAdd(&tr->accepts, sAcc);
        }
    }
}

int sweep_threads(int N) {
    const int sites = N / 2;  // per colour
    int t = 64;
    while (t * 4 < sites && t < 256) t <<= 1;
    return t;
}

bool sweep_threads_supported(int t) {
    return t == 64 || t == 128 || t == 256 || t == 384 || t == 512;
}

static size_t group_smem(const KParams& p) {
    const size_t words_per_entry = 7 + (size_t)p.d;
    return (size_t)p.maxN * 4 + (p.ea ? (size_t)((p.maxN + 15) / 16) * 16 : 0) +
           words_per_entry * 4 * (size_t)queue_capacity(p.maxN);
}

template <int D, bool EA, int NT>
static cudaError_t prepare_nt() {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_group<D, EA, NT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             200 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    return cudaSuccess;
}

template <int D, bool EA, int NT>
static cudaError_t launch_group_nt(const KParams& p, int mode, cudaStream_t s) {
    cudaError_t e = prepare_nt<D, EA, NT>();
    if (e != cudaSuccess) return e;
    k_group<D, EA, NT><<<p.ngrp_total, NT, group_smem(p), s>>>(p, mode);
    return cudaGetLastError();
}

template <int D, bool EA>
static cudaError_t launch_group_t(const KParams& p, int mode, int threads, cudaStream_t s) {
    switch (threads) {
        case 64: return launch_group_nt<D, EA, 64>(p, mode, s);
        case 128: return launch_group_nt<D, EA, 128>(p, mode, s);
        case 384: return launch_group_nt<D, EA, 384>(p, mode, s);
        case 512: return launch_group_nt<D, EA, 512>(p, mode, s);
        default: return launch_group_nt<D, EA, 256>(p, mode, s);
    }
}

static cudaError_t launch_group(const KParams& p, int mode, int threads, cudaStream_t s) {
    if (p.d == 2) return p.ea ? launch_group_t<2, true>(p, mode, threads, s)
                              : launch_group_t<2, false>(p, mode, threads, s);
    return p.ea ? launch_group_t<3, true>(p, mode, threads, s)
                : launch_group_t<3, false>(p, mode, threads, s);
}

template <int D, bool EA>
static cudaError_t prepare_t(int threads) {
    switch (threads) {
        case 64: return prepare_nt<D, EA, 64>();
        case 128: return prepare_nt<D, EA, 128>();
        case 384: return prepare_nt<D, EA, 384>();
        case 512: return prepare_nt<D, EA, 512>();
        default: return prepare_nt<D, EA, 256>();
    }
}

// one-time function attributes, outside any stream capture
cudaError_t prepare_sweep(const KParams& p, int threads) {
    bool done = false;
    cudaError_t e = launch_sweep2d(p, threads, nullptr, true, &done);
    if (e != cudaSuccess) return e;
    for (int k = 0; k < p.n3 && e == cudaSuccess; ++k)
        e = launch_sweep3d(p, p.L3[k], p.c3map[k], p.n3cta[k], nullptr, true);
    if (e != cudaSuccess) return e;
    if (p.d == 2) return p.ea ? prepare_t<2, true>(threads) : prepare_t<2, false>(threads);
    return p.ea ? prepare_t<3, true>(threads) : prepare_t<3, false>(threads);
}

cudaError_t launch_init_spins(const KParams& p, const RunDesc* host_runs, cudaStream_t s) {
    uint64_t most = 0;
    for (int m = 0; m < p.M; ++m) {
        const uint64_t t = (uint64_t)host_runs[m].R * (uint64_t)(host_runs[m].Wp / 4);
        if (t > most) most = t;
    }
    const dim3 grid((unsigned)((most + 255) / 256), (unsigned)p.M);
    k_init_spins<<<grid, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_measure(const KParams& p, int threads, cudaStream_t s) {
    return launch_group(p, 1, threads, s);
}

cudaError_t launch_sweep(const KParams& p, int threads, cudaStream_t s) {
    if (p.n3 > 0) {  // 3D runs of sides 4..16: one launch per side
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < p.n3 && e == cudaSuccess; ++k)
            e = launch_sweep3d(p, p.L3[k], p.c3map[k], p.n3cta[k], s, false);
        return e;
    }
    bool done = false;
    const cudaError_t e = launch_sweep2d(p, threads, s, false, &done);
    if (e != cudaSuccess || done) return e;
    return launch_group(p, 0, threads, s);
}

}  // namespace pa
