// pa_sweep2d.cu -- the temperature step's replica copy, theta checkerboard
// Metropolis sweeps and measurement (Sec. 2 steps 2-4) for two-dimensional
// runs whose side L is a power of two, 16 <= L <= 128: the work of k_group's
// sweep mode, with a lattice layout and a site walk chosen for this case.  The
// random numbers, the order of the updates within a half-sweep (any: sites of
// one colour do not interact) and therefore every result are the same.
//
// Layout.  The CTA's 32 replicas in the multi-spin form (one word per site,
// bit r = replica r) on a halo-padded lattice in shared memory: cell (x, y),
// -1 <= x, y <= L, is word (y+1)(L+2) + x+1, and the halo cells hold copies of
// the opposite boundary, so the four neighbours of every site are at fixed
// offsets +-1 and +-(L+2) with no periodic wrap.  After each half-sweep the
// threads that own boundary sites refresh their copies.  For +-J couplings each
// cell also has a 16-byte record of the bond signs of its four bonds as
// all-ones / all-zeros masks.
//
// Walk.  Thread t keeps one column slot per colour and visits the rows
// y0, y0 + RP, ... (RP = 2 NT / L rows per pass); L and NT are template
// parameters, so every lattice offset of the walk is a compile-time constant
// and the Philox site counter s = x + L y advances by OR-ing a constant.  Rows
// are paired within a warp (half-warp per row) where a row has 16 or more sites
// of a colour, which keeps the warp's shared-memory accesses on distinct banks.
//
// Undecided sites.  After the two unconditional plane blocks (eight bits of the
// uniforms) a site whose replicas are not all decided goes to its warp's queue
// (ballot + prefix count, no atomics); the warp finishes its queue after its
// share of the colour, one site per lane, from plane block 2 on (earlier, should
// the queue run short of room).  The site body has no branches: a decided site
// stores its flips, an undecided one stores no flip and its queue entry, and
// lanes with nothing to queue write a scratch slot of their own.
#include "pa_sweep_common.cuh"

namespace pa {
namespace {

// Philox table of one plane block for the half-sweep: the site-independent
// round-3 values and the threshold bits (0 or 1) of its four planes for the two
// energy classes of d = 2 (dE = 4: B0, dE = 8: B1), class-major for 128-bit
// loads.  The classes' replica masks are disjoint, so the per-replica threshold
// bit word of a plane, (c4 & -B0) | (c8 & -B1), equals the integer c4 B0 + c8 B1:
// two multiply-adds on the multiply pipe instead of logic operations on the
// (busier) integer ALU pipe.
struct Tab2 {
    uint32_t c0k, c1, c2k, pad;
    uint32_t B0[4];
    uint32_t B1[4];
};

__device__ __forceinline__ void build_tab2(Tab2* tab, int g, const KParams& p, uint32_t grp,
                                           uint32_t step, uint32_t t, int colour,
                                           uint32_t thr1, uint32_t thr2) {
    uint32_t h0a, l0a, h1a, l1a, h0b, l0b, h1c, l1c;
    mulhilo(PHILOX_M0, grp, h0a, l0a);
    mulhilo(PHILOX_M1, step, h1a, l1a);
    const uint32_t c1v = DOM_SWEEP | (t << 4) | ((uint32_t)colour << 3) | (uint32_t)g;
    const uint32_t A0 = h1a ^ c1v ^ p.rk0[0];
    mulhilo(PHILOX_M0, A0, h0b, l0b);
    const uint32_t B2 = h0b ^ l0a ^ p.rk1[1];
    mulhilo(PHILOX_M1, B2, h1c, l1c);
    Tab2 e;
    e.c0k = h1c ^ p.rk0[2];
    e.c1 = l1c;
    e.c2k = l0b ^ p.rk1[2];
    e.pad = 0u;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        e.B0[m] = (thr1 >> (31 - (4 * g + m))) & 1u;
        e.B1[m] = (thr2 >> (31 - (4 * g + m))) & 1u;
    }
    tab[g] = e;
}

// rounds 4-10 of two plane blocks, interleaved
__device__ __forceinline__ void draw2(const Tab2& e, const Tab2& f, uint32_t B1, uint32_t h0c,
                                      uint32_t l0c, const KParams& p, uint32_t (&W)[4],
                                      uint32_t (&V)[4]) {
    uint32_t x0 = e.c0k ^ B1, x1 = e.c1, x2 = h0c ^ e.c2k, x3 = l0c;
    uint32_t y0 = f.c0k ^ B1, y1 = f.c1, y2 = h0c ^ f.c2k, y3 = l0c;
#pragma unroll
    for (int rr = 3; rr < 10; ++rr) {
        uint32_t hi0, lo0, hi1, lo1, gi0, go0, gi1, go1;
        mulhilo(PHILOX_M0, x0, hi0, lo0);
        mulhilo(PHILOX_M1, x2, hi1, lo1);
        mulhilo(PHILOX_M0, y0, gi0, go0);
        mulhilo(PHILOX_M1, y2, gi1, go1);
        x0 = hi1 ^ x1 ^ p.rk0[rr];
        x1 = lo1;
        x2 = hi0 ^ x3 ^ p.rk1[rr];
        x3 = lo0;
        y0 = gi1 ^ y1 ^ p.rk0[rr];
        y1 = go1;
        y2 = gi0 ^ y3 ^ p.rk1[rr];
        y3 = go0;
    }
    W[0] = x0; W[1] = x1; W[2] = x2; W[3] = x3;
    V[0] = y0; V[1] = y1; V[2] = y2; V[3] = y3;
}

// rounds 4-10 of one plane block
__device__ __forceinline__ void draw1(const Tab2& e, uint32_t B1, uint32_t h0c, uint32_t l0c,
                                      const KParams& p, uint32_t (&W)[4]) {
    uint32_t x0 = e.c0k ^ B1, x1 = e.c1, x2 = h0c ^ e.c2k, x3 = l0c;
#pragma unroll
    for (int rr = 3; rr < 10; ++rr) {
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo(PHILOX_M0, x0, hi0, lo0);
        mulhilo(PHILOX_M1, x2, hi1, lo1);
        x0 = hi1 ^ x1 ^ p.rk0[rr];
        x1 = lo1;
        x2 = hi0 ^ x3 ^ p.rk1[rr];
        x3 = lo0;
    }
    W[0] = x0; W[1] = x1; W[2] = x2; W[3] = x3;
}

// Site-dependent Philox rounds 2 and 3 (A2s = round-1 lane 2 with the site)
__device__ __forceinline__ void site_rounds(uint32_t A2s, uint32_t B1k, uint32_t& B1,
                                            uint32_t& h0c, uint32_t& l0c) {
    uint32_t h1b, l1b;
    mulhilo(PHILOX_M1, A2s, h1b, l1b);
    B1 = l1b;
    mulhilo(PHILOX_M0, h1b ^ B1k, h0c, l0c);
}

// energy classes of a site from the XORs with its four neighbours (bond signs
// folded in): need = dE > 0 (at most one unsatisfied bond) among the valid
// replicas, c4 = dE = 4 (one), c8 = dE = 8 (none)
__device__ __forceinline__ void classes(uint32_t P0, uint32_t P1, uint32_t P2, uint32_t P3,
                                        uint32_t vmask, uint32_t& need, uint32_t& c4,
                                        uint32_t& c8) {
    const uint32_t any = P0 | P1 | P2 | P3;
    const uint32_t two = (P0 & P1) | (P2 & P3) | ((P0 | P1) & (P2 | P3));
    need = ~two & vmask;
    c8 = ~any;
    c4 = need & any;
}

// the classes of a ferromagnet site from its word and its four neighbours (the same
// values as classes() on P_k = w ^ n_k): each pair term takes the XORs with w inside
// one three-input logic operation, which saves the four separate XORs
__device__ __forceinline__ void classes_w(uint32_t w, uint32_t n0, uint32_t n1, uint32_t n2,
                                          uint32_t n3, uint32_t vmask, uint32_t& need,
                                          uint32_t& c4, uint32_t& c8) {
    const uint32_t a = lop3<0x7E>(w, n0, n1), b = lop3<0x7E>(w, n2, n3);  // (w^x)|(w^y)
    const uint32_t pa = lop3<0x18>(w, n0, n1), pb = lop3<0x18>(w, n2, n3);  // (w^x)&(w^y)
    const uint32_t any = a | b;
    const uint32_t two = pa | pb | (a & b);
    need = ~two & vmask;
    c8 = ~any;
    c4 = need & any;
}

// the top eight planes at once (blocks 0 and 1): b = [u8 < t8] by the borrow of
// u - t from the least significant plane up, eq = [u8 == t8], per replica with
// t the threshold of its class.  ZC: the number of classes, from dE = 8 down,
// whose thresholds have eight zero top bits in this step (their terms of t are
// zero and left out); with both, t = 0: b = 0 and eq = [u8 == 0].
template <int ZC>
__device__ __forceinline__ void cmp8(uint32_t c4, uint32_t c8, const Tab2& e, const Tab2& f,
                                     const uint32_t (&W)[4], const uint32_t (&V)[4], uint32_t& b,
                                     uint32_t& eq) {
    if constexpr (ZC >= 2) {
        b = 0u;
        eq = lop3<0x01>(lop3<0xFE>(V[0], V[1], V[2]), lop3<0xFE>(V[3], W[0], W[1]),
                        W[2] | W[3]);  // ~(a | b | c)
        return;
    }
    b = 0u;
    eq = 0xFFFFFFFFu;
#pragma unroll
    for (int m = 3; m >= 0; --m) {
        const uint32_t t = ZC == 0 ? c4 * f.B0[m] + c8 * f.B1[m] : c4 * f.B0[m];
        b = lop3<0x8E>(V[m], t, b);    // (~V & t) | (~(V ^ t) & b)
        eq = lop3<0x82>(V[m], t, eq);  // eq & ~(V ^ t)
    }
#pragma unroll
    for (int m = 3; m >= 0; --m) {
        const uint32_t t = ZC == 0 ? c4 * e.B0[m] + c8 * e.B1[m] : c4 * e.B0[m];
        b = lop3<0x8E>(W[m], t, b);
        eq = lop3<0x82>(W[m], t, eq);
    }
}

// ZC of a step from its thresholds of dE = 4 and 8 (top eight bits)
__device__ __forceinline__ int zero_classes2(uint32_t thr4, uint32_t thr8) {
    return (thr8 >> 24) != 0u ? 0 : ((thr4 >> 24) != 0u ? 1 : 2);
}

template <int V>
struct IC {
    static constexpr int value = V;
};

// four more planes from the top: replicas leave at the first plane where u and
// thr differ
__device__ __forceinline__ void cmp4(uint32_t c4, uint32_t c8, const Tab2& e,
                                     const uint32_t (&W)[4], uint32_t& und, uint32_t& lt) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const uint32_t t = c4 * e.B0[m] + c8 * e.B1[m];
        lt |= lop3<0x40>(und, t, W[m]);   // und & t & ~W
        und = lop3<0x82>(W[m], t, und);   // und & ~(W ^ t)
    }
}

// planes 8, 9, ... of a site until every replica is decided
__device__ __forceinline__ void finish(uint32_t c4, uint32_t c8, const Tab2* tab, uint32_t B1,
                                       uint32_t h0c, uint32_t l0c, const KParams& p,
                                       uint32_t& und, uint32_t& lt) {
#pragma unroll 1
    for (int g = 2; g < 8 && und; ++g) {
        uint32_t W[4];
        draw1(tab[g], B1, h0c, l0c, p, W);
        cmp4(c4, c8, tab[g], W, und, lt);
    }
}

template <int L>
struct Geo2 {
    static constexpr int P = L + 2;
    __device__ static constexpr int cell(int x, int y) { return (y + 1) * P + x + 1; }
};

// the per-half-sweep state a site body needs
struct Half {
    const Tab2* tab;
    uint32_t A2s0;   // round-1 lane 2 with the thread's first site folded in
    uint32_t B1k;
    uint32_t vmask;
};

// Site k of the thread's walk in pass 1.  la: the site's cell, ja: its bond
// record, s_hi: the high part of its site counter.  A decided site flips now;
// an undecided one is queued as (round-1 lane 2 with the site, und, lt) at slot
// wq + (its rank among the warp's undecided sites); the other lanes write their
// scratch slot qscratch + lane.
template <int L, bool EA, int ZC>
__device__ __forceinline__ void site_pass1(uint32_t* la, const uint4* ja, uint32_t s_hi,
                                           const Half& hs, const KParams& p, uint4* queue,
                                           int qscratch, uint32_t lml, int lane, int& wq,
                                           uint32_t& acc) {
    constexpr int P = L + 2;
    const uint32_t w = la[0];
    uint32_t need, c4, c8;
    if (EA) {
        uint32_t P0 = w ^ la[1], P1 = w ^ la[-1], P2 = w ^ la[P], P3 = w ^ la[-P];
        const uint4 J = *ja;
        P0 ^= J.x;
        P1 ^= J.y;
        P2 ^= J.z;
        P3 ^= J.w;
        classes(P0, P1, P2, P3, hs.vmask, need, c4, c8);
    } else {
        classes_w(w, la[1], la[-1], la[P], la[-P], hs.vmask, need, c4, c8);
    }
    const uint32_t A2s = hs.A2s0 ^ s_hi;
    uint32_t B1, h0c, l0c;
    site_rounds(A2s, hs.B1k, B1, h0c, l0c);
    uint32_t W[4], V[4];
    draw2(hs.tab[0], hs.tab[1], B1, h0c, l0c, p, W, V);
    uint32_t b, eq;
    cmp8<ZC>(c4, c8, hs.tab[0], hs.tab[1], W, V, b, eq);
    const uint32_t lt = b & need;
    const uint32_t und = eq & need;
    const bool undecided = und != 0u;
    const uint32_t ball = __ballot_sync(0xFFFFFFFFu, undecided);
    const int slot = undecided ? wq + __popc(ball & lml) : qscratch + lane;
    queue[slot] = make_uint4(A2s, und, lt, 0u);
    const uint32_t f = (~need | lt) & (undecided ? 0u : hs.vmask);
    la[0] = w ^ f;
    acc += (uint32_t)__popc(f);
    wq += __popc(ball);
}

// Pass 2: the warp's nq queued sites, one per lane, from plane block 2 on.
template <int L, bool EA>
__device__ __forceinline__ void site_pass2(uint32_t* lat, const uint4* jw, const uint4* queue,
                                           int nq, int lane, uint32_t A2x, uint32_t B1k,
                                           uint32_t vmask, const Tab2* tab, const KParams& p,
                                           uint32_t& acc) {
    constexpr int P = L + 2;
    constexpr int LG = (L == 16) ? 4 : (L == 32) ? 5 : (L == 64) ? 6 : 7;
    __syncwarp();
    for (int e = lane; e < nq; e += 32) {
        const uint4 q = queue[e];
        const uint32_t s = q.x ^ A2x;
        uint32_t und = q.y, lt = q.z;
        const int c = Geo2<L>::cell((int)(s & (L - 1)), (int)(s >> LG));
        uint32_t* la = lat + c;
        const uint32_t w = la[0];
        uint32_t need, c4, c8;
        if (EA) {
            uint32_t P0 = w ^ la[1], P1 = w ^ la[-1], P2 = w ^ la[P], P3 = w ^ la[-P];
            const uint4 J = jw[c];
            P0 ^= J.x;
            P1 ^= J.y;
            P2 ^= J.z;
            P3 ^= J.w;
            classes(P0, P1, P2, P3, vmask, need, c4, c8);
        } else {
            classes_w(w, la[1], la[-1], la[P], la[-P], vmask, need, c4, c8);
        }
        uint32_t B1, h0c, l0c;
        site_rounds(q.x, B1k, B1, h0c, l0c);
        finish(c4, c8, tab, B1, h0c, l0c, p, und, lt);
        const uint32_t f = (~need | lt) & vmask;
        la[0] = w ^ f;
        acc += (uint32_t)__popc(f);
    }
    __syncwarp();
}

template <int L, int NT, bool EA>
__global__ void __launch_bounds__(NT, 65536 / (NT * 80)) k_sweep2d(KParams p) {
    constexpr int P = L + 2, N = L * L, TPR = L / 2, RP = NT / TPR, ITERS = L / RP;
    constexpr int NW = NT / 32, W = N / 32;
    constexpr int LG = (L == 16) ? 4 : (L == 32) ? 5 : (L == 64) ? 6 : 7;
    constexpr int LAT_WORDS = (P * P + 3) & ~3;
    // a warp's queue: QW entries, then 32 scratch slots; the warp finishes its
    // queue early when fewer than 32 free entries remain (at most 12% of sites are
    // undecided after eight planes on average, so this practically never happens)
    constexpr int QW = (32 * ITERS) / 4 + 32;
    static_assert((1 << LG) == L && RP % 2 == 0 && ITERS * RP == L, "2D sweep shape");
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t* lat = smem;
    uint4* jw = reinterpret_cast<uint4*>(smem + LAT_WORDS);
    uint4* qbase = reinterpret_cast<uint4*>(smem + LAT_WORDS + (EA ? 4 * P * P : 0));
    __shared__ __align__(16) Tab2 tabs[2][8];
    __shared__ int32_t sU[32];
    __shared__ int32_t sNup[32];
    __shared__ unsigned long long sAcc;

    const RunDesc& r = p.runs[p.grp2run[blockIdx.x]];
    const DevState* st = r.st;
    if (st->status != S_OK) return;
    const int i = st->step + 1;
    const uint32_t R = st->R_cur;
    const uint32_t base = (blockIdx.x - r.grp0) * 32u;
    if (base >= R) return;
    const uint32_t nval = min(32u, R - base);
    const uint32_t vmask = (nval == 32u) ? 0xFFFFFFFFu : ((1u << nval) - 1u);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t* src = r.spins[(i - 1) & 1];
    uint32_t* dst = r.spins[i & 1];
    uint4* queue = qbase + warp * (QW + 32);
    // the queue is finished once it holds more than qflush entries, which leaves
    // room for the next site of every lane (qflush + 32 <= QW).  The test hook can
    // lower it to 0: the queue is then finished after every site of the walk.  A
    // round of the walk always takes at least one site (wq = 0 <= qflush).
    const int qcap = (p.qcap_limit >= 0 && p.qcap_limit < QW) ? p.qcap_limit : QW;
    const int qflush = qcap >= 32 ? qcap - 32 : 0;
    const uint32_t lml = (1u << lane) - 1u;

    if (threadIdx.x < 32) {
        sU[threadIdx.x] = 0;
        sNup[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) sAcc = 0ull;

    const bool valid = (uint32_t)lane < nval;
    uint32_t my_src = base + lane;
    if (valid) my_src = r.anc[base + lane];
    if (warp == 0 && valid) r.fam[i & 1][base + lane] = r.fam[(i - 1) & 1][my_src];

    // gather the 32 parent rows (the copy of step 2) and transpose them into the
    // multi-spin form
    for (int c4 = warp; 4 * c4 < W; c4 += NW) {
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (valid) v = reinterpret_cast<const uint4*>(src + (size_t)my_src * r.Wp)[c4];
        const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int s = 32 * (4 * c4 + k) + lane;
            lat[Geo2<L>::cell(s & (L - 1), s >> LG)] = transpose32(w4[k], lane);
        }
    }
    if (EA) {
        for (int s = threadIdx.x; s < N; s += NT) {
            const int x = s & (L - 1), y = s >> LG;
            const uint32_t js = r.jbits[s];
            const uint32_t jxm = r.jbits[y * L + ((x - 1) & (L - 1))];
            const uint32_t jym = r.jbits[((y - 1) & (L - 1)) * L + x];
            jw[Geo2<L>::cell(x, y)] = make_uint4(0u - (js & 1u), 0u - (jxm & 1u),
                                                 0u - ((js >> 1) & 1u), 0u - ((jym >> 1) & 1u));
        }
    }
    __syncthreads();
    // periodic copies in the halo
    for (int k = threadIdx.x; k < 4 * L; k += NT) {
        const int side = k / L, j = k - side * L;
        if (side == 0) lat[Geo2<L>::cell(L, j)] = lat[Geo2<L>::cell(0, j)];
        else if (side == 1) lat[Geo2<L>::cell(-1, j)] = lat[Geo2<L>::cell(L - 1, j)];
        else if (side == 2) lat[Geo2<L>::cell(j, L)] = lat[Geo2<L>::cell(j, 0)];
        else lat[Geo2<L>::cell(j, -1)] = lat[Geo2<L>::cell(j, L - 1)];
    }

    const uint32_t grp = blockIdx.x;  // global replica group
    uint32_t A2x, B1k;  // round-1 lane 2 without the site; round-2 lane 0 key part
    {
        uint32_t h0a, l0a, h1a, l1a;
        mulhilo(PHILOX_M0, grp, h0a, l0a);
        mulhilo(PHILOX_M1, (uint32_t)i, h1a, l1a);
        A2x = h0a ^ p.rk1[0];
        B1k = l1a ^ p.rk0[1];
    }
    const uint32_t nh = 2u * r.stheta[i - 1];
    const int zc = zero_classes2(r.sthr[4 * (i - 1) + 1], r.sthr[4 * (i - 1) + 2]);
    if (nh > 0 && threadIdx.x < 8)
        build_tab2(tabs[0], threadIdx.x, p, grp, (uint32_t)i, 0u, 0, r.sthr[4 * (i - 1) + 1],
                   r.sthr[4 * (i - 1) + 2]);
    __syncthreads();

    uint32_t acc = 0;
    for (uint32_t h = 0; h < nh; ++h) {
        const int colour = (int)(h & 1u);
        if (h + 1 < nh && threadIdx.x < 8) {
            const int ii = st->step + 1;
            build_tab2(tabs[(h + 1) & 1u], threadIdx.x, p, grp, (uint32_t)ii, (h + 1) >> 1,
                       (int)((h + 1) & 1u), r.sthr[4 * (ii - 1) + 1], r.sthr[4 * (ii - 1) + 2]);
        }
        // the thread's place in the walk: column slot xi of rows y0, y0 + RP, ...
        int y0, xi;
        if constexpr (TPR >= 16) {
            constexpr int CH = TPR / 16;
            y0 = 2 * (warp / CH) + ((threadIdx.x >> 4) & 1);
            xi = 16 * (warp % CH) + (threadIdx.x & 15);
        } else {
            y0 = threadIdx.x / TPR;
            xi = threadIdx.x % TPR;
        }
        const int x = 2 * xi + ((y0 + colour) & 1);
        Half hs;
        hs.tab = tabs[h & 1u];
        hs.B1k = B1k;
        hs.vmask = vmask;
        // the site counter of row y0 + k RP is (x + L y0) | (k RP L), x + L y0 < RP L
        hs.A2s0 = A2x ^ (uint32_t)(x + L * y0);
        uint32_t* la0 = lat + Geo2<L>::cell(x, y0);
        const uint4* ja0 = jw + Geo2<L>::cell(x, y0);
        // pass 1 over rows y0, y0 + RP, ..., pass 2 over the queue (also earlier if
        // the queue runs short of room)
        int k = 0;
        while (true) {
            int wq = 0;
            // a copy of the walk for ZC = 0 and one for ZC >= 1 (the same for the whole
            // launch; a third copy for ZC = 2, which drops the dE = 4 term as well,
            // slowed the ZC = 0 walk more than it saves above beta = ln 256 / 4)
            auto pass1 = [&](auto zc_tag) {
                constexpr int ZC = decltype(zc_tag)::value;
#pragma unroll 1
                for (; k < ITERS && wq <= qflush; ++k)
                    site_pass1<L, EA, ZC>(la0 + k * RP * P, ja0 + k * RP * P,
                                          (uint32_t)(k * RP * L), hs, p, queue, QW, lml, lane,
                                          wq, acc);
            };
            if (zc == 0) pass1(IC<0>{});
            else pass1(IC<1>{});
            site_pass2<L, EA>(lat, jw, queue, wq, lane, A2x, B1k, vmask, hs.tab, p, acc);
            if (k == ITERS) break;
        }
        // periodic copies of the thread's boundary sites (the warp's sites are final)
        if (x == 0)
            for (int kk = 0; kk < ITERS; ++kk) la0[kk * RP * P + L] = la0[kk * RP * P];
        if (x == L - 1)
            for (int kk = 0; kk < ITERS; ++kk) la0[kk * RP * P - L] = la0[kk * RP * P];
        if (y0 == 0) la0[L * P] = la0[0];
        if (y0 == RP - 1) la0[(ITERS - 1) * RP * P - L * P] = la0[(ITERS - 1) * RP * P];
        __syncthreads();
    }

    // measurement: unsatisfied bonds U and up-count per replica, write back.  The
    // thread's unsatisfied-bond words go into a bit-sliced counter (at most 2 per
    // site word it visits), summed per replica at the end.
    constexpr int CB = vc_bits(2 * 4 * ((W / 4 + NW - 1) / NW));
    uint32_t ucnt[CB];
#pragma unroll
    for (int j = 0; j < CB; ++j) ucnt[j] = 0u;
    int32_t nup = 0;
    for (int c4 = warp; 4 * c4 < W; c4 += NW) {
        uint32_t out[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int s = 32 * (4 * c4 + k) + lane;
            const int c = Geo2<L>::cell(s & (L - 1), s >> LG);
            const uint32_t w = lat[c];
            const uint32_t tw = transpose32(w, lane);
            out[k] = tw;
            nup += __popc(tw);
            uint32_t P0 = w ^ lat[c + 1], P1 = w ^ lat[c + P];
            if (EA) {
                const uint4 J = jw[c];
                P0 ^= J.x;
                P1 ^= J.z;
            }
            vc_add2(ucnt, P0, P1);
        }
        if (valid)
            reinterpret_cast<uint4*>(dst + (size_t)(base + lane) * r.Wp)[c4] =
                make_uint4(out[0], out[1], out[2], out[3]);
    }
    const int32_t U = vc_total(ucnt, lane);
    atomicAdd(&sU[lane], U);
    atomicAdd(&sNup[lane], nup);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0 && acc) atomicAdd(&sAcc, (unsigned long long)acc);
    __syncthreads();

    if (warp == 0) {
        long long e = 0, e2 = 0, am = 0, m2 = 0;
        int lvmin = 0x7FFFFFFF, lvmax = -1;  // the warp's histogram levels
        if (valid) {
            const int32_t Uv = sU[lane];
            const int32_t E = 2 * Uv - 2 * N;
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

template <int L, int NT, bool EA>
constexpr size_t smem2d() {
    constexpr int P = L + 2, ITERS = L / (NT / (L / 2));
    constexpr int LAT_WORDS = (P * P + 3) & ~3;
    constexpr int QW = (32 * ITERS) / 4 + 32;
    return (size_t)LAT_WORDS * 4 + (EA ? (size_t)P * P * 16 : 0) + (size_t)(NT / 32) * (QW + 32) * 16;
}

// dynamic shared memory a CTA may take (the opt-in limit less the kernel's static part)
constexpr size_t SMEM2D_MAX = 227 * 1024 - 2048;

// *done = false for a shape whose lattice does not fit one CTA's shared memory (the
// +-J bond records of L = 128): the general kernel takes those runs
template <int L, int NT, bool EA>
cudaError_t launch2d(const KParams& p, cudaStream_t s, bool attr_only, bool* done) {
    constexpr size_t sm = smem2d<L, NT, EA>();
    if constexpr (sm > SMEM2D_MAX) {
        *done = false;
        return cudaSuccess;
    } else {
        static bool attr_set = false;
        if (!attr_set) {
            cudaError_t e = cudaFuncSetAttribute(k_sweep2d<L, NT, EA>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)sm);
            if (e != cudaSuccess) return e;
            attr_set = true;
        }
        if (attr_only) return cudaSuccess;
        k_sweep2d<L, NT, EA><<<p.ngrp_total, NT, sm, s>>>(p);
        return cudaGetLastError();
    }
}

template <bool EA>
cudaError_t launch2d_shape(const KParams& p, int threads, cudaStream_t s, bool attr_only,
                           bool* done) {
    *done = true;
    switch (p.L_all * 1000 + threads) {
        case 16064: return launch2d<16, 64, EA>(p, s, attr_only, done);
        case 16128: return launch2d<16, 128, EA>(p, s, attr_only, done);
        case 32128: return launch2d<32, 128, EA>(p, s, attr_only, done);
        case 32256: return launch2d<32, 256, EA>(p, s, attr_only, done);
        case 32512: return launch2d<32, 512, EA>(p, s, attr_only, done);
        case 64128: return launch2d<64, 128, EA>(p, s, attr_only, done);
        case 64256: return launch2d<64, 256, EA>(p, s, attr_only, done);
        case 64512: return launch2d<64, 512, EA>(p, s, attr_only, done);
        case 128128: return launch2d<128, 128, EA>(p, s, attr_only, done);
        case 128256: return launch2d<128, 256, EA>(p, s, attr_only, done);
        case 128512: return launch2d<128, 512, EA>(p, s, attr_only, done);
        default: *done = false; return cudaSuccess;
    }
}

}  // namespace

// The 2D kernel for runs that all have the same power-of-two side L (16..128)
// at a supported CTA size; *done = false when the shape has no 2D kernel.
// attr_only: set the kernel's function attributes only (before a stream capture).
cudaError_t launch_sweep2d(const KParams& p, int threads, cudaStream_t s, bool attr_only,
                           bool* done) {
    *done = false;
    if (p.d != 2 || p.L_all == 0) return cudaSuccess;
    return p.ea ? launch2d_shape<true>(p, threads, s, attr_only, done)
                : launch2d_shape<false>(p, threads, s, attr_only, done);
}

}  // namespace pa
