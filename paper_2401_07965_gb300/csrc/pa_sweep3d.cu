// pa_sweep3d.cu -- the temperature step's replica copy, theta checkerboard
// Metropolis sweeps and measurement (Sec. 2 steps 2-4) for three-dimensional
// runs of side 4 <= L <= 16: the work of k_group's sweep mode with a layout for
// small lattices.  Random numbers, decisions and results are the same.
//
// Grouping.  A 3D lattice of a few hundred sites gives one group of 32 replicas
// too little work per half-sweep (and per barrier, and per flush of the queue
// of undecided sites), so a CTA of 128 threads holds G replica groups of one
// run (G = 16, 8, 4, 2 for L = 4, 6, 8, 10; 1 above), about eight site words
// per thread and half-sweep: G halo-padded multi-spin lattices in shared
// memory (cell (x, y, z), -1 <= x, y, z <= L, word ((z+1)(L+2) + y+1)(L+2) +
// x+1), each group keeping its own Philox counter (its global replica group).
// Every neighbour of an interior site is at a fixed offset +-1, +-(L+2),
// +-(L+2)^2; a flip of a boundary site also writes its copies in the halo faces.
//
// Walk.  A per-colour table lists the N/2 sites of the colour (lattice word,
// boundary faces, Philox site index) and, for the spin glass, the six bond
// signs of each as byte sign bits; entry e of the CTA's G x N/2 work items is
// group e / (N/2), site e mod (N/2), thread t taking e = t, t + 128, ...
// Consecutive lanes read consecutive table words.  Undecided sites after eight
// planes go to per-warp queues and are finished by the same warp (branch-free
// first pass, as in 2D).
//
// Philox.  Of the round-2 and round-3 values that do not depend on the site,
// the part that does not depend on the group either (the counter word holding
// sweep, colour and plane block) is computed once per half-sweep and plane
// block; the group's part of blocks 0 and 1 is tabulated per group; blocks 2-7,
// needed by few sites, are completed in the queue pass.
//
// Energy classes of d = 3 (n unsatisfied bonds of 6): dE = 4 (n = 2), 8 (n = 1),
// 12 (n = 0), disjoint masks, so a plane's threshold bit word is the sum
// c4 b4 + c8 b8 + c12 b12 (multiply-adds on the multiply pipe).
#include "pa_sweep_common.cuh"

namespace pa {
namespace {

constexpr int NT3 = 128;

// replica groups per CTA of side L
template <int L>
struct Groups3 {
    static constexpr int value = L == 4 ? 16 : (L == 6 ? 8 : (L == 8 ? 4 : (L == 10 ? 2 : 1)));
};

// GM: a multiple of the base group count (the autotuner may double it)
template <int L, int GM = 1>
struct Shape3 {
    static constexpr int P = L + 2, P2 = P * P, N = L * L * L, H = N / 2;
    static constexpr int G = Groups3<L>::value * GM;
    static constexpr int ITERS = (G * H + NT3 - 1) / NT3;
    static constexpr int W = (N + 31) / 32, WP = (W + 3) & ~3;
    static constexpr int CELLS = P * P * P;
    static constexpr int LAT_WORDS = (G * CELLS + 3) & ~3;
    // per warp, then 32 scratch slots
    static constexpr int QW = ((32 * ITERS) / 4 < 64 ? (32 * ITERS) / 4 : 64) + 32;
    __host__ __device__ static constexpr int cell(int x, int y, int z) {
        return ((z + 1) * P + y + 1) * P + x + 1;
    }
};

// The group-independent round-2 product of a plane block's counter word
// (DOM_SWEEP | sweep << 4 | colour << 3 | block) and the key: (h0b, c2k).
__device__ __forceinline__ uint2 block_part(const KParams& p, uint32_t h1a, uint32_t t, int colour,
                                            int b) {
    const uint32_t c1v = DOM_SWEEP | (t << 4) | ((uint32_t)colour << 3) | (uint32_t)b;
    uint32_t h0b, l0b;
    mulhilo(PHILOX_M0, h1a ^ c1v ^ p.rk0[0], h0b, l0b);
    return make_uint2(h0b, l0b ^ p.rk1[2]);
}

// a group's round-3 values of a plane block (c0k, c1, c2k): l0a is the low word
// of the group counter's round-1 product
__device__ __forceinline__ uint4 group_part(const KParams& p, uint2 bp, uint32_t l0a) {
    uint32_t h1c, l1c;
    mulhilo(PHILOX_M1, bp.x ^ l0a ^ p.rk1[1], h1c, l1c);
    return make_uint4(h1c ^ p.rk0[2], l1c, bp.y, 0u);
}

__device__ __forceinline__ void draw2_3(const uint4 e, const uint4 f, uint32_t B1, uint32_t h0c,
                                        uint32_t l0c, const KParams& p, uint32_t (&W)[4],
                                        uint32_t (&V)[4]) {
    uint32_t x0 = e.x ^ B1, x1 = e.y, x2 = h0c ^ e.z, x3 = l0c;
    uint32_t y0 = f.x ^ B1, y1 = f.y, y2 = h0c ^ f.z, y3 = l0c;
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

__device__ __forceinline__ void draw1_3(const uint4 e, uint32_t B1, uint32_t h0c, uint32_t l0c,
                                        const KParams& p, uint32_t (&W)[4]) {
    uint32_t x0 = e.x ^ B1, x1 = e.y, x2 = h0c ^ e.z, x3 = l0c;
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

// classes from the site word w and its six bond partners a[i] (neighbour word,
// XOR the bond's sign for the spin glass; bond i is unsatisfied where w ^ a[i] =
// 1): n unsatisfied bonds as a bit-sliced count (n2 n1 n0); need = n <= 2 among
// the valid replicas.  The sum and carry of a triple of bonds are
// w ^ (a ^ b ^ c) and w ^ maj(a, b, c), so w cancels from n0 and n1 and enters
// only the two carries of the second stage.
__device__ __forceinline__ void classes3_w(uint32_t w, const uint32_t (&a)[6], uint32_t vmask,
                                           uint32_t& need, uint32_t& c4, uint32_t& c8,
                                           uint32_t& c12) {
    const uint32_t x3 = lop3<0x96>(a[0], a[1], a[2]), ma = lop3<0xE8>(a[0], a[1], a[2]);
    const uint32_t y3 = lop3<0x96>(a[3], a[4], a[5]), mb = lop3<0xE8>(a[3], a[4], a[5]);
    const uint32_t n0 = x3 ^ y3;
    const uint32_t kc = lop3<0x18>(w, x3, y3);                         // (w^x3)&(w^y3)
    const uint32_t n1 = lop3<0x96>(ma, mb, kc);
    const uint32_t n2 = lop3<0x18>(w, ma, mb) | lop3<0x60>(kc, ma, mb); // carry of the carries
    need = lop3<0x07>(n2, n1, n0) & vmask;                             // ~n2 & ~(n1 & n0)
    c12 = lop3<0x01>(n0, n1, n2);
    c8 = lop3<0x10>(n0, n1, n2);
    c4 = lop3<0x04>(n0, n1, n2);
}

// threshold bits of a plane block for the three classes (0 or 1 per plane)
struct BlockBits {
    uint4 b4, b8, b12;
};

__device__ __forceinline__ uint32_t lane4(const uint4 v, int m) {
    return m == 0 ? v.x : (m == 1 ? v.y : (m == 2 ? v.z : v.w));
}

__device__ __forceinline__ uint32_t thr_word(uint32_t c4, uint32_t c8, uint32_t c12,
                                             const BlockBits& t, int m) {
    return c4 * lane4(t.b4, m) + c8 * lane4(t.b8, m) + c12 * lane4(t.b12, m);
}

// the threshold word of plane m of a block with the terms of the ZC highest
// classes (dE = 12, then 8, then 4) left out: their top eight bits are zero
template <int ZC>
__device__ __forceinline__ uint32_t thr_word_z(uint32_t c4, uint32_t c8, uint32_t c12,
                                               const BlockBits& t, int m) {
    if constexpr (ZC == 0) return thr_word(c4, c8, c12, t, m);
    if constexpr (ZC == 1) return c4 * lane4(t.b4, m) + c8 * lane4(t.b8, m);
    return c4 * lane4(t.b4, m);
}

// ZC of a step from its thresholds of dE = 4, 8 and 12 (top eight bits)
__device__ __forceinline__ int zero_classes3(uint32_t thr4, uint32_t thr8, uint32_t thr12) {
    if ((thr12 >> 24) != 0u) return 0;
    if ((thr8 >> 24) != 0u) return 1;
    return (thr4 >> 24) != 0u ? 2 : 3;
}

template <int V>
struct IC {
    static constexpr int value = V;
};

// planes 0-7 by the borrow of the subtraction from the least significant plane
// up; with ZC = 3 (every threshold's top eight bits zero) t = 0: b = 0 and
// eq = [u8 == 0]
template <int ZC>
__device__ __forceinline__ void cmp8_3(uint32_t c4, uint32_t c8, uint32_t c12, const BlockBits* bt,
                                       const uint32_t (&W)[4], const uint32_t (&V)[4],
                                       uint32_t& b, uint32_t& eq) {
    if constexpr (ZC >= 3) {
        b = 0u;
        eq = lop3<0x01>(lop3<0xFE>(V[0], V[1], V[2]), lop3<0xFE>(V[3], W[0], W[1]),
                        W[2] | W[3]);  // ~(a | b | c)
        return;
    }
    b = 0u;
    eq = 0xFFFFFFFFu;
    const BlockBits f = bt[1];
#pragma unroll
    for (int m = 3; m >= 0; --m) {
        const uint32_t t = thr_word_z<ZC>(c4, c8, c12, f, m);
        b = lop3<0x8E>(V[m], t, b);    // (~V & t) | (~(V ^ t) & b)
        eq = lop3<0x82>(V[m], t, eq);  // eq & ~(V ^ t)
    }
    const BlockBits e = bt[0];
#pragma unroll
    for (int m = 3; m >= 0; --m) {
        const uint32_t t = thr_word_z<ZC>(c4, c8, c12, e, m);
        b = lop3<0x8E>(W[m], t, b);
        eq = lop3<0x82>(W[m], t, eq);
    }
}

// plane blocks 2-7 of an undecided site, block by block from the top
__device__ __forceinline__ void finish3(uint32_t c4, uint32_t c8, uint32_t c12, const uint2* bpart,
                                        const BlockBits* bt, uint32_t l0a, uint32_t B1,
                                        uint32_t h0c, uint32_t l0c, const KParams& p,
                                        uint32_t& und, uint32_t& lt) {
#pragma unroll 1
    for (int g = 2; g < 8 && und; ++g) {
        uint32_t W[4];
        draw1_3(group_part(p, bpart[g], l0a), B1, h0c, l0c, p, W);
        const BlockBits t = bt[g];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const uint32_t tm = thr_word(c4, c8, c12, t, m);
            lt |= lop3<0x40>(und, tm, W[m]);   // und & tm & ~W
            und = lop3<0x82>(W[m], tm, und);   // und & ~(W ^ tm)
        }
    }
}

// all-ones if the sign bit of byte SEL & 3 of v is set, else zero (prmt with
// every selector nibble 8 + byte replicates the selected byte's sign bit)
template <int SEL>
__device__ __forceinline__ uint32_t sign_of_byte(uint32_t v) {
    uint32_t r;
    asm("prmt.b32 %0, %1, %1, %2;" : "=r"(r) : "r"(v), "n"(SEL));
    return r;
}

// the six bond partners of a site: neighbour words, XOR the bond signs for EA
// (j holds them as byte sign bits: x bytes 0-3 the bonds to +x, -x, +y, -y and
// y bytes 0-1 those to +z, -z)
template <int L, bool EA>
__device__ __forceinline__ void bond_partners(const uint32_t* la, uint2 j, uint32_t (&a)[6]) {
    constexpr int PP = L + 2, P2 = PP * PP;
    a[0] = la[1];
    a[1] = la[-1];
    a[2] = la[PP];
    a[3] = la[-PP];
    a[4] = la[P2];
    a[5] = la[-P2];
    if (EA) {
        a[0] ^= sign_of_byte<0x8888>(j.x);
        a[1] ^= sign_of_byte<0x9999>(j.x);
        a[2] ^= sign_of_byte<0xAAAA>(j.x);
        a[3] ^= sign_of_byte<0xBBBB>(j.x);
        a[4] ^= sign_of_byte<0x8888>(j.y);
        a[5] ^= sign_of_byte<0x9999>(j.y);
    }
}

// store a flipped site and its halo copies
template <int L>
__device__ __forceinline__ void store_site(uint32_t* la, uint32_t v, uint32_t faces) {
    constexpr int P = L + 2, P2 = P * P;
    la[0] = v;
    if (faces & 1u) la[L] = v;
    if (faces & 2u) la[-L] = v;
    if (faces & 4u) la[L * P] = v;
    if (faces & 8u) la[-L * P] = v;
    if (faces & 16u) la[L * P2] = v;
    if (faces & 32u) la[-L * P2] = v;
}

// site-table entry of site s: x = lattice word in group 0 | faces << 16 (bit f:
// the site is on the face x = 0, x = L-1, y = 0, y = L-1, z = 0, z = L-1),
// y = s
template <int L>
__device__ __forceinline__ uint2 site_entry(int s) {
    using S = Shape3<L>;
    const int x = s % L, y = (s / L) % L, z = s / (L * L);
    const uint32_t faces = (x == 0 ? 1u : 0u) | (x == L - 1 ? 2u : 0u) | (y == 0 ? 4u : 0u) |
                           (y == L - 1 ? 8u : 0u) | (z == 0 ? 16u : 0u) | (z == L - 1 ? 32u : 0u);
    return make_uint2((uint32_t)S::cell(x, y, z) | (faces << 16), (uint32_t)s);
}

// the bond-sign word of site s (layout of bond_partners) from the coupling bits
// (bit a of jbits[s]: bond (s, s + e_a) has J = -1)
template <int L>
__device__ __forceinline__ uint2 bond_entry(const uint8_t* jbits, int s) {
    const int x = s % L, y = (s / L) % L, z = s / (L * L);
    const uint32_t js = jbits[s];
    const uint32_t jxm = jbits[z * L * L + y * L + (x + L - 1) % L];
    const uint32_t jym = jbits[z * L * L + ((y + L - 1) % L) * L + x];
    const uint32_t jzm = jbits[((z + L - 1) % L) * L * L + y * L + x];
    const uint32_t bx = ((js & 1u) << 7) | ((jxm & 1u) << 15) | (((js >> 1) & 1u) << 23) |
                        (((jym >> 1) & 1u) << 31);
    const uint32_t by = (((js >> 2) & 1u) << 7) | (((jzm >> 2) & 1u) << 15);
    return make_uint2(bx, by);
}

template <int L, bool EA, int GM>
__global__ void __launch_bounds__(NT3, 6) k_sweep3d(KParams p, const uint32_t* cta2run) {
    using S = Shape3<L, GM>;
    constexpr int G = S::G, H = S::H, N = S::N, P = S::P, P2 = S::P2, NW = NT3 / 32;
    constexpr int W = S::W, WP = S::WP;
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t* lat = smem;                                               // G halo lattices
    uint2* stab = reinterpret_cast<uint2*>(smem + S::LAT_WORDS);       // 2 x H site entries
    uint2* jq = stab + 2 * H;                                          // EA: 2 x H bond words
    uint4* qbase = reinterpret_cast<uint4*>(jq + (EA ? 2 * H : 0));    // NW x (QW + 32)
    __shared__ __align__(16) uint4 gtab[2][G][2];  // group parts of blocks 0, 1 per half-sweep
    __shared__ uint2 bpart[2][8];                  // block parts per half-sweep
    __shared__ BlockBits btab[8];                  // threshold bits of the step's classes
    __shared__ uint32_t sA2x[G], sL0a[G], sVm[G];
    __shared__ int32_t sU[G][32], sNup[G][32];
    __shared__ unsigned long long sAcc;

    const RunDesc& r = p.runs[cta2run[blockIdx.x]];
    const DevState* st = r.st;
    if (st->status != S_OK) return;
    const int i = st->step + 1;
    const uint32_t R = st->R_cur;
    const uint32_t gfirst = (blockIdx.x - r.cta0) * G;   // the CTA's first group in its run
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t* src = r.spins[(i - 1) & 1];
    uint32_t* dst = r.spins[i & 1];
    uint4* queue = qbase + warp * (S::QW + 32);
    const int qcap = (p.qcap_limit >= 0 && p.qcap_limit < S::QW) ? p.qcap_limit : S::QW;
    const int qflush = qcap >= 32 ? qcap - 32 : 0;

    // Philox parts of the step, the groups' counters and the valid-replica masks
    uint32_t B1k, h1a;
    {
        uint32_t l1a;
        mulhilo(PHILOX_M1, (uint32_t)i, h1a, l1a);
        B1k = l1a ^ p.rk0[1];
    }
    if (threadIdx.x < G) {
        const uint32_t g = threadIdx.x;
        const uint32_t base = (gfirst + g) * 32u;
        const uint32_t nval = base < R ? min(32u, R - base) : 0u;
        sVm[g] = nval == 32u ? 0xFFFFFFFFu : ((1u << nval) - 1u);
        uint32_t h0a, l0a;
        mulhilo(PHILOX_M0, r.grp0 + gfirst + g, h0a, l0a);
        sA2x[g] = h0a ^ p.rk1[0];
        sL0a[g] = l0a;
    }
    const uint32_t* thr = r.sthr + 4 * (i - 1);
    if (threadIdx.x < 8 * 3) {
        const int b = threadIdx.x / 3, k = threadIdx.x % 3;
        const uint32_t tk = thr[k + 1];
        const uint4 v = make_uint4((tk >> (31 - 4 * b)) & 1u, (tk >> (30 - 4 * b)) & 1u,
                                   (tk >> (29 - 4 * b)) & 1u, (tk >> (28 - 4 * b)) & 1u);
        if (k == 0) btab[b].b4 = v;
        else if (k == 1) btab[b].b8 = v;
        else btab[b].b12 = v;
    }
    for (int k = threadIdx.x; k < G * 32; k += NT3) {
        sU[k >> 5][k & 31] = 0;
        sNup[k >> 5][k & 31] = 0;
    }
    if (threadIdx.x == 0) sAcc = 0ull;
    // families of the new slots
    for (int k = threadIdx.x; k < G * 32; k += NT3) {
        const uint32_t slot = (gfirst + (k >> 5)) * 32u + (k & 31);
        if (slot < R) r.fam[i & 1][slot] = r.fam[(i - 1) & 1][r.anc[slot]];
    }
    // gather the parent rows of every group and transpose them into the multi-spin form
    for (int k = warp; k < G * (WP / 4); k += NW) {
        const int g = k / (WP / 4), c4 = k % (WP / 4);
        const uint32_t slot = (gfirst + g) * 32u + lane;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (slot < R) v = reinterpret_cast<const uint4*>(src + (size_t)r.anc[slot] * r.Wp)[c4];
        const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int b = 4 * c4 + m;
            if (b < W) {  // warp-uniform
                const uint32_t t = transpose32(w4[m], lane);
                const int s = 32 * b + lane;
                if (s < N)
                    lat[g * S::CELLS + S::cell(s % L, (s / L) % L, s / (L * L))] = t;
            }
        }
    }
    // site tables of the two colours (site q of a colour: s = 2q or 2q + 1), and
    // the bond signs (EA)
    for (int k = threadIdx.x; k < 2 * H; k += NT3) {
        const int colour = k / H, q = k % H;
        const int s0 = 2 * q;
        const int x0 = s0 % L, yz = s0 / L;
        const int s = s0 + ((((yz % L) + (yz / L) + x0) & 1) != colour ? 1 : 0);
        stab[k] = site_entry<L>(s);
        if (EA) jq[k] = bond_entry<L>(r.jbits, s);
    }
    __syncthreads();
    // periodic copies in the halo faces
    for (int k = threadIdx.x; k < G * 6 * L * L; k += NT3) {
        const int g = k / (6 * L * L), f = (k / (L * L)) % 6, a = k % L, b = (k / L) % L;
        uint32_t* lg = lat + g * S::CELLS;
        int d, sidx;
        switch (f) {
            case 0: d = S::cell(L, a, b); sidx = S::cell(0, a, b); break;
            case 1: d = S::cell(-1, a, b); sidx = S::cell(L - 1, a, b); break;
            case 2: d = S::cell(a, L, b); sidx = S::cell(a, 0, b); break;
            case 3: d = S::cell(a, -1, b); sidx = S::cell(a, L - 1, b); break;
            case 4: d = S::cell(a, b, L); sidx = S::cell(a, b, 0); break;
            default: d = S::cell(a, b, -1); sidx = S::cell(a, b, L - 1); break;
        }
        lg[d] = lg[sidx];
    }
    // Philox tables of half-sweep hh: the block parts (all eight blocks) and the
    // groups' parts of blocks 0 and 1
    auto build_tables = [&](uint32_t hh) {
        const uint32_t t = hh >> 1;
        const int colour = (int)(hh & 1u);
        for (int k = threadIdx.x; k < 8 + 2 * G; k += NT3) {
            if (k < 8) {
                bpart[hh & 1u][k] = block_part(p, h1a, t, colour, k);
            } else {
                const int g = (k - 8) >> 1, b = (k - 8) & 1;
                gtab[hh & 1u][g][b] = group_part(p, block_part(p, h1a, t, colour, b), sL0a[g]);
            }
        }
    };
    const uint32_t nh = 2u * r.stheta[i - 1];
    const int zc = zero_classes3(thr[1], thr[2], thr[3]);
    if (nh > 0) build_tables(0u);
    __syncthreads();

    const uint32_t lml = (1u << lane) - 1u;
    uint32_t acc = 0;
    for (uint32_t h = 0; h < nh; ++h) {
        const int colour = (int)(h & 1u);
        if (h + 1 < nh) build_tables(h + 1);
        const uint2* ct = stab + colour * H;
        const uint2* cj = jq + colour * H;
        const uint4(*gt)[2] = gtab[h & 1u];
        int k = 0;
        while (true) {
            int wq = 0;
            // one copy of the walk per ZC (the same for the whole launch)
            auto pass1 = [&](auto zc_tag) {
                constexpr int ZC = decltype(zc_tag)::value;
#pragma unroll 1
                for (; k < S::ITERS && wq <= qflush; ++k) {
                    const int e = threadIdx.x + k * NT3;
                    const bool have = e < G * H;
                    // lanes past the work items run item 0 with no valid replica
                    const int ee = have ? e : 0;
                    const int g = ee / H, q = ee - g * H;
                    const uint2 en = ct[q];
                    uint32_t* la = lat + g * S::CELLS + (en.x & 0xFFFFu);
                    const uint32_t s = en.y;
                    const uint32_t vm = have ? sVm[g] : 0u;
                    const uint32_t w = la[0];
                    uint32_t ab[6];
                    bond_partners<L, EA>(la, EA ? cj[q] : make_uint2(0u, 0u), ab);
                    uint32_t need, c4, c8, c12;
                    classes3_w(w, ab, vm, need, c4, c8, c12);
                    const uint32_t A2s = sA2x[g] ^ s;
                    uint32_t B1, h0c, l0c;
                    {
                        uint32_t h1b, l1b;
                        mulhilo(PHILOX_M1, A2s, h1b, l1b);
                        B1 = l1b;
                        mulhilo(PHILOX_M0, h1b ^ B1k, h0c, l0c);
                    }
                    uint32_t Wd[4], Vd[4];
                    draw2_3(gt[g][0], gt[g][1], B1, h0c, l0c, p, Wd, Vd);
                    uint32_t b, eq;
                    cmp8_3<ZC>(c4, c8, c12, btab, Wd, Vd, b, eq);
                    const uint32_t lt = b & need;
                    const uint32_t und = eq & need;
                    const bool undecided = und != 0u;
                    const uint32_t ball = __ballot_sync(0xFFFFFFFFu, undecided);
                    const int slot = undecided ? wq + __popc(ball & lml) : S::QW + lane;
                    queue[slot] = make_uint4(A2s, und, lt, (uint32_t)ee);
                    const uint32_t f = (~need | lt) & (undecided ? 0u : vm);
                    if (have) store_site<L>(la, w ^ f, en.x >> 16);
                    acc += (uint32_t)__popc(f);
                    wq += __popc(ball);
                }
            };
            if (zc == 0) pass1(IC<0>{});
            else if (zc == 1) pass1(IC<1>{});
            else if (zc == 2) pass1(IC<2>{});
            else pass1(IC<3>{});
            // the warp's undecided sites, one per lane, from plane block 2 on
            __syncwarp();
            for (int e2 = lane; e2 < wq; e2 += 32) {
                const uint4 qe = queue[e2];
                const int g = (int)qe.w / H, q = (int)qe.w - g * H;
                const uint2 en = ct[q];
                uint32_t* la = lat + g * S::CELLS + (en.x & 0xFFFFu);
                const uint32_t vm = sVm[g];
                const uint32_t w = la[0];
                uint32_t ab[6];
                bond_partners<L, EA>(la, EA ? cj[q] : make_uint2(0u, 0u), ab);
                uint32_t need, c4, c8, c12;
                classes3_w(w, ab, vm, need, c4, c8, c12);
                uint32_t B1, h0c, l0c;
                {
                    uint32_t h1b, l1b;
                    mulhilo(PHILOX_M1, qe.x, h1b, l1b);
                    B1 = l1b;
                    mulhilo(PHILOX_M0, h1b ^ B1k, h0c, l0c);
                }
                uint32_t und = qe.y, lt = qe.z;
                finish3(c4, c8, c12, bpart[h & 1u], btab, sL0a[g], B1, h0c, l0c, p, und, lt);
                const uint32_t f = (~need | lt) & vm;
                store_site<L>(la, w ^ f, en.x >> 16);
                acc += (uint32_t)__popc(f);
            }
            __syncwarp();
            if (k == S::ITERS) break;
        }
        __syncthreads();
    }

    // measurement: unsatisfied bonds U and up-count per replica, write back
    for (int k = warp; k < G * (WP / 4); k += NW) {
        const int g = k / (WP / 4), c4 = k % (WP / 4);
        const uint32_t* lg = lat + g * S::CELLS;
        int32_t nup = 0;
        uint32_t out[4];
        uint32_t ucnt[4] = {0u, 0u, 0u, 0u};  // bit-sliced count of up to 12 bonds
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int b = 4 * c4 + m;
            out[m] = 0u;
            if (b < W) {  // warp-uniform
                const int s = 32 * b + lane;
                const bool in = s < N;
                uint32_t w = 0u, P0 = 0u, P1 = 0u, P2v = 0u;
                if (in) {
                    const int c = S::cell(s % L, (s / L) % L, s / (L * L));
                    w = lg[c];
                    P0 = w ^ lg[c + 1];
                    P1 = w ^ lg[c + P];
                    P2v = w ^ lg[c + P2];
                    if (EA) {
                        const uint32_t js = r.jbits[s];
                        P0 ^= 0u - (js & 1u);
                        P1 ^= 0u - ((js >> 1) & 1u);
                        P2v ^= 0u - ((js >> 2) & 1u);
                    }
                }
                const uint32_t tw = transpose32(w, lane);
                out[m] = tw;
                nup += __popc(tw);
                vc_add3(ucnt, P0, P1, P2v);
            }
        }
        const int32_t U = vc_total(ucnt, lane);
        const uint32_t slot = (gfirst + g) * 32u + lane;
        if (slot < R)
            reinterpret_cast<uint4*>(dst + (size_t)slot * r.Wp)[c4] =
                make_uint4(out[0], out[1], out[2], out[3]);
        atomicAdd(&sU[g][lane], U);
        atomicAdd(&sNup[g][lane], nup);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0 && acc) atomicAdd(&sAcc, (unsigned long long)acc);
    __syncthreads();

    for (int g = warp; g < G; g += NW) {
        const uint32_t slot = (gfirst + g) * 32u + lane;
        long long e = 0, e2 = 0, am = 0, m2 = 0;
        int lvmin = 0x7FFFFFFF, lvmax = -1;  // the warp's histogram levels
        if (slot < R) {
            const int32_t Uv = sU[g][lane];
            const int32_t E = 2 * Uv - 3 * N;
            const int32_t M = N - 2 * sNup[g][lane];
            r.E[i & 1][slot] = E;
            r.M[slot] = M;
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
        if (lane == 0 && (e | e2 | am | m2)) {
            TraceRow* tr = r.trace + i;
            atomicAdd(&tr->sumE, (unsigned long long)e);
            atomicAdd(&tr->sumE2, (unsigned long long)e2);
            atomicAdd(&tr->sumAbsM, (unsigned long long)am);
            atomicAdd(&tr->sumM2, (unsigned long long)m2);
        }
    }
    if (threadIdx.x == 0 && sAcc) atomicAdd(&r.trace[i].accepts, sAcc);
}

template <int L, bool EA, int GM>
size_t smem3d() {
    using S = Shape3<L, GM>;
    return (size_t)S::LAT_WORDS * 4 + (size_t)2 * S::H * 8 * (EA ? 2 : 1) +
           (size_t)(NT3 / 32) * (S::QW + 32) * 16;
}

template <int L, bool EA, int GM>
cudaError_t launch3d(const KParams& p, const uint32_t* cta2run, uint32_t ncta, cudaStream_t s,
                     bool attr_only) {
    static bool attr_set = false;
    const size_t sm = smem3d<L, EA, GM>();
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_sweep3d<L, EA, GM>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (attr_only || ncta == 0) return cudaSuccess;
    k_sweep3d<L, EA, GM><<<ncta, NT3, sm, s>>>(p, cta2run);
    return cudaGetLastError();
}

template <bool EA, int GM>
cudaError_t launch3d_L(int L, const KParams& p, const uint32_t* cta2run, uint32_t ncta,
                       cudaStream_t s, bool attr_only) {
    switch (L) {
        case 4: return launch3d<4, EA, GM>(p, cta2run, ncta, s, attr_only);
        case 6: return launch3d<6, EA, GM>(p, cta2run, ncta, s, attr_only);
        case 8: return launch3d<8, EA, GM>(p, cta2run, ncta, s, attr_only);
        case 10: return launch3d<10, EA, GM>(p, cta2run, ncta, s, attr_only);
        case 12: return launch3d<12, EA, GM>(p, cta2run, ncta, s, attr_only);
        case 14: return launch3d<14, EA, GM>(p, cta2run, ncta, s, attr_only);
        default: return launch3d<16, EA, GM>(p, cta2run, ncta, s, attr_only);
    }
}

template <int GM>
int groups_L(int L) {
    switch (L) {
        case 4: return Shape3<4, GM>::G;
        case 6: return Shape3<6, GM>::G;
        case 8: return Shape3<8, GM>::G;
        case 10: return Shape3<10, GM>::G;
        case 12: return Shape3<12, GM>::G;
        case 14: return Shape3<14, GM>::G;
        case 16: return Shape3<16, GM>::G;
        default: return 0;
    }
}

}  // namespace

// replica groups per CTA of the 3D kernel for side L with group multiple gm (1 or 2;
// 0: no 3D kernel for L)
int sweep3d_groups(int L, int gm) { return gm == 2 ? groups_L<2>(L) : groups_L<1>(L); }

// One launch of the 3D kernel over the CTAs of the runs of side L (cta2run: their
// run indices, device memory), with the context's group multiple.  attr_only:
// function attributes only (before a stream capture).
cudaError_t launch_sweep3d(const KParams& p, int L, const uint32_t* cta2run, uint32_t ncta,
                           cudaStream_t s, bool attr_only) {
    if (p.g3mul == 2)
        return p.ea ? launch3d_L<true, 2>(L, p, cta2run, ncta, s, attr_only)
                    : launch3d_L<false, 2>(L, p, cta2run, ncta, s, attr_only);
    return p.ea ? launch3d_L<true, 1>(L, p, cta2run, ncta, s, attr_only)
                : launch3d_L<false, 1>(L, p, cta2run, ncta, s, attr_only);
}

}  // namespace pa
