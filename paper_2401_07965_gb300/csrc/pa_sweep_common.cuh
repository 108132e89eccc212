// pa_sweep_common.cuh -- pieces shared by the sweep kernels: the 32x32 bit
// transpose, the per-half-sweep Philox table of the bit-plane uniforms and the
// rounds that depend on the site, and the plane comparisons.
#pragma once

#include "pa_internal.cuh"

namespace pa {

// three-input logic operation given by its truth table LUT = f(0xF0, 0xCC, 0xAA)
template <int LUT>
__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
    return d;
}

__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
    // lane i holds row i (bit c = element (i, c)); returns column `lane`
    const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int t = 0; t < 5; ++t) {
        const int j = 16 >> t;
        const uint32_t m0 = masks[t];
        uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
        x = (lane & j) ? ((x & ~m0) | ((y >> j) & m0)) : ((x & m0) | ((y << j) & ~m0));
    }
    return x;
}

// Bit-sliced counters for the measurement: plane j of the CB words holds bit j
// of one count per bit position (replica), so adding one-bit words costs a few
// logic operations and the per-replica sums need one transpose per plane
// instead of one per added word.
__host__ __device__ constexpr int vc_bits(int n) { return n > 0 ? 1 + vc_bits(n >> 1) : 0; }

// c += a + b (per bit position)
template <int CB>
__device__ __forceinline__ void vc_add2(uint32_t (&c)[CB], uint32_t a, uint32_t b) {
    uint32_t carry = lop3<0xE8>(c[0], a, b);  // majority: the carry of a full adder
    c[0] = lop3<0x96>(c[0], a, b);
#pragma unroll
    for (int j = 1; j < CB; ++j) {
        const uint32_t t = c[j] & carry;
        c[j] ^= carry;
        carry = t;
    }
}

// c += a + b + d (per bit position), CB >= 2
template <int CB>
__device__ __forceinline__ void vc_add3(uint32_t (&c)[CB], uint32_t a, uint32_t b, uint32_t d) {
    static_assert(CB >= 2, "vc_add3 needs two planes");
    const uint32_t sm = lop3<0x96>(a, b, d), k = lop3<0xE8>(a, b, d);  // a+b+d = sm + 2k
    const uint32_t k2 = c[0] & sm;                                      // c0+sm = (c0^sm) + 2k2
    c[0] ^= sm;
    uint32_t carry = lop3<0xE8>(c[1], k, k2);
    c[1] = lop3<0x96>(c[1], k, k2);
#pragma unroll
    for (int j = 2; j < CB; ++j) {
        const uint32_t t = c[j] & carry;
        c[j] ^= carry;
        carry = t;
    }
}

// lane r: the sum over the warp's lanes of their counts at bit position r
template <int CB>
__device__ __forceinline__ int32_t vc_total(const uint32_t (&c)[CB], int lane) {
    int32_t u = 0;
#pragma unroll
    for (int j = 0; j < CB; ++j) u += __popc(transpose32(c[j], lane)) << j;
    return u;
}

// ---------------------------------------------------------------------------
// Bit-plane uniforms.  The uniform u of replica r (slot base + r) at site s has
// bit 31 - p equal to bit r of plane word p, the lane p & 3 of the Philox draw
// with counter (base >> 5, (sweep << 4) | (colour << 3) | (p >> 2), step, s).
// u < thr is decided from the most significant plane down; a replica leaves
// the comparison at the first plane where u and thr differ, and the planes of
// a site stop once all 32 replicas are decided.
//
// Of the 10 Philox rounds, those parts that depend only on the CTA's replica
// group, the step, the sweep, the colour and the plane block g are the same
// for every thread of the CTA: they are computed once per half-sweep into a
// shared-memory table, together with the threshold bits (0 or 1) of each plane
// for each energy class.  The classes' replica masks are disjoint, so the
// per-replica threshold bit word of a plane, OR over classes of (mask & -bit),
// is the integer sum of mask x bit: multiply-adds on the multiply pipe rather
// than logic operations on the busier integer ALU pipe.  Per site, rounds 2 and 3 need one wide multiply
// each; per block of four planes, rounds 4-10 need 14.
// ---------------------------------------------------------------------------
struct PlaneTab {
    uint32_t c0k, c1, c2k, pad;  // round-3 outputs that do not depend on the site
    uint32_t B[4][4];            // B[m][k-1]: bit 31 - (4g + m) of thr[k] (0 or 1)
};

__device__ __forceinline__ void build_plane_tab(PlaneTab* tab, int g, const KParams& p,
                                                uint32_t grp, uint32_t step, uint32_t t,
                                                int colour, const uint32_t (&thr)[4]) {
    uint32_t h0a, l0a, h1a, l1a, h0b, l0b, h1c, l1c;
    mulhilo(PHILOX_M0, grp, h0a, l0a);
    mulhilo(PHILOX_M1, step, h1a, l1a);
    const uint32_t c1v = DOM_SWEEP | (t << 4) | ((uint32_t)colour << 3) | (uint32_t)g;
    const uint32_t A0 = h1a ^ c1v ^ p.rk0[0];
    const uint32_t A3 = l0a;
    mulhilo(PHILOX_M0, A0, h0b, l0b);
    const uint32_t B2 = h0b ^ A3 ^ p.rk1[1];
    const uint32_t B3 = l0b;
    mulhilo(PHILOX_M1, B2, h1c, l1c);
    PlaneTab e;
    e.c0k = h1c ^ p.rk0[2];
    e.c1 = l1c;
    e.c2k = B3 ^ p.rk1[2];
    e.pad = 0u;
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int k = 0; k < 4; ++k)
            e.B[m][k] = (thr[(k + 1) & 3] >> (31 - (4 * g + m))) & 1u;
    tab[g] = e;
}

// Site state of the plane comparison: the replicas still undecided, those
// already known to have u < thr, the per-site Philox values and the masks of
// the replicas in each energy class (cls[k-1]: dE = 4k).
template <int D>
struct SiteCmp {
    int s;
    uint32_t need, und, lt, B1, h0c, l0c;
    uint32_t cls[D];
};

// rounds 4-10 of the draw of plane block g (its four plane words)
template <int D>
__device__ __forceinline__ void block_draw(const SiteCmp<D>& c, const PlaneTab& e, const KParams& p,
                                           uint32_t (&W)[4]) {
    uint32_t x0 = e.c0k ^ c.B1, x1 = e.c1, x2 = c.h0c ^ e.c2k, x3 = c.l0c;
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
    W[0] = x0;
    W[1] = x1;
    W[2] = x2;
    W[3] = x3;
}

// two independent blocks, rounds interleaved for instruction-level parallelism
template <int D>
__device__ __forceinline__ void block_draw2(const SiteCmp<D>& c, const PlaneTab& e,
                                            const PlaneTab& f, const KParams& p,
                                            uint32_t (&W)[4], uint32_t (&V)[4]) {
    uint32_t x0 = e.c0k ^ c.B1, x1 = e.c1, x2 = c.h0c ^ e.c2k, x3 = c.l0c;
    uint32_t y0 = f.c0k ^ c.B1, y1 = f.c1, y2 = c.h0c ^ f.c2k, y3 = c.l0c;
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

// compare four planes: replicas leave at the first plane where u and thr differ
template <int D>
__device__ __forceinline__ void block_compare(SiteCmp<D>& c, const PlaneTab& e,
                                              const uint32_t (&W)[4]) {
    uint32_t und = c.und, lt = c.lt;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        // the classes' masks are disjoint: OR of the selected masks = their sum
        uint32_t tm = c.cls[0] * e.B[m][0];
#pragma unroll
        for (int a = 1; a < D; ++a) tm += c.cls[a] * e.B[m][a];
        lt |= lop3<0x40>(und, tm, W[m]);  // und & tm & ~W: u bit 0, thr bit 1: u < thr
        und = lop3<0x82>(W[m], tm, und);  // und & ~(W ^ tm): equal bits, still undecided
    }
    c.und = und;
    c.lt = lt;
}

// planes 0-7 (blocks 0 and 1) at once: for each replica, u's top 8 bits
// against thr's, by the borrow of the subtraction run from the least
// significant plane up, b' = (~u & t) | (~(u ^ t) & b): b ends as [u8 < t8],
// eq as [u8 == t8].  Replicas outside the classes see t = 0 and end with
// b = 0.  Same result as the plane-by-plane comparison from the top.
template <int D>
__device__ __forceinline__ void compare8(SiteCmp<D>& c, const PlaneTab& e, const PlaneTab& f,
                                         const uint32_t (&W)[4], const uint32_t (&V)[4]) {
    uint32_t b = 0u, eq = 0xFFFFFFFFu;
#pragma unroll
    for (int m = 3; m >= 0; --m) {
        uint32_t t = c.cls[0] * f.B[m][0];
#pragma unroll
        for (int a = 1; a < D; ++a) t += c.cls[a] * f.B[m][a];
        b = lop3<0x8E>(V[m], t, b);    // (~V & t) | (~(V ^ t) & b)
        eq = lop3<0x82>(V[m], t, eq);  // eq & ~(V ^ t)
    }
#pragma unroll
    for (int m = 3; m >= 0; --m) {
        uint32_t t = c.cls[0] * e.B[m][0];
#pragma unroll
        for (int a = 1; a < D; ++a) t += c.cls[a] * e.B[m][a];
        b = lop3<0x8E>(W[m], t, b);
        eq = lop3<0x82>(W[m], t, eq);
    }
    c.lt = b & c.need;
    c.und = eq & c.need;
}

template <int D>
__device__ __forceinline__ void plane_block(SiteCmp<D>& c, const PlaneTab& e, const KParams& p) {
    uint32_t W[4];
    block_draw<D>(c, e, p, W);
    block_compare<D>(c, e, W);
}

}  // namespace pa
