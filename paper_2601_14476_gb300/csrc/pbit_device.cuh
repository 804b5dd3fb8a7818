// Device helpers shared by the annealing kernels: the counter-based RNG and
// the variability p-bit decision (Eqs. 1 and 6 of arXiv 2601.14476).
#pragma once

#include <cstdint>

namespace pbit {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the 4x32
// S-box with multipliers 0xD2511F53 / 0xCD9E8D57 and key increments
// 0x9E3779B9 / 0xBB67AE85 between rounds.
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                        uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        // one 32x32->64 multiply gives both halves of each product
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0, n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        c0 = n0;
        c1 = (uint32_t)p1;
        c2 = n2;
        c3 = (uint32_t)p0;
    }
    return make_uint4(c0, c1, c2, c3);
}

// Two Philox4x32-10 blocks whose counters differ only in the last word,
// evaluated side by side (independent instruction streams for the scheduler).
// The counters of this library put the per-trial word last: (node, step,
// instance, block index within the node's trial groups).  The first round's
// two products and the second
// round's first product then do not depend on the trial, so a thread that
// draws for many trials of one node shares them (16 rather than 19 wide
// multiplies per block once inlined).
__device__ __forceinline__ void philox_pair(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3a, uint32_t c3b,
                                            uint32_t k0, uint32_t k1, uint4& ra, uint4& rb) {
    uint32_t a0 = c0, a1 = c1, a2 = c2, a3 = c3a, b0 = c0, b1 = c1, b2 = c2, b3 = c3b;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t pa0 = (uint64_t)0xD2511F53u * a0, pa1 = (uint64_t)0xCD9E8D57u * a2;
        const uint64_t pb0 = (uint64_t)0xD2511F53u * b0, pb1 = (uint64_t)0xCD9E8D57u * b2;
        const uint32_t na0 = (uint32_t)(pa1 >> 32) ^ a1 ^ k0, na2 = (uint32_t)(pa0 >> 32) ^ a3 ^ k1;
        const uint32_t nb0 = (uint32_t)(pb1 >> 32) ^ b1 ^ k0, nb2 = (uint32_t)(pb0 >> 32) ^ b3 ^ k1;
        a0 = na0;
        a1 = (uint32_t)pa1;
        a2 = na2;
        a3 = (uint32_t)pa0;
        b0 = nb0;
        b1 = (uint32_t)pb1;
        b2 = nb2;
        b3 = (uint32_t)pb0;
    }
    ra = make_uint4(a0, a1, a2, a3);
    rb = make_uint4(b0, b1, b2, b3);
}

// Philox4x32-10 split at the last counter word.  For counters (c0, c1, c2, c3)
// the first round's two products, and the second round's product of the
// first word, do not depend on c3; PhiloxHead keeps what the rest of the
// rounds need of them, so a thread drawing for many values of c3 (the blocks
// of one node's trial groups) computes them once and each block then costs 16 wide
// multiplies.  philox_tail(philox_head(c0, c1, c2, k), c3, k) equals
// philox(c0, c1, c2, c3, k).
struct PhiloxHead {
    uint32_t y1;   // round-1 output word 1
    uint32_t h2;   // round-1 output word 2 without the c3 term
    uint32_t z3;   // round-2 output word 3
    uint32_t hp1;  // high half of the round-3 product of word 2
    uint32_t w1;   // round-3 output word 1
};

__device__ __forceinline__ PhiloxHead philox_head(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t k0, uint32_t k1) {
    PhiloxHead h;
    // round 1 (keys k0, k1)
    const uint64_t a0 = (uint64_t)0xD2511F53u * c0, a1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t y0 = (uint32_t)(a1 >> 32) ^ c1 ^ k0;
    h.y1 = (uint32_t)a1;
    h.h2 = (uint32_t)(a0 >> 32) ^ k1;
    const uint32_t y3 = (uint32_t)a0;
    // round 2: the product of word 0 (keys + 1 increment)
    const uint64_t b0 = (uint64_t)0xD2511F53u * y0;
    const uint32_t z2 = (uint32_t)(b0 >> 32) ^ y3 ^ (k1 + 0xBB67AE85u);
    h.z3 = (uint32_t)b0;
    // round 3: the product of word 2
    const uint64_t c1p = (uint64_t)0xCD9E8D57u * z2;
    h.hp1 = (uint32_t)(c1p >> 32);
    h.w1 = (uint32_t)c1p;
    return h;
}

__device__ __forceinline__ uint4 philox_tail(const PhiloxHead& h, uint32_t c3, uint32_t k0, uint32_t k1) {
    // round 1, word 2; round 2, word 2 product
    const uint32_t y2 = h.h2 ^ c3;
    const uint64_t b1 = (uint64_t)0xCD9E8D57u * y2;
    const uint32_t z0 = (uint32_t)(b1 >> 32) ^ h.y1 ^ (k0 + 0x9E3779B9u);
    const uint32_t z1 = (uint32_t)b1;
    // round 3, word 0 product (keys + 2 increments)
    const uint64_t c0p = (uint64_t)0xD2511F53u * z0;
    uint32_t x0 = h.hp1 ^ z1 ^ (k0 + 2u * 0x9E3779B9u);
    uint32_t x1 = h.w1;
    uint32_t x2 = (uint32_t)(c0p >> 32) ^ h.z3 ^ (k1 + 2u * 0xBB67AE85u);
    uint32_t x3 = (uint32_t)c0p;
    k0 += 2u * 0x9E3779B9u;
    k1 += 2u * 0xBB67AE85u;
#pragma unroll
    for (int round = 3; round < 10; ++round) {
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
        const uint64_t p0 = (uint64_t)0xD2511F53u * x0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0, n2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        x0 = n0;
        x1 = (uint32_t)p1;
        x2 = n2;
        x3 = (uint32_t)p0;
    }
    return make_uint4(x0, x1, x2, x3);
}

// The random draws of one (node, step, instance) for its trials (the r of
// Eq. 6 and the timing draw u, both on 2^24-point grids).  Trials 8g .. 8g+7
// share three Philox blocks, B0, B1, B2, at last counter words 3g, 3g+1 and
// 3g+2, and all 384 of their bits are used: trial k of the group (k = t mod 8)
// takes word k mod 4 of block k / 4 as its r-word (r from the top 24 bits);
// its 24-bit u has half (k mod 2) of word k / 2 of B2 as its high 16 bits and
// the r-word's low byte as its low 8.  pbit_uword returns u in bits 8..31 of
// a word (bits 0..7 repeat the r-word's low byte), so that callers compare
// (word >> 8) for r and u alike.
__device__ __forceinline__ uint32_t pbit_uword(uint32_t wr, uint32_t w2, bool odd) {
    return __byte_perm(wr, w2, odd ? 0x7600u : 0x5400u);
}

__device__ __forceinline__ uint32_t pbit_word(const uint4& b, int c) {
    return c == 0 ? b.x : (c == 1 ? b.y : (c == 2 ? b.z : b.w));
}

// r- and u-words of the four trials t .. t+3 (t a multiple of 4): the block of
// their r-words (3g + h, h the half of the group) and B2.
__device__ __forceinline__ void pbit_draws4(uint32_t i, uint32_t step, uint32_t instance, uint32_t t, uint32_t k0,
                                            uint32_t k1, uint32_t (&wr)[4], uint32_t (&wu)[4]) {
    const uint32_t g3 = 3u * (t >> 3), h = (t >> 2) & 1u;
    uint4 a, b2;
    philox_pair(i, step, instance, g3 + h, g3 + 2u, k0, k1, a, b2);
    const uint32_t s0 = h ? b2.z : b2.x, s1 = h ? b2.w : b2.y;
    wr[0] = a.x;
    wr[1] = a.y;
    wr[2] = a.z;
    wr[3] = a.w;
    wu[0] = pbit_uword(a.x, s0, false);
    wu[1] = pbit_uword(a.y, s0, true);
    wu[2] = pbit_uword(a.z, s1, false);
    wu[3] = pbit_uword(a.w, s1, true);
}

// The same for the two trials t, t+1 (t even), as (r0, u0, r1, u1).
__device__ __forceinline__ uint4 pbit_draws2(uint32_t i, uint32_t step, uint32_t instance, uint32_t t, uint32_t k0,
                                             uint32_t k1) {
    const uint32_t g3 = 3u * (t >> 3), k = t & 7u;
    uint4 a, b2;
    philox_pair(i, step, instance, g3 + (k >> 2), g3 + 2u, k0, k1, a, b2);
    const uint32_t r0 = (k & 2u) ? a.z : a.x, r1 = (k & 2u) ? a.w : a.y;
    const uint32_t s = pbit_word(b2, (int)(k >> 1));
    return make_uint4(r0, pbit_uword(r0, s, false), r1, pbit_uword(r1, s, true));
}

// The same for one trial t.
__device__ __forceinline__ void pbit_draw1(uint32_t i, uint32_t step, uint32_t instance, uint32_t t, uint32_t k0,
                                           uint32_t k1, uint32_t& wr, uint32_t& wu) {
    const uint4 d = pbit_draws2(i, step, instance, t & ~1u, k0, k1);
    wr = (t & 1u) ? d.z : d.x;
    wu = (t & 1u) ? d.w : d.y;
}

// The r-word alone of trial t (the initial state needs only r).
__device__ __forceinline__ uint32_t pbit_rword(uint32_t i, uint32_t step, uint32_t instance, uint32_t t, uint32_t k0,
                                               uint32_t k1) {
    const uint4 b = philox(i, step, instance, 3u * (t >> 3) + ((t >> 2) & 1u), k0, k1);
    return pbit_word(b, (int)(t & 3u));
}

// The four trial pairs of the group starting at trial t (a multiple of 8) from
// the head of their (node, step, instance): pair q holds trials t + 2q and
// t + 2q + 1 as (r0, u0, r1, u1).
struct PbitPairs8 {
    uint4 p[4];
};

__device__ __forceinline__ PbitPairs8 pbit_pairs8(const PhiloxHead& h, uint32_t t, uint32_t k0, uint32_t k1) {
    const uint32_t g3 = 3u * (t >> 3);
    const uint4 b2 = philox_tail(h, g3 + 2u, k0, k1);
    const uint4 b0 = philox_tail(h, g3, k0, k1);
    const uint4 b1 = philox_tail(h, g3 + 1u, k0, k1);
    PbitPairs8 r;
    r.p[0] = make_uint4(b0.x, pbit_uword(b0.x, b2.x, false), b0.y, pbit_uword(b0.y, b2.x, true));
    r.p[1] = make_uint4(b0.z, pbit_uword(b0.z, b2.y, false), b0.w, pbit_uword(b0.w, b2.y, true));
    r.p[2] = make_uint4(b1.x, pbit_uword(b1.x, b2.z, false), b1.y, pbit_uword(b1.y, b2.z, true));
    r.p[3] = make_uint4(b1.z, pbit_uword(b1.z, b2.w, false), b1.w, pbit_uword(b1.w, b2.w, true));
    return r;
}

// The p-bit input x for an exact integer field D (three placements of the
// offset; see pbit_offset_mode).  Every operation is an explicitly rounded
// float32 operation, so the value does not depend on compiler contraction.
__device__ __forceinline__ float pbit_input(int mode, float I0, float lam, float del, int D) {
    const float d = (float)D;  // exact: |D| < 2^24
    if (mode == 1) return __fmul_rn(__fmul_rn(lam, I0), __fadd_rn(d, del));
    if (mode == 2) return __fmul_rn(lam, __fmaf_rn(I0, d, del));
    return __fmul_rn(I0, __fmaf_rn(lam, d, del));
}

// Decision threshold in the 24-bit r-word domain.  With k = word >> 8 and
// r_k = (2k+1-2^24)/2^24, "tanh(x) - r_k > 0" holds exactly for k < kthr,
// where kthr = (ceil(t*2^24) + 2^24) / 2 (floor) and t = tanh(x) in float32.
// Proof: 2k+1-2^24 is an integer, so it is < t*2^24 iff it is < ceil(t*2^24).
__device__ __forceinline__ uint32_t pbit_kthr(float t) {
    const int c = (int)ceilf(t * 16777216.0f);  // exact scaling by a power of two
    return (uint32_t)(c + (1 << 24)) >> 1;
}

// 2^a from the hardware approximation (ex2.approx.ftz.f32).  For the
// arguments pbit_kthr_of_x passes (|a| <= 57.71: no subnormal results) it
// returned exactly exp2f's value on every float32 tried on GB300.
__device__ __forceinline__ float pbit_exp2(float a) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a));
    return y;
}

// Decision threshold straight from x.  With t = tanh(x) = 1 - 2/(1 + e^(2x))
// and q = 2^25 / (1 + e^(2x)), t * 2^24 = 2^24 - q, so
// ceil(t * 2^24) = 2^24 - floor(q) and kthr = (2^25 - floor(q)) / 2 (floor).
// Evaluated in float32 with x clamped to [-20, 20] (tanh rounds to +-1 there)
// and e^(2x) = 2^(x * 2/ln 2); the threshold it gives corresponds to a tanh
// value within about 2e-7 of the exact one, well inside the 1e-6 band in
// which decisions may differ from the FP64 definition.
__device__ __forceinline__ uint32_t pbit_kthr_of_x(float x) {
    const float xc = fminf(fmaxf(x, -20.0f), 20.0f);
    const float e = pbit_exp2(xc * 2.8853900817779268f);
    const float q = __fdividef(33554432.0f, 1.0f + e);  // in [0, 2^25]
    return (33554432u - (uint32_t)q) >> 1;
}

// New state from the r-word, the u-word, the thresholds and the old state.
__device__ __forceinline__ int pbit_next(uint32_t wr, uint32_t wu, uint32_t kthr, uint32_t thr, int old) {
    const int cand = ((wr >> 8) < kthr) ? 1 : -1;
    return ((wu >> 8) < thr) ? cand : old;
}

}  // namespace pbit
