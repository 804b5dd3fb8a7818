// The per-tile sparse update shared by the one-step kernel and the batched
// persistent kernel: gather over CSR J of trial-major int8 spins, Philox
// draws, variability p-bit decision (Eqs. conv, pbits_variability).
#pragma once

#include <cstdint>

#include "pbit_device.cuh"
#include "pbit_internal.h"

namespace pbit {
namespace tile {

constexpr int kBlock = 256;

template <int G>
struct Pack {
    static constexpr int W = (G + 3) / 4;  // 32-bit words per group
};

template <int G>
__device__ __forceinline__ void load_group(const int8_t* p, uint32_t (&w)[Pack<G>::W]) {
    if constexpr (G == 32) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int4 v = *reinterpret_cast<const int4*>(p + 16 * q);
            w[4 * q] = (uint32_t)v.x;
            w[4 * q + 1] = (uint32_t)v.y;
            w[4 * q + 2] = (uint32_t)v.z;
            w[4 * q + 3] = (uint32_t)v.w;
        }
    } else if constexpr (G == 16) {
        const int4 v = *reinterpret_cast<const int4*>(p);
        w[0] = (uint32_t)v.x;
        w[1] = (uint32_t)v.y;
        w[2] = (uint32_t)v.z;
        w[3] = (uint32_t)v.w;
    } else if constexpr (G == 4) {
        w[0] = *reinterpret_cast<const uint32_t*>(p);
    } else {
        w[0] = (uint32_t)(uint8_t)(*p);
    }
}

template <int G>
__device__ __forceinline__ void store_group(int8_t* p, const uint32_t (&w)[Pack<G>::W]) {
    if constexpr (G == 32) {
#pragma unroll
        for (int q = 0; q < 2; ++q)
            *reinterpret_cast<int4*>(p + 16 * q) =
                make_int4((int)w[4 * q], (int)w[4 * q + 1], (int)w[4 * q + 2], (int)w[4 * q + 3]);
    } else if constexpr (G == 16) {
        *reinterpret_cast<int4*>(p) = make_int4((int)w[0], (int)w[1], (int)w[2], (int)w[3]);
    } else if constexpr (G == 4) {
        *reinterpret_cast<uint32_t*>(p) = w[0];
    } else {
        *p = (int8_t)(w[0] & 0xFF);
    }
}

__device__ __forceinline__ int sbyte(uint32_t w, int k) { return (int)(int8_t)(uint8_t)(w >> (8 * k)); }

// Exact field of node i for trials t0..t0+G-1 read from `in` (global or shared).
template <int G>
__device__ __forceinline__ void gather_field(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                             const int8_t* __restrict__ J, const int8_t* in, int32_t T, int i,
                                             int t0, int (&acc)[G]) {
#pragma unroll
    for (int k = 0; k < G; ++k) acc[k] = 0;
    const int rb = __ldg(row_ptr + i), re = __ldg(row_ptr + i + 1);
    for (int e = rb; e < re; ++e) {
        const int j = __ldg(col + e);
        const int w = __ldg(J + e);
        uint32_t v[Pack<G>::W];
        load_group<G>(in + (size_t)j * T + t0, v);
#pragma unroll
        for (int k = 0; k < G; ++k) acc[k] += w * sbyte(v[k >> 2], k & 3);
    }
}

// Decisions for one group of G trials of node i at `step` (Eq. 6 p-bit with
// timing draw), from exact fields acc (without h) and old state words.
template <int G>
__device__ __forceinline__ void decide_group(const StepArgs& a, int i, int t0, const int (&acc)[G],
                                             const uint32_t (&oldw)[Pack<G>::W], uint32_t (&neww)[Pack<G>::W]) {
    const float I0 = __ldg(a.i0_table + a.step);
    const float lam = a.par.lambda ? __ldg(a.par.lambda + i) : 1.0f;
    const float del = a.par.delta ? __ldg(a.par.delta + i) : 0.0f;
    const uint32_t thr = a.par.thr ? __ldg(a.par.thr + i) : (1u << 24);
    const int hi = a.h ? __ldg(a.h + i) : 0;
#pragma unroll
    for (int k = 0; k < Pack<G>::W; ++k) neww[k] = 0;
    static_assert(G == 1 || G % 4 == 0, "trial groups of 1 or a multiple of 4");
    if constexpr (G == 1) {
        uint32_t wr, wu;
        pbit_draw1((uint32_t)i, (uint32_t)a.step, a.instance, (uint32_t)t0, a.seed_lo, a.seed_hi, wr, wu);
        const uint32_t kthr = pbit_kthr_of_x(pbit_input(a.offset_mode, I0, lam, del, hi + acc[0]));
        const int s = pbit_next(wr, wu, kthr, thr, sbyte(oldw[0], 0));
        neww[0] = (uint32_t)(uint8_t)(int8_t)s;
    } else {
#pragma unroll
        for (int k = 0; k < G; k += 4) {
            uint32_t wr[4], wu[4];
            pbit_draws4((uint32_t)i, (uint32_t)a.step, a.instance, (uint32_t)(t0 + k), a.seed_lo, a.seed_hi, wr, wu);
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const uint32_t kt = pbit_kthr_of_x(pbit_input(a.offset_mode, I0, lam, del, hi + acc[k + b]));
                const int s = pbit_next(wr[b], wu[b], kt, thr, sbyte(oldw[k >> 2], b));
                neww[k >> 2] |= ((uint32_t)(uint8_t)(int8_t)s) << (8 * b);
            }
        }
    }
}

// ------------------------------------------------------------------ step ----
// One thread per (node i, group of G trials); 256-thread blocks cover a
// contiguous range of nodes.
//
// UNIT (every |J| = 1, degree <= 127): the gather counts, per trial byte,
// the neighbours whose product J_ij * s_j is -1.  A spin byte is 0x01 (+1)
// or 0xFF (-1), so (byte & 2) is 2 exactly for -1; XOR with 2 when J = -1
// flips it.  Byte lanes of one 32-bit word add without carries (2 * 127 <
// 256), and sum_j J_ij s_j = deg - 2 * count.
//
// TABLE: the field of node i lies in h_i + [-W_i, W_i] with the parity of
// W_i (W_i = sum_j |J_ij|), so for this step the block first evaluates the
// decision threshold for each of the W_i + 1 possible fields of its nodes
// into shared memory; each update then reads its threshold by index
// (D - h_i + W_i) / 2.  The table entries are computed by the same function
// as the direct path, so both give identical decisions.
constexpr int kTabMax = 4096;  // threshold entries per block (16 KB)

// Byte helpers for the sign-test decisions (see the warp-table tile below).
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}
// byte k of w, zero-extended
__device__ __forceinline__ uint32_t byte_of(uint32_t w, int k) { return prmt(w, 0u, 0x4440u | (uint32_t)k); }
// byte k = 0xFF where v_k < 0 (as int32), else 0x00
__device__ __forceinline__ uint32_t sign_bytes(uint32_t v0, uint32_t v1, uint32_t v2, uint32_t v3) {
    const uint32_t lo = prmt(v0, v1, 0x00FBu);  // bytes 0, 1: sign of v0, v1
    const uint32_t hi = prmt(v2, v3, 0xFB00u);  // bytes 2, 3: sign of v2, v3
    return prmt(lo, hi, 0x7610u);
}

// One warp's 32 consecutive items: this lane's item is `tid` (tid % 32 == lane).
// One tile = kBlock consecutive (node, trial-group) items starting at item
// `first`, processed by the kBlock threads of the calling block.  s_tab is
// shared memory of kTabMax entries (TABLE only).  Every thread of the block
// must call this (the table build has a block barrier).
// item -> node: the host-computed multiply-shift when the launcher set one (items below 2^31),
// else 64-bit division
__device__ __forceinline__ int node_of_item(const StepArgs& a, int64_t item, int groups) {
    if (a.grp_m != 0ull) return (int)(((unsigned long long)item * a.grp_m) >> a.grp_s);
    return (int)(item / groups);
}

template <int G, bool UNIT, bool TABLE>
__device__ __forceinline__ void process_tile(const StepArgs& a, int64_t first, uint32_t* s_tab) {
    const int groups = a.T / G;
    const int64_t total = (int64_t)a.n * groups;
    const int64_t tid = first + threadIdx.x;
    const float I0 = __ldg(a.i0_table + a.step);
    int tab_base = 0;
    if constexpr (TABLE) {
        // W_i + 1 entries per node of the tile: with few nodes (many trials per node) warp w fills
        // nodes i_first + w, i_first + w + 8, ... lane by lane; with many nodes each thread fills one
        const int i_first = node_of_item(a, first, groups);
        const int i_last = node_of_item(a, min(total - 1, first + kBlock - 1), groups);
        tab_base = __ldg(a.tab_off + i_first);
        const bool by_warp = i_last - i_first < 8;
        const int lanes = by_warp ? 32 : 1;
        const int sub = by_warp ? (int)(threadIdx.x & 31) : 0;
        const int stride = by_warp ? kBlock / 32 : kBlock;
        for (int node = i_first + (by_warp ? (int)(threadIdx.x >> 5) : (int)threadIdx.x); node <= i_last;
             node += stride) {
            const int off = __ldg(a.tab_off + node) - tab_base;
            const int W = __ldg(a.wabs + node);
            const int hi_n = a.h ? __ldg(a.h + node) : 0;
            const float lam = a.par.lambda ? __ldg(a.par.lambda + node) : 1.0f;
            const float del = a.par.delta ? __ldg(a.par.delta + node) : 0.0f;
            for (int idx = sub; idx <= W; idx += lanes)
                s_tab[off + idx] = pbit_kthr_of_x(pbit_input(a.offset_mode, I0, lam, del, hi_n - W + 2 * idx));
        }
        __syncthreads();
    }
    if (tid >= total) return;
    const int i = node_of_item(a, tid, groups);
    const int t0 = (int)(tid - (int64_t)i * groups) * G;
    const int hi = a.h ? __ldg(a.h + i) : 0;
    const float lam = a.par.lambda ? __ldg(a.par.lambda + i) : 1.0f;
    const float del = a.par.delta ? __ldg(a.par.delta + i) : 0.0f;
    const uint32_t thr = a.par.thr ? __ldg(a.par.thr + i) : (1u << 24);
    const int rb = __ldg(a.row_ptr + i), re = __ldg(a.row_ptr + i + 1);
    constexpr int NW = Pack<G>::W;
    const int deg = re - rb;

    // UNIT: packed counts c2 = 2 * #(J_ij s_j = -1) per trial byte, field = h + deg - c2;
    // otherwise exact fields acc (without h)
    uint32_t cnt2[UNIT && G >= 4 ? NW : 1];
    int acc[UNIT && G >= 4 ? 1 : G];
    if constexpr (UNIT && G >= 4) {
#pragma unroll
        for (int w = 0; w < NW; ++w) cnt2[w] = 0;
        for (int e = rb; e < re; ++e) {
            const int j = __ldg(a.col + e);
            const uint32_t flip = __ldg(a.J + e) < 0 ? 0x02020202u : 0u;
            uint32_t v[NW];
            load_group<G>(a.in + (size_t)j * a.T + t0, v);
#pragma unroll
            for (int w = 0; w < NW; ++w) cnt2[w] += (v[w] & 0x02020202u) ^ flip;
        }
    } else {
        gather_field<G>(a.row_ptr, a.col, a.J, a.in, a.T, i, t0, acc);
    }
    // table row of node i; for UNIT the entry of count c2 is row[W_i - c2 / 2] (W_i = deg)
    const uint32_t* row = nullptr;
    int W_i = 0;
    if constexpr (TABLE) {
        row = s_tab + (__ldg(a.tab_off + i) - tab_base);
        W_i = __ldg(a.wabs + i);
    }
    auto kthr_at = [&](int k) -> uint32_t {
        if constexpr (UNIT && G >= 4) {
            const int c2 = (int)byte_of(cnt2[k >> 2], k & 3);
            if constexpr (TABLE) return row[W_i - (c2 >> 1)];
            else return pbit_kthr_of_x(pbit_input(a.offset_mode, I0, lam, del, hi + deg - c2));
        } else {
            if constexpr (TABLE) return row[(acc[k] + W_i) >> 1];
            else return pbit_kthr_of_x(pbit_input(a.offset_mode, I0, lam, del, hi + acc[k]));
        }
    };
    uint32_t oldw[NW], neww[NW];
    load_group<G>(a.in + (size_t)i * a.T + t0, oldw);
    if constexpr (G == 1) {
        uint32_t wr, wu;
        pbit_draw1((uint32_t)i, (uint32_t)a.step, a.instance, (uint32_t)t0, a.seed_lo, a.seed_hi, wr, wu);
        const int s = pbit_next(wr, wu, kthr_at(0), thr, sbyte(oldw[0], 0));
        neww[0] = (uint32_t)(uint8_t)(int8_t)s;
    } else {
        // sign tests and byte masks as in the warp-table tile
        const auto decide_word = [&](int w, const uint32_t (&wr)[4], const uint32_t (&wu)[4]) {
            uint32_t dr[4], du[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                dr[b] = (wr[b] >> 8) - kthr_at(4 * w + b);
                du[b] = (wu[b] >> 8) - thr;
            }
            const uint32_t S = sign_bytes(dr[0], dr[1], dr[2], dr[3]);
            const uint32_t U = sign_bytes(du[0], du[1], du[2], du[3]);
            neww[w] = ((U & ~S) | (~U & oldw[w])) | 0x01010101u;
        };
        if constexpr (G == 4) {
            uint32_t wr[4], wu[4];
            pbit_draws4((uint32_t)i, (uint32_t)a.step, a.instance, (uint32_t)t0, a.seed_lo, a.seed_hi, wr, wu);
            decide_word(0, wr, wu);
        } else {
            // whole groups of 8 trials: three Philox blocks per group
            const PhiloxHead ph = philox_head((uint32_t)i, (uint32_t)a.step, a.instance, a.seed_lo, a.seed_hi);
#pragma unroll
            for (int gq = 0; gq < NW / 2; ++gq) {
                const PbitPairs8 d = pbit_pairs8(ph, (uint32_t)(t0 + 8 * gq), a.seed_lo, a.seed_hi);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint4 p0 = d.p[2 * h], p1 = d.p[2 * h + 1];
                    const uint32_t wr[4] = {p0.x, p0.z, p1.x, p1.z}, wu[4] = {p0.y, p0.w, p1.y, p1.w};
                    decide_word(2 * gq + h, wr, wu);
                }
            }
        }
    }
    store_group<G>(a.out + (size_t)i * a.T + t0, neww);
}



// ------------------------------------------------------------ warp table ----
// Unit weights (every |J| = 1) and small degree: the threshold table of a
// node lives in registers of the warp lanes that update it.  A warp covers
// either part of one node's trials (T / G >= 32 groups per node) or several
// whole nodes (T / G divides 32), so each node owns a segment of L lanes,
// L = min(32, T / G).  The update with packed count c2 = 2 * #(J_ij s_j = -1)
// (field h_i + deg_i - c2) reads its threshold with one shuffle from its
// segment.  HALF: lane seg + c holds the negated threshold for the field
// h_i + deg_i - 2c (c = 0..deg_i, needing deg_i + 1 <= L: the field of a node
// with unit weights has the parity of its degree) and the lookup index is
// c2 / 2; otherwise lane seg + c holds the field h_i + deg_i - c (needing
// 2 deg_i + 1 <= L) and the index is c2 itself, which saves the halving.
// No shared memory, no block barrier.
//
// Decisions without branches or multiplies: (w >> 8) - kthr is negative
// exactly when the p-bit draw picks +1 (both sides below 2^25), and
// (u >> 8) - thr when the node updates; the sign bits of four trials are
// turned into byte masks with prmt's sign-replicating selectors, and
//   new = U ? (S ? 0x01 : 0xFF) : old = ((U & ~S) | (~U & old)) | 0x01
// per byte (every spin byte is 0x01 or 0xFF, so bit 0 is always set).
template <int G, bool HALF>
__device__ __forceinline__ void process_warp_items(const StepArgs& a, uint32_t tid) {
    static_assert(G == 16 || G == 32, "warp-table tile needs 4-word trial groups");
    constexpr int NW = Pack<G>::W;
    const uint32_t groups = (uint32_t)a.T / G;
    const uint32_t total = (uint32_t)a.n * groups;
    const bool live = tid < total;
    const uint32_t item = live ? tid : total - 1;  // dead lanes still feed the shuffles
    const int i = (int)(((unsigned long long)item * a.grp_m) >> a.grp_s);
    const int t0 = (int)(item - (uint32_t)i * groups) * G;
    const int lane = (int)(tid & 31u);
    const int L = groups >= 32u ? 32 : (int)groups;  // a power of two: T / G divides 32 or is a multiple
    const int ell = lane & (L - 1);
    const float I0 = __ldg(a.i0_table + a.step);
    const int hi = a.h ? __ldg(a.h + i) : 0;
    const float lam = a.par.lambda ? __ldg(a.par.lambda + i) : 1.0f;
    const float del = a.par.delta ? __ldg(a.par.delta + i) : 0.0f;
    const uint32_t thr = a.par.thr ? __ldg(a.par.thr + i) : (1u << 24);
    const int rb = __ldg(a.row_ptr + i), re = __ldg(a.row_ptr + i + 1);
    const int deg = re - rb;
    const uint32_t negk_lane = 0u - pbit_kthr_of_x(pbit_input(a.offset_mode, I0, lam, del, hi + deg - (HALF ? 2 * ell : ell)));
    uint32_t cnt2[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) cnt2[w] = 0;
    // two neighbours per iteration: both loads in flight, one three-input add per word
    int e = rb;
    for (; e + 1 < re; e += 2) {
        const int j0 = __ldg(a.col + e), j1 = __ldg(a.col + e + 1);
        const uint32_t f0 = __ldg(a.J + e) < 0 ? 0x02020202u : 0u, f1 = __ldg(a.J + e + 1) < 0 ? 0x02020202u : 0u;
        uint32_t v0[NW], v1[NW];
        load_group<G>(a.in + (size_t)j0 * a.T + t0, v0);
        load_group<G>(a.in + (size_t)j1 * a.T + t0, v1);
#pragma unroll
        for (int w = 0; w < NW; ++w) cnt2[w] += ((v0[w] & 0x02020202u) ^ f0) + ((v1[w] & 0x02020202u) ^ f1);
    }
    if (e < re) {
        const int j = __ldg(a.col + e);
        const uint32_t flip = __ldg(a.J + e) < 0 ? 0x02020202u : 0u;
        uint32_t v[NW];
        load_group<G>(a.in + (size_t)j * a.T + t0, v);
#pragma unroll
        for (int w = 0; w < NW; ++w) cnt2[w] += (v[w] & 0x02020202u) ^ flip;
    }
    uint32_t oldw[NW], neww[NW];
    load_group<G>(a.in + (size_t)i * a.T + t0, oldw);
    const PhiloxHead ph = philox_head((uint32_t)i, (uint32_t)a.step, a.instance, a.seed_lo, a.seed_hi);
#pragma unroll
    for (int gq = 0; gq < NW / 2; ++gq) {
        // one group of 8 trials (two words) from three Philox blocks
        const PbitPairs8 d = pbit_pairs8(ph, (uint32_t)(t0 + 8 * gq), a.seed_lo, a.seed_hi);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int w = 2 * gq + h;
            const uint4 p0 = d.p[2 * h], p1 = d.p[2 * h + 1];
            const uint32_t cnt = HALF ? cnt2[w] >> 1 : cnt2[w];  // bytes of cnt2 are even: halving keeps them apart
            // the shuffle width L keeps the source lane inside this node's segment
            uint32_t q[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) q[b] = __shfl_sync(0xFFFFFFFFu, negk_lane, (int)byte_of(cnt, b), L);
            const uint32_t S = sign_bytes((p0.x >> 8) + q[0], (p0.z >> 8) + q[1], (p1.x >> 8) + q[2], (p1.z >> 8) + q[3]);
            const uint32_t U = sign_bytes((p0.y >> 8) - thr, (p0.w >> 8) - thr, (p1.y >> 8) - thr, (p1.w >> 8) - thr);
            neww[w] = ((U & ~S) | (~U & oldw[w])) | 0x01010101u;
        }
    }
    if (live) store_group<G>(a.out + (size_t)i * a.T + t0, neww);
}

template <int G, bool HALF>
__device__ __forceinline__ void process_tile_warp(const StepArgs& a, uint32_t first) {
    process_warp_items<G, HALF>(a, first + threadIdx.x);  // first is a multiple of the block size
}

// The pSA variants of the Methods section (Eq. SpSA, Eq. TApSA) and the
// paper's period timing model, one tile as above (no threshold table: the
// input depends on per-trial state, not on the field alone).
//   timing: node i updates at sub-step q = a.step only when q % nu_i == 0;
//           idle nodes copy their spins and leave their state untouched;
//           I0 = table[q / t_res].
//   SpSA:   stall draw = word (t % 4) of Philox(node, q, t / 4, instance ^ 2^31);
//           stalled: I = Iprev, else I = I0 * D; Iprev <- I.
//   TApSA:  ring[q % window] <- D; I = I0 * (sum of the ring) / window.
//   x:      SCALED lambda I + I0 delta, LISTING lambda (I + I0 delta),
//           EQUATION lambda (I + delta).
__device__ __forceinline__ float variant_x(int mode, float I0, float lam, float del, float I) {
    if (mode == 1) return __fmul_rn(lam, __fmaf_rn(I0, del, I));
    if (mode == 2) return __fmul_rn(lam, __fadd_rn(I, del));
    return __fmaf_rn(lam, I, __fmul_rn(I0, del));
}

template <int G, bool UNIT>
__device__ __forceinline__ void process_tile_variant(const StepArgs& a, int64_t first) {
    const int groups = a.T / G;
    const int64_t total = (int64_t)a.n * groups;
    const int64_t tid = first + threadIdx.x;
    if (tid >= total) return;
    const int i = (int)(tid / groups);
    const int t0 = (int)(tid - (int64_t)i * groups) * G;
    const uint32_t q = (uint32_t)a.step;
    uint32_t oldw[Pack<G>::W];
    load_group<G>(a.in + (size_t)i * a.T + t0, oldw);
    if (a.t_res > 0 && (q % (uint32_t)__ldg(a.nu + i)) != 0u) {
        store_group<G>(a.out + (size_t)i * a.T + t0, oldw);
        return;
    }
    const float I0 = __ldg(a.i0_table + (a.t_res > 0 ? q / (uint32_t)a.t_res : q));
    const int hi = a.h ? __ldg(a.h + i) : 0;
    const float lam = a.par.lambda ? __ldg(a.par.lambda + i) : 1.0f;
    const float del = a.par.delta ? __ldg(a.par.delta + i) : 0.0f;
    const uint32_t thr = a.par.thr ? __ldg(a.par.thr + i) : (1u << 24);
    const int rb = __ldg(a.row_ptr + i), re = __ldg(a.row_ptr + i + 1);
    int D[G];
    if constexpr (UNIT && G >= 4) {
        uint32_t cnt2[Pack<G>::W];
#pragma unroll
        for (int w = 0; w < Pack<G>::W; ++w) cnt2[w] = 0;
        for (int e = rb; e < re; ++e) {
            const int j = __ldg(a.col + e);
            const uint32_t flip = __ldg(a.J + e) < 0 ? 0x02020202u : 0u;
            uint32_t v[Pack<G>::W];
            load_group<G>(a.in + (size_t)j * a.T + t0, v);
#pragma unroll
            for (int w = 0; w < Pack<G>::W; ++w) cnt2[w] += (v[w] & 0x02020202u) ^ flip;
        }
        const int deg = re - rb;
#pragma unroll
        for (int k = 0; k < G; ++k) D[k] = hi + deg - (int)((cnt2[k >> 2] >> (8 * (k & 3))) & 0xFFu);
    } else {
        int acc[G];
        gather_field<G>(a.row_ptr, a.col, a.J, a.in, a.T, i, t0, acc);
#pragma unroll
        for (int k = 0; k < G; ++k) D[k] = hi + acc[k];
    }
    float I[G];
    const size_t base = (size_t)i * a.T + t0;
    if (a.alg == 1) {
        uint4 sw = make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const int t = t0 + k;
            if (k == 0 || (t & 3) == 0)
                sw = philox((uint32_t)i, q, a.instance ^ 0x80000000u, (uint32_t)t >> 2, a.seed_lo, a.seed_hi);
            const uint32_t word = (t & 3) == 0 ? sw.x : ((t & 3) == 1 ? sw.y : ((t & 3) == 2 ? sw.z : sw.w));
            const bool stall = (word >> 8) < a.stall_thr;
            I[k] = stall ? a.Iprev[base + k] : __fmul_rn(I0, (float)D[k]);
            a.Iprev[base + k] = I[k];
        }
    } else if (a.alg == 2) {
        const size_t plane = (size_t)a.n * a.T;
        const int slot = (int)(q % (uint32_t)a.window);
#pragma unroll
        for (int k = 0; k < G; ++k) {
            a.ring[(size_t)slot * plane + base + k] = (int16_t)D[k];
            int sum = 0;
            for (int w = 0; w < a.window; ++w) sum += a.ring[(size_t)w * plane + base + k];
            I[k] = __fmul_rn(I0, __fdiv_rn((float)sum, (float)a.window));
        }
    } else {
#pragma unroll
        for (int k = 0; k < G; ++k) I[k] = __fmul_rn(I0, (float)D[k]);
    }
    uint32_t neww[Pack<G>::W];
#pragma unroll
    for (int w = 0; w < Pack<G>::W; ++w) neww[w] = 0;
    static_assert(G == 1 || G % 4 == 0, "trial groups of 1 or a multiple of 4");
    if constexpr (G == 1) {
        uint32_t wr, wu;
        pbit_draw1((uint32_t)i, q, a.instance, (uint32_t)t0, a.seed_lo, a.seed_hi, wr, wu);
        const uint32_t kthr = pbit_kthr_of_x(variant_x(a.offset_mode, I0, lam, del, I[0]));
        const int s = pbit_next(wr, wu, kthr, thr, sbyte(oldw[0], 0));
        neww[0] = (uint32_t)(uint8_t)(int8_t)s;
    } else {
#pragma unroll
        for (int k = 0; k < G; k += 4) {
            uint32_t wr[4], wu[4];
            pbit_draws4((uint32_t)i, q, a.instance, (uint32_t)(t0 + k), a.seed_lo, a.seed_hi, wr, wu);
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const uint32_t kt = pbit_kthr_of_x(variant_x(a.offset_mode, I0, lam, del, I[k + b]));
                const int s = pbit_next(wr[b], wu[b], kt, thr, sbyte(oldw[k >> 2], b));
                neww[k >> 2] |= ((uint32_t)(uint8_t)(int8_t)s) << (8 * b);
            }
        }
    }
    store_group<G>(a.out + (size_t)i * a.T + t0, neww);
}


// The variants' coalesced word tile, the work of one warp (shared by the one-step variant kernel and the
// batched chunk kernel): node i, trials tb + 128 k of the word span (tb = span start + 4 lane), its
// spins read from `src` and written to `dst`, neighbour e's spins read from nbr(e); I0, the node's
// parameters and its CSR row [rb, re) already loaded.  Every lane of the warp works on node i (the
// threshold table below is shuffled across the warp).
__device__ __forceinline__ uint32_t wld32(const int8_t* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ void wst32(int8_t* p, uint32_t v) { *reinterpret_cast<uint32_t*>(p) = v; }

template <int NW, bool UNIT, int WIN, typename Nbr>
__device__ __forceinline__ void variant_words(const StepArgs& a, int i, int tb, float I0, int hi, float lam, float del,
                                              uint32_t thr, int rb, int re, const int8_t* src, int8_t* dst, Nbr nbr,
                                              int lane) {
    const int T = a.T;
    const uint32_t q = (uint32_t)a.step;
    const size_t row = (size_t)i * T;
    // the carried state first, so that its loads are in flight during the gather:
    // SpSA the last inputs, TApSA the sum of the ring slots other than q % window
    const size_t plane = (size_t)a.n * T;
    const int slot = a.alg == 2 ? (int)(q % (uint32_t)a.window) : 0;
    float4 prev[NW];
    int osum[4 * NW];
#pragma unroll
    for (int k = 0; k < 4 * NW; ++k) osum[k] = 0;
    if (a.alg == 1) {
#pragma unroll
        for (int k = 0; k < NW; ++k) prev[k] = *reinterpret_cast<const float4*>(a.Iprev + row + tb + 128 * k);
    } else if (a.alg == 2) {
        const auto add_slot = [&](int w) {
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                const uint2 v = *reinterpret_cast<const uint2*>(a.ring + (size_t)w * plane + row + tb + 128 * k);
                osum[4 * k] += (int)(int16_t)(v.x & 0xFFFFu);
                osum[4 * k + 1] += (int)(int16_t)(v.x >> 16);
                osum[4 * k + 2] += (int)(int16_t)(v.y & 0xFFFFu);
                osum[4 * k + 3] += (int)(int16_t)(v.y >> 16);
            }
        };
        if constexpr (WIN > 0) {
#pragma unroll
            for (int u = 1; u < WIN; ++u) add_slot(slot + u < WIN ? slot + u : slot + u - WIN);
        } else {
            for (int u = 1; u < a.window; ++u) add_slot(slot + u < a.window ? slot + u : slot + u - a.window);
        }
    }
    // exact fields D = h_i + sum_j J_ij s_j (Eq. 1)
    int D[4 * NW];
    uint32_t cnt2[NW];  // +-1 weights: per trial byte, 2 per neighbour with J_ij s_j = -1
    if constexpr (UNIT) {
        // bit 1 of the spin byte is set for -1; flipped for J = -1
#pragma unroll
        for (int k = 0; k < NW; ++k) cnt2[k] = 0;
        for (int e = rb; e < re; ++e) {
            const int8_t* pj = nbr(e) + (size_t)__ldg(a.col + e) * T + tb;
            const uint32_t flip = __ldg(a.J + e) < 0 ? 0x02020202u : 0u;
#pragma unroll
            for (int k = 0; k < NW; ++k) cnt2[k] += (wld32(pj + 128 * k) & 0x02020202u) ^ flip;
        }
        const int base = hi + (re - rb);
#pragma unroll
        for (int k = 0; k < NW; ++k)
#pragma unroll
            for (int b = 0; b < 4; ++b) D[4 * k + b] = base - (int)((cnt2[k] >> (8 * b)) & 0xFFu);
    } else {
#pragma unroll
        for (int k = 0; k < 4 * NW; ++k) D[k] = hi;
        for (int e = rb; e < re; ++e) {
            const int8_t* pj = nbr(e) + (size_t)__ldg(a.col + e) * T + tb;
            const int w = __ldg(a.J + e);
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                const uint32_t v = wld32(pj + 128 * k);
#pragma unroll
                for (int b = 0; b < 4; ++b) D[4 * k + b] += w * sbyte(v, b);
            }
        }
    }
    // pSA under the timing model with +-1 weights and degree <= 15: the input depends on the count
    // alone, so lane c (every lane of the warp has node i) computes the threshold of count c once and
    // each trial reads its own with a shuffle; the same float operations as the per-trial form
    bool table = false;
    uint32_t negk_lane = 0;
    if constexpr (UNIT) {
        if (a.alg == 0 && 2 * (re - rb) + 1 <= 32) {
            table = true;
            const float Ic = __fmul_rn(I0, (float)(hi + (re - rb) - lane));  // counts above 2 deg are never read
            negk_lane = 0u - pbit_kthr_of_x(variant_x(a.offset_mode, I0, lam, del, Ic));
        }
    }
#pragma unroll
    for (int k = 0; k < NW; ++k) {
        const int t = tb + 128 * k;
        const size_t cell = row + t;
        float I[4];
        if (a.alg == 1) {
            // SpSA: stall draw of trial t + b = word b of Philox(node, q, t / 4, instance ^ 2^31)
            const uint4 sw = philox((uint32_t)i, q, a.instance ^ 0x80000000u, (uint32_t)t >> 2, a.seed_lo, a.seed_hi);
            I[0] = (sw.x >> 8) < a.stall_thr ? prev[k].x : __fmul_rn(I0, (float)D[4 * k]);
            I[1] = (sw.y >> 8) < a.stall_thr ? prev[k].y : __fmul_rn(I0, (float)D[4 * k + 1]);
            I[2] = (sw.z >> 8) < a.stall_thr ? prev[k].z : __fmul_rn(I0, (float)D[4 * k + 2]);
            I[3] = (sw.w >> 8) < a.stall_thr ? prev[k].w : __fmul_rn(I0, (float)D[4 * k + 3]);
            *reinterpret_cast<float4*>(a.Iprev + cell) = make_float4(I[0], I[1], I[2], I[3]);
        } else if (a.alg == 2) {
            // TApSA: ring slot q % window <- D (int16); I = I0 * (sum of the ring) / window
            int16_t d16[4];
            int sum[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                d16[b] = (int16_t)D[4 * k + b];
                sum[b] = osum[4 * k + b] + d16[b];
            }
            *reinterpret_cast<uint2*>(a.ring + (size_t)slot * plane + cell) =
                make_uint2((uint32_t)(uint16_t)d16[0] | ((uint32_t)(uint16_t)d16[1] << 16),
                           (uint32_t)(uint16_t)d16[2] | ((uint32_t)(uint16_t)d16[3] << 16));
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                // sum / window: for the paper's window of 4 a multiply by 0.25, exact like the division
                const float mean = WIN == 4 ? __fmul_rn((float)sum[b], 0.25f) : __fdiv_rn((float)sum[b], (float)a.window);
                I[b] = __fmul_rn(I0, mean);
            }
        } else {
#pragma unroll
            for (int b = 0; b < 4; ++b) I[b] = __fmul_rn(I0, (float)D[4 * k + b]);
        }
        // decisions (Eq. 6): candidate +1 iff r-word k-value < kthr, update iff u-word < thr
        uint32_t wr[4], wu[4];
        pbit_draws4((uint32_t)i, q, a.instance, (uint32_t)t, a.seed_lo, a.seed_hi, wr, wu);
        uint32_t nk[4];
        if (table) {
#pragma unroll
            for (int b = 0; b < 4; ++b) nk[b] = __shfl_sync(0xFFFFFFFFu, negk_lane, (int)byte_of(cnt2[k], b));
        } else {
#pragma unroll
            for (int b = 0; b < 4; ++b) nk[b] = 0u - pbit_kthr_of_x(variant_x(a.offset_mode, I0, lam, del, I[b]));
        }
        const uint32_t S = sign_bytes((wr[0] >> 8) + nk[0], (wr[1] >> 8) + nk[1], (wr[2] >> 8) + nk[2], (wr[3] >> 8) + nk[3]);
        const uint32_t U = sign_bytes((wu[0] >> 8) - thr, (wu[1] >> 8) - thr, (wu[2] >> 8) - thr, (wu[3] >> 8) - thr);
        const uint32_t old = wld32(src + cell);
        wst32(dst + cell, ((U & ~S) | (~U & old)) | 0x01010101u);
    }
}

}  // namespace tile
}  // namespace pbit
