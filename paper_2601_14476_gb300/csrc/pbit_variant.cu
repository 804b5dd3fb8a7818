// The pSA variants of the Methods section (SpSA: a stalled p-bit keeps its
// last input; TApSA: the input is the mean of the last `window` fields) and
// the paper's period timing model (node i updates only at the sub-steps q
// with q % nu_i == 0), one launch per (sub-)step, in a coalesced word tile.
//
// Tile: a warp owns a span of 128 * NW consecutive trials of one node; lane l
// takes the 4-trial words l, l + 32, ... of the span.  So every access of a
// warp for one word index is one contiguous run: 128 B of spins for the node
// and for each neighbour, 512 B of SpSA float32 inputs, 256 B of TApSA int16
// fields per ring slot.  The state keeps its plain [n][T] (SpSA) and
// [window][n][T] (TApSA) layout.
//
// Timing model, two forms.  Parity form (used when the nodes take at most 32
// distinct periods): node i has updated K_i(q) = ceil(q / nu_i) times before
// sub-step q, and its spins live in spins_out when K_i(q) is odd and in the
// scratch buffer when it is even.  A due node reads its spins and its
// neighbours' from where their counts put them and writes the other buffer;
// no neighbour writes a buffer it reads, so the update stays synchronous, and
// a sub-step launches warps for its due nodes alone (the host groups the
// nodes by period and passes the runs of due periods and the parity of every
// period).  One pass at the start places the input by parity, one at the end
// gathers the result into spins_out.  Copy form (otherwise): the Jacobi
// rotation, where a node that is not due copies its spins to the output
// buffer, but only when that buffer lacks them: the output of sub-step q holds
// the state of q - 2 (`carry`), which differs from that of q - 1 only for the
// nodes due at q - 1.
//
// Consecutive (sub-)step launches use programmatic dependent launch: a grid
// runs its constant prologue while the previous one drains and waits for it
// (griddepcontrol.wait) before touching spins or state.
#include "pbit_internal.h"
#include "pbit_device.cuh"
#include "pbit_tile.cuh"

#include <algorithm>
#include <cstdlib>
#include <numeric>

namespace pbit {
namespace {

using tile::sign_bytes;
using tile::variant_x;

constexpr int kVBlock = 256;
constexpr int kMaxRanges = 32;

struct VariantLaunch {
    StepArgs a;
    int32_t slots;            // parity form: a.out holds odd update counts, alt even ones
    int8_t* alt;
    const uint8_t* bkt;       // [n] period bucket of each node
    const uint8_t* ebkt;      // [nnz] period bucket of each edge's column
    uint32_t pmask;           // bit b: ceil(q / period_b) & 1
    uint32_t spans;           // spans per node: T / (128 * NW)
    uint64_t span_m;          // local warp -> node: (w * span_m) >> span_s = w / spans
    int32_t span_s;
    int32_t nranges;          // 0: warps cover all nodes in order; else the perm ranges below
    uint32_t warps;           // warps of the launch
    int32_t rstart[kMaxRanges];     // first perm position of range r
    uint32_t rwarp_end[kMaxRanges]; // prefix sums of the warps of ranges 0..r
};

// Division by d >= 1 for dividends below 2^31 (Granlund-Montgomery).
void magic_divisor(uint32_t d, uint64_t& m, int32_t& s) {
    int l = 0;
    while ((1ull << l) < d) ++l;
    m = ((1ull << (32 + l)) / d) + 1;
    s = 32 + l;
}

__device__ __forceinline__ uint32_t ld32(const int8_t* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ void st32(int8_t* p, uint32_t v) { *reinterpret_cast<uint32_t*>(p) = v; }

// WIN: the TApSA window when it is 4 (the paper's; its other-slot loads unrolled), else 0
template <int NW, bool UNIT, int WIN>
__global__ void __launch_bounds__(kVBlock, NW >= 4 ? 3 : 4) sparse_variant_words_kernel(const __grid_constant__ VariantLaunch L) {
    const StepArgs& a = L.a;
    // programmatic dependent launch: the next (sub-)step's grid may start its prologue now; it reads
    // spins and state only after its own griddepcontrol.wait (below), which returns once this grid
    // has completed and its memory is visible.  Both are no-ops in a launch without the attribute.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const uint32_t warp = (blockIdx.x * (uint32_t)kVBlock + threadIdx.x) >> 5;
    const int lane = (int)(threadIdx.x & 31u);
    if (warp >= L.warps) return;
    uint32_t local = warp;
    int32_t first = 0;
    if (L.nranges > 0) {
        int r = 0;
        while (r + 1 < L.nranges && warp >= L.rwarp_end[r]) ++r;
        local = warp - (r ? L.rwarp_end[r - 1] : 0u);
        first = L.rstart[r];
    }
    const uint32_t nl = (uint32_t)(((unsigned long long)local * L.span_m) >> L.span_s);
    const uint32_t sidx = local - nl * L.spans;
    const int i = L.nranges > 0 ? __ldg(a.perm + first + (int)nl) : (int)nl;
    const int T = a.T;
    const uint32_t q = (uint32_t)a.step;
    const int tb = (int)sidx * (128 * NW) + 4 * lane;  // trial of word 0; word k at tb + 128 k
    const size_t row = (size_t)i * T;
    // everything above and the per-node parameters below are constant over the call; spins and state
    // are written by the previous grid
    const uint32_t nu_i = a.t_res > 0 && !L.slots ? (uint32_t)__ldg(a.nu + i) : 1u;
    const float I0 = __ldg(a.i0_table + (a.t_res > 0 ? q / (uint32_t)a.t_res : q));
    const int hi = a.h ? __ldg(a.h + i) : 0;
    const float lam = a.par.lambda ? __ldg(a.par.lambda + i) : 1.0f;
    const float del = a.par.delta ? __ldg(a.par.delta + i) : 0.0f;
    const uint32_t thr = a.par.thr ? __ldg(a.par.thr + i) : (1u << 24);
    const int rb = __ldg(a.row_ptr + i), re = __ldg(a.row_ptr + i + 1);
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // where the node's spins are read and written, and where neighbour j's are read
    const int8_t* src = a.in;
    int8_t* dst = a.out;
    if (L.slots) {
        const bool odd = (L.pmask >> __ldg(L.bkt + i)) & 1u;
        src = odd ? a.out : L.alt;
        dst = odd ? L.alt : a.out;
    }
    const auto nbr = [&](int e) -> const int8_t* {
        if (!L.slots) return a.in;
        return ((L.pmask >> __ldg(L.ebkt + e)) & 1u) ? a.out : L.alt;
    };
    if (a.t_res > 0 && !L.slots) {
        const uint32_t nu = nu_i;
        if (q % nu != 0u) {
            if (!a.carry || (q - 1u) % nu == 0u) {
#pragma unroll
                for (int k = 0; k < NW; ++k) st32(a.out + row + tb + 128 * k, ld32(a.in + row + tb + 128 * k));
            }
            return;
        }
    }
    tile::variant_words<NW, UNIT, WIN>(a, i, tb, I0, hi, lam, del, thr, rb, re, src, dst, nbr, lane);
}

// Parity form, start and end: node i's row moves from src[P] to dst[P], P the parity of its count.
__global__ void slot_move_kernel(int32_t n, int32_t words, const uint8_t* __restrict__ bkt, uint32_t pmask,
                                 const int8_t* src0, const int8_t* src1, int8_t* dst0, int8_t* dst1) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= (int64_t)n * words) return;
    const int i = (int)(k / words);
    const bool odd = (pmask >> __ldg(bkt + i)) & 1u;
    const int8_t* sp = odd ? src1 : src0;
    int8_t* dp = odd ? dst1 : dst0;
    if ((const void*)sp == (const void*)dp) return;
    reinterpret_cast<uint32_t*>(dp)[k] = reinterpret_cast<const uint32_t*>(sp)[k];
}

__global__ void edge_bucket_kernel(int64_t nnz, const int32_t* __restrict__ col, const uint8_t* __restrict__ bkt,
                                   uint8_t* __restrict__ ebkt) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < nnz) ebkt[e] = __ldg(bkt + __ldg(col + e));
}

// One launch with programmatic stream serialization (the grid may begin while the previous kernel in
// the stream drains; see the kernel's griddepcontrol), or a plain launch when PBIT_NO_PDL is set or
// the attribute is refused.
template <typename K>
cudaError_t launch_pdl(K kernel, unsigned blocks, const VariantLaunch& L, cudaStream_t s) {
    static const bool off = std::getenv("PBIT_NO_PDL") != nullptr;
    if (!off) {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(blocks);
        cfg.blockDim = dim3(kVBlock);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (cudaLaunchKernelEx(&cfg, kernel, L) == cudaSuccess) return cudaSuccess;
        (void)cudaGetLastError();  // clear the refusal, then launch plainly
    }
    kernel<<<blocks, kVBlock, 0, s>>>(L);
    return cudaGetLastError();
}

template <int NW, bool UNIT>
cudaError_t launch_words(const VariantLaunch& L, cudaStream_t s) {
    if (L.warps == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)(((uint64_t)L.warps * 32 + kVBlock - 1) / kVBlock);
    const cudaError_t e = (L.a.alg == 2 && L.a.window == 4)
                              ? launch_pdl(sparse_variant_words_kernel<NW, UNIT, 4>, blocks, L, s)
                              : launch_pdl(sparse_variant_words_kernel<NW, UNIT, 0>, blocks, L, s);
    count_launches(1);
    return e;
}

bool aligned(const void* p, uintptr_t b) { return ((uintptr_t)p % b) == 0; }

}  // namespace

void build_period_buckets(const std::vector<int32_t>& nu, PeriodBuckets& pb) {
    const int32_t n = (int32_t)nu.size();
    pb.host_perm.resize((size_t)n);
    std::iota(pb.host_perm.begin(), pb.host_perm.end(), 0);
    std::stable_sort(pb.host_perm.begin(), pb.host_perm.end(),
                     [&](int32_t x, int32_t y) { return nu[(size_t)x] < nu[(size_t)y]; });
    pb.period.clear();
    pb.start.clear();
    pb.len.clear();
    for (int32_t k = 0; k < n; ++k) {
        const int32_t v = nu[(size_t)pb.host_perm[(size_t)k]];
        if (pb.period.empty() || pb.period.back() != v) {
            pb.period.push_back(v);
            pb.start.push_back(k);
            pb.len.push_back(0);
        }
        ++pb.len.back();
    }
    pb.host_bkt.clear();
    if (pb.period.size() <= 32) {
        pb.host_bkt.resize((size_t)n);
        for (size_t b = 0; b < pb.period.size(); ++b)
            for (int32_t k = pb.start[b]; k < pb.start[b] + pb.len[b]; ++k) pb.host_bkt[(size_t)pb.host_perm[(size_t)k]] = (uint8_t)b;
    }
}

cudaError_t launch_edge_buckets(const Graph& g, const uint8_t* bkt, uint8_t* ebkt, cudaStream_t s) {
    if (g.nnz == 0) return cudaSuccess;
    edge_bucket_kernel<<<(unsigned)((g.nnz + 255) / 256), 256, 0, s>>>(g.nnz, g.col, bkt, ebkt);
    count_launches(1);
    return cudaGetLastError();
}

bool variant_words_ok(const StepArgs& a) {
    return a.T % 128 == 0 && (int64_t)a.n * (a.T / 128) < (1ll << 31) && aligned(a.in, 4) && aligned(a.out, 4) &&
           (a.alg != 1 || aligned(a.Iprev, 16)) && (a.alg != 2 || aligned(a.ring, 8));
}

namespace {

// Words per lane and the warp -> node divisor for the word tile.
void words_config(VariantLaunch& L) {
    // words per lane: up to two (PBIT_VARIANT_NW sets the cap, 1, 2 or 4).  Measured on GB300, 100x200
    // torus, T = 1024, µs per step with one, two and four words: SpSA 96 / 84 / 88, TApSA 112 / 101 / 111,
    // timing model (t_res = 10, copy form) 14.0 / 12.7 / 13.3 per sub-step.
    static const int nw_cap = std::getenv("PBIT_VARIANT_NW") ? std::atoi(std::getenv("PBIT_VARIANT_NW")) : 2;
    const int T = L.a.T;
    const int NW = T % 512 == 0 && nw_cap >= 4 ? 4 : (T % 256 == 0 && nw_cap >= 2 ? 2 : 1);
    L.spans = (uint32_t)(T / (128 * NW));
    magic_divisor(L.spans, L.span_m, L.span_s);
    L.nranges = 0;
    L.warps = (uint32_t)((int64_t)L.a.n * L.spans);
}

cudaError_t launch_words_any(const VariantLaunch& L, SparseVariant v, cudaStream_t s) {
    const int NW = (int)(L.a.T / (128 * L.spans));
    if (NW == 4) return v.unit ? launch_words<4, true>(L, s) : launch_words<4, false>(L, s);
    if (NW == 2) return v.unit ? launch_words<2, true>(L, s) : launch_words<2, false>(L, s);
    return v.unit ? launch_words<1, true>(L, s) : launch_words<1, false>(L, s);
}

cudaError_t launch_move(const Graph& g, int32_t T, const uint8_t* bkt, uint32_t pmask, const int8_t* src0,
                        const int8_t* src1, int8_t* dst0, int8_t* dst1, cudaStream_t s) {
    const int64_t total = (int64_t)g.n * (T / 4);
    if (total == 0) return cudaSuccess;
    slot_move_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(g.n, T / 4, bkt, pmask, src0, src1, dst0, dst1);
    count_launches(1);
    return cudaGetLastError();
}

uint32_t parity_mask(const PeriodBuckets& pb, uint32_t q) {
    uint32_t m = 0;
    for (size_t b = 0; b < pb.period.size(); ++b) {
        const uint32_t p = (uint32_t)pb.period[b];
        m |= (((q + p - 1u) / p) & 1u) << b;
    }
    return m;
}

}  // namespace

cudaError_t launch_timing_slots(const Graph& g, const StepArgs& base, int32_t b, int32_t e, const int8_t* cur,
                                int8_t* X, int8_t* Y, const PeriodBuckets& pb, SparseVariant v, cudaStream_t s) {
    VariantLaunch L{};
    L.a = base;
    L.a.in = X;
    L.a.out = X;
    if (base.t_res <= 0 || !variant_words_ok(L.a) || !aligned(Y, 4) || !aligned(cur, 4) || pb.period.empty() ||
        pb.period.size() > 32 || !pb.bkt || !pb.ebkt || !pb.perm || (int64_t)e + pb.period.back() >= (1ll << 31))
        return cudaErrorNotSupported;
    words_config(L);
    L.slots = 1;
    L.alt = Y;
    L.bkt = pb.bkt;
    L.ebkt = pb.ebkt;
    L.a.perm = pb.perm;
    const int32_t T = base.T;
    cudaError_t err = launch_move(g, T, pb.bkt, parity_mask(pb, (uint32_t)b), cur, cur, Y, X, s);
    if (err != cudaSuccess) return err;
    for (int32_t q = b; q < e; ++q) {
        // the due nodes, as runs of the period-sorted permutation
        int nr = 0;
        uint32_t warps = 0;
        int32_t run_end = -1;
        for (size_t k = 0; k < pb.period.size(); ++k) {
            if ((uint32_t)q % (uint32_t)pb.period[k] != 0u) continue;
            if (pb.start[k] == run_end) {
                L.rwarp_end[nr - 1] += (uint32_t)pb.len[k] * L.spans;
            } else {
                L.rstart[nr] = pb.start[k];
                L.rwarp_end[nr] = warps + (uint32_t)pb.len[k] * L.spans;
                ++nr;
            }
            warps += (uint32_t)pb.len[k] * L.spans;
            run_end = pb.start[k] + pb.len[k];
        }
        if (nr == 0) continue;
        L.a.step = q;
        L.nranges = nr;
        L.warps = warps;
        L.pmask = parity_mask(pb, (uint32_t)q);
        if ((err = launch_words_any(L, v, s)) != cudaSuccess) return err;
    }
    return launch_move(g, T, pb.bkt, parity_mask(pb, (uint32_t)e), Y, X, X, X, s);
}

cudaError_t launch_variant_step(const StepArgs& base, const PeriodBuckets* pb, cudaStream_t s, SparseVariant v) {
    if (!variant_words_ok(base)) {
        StepArgs a = base;
        a.carry = 0;  // the group tile copies every idle node
        return launch_sparse_step(a, s, v);
    }
    VariantLaunch L{};
    L.a = base;
    words_config(L);
    if (base.t_res > 0 && base.carry && pb && pb->perm && !pb->period.empty()) {
        // nodes due at q or q - 1, as runs of the period-sorted permutation
        const uint32_t q = (uint32_t)base.step;
        int nr = 0;
        uint32_t warps = 0;
        int32_t run_end = -1;
        bool fits = true;
        for (size_t b = 0; b < pb->period.size(); ++b) {
            const uint32_t p = (uint32_t)pb->period[b];
            if (q % p != 0u && (q - 1u) % p != 0u) continue;
            if (pb->start[b] == run_end) {
                L.rwarp_end[nr - 1] += (uint32_t)pb->len[b] * L.spans;
            } else {
                if (nr == kMaxRanges) {
                    fits = false;
                    break;
                }
                L.rstart[nr] = pb->start[b];
                L.rwarp_end[nr] = warps + (uint32_t)pb->len[b] * L.spans;
                ++nr;
            }
            warps += (uint32_t)pb->len[b] * L.spans;
            run_end = pb->start[b] + pb->len[b];
        }
        if (fits) {
            L.a.perm = pb->perm;
            L.nranges = nr;
            L.warps = warps;
            if (nr == 0) return cudaSuccess;  // nothing due now or a sub-step ago: both buffers agree
        }
    }
    return launch_words_any(L, v, s);
}

}  // namespace pbit
