// Dense field on the 5th-generation tensor cores (tcgen05) with the p-bit
// update fused into the epilogue.
//
// Field (Eq. conv): D = J * M for a dense J (n x n) and the spins of T trials.
// ptxas for sm_103a has no tcgen05 int8 kind, so the contraction runs as
// kind::f8f6f4 with e4m3 operands and an FP32 accumulator.  It is exact here:
// every J_ij with |J_ij| <= 16 and every spin (+-1, or 0 for padding) is an
// e4m3 value, each product is an integer of magnitude <= 16, and every
// partial sum is an integer below 2^14 in magnitude (K slice of 256 nodes),
// far inside FP32's exact-integer range.  The K-slice partials are summed in
// FP32 (still exact: |D| < 2^24) by a cluster reduction over distributed
// shared memory.
//
// Work decomposition of one step (one launch):
//   grid = (KS, RB, TB) CTAs, cluster = (KS, 1, 1)
//   CTA (ks, rb, tb): rows rb*128..+128 of J, K slice ks*256..+256, trials
//   tb*NT..+NT.  It bulk-copies its J tile (128 x 256 e4m3) and spin tile
//   (NT x 256 e4m3) into shared memory, issues 8 tcgen05.mma (M=128, N=NT,
//   K=32) into TMEM, reads the 128 x NT partial back, publishes it in its
//   shared memory; after a cluster barrier each CTA sums, for its NT/KS
//   trial columns, the KS partials of its 128 rows and applies the p-bit
//   update (Eq. pbits_variability with the timing draw) to them.
//
// Global layouts (both written in the exact no-swizzle K-major core-matrix
// order the MMA reads, so one bulk copy moves a whole tile):
//   J tiles:  [rb][ks][row group (16)][k core (16)][row (8)][16 bytes]
//   spins:    [ks][trial group (T/8)][k core (16)][trial (8)][16 bytes]
// where a "k core" is 16 consecutive nodes j.  Core matrices are 8 x 16 B =
// 128 contiguous bytes: leading byte offset (next core along K) = 128,
// stride byte offset (next 8-row group) = 16 * 128 = 2048.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "pbit_device.cuh"
#include "pbit_internal.h"

namespace cg = cooperative_groups;

namespace pbit {
namespace {

constexpr int kRows = 128;          // MMA M
constexpr int kSlice = 256;         // K slice per CTA (nodes)
constexpr int kCores = kSlice / 16; // k cores per slice
constexpr int kThreads = 256;
constexpr int kPad = 4;             // partial row padding (floats)
constexpr uint8_t kE4m3Plus1 = 0x38, kE4m3Minus1 = 0xB8;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after ~2^31 cycles (about a second) and reports it.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    const long long start = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - start > (1ll << 31)) return false;
    }
    return true;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor, no swizzle, K-major canonical layout.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;                // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor: D f32, A/B e4m3, both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_e4m3(uint32_t n) {
    return (1u << 4)               // D format: f32
           | (0u << 7)             // A format: e4m3
           | (0u << 10)            // B format: e4m3
           | ((n >> 3) << 17)      // N / 8
           | ((uint32_t)(kRows >> 4) << 24);  // M / 16
}

__device__ __forceinline__ void mma_e4m3(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 32 lanes x 32 consecutive 32-bit columns per warp.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
          "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
          "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Byte offset of (trial t, node j) in the tiled spin layout.
__host__ __device__ __forceinline__ size_t spin_off(int t, int j, int T) {
    const int ks = j / kSlice, c = (j % kSlice) >> 4, b = j & 15;
    const int g = t >> 3, r = t & 7;
    return (size_t)ks * ((size_t)T * kSlice) + (size_t)g * (kCores * 128) + (size_t)c * 128 + (size_t)r * 16 + b;
}

struct DenseArgs {
    const uint8_t* Jt;       // tiled J (e4m3)
    const uint8_t* s_in;     // tiled spins (e4m3), current state
    uint8_t* s_out;          // tiled spins, next state (unused when fields_out is set)
    int32_t* fields_out;     // if non-null: write D = h + J s as int32 [n][T] and skip the update
    const int32_t* h;
    NodeParams par;
    const float* i0_table;
    int32_t step;
    int32_t n, T, NT, KS;
    uint32_t seed_lo, seed_hi, instance;
    int32_t offset_mode;
    int* err;
};

__global__ void __launch_bounds__(kThreads, 1) dense_step_kernel(DenseArgs a) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    // 128-align the dynamic shared memory base (descriptors and bulk copies need 16)
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    uint8_t* sA = smem;                                   // 128 x 256 bytes
    uint8_t* sB = sA + kRows * kSlice;                    // NT x 256 bytes
    float* part = (float*)(sB + (size_t)a.NT * kSlice);   // 128 x (NT + kPad)
    uint64_t* bars = (uint64_t*)(part + (size_t)kRows * (a.NT + kPad));
    uint32_t* tmem_slot = (uint32_t*)(bars + 2);

    cg::cluster_group cluster = cg::this_cluster();
    const int ks = blockIdx.x, rb = blockIdx.y, tb = blockIdx.z;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NT = a.NT;
    const uint32_t ncols = NT <= 32 ? 32 : (NT <= 64 ? 64 : (NT <= 128 ? 128 : 256));
    bool ok = true;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // ---- load the J tile and the spin tile, run the MMAs
    if (tid == 0) {
        const uint32_t bytesA = kRows * kSlice, bytesB = (uint32_t)NT * kSlice;
        mbar_expect_tx(&bars[0], bytesA + bytesB);
        const uint8_t* gA = a.Jt + ((size_t)rb * a.KS + ks) * (size_t)(kRows * kSlice);
        const uint8_t* gB = a.s_in + (size_t)ks * ((size_t)a.T * kSlice) + (size_t)tb * NT * kSlice;
        bulk_g2s(sA, gA, bytesA, &bars[0]);
        bulk_g2s(sB, gB, bytesB, &bars[0]);
        if (!mbar_wait_bounded(&bars[0], 0)) {
            atomicExch(a.err, 1);
            ok = false;
        }
        if (ok) {
            tc_fence_after();
            const uint32_t idesc = idesc_e4m3((uint32_t)NT);
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
            for (int kk = 0; kk < kSlice / 32; ++kk) {
                const uint64_t ad = smem_desc(a0 + kk * 256, 128, kCores * 128);
                const uint64_t bd = smem_desc(b0 + kk * 256, 128, kCores * 128);
                mma_e4m3(tmem, ad, bd, idesc, kk > 0 ? 1u : 0u);
            }
            mma_commit(&bars[1]);
        }
    }
    // thread 0 waits (bounded) for the MMA results and broadcasts the outcome,
    // so the warp-collective TMEM loads below are taken uniformly
    __shared__ int s_ok;
    if (tid == 0) {
        if (ok && !mbar_wait_bounded(&bars[1], 0)) {
            atomicExch(a.err, 2);
            ok = false;
        }
        s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    ok = s_ok != 0;
    tc_fence_after();

    // ---- TMEM -> shared partial (warps 0-3: columns [0,128), warps 4-7: [128,256))
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const int stride = NT + kPad;
    if (ok) {
        for (int c0 = (warp >> 2) * 128; c0 < NT; c0 += 256) {
            for (int cc = c0; cc < min(NT, c0 + 128); cc += 32) {
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)cc, v);
                tmem_wait_ld();
                float4* dst = reinterpret_cast<float4*>(part + (size_t)row * stride + cc);
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    dst[q] = make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                                         __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
    cluster.sync();

    // ---- cluster reduction over K slices + fused p-bit update
    // CTA ks owns trial-column pairs [pb, pe) of its row block; the two
    // threads of a row split them.  Columns are processed in chunks of 16.
    const int pairs = NT / 2;
    const int pb = (ks * pairs) / a.KS, pe = ((ks + 1) * pairs) / a.KS;
    const int pm = (pb + pe) / 2;
    const int half = tid >> 7;
    const int r = tid & 127;
    const int i = rb * kRows + r;
    const int cb = 2 * (half == 0 ? pb : pm), ce = 2 * (half == 0 ? pm : pe);
    const bool active = ok && i < a.n;
    const int hi = (active && a.h) ? a.h[i] : 0;
    const float I0 = a.fields_out ? 0.0f : a.i0_table[a.step];
    const float lam = (active && a.par.lambda) ? a.par.lambda[i] : 1.0f;
    const float del = (active && a.par.delta) ? a.par.delta[i] : 0.0f;
    const uint32_t thr = (active && a.par.thr) ? a.par.thr[i] : (1u << 24);
    for (int c = cb; active && c < ce; c += 16) {
        const int cnt = min(16, ce - c);
        float acc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = 0.0f;
        for (int src = 0; src < a.KS; ++src) {
            const float* rp = cluster.map_shared_rank(part, src) + (size_t)r * stride + c;
            if (cnt == 16 && (c & 3) == 0) {
#pragma unroll
                for (int q = 0; q < 16; q += 4) {
                    const float4 v = *reinterpret_cast<const float4*>(rp + q);
                    acc[q] += v.x;
                    acc[q + 1] += v.y;
                    acc[q + 2] += v.z;
                    acc[q + 3] += v.w;
                }
            } else {
                for (int q = 0; q < cnt; ++q) acc[q] += rp[q];
            }
        }
        if (a.fields_out) {
            for (int q = 0; q < cnt; ++q)
                a.fields_out[(size_t)i * a.T + tb * NT + c + q] = hi + __float2int_rn(acc[q]);
            continue;
        }
#pragma unroll
        for (int q = 0; q < 16; q += 2) {
            if (q < cnt) {
                const int t = tb * NT + c + q;  // even
                const uint4 rw =
                    philox((uint32_t)i, (uint32_t)a.step, (uint32_t)t >> 1, a.instance, a.seed_lo, a.seed_hi);
                const int D0 = hi + __float2int_rn(acc[q]);
                const int D1 = hi + __float2int_rn(acc[q + 1]);
                const uint32_t k0 = pbit_kthr_of_x(pbit_input(a.offset_mode, I0, lam, del, D0));
                const uint32_t k1 = pbit_kthr_of_x(pbit_input(a.offset_mode, I0, lam, del, D1));
                const size_t o0 = spin_off(t, i, a.T), o1 = spin_off(t + 1, i, a.T);
                const int old0 = a.s_in[o0] == kE4m3Plus1 ? 1 : -1;
                const int old1 = a.s_in[o1] == kE4m3Plus1 ? 1 : -1;
                a.s_out[o0] = pbit_next(rw.x, rw.y, k0, thr, old0) > 0 ? kE4m3Plus1 : kE4m3Minus1;
                a.s_out[o1] = pbit_next(rw.z, rw.w, k1, thr, old1) > 0 ? kE4m3Plus1 : kE4m3Minus1;
            }
        }
    }
    cluster.sync();  // peers leave only after every CTA has read their partials
}

// int8 trial-major [n][T]  <->  tiled e4m3 (padding nodes written as 0)
__global__ void to_tiled_kernel(const int8_t* __restrict__ s, int32_t n, int32_t n_pad, int32_t T,
                                uint8_t* __restrict__ out) {
    const int64_t total = (int64_t)n_pad * T;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(idx / T), t = (int)(idx - (int64_t)j * T);
        uint8_t v = 0;
        if (j < n) v = s[(size_t)j * T + t] > 0 ? kE4m3Plus1 : kE4m3Minus1;
        out[spin_off(t, j, T)] = v;
    }
}

__global__ void from_tiled_kernel(const uint8_t* __restrict__ in, int32_t n, int32_t T, int8_t* __restrict__ s) {
    const int64_t total = (int64_t)n * T;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(idx / T), t = (int)(idx - (int64_t)j * T);
        s[idx] = in[spin_off(t, j, T)] == kE4m3Plus1 ? 1 : -1;
    }
}

size_t dense_smem_bytes(int NT) {
    return 128 + (size_t)kRows * kSlice + (size_t)NT * kSlice + (size_t)kRows * (NT + kPad) * sizeof(float) + 64;
}

uint8_t e4m3_of_int(int v) {
    // exact e4m3 encoding of an integer with |v| <= 16
    if (v == 0) return 0;
    const uint8_t sign = v < 0 ? 0x80 : 0;
    int a = v < 0 ? -v : v;
    int e = 0;
    while ((a >> (e + 1)) > 0) ++e;            // 2^e <= a < 2^(e+1)
    const int mant = ((a << 3) >> e) & 7;      // 3 fraction bits (exact for a <= 16)
    return (uint8_t)(sign | ((e + 7) << 3) | mant);
}

}  // namespace

// ------------------------------------------------------------- host side ----
bool dense_shape_ok(const Graph& g, int32_t T, std::string* why) {
    if (!g.dense.J_e4m3) {
        if (why) *why = "graph was created without PBIT_GRAPH_DENSE (or |w| > 16 / n > 4096)";
        return false;
    }
    if (T % 32 != 0 || (T > 256 && T % 256 != 0)) {
        if (why) *why = "dense kernel needs trials % 32 == 0 and (trials <= 256 or trials % 256 == 0)";
        return false;
    }
    return true;
}

pbit_status build_dense_operand(Graph& g) {
    const int n_pad = ((g.n + kSlice - 1) / kSlice) * kSlice;
    const int KS = n_pad / kSlice, RB = n_pad / kRows;
    if (KS > 16) return fail(PBIT_E_INVALID, "dense operand: n > 4096 is not supported by the tensor-core path");
    for (size_t k = 0; k < g.h_J.size() && k < (size_t)g.nnz; ++k)
        if (g.h_J[k] > 16 || g.h_J[k] < -16)
            return fail(PBIT_E_INVALID, "dense operand: |w| > 16 is not exact in e4m3");
    std::vector<uint8_t> tiles((size_t)n_pad * n_pad, 0);
    for (int i = 0; i < g.n; ++i) {
        const int rb = i / kRows, rg = (i % kRows) >> 3, rr = i & 7;
        for (int k = g.h_row_ptr[(size_t)i]; k < g.h_row_ptr[(size_t)i + 1]; ++k) {
            const int j = g.h_col[(size_t)k];
            const int ks = j / kSlice, c = (j % kSlice) >> 4, b = j & 15;
            const size_t off = ((size_t)rb * KS + ks) * (size_t)(kRows * kSlice) + (size_t)rg * (kCores * 128) +
                               (size_t)c * 128 + (size_t)rr * 16 + b;
            tiles[off] = e4m3_of_int(g.h_J[(size_t)k]);
        }
    }
    (void)RB;
    cudaError_t e = cudaMalloc((void**)&g.dense.J_e4m3, tiles.size());
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(dense J)");
    e = cudaMemcpy(g.dense.J_e4m3, tiles.data(), tiles.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(dense J)");
    g.dense.n_pad = n_pad;
    g.dense.bytes = tiles.size();
    g.device_bytes += tiles.size();
    return PBIT_OK;
}

size_t dense_spin_bytes(const Graph& g, int32_t T) { return (size_t)g.dense.n_pad * (size_t)T; }

cudaError_t launch_to_tiled(const Graph& g, const int8_t* s, int32_t T, uint8_t* out, cudaStream_t st) {
    to_tiled_kernel<<<152 * 8, 256, 0, st>>>(s, g.n, g.dense.n_pad, T, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_from_tiled(const Graph& g, const uint8_t* in, int32_t T, int8_t* s, cudaStream_t st) {
    from_tiled_kernel<<<152 * 8, 256, 0, st>>>(in, g.n, T, s);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_dense_step(const Graph& g, const StepArgs& sa, const uint8_t* tin, uint8_t* tout,
                              int32_t* fields_out, int* err, cudaStream_t st) {
    DenseArgs a{};
    a.Jt = g.dense.J_e4m3;
    a.s_in = tin;
    a.s_out = tout;
    a.fields_out = fields_out;
    a.h = g.h;
    a.par = sa.par;
    a.i0_table = sa.i0_table;
    a.step = sa.step;
    a.n = g.n;
    a.T = sa.T;
    a.NT = sa.T <= 256 ? sa.T : 256;
    a.KS = g.dense.n_pad / kSlice;
    a.seed_lo = sa.seed_lo;
    a.seed_hi = sa.seed_hi;
    a.instance = sa.instance;
    a.offset_mode = sa.offset_mode;
    a.err = err;
    const size_t smem = dense_smem_bytes(a.NT);
    cudaError_t e = cudaFuncSetAttribute(dense_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (a.KS > 8) {
        e = cudaFuncSetAttribute(dense_step_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)a.KS, (unsigned)(g.dense.n_pad / kRows), (unsigned)(sa.T / a.NT));
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)a.KS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, dense_step_kernel, a);
    count_launches(1);
    return e;
}

}  // namespace pbit
