// Dense field on the 5th-generation tensor cores (tcgen05) with the p-bit
// update fused into the epilogue.
//
// Field (Eq. conv): D = J * M for a dense J (n x n) and the spins of T trials.
// ptxas for sm_103a has no tcgen05 int8 kind, so the contraction runs as
// kind::f8f6f4 with e4m3 operands and an FP32 accumulator.  It is exact here:
// every J_ij with |J_ij| <= 16 and every spin (+-1, or 0 for padding) is an
// e4m3 value, each product is an integer of magnitude <= 16, and every
// partial sum is an integer of magnitude at most 16 * 512 = 2^13 (K slice of
// 512 nodes),
// far inside FP32's exact-integer range.  The K-slice partials are summed in
// FP32 (still exact: |D| < 2^24) by a cluster reduction over distributed
// shared memory.
//
// Work decomposition of one step (one launch):
//   grid = (KS, RB, TB) CTAs, cluster = (KS, 1, 1)
//   CTA (ks, rb, tb): rows rb*128..+128 of J, K slice ks*512..+512, trials
//   tb*NT..+NT (NT <= 128).  It bulk-copies its J tile (128 x 512 e4m3) and
//   spin tile (NT x 512 e4m3) into shared memory, issues 16 tcgen05.mma
//   (M=128, N=NT, K=32) into TMEM, reads the 128 x NT partial back, publishes it in its
//   shared memory; after a cluster barrier each CTA sums, for its NT/KS
//   trial columns, the KS partials of its 128 rows and applies the p-bit
//   update (Eq. pbits_variability with the timing draw) to them.
//
// Global layouts (both written in the exact no-swizzle K-major core-matrix
// order the MMA reads, so one bulk copy moves a whole tile):
//   J tiles:  [rb][ks][row group (16)][k core (32)][row (8)][16 bytes]
//   spins:    [ks][trial group (T/8)][k core (32)][trial (8)][16 bytes]
// where a "k core" is 16 consecutive nodes j.  Core matrices are 8 x 16 B =
// 128 contiguous bytes: leading byte offset (next core along K) = 128,
// stride byte offset (next 8-row group) = 32 * 128 = 4096.
// The K slice is 512 nodes so that a cluster has at most n/512 CTAs: with
// one CTA per SM (about 190-230 KB of shared memory each) GB300 keeps 36
// clusters of 4 resident but only 15 of 8.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "pbit_device.cuh"
#include "pbit_internal.h"

namespace cg = cooperative_groups;

namespace pbit {
namespace {

constexpr int kRows = 128;          // MMA M
constexpr int kSlice = 512;         // K slice per CTA (nodes)
constexpr int kCores = kSlice / 16; // k cores per slice
constexpr int kThreads = 256;
constexpr int kMaxNT = 128;         // trials per CTA tile (MMA N)
constexpr int kFlagsPerSlice = kSlice / kRows;  // row blocks producing one K slice
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

// 32 lanes x 16 consecutive 32-bit columns per warp.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
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
    unsigned long long* obs_out;  // if non-null: add S_t = sum_i s_it (J s)_it per trial, skip the update
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
    uint8_t* sA = smem;                                   // 128 x kSlice bytes
    uint8_t* sB = sA + kRows * kSlice;                    // NT x kSlice bytes
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
    if (warp == 0) {
        if (lane == 0) {
            mbar_init(&bars[0], 1);
            mbar_init(&bars[1], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncwarp();  // the CTA barrier below is warp-aligned: reconverge first
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // ---- load the J tile and the spin tile, run the MMAs (lane 0 of warp 0)
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
    __syncwarp();
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
    __syncwarp();
    __syncthreads();
    ok = s_ok != 0;
    tc_fence_after();

    // ---- TMEM -> shared partial: warp w reads lanes 32*(w%4).., 32-column chunks w/4, w/4+2, ...
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const int stride = NT + kPad;
    if (ok) {
        for (int ch = warp >> 2; ch < NT / 32; ch += 2) {
            {
                const int cc = ch * 32;
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
    const float I0 = (a.fields_out || a.obs_out) ? 0.0f : a.i0_table[a.step];
    const float lam = (active && a.par.lambda) ? a.par.lambda[i] : 1.0f;
    const float del = (active && a.par.delta) ? a.par.delta[i] : 0.0f;
    const uint32_t thr = (active && a.par.thr) ? a.par.thr[i] : (1u << 24);
    for (int c = cb; c < ce; c += 16) {
        const int cnt = min(16, ce - c);
        float acc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = 0.0f;
        if (a.obs_out) {
            // per-trial S_t: every lane of a warp takes part in the warp sums (zeros where inactive)
            for (int src = 0; active && src < a.KS; ++src) {
                const float* rp = cluster.map_shared_rank(part, src) + (size_t)r * stride + c;
                for (int q = 0; q < cnt; ++q) acc[q] += rp[q];
            }
            for (int q = 0; q < cnt; ++q) {
                const int t = tb * NT + c + q;
                int v = 0;
                if (active) v = (a.s_in[spin_off(t, i, a.T)] == kE4m3Plus1 ? 1 : -1) * __float2int_rn(acc[q]);
                v = __reduce_add_sync(0xFFFFFFFFu, v);
                if (lane == 0 && v != 0) atomicAdd(a.obs_out + t, (unsigned long long)(long long)v);
            }
            continue;
        }
        if (!active) continue;
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
                const uint4 rw = pbit_draws2((uint32_t)i, (uint32_t)a.step, a.instance, (uint32_t)t, a.seed_lo, a.seed_hi);
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

// ------------------------------------------------------------------------
// Persistent form: one launch runs steps [b, e).  Each CTA loads its J tile
// once and keeps it in shared memory; per step it waits (bounded) until the
// two clusters that produce its K slice have published the previous step,
// bulk-copies its spin tile, runs the MMAs, and the cluster reduces and
// updates as above.  Progress is published per cluster in `done`.  All
// clusters must be co-resident (checked on the host before launch).
// ------------------------------------------------------------------------
struct PersistArgs {
    DenseArgs d;
    uint8_t* buf0;
    uint8_t* buf1;
    int32_t step_begin, step_end;
    unsigned* done;   // [RB * TB], zero on entry
    int32_t tb_base;  // first trial block of this launch (launches cover consecutive groups)
    long long wait_cycles;  // clock64 budget of each producer-flag wait (about a second; shorter in tests)
    int32_t withhold;       // test-only: CTA (0, 0, tb_base) never publishes its progress
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Warps 0..15 read TMEM and run the epilogue; warp 16 is the control warp
// that waits for the producers, issues the bulk copy and the MMAs.
constexpr int kEpi = 512;                      // epilogue threads
constexpr int kPersistThreads = kEpi + 32;
constexpr int kMaxItems = 4;                   // (NT/2/KS) pairs x 32 row quads <= 4 x 512
static_assert(kEpi == 4 * kRows, "the first kEpi items hold 4 groups of 4 trial pairs over kRows rows");

// 17 warps share 4 SM sub-partitions (one holds 5 warps and 16K registers),
// so the compiler keeps this kernel near 100 registers per thread.
__global__ void __launch_bounds__(kPersistThreads, 1) dense_persistent_kernel(PersistArgs pa) {
    const DenseArgs& a = pa.d;
    extern __shared__ __align__(128) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    const int NT = a.NT;
    uint8_t* sA = smem;                                    // 128 x kSlice bytes, stationary
    uint8_t* sB = sA + kRows * kSlice;                     // NT x kSlice bytes
    // partial fields, column-major [NT][128], two buffers used on alternate steps; they are exact
    // integers of magnitude <= 16 * 512, so int16 holds them
    int16_t* part_buf0 = (int16_t*)(sB + (size_t)NT * kSlice);
    int16_t* part_buf1 = part_buf0 + (size_t)NT * kRows;
    float* s_lam = (float*)(part_buf1 + (size_t)NT * kRows);  // per-row parameters
    float* s_del = s_lam + kRows;
    uint32_t* s_thr = (uint32_t*)(s_del + kRows);
    int32_t* s_h = (int32_t*)(s_thr + kRows);
    uint4* s_rw = (uint4*)(s_h + kRows);                   // Philox words [4][kEpi] of the first item
    uint64_t* bars = (uint64_t*)(s_rw + 4 * kEpi);         // 0: J, 1: spins, 2: MMA
    uint32_t* tmem_slot = (uint32_t*)(bars + 3);
    __shared__ int s_abort;

    cg::cluster_group cluster = cg::this_cluster();
    const int ks = blockIdx.x, rb = blockIdx.y, tb = blockIdx.z + pa.tb_base;
    const int RB = gridDim.y;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool control = warp == kEpi / 32;
    const uint32_t ncols = NT <= 32 ? 32 : (NT <= 64 ? 64 : 128);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (control) {
        if (lane == 0) {
            mbar_init(&bars[0], 1);
            mbar_init(&bars[1], 1);
            mbar_init(&bars[2], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            s_abort = 0;
        }
        __syncwarp();
    }
    // per-row parameters staged in shared memory
    for (int r = tid; r < kRows; r += kPersistThreads) {
        const int i = rb * kRows + r;
        const bool in = i < a.n;
        s_lam[r] = (in && a.par.lambda) ? a.par.lambda[i] : 1.0f;
        s_del[r] = (in && a.par.delta) ? a.par.delta[i] : 0.0f;
        s_thr[r] = (in && a.par.thr) ? a.par.thr[i] : (1u << 24);
        s_h[r] = (in && a.h) ? a.h[i] : 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    if (control) {
        if (lane == 0) {
            mbar_expect_tx(&bars[0], kRows * kSlice);
            bulk_g2s(sA, a.Jt + ((size_t)rb * a.KS + ks) * (size_t)(kRows * kSlice), kRows * kSlice, &bars[0]);
            if (!mbar_wait_bounded(&bars[0], 0)) {
                atomicExch(a.err, 1);
                s_abort = 1;
            }
        }
        __syncwarp();
    }
    const int pairs = NT / 2;
    const int pb = (ks * pairs) / a.KS, pe = ((ks + 1) * pairs) / a.KS;
    const int items = (pe - pb) * (kRows / 4);
    // progress flags, one per CTA: done[((tb * RB) + rb) * KS + ks] = steps published
    const unsigned* prod0 = pa.done + ((size_t)tb * RB + (size_t)kFlagsPerSlice * ks) * a.KS;
    const int nprod = kFlagsPerSlice * a.KS;  // the CTAs that write this CTA's K slice
    const uint32_t idesc = idesc_e4m3((uint32_t)NT);
    const int L = pa.step_end - pa.step_begin;
    // Item `it` = (pair pb + it/32, rows 4*(it%32)..+4).  The thread that
    // writes an item's new spins at step s reads them as old spins at s+1, so
    // they stay in registers between steps.
    uint32_t prev0[kMaxItems], prev1[kMaxItems];

    for (int ls = 0; ls < L; ++ls) {
        const int step = pa.step_begin + ls;
        const uint8_t* cur = (ls & 1) ? pa.buf1 : pa.buf0;
        uint8_t* nxt = (ls & 1) ? pa.buf0 : pa.buf1;
        int16_t* part = (ls & 1) ? part_buf1 : part_buf0;
        if (control) {
            bool ok = s_abort == 0;
            if (ok && ls > 0) {
                // every lane watches some of the producer flags, so their L2 round trips overlap
                const long long start = clock64();
                for (;;) {
                    bool ready = true;
                    for (int f = lane; f < nprod; f += 32) ready = ready && ld_acquire(prod0 + f) >= (unsigned)ls;
                    if (__all_sync(0xFFFFFFFFu, ready)) break;
                    if (__shfl_sync(0xFFFFFFFFu, (int)(clock64() - start > pa.wait_cycles), 0)) {
                        ok = false;
                        break;
                    }
                }
                __syncwarp();
            }
            if (lane == 0 && s_abort == 0) {
                if (ls > 0) fence_proxy_async();
                if (ok) {
                    mbar_expect_tx(&bars[1], (uint32_t)NT * kSlice);
                    bulk_g2s(sB, cur + (size_t)ks * ((size_t)a.T * kSlice) + (size_t)tb * NT * kSlice,
                             (uint32_t)NT * kSlice, &bars[1]);
                    ok = mbar_wait_bounded(&bars[1], (uint32_t)(ls & 1));
                }
                if (ok) {
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
                    for (int kk = 0; kk < kSlice / 32; ++kk)
                        mma_e4m3(tmem, smem_desc(a0 + kk * 256, 128, kCores * 128),
                                 smem_desc(b0 + kk * 256, 128, kCores * 128), idesc, kk > 0 ? 1u : 0u);
                    mma_commit(&bars[2]);
                    ok = mbar_wait_bounded(&bars[2], (uint32_t)(ls & 1));
                }
                if (!ok) {
                    atomicExch(a.err, 3);
                    s_abort = 1;
                }
            }
            __syncwarp();  // reconverge before the warp-aligned CTA barrier
        } else {
            // the Philox words of the first kEpi items for the step, drawn while the control warp
            // waits.  Where their pairs form whole groups of 8 trials, thread (group gl, row r) draws
            // the group's three blocks for row r and hands each pair's words to the thread that
            // decides it (3 blocks per 4 pairs and row instead of 2 per pair)
            const int np0 = min(pe - pb, kEpi / 32);  // pairs of the first kEpi items
            if (((tb * NT + 2 * pb) & 7) == 0 && (np0 & 3) == 0) {
                const int gl = tid / kRows, r = tid % kRows;  // kEpi / kRows = 4 groups of 4 pairs
                if (4 * gl < np0) {
                    const uint32_t i = (uint32_t)(rb * kRows + r);
                    const PhiloxHead ph = philox_head(i, (uint32_t)step, a.instance, a.seed_lo, a.seed_hi);
                    const PbitPairs8 d =
                        pbit_pairs8(ph, (uint32_t)(tb * NT + 2 * (pb + 4 * gl)), a.seed_lo, a.seed_hi);
#pragma unroll
                    for (int q = 0; q < 4; ++q) s_rw[(r & 3) * kEpi + (4 * gl + q) * 32 + (r >> 2)] = d.p[q];
                }
            } else if (tid < items) {
                const int p = pb + (tid >> 5);
                const int t0 = tb * NT + 2 * p;
                const int i0 = rb * kRows + (tid & 31) * 4;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    s_rw[k * kEpi + tid] = pbit_draws2((uint32_t)(i0 + k), (uint32_t)step, a.instance,
                                                       (uint32_t)t0, a.seed_lo, a.seed_hi);
            }
            if (tid < items && ls == 0) {
#pragma unroll
                for (int slot = 0; slot < kMaxItems; ++slot) {
                    const int it = tid + slot * kEpi;
                    if (it < items) {
                        const int tt = tb * NT + 2 * (pb + (it >> 5));
                        const int ii = rb * kRows + (it & 31) * 4;
                        prev0[slot] = *reinterpret_cast<const uint32_t*>(cur + spin_off(tt, ii, a.T));
                        prev1[slot] = *reinterpret_cast<const uint32_t*>(cur + spin_off(tt + 1, ii, a.T));
                    }
                }
            }
        }
        __syncthreads();
        const bool abort = s_abort != 0;
        tc_fence_after();
        if (!abort && !control) {
            // TMEM -> column-major partial: lane = row, 32-column chunks over the four warp groups
            const int quarter = warp & 3;
            const int row = quarter * 32 + lane;
            for (int ch = warp >> 2; ch < NT / 16; ch += 4) {
                const int c = ch * 16;
                uint32_t v[16];
                tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c, v);
                tmem_wait_ld();
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    part[(size_t)(c + q) * kRows + row] = (int16_t)__float2int_rn(__uint_as_float(v[q]));
            }
        }
        tc_fence_before();
        cluster.sync();
        if (!abort && !control) {
            const float I0 = a.i0_table[step];
#pragma unroll
            for (int slot = 0; slot < kMaxItems; ++slot) {
                const int it = tid + slot * kEpi;
                if (it < items) {
                    const int r0 = (it & 31) * 4;
                    const int lc0 = 2 * (pb + (it >> 5));
                    int f0[4] = {0, 0, 0, 0}, f1[4] = {0, 0, 0, 0};
                    const auto add = [&](const uint2 x, const uint2 y) {
                        f0[0] += (int16_t)(x.x & 0xFFFF); f0[1] += (int16_t)(x.x >> 16);
                        f0[2] += (int16_t)(x.y & 0xFFFF); f0[3] += (int16_t)(x.y >> 16);
                        f1[0] += (int16_t)(y.x & 0xFFFF); f1[1] += (int16_t)(y.x >> 16);
                        f1[2] += (int16_t)(y.y & 0xFFFF); f1[3] += (int16_t)(y.y >> 16);
                    };
                    const size_t o0 = (size_t)lc0 * kRows + r0, o1 = o0 + kRows;
                    if (a.KS == 4) {
                        // all eight remote loads issued before the first sum: one DSMEM round trip
                        uint2 x[4], y[4];
#pragma unroll
                        for (int src = 0; src < 4; ++src) {
                            const int16_t* rp = cluster.map_shared_rank(part, src);
                            x[src] = *reinterpret_cast<const uint2*>(rp + o0);
                            y[src] = *reinterpret_cast<const uint2*>(rp + o1);
                        }
#pragma unroll
                        for (int src = 0; src < 4; ++src) add(x[src], y[src]);
                    } else {
                        for (int src = 0; src < a.KS; ++src) {
                            const int16_t* rp = cluster.map_shared_rank(part, src);
                            add(*reinterpret_cast<const uint2*>(rp + o0), *reinterpret_cast<const uint2*>(rp + o1));
                        }
                    }
                    const int t0 = tb * NT + lc0;
                    const int i0 = rb * kRows + r0;
                    const uint32_t old0 = prev0[slot], old1 = prev1[slot];
                    uint32_t n0 = 0u, n1 = 0u;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int i = i0 + k;
                        if (i < a.n) {
                            const int r = r0 + k;
                            const uint4 rw = slot == 0 ? s_rw[k * kEpi + tid]
                                                       : pbit_draws2((uint32_t)i, (uint32_t)step, a.instance,
                                                                     (uint32_t)t0, a.seed_lo, a.seed_hi);
                            const float lam = s_lam[r], del = s_del[r];
                            const uint32_t thr = s_thr[r];
                            const int D0 = s_h[r] + f0[k];
                            const int D1 = s_h[r] + f1[k];
                            const uint32_t k0 = pbit_kthr_of_x(pbit_input(a.offset_mode, I0, lam, del, D0));
                            const uint32_t k1 = pbit_kthr_of_x(pbit_input(a.offset_mode, I0, lam, del, D1));
                            const int s0 = pbit_next(rw.x, rw.y, k0, thr, ((old0 >> (8 * k)) & 0xFF) == kE4m3Plus1 ? 1 : -1);
                            const int s1 = pbit_next(rw.z, rw.w, k1, thr, ((old1 >> (8 * k)) & 0xFF) == kE4m3Plus1 ? 1 : -1);
                            n0 |= (uint32_t)(s0 > 0 ? kE4m3Plus1 : kE4m3Minus1) << (8 * k);
                            n1 |= (uint32_t)(s1 > 0 ? kE4m3Plus1 : kE4m3Minus1) << (8 * k);
                        }
                    }
                    prev0[slot] = n0;
                    prev1[slot] = n1;
                    *reinterpret_cast<uint32_t*>(nxt + spin_off(t0, i0, a.T)) = n0;
                    *reinterpret_cast<uint32_t*>(nxt + spin_off(t0 + 1, i0, a.T)) = n1;
                }
            }
        }
        // Publish this CTA's new spins: the epilogue warps meet at a named
        // barrier (the control warp is not part of it), then one thread makes
        // their stores visible device-wide and raises the CTA's flag.  No
        // second cluster barrier: the partial buffers alternate between steps,
        // and a peer reads this step's buffer before it reaches the next
        // step's cluster barrier, which this CTA passes before writing the
        // same buffer again.
        // The release store is cumulative: it orders every epilogue thread's
        // stores (ordered before it by the named barrier) before the flag; the
        // consumer acquires the flag and fences the async proxy before its bulk copy.
        if (!control) {
            asm volatile("bar.sync 1, %0;" ::"r"(kEpi) : "memory");
            if (tid == 0 && !(pa.withhold && ks == 0 && rb == 0 && tb == pa.tb_base))
                st_release(pa.done + ((size_t)tb * RB + rb) * a.KS + ks, (unsigned)(ls + 1));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
    // The last step's epilogue reads every peer's partials through distributed shared memory and
    // no step follows whose cluster barrier would hold the peers: a CTA leaves only once every CTA
    // of its cluster is done with them (a CTA whose wait gave up skips its epilogue and would
    // otherwise leave first).
    cluster.sync();
}

size_t persist_smem_bytes(int NT) {
    return 128 + (size_t)kRows * kSlice + (size_t)NT * kSlice + 2 * (size_t)NT * kRows * sizeof(int16_t) +
           (size_t)kRows * 16 + (size_t)4 * kEpi * sizeof(uint4) + 64;
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

// cut_t = (S_t + 2W)/4 and H_t = -S_t/2 (h = 0) from S_t = sum_i s_it (J s)_it.
__global__ void finish_dense_observe(long long* v, int32_t T, long long two_w, int energy) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < T) v[t] = energy ? -(v[t] / 2) : (v[t] + two_w) / 4;
}

size_t dense_smem_bytes(int NT) {
    return 128 + (size_t)kRows * kSlice + (size_t)NT * kSlice + (size_t)kRows * (NT + kPad) * sizeof(float) + 64;
}

__host__ __device__ uint8_t e4m3_of_int(int v) {
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
        if (why) *why = "graph was created without PBIT_GRAPH_DENSE";
        return false;
    }
    if (T % 32 != 0 || (T > kMaxNT && T % kMaxNT != 0)) {
        if (why) *why = "dense kernel needs trials % 32 == 0 and (trials <= 128 or trials % 128 == 0)";
        return false;
    }
    return true;
}

// One block per row of J: scatter the row's CSR entries, as e4m3 bytes, into the MMA tile order
// (the zero-filled buffer holds e4m3 zeros elsewhere).
__global__ void dense_operand_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                     const int8_t* __restrict__ J, int32_t KS, uint8_t* __restrict__ tiles) {
    const int i = blockIdx.x;
    const int rb = i / kRows, rg = (i % kRows) >> 3, rr = i & 7;
    const size_t row_base = (size_t)rb * KS * (size_t)(kRows * kSlice) + (size_t)rg * (kCores * 128) + (size_t)rr * 16;
    for (int k = row_ptr[i] + threadIdx.x; k < row_ptr[i + 1]; k += blockDim.x) {
        const int j = col[k];
        const int ks = j / kSlice, c = (j % kSlice) >> 4, b = j & 15;
        tiles[row_base + (size_t)ks * (size_t)(kRows * kSlice) + (size_t)c * 128 + b] = e4m3_of_int(J[k]);
    }
}

pbit_status build_dense_operand(Graph& g) {
    const int n_pad = ((g.n + kSlice - 1) / kSlice) * kSlice;
    const int KS = n_pad / kSlice;
    if (KS > 16) return fail(PBIT_E_INVALID, "dense operand: n > 8192 is not supported by the tensor-core path");
    if (g.max_abs_J > 16) return fail(PBIT_E_INVALID, "dense operand: |w| > 16 is not exact in e4m3");
    const size_t bytes = (size_t)n_pad * n_pad;
    cudaError_t e = cudaMalloc((void**)&g.dense.J_e4m3, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(dense J)");
    e = cudaMemset(g.dense.J_e4m3, 0, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(dense J)");
    if (g.n > 0 && g.nnz > 0) {
        dense_operand_kernel<<<(unsigned)g.n, 256>>>(g.row_ptr, g.col, g.J, KS, g.dense.J_e4m3);
        count_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "dense operand kernel");
        if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, "dense operand kernel");
    }
    g.dense.n_pad = n_pad;
    g.dense.bytes = bytes;
    g.device_bytes += bytes;
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
                              int32_t* fields_out, int* err, cudaStream_t st, unsigned long long* obs_out) {
    DenseArgs a{};
    a.Jt = g.dense.J_e4m3;
    a.s_in = tin;
    a.s_out = tout;
    a.fields_out = fields_out;
    a.obs_out = obs_out;
    a.h = g.h;
    a.par = sa.par;
    a.i0_table = sa.i0_table;
    a.step = sa.step;
    a.n = g.n;
    a.T = sa.T;
    a.NT = sa.T <= kMaxNT ? sa.T : kMaxNT;
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

// Persistent launch over steps [b, e): returns cudaErrorNotSupported (nothing
// launched) when the clusters cannot all be resident at once.
cudaError_t launch_dense_persistent(const Graph& g, const StepArgs& sa, uint8_t* buf0, uint8_t* buf1, int32_t b,
                                    int32_t e, unsigned* done, int* err, cudaStream_t st) {
    PersistArgs pa{};
    DenseArgs& a = pa.d;
    a.Jt = g.dense.J_e4m3;
    a.h = g.h;
    a.par = sa.par;
    a.i0_table = sa.i0_table;
    a.n = g.n;
    a.T = sa.T;
    a.NT = sa.T <= kMaxNT ? sa.T : kMaxNT;
    a.KS = g.dense.n_pad / kSlice;
    a.seed_lo = sa.seed_lo;
    a.seed_hi = sa.seed_hi;
    a.instance = sa.instance;
    a.offset_mode = sa.offset_mode;
    a.err = err;
    pa.buf0 = buf0;
    pa.buf1 = buf1;
    pa.step_begin = b;
    pa.step_end = e;
    pa.done = done;
    const TestFault tf = test_fault("dense", 1ll << 31);
    pa.wait_cycles = tf.wait_cycles;
    pa.withhold = tf.withhold;
    const size_t smem = persist_smem_bytes(a.NT);
    cudaError_t ce = cudaFuncSetAttribute(dense_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem);
    if (ce != cudaSuccess) return ce;
    if (a.KS > 8) {
        ce = cudaFuncSetAttribute(dense_persistent_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (ce != cudaSuccess) return ce;
    }
    cudaLaunchConfig_t cfg{};
    const int RB = g.dense.n_pad / kRows, TB = sa.T / a.NT;
    cfg.gridDim = dim3((unsigned)a.KS, (unsigned)RB, (unsigned)TB);
    cfg.blockDim = dim3(kPersistThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)a.KS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int max_clusters = 0;
    ce = cudaOccupancyMaxActiveClusters(&max_clusters, dense_persistent_kernel, &cfg);
    if (ce != cudaSuccess) return ce;
    // Every CTA of one launch must be resident at once (they wait on one another's flags).  Trial
    // blocks never interact, so when they do not all fit, consecutive groups of trial blocks run as
    // separate launches over the whole step range, each on its own trial columns and flags.
    const int per_launch = std::min(TB, max_clusters / RB);
    if (per_launch < 1) return cudaErrorNotSupported;
    for (int g0 = 0; g0 < TB; g0 += per_launch) {
        pa.tb_base = g0;
        cfg.gridDim.z = (unsigned)std::min(per_launch, TB - g0);
        ce = cudaLaunchKernelEx(&cfg, dense_persistent_kernel, pa);
        count_launches(1);
        if (ce != cudaSuccess) return ce;
    }
    return cudaSuccess;
}

cudaError_t launch_dense_cut_energy(const Graph& g, const int8_t* spins, int32_t T, int64_t* out, bool energy,
                                    uint8_t* tiled_scratch, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int64_t) * (size_t)T, st);
    if (e != cudaSuccess) return e;
    if ((e = launch_to_tiled(g, spins, T, tiled_scratch, st)) != cudaSuccess) return e;
    StepArgs sa{};
    sa.T = T;
    if ((e = launch_dense_step(g, sa, tiled_scratch, nullptr, nullptr, g.err, st,
                               reinterpret_cast<unsigned long long*>(out))) != cudaSuccess)
        return e;
    finish_dense_observe<<<(T + 255) / 256, 256, 0, st>>>(reinterpret_cast<long long*>(out), T,
                                                           2 * (long long)g.total_weight, energy ? 1 : 0);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pbit
