// Dense field on the tcgen05 tensor cores with packed FP4 operands and one
// thread-block cluster per group of trials: the whole anneal runs without any
// grid-wide dependency.
//
// Field (Eq. conv): D = J * M for a dense J (n x n) and the spins of the
// trials.  J and the spins are held as packed e2m1 (FP4: sign, two exponent
// bits, one mantissa bit; two nodes per byte) and contracted by
// tcgen05.mma kind::mxf4 with every block scale factor equal to 1 (UE8M0
// 0x7F) and an FP32 accumulator in tensor memory.  It is exact: e2m1 holds
// the integers 0, +-1, +-2, +-3, +-4 and +-6, a spin is +-1, so every product
// is one of those integers and every partial sum is an integer of magnitude
// at most 6 * 2048 < 2^14, far inside FP32's exact-integer range.
//
// Work decomposition (one launch for the whole step range):
//   cluster = C CTAs (C = ceil(n / 128) <= 16), one cluster per group of N
//   trials (N = 32 or 48; grid = (C, groups)); GB300 keeps 7 clusters of 16
//   CTAs resident, so 256 trials run as 6 groups of 48 in one wave.  CTA r of
//   a cluster holds rows 128r..128r+127 of J over all K = 128C columns in
//   shared memory for the whole anneal (64K bytes: 128 KB at n = 2048) and two
//   buffers of the group's spins in the MMA's B layout (K x N nibbles each).
//   Per step:
//     1. two issuing threads (one per MMA warp) wait until all C slices of
//        the step's spins have arrived in the current buffer, each issues
//        half of the K/64 MMAs (M = 128, N, K = 64; even / odd K chunks)
//        into its own TMEM accumulator and commits them to one mbarrier;
//     2. the epilogue warps (N/4 of them: warp w reads TMEM lanes 32(w%4)..
//        and the 16 trial columns 16(w/4).. of both accumulators, whose
//        sum is exact) take the p-bit decisions
//        (Eq. pbits_variability, timing draw; the Philox words and I0 were
//        drawn during the previous step's copies and MMAs), pack the new
//        spins of their 32 rows with warp ballots into this CTA's slice of
//        the other buffer (64N bytes), and
//     3. one thread stores that slice into a global staging slot (it stays
//        in L2) and loads it back with one multicast bulk load into the
//        same place of the other C-1 CTAs' buffers, completing on each
//        receiver's mbarrier (bytes counted).
//   A CTA's next step therefore waits only for the C-1 slices of its own
//   cluster; J and the spins stay in shared memory, and the only memory
//   traffic between the first and last step is the 64N-byte slice staging.
//   The spins of a step are written to the buffer the step does not read,
//   and a peer can only write a buffer again after this CTA's MMAs on it
//   have completed (its slice depends on this CTA's next slice), so two
//   buffers suffice; for the same reason a staging slot is reused only
//   after every peer has received what it held.  Measured step anatomy
//   (K_2000, 48 trials per cluster, cycles of one CTA, clock64 marks):
//   waiting for the slices 1.2K after the epilogue, 32 MMAs from two
//   issuers 1.5-2.2K (about 47 cycles of tensor time each at N = 48; the
//   issuers share their schedulers with the Philox draws of the next step)
//   and their tail 0.4K, TMEM read and decisions 3.3K, ballot packing and
//   the epilogue barrier 1.1K: about 8.2K in all.  One thread issues a
//   tcgen05.mma only every 66-87 cycles and a bulk copy about every 128,
//   hence two MMA issuers and the multicast: with one issuer the MMAs took
//   2.8K, and with C-1 shared::cta -> shared::cluster copies (45 KB into
//   and out of each SM per step) the slices came 3.3K after the epilogue.
//
// Layouts (no-swizzle K-major core matrices of 8 rows x 16 bytes = 8 x 32
// nodes; leading byte offset = distance of K-adjacent core matrices, stride
// byte offset = distance of the next 8 rows / trials):
//   J (global and shared), per row block r: [k core (K/32)][row group (16)][8][16 B]
//     LBO = 16 * 128 = 2048, SBO = 128
//   spins (shared B buffers): [k core (K/32)][trial group (N/8)][8][16 B]
//     LBO = 16N, SBO = 128; CTA r's slice = k cores 4r..4r+3 = 64N contiguous bytes
//   initial spins (global): the same per trial group, groups consecutive
// Within a byte the even node sits in the low nibble; A and B use the same
// packing, so the contraction does not depend on the convention.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "pbit_device.cuh"
#include "pbit_internal.h"

namespace cg = cooperative_groups;

namespace pbit {
namespace {

constexpr int kR = 128;                 // rows per CTA (MMA M)
constexpr int kMaxC = 16;               // CTAs per cluster
constexpr uint32_t kTmemCols = 256;     // two accumulators (<= 48 columns each) + scale factors
constexpr uint32_t kD1Col = 64;         // second accumulator (odd K chunks)
constexpr uint32_t kSfaCol = 128, kSfbCol = 160;
constexpr uint32_t kUnitScales = 0x7F7F7F7Fu;  // four UE8M0 scale factors equal to 2^0
constexpr long long kWaitBudget = 1ll << 31;   // clock64 cycles (about a second) before a wait gives up

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
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

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long budget) {
    const long long start = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - start > budget) return false;
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

// Bulk store of `bytes` from this CTA's shared memory to global memory, waited for (the data is in
// global memory when it returns).
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Bulk load from global memory into the same shared-memory offset `dst` of every CTA in `mask`, each
// completing `bytes` on its barrier at offset `bar`.
__device__ __forceinline__ void bulk_g2s_multicast(const void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                                   uint16_t mask) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster [%0], [%1], %2, [%3], "
        "%4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "h"(mask)
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
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

// Instruction descriptor of kind::mxf4 (block-scaled): A and B e2m1 (format 1), both K-major,
// N at bits 17-22 (N/8), scale factors UE8M0 (bit 23), M = 128 at bits 24-28 (M/16), scale-factor
// selectors 0, dense K = 64.  The accumulator of the block-scaled kinds is always FP32.
__host__ __device__ constexpr uint32_t idesc_mxf4(uint32_t n) {
    return (1u << 7) | (1u << 10) | ((n >> 3) << 17) | (1u << 23) | ((uint32_t)(kR >> 4) << 24);
}

__device__ __forceinline__ void mma_mxf4(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t tmem_sfa, uint32_t tmem_sfb, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %6, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%5], p;\n\t}" ::"r"(
            tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(tmem_sfa), "r"(tmem_sfb), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_st4(uint32_t taddr, uint32_t v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %1, %1, %1};" ::"r"(taddr), "r"(v) : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// The Philox words of one row's 16 trials t0 .. t0 + 15 (two groups of 8, t0 a
// multiple of 16): rw[j / 2] holds trials t0 + 2 (j / 2) and the next as (r0, u0, r1, u1).
__device__ __forceinline__ void draw16(const PhiloxHead& ph, uint32_t t0, uint32_t k0, uint32_t k1, uint4 (&rw)[8]) {
#pragma unroll
    for (int gq = 0; gq < 2; ++gq) {
        const PbitPairs8 d = pbit_pairs8(ph, t0 + 8u * gq, k0, k1);
#pragma unroll
        for (int q = 0; q < 4; ++q) rw[4 * gq + q] = d.p[q];
    }
}

// The p-bit input x of pbit_input for a field already held as an exact float (|D| < 2^24, so the
// value equals pbit_input's for the same integer field).
__device__ __forceinline__ float pbit_input_f(int mode, float I0, float lam, float del, float d) {
    if (mode == 1) return __fmul_rn(__fmul_rn(lam, I0), __fadd_rn(d, del));
    if (mode == 2) return __fmul_rn(lam, __fmaf_rn(I0, d, del));
    return __fmul_rn(I0, __fmaf_rn(lam, d, del));
}

// Bit m of the low byte of x moved to bit 4m (m = 0..7).
__device__ __forceinline__ uint32_t spread8(uint32_t x) {
    x &= 0xFFu;
    x = (x | (x << 12)) & 0x000F000Fu;
    x = (x | (x << 6)) & 0x03030303u;
    x = (x | (x << 3)) & 0x11111111u;
    return x;
}

// 16 bytes of e2m1 spins for 32 consecutive nodes of one trial: node m's nibble is 0x2 (+1) or
// 0xA (-1), bit m of `neg` set for -1.
__device__ __forceinline__ uint4 pack_row(uint32_t neg) {
    uint4 v;
    v.x = 0x22222222u | (spread8(neg) << 3);
    v.y = 0x22222222u | (spread8(neg >> 8) << 3);
    v.z = 0x22222222u | (spread8(neg >> 16) << 3);
    v.w = 0x22222222u | (spread8(neg >> 24) << 3);
    return v;
}

struct D4Args {
    const uint8_t* J4;        // packed e2m1 J, C row blocks of 64K bytes
    const uint8_t* B0;        // packed e2m1 start spins, groups of K*N/2 bytes
    uint8_t* stage;           // slice staging for the exchange: [group][buffer][rank] slices of 64N bytes
    const int8_t* s_in;       // int8 [n][T] start state (the old spins of the hold rule)
    int8_t* s_out;            // int8 [n][T] final state
    int32_t* fields_out;      // fields only: int32 [n][T] D = h + J s of the start state
    const int32_t* h;
    NodeParams par;
    const float* i0_table;
    int32_t step_begin, step_end;
    int32_t n, T, N, C;
    uint32_t seed_lo, seed_hi, instance;
    int32_t offset_mode;
    int* err;
    long long wait_cycles;    // clock64 budget of each mbarrier wait (about a second; shorter in tests)
    int32_t withhold;         // test-only: CTA 0 of the first cluster never sends its slice to CTA 1
};

// Shared memory: J rows (64K), two buffers of the FP4 spin operand (K N / 2 each), per-row
// parameters, five mbarriers and the TMEM address.
size_t d4_smem_bytes(int C, int N) {
    const size_t K = (size_t)kR * C;
    return 128 + 64 * K + K * (size_t)N + (size_t)kR * 16 + 8 * 5 + 16;
}

// Warps 0 .. E-1 (E = N/4: four lane quarters x N/16 groups of 16 trials) are the epilogue; warps E
// and E+1 issue the MMAs (even and odd K chunks into two accumulators: one thread issues a
// tcgen05.mma only every 66-87 cycles, while the tensor core needs about 47 for M = 128, N = 48,
// K = 64, so two issuers keep it busy).  Warp E also loads J.
template <int N>
__global__ void __launch_bounds__((N / 4 + 2) * 32, 1) dense4_cluster_kernel(D4Args a) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    const int C = a.C;
    const uint32_t K = (uint32_t)kR * C;
    const uint32_t bytesA = 64u * K, bytesB = K * (uint32_t)N / 2u, slice = 64u * (uint32_t)N;
    uint8_t* sA = smem;
    uint8_t* const sB0 = sA + bytesA;  // operand buffer b at sB0 + b * bytesB
    float* s_lam = (float*)(sB0 + 2 * (size_t)bytesB);
    float* s_del = s_lam + kR;
    uint32_t* s_thr = (uint32_t*)(s_del + kR);
    int32_t* s_h = (int32_t*)(s_thr + kR);
    // mbarriers: full[b] = every slice of operand buffer b is in (steps >= 1), then MMA done, J loaded,
    // start spins loaded
    uint64_t* full = (uint64_t*)(s_h + kR);
    uint64_t* bar_mma = full + 2;
    uint64_t* bar_j = bar_mma + 1;
    uint64_t* bar_b0 = bar_mma + 2;
    uint32_t* tmem_slot = (uint32_t*)(bar_mma + 3);
    __shared__ int s_abort;

    constexpr int E = N / 4;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool control = warp >= E;
    const uint32_t issuer = control ? (uint32_t)(warp - E) : 0u;
    const uint32_t rank = cg::this_cluster().block_rank();
    const int g = blockIdx.y;
    const int L = a.step_end - a.step_begin;
    const bool fields_only = a.fields_out != nullptr;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (warp == E && lane == 0) {
        for (int k = 0; k < 5; ++k) mbar_init(&full[k], &full[k] == bar_mma ? 2u : 1u);  // two MMA commits
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    for (int r = tid; r < kR; r += blockDim.x) {
        const int i = (int)rank * kR + r;
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
    // unit block scale factors for A and B (every byte 0x7F = 2^0), written by the four lane quarters
    if (warp < 4) {
        tmem_st4(tmem + ((uint32_t)(warp * 32) << 16) + kSfaCol, kUnitScales);
        tmem_st4(tmem + ((uint32_t)(warp * 32) << 16) + kSfbCol, kUnitScales);
        tmem_wait_st();
    }
    tc_fence_before();
    // every CTA's barriers are initialised before any peer may copy into it
    cluster_sync_all();
    tc_fence_after();

    if (warp == E && lane == 0) {
        // J rows of this CTA (stationary) and the group's start spins
        mbar_arrive_expect_tx(bar_j, bytesA);
        const uint8_t* gA = a.J4 + (size_t)rank * bytesA;
        for (uint32_t off = 0; off < bytesA; off += 65536u)
            bulk_g2s(sA + off, gA + off, min(65536u, bytesA - off), bar_j);
        mbar_arrive_expect_tx(bar_b0, bytesB);
        const uint8_t* gB = a.B0 + (size_t)g * bytesB;
        for (uint32_t off = 0; off < bytesB; off += 65536u)
            bulk_g2s(sB0 + off, gB + off, min(65536u, bytesB - off), bar_b0);
        if (!mbar_wait_bounded(bar_j, 0, a.wait_cycles)) {
            atomicExch(a.err, 11);
            s_abort = 1;
        }
    }

    // epilogue geometry: row rr of this CTA (one k core of 32 rows per warp), trials c0 .. c0 + 15
    const int quarter = warp & 3;
    const int rr = quarter * 32 + lane;
    const int i = (int)rank * kR + rr;
    const int c0 = (warp >> 2) * 16;
    const int t0 = g * N + c0;           // first global trial of this thread
    uint32_t neg = 0;                    // bit j: trial t0 + j is -1 (the current state)
    uint4 rw[8];                         // Philox words of the step about to be decided
    float I0 = 0.0f;                     // I0 of the step about to be decided
    float lam = 1.0f, del = 0.0f, hf = 0.0f;
    uint32_t thr = 1u << 24;
    int hi = 0;
    if (!control) {
        lam = s_lam[rr];
        del = s_del[rr];
        thr = s_thr[rr];
        hi = s_h[rr];
        hf = (float)hi;
        if (i < a.n && !fields_only) {
            for (int j = 0; j < 16; ++j) {
                const int t = t0 + j;
                if (t < a.T && a.s_in[(size_t)i * a.T + t] < 0) neg |= 1u << j;
            }
        }
        if (L > 0) {
            I0 = a.i0_table[a.step_begin];
            const PhiloxHead ph = philox_head((uint32_t)i, (uint32_t)a.step_begin, a.instance, a.seed_lo, a.seed_hi);
            draw16(ph, (uint32_t)t0, a.seed_lo, a.seed_hi, rw);
        }
    }
    const uint32_t idesc = idesc_mxf4((uint32_t)N);
    const uint32_t lboA = 2048u, lboB = 16u * (uint32_t)N;
    const int mma_steps = fields_only ? 1 : L;

    bool good = true;  // this thread's work of every step completed
    for (int ls = 0; ls < mma_steps; ++ls) {
        const int buf = ls & 1;
        if (control) {
            // lane 0 of each MMA warp issues; the warp leaves the loop as a whole once a wait gave up
            uint32_t ok = 1;
            if (lane == 0) {
                ok = s_abort == 0 ? 1u : 0u;
                // the second issuer checks for J itself (warp E waited for it before the loop)
                if (ok && ls == 0 && issuer == 1) ok = mbar_wait_bounded(bar_j, 0, a.wait_cycles) ? 1u : 0u;
                // step 0 reads the start spins; step ls >= 1 the C slices of buffer ls & 1
                if (ok) ok = (ls == 0 ? mbar_wait_bounded(bar_b0, 0, a.wait_cycles)
                                      : mbar_wait_bounded(&full[buf], (uint32_t)(((ls - 1) >> 1) & 1), a.wait_cycles)) ? 1u : 0u;
                if (ok) {
                    tc_fence_after();
                    // K chunks issuer, issuer + 2, ... (K / 64 = 2C is even) into accumulator `issuer`; the
                    // descriptors advance by two chunks (start address field in 16-byte units)
                    const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB0 + (size_t)buf * bytesB);
                    const uint64_t dA = smem_desc(a0 + issuer * 2 * lboA, lboA, 128);
                    const uint64_t dB = smem_desc(b0 + issuer * 2 * lboB, lboB, 128);
                    const uint32_t d = tmem + issuer * kD1Col;
                    for (uint32_t j = 0; j < K / 128; ++j)
                        mma_mxf4(d, dA + (uint64_t)(j * (lboA >> 2)), dB + (uint64_t)(j * (lboB >> 2)), idesc,
                                 tmem + kSfaCol, tmem + kSfbCol, j > 0 ? 1u : 0u);
                    mma_commit(bar_mma);
                } else if (s_abort == 0) {
                    atomicExch(a.err, 12);
                }
            }
            if (__shfl_sync(0xFFFFFFFFu, ok, 0) == 0) break;
            continue;
        }
        // ---- epilogue: wait (bounded) for this step's MMAs; the outcome is made uniform per warp
        uint32_t okw = 1;
        if (lane == 0) okw = mbar_wait_bounded(bar_mma, (uint32_t)(ls & 1), a.wait_cycles) ? 1u : 0u;
        okw = __shfl_sync(0xFFFFFFFFu, okw, 0);
        if (!okw) {
            good = false;
            if (lane == 0) atomicExch(a.err, 13);
        }
        uint32_t v[16];
        if (okw) {
            tc_fence_after();
            uint32_t v1[16];
            tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, v);
            tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + kD1Col + (uint32_t)c0, v1);
            tmem_wait_ld();
            // the two partial sums are integers below 2^14 in magnitude: the float sum is exact
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = __float_as_uint(__fadd_rn(__uint_as_float(v[j]), __uint_as_float(v1[j])));
        }
        tc_fence_before();
        if (fields_only) {
            if (okw && i < a.n) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int t = t0 + j;
                    if (t < a.T) a.fields_out[(size_t)i * a.T + t] = hi + __float2int_rn(__uint_as_float(v[j]));
                }
            }
            break;
        }
        const int step = a.step_begin + ls;
        if (okw) {
            uint32_t nneg = 0;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                // D = h + (J s), both exact integers below 2^24: one float addition, no conversions
                const float D = __fadd_rn(hf, __uint_as_float(v[j]));
                const uint32_t kthr = pbit_kthr_of_x(pbit_input_f(a.offset_mode, I0, lam, del, D));
                const uint4 w = rw[j >> 1];
                const int old = (neg >> j) & 1u ? -1 : 1;
                const int s = (j & 1) ? pbit_next(w.z, w.w, kthr, thr, old) : pbit_next(w.x, w.y, kthr, thr, old);
                nneg |= (s < 0 ? 1u : 0u) << j;
            }
            neg = nneg;
        }
        if (ls + 1 == L) break;
        const uint32_t nb = (uint32_t)(buf ^ 1);
        uint8_t* dstB = sB0 + (size_t)nb * bytesB;
        if (okw) {
            // this warp's 32 rows are one k core (kc = 4 rank + quarter); lane j < 16 writes trial c0 + j
            uint32_t mine = 0;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const uint32_t bj = __ballot_sync(0xFFFFFFFFu, (neg >> j) & 1u);
                if (lane == j) mine = bj;
            }
            if (lane < 16) {
                const int tl = c0 + lane;
                const uint32_t kc = 4u * rank + (uint32_t)quarter;
                *reinterpret_cast<uint4*>(dstB + kc * lboB + (uint32_t)(tl >> 3) * 128u + (uint32_t)(tl & 7) * 16u) =
                    pack_row(mine);
            }
            fence_proxy_async_smem();
        }
        // every epilogue warp meets here each step; a failure anywhere stops all of them together
        uint32_t any_fail;
        asm volatile(
            "{\n\t.reg .pred q, p;\n\t"
            "setp.eq.u32 q, %1, 0;\n\t"
            "bar.red.or.pred p, 1, %2, q;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(any_fail)
            : "r"(okw), "r"(E * 32)
            : "memory");
        if (any_fail) {
            good = false;
            break;
        }
        if (warp == 0 && lane == 0) {
            // This CTA's slice goes to the peers in two bulk operations: a store into its global staging
            // slot (group, buffer, rank), then one load from there multicast into the same place of
            // the C-1 peers' buffers, completing on each peer's barrier.  Measured against C-1
            // shared::cta -> shared::cluster copies (45 KB leaving and entering each SM per step at
            // K_2000, 48 trials): the slices are in 1.2K instead of 3.3K cycles after the epilogue.
            uint64_t* nfull = &full[nb];
            const uint8_t* src = dstB + rank * slice;
            mbar_arrive_expect_tx(nfull, slice * (uint32_t)(C - 1));  // the C-1 peers' slices
            uint8_t* stage = a.stage + (((size_t)g * 2 + nb) * (size_t)C + rank) * slice;
            bulk_s2g(stage, src, slice);
            uint32_t mask = ((1u << C) - 1u) & ~(1u << rank);
            if (a.withhold && g == 0 && rank == 0) mask &= ~2u;  // test-only: CTA 1 never gets this slice
            bulk_g2s_multicast(src, stage, slice, nfull, (uint16_t)mask);
        }
        // I0 and the Philox words of the next step, drawn while the copies and the next MMAs run
        I0 = a.i0_table[step + 1];
        const PhiloxHead ph = philox_head((uint32_t)i, (uint32_t)(step + 1), a.instance, a.seed_lo, a.seed_hi);
        draw16(ph, (uint32_t)t0, a.seed_lo, a.seed_hi, rw);
    }
    // final state of this thread's row and trials (left untouched when a wait gave up: the result of
    // that call is undefined and PBIT_E_TIMEOUT reports it)
    if (!control && !fields_only && good && i < a.n) {
        for (int j = 0; j < 16; ++j) {
            const int t = t0 + j;
            if (t < a.T) a.s_out[(size_t)i * a.T + t] = ((neg >> j) & 1u) ? (int8_t)-1 : (int8_t)1;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
    // no CTA leaves while a peer may still copy into its shared memory
    cluster_sync_all();
}

// int8 trial-major [n][T] -> packed e2m1 start spins, groups of N trials: one thread per
// (group, k core, trial) 16-byte row.  Nodes >= n and trials >= T are written as 0.
__global__ void to_fp4_spins_kernel(const int8_t* __restrict__ s, int32_t n, int32_t T, int32_t K, int32_t N,
                                    int32_t groups, uint8_t* __restrict__ out) {
    const int64_t rows = (int64_t)groups * (K / 32) * N;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < rows;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int tl = (int)(idx % N);
        const int kc = (int)((idx / N) % (K / 32));
        const int g = (int)(idx / ((int64_t)N * (K / 32)));
        const int t = g * N + tl;
        uint32_t w[4] = {0, 0, 0, 0};
        for (int m = 0; m < 32; ++m) {
            const int j = kc * 32 + m;
            uint32_t nib = 0;
            if (j < n && t < T) nib = s[(size_t)j * T + t] < 0 ? 0xAu : 0x2u;
            w[m >> 3] |= nib << (4 * (m & 7));
        }
        uint8_t* dst = out + (size_t)g * ((size_t)K * N / 2) + (size_t)kc * 16 * N + (size_t)(tl >> 3) * 128 +
                       (size_t)(tl & 7) * 16;
        *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

__host__ __device__ uint32_t e2m1_of_int(int v) {
    const uint32_t sign = v < 0 ? 0x8u : 0u;
    const int a = v < 0 ? -v : v;
    const uint32_t mag = a == 0 ? 0u : a == 1 ? 0x2u : a == 2 ? 0x4u : a == 3 ? 0x5u : a == 4 ? 0x6u : 0x7u;  // 6
    return a == 0 ? 0u : (sign | mag);
}

// One block per row of J: OR each entry's nibble into the zero-filled operand (two nodes share a
// byte, so 32-bit atomic ORs).
__global__ void dense4_operand_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                      const int8_t* __restrict__ J, int32_t K, uint8_t* __restrict__ tiles) {
    const int i = blockIdx.x;
    const int rb = i / kR, rg = (i % kR) >> 3, r8 = i & 7;
    const size_t row_base = (size_t)rb * 64 * K + (size_t)rg * 128 + (size_t)r8 * 16;
    for (int k = row_ptr[i] + threadIdx.x; k < row_ptr[i + 1]; k += blockDim.x) {
        const int j = col[k];
        const size_t byte = row_base + (size_t)(j >> 5) * 2048 + (size_t)((j & 31) >> 1);
        const uint32_t nib = e2m1_of_int(J[k]) << (4 * (j & 1));
        unsigned int* word = reinterpret_cast<unsigned int*>(tiles + (byte & ~(size_t)3));
        atomicOr(word, nib << (8 * (byte & 3)));
    }
}

bool e2m1_exact(int v) {
    const int a = v < 0 ? -v : v;
    return a <= 4 || a == 6;
}

}  // namespace

// ------------------------------------------------------------- host side ----

bool dense4_shape_ok(const Graph& g, int32_t T) {
    // PBIT_DENSE_E4M3 forces the e4m3 kernel (tests); read on every call so a process can switch
    return g.dense4.J4 && T % 16 == 0 && std::getenv("PBIT_DENSE_E4M3") == nullptr;
}

pbit_status build_dense4_operand(Graph& g) {
    if (g.n < 1 || g.n > kR * kMaxC) return PBIT_OK;  // not applicable: the e4m3 path serves it
    for (int8_t v : g.h_J)
        if (!e2m1_exact(v)) return PBIT_OK;
    const int C = (g.n + kR - 1) / kR;
    const int K = kR * C;
    const size_t bytes = (size_t)C * 64 * (size_t)K;
    cudaError_t e = cudaMalloc((void**)&g.dense4.J4, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(fp4 dense J)");
    e = cudaMemset(g.dense4.J4, 0, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(fp4 dense J)");
    if (g.nnz > 0) {
        dense4_operand_kernel<<<(unsigned)g.n, 256>>>(g.row_ptr, g.col, g.J, K, g.dense4.J4);
        count_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "fp4 dense operand kernel");
        if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, "fp4 dense operand kernel");
    }
    g.dense4.C = C;
    g.dense4.bytes = bytes;
    g.device_bytes += bytes;
    return PBIT_OK;
}

template <int N>
static int max_clusters_d4(int C);

// Trials per cluster N (32 or 48, the buffers must fit one CTA's shared memory): the smallest N
// whose groups all run at once (ceil(T / N) clusters co-resident), else the largest N that fits.
static int dense4_group(const Graph& g, int32_t T) {
    int dev = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int best = 0;
    for (int N : {32, 48}) {
        if (d4_smem_bytes(g.dense4.C, N) + 256 > (size_t)smem_max) continue;  // + static shared memory
        best = N;
        const int m = N == 32 ? max_clusters_d4<32>(g.dense4.C) : max_clusters_d4<48>(g.dense4.C);
        if (m >= (T + N - 1) / N) return N;
    }
    return best;
}

// Scratch of one launch: the packed start spins (K N / 2 bytes per group), then the slice staging
// (two buffers of C slices of 64N bytes per group: K N bytes).
size_t dense4_spin_bytes(const Graph& g, int32_t T) {
    const int N = dense4_group(g, T);
    if (N == 0) return 0;
    const int groups = (T + N - 1) / N;
    return (size_t)groups * (size_t)(kR * g.dense4.C) * (size_t)N * 3 / 2;
}

template <int N>
static cudaError_t d4_config(int C, cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr) {
    const size_t smem = d4_smem_bytes(C, N);
    cudaError_t ce = cudaFuncSetAttribute(dense4_cluster_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem);
    if (ce != cudaSuccess) return ce;
    if (C > 8) {
        ce = cudaFuncSetAttribute(dense4_cluster_kernel<N>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (ce != cudaSuccess) return ce;
    }
    cfg.blockDim = dim3((unsigned)(N / 4 + 2) * 32, 1, 1);
    cfg.dynamicSmemBytes = smem;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaSuccess;
}

template <int N>
static cudaError_t launch_d4(const D4Args& a, cudaStream_t st) {
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    cudaError_t ce = d4_config<N>(a.C, cfg, attr);
    if (ce != cudaSuccess) return ce;
    cfg.gridDim = dim3((unsigned)a.C, (unsigned)((a.T + N - 1) / N), 1);
    cfg.stream = st;
    int max_clusters = 0;
    ce = cudaOccupancyMaxActiveClusters(&max_clusters, dense4_cluster_kernel<N>, &cfg);
    if (ce != cudaSuccess) return ce;
    if (max_clusters < 1) return cudaErrorNotSupported;
    ce = cudaLaunchKernelEx(&cfg, dense4_cluster_kernel<N>, a);
    count_launches(1);
    return ce;
}

template <int N>
static int max_clusters_d4(int C) {
    // cached per (device, C): an occupancy query per anneal would cost more than a short anneal
    static std::mutex mu;
    static std::map<std::pair<int, int>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find({dev, C});
    if (it != cache.end()) return it->second;
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    int m = 0;
    if (d4_config<N>(C, cfg, attr) == cudaSuccess) {
        cfg.gridDim = dim3((unsigned)C, 1, 1);
        if (cudaOccupancyMaxActiveClusters(&m, dense4_cluster_kernel<N>, &cfg) != cudaSuccess) m = 0;
    }
    cache[{dev, C}] = m;
    return m;
}

cudaError_t launch_dense4(const Graph& g, const StepArgs& sa, const int8_t* s_in, int8_t* s_out, int32_t* fields_out,
                          uint8_t* b0_scratch, int32_t b, int32_t e, cudaStream_t st) {
    const int N = dense4_group(g, sa.T);
    if (N == 0) return cudaErrorNotSupported;
    const int C = g.dense4.C, K = kR * C;
    const int groups = (sa.T + N - 1) / N;
    to_fp4_spins_kernel<<<152 * 4, 256, 0, st>>>(s_in, g.n, sa.T, K, N, groups, b0_scratch);
    count_launches(1);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) return ce;
    D4Args a{};
    a.J4 = g.dense4.J4;
    a.B0 = b0_scratch;
    a.stage = b0_scratch + (size_t)groups * K * N / 2;
    a.s_in = s_in;
    a.s_out = s_out;
    a.fields_out = fields_out;
    a.h = g.h;
    a.par = sa.par;
    a.i0_table = sa.i0_table;
    a.step_begin = b;
    a.step_end = e;
    a.n = g.n;
    a.T = sa.T;
    a.N = N;
    a.C = C;
    a.seed_lo = sa.seed_lo;
    a.seed_hi = sa.seed_hi;
    a.instance = sa.instance;
    a.offset_mode = sa.offset_mode;
    a.err = g.err;
    const TestFault tf = test_fault("dense4", kWaitBudget);
    a.wait_cycles = tf.wait_cycles;
    a.withhold = tf.withhold;
    return N == 48 ? launch_d4<48>(a, st) : launch_d4<32>(a, st);
}

int dense4_max_active_clusters(const Graph& g, int32_t T) {
    const int N = dense4_group(g, T);
    if (N == 0 || !g.dense4.J4) return 0;
    return N == 48 ? max_clusters_d4<48>(g.dense4.C) : max_clusters_d4<32>(g.dense4.C);
}

}  // namespace pbit
