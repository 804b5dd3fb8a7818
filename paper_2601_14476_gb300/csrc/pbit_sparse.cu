// Sparse (CSR) kernels: initial state, one synchronous pSA step, the
// single-CTA resident anneal, exact fields, cut and energy.
//
// Spins are trial-major int8 [n][T]: the T trials of node j are contiguous,
// so the gather of neighbour j for a group of G consecutive trials is one
// vector load (G = 16: int4, G = 4: 32-bit, G = 1: byte), coalesced across
// the threads of a warp that share the node.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdlib>
#include <vector>

#include "pbit_device.cuh"
#include "pbit_internal.h"
#include "pbit_tile.cuh"

namespace pbit {
namespace {

namespace cg = cooperative_groups;

using namespace tile;

// ------------------------------------------------------------------ init ----
__global__ void init_spins_kernel(int32_t n, int32_t T, uint32_t k0, uint32_t k1, uint32_t instance,
                                  int8_t* __restrict__ spins) {
    const int64_t total = (int64_t)n * T;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / T), t = (int)(idx - (int64_t)i * T);
        const uint32_t wr = pbit_rword((uint32_t)i, 0xFFFFFFFFu, instance, (uint32_t)t, k0, k1);
        spins[idx] = ((wr >> 8) < (1u << 23)) ? 1 : -1;  // +1 iff r < 0
    }
}

// --------------------------------------------------------- failure path ----
// Waits (bounded by the global nanosecond timer) on a flag that nothing sets,
// then records the timeout code in the error word and returns: the same exit
// path every bounded wait of the library takes.
__global__ void bounded_wait_selftest_kernel(const unsigned* flag, long long budget_ns, int* err) {
    if (threadIdx.x != 0) return;
    unsigned long long start, now;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(start));
    for (;;) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
        if (v != 0u) return;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
        if ((long long)(now - start) > budget_ns) {
            atomicExch(err, 5);
            return;
        }
    }
}

// ------------------------------------------------------------------ step ----
// Programmatic dependent launch between consecutive step launches: a step's grid may be scheduled
// while the previous one drains and waits (griddepcontrol.wait) until that grid has completed and
// its spins are visible.  Both instructions are no-ops in a launch without the attribute.
__device__ __forceinline__ void step_dependency() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <int G, bool UNIT, bool TABLE>
__global__ void __launch_bounds__(kBlock) sparse_step_kernel(StepArgs a) {
    __shared__ uint32_t s_tab[TABLE ? kTabMax : 1];
    step_dependency();
    process_tile<G, UNIT, TABLE>(a, blockIdx.x * (int64_t)kBlock, s_tab);
}

// Warp-table tile; six resident blocks per SM (40 registers): on the torus at T = 1024 this ran
// 33.5 µs per step, against 33.7 (five), 35.5 (four) and 36.2 (seven or eight, with spills).
template <int G, bool HALF>
__global__ void __launch_bounds__(kBlock, 6) sparse_warp_kernel(StepArgs a) {
    step_dependency();
    process_tile_warp<G, HALF>(a, blockIdx.x * (uint32_t)kBlock);
}

// A step launch with programmatic stream serialization, or a plain one when PBIT_NO_PDL is set or the
// attribute is refused.
template <typename K>
cudaError_t launch_step_pdl(K kernel, unsigned blocks, const StepArgs& a, cudaStream_t s) {
    static const bool off = std::getenv("PBIT_NO_PDL") != nullptr;
    if (!off) {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(blocks);
        cfg.blockDim = dim3(kBlock);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (cudaLaunchKernelEx(&cfg, kernel, a) == cudaSuccess) return cudaSuccess;
        (void)cudaGetLastError();  // clear the refusal, then launch plainly
    }
    kernel<<<blocks, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

template <int G, bool UNIT>
__global__ void __launch_bounds__(kBlock) sparse_variant_kernel(StepArgs a) {
    step_dependency();
    process_tile_variant<G, UNIT>(a, blockIdx.x * (int64_t)kBlock);
}

template <int G, bool UNIT>
cudaError_t launch_variant_g(const StepArgs& a, cudaStream_t s) {
    const int64_t threads = (int64_t)a.n * (a.T / G);
    const int64_t blocks = (threads + kBlock - 1) / kBlock;
    const cudaError_t e = launch_step_pdl(sparse_variant_kernel<G, UNIT>, (unsigned)blocks, a, s);
    count_launches(1);
    return e;
}

template <int G, bool UNIT, bool TABLE>
cudaError_t launch_step_g(const StepArgs& base, cudaStream_t s) {
    StepArgs a = base;
    set_group_divisor(a, G);
    const int64_t threads = (int64_t)a.n * (a.T / G);
    const int64_t blocks = (threads + kBlock - 1) / kBlock;
    const cudaError_t e = launch_step_pdl(sparse_step_kernel<G, UNIT, TABLE>, (unsigned)blocks, a, s);
    count_launches(1);
    return e;
}

template <int G, bool HALF>
cudaError_t launch_warp_g(const StepArgs& base, cudaStream_t s) {
    StepArgs a = base;
    set_group_divisor(a, G);
    const int64_t threads = (int64_t)a.n * (a.T / G);
    const int64_t blocks = (threads + kBlock - 1) / kBlock;
    const cudaError_t e = launch_step_pdl(sparse_warp_kernel<G, HALF>, (unsigned)blocks, a, s);
    count_launches(1);
    return e;
}

template <int G>
cudaError_t launch_step_variant(const StepArgs& a, cudaStream_t s, SparseVariant v) {
    if constexpr (G >= 4) {
        if (v.unit && v.table) return launch_step_g<G, true, true>(a, s);
        if (v.unit) return launch_step_g<G, true, false>(a, s);
    }
    if (v.table) return launch_step_g<G, false, true>(a, s);
    return launch_step_g<G, false, false>(a, s);
}

// -------------------------------------------------------------- resident ----
// All steps [b, e) of one small instance in one launch, the spins held in
// shared memory.  The CTAs of one thread-block cluster (8 when the cluster can
// be placed, else 1) each keep a full copy of both spin buffers: each updates
// the nodes it owns from its local copy and stores the new spins into its own
// next buffer and into every peer's (distributed shared memory); the cluster
// barrier (release / acquire) ends the step.  Nobody reads a buffer that is
// being written: a step writes the buffers read in the step before, and every
// CTA has finished reading those when it arrives at the barrier.
constexpr int kResidentThreads = 512;
constexpr size_t kResidentSmem = 200 * 1024;
constexpr int kResidentCluster = 8;

// UNIT (weights +-1, degree <= 127, G = 4): the field is counted four trials at a time as in the
// tiles (2 per neighbour with J_ij s_j = -1, one 32-bit shared-memory load per neighbour).
template <int G, bool UNIT>
__global__ void __launch_bounds__(kResidentThreads) resident_kernel(StepArgs a, int32_t step_begin, int32_t step_end) {
    extern __shared__ __align__(16) int8_t smem[];
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks(), r = (int)cluster.block_rank();
    const int64_t cells = (int64_t)a.n * a.T;
    int8_t* buf0 = smem;
    int8_t* buf1 = smem + ((cells + 15) / 16) * 16;
    for (int64_t c = threadIdx.x; c < cells; c += blockDim.x) buf0[c] = a.in[c];
    cluster.sync();  // every CTA runs (and holds the state) before any peer writes into it
    const int groups = a.T / G;
    const int node_lo = (int)((int64_t)a.n * r / C), node_hi = (int)((int64_t)a.n * (r + 1) / C);
    const int items = (node_hi - node_lo) * groups;  // < 2^31: both spin copies fit in shared memory
    int8_t* cur = buf0;
    int8_t* nxt = buf1;
    for (int32_t step = step_begin; step < step_end; ++step) {
        StepArgs sa = a;
        sa.step = step;
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            const int li = it / groups;
            const int i = node_lo + li;
            const int t0 = (it - li * groups) * G;
            int acc[G];
            if constexpr (UNIT && G == 4) {
                const int rb = __ldg(a.row_ptr + i), re = __ldg(a.row_ptr + i + 1);
                uint32_t cnt2 = 0;
                for (int e = rb; e < re; ++e) {
                    const int8_t* pj = cur + (size_t)__ldg(a.col + e) * a.T + t0;
                    const uint32_t flip = __ldg(a.J + e) < 0 ? 0x02020202u : 0u;
                    cnt2 += (*reinterpret_cast<const uint32_t*>(pj) & 0x02020202u) ^ flip;
                }
#pragma unroll
                for (int k = 0; k < G; ++k) acc[k] = (re - rb) - (int)((cnt2 >> (8 * k)) & 0xFFu);
            } else {
                gather_field<G>(a.row_ptr, a.col, a.J, cur, a.T, i, t0, acc);
            }
            uint32_t oldw[Pack<G>::W], neww[Pack<G>::W];
            const size_t off = (size_t)i * a.T + t0;
            load_group<G>(cur + off, oldw);
            decide_group<G>(sa, i, t0, acc, oldw, neww);
            store_group<G>(nxt + off, neww);
            for (int q = 1; q < C; ++q) store_group<G>(cluster.map_shared_rank(nxt, (r + q) % C) + off, neww);
        }
        cluster.sync();
        int8_t* tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    for (int64_t c = (int64_t)node_lo * a.T + threadIdx.x; c < (int64_t)node_hi * a.T; c += blockDim.x) a.out[c] = cur[c];
}

template <int G, bool UNIT>
cudaError_t launch_resident_g(const StepArgs& a, int32_t b, int32_t e, cudaStream_t s) {
    const int64_t cells = (int64_t)a.n * a.T;
    const size_t smem = 2 * (size_t)(((cells + 15) / 16) * 16);
    cudaError_t err = cudaFuncSetAttribute(resident_kernel<G, UNIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)kResidentSmem);
    if (err != cudaSuccess) return err;
    static const char* cl_env = std::getenv("PBIT_RESIDENT_CLUSTER");  // tests: 1 forces one CTA
    const int want = cl_env ? std::max(1, std::min(kResidentCluster, std::atoi(cl_env))) : kResidentCluster;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)want, 1, 1);
    cfg.blockDim = dim3(kResidentThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)want;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (want > 1 && cudaOccupancyMaxActiveClusters(&clusters, resident_kernel<G, UNIT>, &cfg) == cudaSuccess && clusters >= 1) {
        err = cudaLaunchKernelEx(&cfg, resident_kernel<G, UNIT>, a, b, e);
        count_launches(1);
        return err;
    }
    (void)cudaGetLastError();
    cfg.gridDim = dim3(1, 1, 1);
    attr[0].val.clusterDim.x = 1;
    err = cudaLaunchKernelEx(&cfg, resident_kernel<G, UNIT>, a, b, e);
    count_launches(1);
    return err;
}

// ---------------------------------------------------------------- fields ----
template <int G>
__global__ void __launch_bounds__(kBlock) fields_kernel(const int32_t* __restrict__ row_ptr,
                                                        const int32_t* __restrict__ col,
                                                        const int8_t* __restrict__ J, const int32_t* __restrict__ h,
                                                        const int8_t* __restrict__ spins, int32_t n, int32_t T,
                                                        int32_t* __restrict__ out) {
    const int groups = T / G;
    const int64_t tid = blockIdx.x * (int64_t)kBlock + threadIdx.x;
    if (tid >= (int64_t)n * groups) return;
    const int i = (int)(tid / groups);
    const int t0 = (int)(tid - (int64_t)i * groups) * G;
    int acc[G];
    gather_field<G>(row_ptr, col, J, spins, T, i, t0, acc);
    const int hi = h ? h[i] : 0;
#pragma unroll
    for (int k = 0; k < G; ++k) out[(size_t)i * T + t0 + k] = hi + acc[k];
}

// ------------------------------------------------------------ cut/energy ----
// Block = 8 warps over a slab of 32*G trials (lane l owns trials l*G..l*G+G-1
// of the slab) and a range of rows.  Per trial it accumulates
//   cut:    sum over directed CSR entries of J_ij (s_i s_j - 1)   (= 4 * cut)
//   energy: -2 h_i s_i - sum over directed entries J_ij s_i s_j   (= 2 * H)
// reduces across the warps in shared memory and adds one int64 per trial.
constexpr int kRowsPerBlock = 128;

template <int G>
__global__ void __launch_bounds__(kBlock) cut_energy_kernel(const int32_t* __restrict__ row_ptr,
                                                            const int32_t* __restrict__ col,
                                                            const int8_t* __restrict__ J,
                                                            const int32_t* __restrict__ h,
                                                            const int8_t* __restrict__ spins, int32_t n, int32_t T,
                                                            bool energy, unsigned long long* __restrict__ out) {
    __shared__ long long red[kBlock / 32][32 * G];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int t0 = blockIdx.y * 32 * G + lane * G;
    const bool active = t0 < T;
    long long acc[G];
#pragma unroll
    for (int k = 0; k < G; ++k) acc[k] = 0;
    const int r0 = blockIdx.x * kRowsPerBlock;
    const int r1 = min(n, r0 + kRowsPerBlock);
    if (active) {
        for (int i = r0 + warp; i < r1; i += kBlock / 32) {
            uint32_t own[Pack<G>::W];
            load_group<G>(spins + (size_t)i * T + t0, own);
            int part[G];
#pragma unroll
            for (int k = 0; k < G; ++k) part[k] = 0;
            const int rb = row_ptr[i], re = row_ptr[i + 1];
            for (int e = rb; e < re; ++e) {
                const int j = col[e];
                const int w = J[e];
                uint32_t v[Pack<G>::W];
                load_group<G>(spins + (size_t)j * T + t0, v);
#pragma unroll
                for (int k = 0; k < G; ++k) {
                    const int ss = sbyte(own[k >> 2], k & 3) * sbyte(v[k >> 2], k & 3);
                    part[k] += energy ? -w * ss : w * (ss - 1);
                }
            }
            const int hi = (energy && h) ? h[i] : 0;
#pragma unroll
            for (int k = 0; k < G; ++k) acc[k] += (long long)part[k] - 2LL * hi * sbyte(own[k >> 2], k & 3);
        }
    }
#pragma unroll
    for (int k = 0; k < G; ++k) red[warp][lane * G + k] = acc[k];
    __syncthreads();
    for (int c = threadIdx.x; c < 32 * G; c += kBlock) {
        long long s = 0;
#pragma unroll
        for (int w = 0; w < kBlock / 32; ++w) s += red[w][c];
        const int t = blockIdx.y * 32 * G + c;
        if (t < T) atomicAdd(out + t, (unsigned long long)s);
    }
}

__global__ void finish_cut_energy(long long* v, int32_t T, bool energy) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < T) v[t] = energy ? v[t] / 2 : v[t] / 4;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
bool aligned4(const void* p) { return ((uintptr_t)p & 3u) == 0; }

int group_size(const StepArgs& a) {
    if (a.T % 16 == 0 && aligned16(a.in) && aligned16(a.out)) return 16;
    if (a.T % 4 == 0 && aligned4(a.in) && aligned4(a.out)) return 4;
    return 1;
}

}  // namespace

// ------------------------------------------------------------- launchers ----
cudaError_t launch_init_spins(int32_t n, int32_t T, uint64_t seed, uint32_t instance, int8_t* spins,
                              cudaStream_t s) {
    const int64_t total = (int64_t)n * T;
    int64_t blocks = (total + kBlock - 1) / kBlock;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (blocks < 1) blocks = 1;
    init_spins_kernel<<<(unsigned)blocks, kBlock, 0, s>>>(n, T, (uint32_t)(seed & 0xFFFFFFFFu),
                                                           (uint32_t)(seed >> 32), instance, spins);
    count_launches(1);
    return cudaGetLastError();
}

// Trials per thread of the warp-table tile for T trials (0: the tile does not apply).  32 trials
// per thread need fewer instructions per update than 16, but give half the threads: a single
// instance takes 32 only when that still fills two waves of the multi-step launch's grid (6 blocks
// of 256 threads per SM); a batch (`wide`) gets its parallelism from its other instances.
int warp_tile_group(const Graph& g, int32_t T, bool wide) {
    if (!g.unit_weights || g.max_degree > 15) return 0;
    int fit32 = 0, fit16 = 0;
    for (const int G : {32, 16}) {
        if (T % G != 0) continue;
        const int64_t groups = T / G;
        if (groups % 32 != 0 && 32 % groups != 0) continue;
        const int64_t L = groups >= 32 ? 32 : groups;
        if ((int64_t)g.max_degree + 1 > L) continue;  // one lane per possible count
        if ((int64_t)g.n * groups >= (int64_t(1) << 31)) continue;
        (G == 32 ? fit32 : fit16) = 1;
    }
    static const int64_t two_waves = [] {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        return 2 * (int64_t)(sms > 0 ? sms : 152) * 6 * kBlock;
    }();
    if (fit32 && (wide || !fit16 || (int64_t)g.n * (T / 32) >= two_waves)) return 32;
    return fit16 ? 16 : 0;
}

SparseVariant choose_sparse_variant(const Graph& g, int32_t T) {
    SparseVariant v;
    static const bool plain = std::getenv("PBIT_SPARSE_PLAIN") != nullptr;  // force the plain variant
    if (plain) return v;
    static const bool no_warp = std::getenv("PBIT_SPARSE_NOWARP") != nullptr;  // force the block-table tile
    v.warp_g = no_warp ? 0 : warp_tile_group(g, T, false);
    // the warp tile indexes its lanes by count / 2 only where 2 deg + 1 lanes do not fit
    v.warp_half = v.warp_g != 0 && 2 * (int64_t)g.max_degree + 1 > std::min<int64_t>(32, T / v.warp_g);
    const int G = T % 16 == 0 ? 16 : (T % 4 == 0 ? 4 : 1);
    v.unit = g.unit_weights && g.max_degree <= 127 && G >= 4;
    // table when its entries stay within shared memory and cost well under one per update
    const int64_t groups = T / G;
    const int64_t nodes_per_block = (kBlock + groups - 1) / groups + 1;
    const int64_t entries = nodes_per_block * ((int64_t)g.max_wabs + 1);
    v.table = g.tab_ok && entries <= kTabMax && entries * 4 <= (int64_t)kBlock * G * 3;
    return v;
}

cudaError_t launch_sparse_step(const StepArgs& a, cudaStream_t s, SparseVariant v) {
    if (v.table && (!a.wabs || !a.tab_off)) v.table = false;
    const int G = group_size(a);
    if (is_variant(a)) {
        if (G == 16) return v.unit ? launch_variant_g<16, true>(a, s) : launch_variant_g<16, false>(a, s);
        if (G == 4) return v.unit ? launch_variant_g<4, true>(a, s) : launch_variant_g<4, false>(a, s);
        return launch_variant_g<1, false>(a, s);
    }
    if (v.warp_g != 0 && G == 16) {  // G == 16: T % 16 == 0 and both buffers 16-byte aligned
        if (v.warp_g == 32) return v.warp_half ? launch_warp_g<32, true>(a, s) : launch_warp_g<32, false>(a, s);
        return v.warp_half ? launch_warp_g<16, true>(a, s) : launch_warp_g<16, false>(a, s);
    }
    if (G == 16) return launch_step_variant<16>(a, s, v);
    if (G == 4) return launch_step_variant<4>(a, s, v);
    return launch_step_variant<1>(a, s, v);
}

void set_group_divisor(StepArgs& a, int32_t G) {
    const uint32_t d = (uint32_t)(a.T / G);
    if (d == 0 || (int64_t)a.n * d + 2 * kBlock >= (int64_t(1) << 31)) {  // items must stay below 2^31
        a.grp_m = 0;
        a.grp_s = 0;
        return;
    }
    int l = 0;
    while ((1ull << l) < d) ++l;
    // floor(2^(32+l) / d) + 1 < 2^33; with item < 2^31 the 64-bit product cannot overflow
    const unsigned long long num_hi = 1ull << l;  // 2^(32+l) = num_hi * 2^32
    const unsigned long long q_hi = num_hi / d, r_hi = num_hi % d;
    const unsigned long long q_lo = ((r_hi << 32)) / d;  // r_hi < d <= 2^31, so r_hi << 32 fits
    a.grp_m = (q_hi << 32) + q_lo + 1ull;
    a.grp_s = 32 + l;
}

cudaError_t launch_bounded_wait_selftest(const unsigned* flag, long long budget_ns, int* err, cudaStream_t s) {
    bounded_wait_selftest_kernel<<<1, 32, 0, s>>>(flag, budget_ns, err);
    count_launches(1);
    return cudaGetLastError();
}

bool resident_preferred(const Graph& g, int32_t T) {
    return resident_fits(g, T) && (double)T * ((double)g.nnz + (double)g.n) <= 1.2e6;
}

bool resident_fits(const Graph& g, int32_t T) {
    const int64_t cells = (int64_t)g.n * T;
    return 2 * (((cells + 15) / 16) * 16) <= (int64_t)kResidentSmem;
}

cudaError_t launch_resident_anneal(const StepArgs& a, int32_t b, int32_t e, bool unit, cudaStream_t s) {
    if (a.T % 4 == 0) return unit ? launch_resident_g<4, true>(a, b, e, s) : launch_resident_g<4, false>(a, b, e, s);
    return launch_resident_g<1, false>(a, b, e, s);
}

cudaError_t launch_fields(const Graph& g, const int8_t* spins, int32_t T, int32_t* fields, cudaStream_t s) {
    const bool g4 = T % 4 == 0 && aligned4(spins);
    const int G = g4 ? 4 : 1;
    const int64_t threads = (int64_t)g.n * (T / G);
    const int64_t blocks = (threads + kBlock - 1) / kBlock;
    if (g4)
        fields_kernel<4><<<(unsigned)blocks, kBlock, 0, s>>>(g.row_ptr, g.col, g.J, g.h, spins, g.n, T, fields);
    else
        fields_kernel<1><<<(unsigned)blocks, kBlock, 0, s>>>(g.row_ptr, g.col, g.J, g.h, spins, g.n, T, fields);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_cut_energy(const Graph& g, const int8_t* spins, int32_t T, int64_t* out, bool energy,
                              cudaStream_t s) {
    cudaError_t err = cudaMemsetAsync(out, 0, sizeof(int64_t) * (size_t)T, s);
    if (err != cudaSuccess) return err;
    const bool g4 = T % 4 == 0 && aligned4(spins);
    const int G = g4 ? 4 : 1;
    dim3 grid((unsigned)((g.n + kRowsPerBlock - 1) / kRowsPerBlock), (unsigned)((T + 32 * G - 1) / (32 * G)));
    auto* o = reinterpret_cast<unsigned long long*>(out);
    if (g4)
        cut_energy_kernel<4><<<grid, kBlock, 0, s>>>(g.row_ptr, g.col, g.J, g.h, spins, g.n, T, energy, o);
    else
        cut_energy_kernel<1><<<grid, kBlock, 0, s>>>(g.row_ptr, g.col, g.J, g.h, spins, g.n, T, energy, o);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    finish_cut_energy<<<(T + 255) / 256, 256, 0, s>>>(reinterpret_cast<long long*>(out), T, energy);
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace pbit
