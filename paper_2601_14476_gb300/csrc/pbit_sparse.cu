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
        const uint4 r = philox((uint32_t)i, 0xFFFFFFFFu, (uint32_t)t >> 1, instance, k0, k1);
        const uint32_t wr = (t & 1) ? r.z : r.x;
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
template <int G, bool UNIT, bool TABLE>
__global__ void __launch_bounds__(kBlock) sparse_step_kernel(StepArgs a) {
    __shared__ uint32_t s_tab[TABLE ? kTabMax : 1];
    process_tile<G, UNIT, TABLE>(a, blockIdx.x * (int64_t)kBlock, s_tab);
}

// Warp-table tile; six resident blocks per SM (40 registers): on the torus at T = 1024 this ran
// 33.5 µs per step, against 33.7 (five), 35.5 (four) and 36.2 (seven or eight, with spills).
template <int G>
__global__ void __launch_bounds__(kBlock, 6) sparse_warp_kernel(StepArgs a) {
    process_tile_warp<G>(a, blockIdx.x * (uint32_t)kBlock);
}

template <int G, bool UNIT>
__global__ void __launch_bounds__(kBlock) sparse_variant_kernel(StepArgs a) {
    process_tile_variant<G, UNIT>(a, blockIdx.x * (int64_t)kBlock);
}

template <int G, bool UNIT>
cudaError_t launch_variant_g(const StepArgs& a, cudaStream_t s) {
    const int64_t threads = (int64_t)a.n * (a.T / G);
    const int64_t blocks = (threads + kBlock - 1) / kBlock;
    sparse_variant_kernel<G, UNIT><<<(unsigned)blocks, kBlock, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

template <int G, bool UNIT, bool TABLE>
cudaError_t launch_step_g(const StepArgs& base, cudaStream_t s) {
    StepArgs a = base;
    set_group_divisor(a, G);
    const int64_t threads = (int64_t)a.n * (a.T / G);
    const int64_t blocks = (threads + kBlock - 1) / kBlock;
    sparse_step_kernel<G, UNIT, TABLE><<<(unsigned)blocks, kBlock, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

template <int G>
cudaError_t launch_warp_g(const StepArgs& base, cudaStream_t s) {
    StepArgs a = base;
    set_group_divisor(a, G);
    const int64_t threads = (int64_t)a.n * (a.T / G);
    const int64_t blocks = (threads + kBlock - 1) / kBlock;
    sparse_warp_kernel<G><<<(unsigned)blocks, kBlock, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
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

// ------------------------------------------------------------------ flow ----
// All steps of one plain-pSA anneal in one persistent launch.  Work items
// (step j, tile t) are claimed in that order from one counter; item (j, t)
// waits until the tiles holding t's neighbours (and t itself) have finished
// step j - 1, or, for tiles with a long list, until all of step j - 1 is done.
// With a symmetric J the same wait covers the write-after-read hazard of the
// two alternating buffers: the tiles that read t's old spins are exactly the
// ones waited for.  Every waited-on item was claimed earlier by a CTA that is
// running it and never waits on a later item, so the waits end without any
// co-residency assumption; each is still bounded (error code 6, then every
// CTA stops claiming).
struct FlowArgs {
    StepArgs a;
    const int8_t* in0;
    int8_t* P;  // written at even j
    int8_t* Q;  // written at odd j
    int32_t k, ntiles;
    const int32_t* dep_ptr;
    const int32_t* dep_idx;
    unsigned* tile_done;   // [ntiles] steps finished in this launch
    unsigned* step_done;   // [k] tiles that finished step j
    unsigned long long* next;
    int* err;
};

constexpr long long kFlowWaitCycles = 1ll << 32;  // about 2 s at 2 GHz

__device__ __forceinline__ unsigned flow_ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void flow_st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void flow_red_release_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <int G, bool WARP, bool UNIT, bool TABLE>
__global__ void __launch_bounds__(kBlock, WARP ? 6 : 1) sparse_flow_kernel(FlowArgs f) {
    __shared__ uint32_t s_tab[TABLE ? kTabMax : 1];
    __shared__ unsigned long long s_item;
    __shared__ int s_ok;
    const unsigned long long total = (unsigned long long)f.k * (unsigned)f.ntiles;
    for (;;) {
        if (threadIdx.x == 0)
            s_item = *(volatile int*)f.err != 0 ? total : atomicAdd(f.next, 1ull);
        __syncthreads();
        const unsigned long long item = s_item;
        if (item >= total) return;  // uniform
        const int j = (int)(item / (unsigned)f.ntiles);
        const int t = (int)(item - (unsigned long long)j * (unsigned)f.ntiles);
        if (j > 0 && threadIdx.x < 32) {
            const int lane = threadIdx.x;
            const int d0 = __ldg(f.dep_ptr + t), d1 = __ldg(f.dep_ptr + t + 1);
            bool ok = true;
            const long long start = clock64();
            if (d1 == d0) {
                if (lane == 0)
                    while (flow_ld_acquire(f.step_done + (j - 1)) < (unsigned)f.ntiles)
                        if (clock64() - start > kFlowWaitCycles) {
                            ok = false;
                            break;
                        }
            } else {
                for (int d = d0 + lane; d < d1 && ok; d += 32) {
                    const unsigned* p = f.tile_done + __ldg(f.dep_idx + d);
                    while (flow_ld_acquire(p) < (unsigned)j)
                        if (clock64() - start > kFlowWaitCycles) {
                            ok = false;
                            break;
                        }
                }
            }
            ok = __all_sync(0xFFFFFFFFu, ok);
            if (lane == 0) s_ok = ok;
        }
        __syncthreads();
        if (j > 0 && !s_ok) {
            if (threadIdx.x == 0) atomicExch(f.err, 6);
            return;
        }
        StepArgs a = f.a;
        a.step = f.a.step + j;
        a.in = j == 0 ? f.in0 : ((j & 1) ? f.P : f.Q);
        a.out = (j & 1) ? f.Q : f.P;
        if constexpr (WARP) process_tile_warp<G>(a, (uint32_t)t * (uint32_t)kBlock);
        else process_tile<G, UNIT, TABLE>(a, (int64_t)t * kBlock, s_tab);
        __syncthreads();  // every spin store of the tile precedes the release below
        if (threadIdx.x == 0) {
            flow_st_release(f.tile_done + t, (unsigned)(j + 1));
            flow_red_release_add(f.step_done + j, 1u);
        }
    }
}

template <int G, bool WARP, bool UNIT, bool TABLE>
cudaError_t launch_flow_g(const FlowArgs& f, int device, cudaStream_t s) {
    static int per_sm[64] = {0};
    static int sms[64] = {0};
    const int dev = device & 63;
    if (per_sm[dev] == 0) {
        int nb = 0, c = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sparse_flow_kernel<G, WARP, UNIT, TABLE>,
                                                                      kBlock, 0);
        if (e != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) return e;
        if (nb < 1) return cudaErrorNotSupported;
        sms[dev] = c;
        per_sm[dev] = nb;
    }
    const unsigned long long items = (unsigned long long)f.k * (unsigned)f.ntiles;
    const unsigned grid = (unsigned)std::min<unsigned long long>(items, (unsigned long long)per_sm[dev] * sms[dev]);
    FlowArgs ff = f;
    set_group_divisor(ff.a, G);
    sparse_flow_kernel<G, WARP, UNIT, TABLE><<<grid, kBlock, 0, s>>>(ff);
    count_launches(1);
    return cudaGetLastError();
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

template <int G>
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
    const int64_t items = (int64_t)(node_hi - node_lo) * groups;
    int8_t* cur = buf0;
    int8_t* nxt = buf1;
    for (int32_t step = step_begin; step < step_end; ++step) {
        StepArgs sa = a;
        sa.step = step;
        for (int64_t it = threadIdx.x; it < items; it += blockDim.x) {
            const int i = node_lo + (int)(it / groups);
            const int t0 = (int)(it - (int64_t)(i - node_lo) * groups) * G;
            int acc[G];
            gather_field<G>(a.row_ptr, a.col, a.J, cur, a.T, i, t0, acc);
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

template <int G>
cudaError_t launch_resident_g(const StepArgs& a, int32_t b, int32_t e, cudaStream_t s) {
    const int64_t cells = (int64_t)a.n * a.T;
    const size_t smem = 2 * (size_t)(((cells + 15) / 16) * 16);
    cudaError_t err = cudaFuncSetAttribute(resident_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
    if (want > 1 && cudaOccupancyMaxActiveClusters(&clusters, resident_kernel<G>, &cfg) == cudaSuccess && clusters >= 1) {
        err = cudaLaunchKernelEx(&cfg, resident_kernel<G>, a, b, e);
        count_launches(1);
        return err;
    }
    (void)cudaGetLastError();
    cfg.gridDim = dim3(1, 1, 1);
    attr[0].val.clusterDim.x = 1;
    err = cudaLaunchKernelEx(&cfg, resident_kernel<G>, a, b, e);
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

// Trials per thread of the warp-table tile for T trials (0: the tile does not apply).
int warp_tile_group(const Graph& g, int32_t T) {
    if (!g.unit_weights || g.max_degree > 15) return 0;
    for (const int G : {32, 16}) {
        if (T % G != 0) continue;
        const int64_t groups = T / G;
        if (groups % 32 != 0 && 32 % groups != 0) continue;
        const int64_t L = groups >= 32 ? 32 : groups;
        if (2 * (int64_t)g.max_degree + 1 > L) continue;
        if ((int64_t)g.n * groups >= (int64_t(1) << 31)) continue;
        return G;
    }
    return 0;
}

SparseVariant choose_sparse_variant(const Graph& g, int32_t T) {
    SparseVariant v;
    static const bool plain = std::getenv("PBIT_SPARSE_PLAIN") != nullptr;  // force the plain variant
    if (plain) return v;
    static const bool no_warp = std::getenv("PBIT_SPARSE_NOWARP") != nullptr;  // force the block-table tile
    v.warp_g = no_warp ? 0 : warp_tile_group(g, T);
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
        if (v.warp_g == 32) return launch_warp_g<32>(a, s);
        return launch_warp_g<16>(a, s);
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

// Trials per thread of the tile the sparse kernels use for T trials and these buffers.
static int32_t tile_trials(int32_t T, const void* const* bufs, int nbufs, SparseVariant v) {
    bool a16 = T % 16 == 0, a4 = T % 4 == 0;
    for (int q = 0; q < nbufs; ++q) {
        a16 = a16 && aligned16(bufs[q]);
        a4 = a4 && aligned4(bufs[q]);
    }
    const int G = a16 ? 16 : (a4 ? 4 : 1);
    if (v.warp_g != 0 && G == 16) return v.warp_g;
    return G;
}

static int32_t flow_groups(int32_t T, const int8_t* in0, const int8_t* P, const int8_t* Q, SparseVariant v) {
    const void* bufs[3] = {in0, P, Q};
    return T / tile_trials(T, bufs, Q ? 3 : 2, v);
}

// Build (or reuse) the per-tile dependency lists for `groups` items per node.
static pbit_status build_flow_deps(Graph& g, int32_t groups) {
    if (g.flow.groups == groups && g.flow.ptr) return PBIT_OK;
    cudaFree(g.flow.ptr);
    cudaFree(g.flow.idx);
    g.flow = FlowDeps();
    constexpr size_t kMaxDeps = 64;  // longer lists wait for the whole previous step
    const int64_t items = (int64_t)g.n * groups;
    const int64_t ntiles = (items + kBlock - 1) / kBlock;
    if (ntiles >= (int64_t(1) << 31)) return fail(PBIT_E_INVALID, "flow: too many tiles");
    std::vector<int32_t> ptr((size_t)ntiles + 1, 0), idx, d;
    int64_t listed = 0;
    g.flow.entries = 0;
    for (int64_t t = 0; t < ntiles; ++t) {
        const int64_t first = t * kBlock, last = std::min(items, first + kBlock) - 1;
        d.clear();
        d.push_back((int32_t)t);
        bool global = false;
        for (int64_t i = first / groups; i <= last / groups && !global; ++i) {
            for (int32_t e = g.h_row_ptr[i]; e < g.h_row_ptr[i + 1]; ++e) {
                const int64_t j = g.h_col[e];
                const int64_t lo = j * groups / kBlock, hi = ((j + 1) * groups - 1) / kBlock;
                for (int64_t x = lo; x <= hi; ++x) d.push_back((int32_t)x);
                if (d.size() > 8 * kMaxDeps) {
                    global = true;
                    break;
                }
            }
        }
        if (!global) {
            std::sort(d.begin(), d.end());
            d.erase(std::unique(d.begin(), d.end()), d.end());
            global = d.size() > kMaxDeps;
        }
        if (!global) {
            idx.insert(idx.end(), d.begin(), d.end());
            ++listed;
            g.flow.entries += (int64_t)d.size();
        }
        ptr[(size_t)t + 1] = (int32_t)idx.size();
    }
    cudaError_t e = cudaMalloc(&g.flow.ptr, sizeof(int32_t) * ptr.size());
    if (e == cudaSuccess) e = cudaMalloc(&g.flow.idx, sizeof(int32_t) * std::max<size_t>(1, idx.size()));
    if (e == cudaSuccess) e = cudaMemcpy(g.flow.ptr, ptr.data(), sizeof(int32_t) * ptr.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !idx.empty())
        e = cudaMemcpy(g.flow.idx, idx.data(), sizeof(int32_t) * idx.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(g.flow.ptr);
        cudaFree(g.flow.idx);
        g.flow = FlowDeps();
        return cuda_fail(e, "flow dependency lists");
    }
    const int64_t entries = g.flow.entries;
    g.flow.groups = groups;
    g.flow.ntiles = (int32_t)ntiles;
    g.flow.listed = listed;
    g.flow.entries = entries;
    return PBIT_OK;
}

pbit_status ensure_flow_deps(Graph& g, int32_t T, const int8_t* in0, const int8_t* P, const int8_t* Q,
                             SparseVariant v) {
    return build_flow_deps(g, flow_groups(T, in0, P, Q, v));
}

cudaError_t launch_sparse_flow(const Graph& g, StepArgs a, int32_t k, const int8_t* in0, int8_t* P, int8_t* Q,
                               unsigned* tile_done, unsigned* step_done, unsigned long long* next,
                               SparseVariant v, cudaStream_t s) {
    if (is_variant(a) || k < 1) return cudaErrorNotSupported;
    if (v.table && (!a.wabs || !a.tab_off)) v.table = false;
    const void* bufs[3] = {in0, P, Q};
    const int32_t G = tile_trials(a.T, bufs, Q ? 3 : 2, v);
    if (g.flow.groups != a.T / G || !g.flow.ptr) return cudaErrorNotSupported;
    FlowArgs f;
    f.a = a;
    f.in0 = in0;
    f.P = P;
    f.Q = Q;
    f.k = k;
    f.ntiles = g.flow.ntiles;
    f.dep_ptr = g.flow.ptr;
    f.dep_idx = g.flow.idx;
    f.tile_done = tile_done;
    f.step_done = step_done;
    f.next = next;
    f.err = g.err;
    const int dev = g.device;
    if (v.warp_g != 0 && G == 32) return launch_flow_g<32, true, false, false>(f, dev, s);
    if (v.warp_g != 0 && G == 16) return launch_flow_g<16, true, false, false>(f, dev, s);
    if (G == 16) {
        if (v.unit && v.table) return launch_flow_g<16, false, true, true>(f, dev, s);
        if (v.unit) return launch_flow_g<16, false, true, false>(f, dev, s);
        if (v.table) return launch_flow_g<16, false, false, true>(f, dev, s);
        return launch_flow_g<16, false, false, false>(f, dev, s);
    }
    if (G == 4) {
        if (v.unit && v.table) return launch_flow_g<4, false, true, true>(f, dev, s);
        if (v.unit) return launch_flow_g<4, false, true, false>(f, dev, s);
        if (v.table) return launch_flow_g<4, false, false, true>(f, dev, s);
        return launch_flow_g<4, false, false, false>(f, dev, s);
    }
    if (v.table) return launch_flow_g<1, false, false, true>(f, dev, s);
    return launch_flow_g<1, false, false, false>(f, dev, s);
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

cudaError_t launch_resident_anneal(const StepArgs& a, int32_t b, int32_t e, cudaStream_t s) {
    if (a.T % 4 == 0) return launch_resident_g<4>(a, b, e, s);
    return launch_resident_g<1>(a, b, e, s);
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
