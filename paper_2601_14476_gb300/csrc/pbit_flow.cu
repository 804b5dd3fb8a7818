// The multi-step sparse launch: all steps of one plain-pSA anneal in one
// persistent kernel with per-tile step dependencies, and the host-built
// dependency lists it waits on.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdlib>
#include <string>
#include <vector>

#include "pbit_device.cuh"
#include "pbit_internal.h"
#include "pbit_tile.cuh"

namespace pbit {
namespace {

using namespace tile;

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
    long long wait_cycles;  // clock64 budget of each dependency wait (about 2 s; shorter in tests)
    int withhold;           // test-only: tile 0 never publishes its progress
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

template <int G, int WARP, bool UNIT, bool TABLE>
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
                        if (clock64() - start > f.wait_cycles) {
                            ok = false;
                            break;
                        }
            } else {
                for (int d = d0 + lane; d < d1 && ok; d += 32) {
                    const unsigned* p = f.tile_done + __ldg(f.dep_idx + d);
                    while (flow_ld_acquire(p) < (unsigned)j)
                        if (clock64() - start > f.wait_cycles) {
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
        if constexpr (WARP != 0) process_tile_warp<G, WARP == 2>(a, (uint32_t)t * (uint32_t)kBlock);
        else process_tile<G, UNIT, TABLE>(a, (int64_t)t * kBlock, s_tab);
        __syncthreads();  // every spin store of the tile precedes the release below
        if (threadIdx.x == 0 && !(f.withhold && t == 0)) {
            flow_st_release(f.tile_done + t, (unsigned)(j + 1));
            flow_red_release_add(f.step_done + j, 1u);
        }
    }
}

template <int G, int WARP, bool UNIT, bool TABLE>
cudaError_t launch_flow_g(const FlowArgs& f, int device, cudaStream_t s) {
    // resident CTAs of this instantiation on each device, computed once (concurrent first calls store
    // the same value)
    static std::atomic<int> resident[64];
    const int dev = device & 63;
    int cap = resident[dev].load(std::memory_order_relaxed);
    if (cap == 0) {
        int nb = 0, c = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sparse_flow_kernel<G, WARP, UNIT, TABLE>,
                                                                      kBlock, 0);
        if (e != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) return e;
        if (nb < 1) return cudaErrorNotSupported;
        cap = nb * c;
        resident[dev].store(cap, std::memory_order_relaxed);
    }
    const unsigned long long items = (unsigned long long)f.k * (unsigned)f.ntiles;
    const unsigned grid = (unsigned)std::min<unsigned long long>(items, (unsigned long long)cap);
    FlowArgs ff = f;
    set_group_divisor(ff.a, G);
    sparse_flow_kernel<G, WARP, UNIT, TABLE><<<grid, kBlock, 0, s>>>(ff);
    count_launches(1);
    return cudaGetLastError();
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
bool aligned4(const void* p) { return ((uintptr_t)p & 3u) == 0; }

}  // namespace

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
    const TestFault tf = test_fault("flow", kFlowWaitCycles);
    f.wait_cycles = tf.wait_cycles;
    f.withhold = tf.withhold;
    f.err = g.err;
    const int dev = g.device;
    // WARP: 0 shared-table tile, 1 warp-table tile, 2 warp-table tile indexed by count / 2
    if (v.warp_g != 0 && G == 32)
        return v.warp_half ? launch_flow_g<32, 2, false, false>(f, dev, s) : launch_flow_g<32, 1, false, false>(f, dev, s);
    if (v.warp_g != 0 && G == 16)
        return v.warp_half ? launch_flow_g<16, 2, false, false>(f, dev, s) : launch_flow_g<16, 1, false, false>(f, dev, s);
    if (G == 16) {
        if (v.unit && v.table) return launch_flow_g<16, 0, true, true>(f, dev, s);
        if (v.unit) return launch_flow_g<16, 0, true, false>(f, dev, s);
        if (v.table) return launch_flow_g<16, 0, false, true>(f, dev, s);
        return launch_flow_g<16, 0, false, false>(f, dev, s);
    }
    if (G == 4) {
        if (v.unit && v.table) return launch_flow_g<4, 0, true, true>(f, dev, s);
        if (v.unit) return launch_flow_g<4, 0, true, false>(f, dev, s);
        if (v.table) return launch_flow_g<4, 0, false, true>(f, dev, s);
        return launch_flow_g<4, 0, false, false>(f, dev, s);
    }
    if (v.table) return launch_flow_g<1, 0, false, true>(f, dev, s);
    return launch_flow_g<1, 0, false, false>(f, dev, s);
}

}  // namespace pbit
