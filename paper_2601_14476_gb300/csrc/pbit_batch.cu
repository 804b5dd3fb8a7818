// Batched annealing of many instances of uneven size in one persistent
// launch per chunk of steps, replayed from a captured CUDA graph.
//
// Work list of one chunk of K steps: items (k, g, tile) in that order, k the
// step within the chunk, g the instance, tile a block of kBlock (node,
// trial-group) items of instance g.  Persistent CTAs claim items with one
// atomic counter.  Before working on (k, g, tile) a CTA waits until all
// tiles of (k-1, g) are done (per-instance counter).  Items are claimed in
// index order, so every item waited on was claimed earlier by a running CTA
// that never waits on a later item: the scheme needs no co-residency and
// cannot deadlock.  The waits are bounded anyway (error flag, then the CTA
// goes on).
//
// Each (instance, step) computes exactly what one pbit_anneal step computes
// (same tile function, same Philox counters), so an instance's result does
// not depend on the batch it runs in, the chunk length or the tiling.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "pbit_device.cuh"
#include "pbit_internal.h"
#include "pbit_tile.cuh"

namespace pbit {
namespace {

using namespace tile;

struct InstDesc {
    StepArgs a;        // graph, parameters, schedule, seeds (in/out/step set per item)
    int8_t* buf[2];    // ping-pong spin buffers
    int32_t cur;       // next schedule step to run
    int32_t end;       // stop before this step
    int32_t parity;    // buf[parity] holds the state at `cur`
    int32_t G, unit, table;
    int32_t tiles;     // work items per step (each up to ChunkArgs::tpi tiles)
    int32_t blocks;    // tiles per step
    int32_t active;    // 0 = slot unused
    int32_t T_real;    // trials the caller asked for; a.T is the padded row stride
    int32_t words;     // 1: SpSA / TApSA in the coalesced word tile (a.T % 128 == 0, no timing model)
    int32_t spans;     // word tile: 128-trial spans per node
    int32_t warp;      // 1: plain pSA in the warp-table tile in this chunk (G = 16 or 32 trials per thread)
    int32_t base_G;    // trials per thread of the shared-table tile
    int32_t wg_wide;   // warp-table tile under a heavy load: trials per thread (0: not applicable)
};

struct ChunkArgs {
    InstDesc* inst;
    const int32_t* tile_prefix;  // [count + 1]
    int32_t count;
    int32_t total_tiles;
    int32_t K;
    int32_t tpi;                 // tiles per work item (1 or 2: the kernel's TPI)
    unsigned* queue;             // item counter
    unsigned* tiles_done;        // [count] tiles finished in this chunk
    int* err;
    long long wait_cycles;       // clock64 budget of each step wait (about a second; shorter in tests)
    int withhold;                // test-only: instance 0's first tile of a chunk is never counted
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <int G, bool UNIT, bool TABLE>
__device__ __forceinline__ void run_tile(const StepArgs& a, int64_t first, uint32_t* s_tab) {
    process_tile<G, UNIT, TABLE>(a, first, s_tab);
}

template <bool VARIANTS, bool WARP>
__device__ void dispatch_tile(const StepArgs& a, int G, int unit, int table, int64_t first, uint32_t* s_tab,
                              int warp) {
    if (WARP && warp) {
        if (G == 32) process_tile_warp<32, true>(a, (uint32_t)first);
        else process_tile_warp<16, true>(a, (uint32_t)first);
        return;
    }
    if (VARIANTS && is_variant(a)) {
        if (G == 16) {
            if (unit) process_tile_variant<16, true>(a, first); else process_tile_variant<16, false>(a, first);
        } else {
            if (unit) process_tile_variant<4, true>(a, first); else process_tile_variant<4, false>(a, first);
        }
        return;
    }
    if (G == 16) {
        if (unit) {
            if (table) run_tile<16, true, true>(a, first, s_tab); else run_tile<16, true, false>(a, first, s_tab);
        } else {
            if (table) run_tile<16, false, true>(a, first, s_tab); else run_tile<16, false, false>(a, first, s_tab);
        }
    } else if (G == 4) {
        if (unit) {
            if (table) run_tile<4, true, true>(a, first, s_tab); else run_tile<4, true, false>(a, first, s_tab);
        } else {
            if (table) run_tile<4, false, true>(a, first, s_tab); else run_tile<4, false, false>(a, first, s_tab);
        }
    } else {
        if (table) run_tile<1, false, true>(a, first, s_tab); else run_tile<1, false, false>(a, first, s_tab);
    }
}

// SpSA and TApSA in the word tile for one batch tile: warp w of the block takes the (node, 128-trial
// span) units (tile * 8 + w) * 4 .. + 3 (an item then holds as many updates as a group-tile item).
constexpr int kWordUnits = 4;  // (node, span) units per warp and item: an item holds 4096 updates

template <bool UNIT>
__device__ void batch_words_unit(const StepArgs& a, int spans, int64_t lw);

template <bool UNIT>
__device__ void batch_words_tile(const StepArgs& a, int spans, int tile_i) {
    const int warp = (int)(threadIdx.x >> 5);
    for (int u = 0; u < kWordUnits; ++u)
        batch_words_unit<UNIT>(a, spans, ((int64_t)tile_i * (kBlock / 32) + warp) * kWordUnits + u);
}

template <bool UNIT>
__device__ void batch_words_unit(const StepArgs& a, int spans, int64_t lw) {
    const int lane = (int)(threadIdx.x & 31u);
    const int i = (int)(lw / spans);
    if (i >= a.n) return;  // uniform across the warp
    const int tb = (int)(lw - (int64_t)i * spans) * 128 + 4 * lane;
    const uint32_t q = (uint32_t)a.step;
    const float I0 = __ldg(a.i0_table + q);
    const int hi = a.h ? __ldg(a.h + i) : 0;
    const float lam = a.par.lambda ? __ldg(a.par.lambda + i) : 1.0f;
    const float del = a.par.delta ? __ldg(a.par.delta + i) : 0.0f;
    const uint32_t thr = a.par.thr ? __ldg(a.par.thr + i) : (1u << 24);
    const int rb = __ldg(a.row_ptr + i), re = __ldg(a.row_ptr + i + 1);
    const auto nbr = [&](int) -> const int8_t* { return a.in; };
    if (a.alg == 2 && a.window == 4)
        variant_words<1, UNIT, 4>(a, i, tb, I0, hi, lam, del, thr, rb, re, a.in, a.out, nbr, lane);
    else
        variant_words<1, UNIT, 0>(a, i, tb, I0, hi, lam, del, thr, rb, re, a.in, a.out, nbr, lane);
}

// VARIANTS = false: plain pSA only (the SpSA / TApSA / timing-model tiles are not compiled in,
// which keeps the register count, and so the residency, of the common case).  TPI: tiles per work
// item (ChunkArgs::tpi), a template parameter so that the one-tile form keeps its straight-line code
// (a runtime loop over tiles cost 19 % of a lone request's latency).
constexpr int kBatchMinBlocks = 8;
constexpr int kBatchMinBlocksVariants = 4;
template <bool VARIANTS, int TPI>
__global__ void __launch_bounds__(kBlock, VARIANTS ? kBatchMinBlocksVariants : kBatchMinBlocks)
    batch_chunk_kernel(ChunkArgs c) {
    __shared__ uint32_t s_tab[kTabMax];
    __shared__ unsigned s_item;
    __shared__ int s_ok;
    const unsigned total = (unsigned)c.K * (unsigned)c.total_tiles;
    for (;;) {
        // once any wait has given up, every CTA stops claiming
        if (threadIdx.x == 0) s_item = *(volatile int*)c.err != 0 ? total : atomicAdd(c.queue, 1u);
        __syncthreads();
        const unsigned idx = s_item;
        __syncthreads();  // s_item is read by everyone before thread 0 may overwrite it
        if (idx >= total) break;
        const int k = (int)(idx / (unsigned)c.total_tiles);
        const int rem = (int)(idx - (unsigned)k * (unsigned)c.total_tiles);
        int lo = 0, hi = c.count - 1;  // instance: last g with tile_prefix[g] <= rem
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (c.tile_prefix[mid] <= rem) lo = mid; else hi = mid - 1;
        }
        const int g = lo;
        const int tile_i = rem - c.tile_prefix[g];
        const InstDesc& d = c.inst[g];
        if (!d.active || d.cur + k >= d.end) continue;  // uniform across the block
        if (threadIdx.x == 0) {
            int ok = 1;
            if (k > 0) {
                const unsigned need = (unsigned)k * (unsigned)d.tiles;
                const long long start = clock64();
                while (ld_acquire_u32(c.tiles_done + g) < need) {
                    if (clock64() - start > c.wait_cycles) {
                        atomicExch(c.err, 4);
                        ok = 0;
                        break;
                    }
                }
            }
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) break;  // uniform: s_ok was written before the barrier
        StepArgs a = d.a;
        a.step = d.cur + k;
        const int par = (d.parity + k) & 1;
        a.in = d.buf[par];
        a.out = d.buf[par ^ 1];
        const int b_first = tile_i * TPI, b_end = min(d.blocks, b_first + TPI);
#pragma unroll
        for (int b = b_first; b < b_end; ++b) {
            if (TPI > 1 && b > b_first) __syncthreads();  // the previous tile's threshold table is read
            if constexpr (VARIANTS) {
                if (d.words) {
                    if (d.unit) batch_words_tile<true>(a, d.spans, b);
                    else batch_words_tile<false>(a, d.spans, b);
                } else {
                    dispatch_tile<VARIANTS, (TPI > 1)>(a, d.G, d.unit, d.table, (int64_t)b * kBlock, s_tab, d.warp);
                }
            } else {
                dispatch_tile<VARIANTS, (TPI > 1)>(a, d.G, d.unit, d.table, (int64_t)b * kBlock, s_tab, d.warp);
            }
        }
        __threadfence();  // this thread's spin stores, before the item is counted
        __syncthreads();
        if (threadIdx.x == 0 && !(c.withhold && g == 0 && k == 0 && tile_i == 0)) atomicAdd(c.tiles_done + g, 1u);
    }
}

// After a chunk: advance every instance by the steps it ran and reset the
// chunk counters, so the same graph can be replayed for the next chunk.
__global__ void batch_advance_kernel(InstDesc* inst, int32_t count, int32_t K, unsigned* queue,
                                     unsigned* tiles_done) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g == 0) *queue = 0u;
    if (g < count) {
        InstDesc& d = inst[g];
        if (d.active) {
            const int ran = min(K, max(0, d.end - d.cur));
            d.cur += ran;
            d.parity = (d.parity + ran) & 1;
        }
        tiles_done[g] = 0u;
    }
}

}  // namespace
}  // namespace pbit

using namespace pbit;

// ------------------------------------------------------------------ host ----
struct pbit_batch_s {
    int device = 0;
    int32_t count = 0;
    std::vector<pbit_graph> graphs;
    std::vector<InstDesc> host_desc;     // host mirror (cur/parity advanced arithmetically)
    std::vector<int32_t> tile_prefix;
    int32_t total_tiles = 0;
    InstDesc* d_inst = nullptr;
    int32_t* d_prefix = nullptr;
    unsigned* d_ctl = nullptr;           // [0] queue, [1..count] tiles_done
    std::vector<void*> allocs;           // per-instance device memory
    bool variants = false;               // some instance runs SpSA, TApSA or the timing model
    // tuning
    int32_t chunk = 32;
    int32_t ctas_per_sm = 0;             // 0 = occupancy maximum
    int32_t tpi = 1;                     // tiles per work item (plan_chunk)
    // captured chunk graph
    cudaGraphExec_t exec = nullptr;
    cudaStream_t exec_stream = nullptr;
    int32_t exec_chunk = 0, exec_grid = 0;
    ~pbit_batch_s() {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(device);
        cudaDeviceSynchronize();
        if (exec) cudaGraphExecDestroy(exec);
        for (void* p : allocs) cudaFree(p);
        cudaFree(d_inst);
        cudaFree(d_prefix);
        cudaFree(d_ctl);
        cudaSetDevice(cur);
    }
};

namespace {

// Tiling of one instance for a chunk: trials per thread and tiles per step (the word tile's tiles are
// fixed), then work items of `tpi` tiles.  Results do not depend on it.
void plan_inst(InstDesc& d, bool wide, int tpi) {
    if (!d.words) {
        d.warp = wide && d.wg_wide != 0 ? 1 : 0;  // the one-tile kernel has no warp-table tile
        d.G = d.warp ? d.wg_wide : d.base_G;
        set_group_divisor(d.a, d.G);
        const int64_t items = (int64_t)d.a.n * (d.a.T / d.G);
        d.blocks = (int32_t)((items + kBlock - 1) / kBlock);
    }
    d.tiles = (d.blocks + tpi - 1) / tpi;
}

// Tiling of a chunk over `count` instances on a grid of at most `max_grid` CTAs.  Under a heavy load
// (at least 16 instances and four tiles per CTA and step) the warp-table tile takes 32 trials per
// thread and an item
// holds two tiles: fewer instructions and claims per update (the 64-instance batch: 146 -> 133 ms).
// Under a light load (a few resident requests) the shared-table tile with 16 trials per thread and
// one tile per item keep every instance's step spread over as many CTAs as possible, which sets its
// latency (a lone request's p50 rose 19 % with two-tile items).  Returns the tiles per item.
int plan_chunk(InstDesc* d, int32_t count, int max_grid) {
    int64_t blocks = 0;
    for (int32_t k = 0; k < count; ++k) {
        plan_inst(d[k], true, 1);
        blocks += d[k].blocks;
    }
    const bool heavy = count >= 16 && blocks >= 4 * (int64_t)max_grid;
    for (int32_t k = 0; k < count; ++k) plan_inst(d[k], heavy, heavy ? 2 : 1);
    return heavy ? 2 : 1;
}

// Device state of one instance: schedule table, per-node parameters, two
// spin buffers (initial state from Philox).  Allocations are appended to
// `allocs`; `host_keep` (optional) receives host arrays that must outlive the
// asynchronous copies.  Stream-ordered on `s`.
pbit_status build_inst(const Graph& g, const pbit_anneal_params& pp, cudaStream_t s, std::vector<void*>& allocs,
                       InstDesc& d, std::vector<std::vector<uint32_t>>* host_keep) {
    const pbit_anneal_params* p = &pp;
    if (p->struct_size != sizeof(pbit_anneal_params)) return fail(PBIT_E_INVALID, "instance: struct_size mismatch");
    const int32_t T = p->trials, S = p->steps;
    if (p->t_res < 0 || (int64_t)S * (p->t_res > 0 ? p->t_res : 1) > INT32_MAX)
        return fail(PBIT_E_INVALID, "instance: bad t_res");
    const int32_t sub = S * (p->t_res > 0 ? p->t_res : 1);
    const int32_t sb = p->step_begin, se = p->step_end == 0 ? sub : p->step_end;
    if (T < 1 || S < 1 || sb < 0 || se < sb || se > sub || p->offset_mode < 0 || p->offset_mode > 2)
        return fail(PBIT_E_INVALID, "instance: bad trials/steps/offset mode");
    if (p->algorithm < 0 || p->algorithm > 2 || (p->algorithm == PBIT_ALG_TAPSA && (p->window < 1 || p->window > 64)) ||
        (p->algorithm == PBIT_ALG_SPSA && !(p->stall_prob >= 0.0f && p->stall_prob <= 1.0f)))
        return fail(PBIT_E_INVALID, "instance: bad algorithm parameters");
    if ((p->algorithm != PBIT_ALG_PSA || p->t_res > 0) && sb != 0)
        return fail(PBIT_E_INVALID, "instance: variants start at step 0 in batches and servers");
    if (p->algorithm == PBIT_ALG_TAPSA && g.max_abs_field > 32767)
        return fail(PBIT_E_UNSUPPORTED, "instance: TApSA keeps fields as int16; |h_i| + sum_j |J_ij| exceeds 32767");
    pbit_status st;
    std::vector<float> tab;
    if ((st = build_schedule(g, p->i0_min, p->i0_max, p->i0_normalize, S, tab)) != PBIT_OK) return st;
    auto alloc = [&](void** ptr, size_t bytes) -> pbit_status {
        cudaError_t e = cudaMallocAsync(ptr, bytes == 0 ? 16 : bytes, s);
        if (e != cudaSuccess) return cuda_fail(e, "instance: cudaMallocAsync");
        allocs.push_back(*ptr);
        return PBIT_OK;
    };
    std::memset(&d, 0, sizeof(d));
    StepArgs& a = d.a;
    a.row_ptr = g.row_ptr;
    a.col = g.col;
    a.J = g.J;
    a.h = g.h;
    a.wabs = g.wabs;
    a.tab_off = g.tab_off;
    // Rows are padded to a multiple of 16 trials (4 below 64 trials) so every
    // instance runs the vectorised tile code; the extra trials are computed
    // like the others (their Philox counters are their own) and never reported.
    const int32_t T_pad = T % 16 == 0 ? T : (T >= 64 ? (T + 15) / 16 * 16 : (T + 3) / 4 * 4);
    a.n = g.n;
    a.T = T_pad;
    a.seed_lo = (uint32_t)(p->seed & 0xFFFFFFFFu);
    a.seed_hi = (uint32_t)(p->seed >> 32);
    a.instance = p->instance;
    a.offset_mode = p->offset_mode;
    const size_t n = (size_t)g.n;
    // one block for the schedule and the parameters, copied from pageable memory (staged by CUDA)
    void* d_tab = nullptr;
    if ((st = alloc(&d_tab, sizeof(float) * tab.size())) != PBIT_OK) return st;
    PBIT_CUDA_TRY(cudaMemcpyAsync(d_tab, tab.data(), sizeof(float) * tab.size(), cudaMemcpyHostToDevice, s));
    a.i0_table = (const float*)d_tab;
    if (p->intensity) {
        void* dp = nullptr;
        if ((st = alloc(&dp, sizeof(float) * n)) != PBIT_OK) return st;
        PBIT_CUDA_TRY(cudaMemcpyAsync(dp, p->intensity, sizeof(float) * n, cudaMemcpyHostToDevice, s));
        a.par.lambda = (const float*)dp;
    }
    if (p->offset) {
        void* dp = nullptr;
        if ((st = alloc(&dp, sizeof(float) * n)) != PBIT_OK) return st;
        PBIT_CUDA_TRY(cudaMemcpyAsync(dp, p->offset, sizeof(float) * n, cudaMemcpyHostToDevice, s));
        a.par.delta = (const float*)dp;
    }
    if (p->p_update) {
        std::vector<uint32_t> thr(n);
        for (size_t i = 0; i < n; ++i) {
            const float pu = p->p_update[i];
            if (!(pu >= 0.0f && pu <= 1.0f)) return fail(PBIT_E_INVALID, "instance: p_update outside [0,1]");
            thr[i] = (uint32_t)std::ceil((double)pu * 16777216.0);
        }
        void* dp = nullptr;
        if ((st = alloc(&dp, sizeof(uint32_t) * n)) != PBIT_OK) return st;
        PBIT_CUDA_TRY(cudaMemcpyAsync(dp, thr.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice, s));
        a.par.thr = (const uint32_t*)dp;
        if (host_keep) host_keep->push_back(std::move(thr));
    }
    const size_t cells = n * (size_t)T_pad;
    void* b0 = nullptr;
    void* b1 = nullptr;
    if ((st = alloc(&b0, cells)) != PBIT_OK) return st;
    if ((st = alloc(&b1, cells)) != PBIT_OK) return st;
    d.buf[0] = (int8_t*)b0;
    d.buf[1] = (int8_t*)b1;
    // variant state (zero = before step 0) and timing periods
    a.alg = p->algorithm;
    a.window = p->window < 1 ? 1 : p->window;
    a.t_res = p->t_res;
    a.stall_thr = (uint32_t)std::ceil((double)p->stall_prob * 16777216.0);
    if (a.alg != PBIT_ALG_PSA) {
        const size_t sbytes = (a.alg == PBIT_ALG_SPSA ? 4 : 2 * (size_t)a.window) * n * (size_t)T_pad;
        void* stt = nullptr;
        if ((st = alloc(&stt, sbytes)) != PBIT_OK) return st;
        PBIT_CUDA_TRY(cudaMemsetAsync(stt, 0, sbytes, s));
        if (a.alg == PBIT_ALG_SPSA) a.Iprev = (float*)stt;
        else a.ring = (int16_t*)stt;
    }
    if (p->t_res > 0) {
        std::vector<uint32_t> nu(n);
        for (size_t i = 0; i < n; ++i) {
            const double v = std::round((double)p->t_res * (1.0 + (p->nu_dev ? (double)p->nu_dev[i] : 0.0)));
            nu[i] = v < 1.0 ? 1u : (uint32_t)std::min(v, 1e9);
        }
        void* dp = nullptr;
        if ((st = alloc(&dp, sizeof(uint32_t) * n)) != PBIT_OK) return st;
        PBIT_CUDA_TRY(cudaMemcpyAsync(dp, nu.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice, s));
        a.nu = (const int32_t*)dp;
    }
    PBIT_CUDA_TRY(launch_init_spins(g.n, T_pad, p->seed, p->instance, d.buf[0], s));
    d.cur = sb;
    d.end = se;
    d.parity = 0;
    d.base_G = T_pad % 16 == 0 ? 16 : 4;
    d.T_real = T;
    const SparseVariant v = choose_sparse_variant(g, T_pad);
    d.unit = v.unit ? 1 : 0;
    d.table = v.table ? 1 : 0;
    // plain pSA takes the warp-table tile where the single-anneal path would (unit weights, every
    // node's deg + 1 thresholds within its lane segment) when the chunk's load is heavy
    if (v.warp_g != 0 && T_pad % 16 == 0 && a.alg == PBIT_ALG_PSA && a.t_res == 0) {
        d.wg_wide = warp_tile_group(g, T_pad, true);
    }
    // SpSA and TApSA take the coalesced word tile when the padded rows hold whole 128-trial spans
    // (measured on the 64-instance batch: 1.06x and 1.03x the group tile's rate); the timing model
    // stays in the group tile, whose idle-node copies ran 1.2x faster there.  PBIT_BATCH_GROUP_TILE,
    // read at every instance setup, keeps every variant in the group tile (comparisons).
    d.words = a.alg != PBIT_ALG_PSA && a.t_res == 0 && T_pad % 128 == 0 &&
              std::getenv("PBIT_BATCH_GROUP_TILE") == nullptr ? 1 : 0;
    if (d.words) {
        d.spans = T_pad / 128;
        const int64_t per_tile = (kBlock / 32) * kWordUnits;
        d.blocks = (int32_t)(((int64_t)g.n * d.spans + per_tile - 1) / per_tile);
    }
    plan_inst(d, false, 1);
    d.active = 1;
    return PBIT_OK;
}

// Exact cuts of the T_real reported trials of an instance (rows padded to a.T).
pbit_status padded_cuts(pbit_graph g, const InstDesc& d, int64_t* cuts, cudaStream_t s) {
    std::vector<int64_t> all((size_t)d.a.T);
    pbit_status st = pbit_cut(g, d.buf[d.parity], d.a.T, all.data(), 1, s);
    if (st != PBIT_OK) return st;
    std::memcpy(cuts, all.data(), sizeof(int64_t) * (size_t)d.T_real);
    return PBIT_OK;
}

// Bytes of device memory one instance needs (spins, schedule, parameters).
size_t inst_bytes(const Graph& g, const pbit_anneal_params& p) {
    const size_t n = (size_t)g.n;
    const size_t T_pad = (size_t)(p.trials + 15) / 16 * 16;
    const size_t state = p.algorithm == PBIT_ALG_SPSA ? 4 * n * T_pad
                         : (p.algorithm == PBIT_ALG_TAPSA ? 2 * (size_t)std::max(1, p.window) * n * T_pad : 0);
    return 2 * n * T_pad + state + sizeof(float) * (size_t)p.steps + 16 * n + 1024;
}

template <typename T>
pbit_status dev_alloc(pbit_batch b, T** p, size_t count) {
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
    if (e != cudaSuccess) return cuda_fail(e, "batch: cudaMalloc");
    b->allocs.push_back((void*)*p);
    return PBIT_OK;
}

int chunk_occupancy(bool variants) {
    int occ = 0;
    if (variants) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_chunk_kernel<true, 1>, kBlock, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_chunk_kernel<false, 1>, kBlock, 0);
    return occ;
}

void launch_chunk(bool variants, int grid, const ChunkArgs& c, cudaStream_t s) {
    if (c.tpi == 2) {
        if (variants) batch_chunk_kernel<true, 2><<<grid, kBlock, 0, s>>>(c);
        else batch_chunk_kernel<false, 2><<<grid, kBlock, 0, s>>>(c);
    } else {
        if (variants) batch_chunk_kernel<true, 1><<<grid, kBlock, 0, s>>>(c);
        else batch_chunk_kernel<false, 1><<<grid, kBlock, 0, s>>>(c);
    }
}

int grid_for(pbit_batch b) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    int occ = chunk_occupancy(b->variants);
    if (occ < 1) occ = 1;
    const int per = b->ctas_per_sm > 0 ? std::min(b->ctas_per_sm, occ) : occ;
    return std::max(1, sms * per);
}

pbit_status upload_desc(pbit_batch b, cudaStream_t s) {
    PBIT_CUDA_TRY(cudaMemcpyAsync(b->d_inst, b->host_desc.data(), sizeof(InstDesc) * b->host_desc.size(),
                                  cudaMemcpyHostToDevice, s));
    PBIT_CUDA_TRY(cudaStreamSynchronize(s));
    return PBIT_OK;
}

// Capture [chunk kernel, advance kernel] once per (chunk length, grid).
pbit_status ensure_graph(pbit_batch b, cudaStream_t user) {
    const int grid = grid_for(b);
    if (b->exec && b->exec_chunk == b->chunk && b->exec_grid == grid) return PBIT_OK;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    cudaStream_t cap = nullptr;
    PBIT_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    ChunkArgs c{};
    c.inst = b->d_inst;
    c.tile_prefix = b->d_prefix;
    c.count = b->count;
    c.total_tiles = b->total_tiles;
    c.K = b->chunk;
    c.tpi = b->tpi;
    c.queue = b->d_ctl;
    c.tiles_done = b->d_ctl + 1;
    c.err = nullptr;
    {
        const TestFault tf = test_fault("batch", 1ll << 31);
        c.wait_cycles = tf.wait_cycles;
        c.withhold = tf.withhold;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        c.err = b->graphs[0]->err;
        launch_chunk(b->variants, grid, c, cap);
        batch_advance_kernel<<<(b->count + 255) / 256, 256, 0, cap>>>(b->d_inst, b->count, b->chunk, b->d_ctl,
                                                                      b->d_ctl + 1);
        e = cudaStreamEndCapture(cap, &graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    (void)user;
    if (e != cudaSuccess) return cuda_fail(e, "batch: graph capture");
    b->exec_chunk = b->chunk;
    b->exec_grid = grid;
    return PBIT_OK;
}

void advance_mirror(pbit_batch b) {
    for (auto& d : b->host_desc) {
        if (!d.active) continue;
        const int ran = std::min(b->chunk, std::max(0, d.end - d.cur));
        d.cur += ran;
        d.parity = (d.parity + ran) & 1;
    }
}

int32_t chunks_left(pbit_batch b) {
    int32_t most = 0;
    for (auto& d : b->host_desc)
        if (d.active) most = std::max(most, d.end - d.cur);
    return (most + b->chunk - 1) / b->chunk;
}

}  // namespace

extern "C" {

pbit_status pbit_batch_create(int32_t count, const pbit_graph* graphs, const pbit_anneal_params* params,
                              pbit_batch* out) {
    if (!out || count < 1 || !graphs || !params) return fail(PBIT_E_INVALID, "batch_create: bad argument");
    *out = nullptr;
    std::unique_ptr<pbit_batch_s> b(new (std::nothrow) pbit_batch_s());
    if (!b) return fail(PBIT_E_NOMEM, "batch_create: host allocation");
    PBIT_CUDA_TRY(cudaGetDevice(&b->device));
    b->count = count;
    b->graphs.assign(graphs, graphs + count);
    b->host_desc.resize((size_t)count);
    b->tile_prefix.assign((size_t)count + 1, 0);
    cudaStream_t s = nullptr;
    pbit_status st;
    for (int32_t k = 0; k < count; ++k) {
        const pbit_graph g = graphs[k];
        if (!g || g->device != b->device)
            return fail(PBIT_E_INVALID, "batch_create: bad graph or graphs on different devices at " + std::to_string(k));
        InstDesc& d = b->host_desc[(size_t)k];
        if ((st = build_inst(*g, params[k], s, b->allocs, d, nullptr)) != PBIT_OK) return st;
        b->variants = b->variants || is_variant(d.a);
    }
    {
        int sms = 0;
        PBIT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
        b->tpi = plan_chunk(b->host_desc.data(), count, sms * std::max(1, chunk_occupancy(b->variants)));
    }
    for (int32_t k = 0; k < count; ++k)
        b->tile_prefix[(size_t)k + 1] = b->tile_prefix[(size_t)k] + b->host_desc[(size_t)k].tiles;
    b->total_tiles = b->tile_prefix[(size_t)count];
    PBIT_CUDA_TRY(cudaMalloc((void**)&b->d_inst, sizeof(InstDesc) * (size_t)count));
    PBIT_CUDA_TRY(cudaMalloc((void**)&b->d_prefix, sizeof(int32_t) * ((size_t)count + 1)));
    PBIT_CUDA_TRY(cudaMalloc((void**)&b->d_ctl, sizeof(unsigned) * ((size_t)count + 1)));
    PBIT_CUDA_TRY(cudaMemcpy(b->d_prefix, b->tile_prefix.data(), sizeof(int32_t) * ((size_t)count + 1),
                             cudaMemcpyHostToDevice));
    PBIT_CUDA_TRY(cudaMemset(b->d_ctl, 0, sizeof(unsigned) * ((size_t)count + 1)));
    PBIT_CUDA_TRY(cudaDeviceSynchronize());
    if ((st = upload_desc(b.get(), s)) != PBIT_OK) return st;
    *out = b.release();
    return PBIT_OK;
}

void pbit_batch_destroy(pbit_batch b) { delete b; }

pbit_status pbit_batch_set_spins(pbit_batch b, int32_t k, const int8_t* spins, void* stream) {
    if (!b || k < 0 || k >= b->count || !spins) return fail(PBIT_E_INVALID, "batch_set_spins: bad argument");
    InstDesc& d = b->host_desc[(size_t)k];
    // both buffers, so the output buffer of the next step never holds a state older than this one
    for (int q = 0; q < 2; ++q)
        PBIT_CUDA_TRY(cudaMemcpy2DAsync(d.buf[q], (size_t)d.a.T, spins, (size_t)d.T_real, (size_t)d.T_real,
                                        (size_t)d.a.n, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return PBIT_OK;
}

pbit_status pbit_batch_run(pbit_batch b, int32_t chunk_steps, int32_t max_chunks, void* stream) {
    if (!b || chunk_steps < 0 || max_chunks < 0) return fail(PBIT_E_INVALID, "batch_run: bad argument");
    int cur = -1;
    PBIT_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != b->device) return fail(PBIT_E_INVALID, "batch_run: current device is not the batch's device");
    if (chunk_steps > 0) b->chunk = chunk_steps;
    pbit_status st = ensure_graph(b, (cudaStream_t)stream);
    if (st != PBIT_OK) return st;
    int32_t n = chunks_left(b);
    if (max_chunks > 0) n = std::min(n, max_chunks);
    cudaStream_t s = (cudaStream_t)stream;
    for (int32_t c = 0; c < n; ++c) {
        PBIT_CUDA_TRY(cudaGraphLaunch(b->exec, s));
        advance_mirror(b);
    }
    count_launches(2 * (int64_t)n);
    return PBIT_OK;
}

pbit_status pbit_batch_progress(pbit_batch b, int32_t k, int32_t* step) {
    if (!b || k < 0 || k >= b->count || !step) return fail(PBIT_E_INVALID, "batch_progress: bad argument");
    *step = b->host_desc[(size_t)k].cur;
    return PBIT_OK;
}

pbit_status pbit_batch_spins(pbit_batch b, int32_t k, int8_t* spins_out, void* stream) {
    if (!b || k < 0 || k >= b->count || !spins_out) return fail(PBIT_E_INVALID, "batch_spins: bad argument");
    const InstDesc& d = b->host_desc[(size_t)k];
    PBIT_CUDA_TRY(cudaMemcpy2DAsync(spins_out, (size_t)d.T_real, d.buf[d.parity], (size_t)d.a.T, (size_t)d.T_real,
                                    (size_t)d.a.n, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return PBIT_OK;
}

pbit_status pbit_batch_cuts(pbit_batch b, int32_t k, int64_t* cuts, void* stream) {
    if (!b || k < 0 || k >= b->count || !cuts) return fail(PBIT_E_INVALID, "batch_cuts: bad argument");
    const InstDesc& d = b->host_desc[(size_t)k];
    return padded_cuts(b->graphs[(size_t)k], d, cuts, (cudaStream_t)stream);
}

// Time one chunk for each candidate (chunk length, CTAs per SM) from the
// current state, restore the state after each trial, keep the fastest.
pbit_status pbit_batch_autotune(pbit_batch b, void* stream, pbit_batch_tuning* chosen) {
    if (!b) return fail(PBIT_E_INVALID, "batch_autotune: NULL batch");
    cudaStream_t s = (cudaStream_t)stream;
    pbit_status st;
    // snapshot of every instance's current spins and the descriptors
    std::vector<InstDesc> saved_desc = b->host_desc;
    std::vector<int8_t*> backup((size_t)b->count, nullptr);
    for (int32_t k = 0; k < b->count; ++k) {
        const InstDesc& d = b->host_desc[(size_t)k];
        const size_t cells = (size_t)d.a.n * (size_t)d.a.T;
        PBIT_CUDA_TRY(cudaMallocAsync((void**)&backup[(size_t)k], cells, s));
        PBIT_CUDA_TRY(cudaMemcpyAsync(backup[(size_t)k], d.buf[d.parity], cells, cudaMemcpyDeviceToDevice, s));
    }
    const int32_t chunks[] = {8, 16, 32, 64};
    const int32_t ctas[] = {1, 2, 4, 0};
    int32_t best_chunk = b->chunk, best_ctas = b->ctas_per_sm;
    float best = 1e30f;
    cudaEvent_t e0, e1;
    PBIT_CUDA_TRY(cudaEventCreate(&e0));
    PBIT_CUDA_TRY(cudaEventCreate(&e1));
    int32_t most = 0;
    for (auto& d : saved_desc)
        if (d.active) most = std::max(most, d.end - d.cur);
    for (int32_t ch : chunks) {
        if (most > 0 && ch > most) continue;
        for (int32_t cp : ctas) {
            b->chunk = ch;
            b->ctas_per_sm = cp;
            if ((st = ensure_graph(b, s)) != PBIT_OK) return st;
            PBIT_CUDA_TRY(cudaEventRecord(e0, s));
            PBIT_CUDA_TRY(cudaGraphLaunch(b->exec, s));
            PBIT_CUDA_TRY(cudaEventRecord(e1, s));
            PBIT_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.0f;
            PBIT_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            const float per_step = ms / (float)std::max(1, std::min(ch, most));
            if (per_step < best) {
                best = per_step;
                best_chunk = ch;
                best_ctas = cp;
            }
            // restore the state
            b->host_desc = saved_desc;
            for (int32_t k = 0; k < b->count; ++k) {
                const InstDesc& d = b->host_desc[(size_t)k];
                const size_t cells = (size_t)d.a.n * (size_t)d.a.T;
                PBIT_CUDA_TRY(cudaMemcpyAsync(d.buf[d.parity], backup[(size_t)k], cells, cudaMemcpyDeviceToDevice, s));
            }
            if ((st = upload_desc(b, s)) != PBIT_OK) return st;
        }
    }
    count_launches(0);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int8_t* p : backup) cudaFreeAsync(p, s);
    PBIT_CUDA_TRY(cudaStreamSynchronize(s));
    b->chunk = best_chunk;
    b->ctas_per_sm = best_ctas;
    if (chosen) {
        chosen->chunk_steps = best_chunk;
        chosen->ctas_per_sm = best_ctas;
        chosen->ms_per_step = best;
    }
    return PBIT_OK;
}

pbit_status pbit_batch_set_tuning(pbit_batch b, int32_t chunk_steps, int32_t ctas_per_sm) {
    if (!b || chunk_steps < 1 || ctas_per_sm < 0) return fail(PBIT_E_INVALID, "batch_set_tuning: bad argument");
    b->chunk = chunk_steps;
    b->ctas_per_sm = ctas_per_sm;
    return PBIT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- server ----
// Continuous batching: a worker thread owns a stream and a slot table of
// resident instances.  Between chunks it retires finished instances (exact
// cuts, latency), frees their memory, and admits queued requests while the
// HBM budget and the slot count allow; each chunk is one persistent launch
// over every resident instance.  Requests that arrive while others run join
// at the next chunk boundary, so their work overlaps on the device.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id = 0;
    pbit_graph g = nullptr;
    pbit_anneal_params p{};
    std::vector<float> lam, del, pu, nudev;
    size_t bytes = 0;
    Clock::time_point t_submit, t_done;
    int state = 0;  // 0 queued, 1 running, 2 done, 3 failed
    pbit_status err = PBIT_OK;
    std::vector<int64_t> cuts;
    InstDesc desc{};
    std::vector<void*> allocs;
    std::vector<std::vector<uint32_t>> keep;
};

}  // namespace

struct pbit_server_s {
    int device = 0;
    size_t budget = 0, in_use = 0;
    int32_t max_slots = 0, chunk = 64;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::deque<uint64_t> queue;
    std::map<uint64_t, std::unique_ptr<Request>> reqs;
    std::vector<uint64_t> running;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread worker;
    cudaStream_t stream = nullptr;
    InstDesc* d_inst = nullptr;
    int32_t* d_prefix = nullptr;
    unsigned* d_ctl = nullptr;
    int* d_err = nullptr;
    // statistics
    uint64_t completed = 0, chunks = 0;
    double updates = 0.0, busy_s = 0.0;
    int32_t peak_resident = 0;
};

namespace {

void server_loop(pbit_server_s* S) {
    cudaSetDevice(S->device);
    std::vector<InstDesc> desc;
    std::vector<int32_t> prefix;
    // FIFO admission while a slot and the budget allow (caller holds the lock)
    auto admit = [S](std::unique_lock<std::mutex>& lk) {
        while (!S->queue.empty() && (int32_t)S->running.size() < S->max_slots) {
            Request* r = S->reqs[S->queue.front()].get();
            if (S->in_use + r->bytes > S->budget) break;
            S->queue.pop_front();
            S->in_use += r->bytes;
            r->state = 1;
            S->running.push_back(r->id);
            lk.unlock();
            pbit_status st = build_inst(*r->g, r->p, S->stream, r->allocs, r->desc, &r->keep);
            lk.lock();
            if (st != PBIT_OK) {
                r->state = 3;
                r->err = st;
                S->running.erase(std::find(S->running.begin(), S->running.end(), r->id));
                S->in_use -= r->bytes;
                S->done_cv.notify_all();
            }
        }
    };
    for (;;) {
        std::vector<Request*> active;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            admit(lk);
            if (S->running.empty()) {
                if (S->stop) return;
                S->cv.wait_for(lk, std::chrono::milliseconds(20));
                continue;
            }
            for (uint64_t id : S->running) active.push_back(S->reqs[id].get());
            S->peak_resident = std::max<int32_t>(S->peak_resident, (int32_t)active.size());
        }
        // one chunk over every resident instance
        const auto t0 = Clock::now();
        const int32_t count = (int32_t)active.size();
        desc.resize((size_t)count);
        prefix.assign((size_t)count + 1, 0);
        double upd = 0.0;
        bool variants = false;
        for (int32_t k = 0; k < count; ++k) {
            desc[(size_t)k] = active[(size_t)k]->desc;
            variants = variants || is_variant(desc[(size_t)k].a);
        }
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, S->device);
        const int occ = chunk_occupancy(variants);
        const int grid = std::max(1, sms * std::max(1, occ));
        const int tpi = plan_chunk(desc.data(), count, grid);  // the resident load sets the tiling
        for (int32_t k = 0; k < count; ++k) {
            prefix[(size_t)k + 1] = prefix[(size_t)k] + desc[(size_t)k].tiles;
            const InstDesc& d = desc[(size_t)k];
            upd += (double)d.a.n * d.a.T * std::min(S->chunk, d.end - d.cur);
        }
        cudaMemcpyAsync(S->d_inst, desc.data(), sizeof(InstDesc) * (size_t)count, cudaMemcpyHostToDevice, S->stream);
        cudaMemcpyAsync(S->d_prefix, prefix.data(), sizeof(int32_t) * ((size_t)count + 1), cudaMemcpyHostToDevice,
                        S->stream);
        cudaMemsetAsync(S->d_ctl, 0, sizeof(unsigned) * ((size_t)count + 1), S->stream);
        ChunkArgs c{};
        c.inst = S->d_inst;
        c.tile_prefix = S->d_prefix;
        c.count = count;
        c.total_tiles = prefix[(size_t)count];
        c.K = S->chunk;
        c.tpi = tpi;
        c.queue = S->d_ctl;
        c.tiles_done = S->d_ctl + 1;
        c.err = S->d_err;
        const TestFault tf = test_fault("batch", 1ll << 31);
        c.wait_cycles = tf.wait_cycles;
        c.withhold = tf.withhold;
        launch_chunk(variants, grid, c, S->stream);
        count_launches(1);
        {
            // requests arriving meanwhile are prepared now and join at the next chunk
            std::unique_lock<std::mutex> lk(S->mu);
            admit(lk);
        }
        cudaError_t ce = cudaStreamSynchronize(S->stream);
        // a bounded wait that gave up stopped the chunk: the resident requests fail with PBIT_E_TIMEOUT
        int herr = 0;
        if (ce == cudaSuccess) {
            ce = cudaMemcpyAsync(&herr, S->d_err, sizeof(int), cudaMemcpyDeviceToHost, S->stream);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(S->stream);
        }
        const bool timed_out = ce == cudaSuccess && herr != 0;
        if (timed_out) {
            cudaMemsetAsync(S->d_err, 0, sizeof(int), S->stream);
            cudaStreamSynchronize(S->stream);
        }
        const auto t1 = Clock::now();
        // retire finished instances
        std::vector<Request*> finished;
        for (int32_t k = 0; k < count; ++k) {
            Request* r = active[(size_t)k];
            InstDesc& d = r->desc;
            const int ran = std::min(S->chunk, std::max(0, d.end - d.cur));
            d.cur += ran;
            d.parity = (d.parity + ran) & 1;
            if (d.cur >= d.end || ce != cudaSuccess || timed_out) finished.push_back(r);
        }
        for (Request* r : finished) {
            r->cuts.assign((size_t)r->p.trials, 0);
            pbit_status st = timed_out ? fail(PBIT_E_TIMEOUT, "server chunk: a bounded device-side wait gave up")
                             : ce == cudaSuccess ? padded_cuts(r->g, r->desc, r->cuts.data(), S->stream)
                                                 : cuda_fail(ce, "server chunk");
            for (void* p : r->allocs) cudaFreeAsync(p, S->stream);
            r->allocs.clear();
            std::lock_guard<std::mutex> lk(S->mu);
            r->t_done = Clock::now();
            r->state = st == PBIT_OK ? 2 : 3;
            r->err = st;
            S->in_use -= r->bytes;
            S->running.erase(std::find(S->running.begin(), S->running.end(), r->id));
            S->completed += 1;
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->chunks += 1;
            S->updates += upd;
            S->busy_s += std::chrono::duration<double>(t1 - t0).count();
        }
        if (!finished.empty()) S->done_cv.notify_all();
    }
}

}  // namespace

extern "C" {

pbit_status pbit_server_create(size_t hbm_budget, int32_t max_slots, int32_t chunk_steps, pbit_server* out) {
    if (!out || hbm_budget == 0 || max_slots < 1 || chunk_steps < 1)
        return fail(PBIT_E_INVALID, "server_create: bad argument");
    *out = nullptr;
    std::unique_ptr<pbit_server_s> S(new (std::nothrow) pbit_server_s());
    if (!S) return fail(PBIT_E_NOMEM, "server_create: host allocation");
    PBIT_CUDA_TRY(cudaGetDevice(&S->device));
    S->budget = hbm_budget;
    S->max_slots = max_slots;
    S->chunk = chunk_steps;
    PBIT_CUDA_TRY(cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking));
    PBIT_CUDA_TRY(cudaMalloc((void**)&S->d_inst, sizeof(InstDesc) * (size_t)max_slots));
    PBIT_CUDA_TRY(cudaMalloc((void**)&S->d_prefix, sizeof(int32_t) * ((size_t)max_slots + 1)));
    PBIT_CUDA_TRY(cudaMalloc((void**)&S->d_ctl, sizeof(unsigned) * ((size_t)max_slots + 1)));
    PBIT_CUDA_TRY(cudaMalloc((void**)&S->d_err, sizeof(int)));
    PBIT_CUDA_TRY(cudaMemset(S->d_err, 0, sizeof(int)));
    pbit_server_s* raw = S.get();
    S->worker = std::thread(server_loop, raw);
    *out = S.release();
    return PBIT_OK;
}

void pbit_server_destroy(pbit_server S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        // queued requests that never started are dropped
        for (uint64_t id : S->queue) {
            S->reqs[id]->state = 3;
            S->reqs[id]->err = PBIT_E_INVALID;
        }
        S->queue.clear();
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(S->device);
    cudaStreamSynchronize(S->stream);
    cudaStreamDestroy(S->stream);
    cudaFree(S->d_inst);
    cudaFree(S->d_prefix);
    cudaFree(S->d_ctl);
    cudaFree(S->d_err);
    cudaSetDevice(cur);
    delete S;
}

pbit_status pbit_server_submit(pbit_server S, pbit_graph g, const pbit_anneal_params* p, uint64_t* req_id) {
    if (!S || !g || !p || !req_id) return fail(PBIT_E_INVALID, "server_submit: bad argument");
    if (p->struct_size != sizeof(pbit_anneal_params)) return fail(PBIT_E_INVALID, "server_submit: struct_size");
    if (g->device != S->device) return fail(PBIT_E_INVALID, "server_submit: graph on another device");
    const int32_t S_ = p->steps, e = p->step_end == 0 ? p->steps : p->step_end;
    if (p->trials < 1 || S_ < 1 || p->step_begin < 0 || e < p->step_begin || e > S_)
        return fail(PBIT_E_INVALID, "server_submit: bad trials/steps");
    std::unique_ptr<Request> r(new (std::nothrow) Request());
    if (!r) return fail(PBIT_E_NOMEM, "server_submit: host allocation");
    r->g = g;
    r->p = *p;
    const size_t n = (size_t)g->n;
    if (p->intensity) {
        r->lam.assign(p->intensity, p->intensity + n);
        r->p.intensity = r->lam.data();
    }
    if (p->offset) {
        r->del.assign(p->offset, p->offset + n);
        r->p.offset = r->del.data();
    }
    if (p->p_update) {
        r->pu.assign(p->p_update, p->p_update + n);
        r->p.p_update = r->pu.data();
    }
    if (p->nu_dev) {
        r->nudev.assign(p->nu_dev, p->nu_dev + n);
        r->p.nu_dev = r->nudev.data();
    }
    r->p.state = nullptr;
    r->bytes = inst_bytes(*g, *p);
    if (r->bytes > S->budget) return fail(PBIT_E_BUDGET, "server_submit: request needs " +
                                                             std::to_string(r->bytes) + " bytes, budget is " +
                                                             std::to_string(S->budget));
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) return fail(PBIT_E_INVALID, "server_submit: server is stopping");
        r->id = S->next_id++;
        *req_id = r->id;
        S->queue.push_back(r->id);
        S->reqs[r->id] = std::move(r);
    }
    S->cv.notify_all();
    return PBIT_OK;
}

static pbit_status take_result(pbit_server S, std::map<uint64_t, std::unique_ptr<Request>>::iterator it,
                               int64_t* cuts, double* latency_s) {
    Request* r = it->second.get();
    if (r->state == 3) {
        const pbit_status e = r->err != PBIT_OK ? r->err : PBIT_E_INVALID;
        S->reqs.erase(it);
        return fail(e, "server: request failed or was cancelled");
    }
    if (cuts) std::memcpy(cuts, r->cuts.data(), sizeof(int64_t) * r->cuts.size());
    if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    S->reqs.erase(it);
    return PBIT_OK;
}

pbit_status pbit_server_poll(pbit_server S, uint64_t req_id, int64_t* cuts, double* latency_s) {
    if (!S) return fail(PBIT_E_INVALID, "server_poll: NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end()) return fail(PBIT_E_NOTFOUND, "server_poll: unknown request id");
    if (it->second->state < 2) return PBIT_PENDING;
    return take_result(S, it, cuts, latency_s);
}

pbit_status pbit_server_wait(pbit_server S, uint64_t req_id, double timeout_s, int64_t* cuts, double* latency_s) {
    if (!S) return fail(PBIT_E_INVALID, "server_wait: NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(
                                             timeout_s > 0 ? timeout_s : 1e9));
    for (;;) {
        auto it = S->reqs.find(req_id);
        if (it == S->reqs.end()) return fail(PBIT_E_NOTFOUND, "server_wait: unknown request id");
        if (it->second->state >= 2) return take_result(S, it, cuts, latency_s);
        if (S->done_cv.wait_until(lk, deadline) == std::cv_status::timeout) return PBIT_PENDING;
    }
}

pbit_status pbit_server_stats(pbit_server S, pbit_server_stats_t* out) {
    if (!S || !out) return fail(PBIT_E_INVALID, "server_stats: bad argument");
    std::lock_guard<std::mutex> lk(S->mu);
    out->completed = S->completed;
    out->queued = (uint64_t)S->queue.size();
    out->resident = (int32_t)S->running.size();
    out->peak_resident = S->peak_resident;
    out->chunks = S->chunks;
    out->spin_updates = S->updates;
    out->busy_seconds = S->busy_s;
    out->hbm_in_use = S->in_use;
    return PBIT_OK;
}

}  // extern "C"
