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
    int32_t tiles;     // tiles per step
    int32_t active;    // 0 = slot unused
};

struct ChunkArgs {
    InstDesc* inst;
    const int32_t* tile_prefix;  // [count + 1]
    int32_t count;
    int32_t total_tiles;
    int32_t K;
    unsigned* queue;             // item counter
    unsigned* tiles_done;        // [count] tiles finished in this chunk
    int* err;
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

__device__ void dispatch_tile(const StepArgs& a, int G, int unit, int table, int64_t first, uint32_t* s_tab) {
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

__global__ void __launch_bounds__(kBlock) batch_chunk_kernel(ChunkArgs c) {
    __shared__ uint32_t s_tab[kTabMax];
    __shared__ unsigned s_item;
    __shared__ int s_ok;
    const unsigned total = (unsigned)c.K * (unsigned)c.total_tiles;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(c.queue, 1u);
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
                    if (clock64() - start > (1ll << 31)) {
                        atomicExch(c.err, 4);
                        ok = 0;
                        break;
                    }
                }
            }
            s_ok = ok;
        }
        __syncthreads();
        StepArgs a = d.a;
        a.step = d.cur + k;
        const int par = (d.parity + k) & 1;
        a.in = d.buf[par];
        a.out = d.buf[par ^ 1];
        dispatch_tile(a, d.G, d.unit, d.table, (int64_t)tile_i * kBlock, s_tab);
        __threadfence();  // this thread's spin stores, before the tile is counted
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(c.tiles_done + g, 1u);
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
    // tuning
    int32_t chunk = 32;
    int32_t ctas_per_sm = 0;             // 0 = occupancy maximum
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

template <typename T>
pbit_status dev_alloc(pbit_batch b, T** p, size_t count) {
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
    if (e != cudaSuccess) return cuda_fail(e, "batch: cudaMalloc");
    b->allocs.push_back((void*)*p);
    return PBIT_OK;
}

int grid_for(pbit_batch b) {
    int sms = 0, occ = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_chunk_kernel, kBlock, 0);
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
    c.queue = b->d_ctl;
    c.tiles_done = b->d_ctl + 1;
    c.err = nullptr;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        c.err = b->graphs[0]->err;
        batch_chunk_kernel<<<grid, kBlock, 0, cap>>>(c);
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
        const pbit_anneal_params* p = &params[k];
        if (!g || p->struct_size != sizeof(pbit_anneal_params))
            return fail(PBIT_E_INVALID, "batch_create: bad graph or params at " + std::to_string(k));
        if (g->device != b->device) return fail(PBIT_E_INVALID, "batch_create: graphs on different devices");
        const int32_t T = p->trials, S = p->steps;
        const int32_t sb = p->step_begin, se = p->step_end == 0 ? S : p->step_end;
        if (T < 1 || S < 1 || sb < 0 || se < sb || se > S || p->offset_mode < 0 || p->offset_mode > 2)
            return fail(PBIT_E_INVALID, "batch_create: bad trials/steps at " + std::to_string(k));
        std::vector<float> tab;
        if ((st = build_schedule(*g, p->i0_min, p->i0_max, p->i0_normalize, S, tab)) != PBIT_OK) return st;
        InstDesc& d = b->host_desc[(size_t)k];
        std::memset(&d, 0, sizeof(d));
        StepArgs& a = d.a;
        a.row_ptr = g->row_ptr;
        a.col = g->col;
        a.J = g->J;
        a.h = g->h;
        a.wabs = g->wabs;
        a.tab_off = g->tab_off;
        a.n = g->n;
        a.T = T;
        a.seed_lo = (uint32_t)(p->seed & 0xFFFFFFFFu);
        a.seed_hi = (uint32_t)(p->seed >> 32);
        a.instance = p->instance;
        a.offset_mode = p->offset_mode;
        float* d_tab = nullptr;
        if ((st = dev_alloc(b.get(), &d_tab, tab.size())) != PBIT_OK) return st;
        PBIT_CUDA_TRY(cudaMemcpy(d_tab, tab.data(), sizeof(float) * tab.size(), cudaMemcpyHostToDevice));
        a.i0_table = d_tab;
        const size_t n = (size_t)g->n;
        if (p->intensity) {
            float* dp = nullptr;
            if ((st = dev_alloc(b.get(), &dp, n)) != PBIT_OK) return st;
            PBIT_CUDA_TRY(cudaMemcpy(dp, p->intensity, sizeof(float) * n, cudaMemcpyHostToDevice));
            a.par.lambda = dp;
        }
        if (p->offset) {
            float* dp = nullptr;
            if ((st = dev_alloc(b.get(), &dp, n)) != PBIT_OK) return st;
            PBIT_CUDA_TRY(cudaMemcpy(dp, p->offset, sizeof(float) * n, cudaMemcpyHostToDevice));
            a.par.delta = dp;
        }
        if (p->p_update) {
            std::vector<uint32_t> thr(n);
            for (size_t i = 0; i < n; ++i) {
                const float pu = p->p_update[i];
                if (!(pu >= 0.0f && pu <= 1.0f)) return fail(PBIT_E_INVALID, "batch_create: p_update outside [0,1]");
                thr[i] = (uint32_t)std::ceil((double)pu * 16777216.0);
            }
            uint32_t* dp = nullptr;
            if ((st = dev_alloc(b.get(), &dp, n)) != PBIT_OK) return st;
            PBIT_CUDA_TRY(cudaMemcpy(dp, thr.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice));
            a.par.thr = dp;
        }
        const size_t cells = n * (size_t)T;
        if ((st = dev_alloc(b.get(), &d.buf[0], (cells + 15) / 16 * 16)) != PBIT_OK) return st;
        if ((st = dev_alloc(b.get(), &d.buf[1], (cells + 15) / 16 * 16)) != PBIT_OK) return st;
        PBIT_CUDA_TRY(launch_init_spins(g->n, T, p->seed, p->instance, d.buf[0], s));
        d.cur = sb;
        d.end = se;
        d.parity = 0;
        d.G = T % 16 == 0 ? 16 : (T % 4 == 0 ? 4 : 1);
        const SparseVariant v = choose_sparse_variant(*g, T);
        d.unit = v.unit ? 1 : 0;
        d.table = v.table ? 1 : 0;
        const int64_t items = (int64_t)g->n * (T / d.G);
        d.tiles = (int32_t)((items + kBlock - 1) / kBlock);
        d.active = 1;
        b->tile_prefix[(size_t)k + 1] = b->tile_prefix[(size_t)k] + d.tiles;
    }
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
    const size_t cells = (size_t)d.a.n * (size_t)d.a.T;
    PBIT_CUDA_TRY(cudaMemcpyAsync(d.buf[d.parity], spins, cells, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
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
    const size_t cells = (size_t)d.a.n * (size_t)d.a.T;
    PBIT_CUDA_TRY(cudaMemcpyAsync(spins_out, d.buf[d.parity], cells, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return PBIT_OK;
}

pbit_status pbit_batch_cuts(pbit_batch b, int32_t k, int64_t* cuts, void* stream) {
    if (!b || k < 0 || k >= b->count || !cuts) return fail(PBIT_E_INVALID, "batch_cuts: bad argument");
    const InstDesc& d = b->host_desc[(size_t)k];
    return pbit_cut(b->graphs[(size_t)k], d.buf[d.parity], d.a.T, cuts, 1, stream);
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
