// pbit_anneal_noalloc: the sparse annealing path with all of its scratch in
// a fixed, file-scope device array instead of memory allocated per call.
//
// Who needs this: callers that must not allocate device memory while they
// run.  Examples are applications whose own caching allocator has reserved
// nearly all of HBM up front (a cudaMalloc from a library would fail, or
// would take memory the application has already promised elsewhere),
// processes that run under a fixed device-memory cap, and latency-bound
// service loops that cannot afford the implicit synchronisation and
// unbounded latency an allocation may bring.
//
// What it still does: it calls the CUDA runtime (cudaGetDevice,
// cudaGetSymbolAddress, cudaMemcpyAsync, kernel launches), so it must not be
// called from a stream callback or host function, where CUDA forbids every
// API call; and its parameter uploads (I0 table, intensity, offset, update
// thresholds) are cudaMemcpyAsync copies from pageable host memory, which
// the runtime stages synchronously, so the call is not meant for stream
// capture (the same as pbit_anneal).
//
// The scratch array is kNoAllocScratchBytes (32 MiB) of global memory,
// reserved on every GPU that loads libpbit.so until the process exits.
// It holds, per call: the float32 I0 table, the per-node intensity, offset
// and update thresholds, and the second spin buffer of the synchronous
// (Jacobi) update.  Each region is completely written before it is read, so
// nothing in it has to start at zero and nothing is cleared.  Every call
// reuses the same array and leaves the last call's data in it; two calls
// whose GPU work overlaps (for example on two streams) race on it.
//
// The steps run the graph's per-step sparse tile (packed +-1 counting, the
// threshold table or the warp-table tile, as pbit_anneal picks them); the
// multi-step launch is not used, because its dependency lists and counters
// are allocated memory.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "pbit_internal.h"

namespace pbit {
namespace {

constexpr size_t kNoAllocScratchBytes = 32u << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the scratch array on the current device.  Host code sees
// only a host-side stand-in under the array's name, so the real address is
// looked up with cudaGetSymbolAddress while the graph's device is current.
// The lookup allocates nothing and is repeated on every call, so no cached
// address can outlive a cudaDeviceReset.
pbit_status scratch_address(unsigned char** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "anneal_noalloc: cudaGetSymbolAddress");
    *out = static_cast<unsigned char*>(p);
    return PBIT_OK;
}

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace pbit

using namespace pbit;

extern "C" pbit_status pbit_anneal_noalloc(pbit_graph g, const pbit_anneal_params* p, const int8_t* spins_in,
                                           int8_t* spins_out) {
    Graph* gr = static_cast<Graph*>(g);
    if (!gr || !p || !spins_out) return fail(PBIT_E_INVALID, "anneal_noalloc: NULL argument");
    if (p->struct_size != sizeof(pbit_anneal_params))
        return fail(PBIT_E_INVALID, "anneal_noalloc: struct_size mismatch");
    const int32_t T = p->trials, S = p->steps;
    const int32_t b = p->step_begin, e = p->step_end == 0 ? S : p->step_end;
    if (T < 1 || S < 1 || b < 0 || e < b || e > S) return fail(PBIT_E_INVALID, "anneal_noalloc: bad trials/steps range");
    if (p->offset_mode < 0 || p->offset_mode > 2) return fail(PBIT_E_INVALID, "anneal_noalloc: bad offset_mode");
    if (p->algorithm != PBIT_ALG_PSA || p->t_res > 0)
        return fail(PBIT_E_UNSUPPORTED, "anneal_noalloc: plain pSA only");
    int device = -1;
    PBIT_CUDA_TRY(cudaGetDevice(&device));
    if (device != gr->device) return fail(PBIT_E_INVALID, "anneal_noalloc: current device is not the graph's device");

    const size_t n = (size_t)gr->n;
    const size_t cells = n * (size_t)T;
    const size_t off_tab = 0;
    const size_t off_lam = off_tab + round256(sizeof(float) * (size_t)S);
    const size_t off_del = off_lam + round256(sizeof(float) * n);
    const size_t off_thr = off_del + round256(sizeof(float) * n);
    const size_t off_spin = off_thr + round256(sizeof(uint32_t) * n);
    const size_t need = off_spin + round256(cells);
    if (need > kNoAllocScratchBytes)
        return fail(PBIT_E_INVALID, "anneal_noalloc: needs " + std::to_string(need) +
                                        " bytes of scratch (4*steps + 12*n + n*trials, each rounded up to 256), "
                                        "more than its fixed " + std::to_string(kNoAllocScratchBytes) + " bytes");

    std::vector<float> tab;
    pbit_status st = build_schedule(*gr, p->i0_min, p->i0_max, p->i0_normalize, S, tab);
    if (st != PBIT_OK) return st;
    std::vector<uint32_t> thr;
    if (p->p_update) {
        thr.resize(n);
        for (size_t i = 0; i < n; ++i) {
            const float pu = p->p_update[i];
            if (!(pu >= 0.0f && pu <= 1.0f)) return fail(PBIT_E_INVALID, "anneal_noalloc: p_update outside [0,1]");
            thr[i] = (uint32_t)std::ceil((double)pu * 16777216.0);
        }
    }
    if (p->intensity)
        for (size_t i = 0; i < n; ++i)
            if (!std::isfinite(p->intensity[i])) return fail(PBIT_E_INVALID, "anneal_noalloc: non-finite intensity");
    if (p->offset)
        for (size_t i = 0; i < n; ++i)
            if (!std::isfinite(p->offset[i])) return fail(PBIT_E_INVALID, "anneal_noalloc: non-finite offset");

    unsigned char* base = nullptr;
    if ((st = scratch_address(&base)) != PBIT_OK) return st;
    cudaStream_t s = (cudaStream_t)p->stream;

    StepArgs a{};
    a.row_ptr = gr->row_ptr;
    a.col = gr->col;
    a.J = gr->J;
    a.h = gr->h;
    a.wabs = gr->wabs;
    a.tab_off = gr->tab_off;
    a.n = gr->n;
    a.T = T;
    a.seed_lo = (uint32_t)(p->seed & 0xFFFFFFFFu);
    a.seed_hi = (uint32_t)(p->seed >> 32);
    a.instance = p->instance;
    a.offset_mode = p->offset_mode;
    float* d_tab = reinterpret_cast<float*>(base + off_tab);
    PBIT_CUDA_TRY(cudaMemcpyAsync(d_tab, tab.data(), sizeof(float) * (size_t)S, cudaMemcpyHostToDevice, s));
    a.i0_table = d_tab;
    if (p->intensity) {
        float* d = reinterpret_cast<float*>(base + off_lam);
        PBIT_CUDA_TRY(cudaMemcpyAsync(d, p->intensity, sizeof(float) * n, cudaMemcpyHostToDevice, s));
        a.par.lambda = d;
    }
    if (p->offset) {
        float* d = reinterpret_cast<float*>(base + off_del);
        PBIT_CUDA_TRY(cudaMemcpyAsync(d, p->offset, sizeof(float) * n, cudaMemcpyHostToDevice, s));
        a.par.delta = d;
    }
    if (p->p_update) {
        uint32_t* d = reinterpret_cast<uint32_t*>(base + off_thr);
        PBIT_CUDA_TRY(cudaMemcpyAsync(d, thr.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice, s));
        a.par.thr = d;
    }
    int8_t* scratch = reinterpret_cast<int8_t*>(base + off_spin);

    // Jacobi rotation between spins_out and the scratch spin buffer so that
    // the last step writes spins_out.
    const int32_t k = e - b;
    const int8_t* cur = spins_in;
    if (!cur) {
        int8_t* init = (k == 0 || (k - 1) % 2 != 0) ? spins_out : scratch;
        PBIT_CUDA_TRY(launch_init_spins(gr->n, T, p->seed, p->instance, init, s));
        cur = init;
    }
    if (k == 0) {
        if (cur != spins_out) PBIT_CUDA_TRY(cudaMemcpyAsync(spins_out, cur, cells, cudaMemcpyDeviceToDevice, s));
        return PBIT_OK;
    }
    if (cur == spins_out && (k - 1) % 2 == 0) {
        PBIT_CUDA_TRY(cudaMemcpyAsync(scratch, cur, cells, cudaMemcpyDeviceToDevice, s));
        cur = scratch;
    }
    const SparseVariant v = choose_sparse_variant(*gr, T);
    for (int32_t j = 0; j < k; ++j) {
        int8_t* dst = ((k - 1 - j) % 2 == 0) ? spins_out : scratch;
        a.step = b + j;
        a.in = cur;
        a.out = dst;
        PBIT_CUDA_TRY(launch_sparse_step(a, s, v));
        cur = dst;
    }
    return PBIT_OK;
}
