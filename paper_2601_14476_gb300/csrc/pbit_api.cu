// C-ABI entry points of libpbit.so (declared in include/pbit.h) and the host
// side of the instance: validation, CSR of J = -w, the I0 schedule, per-node
// parameters, buffer rotation for the synchronous (Jacobi) step loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "pbit_internal.h"

namespace pbit {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};

void count_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_last_error = msg; }

pbit_status fail(pbit_status code, const std::string& msg) {
    set_error(msg);
    return code;
}

pbit_status cuda_fail(cudaError_t err, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(err);
    set_error(m);
    return err == cudaErrorMemoryAllocation ? PBIT_E_NOMEM : PBIT_E_CUDA;
}

// --------------------------------------------------------------- schedule ---
pbit_status build_schedule(const Graph& g, double i0_min, double i0_max, int normalize, int steps,
                           std::vector<float>& out) {
    if (steps < 1) return fail(PBIT_E_INVALID, "schedule: steps must be >= 1");
    if (!(i0_min > 0.0) || !(i0_max > 0.0) || !std::isfinite(i0_min) || !std::isfinite(i0_max))
        return fail(PBIT_E_INVALID, "schedule: I0 end points must be positive and finite");
    double lo = i0_min, hi = i0_max;
    if (normalize) {
        if (!(g.mean_s > 0.0)) return fail(PBIT_E_INVALID, "schedule: mean_s is zero, cannot normalise");
        lo = i0_min / g.mean_s;
        hi = i0_max / g.mean_s;
    }
    out.resize((size_t)steps);
    const double beta = steps > 1 ? std::pow(lo / hi, 1.0 / (double)(steps - 1)) : 1.0;
    double i0 = lo;
    for (int t = 0; t < steps; ++t) {
        out[(size_t)t] = (float)i0;
        i0 = i0 / beta;
    }
    return PBIT_OK;
}

// ---------------------------------------------------------- device memory --
template <typename T>
static pbit_status upload(T** dst, const T* src, size_t count, size_t& bytes) {
    if (count == 0) count = 1;
    PBIT_CUDA_TRY(cudaMalloc((void**)dst, sizeof(T) * count));
    if (src) PBIT_CUDA_TRY(cudaMemcpy(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice));
    bytes += sizeof(T) * count;
    return PBIT_OK;
}

static void release(Graph* g) {
    if (!g) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(g->device);
    cudaDeviceSynchronize();
    cudaFree(g->row_ptr);
    cudaFree(g->col);
    cudaFree(g->J);
    cudaFree(g->h);
    cudaFree(g->dense.J_e4m3);
    cudaFree(g->dense4.J4);
    cudaFree(g->err);
    cudaFree(g->wabs);
    cudaFree(g->tab_off);
    cudaFree(g->flow.ptr);
    cudaFree(g->flow.idx);
    cudaSetDevice(cur);
}

// Per-call device state of one anneal: parameters, schedule and the scratch
// spin buffer, allocated stream-ordered and freed stream-ordered.
struct CallBuffers {
    cudaStream_t s = nullptr;
    std::vector<void*> blocks;
    ~CallBuffers() {
        for (void* p : blocks) cudaFreeAsync(p, s);
    }
    template <typename T>
    pbit_status alloc(T** p, size_t count) {
        if (count == 0) count = 1;
        cudaError_t e = cudaMallocAsync((void**)p, sizeof(T) * count, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
        blocks.push_back((void*)*p);
        return PBIT_OK;
    }
    // copy from (pageable) host memory: CUDA stages the data before the call returns
    template <typename T>
    pbit_status put(T** p, const T* host, size_t count) {
        pbit_status st = alloc(p, count);
        if (st != PBIT_OK) return st;
        cudaError_t e = cudaMemcpyAsync(*p, host, sizeof(T) * count, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
        return PBIT_OK;
    }
};

TestFault test_fault(const char* kernel, long long default_cycles) {
    TestFault f;
    f.wait_cycles = default_cycles;
    const char* w = std::getenv("PBIT_TEST_WITHHOLD");
    if (!w || std::string(w) != kernel) return f;
    f.withhold = 1;
    if (const char* us = std::getenv("PBIT_TEST_WAIT_US")) {
        const long long v = std::atoll(us);
        if (v > 0 && v < 2000000) f.wait_cycles = v * 2000;  // about 2 GHz SM clock
    }
    return f;
}

// Either dense kernel can run T trials on this graph: the cluster-resident FP4 kernel or the e4m3 one.
static bool any_dense_ok(const Graph& g, int32_t T, std::string* why) {
    return dense4_shape_ok(g, T) || dense_shape_ok(g, T, why);
}

// Resolve PBIT_KERNEL_AUTO and check a forced kernel against the shape.
static pbit_status select_kernel(const Graph& g, int requested, int32_t T, int* out, bool variant = false) {
    std::string why;
    if (variant) {
        if (requested == PBIT_KERNEL_DENSE || requested == PBIT_KERNEL_RESIDENT)
            return fail(PBIT_E_UNSUPPORTED, "anneal: SpSA, TApSA and the period timing model run on the sparse kernel");
        *out = PBIT_KERNEL_SPARSE;
        return PBIT_OK;
    }
    if (requested == PBIT_KERNEL_DENSE && !any_dense_ok(g, T, &why)) return fail(PBIT_E_UNSUPPORTED, "anneal: " + why);
    if (requested == PBIT_KERNEL_RESIDENT && !resident_fits(g, T))
        return fail(PBIT_E_UNSUPPORTED, "anneal: n*T too large for the shared-memory resident kernel");
    int k = requested;
    if (k == PBIT_KERNEL_AUTO) {
        if (any_dense_ok(g, T, nullptr))
            k = PBIT_KERNEL_DENSE;
        else
            k = resident_preferred(g, T) ? PBIT_KERNEL_RESIDENT : PBIT_KERNEL_SPARSE;
    }
    *out = k;
    return PBIT_OK;
}

static pbit_status check_device(const Graph* g) {
    int cur = -1;
    PBIT_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != g->device) return fail(PBIT_E_INVALID, "the current CUDA device is not the graph's device");
    return PBIT_OK;
}

// Validate the edge list and build the host CSR of J = -w (rows sorted by
// column), degree and weight statistics and mean_s.  No device work.
static pbit_status build_host(Graph& g, int32_t n, int64_t n_edges, const int32_t* src, const int32_t* dst,
                              const int8_t* w, const int32_t* h) {
    if (n <= 0) return fail(PBIT_E_INVALID, "graph: n must be positive");
    if (n_edges < 0 || n_edges > (int64_t)0x3FFFFFFF) return fail(PBIT_E_INVALID, "graph: bad edge count");
    if (n_edges > 0 && (!src || !dst || !w)) return fail(PBIT_E_INVALID, "graph: NULL edge arrays");
    if (n_edges > (int64_t)n * (n - 1) / 2) return fail(PBIT_E_INVALID, "graph: more edges than node pairs");
    // P host threads for large graphs (at least 256K edges each; per-thread count arrays of n entries)
    const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
    int P = (int)std::max<int64_t>(1, std::min<int64_t>(std::min(hw, 16), n_edges >> 18));
    while (P > 1 && (int64_t)P * n > (int64_t(4) << 20)) --P;
    auto run = [P](auto&& f) {
        std::vector<std::thread> pool;
        for (int t = 1; t < P; ++t) pool.emplace_back(f, t);
        f(0);
        for (auto& th : pool) th.join();
    };
    auto chunk = [&](int t) { return n_edges * t / P; };
    // validation and per-thread endpoint counts; `canonical`: edges strictly increasing in
    // (src, dst) with src < dst
    struct Local {
        int64_t wsum = 0, bad = -1;
        bool unit = true, canonical = true;
    };
    std::vector<Local> loc((size_t)P);
    std::vector<int32_t> cnt_src((size_t)P * n, 0), cnt_dst((size_t)P * n, 0);
    run([&](int t) {
        Local& L = loc[(size_t)t];
        int32_t* cs = cnt_src.data() + (size_t)t * n;
        int32_t* cd = cnt_dst.data() + (size_t)t * n;
        for (int64_t e = chunk(t); e < chunk(t + 1); ++e) {
            const int32_t a = src[e], b = dst[e];
            if (a < 0 || a >= n || b < 0 || b >= n || a == b || w[e] == -128) {
                L.bad = e;
                return;
            }
            L.canonical = L.canonical && a < b && (e == 0 || a > src[e - 1] || (a == src[e - 1] && b > dst[e - 1]));
            cs[a]++;
            cd[b]++;
            L.wsum += w[e];
            if (w[e] != 1 && w[e] != -1) L.unit = false;
        }
    });
    int64_t bad = -1;
    for (const Local& L : loc)
        if (L.bad >= 0 && (bad < 0 || L.bad < bad)) bad = L.bad;
    if (bad >= 0) {
        const int32_t a = src[bad], b = dst[bad];
        if (a < 0 || a >= n || b < 0 || b >= n)
            return fail(PBIT_E_INVALID, "graph: edge endpoint out of range at " + std::to_string(bad));
        if (a == b) return fail(PBIT_E_INVALID, "graph: self loop at " + std::to_string(bad));
        return fail(PBIT_E_INVALID, "graph: weight -128 (J = -w overflows int8)");
    }
    bool canonical = true;
    int64_t wsum = 0;
    g.unit_weights = true;
    for (const Local& L : loc) {
        canonical = canonical && L.canonical;
        wsum += L.wsum;
        g.unit_weights = g.unit_weights && L.unit;
    }
    g.n = n;
    g.n_edges = n_edges;
    g.nnz = 2 * n_edges;
    g.total_weight = wsum;
    // out_deg / in_deg per node, and cnt_dst turned into each thread's first slot among the entries of
    // every destination (exclusive prefix over the threads, which hold consecutive edge ranges)
    std::vector<int32_t> out_deg((size_t)n), in_deg((size_t)n);
    run([&](int t) {
        for (int64_t v = (int64_t)n * t / P; v < (int64_t)n * (t + 1) / P; ++v) {
            int32_t so = 0, si = 0;
            for (int q = 0; q < P; ++q) {
                so += cnt_src[(size_t)q * n + v];
                const int32_t c = cnt_dst[(size_t)q * n + v];
                cnt_dst[(size_t)q * n + v] = si;
                si += c;
            }
            out_deg[(size_t)v] = so;
            in_deg[(size_t)v] = si;
        }
    });
    g.h_row_ptr.assign((size_t)n + 1, 0);
    for (int32_t i = 0; i < n; ++i) g.h_row_ptr[(size_t)i + 1] = g.h_row_ptr[(size_t)i] + out_deg[(size_t)i] + in_deg[(size_t)i];
    g.h_col.resize((size_t)std::max<int64_t>(g.nnz, 1));
    g.h_J.resize((size_t)std::max<int64_t>(g.nnz, 1));
    if (canonical) {
        // Row r holds first the edges (s, r), s < r, in increasing s (= edge order), then the edges
        // (r, d) in increasing d, so it comes out sorted by column.  Edge e = (a, b) lands at
        // row_ptr[a] + in_deg[a] + (e - first edge of a) and at row_ptr[b] + (its rank among the
        // edges into b); the threads write disjoint slots.
        std::vector<int64_t> first((size_t)n + 1, 0);
        for (int32_t i = 0; i < n; ++i) first[(size_t)i + 1] = first[(size_t)i] + out_deg[(size_t)i];
        run([&](int t) {
            int32_t* rank = cnt_dst.data() + (size_t)t * n;
            for (int64_t e = chunk(t); e < chunk(t + 1); ++e) {
                const int8_t J = (int8_t)(-w[e]);
                const int32_t a = src[e], b = dst[e];
                const size_t up = (size_t)(g.h_row_ptr[(size_t)a] + in_deg[(size_t)a] + (e - first[(size_t)a]));
                const size_t lo = (size_t)(g.h_row_ptr[(size_t)b] + rank[b]++);
                g.h_col[up] = b;
                g.h_J[up] = J;
                g.h_col[lo] = a;
                g.h_J[lo] = J;
            }
        });
    } else {
        // any order: two stable counting passes over the 2m directed entries, first bucketed by
        // column (the column pointer equals the row pointer), then, visiting columns in order, by row
        std::vector<int32_t> fill(g.h_row_ptr.begin(), g.h_row_ptr.end() - 1);
        std::vector<int32_t> by_col_row((size_t)std::max<int64_t>(g.nnz, 1));
        std::vector<int8_t> by_col_J((size_t)std::max<int64_t>(g.nnz, 1));
        for (int64_t e = 0; e < n_edges; ++e) {
            const int8_t J = (int8_t)(-w[e]);
            const int32_t a = src[e], b = dst[e];
            by_col_row[(size_t)fill[(size_t)b]] = a;  // entry (a, b) lands in column b
            by_col_J[(size_t)fill[(size_t)b]++] = J;
            by_col_row[(size_t)fill[(size_t)a]] = b;  // entry (b, a) lands in column a
            by_col_J[(size_t)fill[(size_t)a]++] = J;
        }
        std::copy(g.h_row_ptr.begin(), g.h_row_ptr.end() - 1, fill.begin());
        for (int32_t c = 0; c < n; ++c) {
            for (int32_t k = g.h_row_ptr[(size_t)c]; k < g.h_row_ptr[(size_t)c + 1]; ++k) {
                const int32_t r = by_col_row[(size_t)k];
                g.h_col[(size_t)fill[(size_t)r]] = c;
                g.h_J[(size_t)fill[(size_t)r]++] = by_col_J[(size_t)k];
            }
        }
    }
    // per row, in parallel over row ranges: duplicate check, W_i = sum_j |J_ij|, the field bound, and
    // s_i = sqrt((n - 1) Var(J_i,:)) (population variance over the full row of n entries); mean(s_i)
    // is then summed in node order
    struct RowStats {
        int64_t max_field = 0, dup_row = -1;
        int32_t max_degree = 0, max_abs_J = 0, max_wabs = 0;
    };
    std::vector<RowStats> rs((size_t)P);
    std::vector<double> s_row((size_t)n);
    g.h_wabs.assign((size_t)n, 0);
    run([&](int t) {
        RowStats& R = rs[(size_t)t];
        for (int64_t i = (int64_t)n * t / P; i < (int64_t)n * (t + 1) / P; ++i) {
            const int32_t b = g.h_row_ptr[(size_t)i], e = g.h_row_ptr[(size_t)i + 1];
            R.max_degree = std::max(R.max_degree, e - b);
            int64_t absum = 0, s1 = 0, s2 = 0;
            for (int32_t k = b; k < e; ++k) {
                const int32_t J = g.h_J[(size_t)k];
                const int32_t aJ = J < 0 ? -J : J;
                absum += aJ;
                R.max_abs_J = std::max(R.max_abs_J, aJ);
                s1 += J;
                s2 += (int64_t)J * J;
                if (!canonical && k > b && g.h_col[(size_t)k] == g.h_col[(size_t)k - 1] && R.dup_row < 0) R.dup_row = i;
            }
            const int64_t hi = h ? std::llabs((long long)h[i]) : 0;
            R.max_field = std::max(R.max_field, absum + hi);
            const int32_t W = (int32_t)std::min<int64_t>(absum, INT32_MAX);
            g.h_wabs[(size_t)i] = W;
            R.max_wabs = std::max(R.max_wabs, W);
            const double mean = (double)s1 / (double)n;
            double var = (double)s2 / (double)n - mean * mean;
            if (var < 0.0) var = 0.0;
            s_row[(size_t)i] = std::sqrt((double)(n - 1) * var);
        }
    });
    int64_t max_field = 0, dup_row = -1;
    g.max_degree = 0;
    g.max_abs_J = 0;
    g.max_wabs = 0;
    for (const RowStats& R : rs) {
        max_field = std::max(max_field, R.max_field);
        g.max_degree = std::max(g.max_degree, R.max_degree);
        g.max_abs_J = std::max(g.max_abs_J, R.max_abs_J);
        g.max_wabs = std::max(g.max_wabs, R.max_wabs);
        if (R.dup_row >= 0 && (dup_row < 0 || R.dup_row < dup_row)) dup_row = R.dup_row;
    }
    if (dup_row >= 0) {
        const int32_t b = g.h_row_ptr[(size_t)dup_row], e = g.h_row_ptr[(size_t)dup_row + 1];
        int32_t c = -1;
        for (int32_t k = b + 1; k < e && c < 0; ++k)
            if (g.h_col[(size_t)k] == g.h_col[(size_t)k - 1]) c = g.h_col[(size_t)k];
        return fail(PBIT_E_INVALID, "graph: duplicate edge (" + std::to_string(dup_row) + "," + std::to_string(c) + ")");
    }
    g.h_tab_off.assign((size_t)n + 1, 0);
    int64_t acc_off = 0;
    double s_acc = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        g.h_tab_off[(size_t)i] = (int32_t)std::min<int64_t>(acc_off, INT32_MAX);
        acc_off += (int64_t)g.h_wabs[(size_t)i] + 1;
        s_acc += s_row[(size_t)i];
    }
    g.mean_s = s_acc / (double)n;
    if (max_field >= (1 << 24)) return fail(PBIT_E_INVALID, "graph: |field| could reach 2^24");
    g.tab_ok = acc_off < INT32_MAX;
    g.h_tab_off[(size_t)n] = (int32_t)std::min<int64_t>(acc_off, INT32_MAX);
    g.max_abs_field = (int32_t)max_field;
    g.has_h = h != nullptr;
    if (h) g.h_h.assign(h, h + n);
    return PBIT_OK;
}

}  // namespace pbit

using namespace pbit;

extern "C" {

const char* pbit_last_error(void) { return g_last_error.c_str(); }

int32_t pbit_version(void) { return 100; }

int64_t pbit_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

pbit_status pbit_graph_create(int32_t n, int64_t n_edges, const int32_t* src, const int32_t* dst, const int8_t* w,
                              const int32_t* h, uint32_t flags, pbit_graph* out) {
    if (!out) return fail(PBIT_E_INVALID, "graph_create: out is NULL");
    *out = nullptr;
    std::unique_ptr<pbit_graph_s> g(new (std::nothrow) pbit_graph_s());
    if (!g) return fail(PBIT_E_NOMEM, "graph_create: host allocation");
    pbit_status st = build_host(*g, n, n_edges, src, dst, w, h);
    if (st != PBIT_OK) return st;
    PBIT_CUDA_TRY(cudaGetDevice(&g->device));
    if ((st = upload(&g->row_ptr, g->h_row_ptr.data(), (size_t)n + 1, g->device_bytes)) != PBIT_OK) goto err;
    if ((st = upload(&g->col, g->h_col.data(), (size_t)g->nnz, g->device_bytes)) != PBIT_OK) goto err;
    if ((st = upload(&g->J, g->h_J.data(), (size_t)g->nnz, g->device_bytes)) != PBIT_OK) goto err;
    if (h && (st = upload(&g->h, h, (size_t)n, g->device_bytes)) != PBIT_OK) goto err;
    if ((st = upload(&g->wabs, g->h_wabs.data(), (size_t)n, g->device_bytes)) != PBIT_OK) goto err;
    if ((st = upload(&g->tab_off, g->h_tab_off.data(), (size_t)n + 1, g->device_bytes)) != PBIT_OK) goto err;
    if ((st = upload(&g->err, (const int*)nullptr, 1, g->device_bytes)) != PBIT_OK) goto err;
    {
        cudaError_t ce = cudaMemset(g->err, 0, sizeof(int));
        if (ce != cudaSuccess) {
            st = cuda_fail(ce, "cudaMemset(err)");
            goto err;
        }
    }
    if ((flags & PBIT_GRAPH_DENSE) && (st = build_dense_operand(*g)) != PBIT_OK) goto err;
    if ((flags & PBIT_GRAPH_DENSE) && (st = build_dense4_operand(*g)) != PBIT_OK) goto err;
    *out = g.release();
    return PBIT_OK;
err:
    release(g.get());
    return st;
}

pbit_status pbit_mean_s(int32_t n, int64_t n_edges, const int32_t* src, const int32_t* dst, const int8_t* w,
                        double* out) {
    if (!out) return fail(PBIT_E_INVALID, "mean_s: out is NULL");
    Graph g;
    pbit_status st = build_host(g, n, n_edges, src, dst, w, nullptr);
    if (st != PBIT_OK) return st;
    *out = g.mean_s;
    return PBIT_OK;
}

pbit_status pbit_i0_table(double i0_min, double i0_max, int32_t steps, float* table) {
    if (!table) return fail(PBIT_E_INVALID, "i0_table: table is NULL");
    Graph g;
    std::vector<float> tab;
    pbit_status st = build_schedule(g, i0_min, i0_max, 0, steps, tab);
    if (st != PBIT_OK) return st;
    std::memcpy(table, tab.data(), sizeof(float) * tab.size());
    return PBIT_OK;
}

void pbit_graph_destroy(pbit_graph g) {
    if (!g) return;
    release(g);
    delete g;
}

pbit_status pbit_graph_info(pbit_graph g, pbit_graph_info_t* info) {
    if (!g || !info) return fail(PBIT_E_INVALID, "graph_info: NULL argument");
    info->n = g->n;
    info->n_edges = g->n_edges;
    info->max_degree = g->max_degree;
    info->unit_weights = g->unit_weights ? 1 : 0;
    info->has_dense = g->dense.J_e4m3 ? 1 : 0;
    info->has_dense_fp4 = g->dense4.J4 ? 1 : 0;
    info->device = g->device;
    info->mean_s = g->mean_s;
    info->total_weight = g->total_weight;
    info->device_bytes = g->device_bytes;
    return PBIT_OK;
}

pbit_status pbit_schedule(pbit_graph g, double i0_min, double i0_max, int32_t normalize, int32_t steps,
                          float* table) {
    if (!g || !table) return fail(PBIT_E_INVALID, "schedule: NULL argument");
    std::vector<float> tab;
    pbit_status st = build_schedule(*g, i0_min, i0_max, normalize, steps, tab);
    if (st != PBIT_OK) return st;
    std::memcpy(table, tab.data(), sizeof(float) * tab.size());
    return PBIT_OK;
}

void pbit_anneal_params_default(pbit_anneal_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->struct_size = sizeof(pbit_anneal_params);
    p->trials = 1;
    p->steps = 1;
    p->i0_min = 0.1;
    p->i0_max = 10.0;
    p->i0_normalize = 1;
    p->offset_mode = PBIT_OFFSET_SCALED;
    p->kernel = PBIT_KERNEL_AUTO;
    p->algorithm = PBIT_ALG_PSA;
    p->stall_prob = 0.5f;
    p->window = 4;
    p->t_res = 0;
}

size_t pbit_variant_state_bytes(int32_t n, int32_t trials, int32_t algorithm, int32_t window) {
    if (n < 1 || trials < 1) return 0;
    const size_t cells = (size_t)n * (size_t)trials;
    if (algorithm == PBIT_ALG_SPSA) return 4 * cells;
    if (algorithm == PBIT_ALG_TAPSA) return 2 * (size_t)(window < 1 ? 1 : window) * cells;
    return 0;
}

pbit_status pbit_select_kernel(pbit_graph g, int32_t requested, int32_t trials, int32_t* kernel) {
    if (!g || !kernel || trials < 1 || requested < 0 || requested > 3)
        return fail(PBIT_E_INVALID, "select_kernel: bad argument");
    int k = 0;
    pbit_status st = select_kernel(*g, requested, trials, &k);
    if (st != PBIT_OK) return st;
    *kernel = k;
    return PBIT_OK;
}

pbit_status pbit_init_spins(pbit_graph g, int32_t trials, uint64_t seed, uint32_t instance, int8_t* spins,
                            void* stream) {
    if (!g || !spins || trials < 1) return fail(PBIT_E_INVALID, "init_spins: bad argument");
    pbit_status st = check_device(g);
    if (st != PBIT_OK) return st;
    PBIT_CUDA_TRY(launch_init_spins(g->n, trials, seed, instance, spins, (cudaStream_t)stream));
    return PBIT_OK;
}

pbit_status pbit_anneal(pbit_graph g, const pbit_anneal_params* p, const int8_t* spins_in, int8_t* spins_out) {
    if (!g || !p || !spins_out) return fail(PBIT_E_INVALID, "anneal: NULL argument");
    if (p->struct_size != sizeof(pbit_anneal_params)) return fail(PBIT_E_INVALID, "anneal: struct_size mismatch");
    const int32_t T = p->trials, S = p->steps;
    if (p->t_res < 0 || p->t_res > 1000000) return fail(PBIT_E_INVALID, "anneal: bad t_res");
    const int64_t sub = (int64_t)S * (p->t_res > 0 ? p->t_res : 1);  // schedule length in (sub-)steps
    if (sub > INT32_MAX) return fail(PBIT_E_INVALID, "anneal: steps * t_res too large");
    const int32_t b = p->step_begin, e = p->step_end == 0 ? (int32_t)sub : p->step_end;
    if (T < 1 || S < 1 || b < 0 || e < b || e > sub) return fail(PBIT_E_INVALID, "anneal: bad trials/steps range");
    if ((int64_t)g->n * T > ((int64_t)1 << 40)) return fail(PBIT_E_INVALID, "anneal: n*T too large");
    if (p->offset_mode < 0 || p->offset_mode > 2) return fail(PBIT_E_INVALID, "anneal: bad offset_mode");
    if (p->kernel < 0 || p->kernel > 3) return fail(PBIT_E_INVALID, "anneal: bad kernel");
    if (p->algorithm < 0 || p->algorithm > 2) return fail(PBIT_E_INVALID, "anneal: bad algorithm");
    if (p->algorithm == PBIT_ALG_SPSA && !(p->stall_prob >= 0.0f && p->stall_prob <= 1.0f))
        return fail(PBIT_E_INVALID, "anneal: stall_prob outside [0,1]");
    if (p->algorithm == PBIT_ALG_TAPSA && (p->window < 1 || p->window > 64))
        return fail(PBIT_E_INVALID, "anneal: window outside 1..64");
    const bool is_var = p->algorithm != PBIT_ALG_PSA || p->t_res > 0;
    if (p->algorithm == PBIT_ALG_TAPSA && g->max_abs_field > 32767)
        return fail(PBIT_E_UNSUPPORTED, "anneal: TApSA keeps fields as int16; |h_i| + sum_j |J_ij| exceeds 32767");
    if (p->algorithm != PBIT_ALG_PSA && !p->state && b != 0)
        return fail(PBIT_E_INVALID, "anneal: resuming SpSA/TApSA needs the state buffer of the earlier run");
    pbit_status st = check_device(g);
    if (st != PBIT_OK) return st;
    cudaStream_t s = (cudaStream_t)p->stream;
    const int64_t cells = (int64_t)g->n * T;

    int kernel = 0;
    if ((st = select_kernel(*g, p->kernel, T, &kernel, is_var)) != PBIT_OK) return st;

    // host-side tables
    std::vector<float> tab;
    if ((st = build_schedule(*g, p->i0_min, p->i0_max, p->i0_normalize, S, tab)) != PBIT_OK) return st;
    std::vector<uint32_t> thr;
    if (p->p_update) {
        thr.resize((size_t)g->n);
        for (int32_t i = 0; i < g->n; ++i) {
            const float pu = p->p_update[i];
            if (!(pu >= 0.0f && pu <= 1.0f)) return fail(PBIT_E_INVALID, "anneal: p_update outside [0,1]");
            thr[(size_t)i] = (uint32_t)std::ceil((double)pu * 16777216.0);  // u < p  <=>  (u*2^24) < ceil(p*2^24)
        }
    }
    if (p->intensity)
        for (int32_t i = 0; i < g->n; ++i)
            if (!std::isfinite(p->intensity[i])) return fail(PBIT_E_INVALID, "anneal: non-finite intensity");
    if (p->offset)
        for (int32_t i = 0; i < g->n; ++i)
            if (!std::isfinite(p->offset[i])) return fail(PBIT_E_INVALID, "anneal: non-finite offset");

    CallBuffers cb;
    cb.s = s;
    StepArgs a{};
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
    if ((st = cb.put(&d_tab, tab.data(), tab.size())) != PBIT_OK) return st;
    a.i0_table = d_tab;
    if (p->intensity) {
        float* d = nullptr;
        if ((st = cb.put(&d, p->intensity, (size_t)g->n)) != PBIT_OK) return st;
        a.par.lambda = d;
    }
    if (p->offset) {
        float* d = nullptr;
        if ((st = cb.put(&d, p->offset, (size_t)g->n)) != PBIT_OK) return st;
        a.par.delta = d;
    }
    if (p->p_update) {
        uint32_t* d = nullptr;
        if ((st = cb.put(&d, thr.data(), thr.size())) != PBIT_OK) return st;
        a.par.thr = d;
    }
    // variant state and timing periods
    PeriodBuckets buckets;
    a.alg = p->algorithm;
    a.window = p->window < 1 ? 1 : p->window;
    a.t_res = p->t_res;
    a.stall_thr = (uint32_t)std::ceil((double)p->stall_prob * 16777216.0);
    if (p->t_res > 0) {
        std::vector<int32_t> nu((size_t)g->n);
        for (int32_t i = 0; i < g->n; ++i) {
            const double v = std::round((double)p->t_res * (1.0 + (p->nu_dev ? (double)p->nu_dev[i] : 0.0)));
            nu[(size_t)i] = v < 1.0 ? 1 : (int32_t)std::min(v, 1e9);
        }
        int32_t* d = nullptr;
        if ((st = cb.put(&d, nu.data(), nu.size())) != PBIT_OK) return st;
        a.nu = d;
        build_period_buckets(nu, buckets);
        int32_t* dp = nullptr;
        if ((st = cb.put(&dp, buckets.host_perm.data(), buckets.host_perm.size())) != PBIT_OK) return st;
        buckets.perm = dp;
        if (!buckets.host_bkt.empty() && T % 128 == 0) {  // the parity form needs the word tile
            uint8_t* db = nullptr;
            if ((st = cb.put(&db, buckets.host_bkt.data(), buckets.host_bkt.size())) != PBIT_OK) return st;
            buckets.bkt = db;
            if ((st = cb.alloc(&buckets.ebkt, (size_t)g->nnz)) != PBIT_OK) return st;
            PBIT_CUDA_TRY(launch_edge_buckets(*g, buckets.bkt, buckets.ebkt, s));
        }
    }
    if (a.alg != PBIT_ALG_PSA) {
        const size_t sb = pbit_variant_state_bytes(g->n, T, a.alg, a.window);
        uint8_t* stt = (uint8_t*)p->state;
        if (!stt) {
            if ((st = cb.alloc(&stt, sb)) != PBIT_OK) return st;
            PBIT_CUDA_TRY(cudaMemsetAsync(stt, 0, sb, s));
        }
        if (a.alg == PBIT_ALG_SPSA) a.Iprev = (float*)stt;
        else a.ring = (int16_t*)stt;
    }
    // the start state
    const int8_t* cur = spins_in;
    int8_t* init_buf = nullptr;
    if (!cur) {
        if (e == b) {
            init_buf = spins_out;
        } else if ((st = cb.alloc(&init_buf, (size_t)cells)) != PBIT_OK) {
            return st;
        }
        PBIT_CUDA_TRY(launch_init_spins(g->n, T, p->seed, p->instance, init_buf, s));
        cur = init_buf;
    }
    if (e == b) {
        if (cur != spins_out)
            PBIT_CUDA_TRY(cudaMemcpyAsync(spins_out, cur, (size_t)cells, cudaMemcpyDeviceToDevice, s));
        return PBIT_OK;
    }
    if (kernel == PBIT_KERNEL_RESIDENT) {
        a.in = cur;
        a.out = spins_out;
        PBIT_CUDA_TRY(launch_resident_anneal(a, b, e, g->unit_weights && g->max_degree <= 127, s));
        return PBIT_OK;
    }
    if (kernel == PBIT_KERNEL_DENSE && dense4_shape_ok(*g, T)) {
        // cluster-resident FP4 kernel: the whole step range in one launch, int8 in and out
        uint8_t* b0 = nullptr;
        if ((st = cb.alloc(&b0, dense4_spin_bytes(*g, T))) != PBIT_OK) return st;
        const cudaError_t de = launch_dense4(*g, a, cur, spins_out, nullptr, b0, b, e, s);
        if (de == cudaSuccess) return PBIT_OK;
        if (de != cudaErrorNotSupported) return cuda_fail(de, "dense fp4 cluster launch");
    }
    if (kernel == PBIT_KERNEL_DENSE) {
        std::string why;
        if (!dense_shape_ok(*g, T, &why)) return fail(PBIT_E_UNSUPPORTED, "anneal: " + why);
        // tiled e4m3 spin buffers; convert in, step, convert out
        uint8_t* t0 = nullptr;
        uint8_t* t1 = nullptr;
        const size_t tb = dense_spin_bytes(*g, T);
        if ((st = cb.alloc(&t0, tb)) != PBIT_OK) return st;
        if ((st = cb.alloc(&t1, tb)) != PBIT_OK) return st;
        PBIT_CUDA_TRY(launch_to_tiled(*g, cur, T, t0, s));
        // persistent form when every cluster can be resident, else one launch per step
        unsigned* done = nullptr;
        const int RB = g->dense.n_pad / 128, TB = T <= 128 ? 1 : T / 128, KS = g->dense.n_pad / 512;
        const size_t nflags = (size_t)RB * TB * KS;
        if ((st = cb.alloc(&done, nflags)) != PBIT_OK) return st;
        PBIT_CUDA_TRY(cudaMemsetAsync(done, 0, sizeof(unsigned) * nflags, s));
        static const bool stepwise = std::getenv("PBIT_DENSE_STEPWISE") != nullptr;  // force per-step launches
        cudaError_t pe = stepwise ? cudaErrorNotSupported
                                  : launch_dense_persistent(*g, a, t0, t1, b, e, done, g->err, s);
        if (pe == cudaSuccess) {
            if ((e - b) % 2 == 1) std::swap(t0, t1);
        } else if (pe == cudaErrorNotSupported) {
            for (int32_t j = b; j < e; ++j) {
                a.step = j;
                PBIT_CUDA_TRY(launch_dense_step(*g, a, t0, t1, nullptr, g->err, s));
                std::swap(t0, t1);
            }
        } else {
            return cuda_fail(pe, "dense persistent launch");
        }
        PBIT_CUDA_TRY(launch_from_tiled(*g, t0, T, spins_out, s));
        return PBIT_OK;
    }
    const SparseVariant variant = choose_sparse_variant(*g, T);
    static const bool timing_copy = std::getenv("PBIT_TIMING_COPY") != nullptr;  // force the copy form (tests)
    if (a.t_res > 0 && buckets.ebkt && !timing_copy) {
        // timing model, parity form: each node's spins alternate between spins_out and a scratch buffer
        int8_t* other = nullptr;
        if ((st = cb.alloc(&other, (size_t)cells)) != PBIT_OK) return st;
        const cudaError_t te = launch_timing_slots(*g, a, b, e, cur, spins_out, other, buckets, variant, s);
        if (te == cudaSuccess) return PBIT_OK;
        if (te != cudaErrorNotSupported) return cuda_fail(te, "timing model");
    }
    // Jacobi rotation: step j writes spins_out when (k-1-j) is even, else scratch
    int8_t* scratch = nullptr;
    const int32_t k = e - b;
    if (k >= 2 || cur == spins_out) {
        if ((st = cb.alloc(&scratch, (size_t)cells)) != PBIT_OK) return st;
    }
    if (cur == spins_out && ((k - 1) % 2 == 0)) {
        // in place with an odd count: the first write would hit the input
        PBIT_CUDA_TRY(cudaMemcpyAsync(scratch, cur, (size_t)cells, cudaMemcpyDeviceToDevice, s));
        cur = scratch;
    }
    // plain pSA over two or more steps: one persistent launch with per-tile step dependencies
    static const bool stepwise = std::getenv("PBIT_SPARSE_STEPWISE") != nullptr;  // force one launch per step
    // PBIT_SPARSE_FLOW=always takes the multi-step form whatever the dependency structure (tests)
    static const char* flow_env = std::getenv("PBIT_SPARSE_FLOW");
    static const bool flow_forced = flow_env && std::string(flow_env) == "always";
    if (!stepwise && k >= 2 && !is_variant(a)) {
        int8_t* P = ((k - 1) % 2 == 0) ? spins_out : scratch;  // written at even j
        int8_t* Q = P == spins_out ? scratch : spins_out;
        bool use_flow;
        {
            std::lock_guard<std::mutex> lock(g->mu);
            if ((st = ensure_flow_deps(*g, T, cur, P, Q, variant)) != PBIT_OK) return st;
            use_flow = flow_forced || g->flow.local();
        }
        if (use_flow) {
            unsigned* tile_done = nullptr;
            unsigned* step_done = nullptr;
            unsigned long long* next = nullptr;
            if ((st = cb.alloc(&tile_done, (size_t)g->flow.ntiles)) != PBIT_OK) return st;
            if ((st = cb.alloc(&step_done, (size_t)k)) != PBIT_OK) return st;
            if ((st = cb.alloc(&next, 1)) != PBIT_OK) return st;
            PBIT_CUDA_TRY(cudaMemsetAsync(tile_done, 0, sizeof(unsigned) * g->flow.ntiles, s));
            PBIT_CUDA_TRY(cudaMemsetAsync(step_done, 0, sizeof(unsigned) * (size_t)k, s));
            PBIT_CUDA_TRY(cudaMemsetAsync(next, 0, sizeof(unsigned long long), s));
            a.step = b;
            const cudaError_t fe = launch_sparse_flow(*g, a, k, cur, P, Q, tile_done, step_done, next, variant, s);
            if (fe == cudaSuccess) return PBIT_OK;
            if (fe != cudaErrorNotSupported) return cuda_fail(fe, "sparse multi-step launch");
        }
    }
    for (int32_t j = 0; j < k; ++j) {
        int8_t* dst = ((k - 1 - j) % 2 == 0) ? spins_out : scratch;
        a.step = b + j;
        a.in = cur;
        a.out = dst;
        if (is_variant(a)) {
            a.carry = j >= 2 ? 1 : 0;  // dst holds the state of sub-step b + j - 2 from the second write on
            PBIT_CUDA_TRY(launch_variant_step(a, &buckets, s, variant));
        } else {
            PBIT_CUDA_TRY(launch_sparse_step(a, s, variant));
        }
        cur = dst;
    }
    return PBIT_OK;
}

pbit_status pbit_anneal_trace(pbit_graph g, const pbit_anneal_params* p, const int8_t* spins_in, int8_t* spins_out,
                              int32_t every, int32_t what, int64_t* trace) {
    if (!g || !p || !spins_out || !trace || every < 1 || what < 0 || what > 1)
        return fail(PBIT_E_INVALID, "anneal_trace: bad argument");
    if (p->struct_size != sizeof(pbit_anneal_params)) return fail(PBIT_E_INVALID, "anneal_trace: struct_size");
    const int64_t sub = (int64_t)p->steps * (p->t_res > 0 ? p->t_res : 1);
    const int32_t b = p->step_begin, e = p->step_end == 0 ? (int32_t)sub : p->step_end;
    if (b < 0 || e < b || e > sub) return fail(PBIT_E_INVALID, "anneal_trace: bad step range");
    cudaStream_t s = (cudaStream_t)p->stream;
    pbit_anneal_params q = *p;
    CallBuffers cb;
    cb.s = s;
    pbit_status st;
    if (q.algorithm != PBIT_ALG_PSA && !q.state) {  // one state carried across the segments
        if (b != 0) return fail(PBIT_E_INVALID, "anneal_trace: resuming needs the state buffer");
        const size_t sb = pbit_variant_state_bytes(g->n, q.trials, q.algorithm, q.window);
        uint8_t* stt = nullptr;
        if ((st = cb.alloc(&stt, sb)) != PBIT_OK) return st;
        PBIT_CUDA_TRY(cudaMemsetAsync(stt, 0, sb, s));
        q.state = stt;
    }
    const int8_t* in = spins_in;
    int32_t j = 0;
    for (int32_t from = b; from < e; from += every, ++j) {
        q.step_begin = from;
        q.step_end = std::min(e, from + every);
        if ((st = pbit_anneal(g, &q, in, spins_out)) != PBIT_OK) return st;
        in = spins_out;
        int64_t* row = trace + (size_t)j * (size_t)q.trials;
        st = what == 0 ? pbit_energy(g, spins_out, q.trials, row, 0, p->stream)
                       : pbit_cut(g, spins_out, q.trials, row, 0, p->stream);
        if (st != PBIT_OK) return st;
    }
    return PBIT_OK;
}

pbit_status pbit_fields(pbit_graph g, const int8_t* spins, int32_t trials, int32_t* fields, void* stream) {
    if (!g || !spins || !fields || trials < 1) return fail(PBIT_E_INVALID, "fields: bad argument");
    pbit_status st = check_device(g);
    if (st != PBIT_OK) return st;
    PBIT_CUDA_TRY(launch_fields(*g, spins, trials, fields, (cudaStream_t)stream));
    return PBIT_OK;
}

pbit_status pbit_fields_dense(pbit_graph g, const int8_t* spins, int32_t trials, int32_t* fields, void* stream) {
    if (!g || !spins || !fields || trials < 1) return fail(PBIT_E_INVALID, "fields_dense: bad argument");
    pbit_status st = check_device(g);
    if (st != PBIT_OK) return st;
    std::string why;
    if (!any_dense_ok(*g, trials, &why)) return fail(PBIT_E_UNSUPPORTED, "fields_dense: " + why);
    cudaStream_t s = (cudaStream_t)stream;
    CallBuffers cb;
    cb.s = s;
    if (dense4_shape_ok(*g, trials)) {
        uint8_t* b0 = nullptr;
        if ((st = cb.alloc(&b0, dense4_spin_bytes(*g, trials))) != PBIT_OK) return st;
        StepArgs a{};
        a.T = trials;
        const cudaError_t de = launch_dense4(*g, a, spins, nullptr, fields, b0, 0, 0, s);
        if (de == cudaSuccess) return PBIT_OK;
        if (de != cudaErrorNotSupported) return cuda_fail(de, "fields_dense fp4");
    }
    if (!g->dense.J_e4m3) return fail(PBIT_E_UNSUPPORTED, "fields_dense: no e4m3 operand");
    uint8_t* t0 = nullptr;
    if ((st = cb.alloc(&t0, dense_spin_bytes(*g, trials))) != PBIT_OK) return st;
    PBIT_CUDA_TRY(launch_to_tiled(*g, spins, trials, t0, s));
    StepArgs a{};
    a.T = trials;
    PBIT_CUDA_TRY(launch_dense_step(*g, a, t0, nullptr, fields, g->err, s));
    return PBIT_OK;
}

pbit_status pbit_selftest_timeout(pbit_graph g, int32_t budget_us, void* stream) {
    if (!g || budget_us < 1 || budget_us > 2000000) return fail(PBIT_E_INVALID, "selftest_timeout: budget 1..2e6 us");
    pbit_status st = check_device(g);
    if (st != PBIT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned* flag = nullptr;
    PBIT_CUDA_TRY(cudaMallocAsync((void**)&flag, sizeof(unsigned), s));
    PBIT_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(unsigned), s));
    cudaError_t e = launch_bounded_wait_selftest(flag, (long long)budget_us * 1000, g->err, s);
    cudaFreeAsync(flag, s);
    if (e != cudaSuccess) return cuda_fail(e, "selftest_timeout");
    return PBIT_OK;
}

pbit_status pbit_graph_status(pbit_graph g, void* stream) {
    if (!g) return fail(PBIT_E_INVALID, "graph_status: NULL graph");
    pbit_status st = check_device(g);
    if (st != PBIT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    int host = 0;
    PBIT_CUDA_TRY(cudaMemcpyAsync(&host, g->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    PBIT_CUDA_TRY(cudaStreamSynchronize(s));
    if (host != 0) {
        PBIT_CUDA_TRY(cudaMemsetAsync(g->err, 0, sizeof(int), s));
        PBIT_CUDA_TRY(cudaStreamSynchronize(s));
        return fail(PBIT_E_TIMEOUT, "a bounded device-side wait gave up (code " + std::to_string(host) + ")");
    }
    return PBIT_OK;
}

static pbit_status cut_or_energy(pbit_graph g, const int8_t* spins, int32_t trials, int64_t* out, int32_t on_host,
                                 void* stream, bool energy) {
    if (!g || !spins || !out || trials < 1) return fail(PBIT_E_INVALID, "cut/energy: bad argument");
    pbit_status st = check_device(g);
    if (st != PBIT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // tensor-core route when the graph holds the dense operand (and h = 0 for the energy)
    const bool dense = dense_shape_ok(*g, trials, nullptr) && !(energy && g->has_h);
    uint8_t* tiled = nullptr;
    if (dense) PBIT_CUDA_TRY(cudaMallocAsync((void**)&tiled, dense_spin_bytes(*g, trials), s));
    auto run = [&](int64_t* dst) -> cudaError_t {
        return dense ? launch_dense_cut_energy(*g, spins, trials, dst, energy, tiled, s)
                     : launch_cut_energy(*g, spins, trials, dst, energy, s);
    };
    if (!on_host) {
        cudaError_t e1 = run(out);
        if (tiled) cudaFreeAsync(tiled, s);
        if (e1 != cudaSuccess) return cuda_fail(e1, energy ? "energy" : "cut");
        return PBIT_OK;
    }
    int64_t* d = nullptr;
    PBIT_CUDA_TRY(cudaMallocAsync((void**)&d, sizeof(int64_t) * (size_t)trials, s));
    cudaError_t err = run(d);
    if (tiled) cudaFreeAsync(tiled, s);
    if (err == cudaSuccess) err = cudaMemcpyAsync(out, d, sizeof(int64_t) * (size_t)trials, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) return cuda_fail(err, energy ? "energy" : "cut");
    return PBIT_OK;
}

pbit_status pbit_cut(pbit_graph g, const int8_t* spins, int32_t trials, int64_t* out, int32_t out_on_host,
                     void* stream) {
    return cut_or_energy(g, spins, trials, out, out_on_host, stream, false);
}

pbit_status pbit_energy(pbit_graph g, const int8_t* spins, int32_t trials, int64_t* out, int32_t out_on_host,
                        void* stream) {
    return cut_or_energy(g, spins, trials, out, out_on_host, stream, true);
}

}  // extern "C"
