// Internal declarations shared by the translation units of libpbit.so.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "pbit.h"

namespace pbit {

// Process-wide count of kernels this library has launched (for benchmarks).
void count_launches(int64_t k);

// ---------------------------------------------------------------- errors ----
void set_error(const std::string& msg);
pbit_status fail(pbit_status code, const std::string& msg);
pbit_status cuda_fail(cudaError_t err, const char* what);

#define PBIT_CUDA_TRY(expr)                                 \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) return ::pbit::cuda_fail(_e, #expr); \
    } while (0)

// ------------------------------------------------------------- the graph ----
// Device-resident instance: CSR of J = -w (rows sorted by column), biases,
// and optionally the dense tensor-core operand.
struct DenseOperand {
    int32_t n_pad = 0;         // n rounded up to the tile size
    uint8_t* J_e4m3 = nullptr; // device, tile-ordered e4m3 bytes of J (see pbit_dense.cu)
    size_t bytes = 0;
};

// The same J as packed e2m1 (FP4) for the cluster-resident dense kernel (pbit_dense4.cu): built
// when n <= 2048 and every |J_ij| is 0, 1, 2, 3, 4 or 6 (exact in e2m1).
struct Dense4Operand {
    int32_t C = 0;             // row blocks of 128 = CTAs per cluster; K = 128 C
    uint8_t* J4 = nullptr;     // device, C blocks of 64 K bytes
    size_t bytes = 0;
};

// Tile dependencies of the multi-step sparse kernel for one item count per
// node (groups = T / G): tile t may run step j once every tile in
// idx[ptr[t] .. ptr[t+1]) has finished step j - 1; an empty list means "wait
// for the whole previous step".
struct FlowDeps {
    int32_t groups = 0;
    int32_t ntiles = 0;
    int32_t* ptr = nullptr;  // device [ntiles + 1]
    int32_t* idx = nullptr;  // device
    int64_t listed = 0;      // tiles with their own list (the rest wait for the whole step)
    int64_t entries = 0;     // total length of those lists
    // Worth one persistent launch only when the dependencies are local: nearly every tile has a short
    // list and there are enough tiles for steps to overlap.  Measured on GB300 (µs per step, multi-step
    // vs one launch per step): 100x200 torus T=1024 34.9 vs 36.2; random graphs (G(n, 3n), 3-NN points
    // numbered at random) 1.1-2x slower, their tiles all waiting on one step counter.
    bool local() const { return ntiles >= 64 && listed * 10 >= (int64_t)ntiles * 9 && entries <= 16 * listed; }
};

struct Graph {
    int32_t n = 0;
    int64_t n_edges = 0;
    int64_t nnz = 0;              // 2 * n_edges
    int32_t max_degree = 0;
    bool unit_weights = true;
    bool has_h = false;
    int device = 0;
    double mean_s = 0.0;
    int64_t total_weight = 0;
    int32_t max_abs_field = 0;    // max_i |h_i| + sum_j |J_ij|
    int32_t max_abs_J = 0;        // max |J_ij|
    // device arrays
    int32_t* row_ptr = nullptr;   // [n+1]
    int32_t* col = nullptr;       // [nnz]
    int8_t* J = nullptr;          // [nnz]
    int32_t* h = nullptr;         // [n] or null
    int32_t* wabs = nullptr;      // [n] W_i = sum_j |J_ij|: the field of node i lies in h_i + [-W_i, W_i]
    int32_t* tab_off = nullptr;   // [n+1] prefix sums of (W_i + 1): threshold-table offsets
    int32_t max_wabs = 0;
    bool tab_ok = false;          // prefix sums fit int32
    DenseOperand dense;
    Dense4Operand dense4;
    FlowDeps flow;                // built on first use, for the last groups value asked for
    int* err = nullptr;           // device word: nonzero after a bounded wait gave up
    size_t device_bytes = 0;
    // host copies used by the schedule and the dense builder
    std::vector<int32_t> h_row_ptr, h_col;
    std::vector<int8_t> h_J;
    std::vector<int32_t> h_h;
    std::vector<int32_t> h_wabs, h_tab_off;
    std::mutex mu;
};

// Host-side schedule: the float32 I0 table (Methods section).
pbit_status build_schedule(const Graph& g, double i0_min, double i0_max, int normalize, int steps,
                           std::vector<float>& out);

// Per-node parameters in the form the kernels read.
struct NodeParams {
    const float* lambda = nullptr;   // device [n] or null (1)
    const float* delta = nullptr;    // device [n] or null (0)
    const uint32_t* thr = nullptr;   // device [n] update threshold ceil(p*2^24), or null (always)
};

// Everything one synchronous step needs.
struct StepArgs {
    const int32_t* row_ptr;
    const int32_t* col;
    const int8_t* J;
    const int32_t* h;
    const int32_t* wabs;
    const int32_t* tab_off;
    NodeParams par;
    const float* i0_table;
    int32_t step;
    const int8_t* in;
    int8_t* out;
    int32_t n;
    int32_t T;
    uint32_t seed_lo, seed_hi, instance;
    int32_t offset_mode;
    // pSA variants and the period timing model (zero: plain pSA)
    int32_t alg;              // 0 pSA, 1 SpSA, 2 TApSA
    uint32_t stall_thr;       // SpSA: stall iff (s-word >> 8) < stall_thr = ceil(p * 2^24)
    int32_t window;           // TApSA window alpha
    int32_t t_res;            // sub-steps per cycle (0: every node every step, I0 = table[step])
    const int32_t* nu;        // [n] update period in sub-steps (timing model)
    float* Iprev;             // SpSA state [n][T]: the last input
    int16_t* ring;            // TApSA state [window][n][T]: the last fields
    int32_t carry;            // timing model: out holds the state of sub-step step - 2 (see pbit_variant.cu)
    const int32_t* perm;      // timing model: nodes grouped by period (set per launch by the word tile)
    // item -> node for the warp-table tile: node = (item * grp_m) >> grp_s = item / (T / G),
    // exact for item < 2^31 (filled by set_group_divisor for the G the launcher picks)
    uint64_t grp_m;
    int32_t grp_s;
};

// Fill grp_m / grp_s for division by d = T / G (Granlund-Montgomery: m = floor(2^(32+l) / d) + 1
// with l = ceil(log2 d); the quotient is exact for every 32-bit dividend below 2^31).
void set_group_divisor(StepArgs& a, int32_t G);

// Test-only fault switch, off by default and read on every launch: PBIT_TEST_WITHHOLD names one
// persistent kernel ("flow", "batch", "dense" or "dense4") that then never publishes one of its
// progress signals (a software flag, counter or slice copy that peers poll), and PBIT_TEST_WAIT_US
// shortens that kernel's bounded waits to about the given microseconds, so a test can make a real
// wait run out quickly and check PBIT_E_TIMEOUT without faulting the GPU.
struct TestFault {
    int withhold = 0;          // 1: this kernel withholds its designated signal
    long long wait_cycles = 0; // clock64 budget of every bounded wait
};
TestFault test_fault(const char* kernel, long long default_cycles);

// kernels (pbit_sparse.cu)
cudaError_t launch_init_spins(int32_t n, int32_t T, uint64_t seed, uint32_t instance, int8_t* spins,
                              cudaStream_t s);
// Sparse step with the kernel variant chosen for the graph: packed counting
// for +-1 weights (degree <= 127) and a per-block shared-memory table of
// decision thresholds when the node fields take few values.
struct SparseVariant {
    bool unit = false;
    bool table = false;
    int warp_g = 0;      // trials per thread of the warp-table tile (0: not used); see pbit_tile.cuh
    bool warp_half = false;  // the warp-table tile indexes its lanes by count / 2 (HALF)
};
SparseVariant choose_sparse_variant(const Graph& g, int32_t T);
// Trials per thread of the warp-table tile (32, 16, or 0: not applicable); `wide` for many
// instances sharing the GPU (prefers 32 whenever it applies).
int warp_tile_group(const Graph& g, int32_t T, bool wide);
cudaError_t launch_sparse_step(const StepArgs& a, cudaStream_t s, SparseVariant v = SparseVariant());
// Steps [a.step, a.step + k) of plain pSA in one persistent launch: step j reads in0 (j = 0), P (odd j)
// or Q (even j >= 2) and writes P (even j) or Q (odd j).  Scratch: tile_done [ntiles], step_done [k]
// and next (zero on entry).  Returns cudaErrorNotSupported when the tile form has no multi-step kernel.
// The dependency lists are built on the host (and cached in g) under g.mu, held by the caller.
pbit_status ensure_flow_deps(Graph& g, int32_t T, const int8_t* in0, const int8_t* P, const int8_t* Q,
                             SparseVariant v);
cudaError_t launch_sparse_flow(const Graph& g, StepArgs a, int32_t k, const int8_t* in0, int8_t* P, int8_t* Q,
                               unsigned* tile_done, unsigned* step_done, unsigned long long* next,
                               SparseVariant v, cudaStream_t s);
__host__ __device__ inline bool is_variant(const StepArgs& a) { return a.alg != 0 || a.t_res > 0; }
// The variants' coalesced word tile (pbit_variant.cu).  PeriodBuckets groups the nodes by update
// period so that a sub-step with `carry` launches warps only for the nodes due at q or q - 1.
struct PeriodBuckets {
    const int32_t* perm = nullptr;             // device [n]: node ids sorted by period
    const uint8_t* bkt = nullptr;              // device [n]: bucket of each node (at most 32 buckets)
    uint8_t* ebkt = nullptr;                   // device [nnz]: bucket of each edge's column
    std::vector<int32_t> host_perm;
    std::vector<uint8_t> host_bkt;             // empty when there are more than 32 periods
    std::vector<int32_t> period, start, len;   // per distinct period (ascending): its run [start, start + len) of perm
};
void build_period_buckets(const std::vector<int32_t>& nu, PeriodBuckets& pb);
cudaError_t launch_edge_buckets(const Graph& g, const uint8_t* bkt, uint8_t* ebkt, cudaStream_t s);
cudaError_t launch_variant_step(const StepArgs& a, const PeriodBuckets* pb, cudaStream_t s, SparseVariant v);
// Sub-steps [b, e) of the timing model in the parity form (pbit_variant.cu): the result lands in X; Y is
// scratch of n*T bytes; cur may be X.  cudaErrorNotSupported when the form does not apply.
cudaError_t launch_timing_slots(const Graph& g, const StepArgs& a, int32_t b, int32_t e, const int8_t* cur, int8_t* X,
                                int8_t* Y, const PeriodBuckets& pb, SparseVariant v, cudaStream_t s);
cudaError_t launch_fields(const Graph& g, const int8_t* spins, int32_t T, int32_t* fields, cudaStream_t s);
cudaError_t launch_cut_energy(const Graph& g, const int8_t* spins, int32_t T, int64_t* out, bool energy,
                              cudaStream_t s);
// dense tensor-core path (pbit_dense.cu)
bool dense_shape_ok(const Graph& g, int32_t T, std::string* why);
pbit_status build_dense_operand(Graph& g);
size_t dense_spin_bytes(const Graph& g, int32_t T);
cudaError_t launch_to_tiled(const Graph& g, const int8_t* s, int32_t T, uint8_t* out, cudaStream_t st);
cudaError_t launch_from_tiled(const Graph& g, const uint8_t* in, int32_t T, int8_t* s, cudaStream_t st);
cudaError_t launch_dense_step(const Graph& g, const StepArgs& sa, const uint8_t* tin, uint8_t* tout,
                              int32_t* fields_out, int* err, cudaStream_t st,
                              unsigned long long* obs_out = nullptr);
// exact cut (energy when h = 0) through the tensor-core fields; needs n_pad*T bytes of scratch
cudaError_t launch_dense_cut_energy(const Graph& g, const int8_t* spins, int32_t T, int64_t* out, bool energy,
                                    uint8_t* tiled_scratch, cudaStream_t st);
cudaError_t launch_dense_persistent(const Graph& g, const StepArgs& sa, uint8_t* buf0, uint8_t* buf1, int32_t b,
                                    int32_t e, unsigned* done, int* err, cudaStream_t st);
// cluster-resident FP4 dense path (pbit_dense4.cu)
pbit_status build_dense4_operand(Graph& g);
bool dense4_shape_ok(const Graph& g, int32_t T);
size_t dense4_spin_bytes(const Graph& g, int32_t T);
// Steps [b, e) from s_in to s_out in one launch (in place allowed), or, with fields_out, the fields of
// s_in only.  b0_scratch: dense4_spin_bytes(g, T) bytes.  cudaErrorNotSupported: not launched.
cudaError_t launch_dense4(const Graph& g, const StepArgs& sa, const int8_t* s_in, int8_t* s_out, int32_t* fields_out,
                          uint8_t* b0_scratch, int32_t b, int32_t e, cudaStream_t st);
int dense4_max_active_clusters(const Graph& g, int32_t T);
cudaError_t launch_bounded_wait_selftest(const unsigned* flag, long long budget_ns, int* err, cudaStream_t s);
// resident single-CTA anneal: all steps in one launch, spins in shared memory
bool resident_fits(const Graph& g, int32_t T);
// AUTO picks the resident kernel (a cluster of 8 CTAs) only for small steps: the cluster gathers about
// 1.1e11 neighbour-updates per second and a multi-SM sparse step costs at least about 12 µs (measured
// on GB300: G(800, 19176), T = 16 runs 5.8 µs per step resident on the cluster, 32 µs on one CTA,
// 12.4 µs sparse), so the break-even is about 1.3e6 gathers per step.
bool resident_preferred(const Graph& g, int32_t T);
cudaError_t launch_resident_anneal(const StepArgs& base, int32_t step_begin, int32_t step_end, bool unit,
                                   cudaStream_t s);

}  // namespace pbit

// The opaque C handle is the internal Graph.
struct pbit_graph_s : public pbit::Graph {};
