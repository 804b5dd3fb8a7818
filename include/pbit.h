/*
 * pbit.h - C ABI of the GB300 p-bit simulated-annealing library (libpbit.so).
 *
 * The library solves MAX-CUT instances by p-bit simulated annealing (pSA)
 * with the device-variability p-bit of arXiv 2601.14476:
 *
 *   Eq. (3) "eqn:conv":  D_i = h_i + sum_j J_ij sigma_j        (exact integer field)
 *   Eq. (6) "eqn:pbits_variability", in the form
 *            sigma_i <- +1 if tanh(I0(t) * (lambda_i * D_i + delta_i)) - r > 0, else -1,
 *            applied only when the node's timing draw u < p_i (otherwise it holds),
 *            all nodes of a trial updated synchronously;
 *   Methods "CUDA programming and experimental conditions": I0(t+1) = I0(t)/beta,
 *            beta = (I0min/I0max)^(1/(S-1)), I0min = c_min/mean(s_i), I0max = c_max/mean(s_i),
 *            s_i = sqrt((n-1) Var(J_i,:)); MAX-CUT weights w enter as J = -w, h = 0.
 *
 * Conventions shared by every entry point:
 *  - All functions return pbit_status; none aborts.  On failure
 *    pbit_last_error() returns a thread-local message.
 *  - Spins are int8 in {-1,+1}, TRIAL-MAJOR: spins[i*T + t] is node i of trial t.
 *  - "device" pointers are CUDA global memory of the graph's device (e.g. a
 *    torch tensor's data_ptr()); "host" pointers are ordinary CPU memory.
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream.  Work is enqueued on it in order; entry points that return
 *    results in host memory synchronise that stream before returning.
 *  - Random numbers are Philox4x32-10 (Salmon et al., SC'11) with key =
 *    (seed low word, seed high word) and counter = (node, step, instance, c).
 *    The trials 8g .. 8g+7 share the blocks c = 3g, 3g+1, 3g+2 (all 384 bits
 *    used).  Trial k = t mod 8 takes output word k mod 4 of block 3g + k/4 as
 *    its r-word wr: r = (2*(wr>>8)+1-2^24)/2^24; its u = q/2^24 with the
 *    24-bit q = (half (k mod 2) of output word k/2 of block 3g+2) * 2^8 +
 *    (wr & 0xFF).  The
 *    initial state (step counter 0xFFFFFFFF) is +1 iff r < 0.  Results are
 *    therefore a pure function of (graph, parameters, seed, instance) and do
 *    not depend on the kernel, batch or server slot that computed them.
 */
#ifndef PBIT_H
#define PBIT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PBIT_OK = 0,
    PBIT_PENDING = 1,          /* pbit_server_poll: request not finished yet */
    PBIT_E_INVALID = -1,       /* bad argument, bad edge list or shape */
    PBIT_E_NOMEM = -2,         /* host or device allocation failed */
    PBIT_E_CUDA = -3,          /* a CUDA runtime call failed (message has the text) */
    PBIT_E_TIMEOUT = -4,       /* a bounded device-side wait ran out; state undefined */
    PBIT_E_BUDGET = -5,        /* request larger than the server's HBM budget */
    PBIT_E_UNSUPPORTED = -6,   /* the forced kernel cannot run this shape */
    PBIT_E_NOTFOUND = -7       /* unknown request id */
} pbit_status;

/* Thread-local text of the last failure on this thread ("" if none). */
const char* pbit_last_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int32_t pbit_version(void);

/* Number of CUDA kernels this library has launched in this process so far. */
int64_t pbit_launch_count(void);

/* ------------------------------------------------------------------------ */
/* Instance (MAX-CUT problem statement, Methods; Eq. 2 "eqn:Ising")          */
/* ------------------------------------------------------------------------ */

typedef struct pbit_graph_s* pbit_graph;

#define PBIT_GRAPH_DENSE 1u     /* also build the dense tensor-core operands of J: e4m3 (|w| <= 16,
                                   n <= 8192) and, where exact, packed e2m1 (n <= 2048, |w| in
                                   {0,1,2,3,4,6}) for the cluster-resident kernel */

/*
 * Create a MAX-CUT instance on the current CUDA device.
 *   n        number of nodes (1 <= n < 2^31)
 *   n_edges  number of undirected edges (>= 0)
 *   src,dst  HOST int32[n_edges] endpoints, 0 <= src,dst < n, src != dst, no
 *            undirected edge listed twice
 *   w        HOST int8[n_edges] MAX-CUT weights, -127..127 (J = -w)
 *   h        HOST int32[n] Ising biases, or NULL for h = 0
 *   flags    PBIT_GRAPH_DENSE to also build the dense operand (needs |w| <= 16)
 *   out      receives the handle
 * The library copies everything it needs (CSR of J in HBM; the caller keeps
 * ownership of its arrays).  Synchronous.  Errors: PBIT_E_INVALID for a
 * malformed edge list, PBIT_E_NOMEM, PBIT_E_CUDA.
 */
pbit_status pbit_graph_create(int32_t n, int64_t n_edges, const int32_t* src, const int32_t* dst,
                              const int8_t* w, const int32_t* h, uint32_t flags, pbit_graph* out);

/* Release a graph and its device memory (NULL is ignored). Synchronises the device. */
void pbit_graph_destroy(pbit_graph g);

typedef struct {
    int32_t n;             /* nodes */
    int64_t n_edges;       /* undirected edges */
    int32_t max_degree;    /* largest row of the CSR */
    int32_t unit_weights;  /* 1 if every |w| == 1 */
    int32_t has_dense;     /* 1 if the dense tensor-core operand was built */
    int32_t device;        /* CUDA device ordinal the graph lives on */
    double mean_s;         /* mean_i sqrt((n-1) Var(J_i,:)), the schedule's normaliser */
    int64_t total_weight;  /* W = sum of w over edges (cut = (W - H)/2 when h = 0) */
    size_t device_bytes;   /* HBM held by the graph */
    int32_t has_dense_fp4; /* 1 if the packed e2m1 operand of the cluster-resident dense kernel was built
                              (PBIT_GRAPH_DENSE, n <= 2048, every |w| in {0,1,2,3,4,6}) */
} pbit_graph_info_t;

pbit_status pbit_graph_info(pbit_graph g, pbit_graph_info_t* info);

/* ------------------------------------------------------------------------ */
/* Schedule (Methods: I0(t+1) = I0(t)/beta and the I0min/I0max rule)         */
/* ------------------------------------------------------------------------ */

/*
 * Write the float32 I0 table used by pbit_anneal into HOST float[steps]:
 * I0(0) = I0min, I0(t+1) = I0(t)/beta in FP64, each entry rounded to float32,
 * beta = (I0min/I0max)^(1/(steps-1)).  With normalize != 0,
 * I0min = i0_min/mean_s and I0max = i0_max/mean_s (mean_s from
 * pbit_graph_info); otherwise the end points are taken as given.
 * Errors: PBIT_E_INVALID for steps < 1, non-positive end points, or
 * normalize with mean_s == 0.
 */
pbit_status pbit_schedule(pbit_graph g, double i0_min, double i0_max, int32_t normalize, int32_t steps,
                          float* table);

/* Host-only (no device work): the same float32 table between two absolute
 * end points, I0(0) = i0_min ... I0(steps-1) ~ i0_max.  Writes HOST float[steps]. */
pbit_status pbit_i0_table(double i0_min, double i0_max, int32_t steps, float* table);

/* Host-only: validate an edge list like pbit_graph_create and write its
 * mean_s = mean_i sqrt((n-1) Var(J_i,:)) (population variance over the full
 * row of length n, zeros included) to *out. */
pbit_status pbit_mean_s(int32_t n, int64_t n_edges, const int32_t* src, const int32_t* dst, const int8_t* w,
                        double* out);

/* ------------------------------------------------------------------------ */
/* Annealing (Eqs. 1, 3, 6; the schedule of the Methods section)             */
/* ------------------------------------------------------------------------ */

typedef enum {
    PBIT_OFFSET_SCALED = 0,    /* x = I0 * (lambda*D + delta) */
    PBIT_OFFSET_LISTING = 1,   /* x = lambda * I0 * (D + delta)   (the paper's pseudo code) */
    PBIT_OFFSET_EQUATION = 2   /* x = lambda * (I0*D + delta)     (Eq. 6 with Eq. 3) */
} pbit_offset_mode;

typedef enum {
    PBIT_KERNEL_AUTO = 0,      /* pick from the graph shape */
    PBIT_KERNEL_SPARSE = 1,    /* CSR gather kernel: one persistent launch with per-tile step
                                  dependencies when they are local, else one launch per step */
    PBIT_KERNEL_DENSE = 2,     /* tensor-core field kernel (needs PBIT_GRAPH_DENSE) */
    PBIT_KERNEL_RESIDENT = 3   /* whole anneal in one launch on a cluster of up to 8 CTAs, each
                                  holding all spins in shared memory (2*n*T <= 200 KB) */
} pbit_kernel;

typedef struct {
    uint32_t struct_size;    /* sizeof(pbit_anneal_params) */
    int32_t trials;          /* T >= 1 independent trials */
    int32_t steps;           /* S >= 1 schedule length */
    int32_t step_begin;      /* first schedule index to run, 0 <= step_begin <= step_end */
    int32_t step_end;        /* one past the last index to run; 0 means S */
    double i0_min, i0_max;   /* schedule end points (numerators when i0_normalize) */
    int32_t i0_normalize;    /* 1: divide the end points by mean_s (the paper's rule) */
    int32_t offset_mode;     /* pbit_offset_mode */
    uint64_t seed;           /* Philox key */
    uint32_t instance;       /* the third Philox counter word (node, step, instance, c); SpSA's
                                stall draws use instance ^ 0x80000000, so keep instance < 2^31
                                where SpSA runs beside another instance's pSA draws */
    int32_t kernel;          /* pbit_kernel */
    const float* intensity;  /* HOST float[n] lambda_i, NULL = 1 */
    const float* offset;     /* HOST float[n] delta_i, NULL = 0 */
    const float* p_update;   /* HOST float[n] update probability p_i in [0,1], NULL = 1 */
    void* stream;            /* cudaStream_t */
    /* pSA variants (Methods: Eq. SpSA, Eq. TApSA) and the period timing model (Eq. pbits_variability
     * with T_res).  The sparse kernel runs them; DENSE and RESIDENT are pSA only. */
    int32_t algorithm;       /* PBIT_ALG_PSA, PBIT_ALG_SPSA (input kept with probability stall_prob),
                                PBIT_ALG_TAPSA (input = I0 * mean of the last `window` fields) */
    float stall_prob;        /* SpSA p in [0,1] (the paper uses 0.5) */
    int32_t window;          /* TApSA alpha, 1..64 (the paper uses 4) */
    int32_t t_res;           /* 0: off.  > 0: `steps` counts cycles of t_res sub-steps; node i updates at
                                sub-step q only when q % nu_i == 0, nu_i = max(1, round(t_res (1 + nu_dev_i)));
                                I0 = table[q / t_res]; step_begin/step_end then count sub-steps
                                (step_end 0 = steps * t_res).  The paper uses t_res = 10. */
    const float* nu_dev;     /* HOST float[n] timing deviations nu_dev_i ~ N(0, s_nu^2), NULL = 0 */
    void* state;             /* DEVICE variant state of pbit_variant_state_bytes() bytes, read and
                                written in place so a run can be resumed; NULL = a fresh zero state
                                (then step_begin must be 0) */
} pbit_anneal_params;

typedef enum { PBIT_ALG_PSA = 0, PBIT_ALG_SPSA = 1, PBIT_ALG_TAPSA = 2 } pbit_algorithm;

/* Bytes of variant state for n nodes and T trials: SpSA 4*n*T (float32 last input, [n][T]), TApSA
 * 2*window*n*T (int16 last fields, [window][n][T], slot q % window written at sub-step q), pSA 0.
 * Zero-filled memory is the state before step 0.  TApSA needs every field to fit int16
 * (|h_i| + sum_j |J_ij| <= 32767), else pbit_anneal returns PBIT_E_UNSUPPORTED. */
size_t pbit_variant_state_bytes(int32_t n, int32_t trials, int32_t algorithm, int32_t window);

/* Fill `p` with defaults: T=1, S=1, whole schedule, I0 0.1..10 normalised, SCALED, AUTO, pSA. */
void pbit_anneal_params_default(pbit_anneal_params* p);

/*
 * Run schedule steps [step_begin, step_end) of a pSA anneal.
 *   spins_in   DEVICE int8[n*T] start state, or NULL to start from the
 *              Philox initial state of (seed, instance)
 *   spins_out  DEVICE int8[n*T] final state; may equal spins_in
 * Running [0,k) and then [k,S) from its output equals running [0,S).
 * Stream-ordered on p->stream (this call does not wait for the GPU); it
 * allocates its scratch with cudaMallocAsync on that stream and copies the
 * per-node parameters from host memory, so it is not for use under stream
 * capture.  Scratch: up to three n*T spin buffers, the variant state
 * when p->state is NULL, under the timing model 8n + 2m bytes of periods,
 * node order and period buckets, and for the packed-FP4 dense kernel
 * 1.5 * K * T' bytes (K = n rounded up to 128, T' = T rounded up to the
 * kernel's trial group of 32 or 48): the packed start spins and the staging
 * slots through which each step's spin slices are exchanged.  Errors: PBIT_E_INVALID, PBIT_E_UNSUPPORTED
 * (forced kernel cannot run the shape; TApSA fields beyond int16),
 * PBIT_E_NOMEM, PBIT_E_CUDA.
 */
pbit_status pbit_anneal(pbit_graph g, const pbit_anneal_params* p, const int8_t* spins_in, int8_t* spins_out);

/*
 * pbit_anneal without any device allocation (the paper has no counterpart;
 * this is a deployment variant of pbit_anneal).  For callers that cannot
 * allocate device memory while they run: applications whose own caching
 * allocator has reserved nearly all of HBM up front (a library cudaMalloc
 * would fail or take memory promised elsewhere), processes under a fixed
 * device-memory cap, and latency-bound loops that cannot absorb an
 * allocation's synchronisation.  Same arguments, results and Philox stream
 * as pbit_anneal with kernel = PBIT_KERNEL_SPARSE (p->kernel is ignored;
 * plain pSA only, else PBIT_E_UNSUPPORTED); every step runs the graph's
 * per-step sparse tile.  All scratch lives in one fixed 32 MiB device array
 * inside libpbit.so, held on every GPU that loads the library until the
 * process exits; the call needs 4*steps + 12*n + n*trials bytes of it (each
 * part rounded up to 256) and returns PBIT_E_INVALID, with the sizes in
 * pbit_last_error(), when that is more.  It calls no cudaMalloc/cudaFree.
 * It does call the CUDA runtime (the array's address is looked up with
 * cudaGetSymbolAddress on every call; parameters are uploaded with
 * cudaMemcpyAsync from pageable host memory), so it must not be called from
 * a stream callback or host function, and, like pbit_anneal, it is not for
 * use under stream capture.  Non-finite intensity or offset values give
 * PBIT_E_INVALID.  Every call reuses the same array, so calls whose GPU work
 * overlaps (e.g. on two streams) race and must be serialised by the caller.
 */
pbit_status pbit_anneal_noalloc(pbit_graph g, const pbit_anneal_params* p, const int8_t* spins_in,
                                int8_t* spins_out);

/*
 * The kernel pbit_anneal runs for `requested` (a pbit_kernel) and `trials`
 * on this graph: AUTO resolves to DENSE when the graph holds the dense
 * operand and the trial count suits it, else RESIDENT when both spin buffers
 * fit one CTA's shared memory, else SPARSE.  PBIT_E_UNSUPPORTED if a forced
 * kernel cannot run the shape.
 */
pbit_status pbit_select_kernel(pbit_graph g, int32_t requested, int32_t trials, int32_t* kernel);

/*
 * pbit_anneal that also records an observable of the state after every `every`
 * steps (and after the last step): `what` = 0 energy H, 1 cut.  `trace` is
 * DEVICE int64[ceil(k/every)][T] for k = step_end - step_begin steps, written
 * stream-ordered (the paper's energy-vs-cycle curves).
 */
pbit_status pbit_anneal_trace(pbit_graph g, const pbit_anneal_params* p, const int8_t* spins_in, int8_t* spins_out,
                              int32_t every, int32_t what, int64_t* trace);

/* Write the Philox initial state of (seed, instance) to DEVICE int8[n*T]. */
pbit_status pbit_init_spins(pbit_graph g, int32_t trials, uint64_t seed, uint32_t instance, int8_t* spins,
                            void* stream);

/* ------------------------------------------------------------------------ */
/* Exact observables (Eq. 3 fields, Eq. 2 energy, the MAX-CUT objective)     */
/* ------------------------------------------------------------------------ */

/* DEVICE int32[n*T] fields D_i(t) = h_i + sum_j J_ij sigma_j(t). Stream-ordered. */
pbit_status pbit_fields(pbit_graph g, const int8_t* spins, int32_t trials, int32_t* fields, void* stream);

/*
 * The same fields computed by the tensor-core kernel (needs a graph created
 * with PBIT_GRAPH_DENSE and trials % 32 == 0, trials <= 128 or % 128 == 0):
 * J as e4m3 tiles times the spins as e4m3, FP32 accumulation, exact because
 * |J| <= 16 and every partial sum is an integer below 2^24.  DEVICE int32[n*T].
 */
pbit_status pbit_fields_dense(pbit_graph g, const int8_t* spins, int32_t trials, int32_t* fields, void* stream);

/*
 * Synchronise `stream` and report whether any kernel of this graph gave up a
 * bounded device-side wait since the last call (PBIT_E_TIMEOUT; the results
 * of that work are undefined).  Clears the flag.
 */
pbit_status pbit_graph_status(pbit_graph g, void* stream);

/*
 * Exercise the failure path without a fault: one kernel waits for a device
 * flag that nothing sets, gives up after about budget_us microseconds
 * (1..2e6), records the timeout in the graph's error word and returns, so a
 * following pbit_graph_status reports PBIT_E_TIMEOUT and the context stays
 * usable.  Stream-ordered.
 */
pbit_status pbit_selftest_timeout(pbit_graph g, int32_t budget_us, void* stream);

/*
 * Per-trial cut = sum over edges of w * [sigma_src != sigma_dst], and energy
 * H = -sum_i h_i sigma_i - sum_{i<j} J_ij sigma_i sigma_j, exact int64.
 * `out` is HOST int64[T] (the call synchronises `stream`) when out_on_host
 * != 0, else DEVICE int64[T] written stream-ordered.
 */
pbit_status pbit_cut(pbit_graph g, const int8_t* spins, int32_t trials, int64_t* out, int32_t out_on_host,
                     void* stream);
pbit_status pbit_energy(pbit_graph g, const int8_t* spins, int32_t trials, int64_t* out, int32_t out_on_host,
                        void* stream);

/* ------------------------------------------------------------------------ */
/* Batched annealing: many instances of uneven size in one persistent        */
/* launch per chunk of steps, replayed from a captured CUDA graph            */
/* ------------------------------------------------------------------------ */

typedef struct pbit_batch_s* pbit_batch;

/*
 * Build a batch of `count` anneals.  graphs[k] must stay alive until the
 * batch is destroyed; params[k] gives trials, schedule, range, seed,
 * instance, offset mode and HOST variability arrays (copied; `kernel` and
 * `stream` are ignored).  Device memory: two int8 spin buffers of n*T per
 * instance plus its tables.  Each instance starts from the Philox initial
 * state of its (seed, instance) (pbit_batch_set_spins replaces it).
 * Synchronous.  Results equal pbit_anneal's for the same parameters.
 */
pbit_status pbit_batch_create(int32_t count, const pbit_graph* graphs, const pbit_anneal_params* params,
                              pbit_batch* out);
void pbit_batch_destroy(pbit_batch b);

/* Copy DEVICE int8[n*T] spins into instance k's current state (stream-ordered). */
pbit_status pbit_batch_set_spins(pbit_batch b, int32_t k, const int8_t* spins, void* stream);

/*
 * Advance every instance towards its step_end in chunks of `chunk_steps`
 * schedule steps (0 keeps the current tuning), at most `max_chunks` chunks
 * (0 = until every instance is done).  One chunk = one persistent kernel
 * over all instances plus a small bookkeeping kernel, replayed from a CUDA
 * graph.  Stream-ordered; does not wait for the GPU.
 */
pbit_status pbit_batch_run(pbit_batch b, int32_t chunk_steps, int32_t max_chunks, void* stream);

/* Next schedule step of instance k, as enqueued so far. */
pbit_status pbit_batch_progress(pbit_batch b, int32_t k, int32_t* step);

/* Copy instance k's current spins to DEVICE int8[n*T] (stream-ordered). */
pbit_status pbit_batch_spins(pbit_batch b, int32_t k, int8_t* spins_out, void* stream);

/* Per-trial cut of instance k's current state into HOST int64[T]; synchronises `stream`. */
pbit_status pbit_batch_cuts(pbit_batch b, int32_t k, int64_t* cuts, void* stream);

typedef struct {
    int32_t chunk_steps;   /* schedule steps per persistent launch */
    int32_t ctas_per_sm;   /* persistent CTAs per SM (0 = occupancy maximum) */
    float ms_per_step;     /* measured time of one step of the whole batch */
} pbit_batch_tuning;

/*
 * Autotuner: times one chunk for each (chunk_steps in {8,16,32,64},
 * ctas_per_sm in {1,2,4,max}) from the current state, restoring the state
 * after every trial, and keeps the fastest.  Tiling never changes results.
 * Synchronises `stream`.
 */
pbit_status pbit_batch_autotune(pbit_batch b, void* stream, pbit_batch_tuning* chosen);
pbit_status pbit_batch_set_tuning(pbit_batch b, int32_t chunk_steps, int32_t ctas_per_sm);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of MAX-CUT solve requests                    */
/* ------------------------------------------------------------------------ */

typedef struct pbit_server_s* pbit_server;

/*
 * Start a server on the current device: a worker thread with its own stream
 * that keeps up to `max_slots` requests resident, admits queued requests in
 * arrival order while their device memory fits `hbm_budget` bytes, and
 * advances every resident request by up to `chunk_steps` schedule steps per
 * persistent launch.  Finished requests are retired (exact cuts computed)
 * and their memory freed between launches.
 */
pbit_status pbit_server_create(size_t hbm_budget, int32_t max_slots, int32_t chunk_steps, pbit_server* out);

/* Stop the worker after the resident requests finish; queued ones are cancelled. */
void pbit_server_destroy(pbit_server s);

/*
 * Queue one anneal (the same parameters as pbit_anneal; host variability
 * arrays are copied).  `g` must stay alive until the request's result has
 * been taken.  PBIT_E_BUDGET if the request alone needs more device memory
 * than the budget (2*n*T spin bytes + 4*steps + 12*n + 1 KiB).
 */
pbit_status pbit_server_submit(pbit_server s, pbit_graph g, const pbit_anneal_params* p, uint64_t* req_id);

/*
 * PBIT_PENDING while the request is queued or running; PBIT_OK once done,
 * filling HOST int64[T] `cuts` and the seconds from submission to completion
 * in `latency_s` (either may be NULL) and forgetting the request;
 * PBIT_E_NOTFOUND for an unknown or already-taken id.
 */
pbit_status pbit_server_poll(pbit_server s, uint64_t req_id, int64_t* cuts, double* latency_s);

/* As pbit_server_poll, but blocks up to timeout_s seconds (<= 0: no limit). */
pbit_status pbit_server_wait(pbit_server s, uint64_t req_id, double timeout_s, int64_t* cuts, double* latency_s);

typedef struct {
    uint64_t completed;     /* requests finished */
    uint64_t queued;        /* waiting for admission */
    int32_t resident;       /* currently on the device */
    int32_t peak_resident;  /* most requests resident in one launch */
    uint64_t chunks;        /* persistent launches so far */
    double spin_updates;    /* total spin updates executed */
    double busy_seconds;    /* wall time spent inside launches */
    size_t hbm_in_use;      /* device bytes held by resident requests */
} pbit_server_stats_t;

pbit_status pbit_server_stats(pbit_server s, pbit_server_stats_t* out);

#ifdef __cplusplus
}
#endif

#endif /* PBIT_H */
