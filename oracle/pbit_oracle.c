/*
 * Plain CPU oracle for p-bit simulated annealing (pSA) with device variability.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product library never links, calls or falls back to it.  It shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * Arithmetic is FP64 (doubles formed from the same float32 inputs the GPU
 * receives); fields, cuts and energies are exact int64.  Single-threaded,
 * plain loops in the order of the paper's definitions.
 *
 * Paper sections followed (arXiv 2601.14476):
 *   Eq. (1)  "eqn:pbits"               p-bit output sgn(r + tanh(I))
 *   Eq. (2)  "eqn:Ising"               H = -sum_i h_i s_i - sum_{i<j} J_ij s_i s_j
 *   Eq. (3)  "eqn:conv"                I_i = I0 (h_i + sum_j J_ij s_j)
 *   Eq. (6)  "eqn:pbits_variability"   intensity lambda_i, offset delta_i, timing
 *   Eq. (7)  "eqn:variability"         lambda ~ N(1,s^2), delta ~ N(0,s^2), nu ~ N(0,s^2)
 *   Methods, "CUDA programming and experimental conditions": the I0 schedule
 *            I0(t+1) = I0(t)/beta, beta = (I0min/I0max)^(1/(cycle-1)),
 *            I0min = 0.1/mean(s_i), I0max = 10/mean(s_i), s_i = sqrt((n-1) Var(J_i,:)),
 *            and the MAX-CUT objective (maximise the total weight of cut edges).
 *
 * Readings of the paper taken here (each one is listed in the design notes):
 *   - sign convention: the new state is +1 iff tanh(x) - r > 0, else -1
 *     (r is symmetric, so this has the same law as sgn(r + tanh));
 *   - r is uniform on (-1,1), drawn on the 2^24-point midpoint grid
 *     r = (2k+1-2^24)/2^24 with k the top 24 bits of a Philox word;
 *   - timing variability is a per-node update probability p_i: a node updates
 *     at a step iff u < p_i with u = (top 24 bits)/2^24, otherwise it holds;
 *   - all nodes update synchronously (Jacobi: step t+1 reads only step t);
 *   - MAX-CUT weights w map to Ising couplings J = -w, h = 0;
 *   - Var(J_i,:) is the population variance over the full length-n row
 *     (zeros included);
 *   - the schedule recursion runs in FP64 and each entry is rounded to float32.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), written here from that paper's
 * definition.  key = (seed_lo, seed_hi); counter = (node, step, instance, c).
 * The eight trials 8g .. 8g+7 of a (node, step, instance) share the three
 * blocks c = 3g, 3g+1, 3g+2 (384 bits, 48 per trial).  Trial k = trial mod 8:
 * r-word = output word (k mod 4) of block 3g + k/4, r index = its top 24 bits;
 * u index (24 bits) = the 16 bits of half (k mod 2) of output word k/2 of block
 * 3g+2 (the high part), then the r-word's low 8 bits.
 * The initial state uses step = 0xFFFFFFFF and sets +1 iff r < 0.
 *
 * Pins (tests/test_oracle_pins.py): brute-force MAX-CUT for n <= 20, the
 * quadratic-form cut identity for both orientations, cut = (W - H)/2 with
 * h = 0, I0 = 0 gives Bernoulli(1/2) decisions, I0 -> inf gives sgn of the
 * field, fields equal an int64 dense matmul, Philox equals Triton's
 * independent implementation (and so do every trial's r and u indices taken
 * through the layout above), the 16 draws of a group share no bit, the
 * schedule closed form.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_E_INVALID (-1)
#define ORC_E_NOMEM (-2)

/* offset placement readings (design notes): */
#define ORC_OFFSET_SCALED 0 /* x = I0 * (lambda*D + delta)  */
#define ORC_OFFSET_LISTING 1   /* x = lambda * I0 * (D + delta) */
#define ORC_OFFSET_EQUATION 2  /* x = lambda * (I0*D + delta)  */

/* ------------------------------------------------------------------ */
/* Philox4x32-10, Salmon et al. SC'11: 10 rounds of the 4x32 S-box with the  */
/* multipliers 0xD2511F53, 0xCD9E8D57 and the Weyl key increments            */
/* 0x9E3779B9 (golden ratio), 0xBB67AE85 (sqrt(3)-1).                        */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { /* bump the key between rounds */
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The two uniforms one (node, step, trial, instance) draws. */
typedef struct {
    double r;   /* uniform on (-1,1), midpoint grid of 2^24 points */
    double u;   /* uniform on [0,1), grid of 2^24 points            */
} orc_draw;

static orc_draw orc_draw_for(uint64_t seed, uint32_t instance, int32_t node, uint32_t step, int32_t trial) {
    uint32_t group = (uint32_t)trial / 8u, kk = (uint32_t)trial % 8u;
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    uint32_t ctr_r[4] = {(uint32_t)node, step, instance, 3u * group + kk / 4u};
    uint32_t ctr_u[4] = {(uint32_t)node, step, instance, 3u * group + 2u};
    uint32_t wr_block[4], wu_block[4];
    orc_philox4x32_10(ctr_r, key, wr_block);
    orc_philox4x32_10(ctr_u, key, wu_block);
    uint32_t wr = wr_block[kk % 4u];
    uint32_t u_high = (wu_block[kk / 2u] >> (16u * (kk % 2u))) & 0xFFFFu;
    uint32_t k = wr >> 8;                    /* top 24 bits of the r-word */
    uint32_t q = (u_high << 8) | (wr & 0xFFu); /* 16 + 8 bits */
    orc_draw d;
    d.r = ((double)(2.0 * (double)k + 1.0) - 16777216.0) / 16777216.0;
    d.u = (double)q / 16777216.0;
    return d;
}

/* Expose one draw for tests (statistics of r and u). */
void orc_draw_ru(uint64_t seed, uint32_t instance, int32_t node, uint32_t step, int32_t trial,
                 double* r, double* u) {
    orc_draw d = orc_draw_for(seed, instance, node, step, trial);
    *r = d.r;
    *u = d.u;
}

/* ------------------------------------------------------------------ */
/* Instance: MAX-CUT edge list -> Ising couplings J = -w in CSR form.        */
/* ------------------------------------------------------------------ */
/* Validates the edge list (no self loops, endpoints in range, no duplicate  */
/* undirected edge) and fills row_ptr[n+1], col[2m], J[2m] with J = -w.      */
/* Neighbours of each row are sorted by column.                              */
static int cmp_pair(const void* a, const void* b) {
    const int64_t* x = (const int64_t*)a;
    const int64_t* y = (const int64_t*)b;
    if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
    return 0;
}

int orc_build_csr(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, const int8_t* w,
                  int32_t* row_ptr, int32_t* col, int8_t* J) {
    if (n <= 0 || m < 0) return ORC_E_INVALID;
    for (int64_t e = 0; e < m; ++e) {
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return ORC_E_INVALID;
        if (src[e] == dst[e]) return ORC_E_INVALID;
        if (w[e] == -128) return ORC_E_INVALID; /* J = -w must fit int8 */
    }
    /* entries (key = row*n + col, value = -w), both directions */
    int64_t* ent = (int64_t*)malloc(sizeof(int64_t) * 2 * (size_t)(2 * m + 1));
    if (!ent) return ORC_E_NOMEM;
    for (int64_t e = 0; e < m; ++e) {
        ent[2 * (2 * e)] = (int64_t)src[e] * n + dst[e];
        ent[2 * (2 * e) + 1] = -(int64_t)w[e];
        ent[2 * (2 * e + 1)] = (int64_t)dst[e] * n + src[e];
        ent[2 * (2 * e + 1) + 1] = -(int64_t)w[e];
    }
    qsort(ent, (size_t)(2 * m), 2 * sizeof(int64_t), cmp_pair);
    for (int64_t k = 1; k < 2 * m; ++k)
        if (ent[2 * k] == ent[2 * (k - 1)]) { free(ent); return ORC_E_INVALID; }
    for (int32_t i = 0; i <= n; ++i) row_ptr[i] = 0;
    for (int64_t k = 0; k < 2 * m; ++k) row_ptr[ent[2 * k] / n + 1] += 1;
    for (int32_t i = 0; i < n; ++i) row_ptr[i + 1] += row_ptr[i];
    for (int64_t k = 0; k < 2 * m; ++k) {
        col[k] = (int32_t)(ent[2 * k] % n);
        J[k] = (int8_t)ent[2 * k + 1];
    }
    free(ent);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Schedule (Methods): mean(s_i), I0min/I0max, beta, I0(t+1) = I0(t)/beta.  */
/* ------------------------------------------------------------------ */
/* s_i = sqrt((n-1) * Var(J_i,:)), population variance over the full row of */
/* length n (the zero entries included), mean over all n nodes.             */
double orc_mean_s(int32_t n, const int32_t* row_ptr, const int8_t* J) {
    double acc = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        int64_t s1 = 0, s2 = 0;
        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            s1 += J[k];
            s2 += (int64_t)J[k] * J[k];
        }
        double mean = (double)s1 / (double)n;
        double var = (double)s2 / (double)n - mean * mean;
        if (var < 0.0) var = 0.0;
        acc += sqrt((double)(n - 1) * var);
    }
    return acc / (double)n;
}

/* table[t] = float32 of I0(t) for t = 0..steps-1, with I0(0) = i0min and    */
/* I0(t+1) = I0(t) / beta, beta = (i0min/i0max)^(1/(steps-1)), all in FP64.  */
void orc_i0_table(double i0min, double i0max, int32_t steps, float* table) {
    if (steps <= 0) return;
    double beta = steps > 1 ? pow(i0min / i0max, 1.0 / (double)(steps - 1)) : 1.0;
    double i0 = i0min;
    for (int32_t t = 0; t < steps; ++t) {
        table[t] = (float)i0;
        i0 = i0 / beta;
    }
}

/* ------------------------------------------------------------------ */
/* Fields, energy, cut (Eqs. 2-3 and the MAX-CUT objective).                 */
/* ------------------------------------------------------------------ */
/* sigma is trial-major: sigma[i*T + t] is node i of trial t, in {-1,+1}.    */
/* D[i*T + t] = h_i + sum_j J_ij sigma_j(t), exact.                          */
void orc_fields(int32_t n, const int32_t* row_ptr, const int32_t* col, const int8_t* J, const int32_t* h,
                const int8_t* sigma, int32_t T, int64_t* D) {
    for (int32_t i = 0; i < n; ++i)
        for (int32_t t = 0; t < T; ++t) {
            int64_t d = h ? h[i] : 0;
            for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
                d += (int64_t)J[k] * sigma[(int64_t)col[k] * T + t];
            D[(int64_t)i * T + t] = d;
        }
}

/* H(sigma) = -sum_i h_i sigma_i - sum_{i<j} J_ij sigma_i sigma_j per trial. */
void orc_energy(int32_t n, const int32_t* row_ptr, const int32_t* col, const int8_t* J, const int32_t* h,
                const int8_t* sigma, int32_t T, int64_t* H) {
    for (int32_t t = 0; t < T; ++t) {
        int64_t e = 0;
        for (int32_t i = 0; i < n; ++i) {
            int64_t si = sigma[(int64_t)i * T + t];
            if (h) e -= (int64_t)h[i] * si;
            for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                int32_t j = col[k];
                if (i < j) e -= (int64_t)J[k] * si * sigma[(int64_t)j * T + t];
            }
        }
        H[t] = e;
    }
}

/* MAX-CUT value straight from the edge list: sum of w over edges whose      */
/* endpoints lie on different sides.                                         */
void orc_cut(int64_t m, const int32_t* src, const int32_t* dst, const int8_t* w, const int8_t* sigma,
             int32_t T, int64_t* cut) {
    for (int32_t t = 0; t < T; ++t) {
        int64_t c = 0;
        for (int64_t e = 0; e < m; ++e)
            if (sigma[(int64_t)src[e] * T + t] != sigma[(int64_t)dst[e] * T + t]) c += w[e];
        cut[t] = c;
    }
}

/* Exhaustive maximum cut for small n (n <= 24): every partition with node 0 */
/* fixed to side +1.  Returns the maximum and writes one maximiser.          */
int64_t orc_bruteforce_maxcut(int32_t n, int64_t m, const int32_t* src, const int32_t* dst, const int8_t* w,
                              int8_t* best_sigma) {
    if (n <= 0 || n > 24) return INT64_MIN;
    int64_t best = INT64_MIN;
    uint32_t best_mask = 0;
    uint32_t count = 1u << (n - 1);
    for (uint32_t mask = 0; mask < count; ++mask) {
        uint32_t full = mask << 1; /* bit i set: node i on side -1; node 0 on +1 */
        int64_t c = 0;
        for (int64_t e = 0; e < m; ++e)
            if (((full >> src[e]) & 1u) != ((full >> dst[e]) & 1u)) c += w[e];
        if (c > best) { best = c; best_mask = full; }
    }
    if (best_sigma)
        for (int32_t i = 0; i < n; ++i) best_sigma[i] = ((best_mask >> i) & 1u) ? -1 : 1;
    return best;
}

/* ------------------------------------------------------------------ */
/* One synchronous pSA step with the variability p-bit (Eqs. 1, 3, 6).       */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t n;
    const int32_t* row_ptr;
    const int32_t* col;
    const int8_t* J;
    const int32_t* h;        /* may be NULL: h = 0 */
    int32_t T;
    const float* lambda;     /* intensity; NULL = 1 */
    const float* delta;      /* offset;    NULL = 0 */
    const float* p_update;   /* timing;    NULL = 1 */
    int32_t offset_mode;
    uint64_t seed;
    uint32_t instance;
    int32_t trial_base;      /* global index of column 0: column t is trial trial_base + t */
} orc_problem;

/* x for one node given its exact field D and the current I0. */
static double orc_input(const orc_problem* P, int32_t i, int64_t D, float I0f) {
    double I0 = (double)I0f;
    double lam = P->lambda ? (double)P->lambda[i] : 1.0;
    double del = P->delta ? (double)P->delta[i] : 0.0;
    double d = (double)D;
    switch (P->offset_mode) {
    case ORC_OFFSET_LISTING: return lam * I0 * (d + del);
    case ORC_OFFSET_EQUATION: return lam * (I0 * d + del);
    default: return I0 * (lam * d + del);
    }
}

/* Next state of one (node, trial) from the full current state; optionally  */
/* reports gap = tanh(x) - r and whether the node updated.                  */
static int8_t orc_next(const orc_problem* P, const int8_t* sigma, int32_t i, int32_t t, uint32_t step, float I0,
                       double* gap, int* updated) {
    int64_t D = P->h ? P->h[i] : 0;
    for (int32_t k = P->row_ptr[i]; k < P->row_ptr[i + 1]; ++k)
        D += (int64_t)P->J[k] * sigma[(int64_t)P->col[k] * P->T + t];
    double x = orc_input(P, i, D, I0);
    orc_draw dr = orc_draw_for(P->seed, P->instance, i, step, P->trial_base + t);
    double g = tanh(x) - dr.r;
    int8_t cand = g > 0.0 ? 1 : -1;
    double p = P->p_update ? (double)P->p_update[i] : 1.0;
    int upd = dr.u < p;
    if (gap) *gap = g;
    if (updated) *updated = upd;
    return upd ? cand : sigma[(int64_t)i * P->T + t];
}

static void orc_problem_init(orc_problem* P, int32_t n, const int32_t* row_ptr, const int32_t* col, const int8_t* J,
                             const int32_t* h, int32_t T, const float* lambda, const float* delta,
                             const float* p_update, int32_t offset_mode, uint64_t seed, uint32_t instance) {
    P->n = n; P->row_ptr = row_ptr; P->col = col; P->J = J; P->h = h; P->T = T;
    P->lambda = lambda; P->delta = delta; P->p_update = p_update; P->offset_mode = offset_mode;
    P->seed = seed; P->instance = instance; P->trial_base = 0;
}

/* One Jacobi step of the columns of sigma_in (trials trial_base .. trial_base+T-1). */
static void orc_step_cols(const orc_problem* P, uint32_t step, float I0, const int8_t* sigma_in, int8_t* sigma_out,
                          double* gap) {
    for (int32_t i = 0; i < P->n; ++i)
        for (int32_t t = 0; t < P->T; ++t) {
            double g;
            sigma_out[(int64_t)i * P->T + t] = orc_next(P, sigma_in, i, t, step, I0, &g, NULL);
            if (gap) gap[(int64_t)i * P->T + t] = g;
        }
}

/* sigma_out = one Jacobi step of sigma_in at schedule index `step` with I0. */
/* gap (optional, n*T doubles) receives tanh(x) - r for every decision.      */
void orc_step(int32_t n, const int32_t* row_ptr, const int32_t* col, const int8_t* J, const int32_t* h, int32_t T,
              const float* lambda, const float* delta, const float* p_update, int32_t offset_mode, uint64_t seed,
              uint32_t instance, uint32_t step, float I0, const int8_t* sigma_in, int8_t* sigma_out, double* gap) {
    orc_problem P;
    orc_problem_init(&P, n, row_ptr, col, J, h, T, lambda, delta, p_update, offset_mode, seed, instance);
    orc_step_cols(&P, step, I0, sigma_in, sigma_out, gap);
}

/* The same step, evaluated only at the listed (node, trial) pairs.          */
void orc_step_sampled(int32_t n, const int32_t* row_ptr, const int32_t* col, const int8_t* J, const int32_t* h,
                      int32_t T, const float* lambda, const float* delta, const float* p_update,
                      int32_t offset_mode, uint64_t seed, uint32_t instance, uint32_t step, float I0,
                      const int8_t* sigma_in, int64_t count, const int32_t* nodes, const int32_t* trials,
                      int8_t* out, double* gap) {
    orc_problem P;
    orc_problem_init(&P, n, row_ptr, col, J, h, T, lambda, delta, p_update, offset_mode, seed, instance);
    for (int64_t s = 0; s < count; ++s) {
        double g;
        out[s] = orc_next(&P, sigma_in, nodes[s], trials[s], step, I0, &g, NULL);
        if (gap) gap[s] = g;
    }
}

/* Initial state of trials trial_base .. trial_base+T-1 (column t is trial   */
/* trial_base + t): +1 iff the step-0xFFFFFFFF draw has r < 0.               */
void orc_init_spins_trials(int32_t n, int32_t T, int32_t trial_base, uint64_t seed, uint32_t instance,
                           int8_t* sigma) {
    for (int32_t i = 0; i < n; ++i)
        for (int32_t t = 0; t < T; ++t) {
            orc_draw d = orc_draw_for(seed, instance, i, 0xFFFFFFFFu, trial_base + t);
            sigma[(int64_t)i * T + t] = d.r < 0.0 ? 1 : -1;
        }
}

void orc_init_spins(int32_t n, int32_t T, uint64_t seed, uint32_t instance, int8_t* sigma) {
    orc_init_spins_trials(n, T, 0, seed, instance, sigma);
}

/* Full anneal over schedule steps [step_begin, step_end) of `table` for the */
/* trials trial_base .. trial_base+T-1 (every trial is independent, so a    */
/* range of columns equals those columns of a run over all trials).         */
/* sigma holds the start state on entry and the final state on return.       */
int orc_anneal_trials(int32_t n, const int32_t* row_ptr, const int32_t* col, const int8_t* J, const int32_t* h,
                      int32_t T, int32_t trial_base, const float* lambda, const float* delta, const float* p_update,
                      int32_t offset_mode, uint64_t seed, uint32_t instance, const float* table, int32_t step_begin,
                      int32_t step_end, int8_t* sigma) {
    int64_t cells = (int64_t)n * T;
    int8_t* next = (int8_t*)malloc((size_t)cells);
    if (!next) return ORC_E_NOMEM;
    orc_problem P;
    orc_problem_init(&P, n, row_ptr, col, J, h, T, lambda, delta, p_update, offset_mode, seed, instance);
    P.trial_base = trial_base;
    for (int32_t s = step_begin; s < step_end; ++s) {
        orc_step_cols(&P, (uint32_t)s, table[s], sigma, next, NULL);
        memcpy(sigma, next, (size_t)cells);
    }
    free(next);
    return ORC_OK;
}

int orc_anneal(int32_t n, const int32_t* row_ptr, const int32_t* col, const int8_t* J, const int32_t* h, int32_t T,
               const float* lambda, const float* delta, const float* p_update, int32_t offset_mode, uint64_t seed,
               uint32_t instance, const float* table, int32_t step_begin, int32_t step_end, int8_t* sigma) {
    return orc_anneal_trials(n, row_ptr, col, J, h, T, 0, lambda, delta, p_update, offset_mode, seed, instance,
                             table, step_begin, step_end, sigma);
}

/* ------------------------------------------------------------------ */
/* pSA variants of the Methods section and the paper's timing model.        */
/*   SpSA  (Eq. SpSA):  with probability p the input keeps I_i(t-1),        */
/*                      otherwise I_i(t) = I0(t) * (h_i + sum_j J_ij s_j).  */
/*   TApSA (Eq. TApSA): I_i(t) = I0(t) * (1/alpha) * sum_{k<alpha} TI(t-k), */
/*                      TI(t) = h_i + sum_j J_ij s_j(t), TI(t < 0) = 0.      */
/*   Timing (Eq. pbits_variability, T_res): cycle c has T_res sub-steps;    */
/*   node i updates at sub-step q only when q mod nu_i == 0, with           */
/*   nu_i = max(1, round(T_res * (1 + nu_dev_i))); I0 is I0(q / T_res).     */
/* The p-bit then takes x from the input I:                                 */
/*   SCALED x = lambda I + I0 delta, LISTING x = lambda (I + I0 delta),  */
/*   EQUATION x = lambda (I + delta)  (each reduces to the pSA form when    */
/*   I = I0 D).  Random words: (r, u) as for pSA at counter step q; the     */
/*   SpSA stall draw is word (trial mod 4) of Philox at counter (node, q,   */
/*   instance ^ 0x80000000, trial / 4), stall iff top 24 bits / 2^24 < p.   */
/* ------------------------------------------------------------------ */
#define ORC_ALG_PSA 0
#define ORC_ALG_SPSA 1
#define ORC_ALG_TAPSA 2

static double orc_stall_draw(uint64_t seed, uint32_t instance, int32_t node, uint32_t step, int32_t trial) {
    uint32_t ctr[4] = {(uint32_t)node, step, instance ^ 0x80000000u, (uint32_t)trial >> 2};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    return (double)(w[trial & 3] >> 8) / 16777216.0;
}

/* nu_i = max(1, round(T_res * (1 + nu_dev_i))), round half away from zero */
int32_t orc_timing_period(int32_t t_res, float nu_dev) {
    double v = round((double)t_res * (1.0 + (double)nu_dev));
    return v < 1.0 ? 1 : (int32_t)v;
}

/* One sub-step q of a variant.  State (per node, trial):
 *   SpSA : Iprev[i*T+t] (double) the last input, 0 before the first step;
 *   TApSA: ring[(k*n + i)*T + t] (int64) the last `window` fields, slot q mod window.
 * t_res <= 0 disables the timing model (every node updates every step, I0 = table[q]). */
void orc_step_variant(int32_t n, const int32_t* row_ptr, const int32_t* col, const int8_t* J, const int32_t* h,
                      int32_t T, const float* lambda, const float* delta, const float* p_update,
                      int32_t offset_mode, uint64_t seed, uint32_t instance, int32_t algorithm, double stall_prob,
                      int32_t window, int32_t t_res, const float* nu_dev, uint32_t q, const float* table,
                      const int8_t* sigma_in, int8_t* sigma_out, double* Iprev, int64_t* ring, double* gap) {
    for (int32_t i = 0; i < n; ++i) {
        const int32_t nu = t_res > 0 ? orc_timing_period(t_res, nu_dev ? nu_dev[i] : 0.0f) : 1;
        const int due = (q % (uint32_t)nu) == 0;
        const double I0 = (double)table[t_res > 0 ? q / (uint32_t)t_res : q];
        const double lam = lambda ? (double)lambda[i] : 1.0;
        const double del = delta ? (double)delta[i] : 0.0;
        const double p = p_update ? (double)p_update[i] : 1.0;
        for (int32_t t = 0; t < T; ++t) {
            const int64_t c = (int64_t)i * T + t;
            if (!due) {
                sigma_out[c] = sigma_in[c];
                if (gap) gap[c] = 1.0; /* no decision */
                continue;
            }
            int64_t D = h ? h[i] : 0;
            for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) D += (int64_t)J[k] * sigma_in[(int64_t)col[k] * T + t];
            double I;
            if (algorithm == ORC_ALG_SPSA) {
                if (orc_stall_draw(seed, instance, i, q, t) < stall_prob) {
                    I = Iprev[c];
                } else {
                    I = I0 * (double)D;
                }
                Iprev[c] = I;
            } else if (algorithm == ORC_ALG_TAPSA) {
                ring[((int64_t)(q % (uint32_t)window) * n + i) * T + t] = D;
                int64_t sum = 0;
                for (int32_t k = 0; k < window; ++k) sum += ring[((int64_t)k * n + i) * T + t];
                I = I0 * (double)sum / (double)window;
            } else {
                I = I0 * (double)D;
            }
            double x;
            if (offset_mode == ORC_OFFSET_LISTING) x = lam * (I + I0 * del);
            else if (offset_mode == ORC_OFFSET_EQUATION) x = lam * (I + del);
            else x = lam * I + I0 * del;
            orc_draw dr = orc_draw_for(seed, instance, i, q, t);
            const double g = tanh(x) - dr.r;
            if (gap) gap[c] = g;
            sigma_out[c] = (dr.u < p) ? (g > 0.0 ? 1 : -1) : sigma_in[c];
        }
    }
}
