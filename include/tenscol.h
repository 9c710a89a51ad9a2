/*
 * tenscol.h -- C ABI of the GB300 (sm_103a) TensCol population step.
 *
 * TensCol (Goudet, Duval, Hao, "Population-based gradient descent weight
 * learning for graph coloring problems") keeps D candidate k-colourings of a
 * graph G = (V, E), |V| = n, as a real weight tensor W (D x n x k,
 * Section 3.2) and advances all of them at once with one iteration of
 * Algorithm 1 (Sections 3.3, 3.9):
 *   Step 1  S = one_hot(argmax W)                           (Section 3.4)
 *   Step 2  conflicts / fitness f(S_d), equity f_eq (ECP)    (eq. 1-3)
 *   Step 3  group concentration M~ = sum_d S_d S_d^T, penalty kappa and
 *           bonus varpi, loss L, gradient grad_S L           (eq. 4-7, 13-14)
 *   Step 4  softmax straight-through gradient, W <- W - eta grad_W L,
 *           smoothing W <- W / rho every nb_iter iterations  (eq. 8, 10-12)
 * until some individual is legal (f = 0) or the iteration budget ends.
 *
 * Conventions for every entry point:
 *   - Return TC_OK (0) or a negative TC_ERR_* code; tc_strerror() names it.
 *     No call throws across the ABI.  A failed call leaves the context in
 *     the state it had before the call, unless stated otherwise.
 *   - Pointer arguments are HOST memory unless the name ends in _dev.  All
 *     host buffers are caller-owned; the library copies in or out during
 *     the call and keeps no caller pointer.
 *   - A context is bound to one CUDA device and is not thread-safe: callers
 *     serialise calls on one context.  Contexts are independent.
 *   - Integer tensors are row-major: W index (d * n + i) * k + j,
 *     colours index d * n + i, M~ index i * n + m.
 */
#ifndef TENSCOL_H
#define TENSCOL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define TC_OK 0
#define TC_ERR_ARG (-1)            /* invalid argument or size              */
#define TC_ERR_GRAPH_ASYM (-2)     /* adjacency not symmetric / duplicated   */
#define TC_ERR_GRAPH_SELFLOOP (-3) /* a vertex adjacent to itself            */
#define TC_ERR_OOM (-4)            /* device or host allocation failed       */
#define TC_ERR_CUDA (-5)           /* a CUDA runtime call failed             */
#define TC_ERR_TIMEOUT (-6)        /* a bounded device wait expired          */
#define TC_ERR_DEVICE_BOUNDS (-7)  /* a device-side index check failed       */
#define TC_ERR_STATE (-8)          /* call out of order (no graph / no population) */
#define TC_ERR_UNSUPPORTED (-9)    /* size or form outside the built limits  */
#define TC_ERR_INJECTED (-10)      /* host-side fault injection (TC_FAULT)   */

/* ---- problems and step forms -------------------------------------------- */
#define TC_KCOL 0 /* k-colouring, GCP by k-descent (Section 3.5: f = f_color) */
#define TC_ECP 1  /* equitable colouring (eq. 3: f = f_color + f_eq)          */
/* k-partitioning (Section 6): Algorithm 1 with every M_d = S_d S_d^T of
 * eq. 1-7 replaced by J - M_d.  The fitness is the number of cut edges
 * (edges between different groups), the penalty and bonus of eq. 5-6 are
 * taken over sum_d (J - M_d) = D J - M~, and eq. 13's A.S, penalty and bonus
 * terms change sign.  The balanced variant adds f_eq of eq. 3 to the
 * fitness (and nu t grad f_eq to the gradient, as for the ECP). */
#define TC_KPART 2     /* f = cut edges                                      */
#define TC_KPART_BAL 3 /* f = cut edges + f_eq                               */
/* Minimum sum colouring (Section 6): colour l costs z_l >= 0
 * (tc_set_color_costs; z_l = l + 1 by default) and the additive fitness
 * f_mscp(S_d) = sum_i z_{c_d(i)} takes the place of f_eq: f = f_color +
 * f_mscp, nu t f_mscp in eq. 7 and nu t z_l in eq. 13.  With positive costs
 * f never reaches 0: the run goes on and tc_best keeps the lowest f. */
#define TC_MSCP 4

/* How steps 2-3 and the products of eq. 13 are computed.  All forms give
 * identical colours, conflicts and fitness and the same W step to FP32
 * rounding. */
#define TC_FORM_ONEHOT 0     /* gather/compare form: O(D n^2) CUDA-core work  */
#define TC_FORM_DENSE_FP8 1  /* A.S and S S^T as FP8 tcgen05 tensor-core GEMMs */
#define TC_FORM_DENSE_FP32 2 /* A.S and S S^T as FP32 CUDA-core GEMMs         */

/* Limits of this build. */
#define TC_MAX_N 32768
#define TC_MAX_K 1024
#define TC_MAX_D 65535

/* Parameters of Table 2 of the paper plus the run policy. */
typedef struct {
    int problem;     /* TC_KCOL, TC_ECP, TC_KPART, TC_KPART_BAL or TC_MSCP   */
    float sigma0;    /* std of the N(0, sigma0) initial weights (Section 3.2)*/
    float eta;       /* learning rate (Section 3.7)                          */
    float alpha;     /* penalisation exponent, > 1 (eq. 5)                   */
    float lambda_;   /* penalisation weight (eq. 7)                          */
    float beta;      /* bonus exponent, > 1 (eq. 6)                          */
    float mu;        /* bonus weight (eq. 7)                                 */
    float nu;        /* equity weight (eq. 7), 0 for the GCP                 */
    float rho;       /* smoothing divisor >= 1 (eq. 8); 1 disables smoothing */
    int nb_iter;     /* smoothing period in iterations (Step 4-iv)           */
    int stop_on_legal; /* 1: stop once min_d f(S_d) == 0 (Algorithm 1)       */
    int bonus_diag;  /* 1: bar A = J - A keeps its diagonal (Section 3.6.2)  */
    int form;        /* TC_FORM_*                                            */
} tc_params;

typedef struct tc_ctx tc_ctx; /* opaque: one graph + one population */

/* Fills *p with Table 2's column for `problem` (GCP: mu = 1e-6, nu = 0;
 * ECP: mu = 0, nu = 1e-5), rho = 100, stop_on_legal = 1, bonus_diag = 1,
 * form = TC_FORM_ONEHOT.  The paper gives no parameters for partitioning:
 * TC_KPART takes the GCP column, TC_KPART_BAL the GCP column with the ECP's
 * nu = 1e-5; so does TC_MSCP (nu weighs the colour costs).  Returns
 * TC_ERR_ARG for a NULL p or bad problem. */
int tc_params_default(tc_params *p, int problem);

/* Creates a context on CUDA device `device` with its own stream.
 * *out receives the context; on error *out is set to NULL. */
int tc_create(tc_ctx **out, int device);

/* Frees every device and host resource of the context (NULL is accepted). */
int tc_destroy(tc_ctx *ctx);

/* Runs later work on `stream` (a cudaStream_t of the context's device,
 * borrowed, never destroyed by the library); NULL restores the context's own
 * stream.  Captured CUDA graphs are dropped. */
int tc_set_stream(tc_ctx *ctx, void *stream);

/* Step "Input" of Algorithm 1: the graph.  Either CSR (rowptr[n+1],
 * colidx[rowptr[n]], each undirected edge listed from both ends, rows in any
 * order) or, when rowptr == NULL, a dense n*n row-major 0/1 matrix `dense`
 * (A of Section 3.5).  The graph is validated (symmetry, no self loop, ids
 * in range) and copied to the device.  Replaces any previous graph and
 * drops the population. */
int tc_init_graph(tc_ctx *ctx, int n, const int32_t *rowptr, const int32_t *colidx,
                  const uint8_t *dense);

/* Allocates a population of D individuals over k colours and draws
 * W ~ N(0, sigma0) on the device (Philox4x32-10 counter (d, i, j) keyed by
 * `seed`, Box-Muller), sets t = 0 and the best-so-far to "none".  *p is
 * copied; NULL means tc_params_default(TC_KCOL).  Parameters are checked
 * before anything changes; after that, any previous population is dropped
 * first, so a failed allocation leaves the context without a population. */
int tc_init_population(tc_ctx *ctx, uint64_t seed, int D, int k, const tc_params *p);

/* Replaces the parameters of the live population (same D, k). */
int tc_set_params(tc_ctx *ctx, const tc_params *p);

/* Runs up to n_iters iterations of Algorithm 1 (Steps 1-4 each).  Stops
 * early, without updating W, at the first iteration whose population holds a
 * legal individual when stop_on_legal is set.  *iters_done (may be NULL)
 * receives the number of weight updates performed.  The best-so-far
 * individual is tracked on the device at every evaluated iteration. */
int tc_step(tc_ctx *ctx, int64_t n_iters, int64_t *iters_done);

/* Best-so-far individual over all evaluated iterations (lowest fitness f
 * of the problem, lowest d among ties, first iteration reaching the value):
 * coloring[n] (caller-owned), its f_color (monochromatic edges; for the
 * partitioning problems the cut edges are |E| - f_color) and its additive
 * term in `equity` (f_eq, or f_mscp for TC_MSCP), the
 * individual index and the iteration t at which it was seen.  Any output
 * pointer may be NULL.  TC_ERR_STATE if no iteration has been evaluated
 * yet. */
int tc_best(tc_ctx *ctx, int32_t *coloring, int64_t *conflicts, int64_t *equity,
            int32_t *individual, int64_t *iteration);

/* Copies W (D*n*k floats, host memory, [d][i][j] order) and the iteration
 * counter t out / in.  Setting the state also recomputes the assignment S
 * (Step 1) and clears the stop flag; the best-so-far is kept.  Either
 * pointer may be NULL to skip it.  Page-locked W buffers (cudaHostAlloc,
 * cudaHostRegister) are read or written by the device directly, one block
 * per 32-row tile; pageable ones go through a staging copy.  Both return
 * once the transfer is complete. */
int tc_get_state(tc_ctx *ctx, float *W, int64_t *t);
int tc_set_state(tc_ctx *ctx, const float *W, const int64_t *t);

/* Device-resident variants: W_dev is a device pointer on the context's
 * device (D*n*k floats), copied on the context's stream. */
int tc_get_state_dev(tc_ctx *ctx, float *W_dev);
int tc_set_state_dev(tc_ctx *ctx, const float *W_dev);

/* Steps 1-3 for the current W at the current t, without updating W, the
 * counter or the best-so-far.  Outputs (each may be NULL):
 *   colors[D*n]    c_d(i) = argmax_j w_{d,i,j}, lowest j on ties (Section 3.4)
 *   gamma_own[D*n] conflicting neighbours of i in individual d (eq. 1)
 *   f_color[D]     monochromatic edges of individual d (eq. 1)
 *   f_eq[D]        equity fitness (eq. 3); f_mscp for TC_MSCP
 *   Mtilde[n*n]    group concentration matrix (eq. 4)
 *   G[D*n*k]       grad_S L at iteration t (eq. 13)
 *   loss[4]        L (eq. 7), kappa (eq. 5), varpi (eq. 6), sum_d f_color */
int tc_evaluate(tc_ctx *ctx, int32_t *colors, int32_t *gamma_own, int32_t *f_color,
                int32_t *f_eq, int32_t *Mtilde, float *G, float *loss);

/* Enqueues n_iters iterations on the context's stream and returns without
 * waiting (no host synchronisation, no stop polling).  Once the device stop
 * flag is raised the remaining enqueued iterations do nothing.  Read the
 * outcome later with tc_get_state / tc_best (which synchronise). */
int tc_step_async(tc_ctx *ctx, int64_t n_iters);

/* Kernel identifiers for tc_kernel_times. */
#define TC_KID_PAIRS 0   /* pair compare: M~, fitness, pair coefficients    */
#define TC_KID_CLASSES 1 /* colour classes, equity, population reduction    */
#define TC_KID_UPDATE 2  /* fused gradient gather + softmax-ST update        */
#define TC_KID_GEMM_M 3  /* dense forms: M~ = S S^T GEMM                     */
#define TC_KID_GEMM_G 4  /* dense forms: Gamma = A S GEMM                    */
#define TC_KID_GSUM 5    /* grad_S L tiles (class sums of the pair matrix)   */
#define TC_KID_GEMM_F 6  /* dense FP8 form: M~ and Gamma in one launch       */
#define TC_KID_FRONT 7   /* one-hot form: classes and pair terms, one launch */
#define TC_NUM_KID 8

/* Per-kernel device timing with CUDA events recorded around every launch
 * of tc_step / tc_step_async (on=1) or off (on=0; the default).  Graph
 * replay is not timed per kernel.  tc_kernel_times synchronises the stream,
 * adds the elapsed times of all completed launches to ms[TC_NUM_KID] and
 * count[TC_NUM_KID] (totals since timing was switched on) and returns them. */
int tc_set_timing(tc_ctx *ctx, int on);
int tc_kernel_times(tc_ctx *ctx, double *ms, int64_t *count);

/* Hand-written backward of the straight-through estimator (eq. 12-13) for
 * the current population at the current t: gradW_dev[D*n*k] (device) gets
 * grad_W L = S^ (.) (grad_S L - (S^ (.) grad_S L) J) with S^ = softmax(W)
 * and grad_S L of eq. 13 at the one-hot S = g(W), computed by the same code
 * as the fused update (which applies W <- W - eta grad_W L with one rounding
 * per operation, so the two agree bit for bit).  loss_dev[3] (device, may
 * be NULL) gets L (eq. 7), kappa (eq. 5), varpi (eq. 6).  W, t and the
 * best-so-far are unchanged. */
int tc_st_grad_dev(tc_ctx *ctx, float *gradW_dev, float *loss_dev);

/* Relaxation used to check the gradient (Section 3.8): S = softmax(W_dev /
 * tau) row-wise (real valued), eq. 7's GCP terms on it with M_d = S_d S_d^T
 * (nu ignored): loss_dev[4] = L, kappa, varpi, f_color; gradW_dev = dL/dW
 * (eq. 13 through the softmax Jacobian).  Device pointers of D*n*k floats;
 * uses the graph and parameters of the context, k <= 128.  Allocates and
 * frees its own temporaries; the population is not touched.  TC_ERR_ARG for
 * the partitioning problems and TC_MSCP. */
int tc_relaxed_dev(tc_ctx *ctx, const float *W_dev, float tau, int64_t t, float *loss_dev,
                   float *gradW_dev);

/* For callers that cannot allocate device memory: a process that shares a
 * GPU whose memory another framework's pool manages (allocating behind the
 * pool's back can fail or fragment it), a latency-critical loop that must
 * not call cudaMalloc / cudaFree (they can synchronise the whole device), or
 * an embedding whose device memory budget is fixed at start-up.  The paper
 * has no counterpart: this is a library service.  With no allocation of any
 * kind it computes the population pair terms of a population given as
 * colours -- the same kappa and varpi that tc_evaluate reports in loss[1]
 * and loss[2] -- from colors_dev[D*n] (device, uint16, individual-major:
 * colour of vertex i in individual d at d*n + i) and adj_dev[n*n] (device,
 * uint8 0/1, symmetric, zero diagonal), and writes out_dev[0] = kappa and
 * out_dev[1] = varpi (the diagonal of J - A included iff bonus_diag) in FP32
 * (device).  Its scratch is a file-scope device array of
 * TC_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits; n above TC_NOALLOC_MAX_N is rejected with TC_ERR_ARG.
 * The first call on a device (and the first after the device's primary
 * context was reset) looks up the array's device address
 * (cudaGetSymbolAddress), so make that first call before any stream
 * capture.  Every call shares the one array and clears its completion
 * counter first: calls that overlap on the GPU (other streams, other
 * threads) race and must be serialised by the caller.  Runs on the given
 * stream (NULL: the legacy default stream) of the current device and
 * returns without waiting. */
#define TC_NOALLOC_MAX_N 8192
#define TC_NOALLOC_SCRATCH_BYTES 264192
int tc_pair_terms_noalloc(int n, int D, const uint16_t *colors_dev, const uint8_t *adj_dev, float alpha,
                          float beta, int bonus_diag, float *out_dev, void *stream);

/* Limit of every bounded device wait of the context's one-hot kernels (a
 * TMA or record copy that never lands, an arrival that never comes), in
 * nanoseconds; 0 restores the default of one second.  A wait that runs out
 * records TC_ERR_TIMEOUT, which the next tc_step / tc_evaluate returns; the
 * kernel returns without touching memory outside its buffers, and the
 * context stays usable after tc_init_population.  Fault injection for tests
 * (environment, host side): TC_FAULT=alloc | copy | launch makes the next
 * allocation, host-device copy or iteration launch fail with
 * TC_ERR_INJECTED; TC_FAULT=wait makes k_gsum wait for an arrival that never
 * comes (the limit then decides when it gives up); with the device index
 * checks of libtenscol_bounds.so (a build with TC_BOUNDS=1), TC_FAULT=index
 * plants a vertex index past n in the first individual's class list, which
 * the checks report as TC_ERR_DEVICE_BOUNDS.  TC_ERR_ARG for a NULL context
 * or ns outside [0, 6e10]. */
int tc_set_wait_limit(tc_ctx *ctx, int64_t ns);

/* Number of device kernel launches issued by this context since creation
 * (for launch accounting in benchmarks). */
int tc_launch_count(tc_ctx *ctx, int64_t *count);

/* Enables (chunk > 0) or disables (chunk = 0) CUDA-graph replay of tc_step:
 * `chunk` iterations are captured once into one graph and replayed. */
int tc_set_graph_chunk(tc_ctx *ctx, int chunk);

/* k-descent: the GCP (or, with problem = TC_ECP, the ECP) approached as a
 * series of k-COL problems for decreasing k (Section 2 and the opening of
 * Section 3: every k with a legal colouring is an upper bound of the
 * chromatic, resp. equitable chromatic, number).  For k = k_start,
 * k_start - 1, ..., k_min: a fresh population of D individuals (seed + k),
 * Algorithm 1 with stop_on_legal for at most max_iters iterations; a legal
 * colouring (f_color = 0, and f_eq = 0 for the ECP) moves on to k - 1, the
 * first k without one within the budget ends the descent.  *p as for
 * tc_init_population (NULL: Table 2 for TC_KCOL; TC_ERR_ARG for the
 * partitioning problems and TC_MSCP); stop_on_legal is forced on.  Outputs (any may be
 * NULL): *k_best the smallest k solved (-1 if none), coloring[n] its legal
 * colouring, *iters_total the iterations run.  The context keeps the
 * population of the last k tried. */
int tc_kdescent(tc_ctx *ctx, uint64_t seed, int D, int k_start, int k_min, int64_t max_iters,
                const tc_params *p, int32_t *k_best, int32_t *coloring, int64_t *iters_total);

/* The plan the autotuner chose for the dense contractions of this context
 * (tc_init_population / tc_set_params time every candidate on the context's
 * own operands and keep the fastest; the FP32 form keeps one fixed plan).
 * `plan` has 9 entries:
 *   plan[0] Gamma unit rows: 128 (one CTA per unit) or 256 (a CTA pair
 *           running 256-row cta_group::2 MMAs)
 *   plan[1] Gamma column tile (128 or 256)   plan[2] Gamma cluster size
 *   plan[3..5] the same for M~               plan[6] M~ K splits
 *   plan[7] 1: both contractions in one launch (M~ units first)
 *   plan[8] candidates timed
 *   us[0..2] (us may be NULL; else 3 floats): best times of Gamma, M~ and
 *   the single launch of both in microseconds (0 when not timed, or FP32).
 * TC_ERR_STATE when the context has no dense form. */
int tc_dense_plan(tc_ctx *ctx, int32_t *plan, float *us);

/* One record of the iteration trace (tc_set_trace). */
typedef struct {
    int64_t t;          /* iteration of Algorithm 1                          */
    int32_t f_min;      /* min_d f(S_d) of the problem (the stop test)       */
    int32_t individual; /* lowest d attaining it                             */
    int32_t f_color;    /* its f_color (eq. 1)                               */
    int32_t f_add;      /* its additive term: f_eq (eq. 3), or f_mscp        */
    float loss;         /* L(t) of the population (eq. 7)                    */
    float kappa;        /* eq. 5                                             */
    float varpi;        /* eq. 6                                             */
    int32_t pad;
} tc_trace_entry;

/* Iteration trace (the loss and fitness evolution the paper follows in
 * Section 4.3): every `every` iterations t (t % every == 0) of tc_step /
 * tc_step_async / batches, the population reduction writes one record into
 * a device ring of `capacity` records; capacity 0 turns the trace off.
 * Clears the ring.  TC_ERR_ARG for capacity < 0 or every < 1, TC_ERR_STATE
 * without a population; a new population turns the trace off. */
int tc_set_trace(tc_ctx *ctx, int capacity, int every);

/* Copies the retained records, oldest first, up to `max` of them into out
 * (caller-owned; may be NULL to count only); *count receives how many are
 * retained (at most the capacity; 0 with the trace off).  Synchronises the
 * context's stream.  TC_ERR_ARG for max < 0, TC_ERR_STATE without a
 * population, a CUDA error code if the copy fails. */
int tc_get_trace(tc_ctx *ctx, tc_trace_entry *out, int max, int *count);

/* Colour costs z[0..k-1] >= 0 of the minimum sum colouring (TC_MSCP,
 * Section 6), copied; k must be the population's k.  Every population
 * starts with z_l = l + 1.  TC_ERR_ARG for a negative cost or another k,
 * TC_ERR_STATE without a population, TC_ERR_UNSUPPORTED when n max(z) + |E|
 * reaches 2^31 (the fitness is reduced in 32 bits).  Takes effect from the
 * next iteration, also inside captured CUDA graphs. */
int tc_set_color_costs(tc_ctx *ctx, const int32_t *z, int k);

/* Multicolouring (Section 6): vertex i must take demand[i] colours, no
 * colour shared across an edge.  Step 1 then selects the demand[i] colours
 * of largest weight in w_{d,i} (the lower colour first among equal weights)
 * and every other step of Algorithm 1 keeps its formula on the multi-hot S:
 * f_color counts, per edge, the colours its ends share; m~_im the colours i
 * and m share summed over the population (m~_ii = D demand[i]).  Needs the
 * k-COL problem in a dense form (FP8 or FP32: the GEMMs compute A.S and
 * S S^T of the multi-hot S); 1 <= demand[i] <= min(k, 8); n must be the
 * graph's n.  Re-derives the population's colours from W and clears the
 * best-so-far; all demands 1 returns to one colour per vertex.  A new
 * population (tc_init_population) starts with demands 1.  TC_ERR_ARG for a
 * bad demand or n, TC_ERR_STATE without a population, TC_ERR_UNSUPPORTED in
 * the one-hot form, for another problem, or for D max(demand) >= 2^24;
 * tc_set_params refuses to leave the dense forms or k-COL while demands are
 * set.  tc_best reports the best individual's colour of largest weight;
 * tc_best_multi its colour sets.  A failed allocation (TC_ERR_OOM) leaves
 * the context as it was; a CUDA error after that point (TC_ERR_CUDA) leaves
 * it to be re-initialised with tc_init_population. */
int tc_set_demands(tc_ctx *ctx, const int32_t *demand, int n);

/* Best-so-far individual of the multicolouring: colors[i * stride + q] for
 * q < demand[i] its colours of vertex i in increasing order, -1 up to
 * stride (>= the largest demand); *conflicts the colours shared across
 * edges; individual index and iteration as for tc_best.  Any output may be
 * NULL.  TC_ERR_STATE without demands set or before the first iteration. */
int tc_best_multi(tc_ctx *ctx, int32_t *colors, int stride, int64_t *conflicts, int32_t *individual,
                  int64_t *iteration);

/* The current colour sets of the whole population, colors[(d * n + i) *
 * stride + q] as in tc_best_multi (D * n * stride entries, caller-owned). */
int tc_get_multicolors(tc_ctx *ctx, int32_t *colors, int stride);

/* Pins the plan of the dense contractions: plan[0..7] as above (plan[7] = 1
 * needs one shape for both: 128-row units in clusters of 1, or 2 with
 * 256-wide tiles, or 256-row units on CTA pairs; the FP8 form only).  The FP8
 * form accepts, per contraction, unit rows 128 with column tile 128 / 256
 * and clusters sharing the B tile (Gamma: 1 / 2 / 4 dividing the 128-row
 * tiles; M~: 1, or 2 with 256-wide tiles), or unit rows 256 with column tile
 * 128 / 256 and cluster 2 (the pair); K splits 1 .. D k / 128.  The FP32
 * form takes only 128, 256, 1 for both and any K split.  TC_ERR_ARG for a
 * plan outside these, TC_ERR_STATE without a dense form.  Kept until the
 * next tc_init_population or form change, which tune again. */
int tc_dense_set_plan(tc_ctx *ctx, const int32_t *plan);

/* Batches: several independent instances (graphs of uneven n, their own k,
 * D, parameters and form), each a context with a population, stepped
 * together by one CUDA-graph launch per `chunk` iterations.  Algorithm 1
 * (Section 3.9) is run per instance exactly as tc_step runs it: every
 * instance keeps its own t, best-so-far and stop flag, and an instance that
 * has stopped on a legal colouring stays stopped while the others go on.  Inside the
 * graph each instance's iterations form one branch, so small instances run
 * side by side on the GPU.
 *
 * tc_batch_create: an empty batch on `device`.  TC_ERR_ARG for a bad device.
 * tc_batch_add: appends `ctx` (not owned; it must outlive the batch or be
 *   removed by destroying the batch).  The context must have a population
 *   and live on the batch's device, else TC_ERR_STATE / TC_ERR_ARG.  A
 *   context may belong to one batch at a time (TC_ERR_STATE otherwise).
 * tc_batch_step: `n_iters` iterations of every member; `chunk` > 0
 *   iterations are captured once into one graph (re-captured when a member's
 *   configuration changed) and replayed, the remainder launched directly.
 *   Returns once the work has completed, with the first member error (a
 *   bounded device wait that expired: TC_ERR_TIMEOUT).  Members must not be
 *   used concurrently by the caller during the call.
 * tc_batch_size: number of members.
 * tc_batch_destroy: releases the batch (not its members).  NULL is fine. */
typedef struct tc_batch tc_batch;
int tc_batch_create(tc_batch **out, int device);
int tc_batch_add(tc_batch *batch, tc_ctx *ctx);
int tc_batch_step(tc_batch *batch, int64_t n_iters, int chunk);
int tc_batch_size(tc_batch *batch, int *count);
int tc_batch_destroy(tc_batch *batch);

/* Name of a status code (static storage). */
const char *tc_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* TENSCOL_H */
