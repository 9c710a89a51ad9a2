// Internal declarations shared by the CUDA translation units of libtenscol.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tenscol.h"

// Device-resident iteration state.  Every field is written only by device
// code during an iteration; the host reads it after synchronising.
struct tc_dev_state {
    long long t;          // iteration counter of Algorithm 1
    long long evaluated;  // iterations whose Steps 1-2 ran (best-so-far checks)
    long long best_t;     // iteration at which the best-so-far was seen
    long long fcolor_sum; // sum_d f_color of the last evaluated iteration
    int stop;             // 1 once a legal individual is seen (stop_on_legal)
    int err;              // device error word (TC_ERR_* or 0)
    int best_f;           // best-so-far f (-1: none yet)
    int best_fcolor;
    int best_feq;
    int best_d;
    int last_fmin;
    int last_dstar;
    unsigned int done_gsum;     // completion ticket (last-block pattern) of k_gsum's blocks
    unsigned int done_spare;
    float loss, kappa, varpi;
    int best_pending;     // 1: the last evaluation improved the best-so-far, whose colours
                          // (individual last_dstar) k_update copies before it overwrites them
    long long trace_n;    // trace records written so far
};

// Problems whose Algorithm 1 uses J - M_d in place of M_d (Section 6), and
// those whose fitness includes f_eq (eq. 3).
__host__ __device__ inline bool tc_is_partition(int problem) {
    return problem == TC_KPART || problem == TC_KPART_BAL;
}
// Problems whose fitness adds a per-individual term: f_eq (eq. 3) for the ECP
// and the balanced partitioning, f_mscp for the minimum sum colouring.
__host__ __device__ inline bool tc_has_additive(int problem) {
    return problem == TC_ECP || problem == TC_KPART_BAL || problem == TC_MSCP;
}

// Everything a kernel of the step needs, passed by value.
struct tc_kparams {
    int n, D, k;
    int Dp;           // colours per row of cT (D rounded up to a multiple of 4)
    int ct_bytes;     // bytes per colour in cT: 1 when k <= 255, else 2
    int adj_words;    // 32-bit words per adjacency-bitmask row
    int problem, nb_iter, bonus_diag, stop_on_legal, commit;
    long long n_edges;  // |E| (the partitioning fitness is |E| - f_color)
    int csr_walk;     // grad_S L by adjacency lists (mu = 0, sparse graph)
    int max_degree;   // largest vertex degree (the staged adjacency walk's [degree][32] tiles)
    float eta, rho, lambda_, mu, nu, alpha, beta;
    float* W;                 // weights, tile-transposed (tc_w_index)
    uint16_t* c;              // D x n colours
    uint16_t* c_snap;         // D x n colours of the iteration, for the adjacency walk
    uint16_t* cT;             // n x Dp colours (vertex-major, ct_bytes each), pads all-ones
    uint32_t* planes;         // k <= 128, one colour per vertex: n x png x 8 bit-plane words, word
                              // p of group g of vertex i holding bit p of c_d(i) at bit d - 32 g
                              // (d in 32 g .. 32 g + 31; plane 7 and absent individuals 0)
    int png;                  // groups of 32 individuals, ceil(D / 32)
    const uint32_t* adj;      // n x adj_words adjacency bitmask
    const int* rowptr;        // CSR
    const int* colidx;
    float* B;                 // (n + 1) x ldb pair coefficients of eq. 13 (symmetric); row n = 0
    int ldb;                  // row stride of B: n rounded up to a multiple of 4
    // Per individual d, one record of rec_stride words at rec + d rec_stride
    // (tc_rec_* below): the vertices sorted by colour (stable; every class
    // padded to a multiple of 4 with vertex n), the padded class offsets, the
    // gradient factor of the additive fitness term by s_{d,i,j} (the equity
    // sign of eq. 14, or the colour cost z_j of the minimum sum colouring),
    // the classes by decreasing padded length (k_gsum's slot walk) and a chunk
    // of 4 padding vertices.  One record is one contiguous 16-byte-aligned copy.
    uint32_t* rec;
    int rec_stride;           // words per record
    int perm_stride;          // list entries per record: n + 3k (or the demands' sum + 3k) rounded to 8
    const int* zcost;         // k colour costs of the minimum sum colouring
    int* fcolor;              // D conflicts (eq. 1): k_gsum adds twice each, the reduction halves them
    int* feq;                 // D additive fitness: f_eq (eq. 3), or f_mscp (minimum sum colouring)
    float* loss_part;         // 2 x n_pair_blocks partial kappa / varpi
    int n_pair_blocks;
    const int2* pair_tiles;   // upper-triangular 32x32 tile list
    // tables over v = m~ in [0..D], with x = v for the colouring problems and
    // x = D - v (the entry of sum_d (J - M_d)) for the partitioning problems
    const float* lutA;        // 2 alpha x^(alpha-1)
    const float* lutB;        // 2 beta x^(beta-1)
    const float* powA;        // x^alpha
    const float* powB;        // x^beta
    tc_dev_state* st;
    uint16_t* best;           // n best-so-far colours
    // multicolouring (Section 6; dense forms only), NULL / 0 otherwise
    const int* dem;           // n demands c_i in [1, TC_MAX_DEMAND]
    uint16_t* cm;             // D x n x cmax colour sets, increasing, 0xFFFF past c_i
    uint16_t* best_m;         // n x cmax colour sets of the best-so-far individual
    int cmax;                 // largest demand
    int mt_max;               // largest value of m~: D, or D cmax in the multicolouring
    // iteration trace (NULL: off): ring of trace_cap records, one every trace_every t
    tc_trace_entry* trace;
    int trace_cap, trace_every;
    // dense forms (NULL in the one-hot form)
    float* M32;               // n_pad x n_pad group concentration from a GEMM (k_pairs zeroes it)
    int ldm;
    const uint16_t* G16;      // n_pad x ldg gamma matrix A.S_cat from a GEMM
    int ldg;
    uint8_t* S8;              // n_pad x ldg one-hot S_cat, FP8 E4M3 (1.0 = 0x38)
    uint8_t* S8T;             // ldg x n_pad its transpose
    int n_pad;
    int* dbg_Mt;              // optional n x n group concentration output
    float* dbg_G;             // optional D x n x k grad_S L output
    float* Gbuf;              // D x nT x k x 32 grad_S L tiles of the split update
    int* dbg_gamma;           // optional D x n conflicting-neighbour counts
    // failure handling: the limit of every bounded device wait (ns), and the
    // host-side fault injections that reach the device (TC_FAULT=wait: k_gsum
    // waits for an arrival that never comes; TC_FAULT=index, TC_BOUNDS builds
    // only: k_classes plants a vertex index past n that the checks must catch)
    unsigned long long wait_ns;
    int dbg_withhold, dbg_plant;
};

// Layout of an individual's record (words): the colour-sorted list
// [perm_stride], the k + 1 class offsets, the k additive-term factors, the k
// classes by decreasing padded length (uint16), 4 padding vertices.
__host__ __device__ inline int tc_off_words(int k) { return (k + 1 + 3) & ~3; }
__host__ __device__ inline int tc_e_words(int k) { return (k + 3) & ~3; }
__host__ __device__ inline int tc_cord_words(int k) { return ((k + 1) / 2 + 3) & ~3; }
__host__ __device__ inline int tc_rec_words(int perm_stride, int k) {
    return perm_stride + tc_off_words(k) + tc_e_words(k) + tc_cord_words(k) + 4;
}
__host__ __device__ inline int* tc_rec_off(uint32_t* r, int perm_stride) { return reinterpret_cast<int*>(r + perm_stride); }
__host__ __device__ inline float* tc_rec_E(uint32_t* r, int perm_stride, int k) {
    return reinterpret_cast<float*>(r + perm_stride + tc_off_words(k));
}
__host__ __device__ inline uint16_t* tc_rec_cord(uint32_t* r, int perm_stride, int k) {
    return reinterpret_cast<uint16_t*>(r + perm_stride + tc_off_words(k) + tc_e_words(k));
}
__host__ __device__ inline uint32_t* tc_rec_zchunk(uint32_t* r, int perm_stride, int k) {
    return r + perm_stride + tc_off_words(k) + tc_e_words(k) + tc_cord_words(k);
}

// The weight tensor W (D x n x k) is kept on the device tile-transposed:
// vertex tiles of 32 rows, each stored colour-major, so that a 32-row tile
// of one individual is one contiguous k x 32 block (one bulk copy) in which
// the 32 rows of one colour are one 128-byte line.  Rows n .. 32 nT - 1 of
// the last tile are padding (zero, never read).
constexpr int TC_WT = 32;
constexpr int TC_MAX_DEMAND = 8;  // colours a vertex may take in the multicolouring
__host__ __device__ inline size_t tc_w_index(int d, int i, int j, int nT, int k) {
    return (((size_t)d * nT + i / TC_WT) * k + j) * TC_WT + (i % TC_WT);
}
// The gamma matrix of the dense forms (Gamma_d[i][j] = #neighbours of i in
// colour j of individual d, uint16) is stored transposed, column-major over
// the padded rows: entry (d, i, j) at (d k + j) n_pad + i.  A run of 32 rows
// of one colour is one 64-byte line, and a 32-column x 128-row block of the
// GEMM output is one TMA box.
__host__ __device__ inline size_t tc_gamma_index(int d, int i, int j, int n_pad, int k) {
    return ((size_t)d * k + j) * (size_t)n_pad + (size_t)i;
}
// src (standard D x n x k) -> dst (tiled) when to_tiled, else back.
cudaError_t tc_launch_w_layout(const float* src, float* dst, int D, int n, int k, bool to_tiled,
                               cudaStream_t s);
// The same conversion by (individual, 32-row tile) blocks, whole lines on both
// sides (for host memory the device reads or writes directly);
// cudaErrorInvalidValue when a tile does not fit 48 KB of shared memory.
cudaError_t tc_launch_w_tiles(const float* src, float* dst, int D, int n, int k, bool to_tiled, cudaStream_t s);

// Programmatic dependent launch: a kernel launched with tc_launch_pdl may be
// scheduled while the previous kernel on the stream still runs; pdl_wait()
// returns once that kernel has completed and its writes are visible (without
// a programmatic dependency it returns at once).  pdl_trigger() lets the next
// kernel be scheduled early; it orders nothing by itself.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t tc_launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                          Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

// Population reduction of one iteration, run by the last block of k_gsum
// once every individual's conflicts (counted twice, over both ends of each
// edge) and additive term are in: min_d f(S_d) with the lowest d on ties (Algorithm 1 stop test),
// the best-so-far record, the loss of eq. 7, the stop flag and the trace.
// It sits between the last walk and k_update on the iteration's critical
// path, so every load it needs is issued at once (one memory round trip);
// the colours of an improved best are copied by k_update, which reads each
// row's colour before overwriting it (best_pending), except in the
// multicolouring, whose colour sets change in another kernel.  t is the
// iteration's counter, which the block read at its start.
// `scratch`: TC_FINALIZE_SCRATCH bytes of shared memory, 8-byte aligned; any
// block size up to 1024 threads (fixed-order sums: deterministic for a given
// block size).
constexpr int TC_FINALIZE_SCRATCH = 1296;
__device__ __forceinline__ void finalize_population(const tc_kparams& P, void* scratch, long long t) {
    // one pass: per-thread partials, warp trees, then warp 0 over the warps
    // (fixed order: deterministic for a given block size, at most 1024)
    long long* sh_fc = reinterpret_cast<long long*>(scratch);
    long long* sh_fe = sh_fc + 32;
    unsigned long long* sh_key = reinterpret_cast<unsigned long long*>(sh_fe + 32);
    unsigned long long* sh_ab = sh_key + 32;  // f_color, additive term of the key's individual
    float* sh_ka = reinterpret_cast<float*>(sh_ab + 32);
    float* sh_va = sh_ka + 32;
    int& s_dstar = *reinterpret_cast<int*>(sh_va + 32);
    int& s_better = *(reinterpret_cast<int*>(sh_va + 32) + 1);
    tc_dev_state* st = P.st;
    const int D = P.D, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    // the state thread 0 needs below, loaded with the per-individual values
    int prev_best = 0;
    long long trace_n = 0, evaluated = 0;
    if (threadIdx.x == 0) {
        prev_best = __ldcg(&st->best_f);
        trace_n = __ldcg(&st->trace_n);
        evaluated = __ldcg(&st->evaluated);
    }
    long long fc = 0, fe = 0;
    unsigned long long key = ~0ull, ab = 0ull;
    float ka = 0.f, va = 0.f;
    const bool part = tc_is_partition(P.problem), with_eq = tc_has_additive(P.problem);
    for (int d = threadIdx.x; d < D; d += blockDim.x) {
        // k_gsum summed gamma_d(i) over the vertices: each conflict twice
        const int a = __ldcg(P.fcolor + d) / 2, b = __ldcg(P.feq + d);
        P.fcolor[d] = a;
        fc += a;
        fe += b;
        // the fitness of the problem: monochromatic or (partitioning) cut edges,
        // plus f_eq for the ECP and the balanced partitioning, or f_mscp for
        // the minimum sum colouring
        const long long fobj = part ? P.n_edges - a : (long long)a;
        const unsigned long long f = (unsigned long long)(fobj + (with_eq ? b : 0));
        const unsigned long long kk = (f << 32) | (unsigned)d;
        if (kk < key) {
            key = kk;
            ab = ((unsigned long long)(unsigned)a << 32) | (unsigned)b;
        }
    }
    for (int b = threadIdx.x; b < P.n_pair_blocks; b += blockDim.x) {
        ka += __ldcg(P.loss_part + 2 * b);
        va += __ldcg(P.loss_part + 2 * b + 1);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        fc += __shfl_xor_sync(0xffffffffu, fc, o);
        fe += __shfl_xor_sync(0xffffffffu, fe, o);
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, key, o);
        const unsigned long long uab = __shfl_xor_sync(0xffffffffu, ab, o);
        if (u < key) {  // keys are distinct (they hold d)
            key = u;
            ab = uab;
        }
        ka += __shfl_xor_sync(0xffffffffu, ka, o);
        va += __shfl_xor_sync(0xffffffffu, va, o);
    }
    if (lane == 0) {
        sh_fc[warp] = fc;
        sh_fe[warp] = fe;
        sh_key[warp] = key;
        sh_ab[warp] = ab;
        sh_ka[warp] = ka;
        sh_va[warp] = va;
    }
    __syncthreads();
    if (warp == 0) {  // the warps' partials, by the same butterfly
        const bool in = lane < nw;
        fc = in ? sh_fc[lane] : 0;
        fe = in ? sh_fe[lane] : 0;
        key = in ? sh_key[lane] : ~0ull;
        ab = in ? sh_ab[lane] : 0ull;
        ka = in ? sh_ka[lane] : 0.f;
        va = in ? sh_va[lane] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            fc += __shfl_xor_sync(0xffffffffu, fc, o);
            fe += __shfl_xor_sync(0xffffffffu, fe, o);
            const unsigned long long u = __shfl_xor_sync(0xffffffffu, key, o);
            const unsigned long long uab = __shfl_xor_sync(0xffffffffu, ab, o);
            if (u < key) {
                key = u;
                ab = uab;
            }
            ka += __shfl_xor_sync(0xffffffffu, ka, o);
            va += __shfl_xor_sync(0xffffffffu, va, o);
        }
    }
    if (threadIdx.x == 0) {
        const int fmin = (int)(key >> 32), dstar = (int)(key & 0xffffffffu);
        const int fcol_star = (int)(ab >> 32), fadd_star = (int)(unsigned)(ab & 0xffffffffu);
        const double tt = (double)t;
        const long long fsum = part ? (long long)D * P.n_edges - fc : fc;  // the fitness term of eq. 7
        st->loss = (float)fsum + (float)((double)P.nu * tt) * (float)fe +
                   (float)((double)P.lambda_ * tt) * ka - (float)((double)P.mu * tt) * va;
        st->kappa = ka;
        st->varpi = va;
        st->fcolor_sum = fc;
        st->last_fmin = fmin;
        st->last_dstar = dstar;
        if (P.trace && P.commit && t % P.trace_every == 0) {  // the iteration trace
            tc_trace_entry e;
            e.t = t;
            e.f_min = fmin;
            e.individual = dstar;
            e.f_color = fcol_star;
            e.f_add = fadd_star;
            e.loss = st->loss;
            e.kappa = ka;
            e.varpi = va;
            e.pad = 0;
            P.trace[trace_n % P.trace_cap] = e;
            st->trace_n = trace_n + 1;
        }
        int better = 0;
        if (P.commit) {
            st->evaluated = evaluated + 1;
            if (prev_best < 0 || fmin < prev_best) {
                better = 1;
                st->best_f = fmin;
                st->best_fcolor = fcol_star;
                st->best_feq = fadd_star;
                st->best_d = dstar;
                st->best_t = t;
            }
            // the iteration ends here unless it stops before Step 3; its update
            // (k_update) reads the new counter
            if (P.stop_on_legal && fmin == 0)
                st->stop = 1;
            else
                st->t = t + 1;
        }
        // k_update copies the colours (one colour per vertex)
        st->best_pending = better && !P.cm;
        s_dstar = dstar;
        s_better = better && P.cm;
    }
    __syncthreads();
    if (s_better) {  // multicolouring: the colours and the colour sets here
        for (int i = threadIdx.x; i < P.n; i += blockDim.x)
            P.best[i] = P.c[(size_t)s_dstar * P.n + i];
        if (P.cm)
            for (size_t e = threadIdx.x; e < (size_t)P.n * P.cmax; e += blockDim.x)
                P.best_m[e] = P.cm[(size_t)s_dstar * P.n * P.cmax + e];
    }
    if (threadIdx.x == 0) st->done_gsum = 0u;
}


// Launchers (tc_onehot.cu).  All return cudaGetLastError() of the launch.
cudaError_t tc_launch_init_weights(float* W, int D, int n, int k, unsigned long long seed,
                                   float sigma0, cudaStream_t s);
cudaError_t tc_launch_assign(const tc_kparams& P, cudaStream_t s);
cudaError_t tc_launch_pairs(const tc_kparams& P, cudaStream_t s);
cudaError_t tc_launch_classes(const tc_kparams& P, cudaStream_t s);
// The class blocks and the pair blocks in one launch (one-hot form, one colour per vertex).
cudaError_t tc_launch_front(const tc_kparams& P, cudaStream_t s);
cudaError_t tc_launch_gsum(const tc_kparams& P, const CUtensorMap& tmB, int num_sms, cudaStream_t s);
cudaError_t tc_launch_update(const tc_kparams& P, int num_sms, cudaStream_t s, int debug_only);
// Tiled 2-D tensor map (TMA) over a row-major matrix: `inner` elements per
// row (contiguous), `outer` rows, `row_bytes` between rows (multiple of 16).
int tc_encode_tmap_2d(CUtensorMap* out, CUtensorMapDataType dt, void* base, uint64_t inner,
                      uint64_t outer, uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer,
                      CUtensorMapSwizzle swizzle);
constexpr int TC_BT_BOX_ROWS = 128;  // rows per TMA box of the B column panel
// Dense contractions (tc_dense.cu): C = X . Y^T over FP8 0/1 operands.
#define TC_GEMM_GAMMA 0  /* C uint16 transposed (tc_gamma_index); ldc = k, cols_alloc = D k */
#define TC_GEMM_MTILDE 1 /* C float, atomic adds (K may be split)       */
struct tc_gemm_args {
    const int4* units;  // (tile row, tile column, first K block, end K block); bit 30
                        // of the column marks a unit of the second contraction
    int n_units;
    int mode;
    void* C;
    int ldc;
    int rows_alloc, cols_alloc;
    int* err;
    // one launch for both contractions: the marked units use the second set
    // of tensor maps, this mode and column bound (fused = 0: no marked units)
    int fused, mode2, cols_alloc2;
};
constexpr int TC_UNIT_SECOND = 1 << 30;
// Shape of one contraction's work: rows of a unit (128 on one CTA, 256 on a
// CTA pair), column tile, CTAs per cluster (sharing the B tile, or the pair).
struct tc_gemm_shape {
    int tm = 128, bn = 256, cl = 1;
    bool operator==(const tc_gemm_shape& o) const { return tm == o.tm && bn == o.bn && cl == o.cl; }
};
int tc_gemm_tile_m();
int tc_gemm_tile_n();
int tc_gemm_tile_k();
cudaError_t tc_launch_gemm_tc(const CUtensorMap& tmX, const CUtensorMap& tmY, const CUtensorMap& tmC,
                              const tc_gemm_args& g, int slots, int tm, int cluster, int bn, bool pdl,
                              cudaStream_t s);
// Both contractions in one launch: the units marked TC_UNIT_SECOND use tmX2,
// tmY2, tmC2, g.mode2 and g.cols_alloc2 (g.fused = 1).
cudaError_t tc_launch_gemm_tc2(const CUtensorMap& tmX, const CUtensorMap& tmY, const CUtensorMap& tmC,
                               const CUtensorMap& tmX2, const CUtensorMap& tmY2, const CUtensorMap& tmC2,
                               const tc_gemm_args& g, int slots, int tm, int cluster, int bn, bool pdl,
                               cudaStream_t s);
int tc_gemm_cluster_slots(int tm, int cluster, int bn, int num_sms);
cudaError_t tc_launch_gemm_simt(const uint8_t* X, const uint8_t* Y, int ldk, const tc_gemm_args& g,
                                int num_sms, cudaStream_t s);
cudaError_t tc_launch_assign_multi(const tc_kparams& P, int clear_old, cudaStream_t s);
cudaError_t tc_launch_classes_multi(const tc_kparams& P, cudaStream_t s);
cudaError_t tc_launch_onehot_build(const tc_kparams& P, cudaStream_t s);

int tc_relaxed_run(const tc_kparams& P, const float* W, float tau, long long t, float* loss, float* gradW,
                   float* S, float* M, float* Bp, float* part, cudaStream_t s);
int tc_relaxed_partials(int n);

int tc_pair_tile_edge();
int tc_pair_tile_count(int n);
int tc_update_fits(int k);
