// Host engine of libtenscol: the C ABI of include/tenscol.h.
//
// One context = one graph + one population on one device.  Per iteration of
// Algorithm 1 the engine issues, on the context's stream,
//   memset(f_color) -> k_pairs -> k_classes -> k_update
// (see tc_onehot.cu).  The iteration counter, stop flag and best-so-far live
// in device memory, so any number of iterations can be queued (or captured
// in one CUDA graph) without a host round trip; the host polls the stop flag
// between chunks.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "tc_internal.cuh"

// NVTX ranges (header-only; inert unless a profiler is attached): one per
// iteration and one per kernel launch, named as the kernel timing names them
#include <nvtx3/nvToolsExt.h>

struct tc_batch;

struct tc_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t own = nullptr;
    cudaStream_t stream = nullptr;
    long long launches = 0;
    // graph
    int n = 0;
    long long nnz = 0;
    int max_degree = 0;      // largest vertex degree
    int* d_rowptr = nullptr;
    int* d_colidx = nullptr;
    uint32_t* d_adj = nullptr;
    int adj_words = 0;
    int2* d_tiles = nullptr;
    int n_tiles = 0;
    // population
    bool pop = false;
    int D = 0, k = 0, Dp = 0;
    tc_params p{};
    float* d_W = nullptr;
    uint16_t* d_c = nullptr;
    uint16_t* d_csnap = nullptr;
    uint32_t* d_planes = nullptr;  // bit planes of the colours (k <= 128; k_pairs' compares)
    uint16_t* d_cT = nullptr;
    float* d_B = nullptr;
    float* d_Gbuf = nullptr;  // grad_S L tiles between k_gsum and k_update
    uint32_t* d_rec = nullptr;  // per-individual records: class lists, offsets, additive terms, class order
    int* d_z = nullptr;         // k colour costs (minimum sum colouring), z_j = j + 1 unless set
    // multicolouring (tc_set_demands; dense forms): demands, colour sets
    int cmax = 0;                // largest demand; 0: one colour per vertex
    long long dem_sum = 0;       // sum of the demands
    int* d_dem = nullptr;
    uint16_t* d_cm = nullptr;
    uint16_t* d_best_m = nullptr;
    // iteration trace (tc_set_trace)
    tc_trace_entry* d_trace = nullptr;
    int trace_cap = 0, trace_every = 1;
    int* d_fcolor = nullptr;
    int* d_feq = nullptr;
    float* d_loss_part = nullptr;
    float* d_lut = nullptr;  // 4 x (D + 1): lutA, lutB, powA, powB
    tc_dev_state* d_st = nullptr;
    uint16_t* d_best = nullptr;
    int ldb = 0;
    alignas(64) CUtensorMap tmB;  // B column panels for k_update
    // dense forms: FP8 operands, GEMM outputs, tensor maps, work units
    std::vector<int> h_rowptr, h_colidx;
    int n_pad = 0, ldg = 0;
    uint8_t* d_A8 = nullptr;
    uint8_t* d_S8 = nullptr;
    uint8_t* d_S8T = nullptr;
    uint16_t* d_G16 = nullptr;
    float* d_M32 = nullptr;
    int4* d_units_g = nullptr;
    int4* d_units_m = nullptr;
    int n_units_g = 0, n_units_m = 0;
    tc_gemm_shape sh_g, sh_m;    // tiles and clusters of the two contractions (Gamma, M~)
    bool fused = false;          // both contractions in one launch (same shape; M~ units first)
    int4* d_units_f = nullptr;
    int n_units_f = 0;
    int split_m = 1;             // K splits of M~
    int slots_g = 0, slots_m = 0;  // clusters of those sizes resident at once
    int tune_candidates = 0;       // configurations timed by the autotuner
    float tune_us_g = 0.f, tune_us_m = 0.f;  // their best times
    float tune_us_f = 0.f;                   // best time of one launch for both (0: none timed)
    alignas(64) CUtensorMap tmA8;
    alignas(64) CUtensorMap tmS8T;
    alignas(64) CUtensorMap tmS8x;
    alignas(64) CUtensorMap tmS8y;
    alignas(64) CUtensorMap tmG16;  // output of Gamma (TMA store)
    alignas(64) CUtensorMap tmM32;  // output of M~ (TMA reduce-add)
    // CUDA graph of graph_chunk iterations
    int graph_chunk = 0;
    cudaGraphExec_t gexec = nullptr;
    long long gen = 0;          // bumped whenever captured work would go stale
    tc_batch* batch = nullptr;  // the batch this context belongs to, if any
    unsigned long long wait_ns = 1000000000ull;  // limit of every bounded device wait (tc_set_wait_limit)
    // per-kernel event timing
    int timing = 0;
    bool capturing = false;
    struct Timed {
        int kid;
        cudaEvent_t a, b;
    };
    std::vector<Timed> pending;
    std::vector<cudaEvent_t> spare;
    double kms[TC_NUM_KID] = {0};
    long long kcount[TC_NUM_KID] = {0};
};

namespace {

bool fault(const char* where) {
    const char* f = getenv("TC_FAULT");
    return f && strcmp(f, where) == 0;
}

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return TC_OK;
    if (e == cudaErrorMemoryAllocation) return TC_ERR_OOM;
    return TC_ERR_CUDA;
}

#define TC_CHECK(expr)                          \
    do {                                        \
        cudaError_t _e = (expr);                \
        if (_e != cudaSuccess) {                \
            (void)cudaGetLastError();           \
            return cuda_status(_e);             \
        }                                       \
    } while (0)

template <typename T>
int dalloc(T** p, size_t count) {
    *p = nullptr;
    if (fault("alloc")) return TC_ERR_INJECTED;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        *p = nullptr;
        return TC_ERR_OOM;
    }
    return TC_OK;
}

template <typename T>
void dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

void drop_graph_exec(tc_ctx* c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    c->gen += 1;  // batches holding this context re-capture
}

void free_dense(tc_ctx* c) {
    dfree(c->d_A8);
    dfree(c->d_S8);
    dfree(c->d_S8T);
    dfree(c->d_G16);
    dfree(c->d_M32);
    dfree(c->d_units_g);
    dfree(c->d_units_m);
    dfree(c->d_units_f);
    c->n_units_g = c->n_units_m = c->n_units_f = 0;
    c->fused = false;
    c->n_pad = c->ldg = 0;
}

void free_population(tc_ctx* c) {
    drop_graph_exec(c);
    free_dense(c);
    dfree(c->d_W);
    dfree(c->d_c);
    dfree(c->d_csnap);
    dfree(c->d_planes);
    dfree(c->d_cT);
    dfree(c->d_B);
    dfree(c->d_Gbuf);
    dfree(c->d_rec);
    dfree(c->d_z);
    dfree(c->d_fcolor);
    dfree(c->d_feq);
    dfree(c->d_loss_part);
    dfree(c->d_lut);
    dfree(c->d_st);
    dfree(c->d_best);
    dfree(c->d_dem);
    dfree(c->d_cm);
    dfree(c->d_best_m);
    dfree(c->d_trace);
    c->trace_cap = 0;
    c->cmax = 0;
    c->dem_sum = 0;
    c->pop = false;
    c->D = c->k = c->Dp = 0;
}

void free_graph(tc_ctx* c) {
    free_population(c);
    dfree(c->d_rowptr);
    dfree(c->d_colidx);
    dfree(c->d_adj);
    dfree(c->d_tiles);
    c->n = 0;
    c->nnz = 0;
}

int check_params(const tc_params* p) {
    if (p->problem < TC_KCOL || p->problem > TC_MSCP) return TC_ERR_ARG;
    if (!(p->eta >= 0.f) || !(p->rho >= 1.f) || p->nb_iter < 1) return TC_ERR_ARG;
    if (!(p->alpha > 1.f) || !(p->beta > 1.f)) return TC_ERR_ARG;
    if (!(p->lambda_ >= 0.f) || !(p->mu >= 0.f) || !(p->nu >= 0.f) || !(p->sigma0 >= 0.f))
        return TC_ERR_ARG;
    if (p->form != TC_FORM_ONEHOT && p->form != TC_FORM_DENSE_FP8 && p->form != TC_FORM_DENSE_FP32)
        return TC_ERR_UNSUPPORTED;
    return TC_OK;
}

// Entries per individual of the colour-class lists (each vertex once per
// colour it takes, each class padded to a multiple of 4) and the largest
// value of m~ (the tables of k_pairs hold that many + 1 entries).
int perm_stride_for(int n, int k, int cmax, long long dem_sum) {
    const long long entries = cmax > 0 ? dem_sum : n;
    return (int)((entries + 3ll * k + 7) & ~7ll);
}
int mt_max_for(int D, int cmax) { return D * (cmax > 0 ? cmax : 1); }
int perm_stride(const tc_ctx* c) { return perm_stride_for(c->n, c->k, c->cmax, c->dem_sum); }
int rec_stride_for(int n, int k, int cmax, long long dem_sum) {
    return tc_rec_words(perm_stride_for(n, k, cmax, dem_sum), k);
}
int mt_max(const tc_ctx* c) { return mt_max_for(c->D, c->cmax); }

tc_kparams make_kparams(tc_ctx* c, int commit) {
    tc_kparams P;
    memset(&P, 0, sizeof(P));
    P.n = c->n;
    P.D = c->D;
    P.k = c->k;
    P.Dp = c->Dp;
    P.ct_bytes = c->k <= 255 ? 1 : 2;
    P.adj_words = c->adj_words;
    P.problem = c->p.problem;
    P.n_edges = c->nnz / 2;
    P.nb_iter = c->p.nb_iter;
    P.bonus_diag = c->p.bonus_diag;
    P.stop_on_legal = c->p.stop_on_legal;
    P.commit = commit;
    P.eta = c->p.eta;
    P.rho = c->p.rho;
    P.lambda_ = c->p.lambda_;
    P.mu = c->p.mu;
    P.nu = c->p.nu;
    P.alpha = c->p.alpha;
    P.beta = c->p.beta;
    P.W = c->d_W;
    P.c = c->d_c;
    P.c_snap = c->d_csnap;
    P.cT = c->d_cT;
    // the bit planes are kept with every colour store while k <= 128 and one
    // colour per vertex; the colour assignment rebuilds them
    P.png = (c->D + 31) / 32;
    P.planes = c->k <= 128 && c->cmax == 0 ? c->d_planes : nullptr;
    P.adj = c->d_adj;
    P.rowptr = c->d_rowptr;
    P.colidx = c->d_colidx;
    P.B = c->d_B;
    P.Gbuf = c->d_Gbuf;
    P.ldb = c->ldb;
    P.rec = c->d_rec;
    P.perm_stride = perm_stride(c);
    P.rec_stride = tc_rec_words(P.perm_stride, c->k);
    P.zcost = c->d_z;
    P.fcolor = c->d_fcolor;
    P.feq = c->d_feq;
    P.loss_part = c->d_loss_part;
    P.n_pair_blocks = c->n_tiles;
    P.pair_tiles = c->d_tiles;
    P.mt_max = mt_max(c);
    const int D1 = P.mt_max + 1;
    P.lutA = c->d_lut;
    P.lutB = c->d_lut + D1;
    P.powA = c->d_lut + 2 * D1;
    P.powB = c->d_lut + 3 * D1;
    P.st = c->d_st;
    P.best = c->d_best;
    P.wait_ns = c->wait_ns;
    P.dbg_withhold = fault("wait") ? 1 : 0;
    P.dbg_plant = fault("index") ? 1 : 0;
    // with mu = 0 the pair matrix vanishes off the edges; below a density of
    // 1/8 walking the adjacency lists beats walking all n vertices per class
    P.csr_walk = c->p.mu == 0.0f && c->nnz * 8 < (long long)c->n * c->n && c->cmax == 0;
    P.max_degree = c->max_degree;
    if (c->trace_cap > 0) {
        P.trace = c->d_trace;
        P.trace_cap = c->trace_cap;
        P.trace_every = c->trace_every;
    }
    if (c->cmax > 0) {  // multicolouring
        P.dem = c->d_dem;
        P.cm = c->d_cm;
        P.best_m = c->d_best_m;
        P.cmax = c->cmax;
    }
    if (c->p.form != TC_FORM_ONEHOT && c->d_M32) {
        P.M32 = c->d_M32;
        P.ldm = c->n_pad;
        P.G16 = c->d_G16;
        P.ldg = c->ldg;
        P.S8 = c->d_S8;
        P.S8T = c->d_S8T;
        P.n_pad = c->n_pad;
    }
    return P;
}

// Work units of Gamma = A . S_cat: every (row tile, column tile), row tiles
// fastest so that `cl` consecutive units share the column tile.
std::vector<int4> units_gamma(int mt, int nt, int kblocks) {
    std::vector<int4> u;
    for (int bn = 0; bn < nt; ++bn)
        for (int bm = 0; bm < mt; ++bm) u.push_back(make_int4(bm, bn, 0, kblocks));
    return u;
}

// Work units of M~ = S_cat . S_cat^T: the (row, column) tiles of tm x bn
// touching the upper triangle, each K range split `split` ways (partial sums
// added in L2 by the TMA reduce).  With tm = 128 and bn = 256 every column
// holds an even number of such row tiles, so row pairs share the column tile
// (clusters of 2).
std::vector<int4> units_mtilde(int mt, int tm, int bn, int ntm, int kblocks, int split) {
    std::vector<int2> tri;
    for (int c = 0; c < ntm; ++c)
        for (int bm = 0; bm < mt; ++bm)
            if ((long long)c * bn + bn - 1 >= (long long)bm * tm) tri.push_back(make_int2(bm, c));
    std::vector<int4> u;
    for (int sidx = 0; sidx < split; ++sidx)
        for (auto& tt : tri) {
            const int k0 = (int)((long long)kblocks * sidx / split), k1 = (int)((long long)kblocks * (sidx + 1) / split);
            if (k1 > k0) u.push_back(make_int4(tt.x, tt.y, k0, k1));
        }
    return u;
}

int upload_units(tc_ctx* c, int4* dst, const std::vector<int4>& u) {
    TC_CHECK(cudaMemcpyAsync(dst, u.data(), u.size() * sizeof(int4), cudaMemcpyHostToDevice, c->stream));
    return TC_OK;
}

// Whether a plan suits the context's dense form and sizes.
bool shape_valid(const tc_ctx* c, const tc_gemm_shape& q, bool mtilde) {
    const int BMt = tc_gemm_tile_m();
    if (q.bn != 128 && q.bn != 256) return false;
    if (q.tm == 2 * BMt) return q.cl == 2 && c->n_pad % q.tm == 0;  // a CTA pair per unit
    if (q.tm != BMt) return false;
    if (mtilde) return q.cl == 1 || (q.cl == 2 && q.bn == 256);
    return (q.cl == 1 || q.cl == 2 || q.cl == 4) && (c->n_pad / BMt) % q.cl == 0;
}

bool plan_valid(const tc_ctx* c, const tc_gemm_shape& g, const tc_gemm_shape& m, int split) {
    const int km = c->ldg / tc_gemm_tile_k();
    if (split < 1 || split > km) return false;
    if (c->p.form == TC_FORM_DENSE_FP32) {  // the CUDA-core comparator: 128 x 256 tiles
        const tc_gemm_shape f;
        return g == f && m == f;
    }
    return shape_valid(c, g, false) && shape_valid(c, m, true);
}

// Box rows of the B operand each CTA loads: its slice of the shared tile
// (cluster multicast) or its half of the pair's tile.
int b_box_rows(const tc_gemm_shape& q) { return q.tm == 2 * tc_gemm_tile_m() ? q.bn / 2 : q.bn / q.cl; }

std::vector<int4> plan_units_gamma(const tc_ctx* c, const tc_gemm_shape& q) {
    return units_gamma(c->n_pad / q.tm, (int)(c->ldg / q.bn), c->n_pad / tc_gemm_tile_k());
}

std::vector<int4> plan_units_mtilde(const tc_ctx* c, const tc_gemm_shape& q, int kblocks, int split) {
    return units_mtilde(c->n_pad / q.tm, q.tm, q.bn, c->n_pad / q.bn, kblocks, split);
}

// The unit list of one launch for both contractions: the M~ units (long K
// ranges) first, then the Gamma units marked as the second contraction; the
// persistent CTAs take units round robin, so the long ones start first.
std::vector<int4> plan_units_fused(const tc_ctx* c, const tc_gemm_shape& q, int split) {
    std::vector<int4> u = plan_units_mtilde(c, q, (int)(c->ldg / tc_gemm_tile_k()), split);
    for (int4 w : plan_units_gamma(c, q)) {
        w.y |= TC_UNIT_SECOND;
        u.push_back(w);
    }
    return u;
}

// Whether both contractions can share a launch: one shape for both, either
// 128-row units in clusters of 1 or 2 (a cluster's units must share the
// column tile in both lists: the M~ list comes in such pairs when bn = 2 x
// 128) or 256-row units on CTA pairs (a unit per pair).
bool fusable(const tc_ctx* c, const tc_gemm_shape& g, const tc_gemm_shape& m) {
    if (c->p.form != TC_FORM_DENSE_FP8 || !(g == m)) return false;
    if (g.tm == 2 * tc_gemm_tile_m()) return g.cl == 2;
    return g.tm == tc_gemm_tile_m() && (g.cl == 1 || (g.cl == 2 && g.bn == 256));
}

// Makes a plan current: unit lists, the B operands' tensor maps, resident
// cluster counts.
int apply_plan(tc_ctx* c, const tc_gemm_shape& sg, const tc_gemm_shape& sm, int split, bool fused) {
    if (fused && !fusable(c, sg, sm)) return TC_ERR_ARG;
    const int BKt = tc_gemm_tile_k();
    const int n_pad = c->n_pad;
    const long long ldg = c->ldg;
    const CUtensorMapDataType u8 = CU_TENSOR_MAP_DATA_TYPE_UINT8;
    const CUtensorMapSwizzle sw = CU_TENSOR_MAP_SWIZZLE_128B;
    const std::vector<int4> ug = plan_units_gamma(c, sg);
    const std::vector<int4> um = plan_units_mtilde(c, sm, (int)(ldg / BKt), split);
    int rc;
    if ((rc = upload_units(c, c->d_units_g, ug)) || (rc = upload_units(c, c->d_units_m, um))) return rc;
    if ((rc = tc_encode_tmap_2d(&c->tmS8T, u8, c->d_S8T, n_pad, ldg, n_pad, BKt, b_box_rows(sg), sw)) ||
        (rc = tc_encode_tmap_2d(&c->tmS8y, u8, c->d_S8, ldg, n_pad, ldg, BKt, b_box_rows(sm), sw)))
        return rc;
    c->n_units_g = (int)ug.size();
    c->n_units_m = (int)um.size();
    c->fused = fused;
    c->n_units_f = 0;
    if (fused) {
        const std::vector<int4> uf = plan_units_fused(c, sg, split);
        if ((rc = upload_units(c, c->d_units_f, uf))) return rc;
        c->n_units_f = (int)uf.size();
    }
    c->sh_g = sg;
    c->sh_m = sm;
    c->split_m = split;
    c->slots_g = tc_gemm_cluster_slots(sg.tm, sg.cl, sg.bn, c->num_sms);
    c->slots_m = tc_gemm_cluster_slots(sm.tm, sm.cl, sm.bn, c->num_sms);
    TC_CHECK(cudaStreamSynchronize(c->stream));
    return TC_OK;
}

// Autotuner of the FP8 tensor-core contractions: times every candidate
// (128-row units on one CTA with column tile 128 or 256 and clusters
// sharing the B tile, or 256-row units on a CTA pair; K splits of M~) on the
// context's own operands, one warm-up and three timed launches each, and
// keeps the fastest (the shapes differ from instance to instance).  The FP32
// comparator keeps the 128 x 256 tiles.
int plan_dense(tc_ctx* c) {
    const int BMt = tc_gemm_tile_m(), BKt = tc_gemm_tile_k();
    const int n_pad = c->n_pad;
    const long long ldg = c->ldg;
    const int km = (int)(ldg / BKt);
    const CUtensorMapDataType u8 = CU_TENSOR_MAP_DATA_TYPE_UINT8;
    const CUtensorMapSwizzle sw = CU_TENSOR_MAP_SWIZZLE_128B;
    int rc;
    if ((rc = tc_encode_tmap_2d(&c->tmA8, u8, c->d_A8, n_pad, n_pad, n_pad, BKt, BMt, sw)) ||
        (rc = tc_encode_tmap_2d(&c->tmS8x, u8, c->d_S8, ldg, n_pad, ldg, BKt, BMt, sw)) ||
        // outputs: Gamma transposed [D k][n_pad] uint16 and M~ [n_pad][n_pad]
        // f32 (128-byte swizzled), each in boxes of 32 rows x 32 columns
        (rc = tc_encode_tmap_2d(&c->tmG16, CU_TENSOR_MAP_DATA_TYPE_UINT16, c->d_G16, n_pad,
                                (uint64_t)c->D * c->k, 2ull * n_pad, 32, 32, CU_TENSOR_MAP_SWIZZLE_NONE)) ||
        (rc = tc_encode_tmap_2d(&c->tmM32, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, c->d_M32, n_pad, n_pad, 4ull * n_pad, 32,
                                32, sw)))
        return rc;
    // CTAs resident at once for a shape, and the triangle's tile count
    auto ctas = [&](const tc_gemm_shape& q) { return tc_gemm_cluster_slots(q.tm, q.cl, q.bn, c->num_sms) * q.cl; };
    auto tri_tiles = [&](const tc_gemm_shape& q) { return (int)plan_units_mtilde(c, q, 1, 1).size(); };
    struct Cand {
        tc_gemm_shape q;
        int split;
    };
    std::vector<Cand> cg, cm;
    const bool tc = c->p.form == TC_FORM_DENSE_FP8;
    if (tc) {
        std::vector<tc_gemm_shape> shapes;
        for (int bn : {256, 128}) {
            for (int cl : {1, 2, 4}) shapes.push_back({BMt, bn, cl});
            shapes.push_back({2 * BMt, bn, 2});
        }
        for (const tc_gemm_shape& q : shapes)
            if (shape_valid(c, q, false)) cg.push_back({q, 1});
        for (const tc_gemm_shape& q : shapes) {
            if (!shape_valid(c, q, true)) continue;
            // splits around the one that fills the resident CTAs: those that
            // give one or two full waves of units, and fewer (less reduction)
            const int slots = ctas(q) / (q.tm == 2 * BMt ? 2 : 1), tri = tri_tiles(q);
            std::vector<int> sps = {slots / tri, 2 * slots / tri, (slots + tri - 1) / tri, slots / tri / 2};
            for (int& sp : sps) sp = std::max(1, std::min(sp, km));  // 1 .. K blocks
            std::sort(sps.begin(), sps.end());
            sps.erase(std::unique(sps.begin(), sps.end()), sps.end());
            for (int sp : sps) cm.push_back({q, sp});
        }
        if (cg.empty() || cm.empty()) return TC_ERR_UNSUPPORTED;  // no shape fits (n_pad is a multiple of 256)
    } else {
        const tc_gemm_shape f;
        cg.push_back({f, 1});
        cm.push_back({f, std::max(1, std::min((c->num_sms + tri_tiles(f) - 1) / tri_tiles(f), km))});
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    TC_CHECK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        (void)cudaGetLastError();
        return TC_ERR_CUDA;
    }
    // time one candidate: 1 warm-up + 3 launches, the fastest (ms), or a
    // negative value when the launch configuration is refused
    auto time_it = [&](auto launch) -> float {
        if (launch() != cudaSuccess) {
            (void)cudaGetLastError();
            return -1.f;
        }
        float best = 1e30f;
        for (int r = 0; r < 3; ++r) {
            float ms = 0.f;
            if (cudaEventRecord(e0, c->stream) != cudaSuccess || launch() != cudaSuccess ||
                cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                (void)cudaGetLastError();
                return -1.f;
            }
            best = std::min(best, ms);
        }
        return best;
    };
    float best_g = 1e30f, best_m = 1e30f;
    Cand pick_g = cg[0], pick_m = cm[0];
    int timed = 0;
    rc = TC_OK;
    for (const Cand& q : cg) {
        if (!tc) break;
        const std::vector<int4> u = plan_units_gamma(c, q.q);
        CUtensorMap tmY;
        const int slots = tc_gemm_cluster_slots(q.q.tm, q.q.cl, q.q.bn, c->num_sms);
        if ((rc = tc_encode_tmap_2d(&tmY, u8, c->d_S8T, n_pad, ldg, n_pad, BKt, b_box_rows(q.q), sw)) ||
            (rc = upload_units(c, c->d_units_g, u)))
            break;
        tc_gemm_args g = {c->d_units_g, (int)u.size(), TC_GEMM_GAMMA, c->d_G16, c->k, c->n_pad, c->D * c->k,
                          &c->d_st->err};
        const float ms = time_it(
            [&] { return tc_launch_gemm_tc(c->tmA8, tmY, c->tmG16, g, slots, q.q.tm, q.q.cl, q.q.bn, false, c->stream); });
        ++timed;
        if (ms >= 0.f && ms < best_g) {
            best_g = ms;
            pick_g = q;
        }
    }
    for (const Cand& q : cm) {
        if (!tc || rc) break;
        const std::vector<int4> u = plan_units_mtilde(c, q.q, km, q.split);
        CUtensorMap tmY;
        const int slots = tc_gemm_cluster_slots(q.q.tm, q.q.cl, q.q.bn, c->num_sms);
        if ((rc = tc_encode_tmap_2d(&tmY, u8, c->d_S8, ldg, n_pad, ldg, BKt, b_box_rows(q.q), sw)) ||
            (rc = upload_units(c, c->d_units_m, u)))
            break;
        tc_gemm_args g = {c->d_units_m, (int)u.size(), TC_GEMM_MTILDE, c->d_M32, c->n_pad, c->n_pad, c->n_pad,
                          &c->d_st->err};
        const float ms = time_it(
            [&] { return tc_launch_gemm_tc(c->tmS8x, tmY, c->tmM32, g, slots, q.q.tm, q.q.cl, q.q.bn, false, c->stream); });
        ++timed;
        if (ms >= 0.f && ms < best_m) {
            best_m = ms;
            pick_m = q;
        }
    }
    // one launch for both contractions (M~ units first, then Gamma's): every
    // M~ candidate whose shape both can share, kept if it beats the two
    // best separate launches together
    float best_f = 1e30f;
    Cand pick_f = pick_m;
    for (const Cand& q : cm) {
        if (!tc || rc) break;
        if (!fusable(c, q.q, q.q)) continue;
        const std::vector<int4> u = plan_units_fused(c, q.q, q.split);
        CUtensorMap tmYm, tmYg;
        const int slots = tc_gemm_cluster_slots(q.q.tm, q.q.cl, q.q.bn, c->num_sms);
        if ((rc = tc_encode_tmap_2d(&tmYm, u8, c->d_S8, ldg, n_pad, ldg, BKt, b_box_rows(q.q), sw)) ||
            (rc = tc_encode_tmap_2d(&tmYg, u8, c->d_S8T, n_pad, ldg, n_pad, BKt, b_box_rows(q.q), sw)) ||
            (rc = upload_units(c, c->d_units_f, u)))
            break;
        tc_gemm_args g = {c->d_units_f, (int)u.size(), TC_GEMM_MTILDE, c->d_M32, c->n_pad, c->n_pad, c->n_pad,
                          &c->d_st->err, 1, TC_GEMM_GAMMA, c->D * c->k};
        const float ms = time_it([&] {
            return tc_launch_gemm_tc2(c->tmS8x, tmYm, c->tmM32, c->tmA8, tmYg, c->tmG16, g, slots, q.q.tm, q.q.cl,
                                      q.q.bn, false, c->stream);
        });
        ++timed;
        if (ms >= 0.f && ms < best_f) {
            best_f = ms;
            pick_f = q;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (tc && (best_g >= 1e30f || best_m >= 1e30f)) return TC_ERR_CUDA;  // no configuration ran
    // the timed M~ launches left sums behind; the iteration expects zeros
    // (k_pairs zeroes M~ after reading it)
    TC_CHECK(cudaMemsetAsync(c->d_M32, 0, sizeof(float) * (size_t)n_pad * n_pad, c->stream));
    const bool fuse = tc && best_f < best_g + best_m;
    if ((rc = fuse ? apply_plan(c, pick_f.q, pick_f.q, pick_f.split, true)
                   : apply_plan(c, pick_g.q, pick_m.q, pick_m.split, false)))
        return rc;
    c->tune_candidates = timed;
    c->tune_us_g = tc ? 1e3f * best_g : 0.f;
    c->tune_us_m = tc ? 1e3f * best_m : 0.f;
    c->tune_us_f = tc && best_f < 1e30f ? 1e3f * best_f : 0.f;
    return TC_OK;
}

// Dense forms: FP8 adjacency, one-hot operands, GEMM outputs, then the plan
// of the two contractions (plan_dense).  n_pad is a multiple of every GEMM
// tile edge, ldg (the padded D k) a multiple of the widest column tile.
int setup_dense(tc_ctx* c) {
    free_dense(c);
    const int BMt = tc_gemm_tile_m(), BNt = tc_gemm_tile_n();
    const int n = c->n;
    const int n_pad = (n + BNt - 1) / BNt * BNt;
    const long long Kc = (long long)c->D * c->k;
    const long long ldg = (Kc + BNt - 1) / BNt * BNt;
    if (ldg > (1ll << 31) / 4) return TC_ERR_UNSUPPORTED;
    // unit lists sized for the most units any valid plan uses (128-wide
    // tiles, M~ split to single K blocks)
    const int mt = n_pad / BMt;
    const size_t max_ug = (size_t)mt * (size_t)(ldg / 128);
    const size_t max_um = (size_t)mt * (size_t)(n_pad / 128) * (size_t)(ldg / tc_gemm_tile_k());
    int rc;
    if ((rc = dalloc(&c->d_A8, (size_t)n_pad * n_pad)) || (rc = dalloc(&c->d_S8, (size_t)n_pad * ldg)) ||
        (rc = dalloc(&c->d_S8T, (size_t)ldg * n_pad)) || (rc = dalloc(&c->d_G16, (size_t)n_pad * ldg)) ||
        (rc = dalloc(&c->d_M32, (size_t)n_pad * n_pad)) || (rc = dalloc(&c->d_units_g, max_ug)) ||
        (rc = dalloc(&c->d_units_m, max_um)) || (rc = dalloc(&c->d_units_f, max_ug + max_um))) {
        free_dense(c);
        return rc;
    }
    c->n_pad = n_pad;
    c->ldg = (int)ldg;
    std::vector<uint8_t> a8((size_t)n_pad * n_pad, 0);
    for (int i = 0; i < n; ++i)
        for (int e = c->h_rowptr[i]; e < c->h_rowptr[i + 1]; ++e) a8[(size_t)i * n_pad + c->h_colidx[e]] = 0x38;
    cudaError_t e = cudaMemcpyAsync(c->d_A8, a8.data(), a8.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        free_dense(c);
        return cuda_status(e);
    }
    if ((rc = plan_dense(c))) {
        (void)cudaGetLastError();
        free_dense(c);
        return rc;
    }
    return TC_OK;
}


// Rebuilds the FP8 one-hot operands from the current colours.
cudaError_t rebuild_onehot(tc_ctx* c) {
    if (!c->d_S8) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(c->d_S8, 0, (size_t)c->n_pad * c->ldg, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_S8T, 0, (size_t)c->ldg * c->n_pad, c->stream);
    if (e == cudaSuccess)  // multicolouring: the colour sets of Step 1 from W (they replace c)
        e = c->cmax > 0 ? tc_launch_assign_multi(make_kparams(c, 0), 0, c->stream)
                        : tc_launch_onehot_build(make_kparams(c, 0), c->stream);
    c->launches += 1;
    return e;
}

// The LUTs of the pair terms over the integer values v = 0..D of m~ (eq. 5,
// 6, 13), computed once in double precision on the host.
int upload_luts(tc_ctx* c) {
    const int D1 = mt_max(c) + 1;
    std::vector<float> h(4 * (size_t)D1);
    const double a = c->p.alpha, b = c->p.beta;
    const bool part = tc_is_partition(c->p.problem);
    for (int v = 0; v < D1; ++v) {
        // v = m~; the partitioning problems weigh sum_d (J - M_d) = D - m~
        const double x = part ? (double)(c->D - v) : (double)v;
        h[v] = (float)(2.0 * a * pow(x, a - 1.0));
        h[D1 + v] = (float)(2.0 * b * pow(x, b - 1.0));
        h[2 * D1 + v] = (float)pow(x, a);
        h[3 * D1 + v] = (float)pow(x, b);
    }
    if (fault("copy")) return TC_ERR_INJECTED;
    TC_CHECK(cudaMemcpyAsync(c->d_lut, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice,
                             c->stream));
    TC_CHECK(cudaStreamSynchronize(c->stream));
    return TC_OK;
}

cudaEvent_t take_event(tc_ctx* c) {
    if (!c->spare.empty()) {
        cudaEvent_t e = c->spare.back();
        c->spare.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return e;
}

const char* kernel_name(int kid) {
    static const char* names[TC_NUM_KID] = {"k_pairs", "k_classes", "k_update", "gemm_mtilde",
                                            "gemm_gamma", "k_gsum", "gemm_fused", "k_front"};
    return kid >= 0 && kid < TC_NUM_KID && names[kid] ? names[kid] : "kernel";
}

// Launches one kernel through `fn`, bracketed by timing events when enabled
// and by an NVTX range.
template <typename F>
cudaError_t timed(tc_ctx* c, int kid, F fn, cudaStream_t s = nullptr) {
    if (!s) s = c->stream;
    const bool on = c->timing && !c->capturing;
    cudaEvent_t a = on ? take_event(c) : nullptr;
    cudaEvent_t b = on ? take_event(c) : nullptr;
    if (a && b) cudaEventRecord(a, s);
    nvtxRangePushA(kernel_name(kid));
    cudaError_t e = fn();
    nvtxRangePop();
    if (a && b) {
        cudaEventRecord(b, s);
        c->pending.push_back({kid, a, b});
    } else {
        if (a) c->spare.push_back(a);
        if (b) c->spare.push_back(b);
    }
    c->launches += 1;
    return e;
}

int collect_timing(tc_ctx* c) {
    if (c->pending.empty()) return TC_OK;
    TC_CHECK(cudaStreamSynchronize(c->stream));
    for (auto& t : c->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
            c->kms[t.kid] += ms;
            c->kcount[t.kid] += 1;
        } else {
            (void)cudaGetLastError();
        }
        c->spare.push_back(t.a);
        c->spare.push_back(t.b);
    }
    c->pending.clear();
    return TC_OK;
}

void free_events(tc_ctx* c) {
    for (auto& t : c->pending) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    c->pending.clear();
    for (auto e : c->spare) cudaEventDestroy(e);
    c->spare.clear();
}

// The two dense contractions of the dense forms: M~ (into d_M32) and Gamma
// (into d_G16), on the tensor cores (FP8) or the CUDA cores (FP32).
int launch_dense_gemms(tc_ctx* c, int which, cudaStream_t s) {
    tc_gemm_args gm = {c->d_units_m, c->n_units_m, TC_GEMM_MTILDE, c->d_M32, c->n_pad, c->n_pad, c->n_pad,
                       &c->d_st->err};
    tc_gemm_args gg = {c->d_units_g, c->n_units_g, TC_GEMM_GAMMA, c->d_G16, c->k, c->n_pad, c->D * c->k,
                       &c->d_st->err};
    const bool tc = c->p.form == TC_FORM_DENSE_FP8;
    if (tc && c->fused) {  // both contractions in the first launch (M~ is zero: k_pairs zeroes it)
        if (which != 0) return TC_OK;
        tc_gemm_args gf = {c->d_units_f, c->n_units_f, TC_GEMM_MTILDE, c->d_M32, c->n_pad, c->n_pad, c->n_pad,
                           &c->d_st->err, 1, TC_GEMM_GAMMA, c->D * c->k};
        TC_CHECK(timed(c, TC_KID_GEMM_F, [&] {
            return tc_launch_gemm_tc2(c->tmS8x, c->tmS8y, c->tmM32, c->tmA8, c->tmS8T, c->tmG16, gf, c->slots_m,
                                      c->sh_m.tm, c->sh_m.cl, c->sh_m.bn, true, s);
        }, s));
        return TC_OK;
    }
    if (which == 0) {  // M~ is zero here: k_pairs zeroes it after reading it
        TC_CHECK(timed(c, TC_KID_GEMM_M, [&] {
            return tc ? tc_launch_gemm_tc(c->tmS8x, c->tmS8y, c->tmM32, gm, c->slots_m, c->sh_m.tm, c->sh_m.cl,
                                          c->sh_m.bn, true, s)
                      : tc_launch_gemm_simt(c->d_S8, c->d_S8, c->ldg, gm, c->num_sms, s);
        }, s));
    } else {
        TC_CHECK(timed(c, TC_KID_GEMM_G, [&] {
            return tc ? tc_launch_gemm_tc(c->tmA8, c->tmS8T, c->tmG16, gg, c->slots_g, c->sh_g.tm, c->sh_g.cl,
                                          c->sh_g.bn, true, s)
                      : tc_launch_gemm_simt(c->d_A8, c->d_S8T, c->n_pad, gg, c->num_sms, s);
        }, s));
    }
    return TC_OK;
}

// Step 3-ii (k_gsum) then Step 4 (k_update).
cudaError_t launch_grad_update(tc_ctx* c, const tc_kparams& P, int debug_only) {
    cudaError_t e = timed(c, TC_KID_GSUM, [&] { return tc_launch_gsum(P, c->tmB, c->num_sms, c->stream); });
    if (e != cudaSuccess) return e;
    e = timed(c, TC_KID_UPDATE, [&] { return tc_launch_update(P, c->num_sms, c->stream, debug_only); });
    // multicolouring: Step 1 of the next iteration (top-c_i sets, FP8 operands)
    if (e == cudaSuccess && P.cm && debug_only == 0) e = tc_launch_assign_multi(P, 1, c->stream);
    return e;
}

int launch_iteration_body(tc_ctx* c);

int launch_iteration(tc_ctx* c) {
    if (fault("launch")) return TC_ERR_INJECTED;
    nvtxRangePushA("tc_iteration");
    const int rc = launch_iteration_body(c);
    nvtxRangePop();
    return rc;
}

int launch_iteration_body(tc_ctx* c) {
    tc_kparams P = make_kparams(c, 1);
    const bool dense = P.M32 != nullptr;
    int rc;
    // k_pairs and k_classes share no data: k_classes builds its class lists
    // while k_pairs runs (it is launched once k_pairs has passed its wait)
    // and waits for k_pairs only before it lets k_gsum start
    if (!dense && !P.cm) {  // one-hot form: the class and pair blocks in one launch
        TC_CHECK(timed(c, TC_KID_FRONT, [&] { return tc_launch_front(P, c->stream); }));
    } else {
        if (dense && (rc = launch_dense_gemms(c, 0, c->stream))) return rc;
        TC_CHECK(timed(c, TC_KID_PAIRS, [&] { return tc_launch_pairs(P, c->stream); }));
        if (dense && (rc = launch_dense_gemms(c, 1, c->stream))) return rc;
        TC_CHECK(timed(c, TC_KID_CLASSES, [&] { return tc_launch_classes(P, c->stream); }));
    }
    TC_CHECK(launch_grad_update(c, P, 0));
    return TC_OK;
}

int launches_per_iteration(const tc_ctx* c) {
    if (c->p.form == TC_FORM_ONEHOT && c->cmax == 0) return 3;  // k_front, k_gsum, k_update
    const int gemms = c->p.form == TC_FORM_ONEHOT ? 0 : (c->fused ? 1 : 2);
    return 4 + gemms + (c->cmax > 0 ? 1 : 0);
}

int read_state(tc_ctx* c, tc_dev_state* h) {
    TC_CHECK(cudaMemcpyAsync(h, c->d_st, sizeof(*h), cudaMemcpyDeviceToHost, c->stream));
    TC_CHECK(cudaStreamSynchronize(c->stream));
    return TC_OK;
}

int build_graph_exec(tc_ctx* c) {
    drop_graph_exec(c);
    cudaGraph_t g = nullptr;
    TC_CHECK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int rc = TC_OK;
    long long before = c->launches;
    c->capturing = true;
    for (int it = 0; it < c->graph_chunk && rc == TC_OK; ++it) rc = launch_iteration(c);
    c->capturing = false;
    c->launches = before;  // counted at replay
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (rc != TC_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    TC_CHECK(e);
    e = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    TC_CHECK(e);
    return TC_OK;
}

}  // namespace

// A batch: member contexts stepped together, one graph branch per member.
struct tc_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<tc_ctx*> members;
    std::vector<cudaEvent_t> joins;  // one per member
    std::vector<long long> gens;     // members' generations at capture
    int chunk = 0;
    cudaGraphExec_t gexec = nullptr;
};

namespace {

void batch_drop_graph(tc_batch* b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
}

void batch_forget(tc_batch* b, tc_ctx* c) {
    for (size_t i = 0; i < b->members.size(); ++i)
        if (b->members[i] == c) {
            b->members.erase(b->members.begin() + i);
            cudaEventDestroy(b->joins[i]);
            b->joins.erase(b->joins.begin() + i);
            break;
        }
    c->batch = nullptr;
    batch_drop_graph(b);
}

// `iters` iterations of every member: fork from the batch stream, each
// member's iterations on its own stream, join back.  Inside a capture the
// member streams join the batch stream's capture through the fork event.
int batch_launch(tc_batch* b, int iters, bool capture) {
    TC_CHECK(cudaEventRecord(b->fork, b->stream));
    for (size_t i = 0; i < b->members.size(); ++i) {
        tc_ctx* m = b->members[i];
        TC_CHECK(cudaStreamWaitEvent(m->stream, b->fork, 0));
        m->capturing = capture;
        int rc = TC_OK;
        for (int it = 0; it < iters && rc == TC_OK; ++it) rc = launch_iteration(m);
        m->capturing = false;
        if (rc) return rc;
        TC_CHECK(cudaEventRecord(b->joins[i], m->stream));
        TC_CHECK(cudaStreamWaitEvent(b->stream, b->joins[i], 0));
    }
    return TC_OK;
}

int batch_capture(tc_batch* b, int chunk) {
    batch_drop_graph(b);
    std::vector<long long> before(b->members.size());
    for (size_t i = 0; i < b->members.size(); ++i) before[i] = b->members[i]->launches;
    TC_CHECK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int rc = batch_launch(b, chunk, true);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    for (size_t i = 0; i < b->members.size(); ++i) b->members[i]->launches = before[i];  // counted at replay
    if (rc != TC_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        (void)cudaGetLastError();
        return rc != TC_OK ? rc : TC_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    TC_CHECK(e);
    b->chunk = chunk;
    b->gens.resize(b->members.size());
    for (size_t i = 0; i < b->members.size(); ++i) b->gens[i] = b->members[i]->gen;
    return TC_OK;
}

bool batch_graph_current(const tc_batch* b, int chunk) {
    if (!b->gexec || b->chunk != chunk || b->gens.size() != b->members.size()) return false;
    for (size_t i = 0; i < b->members.size(); ++i)
        if (b->gens[i] != b->members[i]->gen) return false;
    return true;
}

}  // namespace

int tc_encode_tmap_2d(CUtensorMap* out, CUtensorMapDataType dt, void* base, uint64_t inner,
                      uint64_t outer, uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer,
                      CUtensorMapSwizzle swizzle) {
    typedef CUresult (*encode_fn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);
    static encode_fn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p) {
            (void)cudaGetLastError();
            return TC_ERR_CUDA;
        }
        fn = (encode_fn)p;
    }
    const cuuint64_t dims[2] = {inner, outer};
    const cuuint64_t strides[1] = {row_bytes};
    const cuuint32_t box[2] = {box_inner, box_outer};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(out, dt, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? TC_OK : TC_ERR_CUDA;
}

extern "C" {

const char* tc_strerror(int code) {
    switch (code) {
        case TC_OK: return "ok";
        case TC_ERR_ARG: return "invalid argument";
        case TC_ERR_GRAPH_ASYM: return "adjacency is not symmetric or has duplicate/out-of-range entries";
        case TC_ERR_GRAPH_SELFLOOP: return "adjacency has a self loop";
        case TC_ERR_OOM: return "out of memory";
        case TC_ERR_CUDA: return "CUDA runtime error";
        case TC_ERR_TIMEOUT: return "bounded device wait expired";
        case TC_ERR_DEVICE_BOUNDS: return "device-side index check failed";
        case TC_ERR_STATE: return "call out of order (no graph or no population)";
        case TC_ERR_UNSUPPORTED: return "size or form not supported by this build";
        case TC_ERR_INJECTED: return "injected fault (TC_FAULT)";
        default: return "unknown status";
    }
}

int tc_params_default(tc_params* p, int problem) {
    if (!p || problem < TC_KCOL || problem > TC_MSCP) return TC_ERR_ARG;
    memset(p, 0, sizeof(*p));
    p->problem = problem;
    p->sigma0 = 0.01f;
    p->eta = 1e-3f;
    p->alpha = 2.5f;
    p->lambda_ = 1e-5f;
    p->beta = 1.2f;
    p->mu = problem == TC_ECP ? 0.0f : 1e-6f;
    p->nu = tc_has_additive(problem) ? 1e-5f : 0.0f;
    p->rho = 100.0f;
    p->nb_iter = 5;
    p->stop_on_legal = 1;
    p->bonus_diag = 1;
    p->form = TC_FORM_ONEHOT;
    return TC_OK;
}

int tc_create(tc_ctx** out, int device) {
    if (!out) return TC_ERR_ARG;
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count == 0) {
        (void)cudaGetLastError();
        return TC_ERR_CUDA;
    }
    if (device < 0 || device >= count) return TC_ERR_ARG;
    DeviceGuard g(device);
    tc_ctx* c = new (std::nothrow) tc_ctx();
    if (!c) return TC_ERR_OOM;
    c->device = device;
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking) != cudaSuccess) {
        (void)cudaGetLastError();
        delete c;
        return TC_ERR_CUDA;
    }
    c->stream = c->own;
    *out = c;
    return TC_OK;
}

int tc_destroy(tc_ctx* c) {
    if (!c) return TC_OK;
    DeviceGuard g(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->batch) batch_forget(c->batch, c);
    free_graph(c);
    free_events(c);
    if (c->own) cudaStreamDestroy(c->own);
    delete c;
    return TC_OK;
}

int tc_set_stream(tc_ctx* c, void* stream) {
    if (!c) return TC_ERR_ARG;
    DeviceGuard g(c->device);
    TC_CHECK(cudaStreamSynchronize(c->stream));
    drop_graph_exec(c);
    c->stream = stream ? (cudaStream_t)stream : c->own;
    return TC_OK;
}

int tc_init_graph(tc_ctx* c, int n, const int32_t* rowptr, const int32_t* colidx,
                  const uint8_t* dense) {
    if (!c || n < 1 || n > TC_MAX_N) return TC_ERR_ARG;
    if (!rowptr && !dense) return TC_ERR_ARG;
    if (rowptr && !colidx && rowptr[n] > 0) return TC_ERR_ARG;
    // host-side CSR + bitmask, validated
    const int aw = (n + 127) / 128 * 4;  // bitmask rows padded to 16 bytes
    std::vector<uint32_t> bits((size_t)n * aw, 0u);
    std::vector<int> rp(n + 1, 0), ci;
    if (rowptr) {
        if (rowptr[0] != 0) return TC_ERR_ARG;
        for (int i = 0; i < n; ++i)
            if (rowptr[i + 1] < rowptr[i]) return TC_ERR_ARG;
        for (int i = 0; i < n; ++i)
            for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                const int m = colidx[e];
                if (m < 0 || m >= n) return TC_ERR_GRAPH_ASYM;
                if (m == i) return TC_ERR_GRAPH_SELFLOOP;
                uint32_t& w = bits[(size_t)i * aw + (m >> 5)];
                if (w & (1u << (m & 31))) return TC_ERR_GRAPH_ASYM;  // duplicate
                w |= 1u << (m & 31);
            }
    } else {
        for (int i = 0; i < n; ++i)
            for (int m = 0; m < n; ++m)
                if (dense[(size_t)i * n + m]) {
                    if (dense[(size_t)i * n + m] != 1) return TC_ERR_ARG;
                    if (m == i) return TC_ERR_GRAPH_SELFLOOP;
                    bits[(size_t)i * aw + (m >> 5)] |= 1u << (m & 31);
                }
    }
    for (int i = 0; i < n; ++i)  // symmetry
        for (int w = 0; w < aw; ++w) {
            uint32_t x = bits[(size_t)i * aw + w];
            while (x) {
                const int b = __builtin_ctz(x);
                x &= x - 1;
                const int m = w * 32 + b;
                if (!((bits[(size_t)m * aw + (i >> 5)] >> (i & 31)) & 1u)) return TC_ERR_GRAPH_ASYM;
            }
        }
    for (int i = 0; i < n; ++i) {  // canonical CSR: sorted neighbour lists
        for (int w = 0; w < aw; ++w) {
            uint32_t x = bits[(size_t)i * aw + w];
            while (x) {
                const int b = __builtin_ctz(x);
                x &= x - 1;
                ci.push_back(w * 32 + b);
            }
        }
        rp[i + 1] = (int)ci.size();
    }
    // tile list of the upper triangle for k_pairs
    const int T = (n + tc_pair_tile_edge() - 1) / tc_pair_tile_edge();
    std::vector<int2> tiles;
    tiles.reserve((size_t)T * (T + 1) / 2);
    for (int I = 0; I < T; ++I)
        for (int M = I; M < T; ++M) tiles.push_back(make_int2(I, M));

    DeviceGuard g(c->device);
    TC_CHECK(cudaStreamSynchronize(c->stream));
    free_graph(c);
    int rc;
    if ((rc = dalloc(&c->d_rowptr, n + 1)) || (rc = dalloc(&c->d_colidx, ci.size())) ||
        (rc = dalloc(&c->d_adj, bits.size())) || (rc = dalloc(&c->d_tiles, tiles.size()))) {
        free_graph(c);
        return rc;
    }
    if (fault("copy")) {
        free_graph(c);
        return TC_ERR_INJECTED;
    }
    cudaError_t e = cudaMemcpyAsync(c->d_rowptr, rp.data(), rp.size() * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && !ci.empty())
        e = cudaMemcpyAsync(c->d_colidx, ci.data(), ci.size() * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_adj, bits.data(), bits.size() * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_tiles, tiles.data(), tiles.size() * sizeof(int2),
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        free_graph(c);
        return cuda_status(e);
    }
    c->n = n;
    c->nnz = (long long)ci.size();
    c->max_degree = 0;
    for (int i = 0; i < n; ++i) c->max_degree = std::max(c->max_degree, rp[i + 1] - rp[i]);
    c->adj_words = aw;
    c->h_rowptr = rp;
    c->h_colidx = ci;
    c->n_tiles = (int)tiles.size();
    return TC_OK;
}

int tc_init_population(tc_ctx* c, uint64_t seed, int D, int k, const tc_params* p_in) {
    if (!c) return TC_ERR_ARG;
    if (c->n < 1) return TC_ERR_STATE;
    if (D < 1 || D > TC_MAX_D || k < 1 || k > TC_MAX_K) return TC_ERR_ARG;
    tc_params p;
    if (p_in) p = *p_in;
    else tc_params_default(&p, TC_KCOL);
    int rc = check_params(&p);
    if (rc) return rc;
    if (tc_update_fits(k) != TC_OK) return TC_ERR_UNSUPPORTED;
    DeviceGuard g(c->device);
    TC_CHECK(cudaStreamSynchronize(c->stream));
    free_population(c);
    const int n = c->n;
    const int Dp = (D + 3) & ~3;
    const size_t Wtiled = (size_t)D * ((n + TC_WT - 1) / TC_WT) * TC_WT * k;
    if ((rc = dalloc(&c->d_W, Wtiled)) || (rc = dalloc(&c->d_c, (size_t)D * n)) || (rc = dalloc(&c->d_csnap, (size_t)D * n)) ||
        (rc = dalloc(&c->d_cT, (size_t)n * Dp)) || (rc = dalloc(&c->d_planes, (size_t)n * ((D + 31) / 32) * 8)) || (rc = dalloc(&c->d_B, (size_t)(n + 1) * ((n + 3) & ~3))) ||
        (rc = dalloc(&c->d_Gbuf, (size_t)D * ((n + 31) / 32) * 32 * k)) ||
        (rc = dalloc(&c->d_rec, (size_t)D * rec_stride_for(n, k, 0, 0))) || (rc = dalloc(&c->d_z, (size_t)k)) || (rc = dalloc(&c->d_fcolor, D)) ||
        (rc = dalloc(&c->d_feq, D)) || (rc = dalloc(&c->d_loss_part, 2 * (size_t)c->n_tiles)) ||
        (rc = dalloc(&c->d_lut, 4 * (size_t)(D + 1))) || (rc = dalloc(&c->d_st, 1)) ||
        (rc = dalloc(&c->d_best, n))) {
        free_population(c);
        return rc;
    }
    c->D = D;
    c->k = k;
    c->Dp = Dp;
    c->p = p;
    c->ldb = (n + 3) & ~3;
    c->pop = true;
    rc = tc_encode_tmap_2d(&c->tmB, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, c->d_B, (uint64_t)n, (uint64_t)n,
                           4ull * c->ldb, 32, TC_BT_BOX_ROWS, CU_TENSOR_MAP_SWIZZLE_NONE);
    if (rc) {
        free_population(c);
        return rc;
    }
    tc_dev_state st;
    memset(&st, 0, sizeof(st));
    st.best_f = -1;
    st.best_d = -1;
    st.best_t = -1;
    cudaError_t e = cudaMemsetAsync(c->d_cT, 0xFF, sizeof(uint16_t) * (size_t)n * Dp, c->stream);
    if (e == cudaSuccess)  // row n of B is the zero row the padded classes point at
        e = cudaMemsetAsync(c->d_B, 0, sizeof(float) * (size_t)(n + 1) * ((n + 3) & ~3), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_fcolor, 0, sizeof(int) * D, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_best, 0, sizeof(uint16_t) * n, c->stream);
    std::vector<int> zdef(k);
    for (int j = 0; j < k; ++j) zdef[j] = j + 1;  // colours numbered 1..k
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_z, zdef.data(), sizeof(int) * k, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_st, &st, sizeof(st), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)  // padding rows of the last vertex tile stay zero
        e = cudaMemsetAsync(c->d_W, 0, sizeof(float) * Wtiled, c->stream);
    if (e == cudaSuccess) e = tc_launch_init_weights(c->d_W, D, n, k, seed, p.sigma0, c->stream);
    if (e == cudaSuccess) e = tc_launch_assign(make_kparams(c, 0), c->stream);
    c->launches += 2;
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        free_population(c);
        return cuda_status(e);
    }
    rc = upload_luts(c);
    if (!rc && p.form != TC_FORM_ONEHOT) rc = setup_dense(c);
    if (!rc && rebuild_onehot(c) != cudaSuccess) rc = TC_ERR_CUDA;
    if (!rc && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = TC_ERR_CUDA;
    if (rc) {
        (void)cudaGetLastError();
        free_population(c);
        return rc;
    }
    return TC_OK;
}

int tc_set_params(tc_ctx* c, const tc_params* p) {
    if (!c || !p) return TC_ERR_ARG;
    if (!c->pop) return TC_ERR_STATE;
    int rc = check_params(p);
    if (rc) return rc;
    if (c->cmax > 0 && (p->form == TC_FORM_ONEHOT || p->problem != TC_KCOL))
        return TC_ERR_UNSUPPORTED;  // the multicolouring runs the k-COL problem in a dense form
    DeviceGuard g(c->device);
    TC_CHECK(cudaStreamSynchronize(c->stream));
    tc_params old = c->p;
    c->p = *p;
    rc = upload_luts(c);
    if (!rc && p->form != old.form) {
        if (p->form == TC_FORM_ONEHOT) {
            free_dense(c);
        } else if (!c->d_M32) {
            rc = setup_dense(c);
            if (!rc && rebuild_onehot(c) != cudaSuccess) rc = TC_ERR_CUDA;
            if (!rc && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = TC_ERR_CUDA;
        } else {
            rc = plan_dense(c);  // the other dense form: its own tiles
        }
    }
    if (rc) {
        (void)cudaGetLastError();
        c->p = old;
        upload_luts(c);
        // a dense form keeps a plan that matches its own kernels
        if (old.form != TC_FORM_ONEHOT && c->d_M32 && plan_dense(c) != TC_OK) {
            (void)cudaGetLastError();
            free_dense(c);
            c->p.form = TC_FORM_ONEHOT;
        }
        drop_graph_exec(c);
        return rc;
    }
    drop_graph_exec(c);
    return TC_OK;
}

int tc_step(tc_ctx* c, int64_t n_iters, int64_t* iters_done) {
    if (iters_done) *iters_done = 0;
    if (!c || n_iters < 0) return TC_ERR_ARG;
    if (!c->pop) return TC_ERR_STATE;
    DeviceGuard g(c->device);
    tc_dev_state h;
    int rc = read_state(c, &h);
    if (rc) return rc;
    const long long t0 = h.t;
    TC_CHECK(cudaMemsetAsync(&c->d_st->stop, 0, sizeof(int), c->stream));
    long long left = n_iters;
    // poll the device stop flag between chunks only when it can be raised
    const long long poll = c->p.stop_on_legal ? 64 : (long long)1 << 62;
    long long since_poll = 0;
    while (left > 0) {
        if (c->graph_chunk > 0 && left >= c->graph_chunk) {
            if (!c->gexec) {
                rc = build_graph_exec(c);
                if (rc) return rc;
            }
            TC_CHECK(cudaGraphLaunch(c->gexec, c->stream));
            c->launches += (long long)launches_per_iteration(c) * c->graph_chunk;
            left -= c->graph_chunk;
            since_poll += c->graph_chunk;
        } else {
            rc = launch_iteration(c);
            if (rc) return rc;
            left -= 1;
            since_poll += 1;
        }
        if (since_poll >= poll && left > 0) {
            since_poll = 0;
            rc = read_state(c, &h);
            if (rc) return rc;
            if (h.stop) break;
        }
    }
    rc = read_state(c, &h);
    if (rc) return rc;
    if (h.err) return h.err;
    if (iters_done) *iters_done = h.t - t0;
    return TC_OK;
}

int tc_best(tc_ctx* c, int32_t* coloring, int64_t* conflicts, int64_t* equity, int32_t* individual,
            int64_t* iteration) {
    if (!c) return TC_ERR_ARG;
    if (!c->pop) return TC_ERR_STATE;
    DeviceGuard g(c->device);
    tc_dev_state h;
    int rc = read_state(c, &h);
    if (rc) return rc;
    if (h.best_f < 0) return TC_ERR_STATE;
    if (coloring) {
        std::vector<uint16_t> b(c->n);
        TC_CHECK(cudaMemcpyAsync(b.data(), c->d_best, sizeof(uint16_t) * c->n, cudaMemcpyDeviceToHost,
                                 c->stream));
        TC_CHECK(cudaStreamSynchronize(c->stream));
        for (int i = 0; i < c->n; ++i) coloring[i] = b[i];
    }
    if (conflicts) *conflicts = h.best_fcolor;
    if (equity) *equity = h.best_feq;
    if (individual) *individual = h.best_d;
    if (iteration) *iteration = h.best_t;
    return TC_OK;
}

// Device address of a page-locked host buffer (cudaHostAlloc or
// cudaHostRegister memory, torch's pin_memory included), or null for
// pageable memory: the weight conversions read and write page-locked
// buffers directly, in whole lines, instead of staging them with a copy.
static void* pinned_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int tc_get_state(tc_ctx* c, float* W, int64_t* t) {
    if (!c) return TC_ERR_ARG;
    if (!c->pop) return TC_ERR_STATE;
    DeviceGuard g(c->device);
    if (W) {
        if (fault("copy")) return TC_ERR_INJECTED;
        float* Wd = static_cast<float*>(pinned_device_ptr(W));
        // (a null address, a tile beyond 48 KB or a failed launch: the staged path;
        // the launcher has taken the error of its launch)
        if (Wd && tc_launch_w_tiles(c->d_W, Wd, c->D, c->n, c->k, false, c->stream) == cudaSuccess) {
            c->launches += 1;  // untiled straight into the page-locked buffer
        } else {
            // untile into the grad_S buffer (free between iterations), then copy
            TC_CHECK(tc_launch_w_layout(c->d_W, c->d_Gbuf, c->D, c->n, c->k, false, c->stream));
            c->launches += 1;
            TC_CHECK(cudaMemcpyAsync(W, c->d_Gbuf, sizeof(float) * (size_t)c->D * c->n * c->k,
                                     cudaMemcpyDeviceToHost, c->stream));
        }
    }
    if (t) {
        long long tv = 0;
        TC_CHECK(cudaMemcpyAsync(&tv, &c->d_st->t, sizeof(tv), cudaMemcpyDeviceToHost, c->stream));
        TC_CHECK(cudaStreamSynchronize(c->stream));
        *t = tv;
    }
    TC_CHECK(cudaStreamSynchronize(c->stream));
    return TC_OK;
}

static int set_state_common(tc_ctx* c, const float* W, const int64_t* t, cudaMemcpyKind kind) {
    if (!c) return TC_ERR_ARG;
    if (!c->pop) return TC_ERR_STATE;
    if (t && *t < 0) return TC_ERR_ARG;
    DeviceGuard g(c->device);
    if (W) {
        if (fault("copy")) return TC_ERR_INJECTED;
        const float* src = W;
        const float* Wd = kind == cudaMemcpyHostToDevice ? static_cast<const float*>(pinned_device_ptr(W)) : nullptr;
        if (Wd && tc_launch_w_tiles(Wd, c->d_W, c->D, c->n, c->k, true, c->stream) == cudaSuccess) {
            c->launches += 1;  // tiled straight from the page-locked buffer
        } else {
            if (kind == cudaMemcpyHostToDevice) {  // through the grad_S buffer
                TC_CHECK(cudaMemcpyAsync(c->d_Gbuf, W, sizeof(float) * (size_t)c->D * c->n * c->k, kind, c->stream));
                src = c->d_Gbuf;
            }
            TC_CHECK(tc_launch_w_layout(src, c->d_W, c->D, c->n, c->k, true, c->stream));
            c->launches += 1;
        }
    }
    if (t) {
        const long long tv = *t;
        TC_CHECK(cudaMemcpyAsync(&c->d_st->t, &tv, sizeof(tv), cudaMemcpyHostToDevice, c->stream));
    }
    TC_CHECK(cudaMemsetAsync(&c->d_st->stop, 0, sizeof(int), c->stream));
    TC_CHECK(tc_launch_assign(make_kparams(c, 0), c->stream));
    c->launches += 1;
    TC_CHECK(rebuild_onehot(c));
    TC_CHECK(cudaStreamSynchronize(c->stream));
    return TC_OK;
}

int tc_set_state(tc_ctx* c, const float* W, const int64_t* t) {
    return set_state_common(c, W, t, cudaMemcpyHostToDevice);
}

int tc_get_state_dev(tc_ctx* c, float* W_dev) {
    if (!c || !W_dev) return TC_ERR_ARG;
    if (!c->pop) return TC_ERR_STATE;
    DeviceGuard g(c->device);
    TC_CHECK(tc_launch_w_layout(c->d_W, W_dev, c->D, c->n, c->k, false, c->stream));
    c->launches += 1;
    TC_CHECK(cudaStreamSynchronize(c->stream));
    return TC_OK;
}

int tc_set_state_dev(tc_ctx* c, const float* W_dev) {
    if (!W_dev) return TC_ERR_ARG;
    return set_state_common(c, W_dev, nullptr, cudaMemcpyDeviceToDevice);
}

int tc_evaluate(tc_ctx* c, int32_t* colors, int32_t* gamma_own, int32_t* f_color, int32_t* f_eq,
                int32_t* Mtilde, float* G, float* loss) {
    if (!c) return TC_ERR_ARG;
    if (!c->pop) return TC_ERR_STATE;
    DeviceGuard g(c->device);
    const int n = c->n, D = c->D, k = c->k;
    int* d_mt = nullptr;
    float* d_G = nullptr;
    int* d_gam = nullptr;
    int rc = TC_OK;
    if (Mtilde && (rc = dalloc(&d_mt, (size_t)n * n))) return rc;
    if (G && (rc = dalloc(&d_G, (size_t)D * n * k))) {
        dfree(d_mt);
        return rc;
    }
    if (gamma_own && (rc = dalloc(&d_gam, (size_t)D * n))) {
        dfree(d_mt);
        dfree(d_G);
        return rc;
    }
    tc_kparams P = make_kparams(c, 0);
    P.dbg_Mt = d_mt;
    P.dbg_G = d_G;
    P.dbg_gamma = d_gam;
    const bool dense = P.M32 != nullptr;
    cudaError_t e = cudaSuccess;
    if (dense && launch_dense_gemms(c, 0, c->stream)) e = cudaErrorUnknown;
    if (e == cudaSuccess) e = tc_launch_pairs(P, c->stream);
    if (e == cudaSuccess && dense && launch_dense_gemms(c, 1, c->stream)) e = cudaErrorUnknown;
    if (e == cudaSuccess) e = tc_launch_classes(P, c->stream);
    // k_gsum counts the conflicts and reduces the population; k_update only
    // copies grad_S L out (debug mode 1) when G is wanted
    if (e == cudaSuccess)
        e = G ? launch_grad_update(c, P, 1) : tc_launch_gsum(P, c->tmB, c->num_sms, c->stream);
    c->launches += 2;
    std::vector<uint16_t> hc;
    tc_dev_state h;
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess && colors) {
        hc.resize((size_t)D * n);
        e = cudaMemcpy(hc.data(), c->d_c, hc.size() * 2, cudaMemcpyDeviceToHost);
        for (size_t q = 0; q < hc.size(); ++q) colors[q] = hc[q];
    }
    if (e == cudaSuccess && gamma_own)
        e = cudaMemcpy(gamma_own, d_gam, sizeof(int) * (size_t)D * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && f_color) e = cudaMemcpy(f_color, c->d_fcolor, sizeof(int) * D, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && f_eq) e = cudaMemcpy(f_eq, c->d_feq, sizeof(int) * D, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && Mtilde)
        e = cudaMemcpy(Mtilde, d_mt, sizeof(int) * (size_t)n * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && G) e = cudaMemcpy(G, d_G, sizeof(float) * (size_t)D * n * k, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && loss) {
        e = cudaMemcpy(&h, c->d_st, sizeof(h), cudaMemcpyDeviceToHost);
        loss[0] = h.loss;
        loss[1] = h.kappa;
        loss[2] = h.varpi;
        loss[3] = (float)h.fcolor_sum;
    }
    if (e == cudaSuccess && !loss) e = cudaMemcpy(&h, c->d_st, sizeof(h), cudaMemcpyDeviceToHost);
    dfree(d_mt);
    dfree(d_G);
    dfree(d_gam);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return cuda_status(e);
    }
    return h.err ? h.err : TC_OK;
}

int tc_step_async(tc_ctx* c, int64_t n_iters) {
    if (!c || n_iters < 0) return TC_ERR_ARG;
    if (!c->pop) return TC_ERR_STATE;
    DeviceGuard g(c->device);
    for (long long it = 0; it < n_iters;) {
        int rc;
        if (c->graph_chunk > 0 && n_iters - it >= c->graph_chunk) {
            if (!c->gexec && (rc = build_graph_exec(c))) return rc;
            TC_CHECK(cudaGraphLaunch(c->gexec, c->stream));
            c->launches += (long long)launches_per_iteration(c) * c->graph_chunk;
            it += c->graph_chunk;
        } else {
            if ((rc = launch_iteration(c))) return rc;
            it += 1;
        }
    }
    return TC_OK;
}

int tc_set_timing(tc_ctx* c, int on) {
    if (!c) return TC_ERR_ARG;
    DeviceGuard g(c->device);
    int rc = collect_timing(c);
    if (rc) return rc;
    c->timing = on ? 1 : 0;
    for (int q = 0; q < TC_NUM_KID; ++q) {
        c->kms[q] = 0.0;
        c->kcount[q] = 0;
    }
    return TC_OK;
}

int tc_kernel_times(tc_ctx* c, double* ms, int64_t* count) {
    if (!c) return TC_ERR_ARG;
    DeviceGuard g(c->device);
    int rc = collect_timing(c);
    if (rc) return rc;
    for (int q = 0; q < TC_NUM_KID; ++q) {
        if (ms) ms[q] = c->kms[q];
        if (count) count[q] = c->kcount[q];
    }
    return TC_OK;
}

int tc_st_grad_dev(tc_ctx* c, float* gradW_dev, float* loss_dev) {
    if (!c || !gradW_dev) return TC_ERR_ARG;
    if (!c->pop) return TC_ERR_STATE;
    DeviceGuard g(c->device);
    tc_kparams P = make_kparams(c, 0);
    P.dbg_G = gradW_dev;
    const bool dense = P.M32 != nullptr;
    int rc;
    if (dense && (rc = launch_dense_gemms(c, 0, c->stream))) return rc;
    TC_CHECK(tc_launch_pairs(P, c->stream));
    if (dense && (rc = launch_dense_gemms(c, 1, c->stream))) return rc;
    TC_CHECK(tc_launch_classes(P, c->stream));
    TC_CHECK(launch_grad_update(c, P, 2));
    c->launches += 2;
    if (loss_dev)  // loss, kappa, varpi are consecutive floats of the state
        TC_CHECK(cudaMemcpyAsync(loss_dev, &c->d_st->loss, 3 * sizeof(float), cudaMemcpyDeviceToDevice,
                                 c->stream));
    tc_dev_state h;
    rc = read_state(c, &h);
    if (rc) return rc;
    return h.err ? h.err : TC_OK;
}

int tc_relaxed_dev(tc_ctx* c, const float* W_dev, float tau, int64_t t, float* loss_dev, float* gradW_dev) {
    if (!c || !W_dev || !loss_dev || !gradW_dev || !(tau > 0.f) || t < 0) return TC_ERR_ARG;
    if (!c->pop) return TC_ERR_STATE;
    if (tc_is_partition(c->p.problem) || c->p.problem == TC_MSCP) return TC_ERR_ARG;  // the GCP terms only
    if (c->k > 128) return TC_ERR_UNSUPPORTED;
    DeviceGuard g(c->device);
    const int n = c->n;
    float *S = nullptr, *M = nullptr, *Bp = nullptr, *part = nullptr;
    int rc;
    if ((rc = dalloc(&S, (size_t)c->D * n * c->k)) || (rc = dalloc(&M, (size_t)n * n)) ||
        (rc = dalloc(&Bp, (size_t)n * n)) || (rc = dalloc(&part, 3 * (size_t)tc_relaxed_partials(n)))) {
        dfree(S); dfree(M); dfree(Bp); dfree(part);
        return rc;
    }
    rc = tc_relaxed_run(make_kparams(c, 0), W_dev, tau, t, loss_dev, gradW_dev, S, M, Bp, part, c->stream);
    c->launches += 5;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    dfree(S); dfree(M); dfree(Bp); dfree(part);
    if (rc) return rc;
    TC_CHECK(e);
    return TC_OK;
}

int tc_set_wait_limit(tc_ctx* c, int64_t ns) {
    if (!c || ns < 0 || ns > 60000000000ll) return TC_ERR_ARG;
    DeviceGuard g(c->device);
    drop_graph_exec(c);
    c->wait_ns = ns > 0 ? (unsigned long long)ns : 1000000000ull;
    return TC_OK;
}

int tc_launch_count(tc_ctx* c, int64_t* count) {
    if (!c || !count) return TC_ERR_ARG;
    *count = c->launches;
    return TC_OK;
}

int tc_set_graph_chunk(tc_ctx* c, int chunk) {
    if (!c || chunk < 0 || chunk > 100000) return TC_ERR_ARG;
    DeviceGuard g(c->device);
    drop_graph_exec(c);
    c->graph_chunk = chunk;
    return TC_OK;
}

int tc_kdescent(tc_ctx* c, uint64_t seed, int D, int k_start, int k_min, int64_t max_iters, const tc_params* p_in,
                int32_t* k_best, int32_t* coloring, int64_t* iters_total) {
    if (k_best) *k_best = -1;
    if (iters_total) *iters_total = 0;
    if (!c || D < 1 || k_min < 1 || k_start < k_min || k_start > TC_MAX_K || max_iters < 1) return TC_ERR_ARG;
    if (c->n < 1) return TC_ERR_STATE;
    tc_params p;
    if (p_in) p = *p_in;
    else tc_params_default(&p, TC_KCOL);
    p.stop_on_legal = 1;
    int rc = check_params(&p);
    if (rc) return rc;
    // k-descent is for the problems whose fitness reaches 0 on a solution
    if (tc_is_partition(p.problem) || p.problem == TC_MSCP) return TC_ERR_ARG;
    std::vector<int32_t> col(c->n);
    long long total = 0;
    for (int k = k_start; k >= k_min; --k) {
        if ((rc = tc_init_population(c, seed + (uint64_t)k, D, k, &p))) return rc;
        int64_t done = 0;
        if ((rc = tc_step(c, max_iters, &done))) return rc;
        total += done;
        if (iters_total) *iters_total = total;
        int64_t conf = -1, eq = -1;
        if ((rc = tc_best(c, col.data(), &conf, &eq, nullptr, nullptr))) return rc;
        const bool legal = conf == 0 && (p.problem != TC_ECP || eq == 0);
        if (!legal) break;
        if (k_best) *k_best = k;
        if (coloring) memcpy(coloring, col.data(), sizeof(int32_t) * (size_t)c->n);
    }
    return TC_OK;
}

int tc_set_color_costs(tc_ctx* c, const int32_t* z, int k) {
    if (!c || !z) return TC_ERR_ARG;
    if (!c->pop) return TC_ERR_STATE;
    if (k != c->k) return TC_ERR_ARG;
    long long zmax = 0;
    for (int j = 0; j < k; ++j) {
        if (z[j] < 0) return TC_ERR_ARG;
        zmax = std::max(zmax, (long long)z[j]);
    }
    // the reduction keeps f = f_color + f_mscp in 31 bits
    if (zmax * c->n + c->nnz / 2 >= (1ll << 31)) return TC_ERR_UNSUPPORTED;
    DeviceGuard g(c->device);
    TC_CHECK(cudaMemcpyAsync(c->d_z, z, sizeof(int) * (size_t)k, cudaMemcpyHostToDevice, c->stream));
    TC_CHECK(cudaStreamSynchronize(c->stream));
    return TC_OK;
}

int tc_set_trace(tc_ctx* c, int capacity, int every) {
    if (!c || capacity < 0 || every < 1) return TC_ERR_ARG;
    if (!c->pop) return TC_ERR_STATE;
    DeviceGuard g(c->device);
    TC_CHECK(cudaStreamSynchronize(c->stream));
    tc_trace_entry* ring = nullptr;
    int rc;
    if (capacity > 0 && (rc = dalloc(&ring, (size_t)capacity))) return rc;
    dfree(c->d_trace);
    c->d_trace = ring;
    c->trace_cap = capacity;
    c->trace_every = every;
    const long long zero = 0;
    TC_CHECK(cudaMemcpyAsync(&c->d_st->trace_n, &zero, sizeof(zero), cudaMemcpyHostToDevice, c->stream));
    TC_CHECK(cudaStreamSynchronize(c->stream));
    drop_graph_exec(c);  // captured launches carry the old ring
    return TC_OK;
}

int tc_get_trace(tc_ctx* c, tc_trace_entry* out, int max, int* count) {
    if (!c || max < 0) return TC_ERR_ARG;
    if (count) *count = 0;
    if (!c->pop) return TC_ERR_STATE;
    if (c->trace_cap == 0) return TC_OK;
    DeviceGuard g(c->device);
    tc_dev_state h;
    int rc = read_state(c, &h);
    if (rc) return rc;
    const long long kept = std::min<long long>(h.trace_n, c->trace_cap);
    if (count) *count = (int)kept;
    if (!out || max == 0 || kept == 0) return TC_OK;
    std::vector<tc_trace_entry> ring((size_t)c->trace_cap);
    TC_CHECK(cudaMemcpyAsync(ring.data(), c->d_trace, sizeof(tc_trace_entry) * ring.size(), cudaMemcpyDeviceToHost,
                             c->stream));
    TC_CHECK(cudaStreamSynchronize(c->stream));
    const long long first = h.trace_n - kept;  // oldest retained record
    for (long long r = 0; r < kept && r < max; ++r) out[r] = ring[(size_t)((first + r) % c->trace_cap)];
    return TC_OK;
}

int tc_set_demands(tc_ctx* c, const int32_t* demand, int n) {
    if (!c || !demand) return TC_ERR_ARG;
    if (!c->pop) return TC_ERR_STATE;
    if (n != c->n) return TC_ERR_ARG;
    if (c->p.form == TC_FORM_ONEHOT || c->p.problem != TC_KCOL) return TC_ERR_UNSUPPORTED;
    int cmax = 1;
    long long sum = 0;
    for (int i = 0; i < n; ++i) {
        if (demand[i] < 1 || demand[i] > std::min(c->k, TC_MAX_DEMAND)) return TC_ERR_ARG;
        cmax = std::max(cmax, (int)demand[i]);
        sum += demand[i];
    }
    if ((long long)c->D * cmax >= (1ll << 24)) return TC_ERR_UNSUPPORTED;  // M~ exact in FP32
    DeviceGuard g(c->device);
    TC_CHECK(cudaStreamSynchronize(c->stream));
    const int new_cmax = cmax > 1 ? cmax : 0;  // all demands 1: one colour per vertex
    const long long new_sum = cmax > 1 ? sum : 0;
    // new buffers first: a failed allocation leaves the context as it was
    uint32_t* rec = nullptr;
    float* lut = nullptr;
    int* dem = nullptr;
    uint16_t *cm = nullptr, *best_m = nullptr;
    int rc;
    if ((rc = dalloc(&rec, (size_t)c->D * rec_stride_for(c->n, c->k, new_cmax, new_sum))) ||
        (rc = dalloc(&lut, 4 * (size_t)(mt_max_for(c->D, new_cmax) + 1))) ||
        (new_cmax > 0 && ((rc = dalloc(&dem, (size_t)n)) || (rc = dalloc(&cm, (size_t)c->D * n * new_cmax)) ||
                          (rc = dalloc(&best_m, (size_t)n * new_cmax))))) {
        dfree(rec);
        dfree(lut);
        dfree(dem);
        dfree(cm);
        dfree(best_m);
        return rc;
    }
    dfree(c->d_rec);
    dfree(c->d_lut);
    dfree(c->d_dem);
    dfree(c->d_cm);
    dfree(c->d_best_m);
    c->d_rec = rec;
    c->d_lut = lut;
    c->d_dem = dem;
    c->d_cm = cm;
    c->d_best_m = best_m;
    c->cmax = new_cmax;
    c->dem_sum = new_sum;
    if (dem) TC_CHECK(cudaMemcpyAsync(dem, demand, sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, c->stream));
    if ((rc = upload_luts(c))) return rc;
    // Step 1 again under the new demands, and a fresh best-so-far
    TC_CHECK(tc_launch_assign(make_kparams(c, 0), c->stream));
    TC_CHECK(rebuild_onehot(c));
    c->launches += 1;
    tc_dev_state h;
    if ((rc = read_state(c, &h))) return rc;
    h.best_f = -1;
    h.best_d = -1;
    h.best_t = -1;
    h.stop = 0;
    TC_CHECK(cudaMemcpyAsync(c->d_st, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream));
    TC_CHECK(cudaStreamSynchronize(c->stream));
    drop_graph_exec(c);
    return TC_OK;
}

int tc_best_multi(tc_ctx* c, int32_t* colors, int stride, int64_t* conflicts, int32_t* individual,
                  int64_t* iteration) {
    if (!c) return TC_ERR_ARG;
    if (!c->pop || c->cmax == 0) return TC_ERR_STATE;
    if (colors && stride < c->cmax) return TC_ERR_ARG;
    DeviceGuard g(c->device);
    tc_dev_state h;
    int rc = read_state(c, &h);
    if (rc) return rc;
    if (h.best_f < 0) return TC_ERR_STATE;
    if (colors) {
        std::vector<uint16_t> b((size_t)c->n * c->cmax);
        TC_CHECK(cudaMemcpyAsync(b.data(), c->d_best_m, sizeof(uint16_t) * b.size(), cudaMemcpyDeviceToHost,
                                 c->stream));
        TC_CHECK(cudaStreamSynchronize(c->stream));
        for (int i = 0; i < c->n; ++i)
            for (int q = 0; q < stride; ++q) {
                const int v = q < c->cmax ? b[(size_t)i * c->cmax + q] : 0xFFFF;
                colors[(size_t)i * stride + q] = v == 0xFFFF ? -1 : v;
            }
    }
    if (conflicts) *conflicts = h.best_fcolor;
    if (individual) *individual = h.best_d;
    if (iteration) *iteration = h.best_t;
    return TC_OK;
}

int tc_get_multicolors(tc_ctx* c, int32_t* colors, int stride) {
    if (!c || !colors) return TC_ERR_ARG;
    if (!c->pop || c->cmax == 0) return TC_ERR_STATE;
    if (stride < c->cmax) return TC_ERR_ARG;
    DeviceGuard g(c->device);
    std::vector<uint16_t> b((size_t)c->D * c->n * c->cmax);
    TC_CHECK(cudaMemcpyAsync(b.data(), c->d_cm, sizeof(uint16_t) * b.size(), cudaMemcpyDeviceToHost, c->stream));
    TC_CHECK(cudaStreamSynchronize(c->stream));
    for (size_t r = 0; r < (size_t)c->D * c->n; ++r)
        for (int q = 0; q < stride; ++q) {
            const int v = q < c->cmax ? b[r * c->cmax + q] : 0xFFFF;
            colors[r * stride + q] = v == 0xFFFF ? -1 : v;
        }
    return TC_OK;
}

int tc_dense_plan(tc_ctx* c, int32_t* plan, float* us) {
    if (!c || !plan) return TC_ERR_ARG;
    if (!c->pop || !c->d_M32) return TC_ERR_STATE;
    const int v[9] = {c->sh_g.tm, c->sh_g.bn, c->sh_g.cl, c->sh_m.tm,      c->sh_m.bn,
                      c->sh_m.cl, c->split_m, c->fused ? 1 : 0, c->tune_candidates};
    memcpy(plan, v, sizeof(v));
    if (us) {
        us[0] = c->tune_us_g;
        us[1] = c->tune_us_m;
        us[2] = c->tune_us_f;
    }
    return TC_OK;
}

int tc_dense_set_plan(tc_ctx* c, const int32_t* plan) {
    if (!c || !plan) return TC_ERR_ARG;
    if (!c->pop || !c->d_M32) return TC_ERR_STATE;
    const tc_gemm_shape sg{plan[0], plan[1], plan[2]}, sm{plan[3], plan[4], plan[5]};
    if (!plan_valid(c, sg, sm, plan[6]) || (plan[7] != 0 && plan[7] != 1)) return TC_ERR_ARG;
    if (plan[7] == 1 && !fusable(c, sg, sm)) return TC_ERR_ARG;
    DeviceGuard g(c->device);
    TC_CHECK(cudaStreamSynchronize(c->stream));
    const tc_gemm_shape og = c->sh_g, om = c->sh_m;
    const int osplit = c->split_m;
    const bool ofused = c->fused;
    int rc = apply_plan(c, sg, sm, plan[6], plan[7] == 1);
    if (rc) {
        (void)cudaGetLastError();
        apply_plan(c, og, om, osplit, ofused);
        return rc;
    }
    drop_graph_exec(c);
    return TC_OK;
}

int tc_batch_create(tc_batch** out, int device) {
    if (!out) return TC_ERR_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
        (void)cudaGetLastError();
        return TC_ERR_CUDA;
    }
    if (device < 0 || device >= count) return TC_ERR_ARG;
    DeviceGuard g(device);
    tc_batch* b = new (std::nothrow) tc_batch();
    if (!b) return TC_ERR_OOM;
    b->device = device;
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
        (void)cudaGetLastError();
        if (b->stream) cudaStreamDestroy(b->stream);
        delete b;
        return TC_ERR_CUDA;
    }
    *out = b;
    return TC_OK;
}

int tc_batch_add(tc_batch* b, tc_ctx* c) {
    if (!b || !c) return TC_ERR_ARG;
    if (c->device != b->device) return TC_ERR_ARG;
    if (!c->pop || c->batch) return TC_ERR_STATE;
    DeviceGuard g(b->device);
    cudaEvent_t e = nullptr;
    TC_CHECK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    b->members.push_back(c);
    b->joins.push_back(e);
    c->batch = b;
    batch_drop_graph(b);
    return TC_OK;
}

int tc_batch_size(tc_batch* b, int* count) {
    if (!b || !count) return TC_ERR_ARG;
    *count = (int)b->members.size();
    return TC_OK;
}

int tc_batch_step(tc_batch* b, int64_t n_iters, int chunk) {
    if (!b || n_iters < 0 || chunk < 0 || chunk > 100000) return TC_ERR_ARG;
    for (tc_ctx* m : b->members)
        if (!m->pop) return TC_ERR_STATE;
    DeviceGuard g(b->device);
    // earlier work of the members first; every member starts with its stop
    // flag cleared, as tc_step does
    for (size_t i = 0; i < b->members.size(); ++i) {
        tc_ctx* m = b->members[i];
        TC_CHECK(cudaEventRecord(b->joins[i], m->stream));
        TC_CHECK(cudaStreamWaitEvent(b->stream, b->joins[i], 0));
        TC_CHECK(cudaMemsetAsync(&m->d_st->stop, 0, sizeof(int), b->stream));
    }
    const long long full = chunk > 0 ? n_iters / chunk : 0;
    const int rem = (int)(n_iters - full * chunk);
    int rc;
    if (full > 0) {
        if (!batch_graph_current(b, chunk) && (rc = batch_capture(b, chunk))) return rc;
        for (long long f = 0; f < full; ++f) TC_CHECK(cudaGraphLaunch(b->gexec, b->stream));
        for (tc_ctx* m : b->members) m->launches += (long long)launches_per_iteration(m) * chunk * full;
    }
    if (rem > 0 && (rc = batch_launch(b, rem, false))) return rc;
    TC_CHECK(cudaStreamSynchronize(b->stream));
    for (tc_ctx* m : b->members) {
        tc_dev_state h;
        if ((rc = read_state(m, &h))) return rc;
        if (h.err) return h.err;
    }
    return TC_OK;
}

int tc_batch_destroy(tc_batch* b) {
    if (!b) return TC_OK;
    DeviceGuard g(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (tc_ctx* m : b->members) m->batch = nullptr;
    batch_drop_graph(b);
    for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return TC_OK;
}

}  // extern "C"
