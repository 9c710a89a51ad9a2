// Multicolouring (Goudet, Duval, Hao, Section 6): vertex i must take c_i
// colours, no colour shared across an edge.  Step 1 of Algorithm 1 selects
// the c_i colours of largest weight in w_{d,i}; S_d becomes a 0/1 matrix
// with c_i ones in row i and every other step keeps its formula on it
// (M_d = S_d S_d^T counts shared colours, M~ = sum_d M_d with m~_ii = D c_i,
// gamma = A.S counts neighbours per colour, eq. 13 sums over each colour's
// members).  The dense forms compute M~ and A.S as GEMMs over the multi-hot
// FP8 operands unchanged; this file holds the two steps that differ:
//
//   k_assign_multi   top-c_i selection per row (lower colour first among
//                    equal weights), colour sets, FP8 operand entries
//   k_classes_multi  colour classes of the multi-hot S (a vertex is listed
//                    in each of its c_i classes, in vertex order), padded to
//                    multiples of 4 with the zero row n of B
#include "tc_internal.cuh"

namespace {

constexpr int MC_THREADS = 256;

// One thread per (d, i) row, lanes over the 32 rows of a weight tile (the
// tiled layout makes each colour's loads one 128-byte line).  clear_old:
// the row's previous colours are taken out of the FP8 operands first.
__global__ void __launch_bounds__(MC_THREADS) k_assign_multi(tc_kparams P, int clear_old) {
    const int nT = (P.n + TC_WT - 1) / TC_WT;
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (long long)P.D * nT * TC_WT) return;
    const int d = (int)(r / ((long long)nT * TC_WT));
    const int i = (int)(r % ((long long)nT * TC_WT));
    if (i >= P.n) return;
    const int k = P.k, c = P.dem[i];
    float bv[TC_MAX_DEMAND];
    int bj[TC_MAX_DEMAND];
    for (int q = 0; q < c; ++q) {
        bv[q] = -INFINITY;
        bj[q] = -1;
    }
    for (int j = 0; j < k; ++j) {
        const float w = P.W[tc_w_index(d, i, j, nT, k)];
        // insert behind every kept weight >= w: equal weights keep the lower colour first
        if (bj[c - 1] >= 0 && !(w > bv[c - 1])) continue;
        int q = c - 1;
        while (q > 0 && (bj[q - 1] < 0 || w > bv[q - 1])) {
            bv[q] = bv[q - 1];
            bj[q] = bj[q - 1];
            --q;
        }
        bv[q] = w;
        bj[q] = j;
    }
    uint16_t* set = P.cm + ((size_t)d * P.n + i) * P.cmax;
    if (clear_old)
        for (int q = 0; q < P.cmax; ++q) {
            const int o = set[q];
            if (o == 0xFFFF) break;
            const size_t col = (size_t)d * k + o;
            P.S8[(size_t)i * P.ldg + col] = 0;
            P.S8T[col * P.n_pad + i] = 0;
        }
    // the set in increasing colour order; the first colour of largest weight
    // is the row's representative colour
    int sorted[TC_MAX_DEMAND];
    for (int q = 0; q < c; ++q) sorted[q] = bj[q];
    for (int a = 1; a < c; ++a)
        for (int b = a; b > 0 && sorted[b - 1] > sorted[b]; --b) {
            const int t = sorted[b];
            sorted[b] = sorted[b - 1];
            sorted[b - 1] = t;
        }
    for (int q = 0; q < P.cmax; ++q) set[q] = q < c ? (uint16_t)sorted[q] : (uint16_t)0xFFFF;
    for (int q = 0; q < c; ++q) {
        const size_t col = (size_t)d * k + sorted[q];
        P.S8[(size_t)i * P.ldg + col] = 0x38;  // E4M3 1.0
        P.S8T[col * P.n_pad + i] = 0x38;
    }
    P.c[(size_t)d * P.n + i] = (uint16_t)bj[0];
}

__device__ __forceinline__ bool has_colour(const uint16_t* set, int c, int j) {
    for (int q = 0; q < c; ++q)
        if (set[q] == j) return true;
    return false;
}

// One block per individual: class sizes, padded offsets, class lists; the
// additive term is absent (multicolouring is a k-COL variant): E = 0, f_eq = 0.
// masks (k x adj_words words of dynamic shared memory, or 0): the class
// membership bitmasks, from which a warp writes a class's members in vertex
// order with a popcount scan over n / 32 words; without them it tests every
// vertex for the class.
__global__ void __launch_bounds__(MC_THREADS) k_classes_multi(tc_kparams P, int masks) {
    // k_gsum reads the pair matrix of k_pairs before its own wait: it may
    // start only once this kernel's predecessors are complete
    pdl_wait();
    pdl_trigger();
    if (P.commit && P.st->stop) return;
    __shared__ int s_hist[TC_MAX_K];
    __shared__ int s_off[TC_MAX_K + 1];
    const int n = P.n, k = P.k, d = blockIdx.x, cmax = P.cmax;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwp = MC_THREADS / 32;
    const uint16_t* cmd = P.cm + (size_t)d * n * cmax;
    uint32_t* rd = P.rec + (size_t)d * P.rec_stride;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        s_hist[j] = 0;
        tc_rec_E(rd, P.perm_stride, k)[j] = 0.0f;
    }
    extern __shared__ uint32_t mk[];  // masks: bit b of mk[j aw + w]: vertex 32 w + b has colour j
    const int aw = P.adj_words;
    if (masks)
        for (int e = threadIdx.x; e < k * aw; e += blockDim.x) mk[e] = 0u;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int c = P.dem[i];
        for (int q = 0; q < c; ++q) {
            const int col = cmd[(size_t)i * cmax + q];
            atomicAdd(&s_hist[col], 1);
            if (masks) atomicOr(&mk[col * aw + (i >> 5)], 1u << (i & 31));
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // padded exclusive scan (k <= TC_MAX_K, once per individual)
        int run = 0;
        for (int j = 0; j < k; ++j) {
            s_off[j] = run;
            run += (s_hist[j] + 3) & ~3;
        }
        s_off[k] = run;
        P.feq[d] = 0;
        P.fcolor[d] = 0;  // k_gsum counts the conflicts over these class lists
    }
    __syncthreads();
    int* od = tc_rec_off(rd, P.perm_stride);
    uint32_t* pd = rd;
    for (int j = threadIdx.x; j <= k; j += blockDim.x) od[j] = s_off[j];
    // a warp per class, members in vertex order
    for (int j = warp; j < k; j += nwp) {
        int pos = s_off[j];
        if (masks) {  // lane w: the members in word w, after those of the lower words
            for (int w0 = 0; w0 < aw; w0 += 32) {
                const int w = w0 + lane;
                uint32_t bits = w < aw ? mk[j * aw + w] : 0u;
                const int cnt = __popc(bits);
                int incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                for (int q = pos + incl - cnt; bits; bits &= bits - 1u, ++q)
                    pd[q] = (uint32_t)(32 * w + __ffs(bits) - 1);
                pos += __shfl_sync(0xffffffffu, incl, 31);
            }
        } else {  // vertices in order, members compacted by ballot
            for (int base = 0; base < n; base += 32) {
                const int i = base + lane;
                const bool in = i < n && has_colour(cmd + (size_t)i * cmax, P.dem[i], j);
                const unsigned m = __ballot_sync(0xffffffffu, in);
                if (in) pd[pos + __popc(m & ((1u << lane) - 1u))] = (uint32_t)i;
                pos += __popc(m);
            }
        }
        for (int q = pos + lane; q < s_off[j + 1]; q += 32) pd[q] = (uint32_t)n;  // padding entries
    }
}

}  // namespace

cudaError_t tc_launch_assign_multi(const tc_kparams& P, int clear_old, cudaStream_t s) {
    const int nT = (P.n + TC_WT - 1) / TC_WT;
    const long long rows = (long long)P.D * nT * TC_WT;
    k_assign_multi<<<(unsigned)((rows + MC_THREADS - 1) / MC_THREADS), MC_THREADS, 0, s>>>(P, clear_old);
    return cudaGetLastError();
}

cudaError_t tc_launch_classes_multi(const tc_kparams& P, cudaStream_t s) {
    const long long mask_bytes = 4ll * P.k * P.adj_words;
    const int masks = mask_bytes <= 96 * 1024 ? 1 : 0;
    const int smem = masks ? (int)mask_bytes : 0;
    if (masks) {
        cudaError_t e = cudaFuncSetAttribute(k_classes_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    return tc_launch_pdl(k_classes_multi, dim3(P.D), dim3(MC_THREADS), smem, s, P, masks);
}
