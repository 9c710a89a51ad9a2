// One-hot form of the TensCol iteration (Algorithm 1 of Goudet, Duval, Hao):
// every product with the one-hot population S is computed as the gather or
// compare it reduces to, never as a dense contraction.
//
//   k_pairs    Step 2 + Step 3-i: for every vertex pair (i, m) of the upper
//              triangle, m~_im = #{d : c_d(i) = c_d(m)} (eq. 4) by packed
//              16-bit colour compares; per-individual conflicts f_color (eq. 1)
//              from the equal colours on edges; the pair coefficient
//              B_im = a_im (1 + 2 alpha lambda t m~^(alpha-1))
//                     - (1 - a_im) 2 beta mu t m~^(beta-1)
//              of eq. 13 (A.S and both population terms in one matrix);
//              partial sums of kappa (eq. 5) and varpi (eq. 6).
//   k_classes  per individual: colour-class sizes #V_{d,j}, f_eq (eq. 3), the
//              equity gradient sign (eq. 14), a stable counting sort of the
//              vertices by colour; the last block reduces the population
//              (min_d f, best-so-far, loss of eq. 7, stop rule).
//   k_update   Step 3-ii + Step 4 fused: grad_S L[d,i,j] = sum of B_im over
//              the colour class j of individual d (a segment sum over the
//              sorted vertices) + nu t E_dj, then the softmax straight-through
//              step of eq. 10-12, W -= eta grad, smoothing (eq. 8) and the
//              next Step 1 argmax, one 32-vertex tile of one individual per
//              warp, W streamed through shared memory once.
#include <limits.h>
#include <algorithm>
#include <math.h>
#include <stdio.h>

#include "tc_internal.cuh"

#ifndef TC_BOUNDS
#define TC_BOUNDS 0  // 1: device-side index checks of the class walk (libtenscol_bounds.so)
#endif

namespace {

constexpr int PT = 32;              // pair tile edge
constexpr int PP = PT / 16;         // pairs per thread along each tile edge
constexpr int PAIR_THREADS = 256;   // 16 x 16 threads, PP x PP pairs each
constexpr int PAIR_CW = 64;         // colour words per chunk (< 256: lane counters)
constexpr int CLS_THREADS = 256;
constexpr int UPD_GW = 4;          // k_update: warps per item, each a quarter of the colours
constexpr int UPD_MAX_WARPS = 21;  // a producer warp and 5 groups

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// Initial weights: W ~ N(0, sigma0) (Section 3.2).  Philox4x32-10 as defined
// by Salmon, Moraes, Dror, Shaw (SC'11): 10 rounds of the 4x32 S-box with
// multipliers 0xD2511F53 / 0xCD9E8D57 and Weyl key increments 0x9E3779B9 /
// 0xBB67AE85.  Counter = (g mod 2^32, g div 2^32, 0, 0) for the 4-element
// group g, key = (seed mod 2^32, seed div 2^32); the four 32-bit outputs
// become two Box-Muller pairs.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ float u01(uint32_t x) {  // (0, 1), exact in float
    return ((float)(x >> 8) + 0.5f) * (1.0f / 16777216.0f);
}

// Element e of the standard D x n x k order draws from Philox counter e / 4
// (lane e % 4), whatever layout the values are stored in.
__global__ void k_init_weights(float* W, int D, int n, int k, unsigned long long seed, float sigma0) {
    const long long count = (long long)D * n * k;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g * 4 >= count) return;
    const uint4 r = philox4x32_10(make_uint4((uint32_t)g, (uint32_t)(g >> 32), 0u, 0u),
                                  (uint32_t)seed, (uint32_t)(seed >> 32));
    float z[4];
    {
        const float rad = sqrtf(-2.0f * logf(u01(r.x)));
        float s, c;
        sincospif(2.0f * u01(r.y), &s, &c);
        z[0] = rad * c;
        z[1] = rad * s;
    }
    {
        const float rad = sqrtf(-2.0f * logf(u01(r.z)));
        float s, c;
        sincospif(2.0f * u01(r.w), &s, &c);
        z[2] = rad * c;
        z[3] = rad * s;
    }
    const int nT = (n + TC_WT - 1) / TC_WT;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const long long e = g * 4 + q;
        if (e >= count) break;
        const long long row = e / k;
        const int j = (int)(e - row * k), d = (int)(row / n), i = (int)(row - (long long)d * n);
        W[tc_w_index(d, i, j, nT, k)] = z[q] * sigma0;
    }
}

// Standard (D x n x k) <-> tile-transposed weights, one thread per tiled
// element (padding rows: written as 0 going in, skipped coming out).
__global__ void k_w_layout(const float* src, float* dst, int D, int n, int k, bool to_tiled) {
    const int nT = (n + TC_WT - 1) / TC_WT;
    const long long total = (long long)D * nT * k * TC_WT;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int r = (int)(t % TC_WT);
    const long long q = t / TC_WT;
    const int j = (int)(q % k);
    const long long dT = q / k;
    const int d = (int)(dT / nT), i = (int)(dT % nT) * TC_WT + r;
    const size_t e = ((size_t)d * n + i) * k + j;
    if (to_tiled)
        dst[t] = i < n ? src[e] : 0.f;
    else if (i < n)
        dst[e] = src[t];
}

// The same conversion one (individual, 32-row tile) per block: the tile's
// rows are one contiguous block of 32 k weights in either layout, so both
// sides are read and written in whole lines (host memory reached over the
// chip-to-chip link included), the transpose going through shared memory
// (32 x (k + 1) floats: an odd row stride for even k, so neither phase has
// bank conflicts worth counting).
__global__ void k_w_tiles(const float* src, float* dst, int n, int k, bool to_tiled) {
    extern __shared__ float tl[];
    const int nT = (n + TC_WT - 1) / TC_WT;
    const long long b = blockIdx.x;  // d nT + T
    const int d = (int)(b / nT), T = (int)(b - (long long)d * nT);
    const int rows = min(TC_WT, n - T * TC_WT), ld = k + 1;
    const size_t s0 = ((size_t)d * n + (size_t)T * TC_WT) * k, t0 = (size_t)b * k * TC_WT;
    if (to_tiled) {
        for (int e = threadIdx.x; e < rows * k; e += blockDim.x) {
            const int r = e / k;
            tl[r * ld + (e - r * k)] = src[s0 + e];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < TC_WT * k; e += blockDim.x) {
            const int j = e / TC_WT, r = e - j * TC_WT;
            dst[t0 + e] = r < rows ? tl[r * ld + j] : 0.f;
        }
    } else {
        for (int e = threadIdx.x; e < TC_WT * k; e += blockDim.x) {
            const int j = e / TC_WT, r = e - j * TC_WT;
            tl[r * ld + j] = src[t0 + e];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < rows * k; e += blockDim.x) {
            const int r = e / k;
            dst[s0 + e] = tl[r * ld + (e - r * k)];
        }
    }
}

// Step 1 (Section 3.4) for a fresh W: c_d(i) = lowest j with maximal w.
// ---------------------------------------------------------------------------
// old: the colour being replaced (the bit planes change by its difference)
__device__ __forceinline__ void store_colour(const tc_kparams& P, int d, int i, int old, int c) {
    if (P.planes && old != c) {
        const unsigned x = (unsigned)(old ^ c), bit = 1u << (d & 31);
        uint32_t* w = P.planes + ((size_t)i * P.png + (d >> 5)) * 8;
        for (int p = 0; p < 7; ++p)
            if ((x >> p) & 1u) atomicXor(w + p, bit);
    }
    P.c[(size_t)d * P.n + i] = (uint16_t)c;
    if (P.ct_bytes == 1)
        reinterpret_cast<uint8_t*>(P.cT)[(size_t)i * P.Dp + d] = (uint8_t)c;
    else
        P.cT[(size_t)i * P.Dp + d] = (uint16_t)c;
}

__global__ void k_assign(tc_kparams P) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (long long)P.D * P.n) return;
    const int d = (int)(r / P.n), i = (int)(r % P.n);
    const float* w = P.W + tc_w_index(d, i, 0, (P.n + TC_WT - 1) / TC_WT, P.k);
    int best = 0;
    float bv = w[0];
    for (int j = 1; j < P.k; ++j) {
        const float v = w[j * TC_WT];
        if (v > bv) {
            bv = v;
            best = j;
        }
    }
    store_colour(P, d, i, best, best);  // (the planes are rebuilt after the assignment)
}

// ---------------------------------------------------------------------------
// k_pairs: one 32x32 tile (I <= M) of vertex pairs per block, 2x2 pairs per
// thread.  Colours are packed 4 (8-bit, k <= 255) or 2 (16-bit) to a word of
// cT; equal colours are counted without branches: x = a ^ b has a zero lane
// exactly where the colours agree, ~(((x & 0x7f..) + 0x7f..) | x) sets the
// top bit of precisely those lanes (no carry crosses a lane), and a dp4a
// with 0x01010101 adds the marked bytes: 128 per equal colour.  C7 (8-bit
// lanes, k <= 128): colours fit in 7 bits and the padding slots (all ones)
// cancel in x, so no lane of x has its top bit set, x & 0x7f.. is x and the
// mark is ~(x + 0x7f..) & 0x80.. (one operation fewer per word).
// ---------------------------------------------------------------------------
// FRONT: a pair block of k_front (the class blocks run in the same launch):
// it lets k_gsum start once its pair coefficients are written and fenced.
template <int CB, bool C7, bool DN, bool FRONT>  // DN: M~ comes from the dense forms' GEMM
__device__ __forceinline__ void pairs_block(const tc_kparams& P, int blk) {
    static_assert(!C7 || CB == 1, "7-bit colours are packed in bytes");
    pdl_wait();  // colours from the previous k_update (dense forms: M~ from the GEMM)
    // k_classes reads the colours before its own wait: it may start only
    // once this kernel's predecessors are complete
    if (!FRONT) pdl_trigger();
    const int2 tile = P.pair_tiles[blk];
    if (P.commit && P.st->stop) {
        // the dense forms' M~ accumulates by reduce-adds: every block leaves
        // its entries zero for the next GEMM, also when it has nothing to do
        if (DN)
            for (int e = threadIdx.x; e < PT * PT; e += PAIR_THREADS) {
                const int i = tile.x * PT + e / PT, m = tile.y * PT + e % PT;
                if (i < P.n && m < P.n) {
                    P.M32[(size_t)i * P.ldm + m] = 0.f;
                    P.M32[(size_t)m * P.ldm + i] = 0.f;
                }
            }
        return;
    }
    // colour words of the tile's rows (odd stride: the column reads are free
    // of bank conflicts), or their bit planes at a 68-word stride (16-byte rows)
    __shared__ __align__(16) uint32_t s_a[PT][PAIR_CW + 5];
    __shared__ __align__(16) uint32_t s_b[PT][PAIR_CW + 5];
    __shared__ float s_red[2][PAIR_THREADS / 32];
    constexpr uint32_t LOW = CB == 1 ? 0x7F7F7F7Fu : 0x7FFF7FFFu;
    constexpr uint32_t HIGH = CB == 1 ? 0x80808080u : 0x80008000u;

    const int n = P.n, D = P.D;
    const int I = tile.x, M = tile.y;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int Dw = P.Dp * CB / 4;
    const uint32_t* cTw = reinterpret_cast<const uint32_t*>(P.cT);

    uint32_t wide[PP][PP];
    int mis[PP][PP];  // bit-plane path: individuals whose colours differ
#pragma unroll
    for (int a = 0; a < PP; ++a)
#pragma unroll
        for (int b = 0; b < PP; ++b) {
            wide[a][b] = 0u;
            mis[a][b] = 0;
        }
    constexpr bool from_gemm = DN;  // dense form: M~ came from a GEMM
    const bool planes = C7 && !from_gemm && P.planes != nullptr;
    if (planes) {
        // 32 individuals at a time: the colours of i and m agree in individual
        // d exactly when no bit plane differs at bit d, so the OR of the seven
        // planes' XORs marks the individuals that differ (absent individuals
        // have all planes 0 for every vertex: they never differ)
        constexpr int PLS = 68;
        uint32_t* pa = &s_a[0][0];
        uint32_t* pb = &s_b[0][0];
        const int ng = P.png;
        for (int g0 = 0; g0 < ng; g0 += 8) {
            const int gc = min(8, ng - g0);
            __syncthreads();
            for (int e = tid; e < PT * gc * 2; e += PAIR_THREADS) {
                const int r = e / (gc * 2), q = e - r * (gc * 2);
                const int ii = I * PT + r, mm = M * PT + r;
                const uint4 z = make_uint4(0u, 0u, 0u, 0u);
                reinterpret_cast<uint4*>(pa + r * PLS)[q] =
                    ii < n ? __ldg(reinterpret_cast<const uint4*>(P.planes + ((size_t)ii * ng + g0) * 8) + q) : z;
                reinterpret_cast<uint4*>(pb + r * PLS)[q] =
                    mm < n ? __ldg(reinterpret_cast<const uint4*>(P.planes + ((size_t)mm * ng + g0) * 8) + q) : z;
            }
            __syncthreads();
            for (int g = 0; g < gc; ++g) {
                uint4 a0[PP], a1[PP], b0[PP], b1[PP];
#pragma unroll
                for (int r = 0; r < PP; ++r) {
                    const uint4* ar = reinterpret_cast<const uint4*>(pa + (ty + 16 * r) * PLS + 8 * g);
                    const uint4* br = reinterpret_cast<const uint4*>(pb + (tx + 16 * r) * PLS + 8 * g);
                    a0[r] = ar[0];
                    a1[r] = ar[1];
                    b0[r] = br[0];
                    b1[r] = br[1];
                }
#pragma unroll
                for (int a = 0; a < PP; ++a)
#pragma unroll
                    for (int b = 0; b < PP; ++b) {
                        const uint32_t x = (a0[a].x ^ b0[b].x) | (a0[a].y ^ b0[b].y) | (a0[a].z ^ b0[b].z) |
                                           (a0[a].w ^ b0[b].w) | (a1[a].x ^ b1[b].x) | (a1[a].y ^ b1[b].y) |
                                           (a1[a].z ^ b1[b].z);
                        mis[a][b] += __popc(x);
                    }
            }
        }
    }
    for (int w0 = 0; w0 < (from_gemm || planes ? 0 : Dw); w0 += PAIR_CW) {
        const int cw = min(PAIR_CW, Dw - w0);
        __syncthreads();
        for (int e = tid; e < PT * cw; e += PAIR_THREADS) {
            const int r = e / cw, w = e - r * cw;
            const int ii = I * PT + r, mm = M * PT + r;
            s_a[r][w] = ii < n ? cTw[(size_t)ii * Dw + w0 + w] : 0u;
            s_b[r][w] = mm < n ? cTw[(size_t)mm * Dw + w0 + w] : 0u;
        }
        __syncthreads();
        for (int w = 0; w < cw; ++w) {
            uint32_t av[PP], bv[PP];
#pragma unroll
            for (int r = 0; r < PP; ++r) {
                av[r] = s_a[ty + 16 * r][w];
                bv[r] = s_b[tx + 16 * r][w];
            }
#pragma unroll
            for (int a = 0; a < PP; ++a)
#pragma unroll
                for (int b = 0; b < PP; ++b) {
                    const uint32_t x = av[a] ^ bv[b];
                    const uint32_t mark = C7 ? ~(x + LOW) & HIGH : ~(((x & LOW) + LOW) | x) & HIGH;
                    // the byte sum of the marks (0x80 per equal colour): 128
                    // per equal colour, one dp4a instead of a shift and an add
                    wide[a][b] = __dp4a(mark, 0x01010101u, wide[a][b]);
                }
        }
    }

    // pair coefficient of eq. 13 and loss terms of eq. 5-6; the partitioning
    // problems (M_d -> J - M_d, tables over D - m~) negate every term
    const long long t = P.st->t;
    const float cA = (float)((double)P.lambda_ * (double)t);
    const float cB = (float)((double)P.mu * (double)t);
    const float sg = tc_is_partition(P.problem) ? -1.0f : 1.0f;
    const int pad = P.Dp - D;  // padded colour slots always compare equal
    float kap = 0.f, var = 0.f;
    __syncthreads();  // s_a / s_b are reused as transpose tiles
    float(*s_t)[PT + 1] = reinterpret_cast<float(*)[PT + 1]>(&s_a[0][0]);
    int(*s_m)[PT + 1] = reinterpret_cast<int(*)[PT + 1]>(&s_b[0][0]);
    // dense forms: this thread's M~ entries, all loaded before any store (the
    // entries are zeroed after use for the next iteration's reduce-adds)
    int mg[PP][PP];
    if (from_gemm) {
#pragma unroll
        for (int a = 0; a < PP; ++a)
#pragma unroll
            for (int b = 0; b < PP; ++b) {
                const int il = ty + 16 * a, ml = tx + 16 * b, i = I * PT + il, m = M * PT + ml;
                mg[a][b] = (i < n && m < n && (I < M || ml >= il)) ? __float2int_rn(__ldcg(P.M32 + (size_t)i * P.ldm + m))
                                                                   : 0;
            }
    }
#pragma unroll
    for (int a = 0; a < PP; ++a) {
        const int il = ty + 16 * a, i = I * PT + il;
#pragma unroll
        for (int b = 0; b < PP; ++b) {
            const int ml = tx + 16 * b, m = M * PT + ml;
            float bb = 0.f;
            int mt = 0;
            if (i < n && m < n && (I < M || ml >= il)) {
                if (from_gemm) {
                    mt = mg[a][b];
                    P.M32[(size_t)i * P.ldm + m] = 0.f;
                } else {
                    mt = planes ? D - mis[a][b] : (int)(wide[a][b] >> 7) - pad;
                }
                // a count of shared colours: the tables hold mt_max + 1 entries
                mt = min(max(mt, 0), P.mt_max);
                const bool edge = (P.adj[(size_t)i * P.adj_words + (m >> 5)] >> (m & 31)) & 1u;
                if (m == i) {
                    // m~_ii: D (one colour per vertex), from the GEMM D c_i in the multicolouring
                    if (!from_gemm) mt = D;
                    if (P.bonus_diag) {
                        bb = -sg * (cB * P.lutB[mt]);
                        var += P.powB[mt];
                    }
                } else if (edge) {
                    // the A.S term enters through B only in the one-hot form
                    bb = sg * (from_gemm ? cA * P.lutA[mt] : fmaf(cA, P.lutA[mt], 1.0f));
                    kap += 2.0f * P.powA[mt];
                } else {
                    bb = -sg * (cB * P.lutB[mt]);
                    var += 2.0f * P.powB[mt];
                }
                P.B[(size_t)i * P.ldb + m] = bb;
                if (P.dbg_Mt) P.dbg_Mt[(size_t)i * n + m] = mt;
            }
            s_t[ml][il] = bb;
            s_m[ml][il] = mt;
        }
    }
    __syncthreads();
    // transposed counterpart B[m][i] = B[i][m] for the strictly-lower half
    for (int e = tid; e < PT * PT; e += PAIR_THREADS) {
        const int ml = e / PT, il = e % PT;
        const int mm = M * PT + ml, ii = I * PT + il;
        if (mm < n && ii < n && (I < M || il < ml)) {
            P.B[(size_t)mm * P.ldb + ii] = s_t[ml][il];
            if (from_gemm) P.M32[(size_t)mm * P.ldm + ii] = 0.f;  // the GEMM's tiles reach below the diagonal
            if (P.dbg_Mt) P.dbg_Mt[(size_t)mm * n + ii] = s_m[ml][il];
        }
    }
    // block partial sums (fixed order -> deterministic)
    kap = warp_sum(kap);
    var = warp_sum(var);
    if ((tid & 31) == 0) {
        s_red[0][tid >> 5] = kap;
        s_red[1][tid >> 5] = var;
    }
    __syncthreads();
    if (tid == 0) {
        float ka = 0.f, va = 0.f;
        for (int q = 0; q < PAIR_THREADS / 32; ++q) {
            ka += s_red[0][q];
            va += s_red[1][q];
        }
        P.loss_part[2 * blk] = ka;
        P.loss_part[2 * blk + 1] = va;
    }
    if (FRONT) {  // k_gsum reads B before its own wait
        __threadfence();
        __syncthreads();
        pdl_trigger();
    }
}

template <int CB, bool C7, bool DN>
__global__ void __launch_bounds__(PAIR_THREADS) k_pairs(tc_kparams P) {
    pairs_block<CB, C7, DN, false>(P, blockIdx.x);
}

// ---------------------------------------------------------------------------
// block-wide helpers (any block size up to 1024 threads)
// ---------------------------------------------------------------------------
template <typename T>
__device__ T block_sum(T v, T* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    T s = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += sh[q];
    return s;
}



// ---------------------------------------------------------------------------
// k_classes: one individual per block.  Class sizes, equity (eq. 3, eq. 14)
// and a stable counting sort of the vertices by colour into `perm` with every
// class padded to a multiple of 4 entries (padding = vertex n, a zero row of
// the pair matrix) and the class order of k_gsum's slot walk.  Dynamic
// shared memory: the individual's colours, then the per-warp colour counts of
// the sort.
// ---------------------------------------------------------------------------
// FRONT: a class block of k_front, launched with the pair blocks: it waits
// for the previous k_update at its start and does not hold k_gsum back
// (k_gsum reads the class lists only after its own wait).
template <bool FRONT>
__device__ __forceinline__ void classes_block(const tc_kparams& P, int d) {
    // Launched once k_pairs has passed its own wait, so the colours of the
    // previous update (and the stop flag) are final: the class lists need
    // nothing from k_pairs and are built while it runs.  The wait for k_pairs
    // comes at the end, before this kernel lets k_gsum start (k_gsum reads
    // the pair matrix of k_pairs before its own wait).
    if (FRONT) {
        pdl_wait();
        pdl_trigger();
    }
    if (P.commit && P.st->stop) {
        if (!FRONT) pdl_wait();
        return;
    }
    __shared__ int s_hist[TC_MAX_K];
    __shared__ int s_cur[TC_MAX_K];
    __shared__ int s_scan[64];
    __shared__ int s_bk[64];
    __shared__ long long sh_ll[CLS_THREADS / 32];
    extern __shared__ __align__(16) uint32_t s_dyn[];
    const int n = P.n, k = P.k;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwp = CLS_THREADS / 32;
    uint16_t* cs = reinterpret_cast<uint16_t*>(s_dyn);  // n colours
    int* wcnt = reinterpret_cast<int*>(s_dyn + ((n + 7) / 8) * 4);  // after the colours: nwp x k counts
    const uint16_t* cd = P.c + (size_t)d * n;
    for (int j = threadIdx.x; j < k; j += blockDim.x) s_hist[j] = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const uint16_t c = cd[i];
        cs[i] = c;
        // the adjacency-list walk of k_update reads this iteration's colours
        // while k_update overwrites c with the next ones: give it a snapshot
        if (P.csr_walk) P.c_snap[(size_t)d * n + i] = c;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&s_hist[cs[i]], 1);
    for (int b = threadIdx.x; b < 64; b += blockDim.x) s_bk[b] = 0;
    __syncthreads();
    // the class order of k_gsum's slot walk: classes by decreasing padded
    // length (in 4-entry chunks; 63 chunks or more share the first bucket),
    // by colour within a bucket (a stable, run-independent order)
    auto bucket = [&](int j) { return 63 - min((s_hist[j] + 3) >> 2, 63); };
    for (int j = threadIdx.x; j < k; j += blockDim.x) atomicAdd(&s_bk[bucket(j)], 1);
    __syncthreads();
    if (warp == 0) {  // exclusive scan of the 64 bucket counts, two per lane
        const int a0 = s_bk[2 * lane], a1 = s_bk[2 * lane + 1];
        int incl = a0 + a1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        s_bk[2 * lane] = incl - a0 - a1;
        s_bk[2 * lane + 1] = incl - a1;
    }
    __syncthreads();
    if (warp == 0) {  // stable scatter, 32 classes at a time (ranks among equal buckets by warp matching)
        uint16_t* cod = tc_rec_cord(P.rec + (size_t)d * P.rec_stride, P.perm_stride, k);
        for (int j0 = 0; j0 < k; j0 += 32) {
            const int j = j0 + lane;
            const unsigned valid = __ballot_sync(0xffffffffu, j < k);
            if (j < k) {
                const int b = bucket(j);
                const unsigned peers = __match_any_sync(valid, b);
                cod[s_bk[b] + __popc(peers & ((1u << lane) - 1u))] = (uint16_t)j;
                __syncwarp(valid);
                if ((__ffs(peers) - 1) == lane) s_bk[b] += __popc(peers);
            }
            __syncwarp();
        }
    }
    // exclusive scan of the padded class sizes: contiguous chunks per thread,
    // warp shuffles, then the warp totals
    const int per = (k + CLS_THREADS - 1) / CLS_THREADS;
    const int j0 = threadIdx.x * per, j1 = min(k, j0 + per);
    int local = 0;
    for (int j = j0; j < j1; ++j) local += (s_hist[j] + 3) & ~3;
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) s_scan[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int wt = lane < nwp ? s_scan[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, wt, o);
            if (lane >= o) wt += v;
        }
        if (lane < nwp) s_scan[32 + lane] = wt;  // inclusive warp totals
    }
    __syncthreads();
    int run = (warp > 0 ? s_scan[32 + warp - 1] : 0) + incl - local;
    uint32_t* rd = P.rec + (size_t)d * P.rec_stride;
    int* od = tc_rec_off(rd, P.perm_stride);
    uint32_t* pd = rd;
    float* Ed = tc_rec_E(rd, P.perm_stride, k);
    if (threadIdx.x < 4) tc_rec_zchunk(rd, P.perm_stride, k)[threadIdx.x] = (uint32_t)n;
    for (int j = j0; j < j1; ++j) {
        const int h = s_hist[j], ph = (h + 3) & ~3;
        od[j] = run;
        s_cur[j] = run;
        for (int q = h; q < ph; ++q) pd[run + q] = (uint32_t)n;  // padding entries
        run += ph;
    }
    if (threadIdx.x == CLS_THREADS - 1) od[k] = s_scan[32 + nwp - 1];
    // the additive fitness term and its gradient factor: equity (eq. 3)
    // with the sign of eq. 14, or for the minimum sum colouring the colour
    // costs f_mscp = sum_j #V_{d,j} z_j, whose gradient is z_j (Section 6)
    const int c1 = n / k, c2 = (n + k - 1) / k;
    const bool mscp = P.problem == TC_MSCP;
    long long fe = 0;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        const int h = s_hist[j];
        if (mscp) {
            const int z = __ldg(P.zcost + j);
            fe += (long long)h * z;
            Ed[j] = (float)z;
        } else {
            fe += min(abs(h - c1), abs(h - c2));
            Ed[j] = h > c2 ? 1.0f : (h < c1 ? -1.0f : 0.0f);
        }
    }
    fe = block_sum<long long>(fe, sh_ll);
    if (threadIdx.x == 0) P.feq[d] = (int)fe;
    __syncthreads();
    // stable counting sort: each warp owns a contiguous chunk of vertices;
    // per-warp colour counts give every (warp, colour) its base, ranks within
    // 32-vertex rounds come from warp matching
    for (int e = threadIdx.x; e < nwp * k; e += blockDim.x) wcnt[e] = 0;
    __syncthreads();
    const int chunk = (n + nwp - 1) / nwp;
    const int cbeg = min(n, warp * chunk), cend = min(n, cbeg + chunk);
    for (int base = cbeg; base < cend; base += 32) {
        const int i = base + lane;
        const unsigned valid = __ballot_sync(0xffffffffu, i < cend);
        if (i < cend) {
            const int col = cs[i];
            const unsigned peers = __match_any_sync(valid, col);
            if ((__ffs(peers) - 1) == lane) wcnt[warp * k + col] += __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        int r = s_cur[j];
        for (int w = 0; w < nwp; ++w) {
            const int c = wcnt[w * k + j];
            wcnt[w * k + j] = r;
            r += c;
        }
    }
    __syncthreads();
    for (int base = cbeg; base < cend; base += 32) {
        const int i = base + lane;
        const unsigned valid = __ballot_sync(0xffffffffu, i < cend);
        if (i < cend) {
            const int col = cs[i];
            const unsigned peers = __match_any_sync(valid, col);
            const int rank = __popc(peers & ((1u << lane) - 1u));
            pd[wcnt[warp * k + col] + rank] = (uint32_t)i;
            __syncwarp(valid);
            if ((__ffs(peers) - 1) == lane) wcnt[warp * k + col] += __popc(peers);
        }
        __syncwarp();
    }
    // conflicts (eq. 1) are counted by k_gsum, which walks these class lists
    if (threadIdx.x == 0) P.fcolor[d] = 0;
#if TC_BOUNDS
    __syncthreads();  // the sort's entries are written
    if (P.dbg_plant && d == 0 && threadIdx.x == 0) pd[0] = (uint32_t)(n + 1);  // TC_FAULT=index
#endif
    if (!FRONT) {
        pdl_wait();
        pdl_trigger();
    }
}

__global__ void __launch_bounds__(CLS_THREADS) k_classes(tc_kparams P) { classes_block<false>(P, blockIdx.x); }

// k_front (one-hot form): the colour classes (the first D blocks,
// classes_block) and Step 3-i with the pair coefficients (the n_pair_blocks
// after them, pairs_block) in one launch.  The class blocks are short and
// latency-bound, the pair blocks long and ALU-bound: dispatched first, the
// class blocks' warps are the older ones an SM's schedulers favour, so their
// chain of barriers runs in the pair blocks' shadow instead of after them.
template <int CB, bool C7>
__global__ void __launch_bounds__(PAIR_THREADS) k_front(tc_kparams P) {
    static_assert(PAIR_THREADS == CLS_THREADS, "one block size for both roles");
    if ((int)blockIdx.x < P.D)
        classes_block<true>(P, (int)blockIdx.x);
    else
        pairs_block<CB, C7, false, true>(P, (int)blockIdx.x - P.D);
}


// ---------------------------------------------------------------------------
// Step 3-ii and Step 4 run as two kernels over (32-vertex tile, individual)
// items, tile-major:
//   k_gsum    grad_S L of eq. 13 for the item's 32 vertices and all k colours
//             into Gbuf[item][j][lane] (coalesced 128-byte rows).  A block
//             owns a contiguous run of items and keeps the tile's 32 columns
//             of B in shared memory (2-D TMA boxes); each warp sums B over the
//             individual's colour classes, one vertex per lane.
//   k_update  streams the item's grad_S tile and its 32 x k weight rows into
//             shared memory with bulk async copies, lane r of four warps
//             updates row r (softmax, straight-through gradient of eq. 12,
//             descent step, smoothing of eq. 8, the next argmax) and the rows
//             go back with a bulk async store.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// try_wait with a suspend-time hint: a thread whose phase is not complete
// sleeps (up to `ns` nanoseconds) until it completes instead of spinning.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, unsigned parity, unsigned ns) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait: the thread sleeps in try_wait (up to 20 us per attempt) until
// the phase completes; gives up after `limit_ns` (the context's wait limit,
// one second by default) and reports TC_ERR_TIMEOUT.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, int* err,
                                                  unsigned long long limit_ns = 1000000000ull) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    const unsigned hint = limit_ns < 20000ull ? (unsigned)limit_ns : 20000u;
    for (;;) {
        if (mbar_try_wait_sleep(bar, parity, hint)) return true;
        if (global_ns() - t0 > limit_ns) break;
    }
    atomicCAS(err, 0, TC_ERR_TIMEOUT);
    return false;
}

// L2 eviction policy for the bytes that k_update moves once (the weight
// tiles it reads and writes back, the grad_S tiles it reads): they go first,
// so the grad_S tiles that k_gsum has just written stay in L2 longer
// (k_update 43.5 -> 40.0 us at the benchmark shape; marking k_gsum's stores
// evict_last as well slowed k_gsum by as much).
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ void bulk_load_hint(void* smem_dst, const void* gsrc, unsigned bytes, uint64_t* bar,
                                               uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
            "r"(smem_u32(smem_dst)),
        "l"(gsrc), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

__device__ __forceinline__ void bulk_load(void* smem_dst, const void* gsrc, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(smem_dst)),
                 "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void bulk_store_hint(void* gdst, const void* smem_src, unsigned bytes, uint64_t pol) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;" ::"l"(gdst),
                 "r"(smem_u32(smem_src)), "r"(bytes), "l"(pol)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

__device__ __forceinline__ void pair_sync(int pair) {  // warps 2 pair, 2 pair + 1 (named barrier pair + 1)
    asm volatile("bar.sync %0, 64;" ::"r"(pair + 1) : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// grad_S L of one vertex (i0 + lane) for every colour of one individual
// (eq. 13): class j occupies the padded range [of[j], of[j+1]) of the
// colour-sorted vertices (length a multiple of 4; padding is vertex n, a zero
// row of B), so a class is a loop of 4-wide chunks: one 16-byte index load
// and four independent loads of B.  BS > 0: B rows BS floats apart (the
// shared panel), else `bstride`.  STG: pm, of and xs (= E_dj) are the
// warp's shared-memory copies; else pm, of in global memory and xs unused
// (Ed gives E).  Gout[j * 32] receives the class sum +
// nu t E_dj (+ gs times the gamma-matrix entry in the dense forms: gs = -1 for
// the partitioning problems, whose A.S term changes sign).
template <int BS, bool STG>
__device__ __forceinline__ void class_sums(const uint32_t* pm, const int* of, const float* xs, const float* Ed,
                                           const uint16_t* grow, float gs, int gstride, const float* Bl,
                                           int bstride, float nut, int k, int jb, int je, float* Gout) {
    const int bs = BS > 0 ? BS : bstride;
    if (jb >= je) return;
    int s = STG ? of[jb] : __ldg(of + jb);
    int e = STG ? of[jb + 1] : __ldg(of + jb + 1);
    // gamma entries travel 4 classes ahead of use (an L2 round trip each)
    uint16_t g0 = 0, g1 = 0, g2 = 0, g3 = 0;
    if (grow) {
        g0 = __ldg(grow + (size_t)jb * gstride);
        if (jb + 1 < je) g1 = __ldg(grow + (size_t)(jb + 1) * gstride);
        if (jb + 2 < je) g2 = __ldg(grow + (size_t)(jb + 2) * gstride);
        if (jb + 3 < je) g3 = __ldg(grow + (size_t)(jb + 3) * gstride);
    }
    for (int j = jb; j < je; ++j) {
        int e_next;
        float extra;
        if (STG) {
            e_next = of[j + 2 <= k ? j + 2 : k];
            extra = nut * xs[j];
        } else {
            e_next = (j + 2 <= k) ? __ldg(of + j + 2) : 0;  // next bound, ahead of use
            extra = nut * __ldg(Ed + j);
        }
        if (grow) {
            extra += gs * (float)g0;
            g0 = g1;
            g1 = g2;
            g2 = g3;
            g3 = j + 4 < je ? __ldg(grow + (size_t)(j + 4) * gstride) : (uint16_t)0;
        }
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll 2
        for (int p = s; p < e; p += 4) {
            const uint4 v = STG ? *reinterpret_cast<const uint4*>(pm + p)
                                : __ldg(reinterpret_cast<const uint4*>(pm + p));
            a0 += Bl[(int)v.x * bs];
            a1 += Bl[(int)v.y * bs];
            a2 += Bl[(int)v.z * bs];
            a3 += Bl[(int)v.w * bs];
        }
        // (B from global memory: the grad_S tiles stream past L2, which then
        // keeps more of B's columns)
        if (BS == 0)
            __stcs(Gout + j * 32, ((a0 + a1) + (a2 + a3)) + extra);
        else
            Gout[j * 32] = ((a0 + a1) + (a2 + a3)) + extra;
        s = e;
        e = e_next;
    }
}

// class_sums for the hot configuration (the tile's B columns and the item's
// lists both in shared memory), given as 32-bit shared addresses: the B
// entry of vertex v for this lane sits at bl + 128 v.
__device__ __forceinline__ void class_sums_shared(uint32_t pm, const int* of, const float* xs, float nut,
                                                  const uint16_t* grow, float gs, int gstride, uint32_t bl, int k,
                                                  int jb, int je, float* Gout) {
    if (jb >= je) return;
    // the list and the lane's panel column as pointers into the dynamic shared
    // array: plain indexed loads took 2 % fewer warp instructions per launch
    // than inline-asm shared loads on the 32-bit addresses (55.5 M against 56.7 M)
    extern __shared__ __align__(1024) float sm[];
    const char* list = reinterpret_cast<const char*>(sm) + (pm - smem_u32(sm));
    const float* col = reinterpret_cast<const float*>(reinterpret_cast<const char*>(sm) + (bl - smem_u32(sm)));
    uint32_t p = pm + 4u * (uint32_t)of[jb];
    uint32_t e = pm + 4u * (uint32_t)of[jb + 1];
    uint16_t g0 = 0, g1 = 0, g2 = 0, g3 = 0;  // gamma entries, 4 classes ahead
    if (grow) {
        g0 = __ldg(grow + (size_t)jb * gstride);
        if (jb + 1 < je) g1 = __ldg(grow + (size_t)(jb + 1) * gstride);
        if (jb + 2 < je) g2 = __ldg(grow + (size_t)(jb + 2) * gstride);
        if (jb + 3 < je) g3 = __ldg(grow + (size_t)(jb + 3) * gstride);
    }
    for (int j = jb; j < je; ++j) {
        const uint32_t e_next = pm + 4u * (uint32_t)of[j + 2 <= k ? j + 2 : k];
        float extra = nut * xs[j];
        if (grow) {
            extra += gs * (float)g0;
            g0 = g1;
            g1 = g2;
            g2 = g3;
            g3 = j + 4 < je ? __ldg(grow + (size_t)(j + 4) * gstride) : (uint16_t)0;
        }
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        // not unrolled: classes are ~3 chunks long, and the remainder handling
        // of an unrolled loop cost more than it saved (56.1 M against 59.1 M
        // warp instructions per launch; 60.4 M unrolled by 4)
#pragma unroll 1
        for (; p < e; p += 16) {
            const uint4 v = *reinterpret_cast<const uint4*>(list + (p - pm));
            a0 += col[v.x * 32];
            a1 += col[v.y * 32];
            a2 += col[v.z * 32];
            a3 += col[v.w * 32];
        }
        Gout[j * 32] = ((a0 + a1) + (a2 + a3)) + extra;
        p = e;
        e = e_next;
    }
}

// ---------------------------------------------------------------------------
// Slot walk (the one-hot form's staged walk).  The two warps of a pair split
// into 8 lane groups of 8 lanes; lane l8 of a group covers the tile rows
// 4 l8 .. 4 l8 + 3, so one 16-byte load of panel row m brings
// B[m][4 l8 .. 4 l8 + 3] = B[i][m] for its four rows (B is symmetric) and a
// group's 8 loads of one vertex are one 128-byte line.  k_classes lists each
// individual's classes by decreasing padded length (cord).  Classes of at
// least SW_LONG entries (they come first) are walked one at a time by the
// four groups of a warp; the others form quads, consecutive in that order,
// whose four classes the four groups of a warp walk side by side, so they
// have nearly equal lengths.  The warp loops to the longest of the four; a
// group whose class is shorter reads a chunk of padding vertices (the zero
// row n of B) instead of branching, and all four groups store their class
// sums together at the end of the quad.  Each long class goes to the warp of
// the pair with fewer long-class entries so far; the quads alternate between
// the two warps.
// ---------------------------------------------------------------------------
// One 4-entry chunk of a class walk, on 32-bit shared-memory addresses:
// the chunk's vertex indices v0..v3 at `src`, and for each the 16 bytes
// B[v][4 l8 .. 4 l8 + 3] at colb + 128 v (the lane's four rows of the
// panel row v).  acc01 / acc23 hold the rows' running sums as packed pairs
// (add.rn.f32x2, IEEE per element): acc += (b0 + b1) + (b2 + b3) per row.
__device__ __forceinline__ void walk_chunk(uint32_t src, uint32_t colb, uint64_t& acc01, uint64_t& acc23) {
    asm volatile(
        "{\n"
        " .reg .u32 v0, v1, v2, v3, a0, a1, a2, a3;\n"
        " .reg .b64 p0, q0, p1, q1, p2, q2, p3, q3, s, t;\n"
        " ld.shared.v4.u32 {v0, v1, v2, v3}, [%2];\n"
        " mad.lo.u32 a0, v0, 128, %3;\n"
        " mad.lo.u32 a1, v1, 128, %3;\n"
        " mad.lo.u32 a2, v2, 128, %3;\n"
        " mad.lo.u32 a3, v3, 128, %3;\n"
        " ld.shared.v2.b64 {p0, q0}, [a0];\n"
        " ld.shared.v2.b64 {p1, q1}, [a1];\n"
        " ld.shared.v2.b64 {p2, q2}, [a2];\n"
        " ld.shared.v2.b64 {p3, q3}, [a3];\n"
        " add.rn.f32x2 s, p0, p1;\n"
        " add.rn.f32x2 t, p2, p3;\n"
        " add.rn.f32x2 s, s, t;\n"
        " add.rn.f32x2 %0, %0, s;\n"
        " add.rn.f32x2 s, q0, q1;\n"
        " add.rn.f32x2 t, q2, q3;\n"
        " add.rn.f32x2 s, s, t;\n"
        " add.rn.f32x2 %1, %1, s;\n"
        "}\n"
        : "+l"(acc01), "+l"(acc23)
        : "r"(src), "r"(colb)
        : "memory");
}

// The four row sums of a class walk (the packed pairs) plus nu t E_dj.
__device__ __forceinline__ float4 walk_result(uint64_t acc01, uint64_t acc23, float ex) {
    float x, y, z, w;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(acc01));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(z), "=f"(w) : "l"(acc23));
    return make_float4(x + ex, y + ex, z + ex, w + ex);
}

// The chunks c = 0, 4, ... < m of entries c0 + c of the class at p0 of the
// list (entries at or past len: the padding chunk); m is the same in the
// whole warp, so the groups run in lockstep.  TC_BOUNDS builds check every
// vertex index against the panel (rows 0 .. n) and skip a chunk that names
// another row, recording TC_ERR_DEVICE_BOUNDS in *err.
__device__ __forceinline__ void walk_chunks(const uint32_t* list, const uint32_t* zchunk, uint32_t lists,
                                            uint32_t zcs, uint32_t colb, int p0, int c0, int len, int m, int nmax,
                                            int* err, uint64_t& a01, uint64_t& a23) {
    const uint32_t srcb = lists + 4u * (uint32_t)(p0 + c0);
#pragma unroll 1
    for (int c = 0; c < m; c += 4) {
        const bool in = c0 + c < len;
#if TC_BOUNDS
        const uint4 v = *reinterpret_cast<const uint4*>(in ? list + p0 + c0 + c : zchunk);
        if (v.x > (uint32_t)nmax || v.y > (uint32_t)nmax || v.z > (uint32_t)nmax || v.w > (uint32_t)nmax) {
            atomicCAS(err, 0, TC_ERR_DEVICE_BOUNDS);
            continue;
        }
#else
        (void)list;
        (void)zchunk;
        (void)nmax;
        (void)err;
#endif
        walk_chunk(in ? srcb + 4u * (uint32_t)c : zcs, colb, a01, a23);
    }
}

// Classes of at least SW_LONG entries lead the class order.  Side by side
// with short classes they would leave three groups of their warp walking
// padding: after the smoothing of Step 4-iv the weights are a hundredth of
// their size, the next update moves about one colour in seven, and a few
// classes of hundreds of vertices follow (the iteration after it took 13 us
// longer in the walk at the benchmark shape).  Each such class is walked by
// the four groups of one warp, a quarter of its chunks each, and their sums
// combined by two shuffles in a fixed order; it goes to the warp of the pair
// with fewer chunks so far (warp 0 on ties), the same choice in both warps.
constexpr int SW_LONG = 32;

// TC_BOUNDS builds check the record the walk reads (class order, offsets,
// vertex indices <= n) and replace what is out of range, recording
// TC_ERR_DEVICE_BOUNDS in *err instead of reading outside the record or panel.
__device__ __forceinline__ bool class_ok(int j, int p0, int len, int k, int plen, int* err) {
#if TC_BOUNDS
    if (j < 0 || j >= k || p0 < 0 || len < 0 || p0 + len > plen || (len & 3)) {
        atomicCAS(err, 0, TC_ERR_DEVICE_BOUNDS);
        return false;
    }
#else
    (void)j;
    (void)p0;
    (void)len;
    (void)k;
    (void)plen;
    (void)err;
#endif
    return true;
}

// The class sum of the four rows plus nu t E_dj, plus in the dense forms
// gs times the gamma-matrix entries of the four rows (gam: colour j of rows
// 4 l8 .. 4 l8 + 3 at gam + j gstride + 4 l8, four uint16).
template <bool GM>
__device__ __forceinline__ float4 class_result(float4 r, float ex, const uint16_t* gam, int gstride, float gs, int j,
                                               int l8) {
    r = make_float4(r.x + ex, r.y + ex, r.z + ex, r.w + ex);
    if (GM) {
        const uint2 g = __ldg(reinterpret_cast<const uint2*>(gam + (size_t)j * gstride + 4 * l8));
        r.x += gs * (float)(g.x & 0xffffu);
        r.y += gs * (float)(g.x >> 16);
        r.z += gs * (float)(g.y & 0xffffu);
        r.w += gs * (float)(g.y >> 16);
    }
    return r;
}

// Returns the number of long classes.  GM: the dense forms, whose pair
// matrix leaves out the A.S term; it is added from the gamma matrix (gam).
template <bool GM>
__device__ __forceinline__ int slot_walk(const uint32_t* list, const int* of, const uint16_t* cord,
                                          const float* xs, const uint32_t* zchunk, float nut, const float* panel,
                                          int k, int h, int lane, float* gtile, int nmax, int plen, int* err,
                                          const uint16_t* gam, int gstride, float gs) {
    const int grp = lane >> 3, l8 = lane & 7;
    const uint32_t colb = smem_u32(panel) + 16u * (uint32_t)l8, lists = smem_u32(list), zcs = smem_u32(zchunk);
    int nlong = 0;
    while (nlong < k) {
        const int j = cord[nlong];
#if TC_BOUNDS
        if (j >= k) break;  // reported by the slots below
#endif
        if (of[j + 1] - of[j] < SW_LONG) break;
        ++nlong;
    }
    int w0 = 0, w1 = 0;  // chunks per group given to each warp
    for (int i = 0; i < nlong; ++i) {
        const int j = cord[i], p0 = of[j], len = of[j + 1] - p0;
        if (!class_ok(j, p0, len, k, plen, err)) continue;
        const int per = 4 * (((len >> 2) + 3) >> 2);  // entries per group
        const int w = w1 < w0 ? 1 : 0;
        if (w)
            w1 += per;
        else
            w0 += per;
        if (w != h) continue;
        uint64_t a01 = 0ull, a23 = 0ull;
        walk_chunks(list, zchunk, lists, zcs, colb, p0, grp * per, len, per, nmax, err, a01, a23);
        float4 r = walk_result(a01, a23, -0.0f);  // (x + -0 = x)
        r.x += __shfl_xor_sync(0xffffffffu, r.x, 8);
        r.y += __shfl_xor_sync(0xffffffffu, r.y, 8);
        r.z += __shfl_xor_sync(0xffffffffu, r.z, 8);
        r.w += __shfl_xor_sync(0xffffffffu, r.w, 8);
        r.x += __shfl_xor_sync(0xffffffffu, r.x, 16);
        r.y += __shfl_xor_sync(0xffffffffu, r.y, 16);
        r.z += __shfl_xor_sync(0xffffffffu, r.z, 16);
        r.w += __shfl_xor_sync(0xffffffffu, r.w, 16);
        if (grp == 0)
            __stcg(reinterpret_cast<float4*>(gtile + j * 32 + 4 * l8),
                   class_result<GM>(r, nut * xs[j], gam, gstride, gs, j, l8));
    }
    // the other classes four side by side: in slot s, group g of warp h
    // walks the class at position nlong + 8 s + 4 h + g (quads of nearly
    // equal lengths, alternating between the warps: handing each quad to
    // the warp with fewer entries so far took 57.1 against 53.2 us at the
    // benchmark shape, the extra per-quad work outweighing the balance)
    const int nslots = (k - nlong + 7) >> 3;
    for (int s = 0; s < nslots; ++s) {
        const int pos = nlong + 8 * s + 4 * h + grp;
        int j = pos < k ? (int)cord[pos] : -1;
        int p0 = j >= 0 ? of[j] : 0;
        int len = j >= 0 ? of[j + 1] - p0 : 0;
        if (j >= 0 && !class_ok(j, p0, len, k, plen, err)) {
            j = -1;
            p0 = 0;
            len = 0;
        }
        int m = max(len, __shfl_xor_sync(0xffffffffu, len, 8));
        m = max(m, __shfl_xor_sync(0xffffffffu, m, 16));
        uint64_t a01 = 0ull, a23 = 0ull;  // +0.0f pairs
        walk_chunks(list, zchunk, lists, zcs, colb, p0, 0, len, m, nmax, err, a01, a23);
        if (j >= 0)
            __stcg(reinterpret_cast<float4*>(gtile + j * 32 + 4 * l8),
                   class_result<GM>(walk_result(a01, a23, -0.0f), nut * xs[j], gam, gstride, gs, j, l8));
    }
    return nlong;
}

// Sparse form of the same sums, used when B vanishes off the edges (mu = 0:
// no bonus term, so B_im = 0 unless a_im = 1): vertex i walks its adjacency
// list (CSR) and adds B_im into the colour of each neighbour, D 2|E|
// additions per iteration instead of D n^2.  Accumulates in Gs[j * 32].
// Also counts gamma_d(i) (eq. 1): the neighbours sharing i's colour.
__device__ __forceinline__ int neighbour_sums(const int* rowptr, const int* colidx, const uint16_t* cd,
                                              const float* Ed, const uint16_t* grow, float gs, int gstride,
                                              const float* Bl, int bstride, float nut, int k, float* Gs, int i,
                                              bool valid) {
    for (int j = 0; j < k; ++j) {
        float g0 = nut * __ldg(Ed + j);
        if (grow) g0 += gs * (float)__ldg(grow + (size_t)j * gstride);
        Gs[j * 32] = g0;
    }
    if (!valid) return 0;
    const int ci = __ldg(cd + i);
    int conf = 0;
    const int e0 = __ldg(rowptr + i), e1 = __ldg(rowptr + i + 1);
    int e = e0;
    for (; e + 4 <= e1; e += 4) {
        const int m0 = __ldg(colidx + e), m1 = __ldg(colidx + e + 1), m2 = __ldg(colidx + e + 2),
                  m3 = __ldg(colidx + e + 3);
        const int c0 = __ldg(cd + m0), c1 = __ldg(cd + m1), c2 = __ldg(cd + m2), c3 = __ldg(cd + m3);
        const float b0 = Bl[m0 * bstride], b1 = Bl[m1 * bstride], b2 = Bl[m2 * bstride], b3 = Bl[m3 * bstride];
        Gs[c0 * 32] += b0;
        Gs[c1 * 32] += b1;
        Gs[c2 * 32] += b2;
        Gs[c3 * 32] += b3;
        conf += (c0 == ci) + (c1 == ci) + (c2 == ci) + (c3 == ci);
    }
    for (; e < e1; ++e) {
        const int m = __ldg(colidx + e), cm = __ldg(cd + m);
        Gs[cm * 32] += Bl[m * bstride];
        conf += cm == ci;
    }
    return conf;
}

// gamma_d(i) (eq. 1) from the individual's class lists: the members of i's
// own class that are adjacent to i.  In the one-hot form the pair matrix
// tells them apart exactly: sg B_im >= 1 on edges (1 + lambda t (...) >= 1)
// and sg B_im <= 0 off them (-mu t (...) <= 0, the diagonal, the padding
// row), sg = -1 for the partitioning problems (whose B is negated), else 1.
// half: 0 the whole class, 1 / 2 its first / second half (in 4-wide chunks).
template <bool STG>
__device__ __forceinline__ int own_class_conflicts(const uint32_t* pm, const int* of, int ci, const float* Bl,
                                                   int bstride, float sg, int half = 0) {
    int s = STG ? of[ci] : __ldg(of + ci), e = STG ? of[ci + 1] : __ldg(of + ci + 1);
    if (half) {
        const int mid = s + 4 * ((e - s) >> 3);
        if (half == 1)
            e = mid;
        else
            s = mid;
    }
    int conf = 0;
    for (int p = s; p < e; p += 4) {  // padded class: whole 4-wide chunks
        const uint4 v = STG ? *reinterpret_cast<const uint4*>(pm + p) : __ldg(reinterpret_cast<const uint4*>(pm + p));
        conf += (sg * Bl[(int)v.x * bstride] >= 0.5f) + (sg * Bl[(int)v.y * bstride] >= 0.5f) +
                (sg * Bl[(int)v.z * bstride] >= 0.5f) + (sg * Bl[(int)v.w * bstride] >= 0.5f);
    }
    return conf;
}

// One 128-byte line per lane: the item's sorted vertices, class offsets and
// equity signs arrive in L1 in parallel instead of one L2 round trip per line.
__device__ __forceinline__ void prefetch_item(const uint32_t* pm, int plen, const int* of, int k, const float* Ed,
                                              int lane) {
    const int lp = (4 * plen + 127) / 128, lo = (4 * (k + 1) + 127) / 128, le = (4 * k + 127) / 128;
    for (int l = lane; l < lp + lo + le; l += 32) {
        const char* a = l < lp ? (const char*)pm + 128 * l
                               : (l < lp + lo ? (const char*)of + 128 * (l - lp)
                                              : (const char*)Ed + 128 * (l - lp - lo));
        asm volatile("prefetch.global.L1 [%0];" ::"l"(a));
    }
}

// The same sums on shared-memory copies: the tile's adjacency entries, entry
// t of row r at t * 32 + r (col: neighbour, bv: pair coefficient; staged
// once per tile for all its items, so the 32 lanes read one contiguous line
// per step), and the individual's colours (cw, staged once per item); vertex
// i0 + lane walks its own deg entries, the warp to the tile's largest degree.
__device__ __forceinline__ int neighbour_sums_staged(const uint16_t* col, const float* bv, const uint16_t* cw,
                                                     int deg, int tmax, const float* Ed, const uint16_t* grow,
                                                     float gs, int gstride, float nut, int k, float* Gs, int i0,
                                                     int lane, bool valid) {
    for (int j = 0; j < k; ++j) {
        float g0 = nut * __ldg(Ed + j);
        if (grow) g0 += gs * (float)__ldg(grow + (size_t)j * gstride);
        Gs[j * 32] = g0;
    }
    const int ci = valid ? cw[i0 + lane] : -1;
    int conf = 0;
    for (int t = 0; t < tmax; t += 4) {  // four entries' loads ahead of their additions
        int c[4];
        float b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            c[u] = -1;
            b[u] = 0.f;
            if (t + u < deg) {
                c[u] = cw[col[(t + u) * 32 + lane]];
                b[u] = bv[(t + u) * 32 + lane];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (c[u] >= 0) {
                Gs[c[u] * 32] += b[u];
                conf += c[u] == ci;
            }
    }
    return valid ? conf : 0;
}

// ---------------------------------------------------------------------------
// k_gsum: one block per SM, 16 warps (the adjacency walk keeps a shared
// 32 x k accumulator per warp and runs fewer).
// ---------------------------------------------------------------------------
constexpr int GSUM_MAX_WARPS = 30;  // the staged class walk: 15 warp pairs (named barriers 1..15)
constexpr int GSUM_CSR_WARPS = 32;  // the adjacency walk: one warp per item, no named barriers

// Staging (STG): the item's colour-sorted vertices, class offsets and equity
// terms, copied to shared memory once per item by the PAIR of warps that
// share it; warp h of the pair sums the colours [h kh, min(k, (h+1) kh)),
// kh = ceil(k / 2).
__host__ __device__ inline int gsum_stage_words(int perm_stride, int k) {
    return tc_rec_words(perm_stride, k);  // one individual's record
}

// Items (32-vertex tile T, individual d) run tile-major; each tile's D
// items form ceil(D / units) chunks of about one item per unit (a warp, or a
// warp pair when staged), and every block takes a contiguous run of whole
// chunks.  A block whose run crosses a tile boundary reloads the B panel
// between two barriers; with whole chunks on both sides its units still
// need no more rounds than a block inside one tile.
__host__ __device__ inline long long gsum_chunk_item(long long c, int cpt, int D) {
    return (c / cpt) * D + ((c % cpt) * D) / cpt;
}

// DN: the dense forms' gamma matrix (and the multicolouring's colour sets)
// may be present; without it their code is compiled out of the one-hot walk.
template <bool BTS, bool CSR, bool STG, bool DN>
__global__ void __launch_bounds__((CSR ? GSUM_CSR_WARPS : GSUM_MAX_WARPS) * 32, 1)
    k_gsum(tc_kparams P, const __grid_constant__ CUtensorMap tmB, int dbuf) {
    // dbuf (STG): two record buffers per warp pair, the next item's record
    // arriving by one bulk copy while the pair walks the current one
    pdl_trigger();
    // k_classes lets this kernel start only after its own predecessors (k_pairs
    // and, in the dense forms, the GEMMs) are complete: the stop flag of the
    // previous iteration and B can be read now, and the first panel of B is
    // loaded while k_classes finishes; its class lists need the wait below
    tc_dev_state* st = P.st;
    if (P.commit && st->stop) {
        pdl_wait();
        return;
    }
    // the grouped walk: staged lists, the B panel in shared memory, one
    // colour per vertex (the multicolouring keeps the per-warp class loop)
    constexpr bool GROUPED_OK = STG && BTS && !CSR;
    const bool GROUPED = GROUPED_OK && !(DN && P.cm);
    extern __shared__ __align__(1024) float sm[];
    __shared__ __align__(8) uint64_t s_bbar;
    __shared__ __align__(8) uint64_t s_rbar[GSUM_MAX_WARPS / 2][2];  // dbuf: the record buffers' barriers
    __shared__ __align__(8) uint64_t s_never;  // TC_FAULT=wait: a barrier nothing arrives at
    const int n = P.n, D = P.D, k = P.k;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nbox = (n + TC_BT_BOX_ROWS) / TC_BT_BOX_ROWS;  // rows 0..n, row n zero
    float* Bt = sm;
    // CSR: the per-warp grad_S tiles; staged (dbuf = 1): after the tile's
    // adjacency entries (neighbours, pair coefficients), and each warp's
    // tile followed by its copy of the individual's colours
    const bool cstaged = CSR && dbuf;
    const int ce_words = cstaged ? 16 * P.max_degree + 32 * P.max_degree : 0;  // [deg][32] uint16, then FP32
    const int cw_words = cstaged ? ((n + 7) / 8) * 4 : 0;
    uint16_t* s_col = reinterpret_cast<uint16_t*>(sm);
    float* s_bv = sm + 16 * P.max_degree;
    float* Gw = sm + (BTS ? (size_t)nbox * TC_BT_BOX_ROWS * 32 : 0) + ce_words +
                (size_t)warp * (32 * k + cw_words);  // CSR only
    uint16_t* cw = reinterpret_cast<uint16_t*>(Gw + 32 * k);
    __shared__ int s_rp[33];
    const int unit = STG ? warp >> 1 : warp, nunits = STG ? nw >> 1 : nw, h = STG ? (warp & 1) : 0;
    const int sw = gsum_stage_words(P.perm_stride, k);
    uint32_t* const psb = reinterpret_cast<uint32_t*>(sm + (BTS ? (size_t)nbox * TC_BT_BOX_ROWS * 32 : 0)) +
                          (size_t)unit * (dbuf ? 2 : 1) * sw;  // STG only
    const unsigned rec_bytes = 4u * (unsigned)P.rec_stride;
    unsigned bphase = 0;
    if (P.dbg_withhold && threadIdx.x == 0) {
        // injected failure: a device wait whose arrival is withheld, before
        // any copy is in flight; it runs out after the context's wait limit
        // and records TC_ERR_TIMEOUT, and the kernel then goes on as usual
        mbar_init(&s_never, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_wait_bounded(&s_never, 0u, &st->err, P.wait_ns);
    }
    if (threadIdx.x == 0 && (BTS || STG)) {
        if (BTS) mbar_init(&s_bbar, 1);
        if (STG)  // the record buffers' barriers (one used per pair without dbuf)
            for (int u = 0; u < nunits; ++u) {
                mbar_init(&s_rbar[u][0], 1);
                mbar_init(&s_rbar[u][1], 1);
            }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    __syncthreads();
    const long long t = st->t;
    const float nut = (float)((double)P.nu * (double)t);
    const int nT = (n + 31) / 32;
    const int cpt = (D + nunits - 1) / nunits;  // chunks per tile
    const long long C = (long long)nT * cpt;
    long long q = gsum_chunk_item(C * blockIdx.x / gridDim.x, cpt, D);
    const long long qend = gsum_chunk_item(C * (blockIdx.x + 1) / gridDim.x, cpt, D);
    // B[0..n] x [32 T, 32 T + 32) -> Bt by 2-D TMA boxes, zero filled past
    // the matrix edge; B is symmetric, so these are its columns
    auto load_panel = [&](int T) {
        fence_proxy_async();
        mbar_expect_tx(&s_bbar, (unsigned)(nbox * TC_BT_BOX_ROWS * 32 * 4));
        for (int b = 0; b < nbox; ++b)
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(Bt + (size_t)b * TC_BT_BOX_ROWS * 32)),
                "l"(reinterpret_cast<uint64_t>(&tmB)), "r"(T * 32), "r"(b * TC_BT_BOX_ROWS), "r"(smem_u32(&s_bbar))
                : "memory");
    };
    if (BTS && threadIdx.x == 0 && q < qend) load_panel((int)(q / D));
    // this pair's item after qq (tile T), across tile segments; qend: none
    auto unit_next = [&](long long qq, int T) -> long long {
        long long a = (long long)(T + 1) * D;  // the next segment's start
        if (qq + nunits < min(qend, a)) return qq + nunits;
        while (a < qend) {
            const long long se = min(qend, a + D);
            if (a + unit < se) return a + unit;
            a = se;
        }
        return qend;
    };
    const bool leader = STG && h == 0 && lane == 0;
    pdl_wait();  // the class lists (and equity terms) from k_classes
    if (STG && dbuf && leader && q < qend) {  // the pair's first record
        long long q1 = q + unit;
        const int T0 = (int)(q / D);
        if (q1 >= min(qend, (long long)(T0 + 1) * D)) q1 = unit_next(q1 - nunits, T0);
        if (q1 < qend) {
            const int d1 = (int)(q1 - (q1 / D) * D);
            mbar_expect_tx(&s_rbar[unit][0], rec_bytes);
            bulk_load(psb, P.rec + (size_t)d1 * P.rec_stride, rec_bytes, &s_rbar[unit][0]);
        }
    }
    int it = 0;  // items this pair has started (dbuf: buffer it & 1, phase (it >> 1) & 1)
    bool first = true;
    while (q < qend) {
        const int T = (int)(q / D);
        const long long seg_end = min(qend, (long long)(T + 1) * D);
        // Each warp waits for the segment's panel just before its first walk,
        // so that the staging of its first item overlaps the panel's load.
        // Every segment holds an item, so some warp has waited for the
        // previous panel before the barrier below lets the next one start.
        bool panel_pending = false;
        unsigned seg_phase = 0;
        if (cstaged) {  // the tile's adjacency entries: lane = row, warp w takes the steps t = w, w + nw, ...
            const int i = T * 32 + lane;
            __syncthreads();  // every warp is done with the previous tile's entries
            const int a = i < n ? __ldg(P.rowptr + i) : 0, deg = i < n ? __ldg(P.rowptr + i + 1) - a : 0;
            int tmax = deg;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) tmax = max(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
            if (warp == 0) {
                s_rp[lane] = deg;
                if (lane == 0) s_rp[32] = tmax;
            }
            for (int t = warp; t < tmax; t += nw)
                if (t < deg) {
                    const int m = __ldg(P.colidx + a + t);
                    s_col[t * 32 + lane] = (uint16_t)m;
                    s_bv[t * 32 + lane] = __ldg(P.B + (size_t)i * P.ldb + m);
                }
            __syncthreads();
        }
        if (BTS) {
            if (!first) {
                __syncthreads();  // every pair is done with the previous panel
                if (threadIdx.x == 0) load_panel(T);
            }
            first = false;
            seg_phase = bphase;
            bphase ^= 1u;
            panel_pending = true;
        }
        const int i0 = T * 32, rows = min(32, n - i0);
        for (long long qq = q + unit; qq < seg_end; qq += nunits) {
            const int d = (int)(qq - (long long)T * D);
            uint32_t* rd = P.rec + (size_t)d * P.rec_stride;
            const uint32_t* pm = rd;
            const int* of = tc_rec_off(rd, P.perm_stride);
            const float* Ed = tc_rec_E(rd, P.perm_stride, k);
            // the staged record (STG): list, offsets, additive-term factors,
            // class order, padding chunk
            uint32_t* ps = psb + (dbuf ? (size_t)(it & 1) * sw : 0);
            int* os = tc_rec_off(ps, P.perm_stride);
            float* xs = tc_rec_E(ps, P.perm_stride, k);
            uint16_t* cs = tc_rec_cord(ps, P.perm_stride, k);
            uint32_t* zc = tc_rec_zchunk(ps, P.perm_stride, k);
            if (STG && dbuf) {
                pair_sync(unit);  // the pair's reads of the previous item (the other buffer) are done
                if (leader) {
                    const long long nx = unit_next(qq, T);
                    if (nx < qend) {
                        const int dn = (int)(nx - (nx / D) * D);
                        uint64_t* bar = &s_rbar[unit][(it + 1) & 1];
                        fence_proxy_async();
                        mbar_expect_tx(bar, rec_bytes);
                        bulk_load(psb + (size_t)((it + 1) & 1) * sw, P.rec + (size_t)dn * P.rec_stride, rec_bytes,
                                  bar);
                    }
                }
                mbar_wait_bounded(&s_rbar[unit][it & 1], (unsigned)(it >> 1) & 1u, &st->err, P.wait_ns);
            } else if (STG) {
                pair_sync(unit);  // the pair's reads of the previous item are done
                // the whole record (a multiple of 16 bytes) by one bulk copy:
                // the copy engine writes shared memory without load/store
                // instructions of the pair (the class walk's own pipe)
                if (leader) {
                    fence_proxy_async();
                    mbar_expect_tx(&s_rbar[unit][0], rec_bytes);
                    bulk_load(ps, pm, rec_bytes, &s_rbar[unit][0]);
                }
                mbar_wait_bounded(&s_rbar[unit][0], (unsigned)it & 1u, &st->err, P.wait_ns);
            } else if (!CSR) {
                prefetch_item(pm, P.perm_stride, of, k, Ed, lane);
            }
            if (BTS && panel_pending) {
                mbar_wait_bounded(&s_bbar, seg_phase, &st->err, P.wait_ns);
                panel_pending = false;
            }
            const float* Bl = BTS ? (Bt + lane) : (P.B + min(i0 + lane, n - 1));
            // the item's gamma entries: colour j of row i0 + lane at grow[j * gstride]
            const uint16_t* grow = DN && P.G16 ? P.G16 + tc_gamma_index(d, i0 + lane, 0, P.n_pad, k) : nullptr;
            const int gstride = P.n_pad;
            const float gs = tc_is_partition(P.problem) ? -1.0f : 1.0f;  // sign of the A.S term
            float* Gout = P.Gbuf + ((size_t)d * nT + T) * k * 32 + lane;
            const bool live = lane < rows;
            const int bstride = BTS ? 32 : P.ldb;
            const bool counter = !CSR && h == (STG ? 1 : 0);  // the warp that counts the conflicts
            const int ci = counter && live ? (int)__ldg(P.c + (size_t)d * n + i0 + lane) : 0;  // ahead of use
            int conf = -1;  // gamma_d(i0 + lane), counted by one warp of the item
            if (GROUPED_OK && GROUPED) {
                int nlong;
                if (DN && P.G16) {  // the dense forms: A.S and gamma_d(i) from the gamma matrix
                    nlong = slot_walk<true>(ps, os, cs, xs, zc, nut, Bt, k, h, lane,
                                            P.Gbuf + ((size_t)d * nT + T) * k * 32, n, P.perm_stride, &st->err,
                                            P.G16 + tc_gamma_index(d, i0, 0, P.n_pad, k), P.n_pad, gs);
                    if (counter) conf = live ? (int)__ldg(grow + (size_t)ci * gstride) : 0;
                    nlong = 0;  // (no own-class walks to share)
                } else {
                    nlong = slot_walk<false>(ps, os, cs, xs, zc, nut, Bt, k, h, lane,
                                             P.Gbuf + ((size_t)d * nT + T) * k * 32, n, P.perm_stride, &st->err,
                                             nullptr, 0, gs);
                }
                // with classes of 32 entries or more the rows' own classes are
                // mostly long as well: both warps count half of each (the
                // partitioning problems keep most vertices in a few classes,
                // where warp 1 counting whole classes took about as long as the
                // walk itself); tc_evaluate's per-vertex counts come whole
                // from warp 1
                const bool split = nlong > 0 && P.dbg_gamma == nullptr;
                if (!(DN && P.G16) && (counter || split)) {
                    conf = 0;
                    if (live) {
                        const int cc = counter ? ci : (int)__ldg(P.c + (size_t)d * n + i0 + lane);
                        conf = own_class_conflicts<true>(ps, os, cc, Bt + lane, 32, gs, split ? 1 + h : 0);
                    }
                }
            } else if (CSR) {
                if (cstaged) {
                    const uint32_t* src = reinterpret_cast<const uint32_t*>(P.c_snap + (size_t)d * n);
                    uint32_t* dst = reinterpret_cast<uint32_t*>(cw);
                    if ((((size_t)d * n) & 1) == 0)  // 4-byte aligned row
                        for (int x = lane; x < n / 2; x += 32) dst[x] = __ldg(src + x);
                    else
                        for (int x = lane; x < n / 2; x += 32)
                            cw[2 * x] = P.c_snap[(size_t)d * n + 2 * x], cw[2 * x + 1] = P.c_snap[(size_t)d * n + 2 * x + 1];
                    if ((n & 1) && lane == 0) cw[n - 1] = P.c_snap[(size_t)d * n + n - 1];
                    __syncwarp();
                    conf = neighbour_sums_staged(s_col, s_bv, cw, s_rp[lane], s_rp[32], Ed, grow, gs, gstride, nut, k,
                                                 Gw + lane, i0, lane, live);
                } else {
                    conf = neighbour_sums(P.rowptr, P.colidx, P.c_snap + (size_t)d * n, Ed, grow, gs, gstride, Bl,
                                          bstride, nut, k, Gw + lane, i0 + lane, live);
                }
                __syncwarp();
                for (int j = 0; j < k; ++j) Gout[j * 32] = Gw[j * 32 + lane];
                __syncwarp();
            } else {
                // the counting warp takes a few colours fewer
                const int kh = min(k, (k + 4) >> 1), jb = STG ? h * kh : 0, je = STG ? (h ? k : kh) : k;
                if (STG) {
                    if (BTS)
                        class_sums_shared(smem_u32(ps), os, xs, nut, grow, gs, gstride, smem_u32(Bl), k, jb, je,
                                          Gout);
                    else
                        class_sums<0, true>(ps, os, xs, Ed, grow, gs, gstride, Bl, P.ldb, nut, k, jb, je, Gout);
                } else if (BTS) {
                    class_sums<32, false>(pm, of, nullptr, Ed, grow, gs, gstride, Bl, 32, nut, k, 0, k, Gout);
                } else {
                    class_sums<0, false>(pm, of, nullptr, Ed, grow, gs, gstride, Bl, P.ldb, nut, k, 0, k, Gout);
                }
                if (counter) {
                    conf = 0;
                    if (live) {
                        if (DN && P.cm) {  // multicolouring: shared colours with the neighbours, over i's colours
                            const uint16_t* set = P.cm + ((size_t)d * n + i0 + lane) * P.cmax;
                            const int ci_n = __ldg(P.dem + i0 + lane);
                            for (int qq = 0; qq < ci_n; ++qq) conf += __ldg(grow + (size_t)set[qq] * gstride);
                        } else if (DN && P.G16)
                            conf = __ldg(grow + (size_t)ci * gstride);  // the gamma matrix of the dense forms
                        else if (STG)
                            conf = own_class_conflicts<true>(ps, os, ci, Bl, bstride, gs);
                        else
                            conf = own_class_conflicts<false>(pm, of, ci, Bl, bstride, gs);
                    }
                }
            }
            if (conf >= 0) {  // warp-uniform
                if (P.dbg_gamma && live) P.dbg_gamma[(size_t)d * n + i0 + lane] = conf;
                int sum = conf;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
                if (lane == 0 && sum) atomicAdd(P.fcolor + d, sum);  // twice the conflicts of the item's rows
            }
            ++it;
        }
        q = seg_end;
    }
    // completion ticket: the last block reduces the population (Algorithm 1's
    // stop test, the best-so-far record, the loss of eq. 7) before k_update.
    // The ticket is an acquire-release atomic taken after the block barrier:
    // it releases the block's conflict counts and, for the last block,
    // acquires every other block's (the barrier below passes both on)
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned ticket;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(ticket) : "l"(&st->done_gsum) : "memory");
        s_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last) finalize_population(P, sm, t);  // the panel and staging areas are free now
}

// ---------------------------------------------------------------------------
// k_update: per item, bulk copies bring the grad_S tile and the weight tile
// (both [k][32], contiguous: the tile-transposed weight layout) into shared
// memory; lane r of each warp of a group of four updates its quarter of row
// r with loops uniform across the warp and free of bank conflicts, and the
// tile goes back with a bulk store.
// debug_only: 1 = copy grad_S L to P.dbg_G; 2 = write grad_W L to P.dbg_G
// instead of updating W.
// ---------------------------------------------------------------------------
// k_update is warp-specialised.  Warp 0 streams the block's items through a
// ring of S stages (grad_S tile and weight tile, each k x 32 floats and
// contiguous in the tiled layouts) with bulk copies.  P groups of UPD_GW
// warps take the items in turn (latency, not issue, bounds one lane walking
// a whole row): warp h of a group updates the colours [jb, je) (a quarter)
// of all 32 rows in place, lane r owning row r, and the quarters meet twice
// through shared memory (softmax sums, then argmax); the producer writes
// each updated weight tile back with a bulk store before its stage is
// refilled.  A group holds its stage while it computes, so the quarters
// (half the time per item of halves) leave more of the ring loading.
// Shared memory: full[S], done[S] mbarriers, S stages of 64 k floats
// ([Gs | Ws], 16-byte aligned), P exchange slots of 512 floats (xa [4][2][32]:
// Z, num per quarter; xb [4][2][32]: best value, colour per quarter).
constexpr int UPD_MAX_GROUPS = (UPD_MAX_WARPS - 1) / UPD_GW;
constexpr int UPD_MAX_STAGES = 16;

__host__ __device__ constexpr long long upd_smem_bytes(int k, int S, int P) {
    return 16ll * S + 256ll * k * S + 2048ll * P;
}

__device__ __forceinline__ void group_sync(int grp) {  // the UPD_GW warps of group grp (named barrier grp + 1)
    asm volatile("bar.sync %0, %1;" ::"r"(grp + 1), "n"(UPD_GW * 32) : "memory");
}

__device__ __forceinline__ float ex2_approx(float x) {  // 2^x, PTX ex2.approx
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// One item (32-row tile T of individual d) by warp h (a quarter of the
// colours) of group `grp`, its tiles already in Gs, Ws.  xa, xb: the group's
// exchange slots of 256 floats each.  Returns with all the group's warps
// done with the stage.
__device__ __forceinline__ void update_item(const tc_kparams& P, float* Gs, float* Ws, float* xa, float* xb,
                                            int grp, int h, int T, int d, int cur, bool smooth,
                                            int debug_only, bool dn) {
    static_assert(UPD_GW == 4, "the sums below combine four quarters");
    const int n = P.n, k = P.k;
    const int lane = threadIdx.x & 31;
    const int i0 = T * 32;
    const int rows = min(32, n - i0);
    const int kq = (k + UPD_GW - 1) / UPD_GW, jb = min(k, h * kq), je = min(k, jb + kq);
    const bool live = lane < rows;
    if (debug_only == 1) {
        if (live) {
            float* g = P.dbg_G + ((size_t)d * n + i0 + lane) * k;
            for (int jj = jb; jj < je; ++jj) g[jj] = Gs[jj * 32 + lane];
        }
        group_sync(grp);
        return;
    }
    float* wr = Ws + lane;
    const float* gr = Gs + lane;
    constexpr float kL2E = 1.4426950408889634f;  // log2(e)
    // the row maximum is the weight of the row's current colour: the colours
    // are the argmax of W, kept in step with it by every update
    const float nml = live ? -wr[cur * 32] * kL2E : 0.f;
    // softmax sums of this quarter: e_j = 2^(w_j log2 e - max log2 e)
    float z4[4] = {0.f, 0.f, 0.f, 0.f}, n4[4] = {0.f, 0.f, 0.f, 0.f};
    if (live) {
        int j = jb;
        for (; j + 4 <= je; j += 4)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float e = ex2_approx(fmaf(wr[(j + u) * 32], kL2E, nml));
                z4[u] += e;
                n4[u] = fmaf(e, gr[(j + u) * 32], n4[u]);
            }
        for (; j < je; ++j) {
            const float e = ex2_approx(fmaf(wr[j * 32], kL2E, nml));
            z4[0] += e;
            n4[0] = fmaf(e, gr[j * 32], n4[0]);
        }
    }
    xa[h * 64 + lane] = (z4[0] + z4[1]) + (z4[2] + z4[3]);
    xa[h * 64 + 32 + lane] = (n4[0] + n4[1]) + (n4[2] + n4[3]);
    group_sync(grp);
    // same order in every warp of the group
    const float Z = (xa[lane] + xa[64 + lane]) + (xa[128 + lane] + xa[192 + lane]);
    const float num = (xa[32 + lane] + xa[96 + lane]) + (xa[160 + lane] + xa[224 + lane]);
    const float invZ = 1.0f / Z;
    const float dot = num * invZ;  // (S^ (.) grad_S L) . J of eq. 12
    // Step 4-iv: W / rho as a product with the rounded reciprocal (within
    // one rounding of the quotient; the IEEE division cost 7.7 us in every
    // smoothing iteration at the benchmark shape)
    const float rrho = 1.0f / P.rho;
    float bestv = -INFINITY;
    int newc = jb;
    if (live) {
#pragma unroll 4
        for (int j = jb; j < je; ++j) {
            // eq. 12, the descent step and eq. 8, each rounded once (no
            // contraction): W_next == W - eta * gW holds bit for bit
            const float w = wr[j * 32];
            const float sj = __fmul_rn(ex2_approx(fmaf(w, kL2E, nml)), invZ);
            const float gw = __fmul_rn(sj, __fsub_rn(gr[j * 32], dot));
            if (debug_only == 2) {
                P.dbg_G[((size_t)d * n + i0 + lane) * k + j] = gw;
                continue;
            }
            float wn = __fsub_rn(w, __fmul_rn(P.eta, gw));
            if (smooth) wn = __fmul_rn(wn, rrho);
            wr[j * 32] = wn;
            if (wn > bestv) {  // first maximum wins
                bestv = wn;
                newc = j;
            }
        }
    }
    if (debug_only == 2) {
        group_sync(grp);
        return;
    }
    xb[h * 64 + lane] = bestv;
    xb[h * 64 + 32 + lane] = __int_as_float(newc);
    fence_proxy_async();  // this lane's writes of Ws, before the producer's bulk store
    group_sync(grp);
    if (h != 0) return;
    // the lowest quarter wins ties: it holds the lower colours
    bestv = xb[lane];
#pragma unroll
    for (int q = 1; q < UPD_GW; ++q)
        if (xb[q * 64 + lane] > bestv) {
            bestv = xb[q * 64 + lane];
            newc = __float_as_int(xb[q * 64 + 32 + lane]);
        }
    if (live && !(dn && P.cm)) {  // (the multicolouring's next assignment is k_assign_multi)
        const int i = i0 + lane;
        if (dn && P.S8 && cur != newc) {  // dense forms: move the one-hot entry of (d, i) in both operands
            const size_t co = (size_t)d * k + cur, cn = (size_t)d * k + newc;
            P.S8[(size_t)i * P.ldg + co] = 0;
            P.S8[(size_t)i * P.ldg + cn] = 0x38;  // E4M3 1.0
            P.S8T[co * P.n_pad + i] = 0;
            P.S8T[cn * P.n_pad + i] = 0x38;
        }
        store_colour(P, d, i, cur, newc);
    }
}

template <int DBG, bool DN>
__global__ void __launch_bounds__(UPD_MAX_WARPS * 32, 1)
    k_update(tc_kparams P, int items_per_block, int S) {
    // DBG: the debug mode (compile time); DN: the dense forms' FP8 operands
    // or the multicolouring may be present (else their code is compiled out)
    constexpr int debug_only = DBG;
    pdl_trigger();
    // Before the wait for k_gsum: only what earlier kernels wrote (the weight
    // tiles, t) is read; the stop flag and the grad_S tiles come after it.
    tc_dev_state* st = P.st;
    extern __shared__ __align__(1024) float sm[];
    const int n = P.n, D = P.D, k = P.k;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, ngroups = ((int)(blockDim.x >> 5) - 1) / UPD_GW;
    uint64_t* full = reinterpret_cast<uint64_t*>(sm);
    uint64_t* done = full + S;
    float* stages = sm + 4 * S;  // after 2 S mbarriers (16 S bytes)
    float* xch = stages + (size_t)S * 64 * k;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full + s, 1);
            mbar_init(done + s, 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    __syncthreads();
    const int nT = (n + 31) / 32;
    const long long Q = (long long)nT * D;
    const long long q0 = (long long)blockIdx.x * items_per_block;
    const int R = (int)max(0ll, min(Q, q0 + items_per_block) - q0);
    const unsigned bytes = (unsigned)(k * 32 * 4);
    const uint64_t spol = l2_policy_evict_first();  // W and the grad_S tiles pass through once
    auto tile_of = [&](int r) {  // same offset in Gbuf and W
        const long long qq = q0 + r;
        const int T = (int)(qq / D);
        return ((size_t)(qq - (long long)T * D) * nT + T) * k * 32;
    };
    // the weight tiles of the first stages load while k_gsum finishes
    const int pre = debug_only == 1 ? 0 : min(S, R);
    if (warp == 0 && lane == 0)
        for (int r = 0; r < pre; ++r) {
            mbar_expect_tx(full + r, 2 * bytes);
            bulk_load_hint(stages + (size_t)r * 64 * k + 32 * k, P.W + tile_of(r), bytes, full + r, spol);
        }
    pdl_wait();  // the grad_S tiles and the stop flag from k_gsum
    // an improved best-so-far (k_gsum's population reduction): its colours
    // are copied here, each row just before its update overwrites it
    const int best_d = debug_only == 0 && __ldcg(&st->best_pending) ? __ldcg(&st->last_dstar) : -1;
    // Step 4-iv after the update of iteration t: the population reduction of
    // a committed iteration that goes on has already set the counter to t + 1
    const long long tc = __ldcg(&st->t);
    const bool smooth = ((debug_only ? tc + 1 : tc) % P.nb_iter) == 0;
    if (!debug_only && st->stop) {
        if (warp == 0 && lane == 0) {  // no copy may still be landing when the block exits
            for (int r = 0; r < pre; ++r)
                bulk_load_hint(stages + (size_t)r * 64 * k, P.Gbuf + tile_of(r), bytes, full + r, spol);
            for (int r = 0; r < pre; ++r) mbar_wait_bounded(full + r, 0u, &st->err, P.wait_ns);
        }
        if (best_d >= 0 && blockIdx.x == 0)  // no update: the colours are the evaluated ones
            for (int i = threadIdx.x; i < n; i += blockDim.x) P.best[i] = P.c[(size_t)best_d * n + i];
        return;
    }
    if (warp == 0) {
        if (lane == 0) {  // producer: item r into stage r % S once its previous use is released
            for (int r = 0; r < R; ++r) {
                const int s = r % S, u = r / S;
                float* Gs = stages + (size_t)s * 64 * k;
                const size_t tile = tile_of(r);
                if (r < pre) {  // its weight tile is on the way
                    bulk_load_hint(Gs, P.Gbuf + tile, bytes, full + s, spol);
                    continue;
                }
                if (u > 0) mbar_wait_bounded(done + s, (unsigned)(u - 1) & 1u, &st->err, P.wait_ns);
                mbar_expect_tx(full + s, debug_only == 1 ? bytes : 2 * bytes);
                bulk_load_hint(Gs, P.Gbuf + tile, bytes, full + s, spol);
                if (debug_only != 1) bulk_load_hint(Gs + 32 * k, P.W + tile, bytes, full + s, spol);
            }
        }
        __syncwarp();
    } else {  // consumer groups
        const int grp = (warp - 1) / UPD_GW, h = (warp - 1) % UPD_GW;
        float* xa = xch + (size_t)grp * 512;
        float* xb = xa + 256;
        // the rows' current colours, one item ahead (an L2 round trip)
        auto colour_of = [&](int r) {
            const long long qq = q0 + r;
            const int T = (int)(qq / D), d = (int)(qq - (long long)T * D), i = T * 32 + lane;
            return i < n ? (int)__ldg(P.c + (size_t)d * n + i) : 0;
        };
        int cur_next = grp < R ? colour_of(grp) : 0;
        for (int r = grp; r < R; r += ngroups) {
            const long long qq = q0 + r;
            const int T = (int)(qq / D), d = (int)(qq - (long long)T * D);
            const int s = r % S, u = r / S;
            const int cur = cur_next;
            if (r + ngroups < R) cur_next = colour_of(r + ngroups);
            if (d == best_d && h == 0 && T * 32 + lane < n) P.best[T * 32 + lane] = (uint16_t)cur;
            // A parity wait is only sound within one phase of the barrier.
            // Another group may still hold use u - 1 of this stage (the loads
            // of use u - 1 were issued, since this group's previous item,
            // loaded later, was; their bytes may not have landed): wait for
            // that use to be released first, then for use u's bytes.
            if (u > 0) mbar_wait_bounded(done + s, (unsigned)(u - 1) & 1u, &st->err, P.wait_ns);
            mbar_wait_bounded(full + s, (unsigned)u & 1u, &st->err, P.wait_ns);
            float* Gs = stages + (size_t)s * 64 * k;
            update_item(P, Gs, Gs + 32 * k, xa, xb, grp, h, T, d, cur, smooth, debug_only, DN);
            // all the group's warps are past its last barrier of the item (their
            // writes of the weight tile fenced for the async proxy): one lane
            // writes the tile back and frees the stage once the store has read it
            if (h == 0 && lane == 0) {
                if (debug_only == 0) {
                    bulk_store_hint(P.W + tile_of(r), Gs + 32 * k, bytes, spol);
                    bulk_wait_read();
                }
                mbar_arrive(done + s);
            }
        }
        if (h == 0 && lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // stores complete
    }
}

constexpr int kSmemOptin = 232448 - 1024;  // 227 KB per block on sm_103, less static slack

}  // namespace

int tc_pair_tile_edge() { return PT; }

int tc_pair_tile_count(int n) {
    const int T = (n + PT - 1) / PT;
    return T * (T + 1) / 2;
}

// Whether a population of this shape fits the update kernel (one warp's
// grad_S and weight tiles in shared memory).
int tc_update_fits(int k) { return upd_smem_bytes(k, 1, 1) <= kSmemOptin ? TC_OK : TC_ERR_UNSUPPORTED; }

cudaError_t tc_launch_init_weights(float* W, int D, int n, int k, unsigned long long seed, float sigma0,
                                   cudaStream_t s) {
    const long long groups = ((long long)D * n * k + 3) / 4;
    const int th = 256;
    k_init_weights<<<(unsigned)((groups + th - 1) / th), th, 0, s>>>(W, D, n, k, seed, sigma0);
    return cudaGetLastError();
}

cudaError_t tc_launch_w_layout(const float* src, float* dst, int D, int n, int k, bool to_tiled,
                               cudaStream_t s) {
    const long long total = (long long)D * ((n + TC_WT - 1) / TC_WT) * k * TC_WT;
    k_w_layout<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(src, dst, D, n, k, to_tiled);
    return cudaGetLastError();
}

cudaError_t tc_launch_w_tiles(const float* src, float* dst, int D, int n, int k, bool to_tiled, cudaStream_t s) {
    const size_t smem = sizeof(float) * TC_WT * ((size_t)k + 1);
    if (smem > 48 * 1024) return cudaErrorInvalidValue;  // (k > 374: the element-wise conversion)
    const long long blocks = (long long)D * ((n + TC_WT - 1) / TC_WT);
    k_w_tiles<<<(unsigned)blocks, 256, smem, s>>>(src, dst, n, k, to_tiled);
    return cudaGetLastError();
}

// The bit planes from the colours: one warp per (vertex, group of 32
// individuals), a ballot per bit.
__global__ void k_planes(tc_kparams P) {
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= (long long)P.n * P.png) return;
    const int i = (int)(wid / P.png), g = (int)(wid % P.png), d = 32 * g + lane;
    const unsigned c = d < P.D ? P.c[(size_t)d * P.n + i] : 0u;
    unsigned mine = 0u;
#pragma unroll
    for (int p = 0; p < 7; ++p) {
        const unsigned b = __ballot_sync(0xffffffffu, (c >> p) & 1u);
        if (lane == p) mine = b;
    }
    if (lane < 8) P.planes[((size_t)i * P.png + g) * 8 + lane] = mine;  // plane 7: 0
}

cudaError_t tc_launch_assign(const tc_kparams& P, cudaStream_t s) {
    const long long rows = (long long)P.D * P.n;
    k_assign<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(P);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && P.planes) {
        const long long warps = (long long)P.n * P.png;
        k_planes<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(P);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t tc_launch_pairs(const tc_kparams& P, cudaStream_t s) {
    if (P.M32)  // the dense forms: M~ read from the GEMM, no colour compares
        return tc_launch_pdl(k_pairs<1, false, true>, dim3(P.n_pair_blocks), dim3(PAIR_THREADS), 0, s, P);
    if (P.ct_bytes == 1)
        return P.k <= 128 ? tc_launch_pdl(k_pairs<1, true, false>, dim3(P.n_pair_blocks), dim3(PAIR_THREADS), 0, s, P)
                          : tc_launch_pdl(k_pairs<1, false, false>, dim3(P.n_pair_blocks), dim3(PAIR_THREADS), 0, s,
                                          P);
    return tc_launch_pdl(k_pairs<2, false, false>, dim3(P.n_pair_blocks), dim3(PAIR_THREADS), 0, s, P);
}

cudaError_t tc_launch_front(const tc_kparams& P, cudaStream_t s) {
    const long long counts = 4ll * (CLS_THREADS / 32) * P.k;  // the class blocks' per-warp colour counts
    const int smem = (int)(counts + 16ll * ((P.n + 7) / 8));  // + the individual's colours
    auto fn = P.ct_bytes == 1 ? (P.k <= 128 ? k_front<1, true> : k_front<1, false>) : k_front<2, false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return tc_launch_pdl(fn, dim3(P.D + P.n_pair_blocks), dim3(PAIR_THREADS), smem, s, P);
}

cudaError_t tc_launch_classes(const tc_kparams& P, cudaStream_t s) {
    if (P.cm) return tc_launch_classes_multi(P, s);  // multicolouring: a vertex in several classes
    const long long counts = 4ll * (CLS_THREADS / 32) * P.k;  // per-warp colour counts
    const int smem = (int)(counts + 16ll * ((P.n + 7) / 8));  // + the individual's colours
    cudaError_t e = cudaFuncSetAttribute(k_classes, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return tc_launch_pdl(k_classes, dim3(P.D), dim3(CLS_THREADS), smem, s, P);
}

template <bool BTS, bool CSR, bool STG>
static cudaError_t launch_gsum_t(const tc_kparams& P, const CUtensorMap& tmB, int num_sms, int warps, int smem,
                                 int dbuf, cudaStream_t s) {
    auto fn = (P.G16 || P.cm) ? k_gsum<BTS, CSR, STG, true> : k_gsum<BTS, CSR, STG, false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int units = STG ? warps / 2 : warps;
    const long long chunks = (long long)((P.n + 31) / 32) * ((P.D + units - 1) / units);
    const int blocks = (int)std::max(1ll, std::min<long long>(num_sms, chunks));
    return tc_launch_pdl(fn, dim3(blocks), dim3(warps * 32), smem, s, P, tmB, dbuf);
}

// grad_S L tiles (k_gsum) into P.Gbuf: the B panel in shared memory when it
// fits, 16 warps, or fewer with the per-warp tiles of the adjacency walk; the
// class walk stages each item in shared memory when 8 or more warps fit so.
cudaError_t tc_launch_gsum(const tc_kparams& P, const CUtensorMap& tmB, int num_sms, cudaStream_t s) {
    const long long bt = 4ll * 32 * ((P.n + TC_BT_BOX_ROWS) / TC_BT_BOX_ROWS) * TC_BT_BOX_ROWS;
    const long long stage = 4ll * gsum_stage_words(P.perm_stride, P.k);
    if (P.csr_walk && P.n < 65536) {
        // the staged adjacency walk: the tile's entries ([degree][32] uint16
        // neighbours and FP32 pair coefficients) once per tile, then per warp
        // its grad_S tile and the individual's colours (G(1000, 0.1), k = 25,
        // D = 128: 64.2 -> 35.0 us; entries read from global memory before)
        const long long ce = 4ll * 48 * P.max_degree;  // [max degree][32] uint16 + FP32
        const long long pw = 4ll * (32ll * P.k + ((P.n + 7) / 8) * 4);
        // 32 warps: D = 128 items per tile make 4 chunks of 32, one round per
        // block (30 warps made 5 chunks of ~26 and two rounds for some blocks)
        const long long w = std::min<long long>(GSUM_CSR_WARPS, (kSmemOptin - ce) / pw);
        if (w >= 8) {
            const int smem = (int)std::max(ce + w * pw, 2048ll);
            return launch_gsum_t<false, true, false>(P, tmB, num_sms, (int)w, smem, 1, s);
        }
    }
    long long per_warp = P.csr_walk ? 4ll * 32 * P.k : 0;
    const bool bts = bt + per_warp <= kSmemOptin;
    const long long base = bts ? bt : 0;
    const bool stg = !P.csr_walk && base + 4 * stage <= kSmemOptin;  // 4 pairs or more
    int warps = GSUM_MAX_WARPS;
    long long smem_ll = base;
    // two record buffers per warp pair only when the most pairs still fit
    // (at the benchmark shape 8 double-buffered pairs took 61.3 us against
    // 55.4 us for 15 pairs with one buffer each)
    const int dbuf = stg && (kSmemOptin - base) / (2 * stage) >= GSUM_MAX_WARPS / 2 ? 1 : 0;
    if (stg) {  // one or two staging areas per warp pair
        const int pairs = (int)std::min<long long>(GSUM_MAX_WARPS / 2, (kSmemOptin - base) / ((1 + dbuf) * stage));
        warps = 2 * pairs;
        smem_ll += (1 + dbuf) * stage * pairs;
    } else if (per_warp > 0) {
        warps = (int)std::min<long long>(GSUM_MAX_WARPS, (kSmemOptin - base) / per_warp);
        smem_ll += per_warp * warps;
    }
    if (warps < 1) return cudaErrorInvalidValue;
    const int smem = (int)std::max(smem_ll, 2048ll);  // the population reduction's scratch at least
    if (P.csr_walk)
        return bts ? launch_gsum_t<true, true, false>(P, tmB, num_sms, warps, smem, 0, s)
                   : launch_gsum_t<false, true, false>(P, tmB, num_sms, warps, smem, 0, s);
    if (stg)
        return bts ? launch_gsum_t<true, false, true>(P, tmB, num_sms, warps, smem, dbuf, s)
                   : launch_gsum_t<false, false, true>(P, tmB, num_sms, warps, smem, dbuf, s);
    return bts ? launch_gsum_t<true, false, false>(P, tmB, num_sms, warps, smem, 0, s)
               : launch_gsum_t<false, false, false>(P, tmB, num_sms, warps, smem, 0, s);
}

// k_update: as many stages as fit (at most 16), at most 5 consumer groups,
// three stages fewer; one block per SM.
cudaError_t tc_launch_update(const tc_kparams& P, int num_sms, cudaStream_t s, int debug_only) {
    const long long per_stage = 16ll + 256ll * P.k;
    int S = (int)std::min<long long>(UPD_MAX_STAGES, (kSmemOptin - 1024ll) / per_stage);
    if (S < 1) return cudaErrorInvalidValue;
    // groups of UPD_GW warps, three stages loading ahead of them (at the
    // benchmark shape 9 stages: 3, 4, 5 groups measured 50.9, 43.5, 42.6 us);
    // with fewer than four stages (k above ~220) one stage loads ahead of
    // S - 1 groups (k = 230: 3 stages, 2 groups 78.9 us against 137.5 us for
    // one group)
    int pairs = S >= 4 ? std::min(UPD_MAX_GROUPS, S - 3) : std::max(1, S - 1);
    while (S > 1 && upd_smem_bytes(P.k, S, pairs) > kSmemOptin) --S;
    if (upd_smem_bytes(P.k, S, pairs) > kSmemOptin) return cudaErrorInvalidValue;
    const int smem = (int)upd_smem_bytes(P.k, S, pairs);
    const long long items = (long long)((P.n + 31) / 32) * P.D;
    long long blocks = std::min<long long>(num_sms, items);
    if (blocks < 1) blocks = 1;
    const int per_block = (int)((items + blocks - 1) / blocks);
    const bool dn = P.S8 != nullptr || P.cm != nullptr;
    auto fn = debug_only == 1 ? (dn ? k_update<1, true> : k_update<1, false>)
            : debug_only == 2 ? (dn ? k_update<2, true> : k_update<2, false>)
                              : (dn ? k_update<0, true> : k_update<0, false>);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return tc_launch_pdl(fn, dim3((unsigned)blocks), dim3((1 + UPD_GW * pairs) * 32), smem, s, P, per_block, S);
}
