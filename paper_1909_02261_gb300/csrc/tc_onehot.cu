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
#include <math.h>
#include <stdio.h>

#include "tc_internal.cuh"

namespace {

constexpr int PT = 32;              // pair tile edge
constexpr int PAIR_THREADS = 256;   // 8 warps x 4 rows each
constexpr int PAIR_CW = 128;        // colour words (2 individuals each) per chunk
constexpr int CLS_THREADS = 256;
constexpr int UPD_MAX_WARPS = 8;

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

__global__ void k_init_weights(float* W, long long count, unsigned long long seed, float sigma0) {
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
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (g * 4 + q < count) W[g * 4 + q] = z[q] * sigma0;
}

// ---------------------------------------------------------------------------
// Step 1 (Section 3.4) for a fresh W: c_d(i) = lowest j with maximal w.
// ---------------------------------------------------------------------------
__global__ void k_assign(tc_kparams P) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (long long)P.D * P.n) return;
    const float* w = P.W + r * P.k;
    int best = 0;
    float bv = w[0];
    for (int j = 1; j < P.k; ++j) {
        const float v = w[j];
        if (v > bv) {
            bv = v;
            best = j;
        }
    }
    const int d = (int)(r / P.n), i = (int)(r % P.n);
    P.c[r] = (uint16_t)best;
    P.cT[(size_t)i * P.Dp + d] = (uint16_t)best;
}

// ---------------------------------------------------------------------------
// k_pairs: one 32x32 tile (I <= M) of vertex pairs per block.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(PAIR_THREADS) k_pairs(tc_kparams P) {
    if (P.commit && P.st->stop) return;
    __shared__ uint32_t s_ci[PT][PAIR_CW + 1];
    __shared__ uint32_t s_cm[PT][PAIR_CW + 1];
    __shared__ int s_conf[2 * PAIR_CW];
    __shared__ float s_bt[PT][PT + 1];
    __shared__ int s_mt[PT][PT + 1];
    __shared__ float s_red[2][PAIR_THREADS / 32];

    const int n = P.n, D = P.D;
    const int2 tile = P.pair_tiles[blockIdx.x];
    const int I = tile.x, M = tile.y;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const int m = M * PT + tx;
    const int Dw = P.Dp >> 1;
    const uint32_t* cTw = reinterpret_cast<const uint32_t*>(P.cT);

    // which of my 4 pairs are edges / count towards the fitness (strict upper)
    bool edge[4], upper[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int i = I * PT + ty + 8 * r;
        const bool ok = (i < n) && (m < n);
        edge[r] = ok && ((P.adj[(size_t)i * P.adj_words + (m >> 5)] >> (m & 31)) & 1u);
        upper[r] = ok && (I < M || tx > ty + 8 * r);
    }

    int cnt[4] = {0, 0, 0, 0};
    for (int w0 = 0; w0 < Dw; w0 += PAIR_CW) {
        const int cw = min(PAIR_CW, Dw - w0);
        __syncthreads();
        for (int e = tid; e < PT * cw; e += PAIR_THREADS) {
            const int r = e / cw, w = e - r * cw;
            const int ii = I * PT + r, mm = M * PT + r;
            s_ci[r][w] = ii < n ? cTw[(size_t)ii * Dw + w0 + w] : 0xFFFFFFFFu;
            s_cm[r][w] = mm < n ? cTw[(size_t)mm * Dw + w0 + w] : 0xFFFFFFFFu;
        }
        for (int e = tid; e < 2 * PAIR_CW; e += PAIR_THREADS) s_conf[e] = 0;
        __syncthreads();
        for (int w = 0; w < cw; ++w) {
            const uint32_t b = s_cm[tx][w];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const uint32_t eq = __vcmpeq2(s_ci[ty + 8 * r][w], b);
                cnt[r] += __popc(eq);
                if (eq && edge[r] && upper[r]) {  // conflicts on this edge
                    if (eq & 1u) atomicAdd(&s_conf[2 * w], 1);
                    if (eq & 0x10000u) atomicAdd(&s_conf[2 * w + 1], 1);
                }
            }
        }
        __syncthreads();
        for (int e = tid; e < 2 * cw; e += PAIR_THREADS) {
            const int d = 2 * w0 + e;
            const int v = s_conf[e];
            if (v && d < D) atomicAdd(&P.fcolor[d], v);
        }
    }

    // pair coefficient of eq. 13 and loss terms of eq. 5-6
    const long long t = P.st->t;
    const float cA = (float)((double)P.lambda_ * (double)t);
    const float cB = (float)((double)P.mu * (double)t);
    const int pad = P.Dp - D;  // padded colour slots always compare equal
    float kap = 0.f, var = 0.f;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int il = ty + 8 * r;
        const int i = I * PT + il;
        float b = 0.f;
        int mt = 0;
        if (i < n && m < n && (I < M || tx >= il)) {
            mt = (cnt[r] >> 4) - pad;
            if (m == i) {
                mt = D;
                if (P.bonus_diag) {
                    b = -cB * P.lutB[D];
                    var += P.powB[D];
                }
            } else if (edge[r]) {
                b = fmaf(cA, P.lutA[mt], 1.0f);
                kap += 2.0f * P.powA[mt];
            } else {
                b = -cB * P.lutB[mt];
                var += 2.0f * P.powB[mt];
            }
            P.B[(size_t)i * n + m] = b;
            if (P.dbg_Mt) P.dbg_Mt[(size_t)i * n + m] = mt;
        }
        s_bt[tx][il] = b;
        s_mt[tx][il] = mt;
    }
    __syncthreads();
    // transposed write of the strictly-lower counterpart: B[m][i] = B[i][m]
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int ml = ty + 8 * r;    // row of the transposed tile
        const int mm = M * PT + ml;
        const int ii = I * PT + tx;
        if (mm < n && ii < n && (I < M || tx < ml)) {
            P.B[(size_t)mm * n + ii] = s_bt[ml][tx];
            if (P.dbg_Mt) P.dbg_Mt[(size_t)mm * n + ii] = s_mt[ml][tx];
        }
    }
    // block partial sums (fixed order -> deterministic)
    kap = warp_sum(kap);
    var = warp_sum(var);
    if (tx == 0) {
        s_red[0][ty] = kap;
        s_red[1][ty] = var;
    }
    __syncthreads();
    if (tid == 0) {
        float a = 0.f, v = 0.f;
        for (int q = 0; q < PAIR_THREADS / 32; ++q) {
            a += s_red[0][q];
            v += s_red[1][q];
        }
        P.loss_part[2 * blockIdx.x] = a;
        P.loss_part[2 * blockIdx.x + 1] = v;
    }
}

// ---------------------------------------------------------------------------
// block-wide helpers for k_classes (CLS_THREADS threads)
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

__device__ unsigned long long block_min_u64(unsigned long long v, unsigned long long* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u < v ? u : v;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    unsigned long long s = sh[0];
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) s = sh[q] < s ? sh[q] : s;
    return s;
}

// Population reduction of one iteration, run by the last k_classes block:
// min_d f(S_d) with the lowest d on ties (Algorithm 1 stop test), the
// best-so-far copy, the loss of eq. 7 and the stop flag.
__device__ void finalize_population(const tc_kparams& P) {
    __shared__ long long sh_ll[CLS_THREADS / 32];
    __shared__ float sh_f[CLS_THREADS / 32];
    __shared__ unsigned long long sh_u[CLS_THREADS / 32];
    __shared__ int s_dstar, s_better;
    tc_dev_state* st = P.st;
    const int D = P.D;
    long long fc = 0, fe = 0;
    unsigned long long key = ~0ull;
    for (int d = threadIdx.x; d < D; d += blockDim.x) {
        const int a = __ldcg(P.fcolor + d), b = __ldcg(P.feq + d);
        fc += a;
        fe += b;
        const unsigned long long f = (unsigned long long)(a + (P.problem == TC_ECP ? b : 0));
        const unsigned long long kk = (f << 32) | (unsigned)d;
        key = kk < key ? kk : key;
    }
    fc = block_sum<long long>(fc, sh_ll);
    fe = block_sum<long long>(fe, sh_ll);
    key = block_min_u64(key, sh_u);
    float ka = 0.f, va = 0.f;
    for (int b = threadIdx.x; b < P.n_pair_blocks; b += blockDim.x) {
        ka += __ldcg(P.loss_part + 2 * b);
        va += __ldcg(P.loss_part + 2 * b + 1);
    }
    ka = block_sum<float>(ka, sh_f);
    va = block_sum<float>(va, sh_f);
    const int fmin = (int)(key >> 32), dstar = (int)(key & 0xffffffffu);
    const long long t = st->t;
    if (threadIdx.x == 0) {
        const double tt = (double)t;
        st->loss = (float)fc + (float)((double)P.nu * tt) * (float)fe +
                   (float)((double)P.lambda_ * tt) * ka - (float)((double)P.mu * tt) * va;
        st->kappa = ka;
        st->varpi = va;
        st->fcolor_sum = fc;
        st->last_fmin = fmin;
        st->last_dstar = dstar;
        int better = 0;
        if (P.commit) {
            st->evaluated += 1;
            if (st->best_f < 0 || fmin < st->best_f) {
                better = 1;
                st->best_f = fmin;
                st->best_fcolor = __ldcg(P.fcolor + dstar);
                st->best_feq = __ldcg(P.feq + dstar);
                st->best_d = dstar;
                st->best_t = t;
            }
            if (P.stop_on_legal && fmin == 0) st->stop = 1;
        }
        s_dstar = dstar;
        s_better = better;
    }
    __syncthreads();
    if (s_better)
        for (int i = threadIdx.x; i < P.n; i += blockDim.x)
            P.best[i] = P.c[(size_t)s_dstar * P.n + i];
    if (threadIdx.x == 0) st->done_classes = 0u;
}

// ---------------------------------------------------------------------------
// k_classes: one individual per block.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(CLS_THREADS) k_classes(tc_kparams P) {
    if (P.commit && P.st->stop) return;
    __shared__ int s_hist[TC_MAX_K];
    __shared__ int s_cur[TC_MAX_K];
    __shared__ int s_scan[CLS_THREADS];
    __shared__ long long sh_ll[CLS_THREADS / 32];
    __shared__ int s_last;
    const int n = P.n, k = P.k, d = blockIdx.x;
    const uint16_t* cd = P.c + (size_t)d * n;
    for (int j = threadIdx.x; j < k; j += blockDim.x) s_hist[j] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&s_hist[cd[i]], 1);
    __syncthreads();
    // exclusive scan of the class sizes: contiguous chunks per thread
    const int per = (k + CLS_THREADS - 1) / CLS_THREADS;
    const int j0 = threadIdx.x * per, j1 = min(k, j0 + per);
    int local = 0;
    for (int j = j0; j < j1; ++j) local += s_hist[j];
    s_scan[threadIdx.x] = local;
    __syncthreads();
    for (int o = 1; o < CLS_THREADS; o <<= 1) {  // Hillis-Steele inclusive scan
        const int v = threadIdx.x >= o ? s_scan[threadIdx.x - o] : 0;
        __syncthreads();
        s_scan[threadIdx.x] += v;
        __syncthreads();
    }
    int run = s_scan[threadIdx.x] - local;
    int* od = P.off + (size_t)d * (k + 1);
    for (int j = j0; j < j1; ++j) {
        od[j] = run;
        s_cur[j] = run;
        run += s_hist[j];
    }
    if (threadIdx.x == 0) od[k] = n;
    // equity fitness (eq. 3) and its gradient sign (eq. 14)
    const int c1 = n / k, c2 = (n + k - 1) / k;
    long long fe = 0;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        const int h = s_hist[j];
        fe += min(abs(h - c1), abs(h - c2));
        P.E[(size_t)d * k + j] = (int8_t)(h > c2 ? 1 : (h < c1 ? -1 : 0));
    }
    fe = block_sum<long long>(fe, sh_ll);
    if (threadIdx.x == 0) P.feq[d] = (int)fe;
    __syncthreads();
    // stable counting sort of the vertices by colour (warp 0, 32 at a time)
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        uint16_t* pd = P.perm + (size_t)d * n;
        for (int base = 0; base < n; base += 32) {
            const int i = base + lane;
            const unsigned valid = __ballot_sync(0xffffffffu, i < n);
            if (i < n) {
                const int col = cd[i];
                const unsigned peers = __match_any_sync(valid, col);
                const int rank = __popc(peers & ((1u << lane) - 1u));
                pd[s_cur[col] + rank] = (uint16_t)i;
                __syncwarp(valid);
                if ((__ffs(peers) - 1) == lane) s_cur[col] += __popc(peers);
            }
            __syncwarp();
        }
    }
    // completion ticket: the last block reduces the population
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned ticket = atomicAdd(&P.st->done_classes, 1u);
        s_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        finalize_population(P);
    }
}

// ---------------------------------------------------------------------------
// k_update: Step 3-ii + Step 4 for (32-vertex tile, individual) items.
// KREG > 0 keeps the tile's grad_S rows in registers (k <= KREG), else in
// shared memory.  BTS stages the tile's columns of B in shared memory.
// ---------------------------------------------------------------------------
template <int KREG, bool BTS>
__device__ __forceinline__ void update_item(const tc_kparams& P, const float* Bt, float* Ws,
                                            float* Gs, int T, int d, float nut, bool smooth,
                                            int debug_only) {
    const int n = P.n, k = P.k, k1 = k + 1;
    const int lane = threadIdx.x & 31;
    const int i0 = T * 32;
    const int rows = min(32, n - i0);
    const uint16_t* pm = P.perm + (size_t)d * n;
    const int* of = P.off + (size_t)d * (k + 1);
    const int8_t* Ed = P.E + (size_t)d * k;
    const float* Bcol;
    int bstride;
    if (BTS) {
        Bcol = Bt + lane;
        bstride = 32;
    } else {
        Bcol = P.B + min(i0 + lane, n - 1);
        bstride = n;
    }
    float Gr[KREG > 0 ? KREG : 1];

    // Phase A: grad_S L row of vertex i0 + lane, one colour class at a time
    auto class_sum = [&](int j) -> float {
        const int s = __ldg(of + j), e = __ldg(of + j + 1);
        float a0 = 0.f, a1 = 0.f;
        int p = s;
        for (; p + 1 < e; p += 2) {
            const int m0 = __ldg(pm + p), m1 = __ldg(pm + p + 1);
            a0 += Bcol[m0 * bstride];
            a1 += Bcol[m1 * bstride];
        }
        if (p < e) a0 += Bcol[__ldg(pm + p) * bstride];
        return (a0 + a1) + nut * (float)__ldg(Ed + j);
    };
    if (KREG > 0) {
#pragma unroll
        for (int j = 0; j < (KREG > 0 ? KREG : 1); ++j)
            if (j < k) Gr[j] = class_sum(j);
    } else {
        for (int j = 0; j < k; ++j) Gs[j * 33 + lane] = class_sum(j);
    }
    if (debug_only) {
        if (lane < rows) {
            float* g = P.dbg_G + ((size_t)d * n + i0 + lane) * k;
            if (KREG > 0) {
#pragma unroll
                for (int j = 0; j < (KREG > 0 ? KREG : 1); ++j)
                    if (j < k) g[j] = Gr[j];
            } else {
                for (int j = 0; j < k; ++j) g[j] = Gs[j * 33 + lane];
            }
        }
        __syncwarp();
        return;
    }
    auto Gget = [&](int j) -> float { return KREG > 0 ? Gr[j] : Gs[j * 33 + lane]; };

    // Phase B: the 32 x k weight tile through shared memory (coalesced)
    const size_t wbase = ((size_t)d * n + i0) * k;
    const int cnt = rows * k;
    {
        int r = 0, j = lane;
        while (j >= k) { j -= k; ++r; }
        for (int e = lane; e < cnt; e += 32) {
            Ws[r * k1 + j] = P.W[wbase + e];
            j += 32;
            while (j >= k) { j -= k; ++r; }
        }
    }
    __syncwarp();
    int newc = 0;
    if (lane < rows) {
        float* w = Ws + lane * k1;
        float mx = w[0];
        for (int j = 1; j < k; ++j) mx = fmaxf(mx, w[j]);
        float Z = 0.f, num = 0.f;
        if (KREG > 0) {
#pragma unroll
            for (int j = 0; j < (KREG > 0 ? KREG : 1); ++j)
                if (j < k) {
                    const float e = __expf(w[j] - mx);
                    Z += e;
                    num = fmaf(e, Gget(j), num);
                }
        } else {
            for (int j = 0; j < k; ++j) {
                const float e = __expf(w[j] - mx);
                Z += e;
                num = fmaf(e, Gget(j), num);
            }
        }
        const float invZ = 1.0f / Z;
        const float dot = num * invZ;  // (S^ (.) grad_S L) . J of eq. 12
        float bestv = -INFINITY;
        auto upd = [&](int j) {
            const float s = __expf(w[j] - mx) * invZ;
            float wn = w[j] - P.eta * (s * (Gget(j) - dot));
            if (smooth) wn = wn / P.rho;
            w[j] = wn;
            if (wn > bestv) {
                bestv = wn;
                newc = j;
            }
        };
        if (KREG > 0) {
#pragma unroll
            for (int j = 0; j < (KREG > 0 ? KREG : 1); ++j)
                if (j < k) upd(j);
        } else {
            for (int j = 0; j < k; ++j) upd(j);
        }
    }
    __syncwarp();
    {
        int r = 0, j = lane;
        while (j >= k) { j -= k; ++r; }
        for (int e = lane; e < cnt; e += 32) {
            P.W[wbase + e] = Ws[r * k1 + j];
            j += 32;
            while (j >= k) { j -= k; ++r; }
        }
    }
    if (lane < rows) {
        P.c[(size_t)d * n + i0 + lane] = (uint16_t)newc;
        P.cT[(size_t)(i0 + lane) * P.Dp + d] = (uint16_t)newc;
    }
    __syncwarp();
}

template <int KREG, bool BTS>
__global__ void __launch_bounds__(UPD_MAX_WARPS * 32, 1) k_update(tc_kparams P, int items_per_block,
                                                               int debug_only) {
    tc_dev_state* st = P.st;
    if (!debug_only && st->stop) return;
    extern __shared__ __align__(16) float sm[];
    const int n = P.n, D = P.D, k = P.k;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float* Bt = sm;
    float* Ws = sm + (BTS ? (size_t)n * 32 : 0) + (size_t)warp * (32 * (k + 1) + (KREG > 0 ? 0 : k * 33));
    float* Gs = Ws + 32 * (k + 1);
    const long long t = st->t;
    const float nut = (float)((double)P.nu * (double)t);
    const bool smooth = ((t + 1) % P.nb_iter) == 0;
    const int nT = (n + 31) / 32;
    const long long Q = (long long)nT * D;
    long long q = (long long)blockIdx.x * items_per_block;
    const long long qend = min(Q, q + items_per_block);
    while (q < qend) {
        const int T = (int)(q / D);
        const long long seg_end = min(qend, (long long)(T + 1) * D);
        if (BTS) {
            const int i0 = T * 32;
            __syncthreads();
            for (int m = warp; m < n; m += nw)
                Bt[m * 32 + lane] = (i0 + lane < n) ? P.B[(size_t)m * n + i0 + lane] : 0.f;
            __syncthreads();
        }
        for (long long qq = q + warp; qq < seg_end; qq += nw)
            update_item<KREG, BTS>(P, Bt, Ws, Gs, T, (int)(qq - (long long)T * D), nut, smooth,
                                   debug_only);
        q = seg_end;
    }
    if (!debug_only) {
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned ticket = atomicAdd(&st->done_update, 1u);
            if (ticket == gridDim.x - 1) {
                st->done_update = 0u;
                st->t = t + 1;
                __threadfence();
            }
        }
    }
}

// gamma_own[d, i] = conflicting neighbours (eq. 1), for tc_evaluate only.
__global__ void k_debug_gamma(tc_kparams P) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (long long)P.D * P.n) return;
    const int d = (int)(r / P.n), i = (int)(r % P.n);
    const uint16_t* cd = P.c + (size_t)d * P.n;
    const int ci = cd[i];
    int g = 0;
    for (int e = P.rowptr[i]; e < P.rowptr[i + 1]; ++e) g += (cd[P.colidx[e]] == ci);
    P.dbg_gamma[r] = g;
}

constexpr int kSmemOptin = 232448;  // 227 KB per block on sm_100 / sm_103

int pick_kreg(int k) { return k <= 32 ? 32 : (k <= 64 ? 64 : (k <= 96 ? 96 : 0)); }

}  // namespace

int tc_pair_tile_count(int n) {
    const int T = (n + PT - 1) / PT;
    return T * (T + 1) / 2;
}

int tc_update_config(int n, int k, int* warps, int* smem_bytes, int* bt_in_smem) {
    const int kreg = pick_kreg(k);
    const long long per_warp = 4ll * (32ll * (k + 1) + (kreg > 0 ? 0 : 33ll * k));
    const long long bt = 4ll * 32 * n;
    int w = 0, bts = 0;
    if (bt + per_warp <= kSmemOptin) {
        bts = 1;
        w = (int)((kSmemOptin - bt) / per_warp);
    } else {
        w = (int)(kSmemOptin / per_warp);
    }
    w = w > UPD_MAX_WARPS ? UPD_MAX_WARPS : w;
    if (w < 1) return TC_ERR_UNSUPPORTED;
    *warps = w;
    *bt_in_smem = bts;
    *smem_bytes = (int)((bts ? bt : 0) + per_warp * w);
    return TC_OK;
}

cudaError_t tc_launch_init_weights(float* W, long long count, unsigned long long seed, float sigma0,
                                   cudaStream_t s) {
    const long long groups = (count + 3) / 4;
    const int th = 256;
    k_init_weights<<<(unsigned)((groups + th - 1) / th), th, 0, s>>>(W, count, seed, sigma0);
    return cudaGetLastError();
}

cudaError_t tc_launch_assign(const tc_kparams& P, cudaStream_t s) {
    const long long rows = (long long)P.D * P.n;
    k_assign<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t tc_launch_pairs(const tc_kparams& P, cudaStream_t s) {
    k_pairs<<<P.n_pair_blocks, PAIR_THREADS, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t tc_launch_classes(const tc_kparams& P, cudaStream_t s) {
    k_classes<<<P.D, CLS_THREADS, 0, s>>>(P);
    return cudaGetLastError();
}

template <int KREG, bool BTS>
static cudaError_t launch_update_t(const tc_kparams& P, int blocks, int warps, int smem,
                                   int per_block, cudaStream_t s, int debug_only) {
    auto fn = k_update<KREG, BTS>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    fn<<<blocks, warps * 32, smem, s>>>(P, per_block, debug_only);
    return cudaGetLastError();
}

cudaError_t tc_launch_update(const tc_kparams& P, int num_sms, cudaStream_t s, int debug_only) {
    int warps = 0, smem = 0, bts = 0;
    if (tc_update_config(P.n, P.k, &warps, &smem, &bts) != TC_OK) return cudaErrorInvalidValue;
    const long long items = (long long)((P.n + 31) / 32) * P.D;
    long long blocks = num_sms;  // one resident block per SM (shared-memory bound)
    if (blocks > items) blocks = items;
    if (blocks < 1) blocks = 1;
    const int per_block = (int)((items + blocks - 1) / blocks);
    const int kreg = pick_kreg(P.k);
#define TC_UPD(KR)                                                                                \
    return bts ? launch_update_t<KR, true>(P, (int)blocks, warps, smem, per_block, s, debug_only)  \
               : launch_update_t<KR, false>(P, (int)blocks, warps, smem, per_block, s, debug_only)
    switch (kreg) {
        case 32: TC_UPD(32);
        case 64: TC_UPD(64);
        case 96: TC_UPD(96);
        default: TC_UPD(0);
    }
#undef TC_UPD
}

cudaError_t tc_launch_debug_gamma(const tc_kparams& P, cudaStream_t s) {
    const long long rows = (long long)P.D * P.n;
    k_debug_gamma<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(P);
    return cudaGetLastError();
}
