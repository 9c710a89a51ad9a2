// Relaxed loss of the TensCol iteration and its hand-written gradient, used to
// check the differentiation of eq. 7 / eq. 13 (Goudet, Duval, Hao, Section
// 3.8) against finite differences: S = softmax(W / tau) row-wise (real
// valued), eq. 7 with its GCP terms evaluated literally on S,
//   L = 1/2 sum_{i,m} a_im M~_im + lambda t kappa(M~) - mu t varpi(M~),
//   M~ = sum_d S_d S_d^T,
// and dL/dW = (1/tau) S (.) (G - (S (.) G) J) with G = B'(M~) . S_d (eq. 13),
// B'_im = a_im (1 + 2 alpha lambda t M~^(alpha-1)) - (1 - a_im) 2 beta mu t M~^(beta-1).
// FP32 CUDA-core kernels; not on the hot path.
#include <math.h>

#include "tc_internal.cuh"

namespace {

constexpr int RT = 32;  // tile edge

// S = softmax(W / tau): one warp per row.
__global__ void k_rx_softmax(const float* W, float* S, long long rows, int k, float inv_tau) {
    const long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    const float* w = W + r * k;
    float mx = -INFINITY;
    for (int j = lane; j < k; j += 32) mx = fmaxf(mx, w[j] * inv_tau);
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    float z = 0.f;
    for (int j = lane; j < k; j += 32) z += expf(w[j] * inv_tau - mx);
    for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
    for (int j = lane; j < k; j += 32) S[r * k + j] = expf(w[j] * inv_tau - mx) / z;
}

// M~[i][m] = sum_d sum_j S[d][i][j] S[d][m][j], 32 x 32 tiles, thread per entry.
__global__ void k_rx_mtilde(const float* S, float* M, int n, int D, int k) {
    __shared__ float a[RT][RT + 1], b[RT][RT + 1];
    const int i = blockIdx.y * RT + threadIdx.y, m = blockIdx.x * RT + threadIdx.x;
    float acc = 0.f;
    for (int d = 0; d < D; ++d)
        for (int j0 = 0; j0 < k; j0 += RT) {
            const int ia = blockIdx.y * RT + threadIdx.y, ma = blockIdx.x * RT + threadIdx.y;
            const int jj = j0 + threadIdx.x;
            a[threadIdx.y][threadIdx.x] = (ia < n && jj < k) ? S[((size_t)d * n + ia) * k + jj] : 0.f;
            b[threadIdx.y][threadIdx.x] = (ma < n && jj < k) ? S[((size_t)d * n + ma) * k + jj] : 0.f;
            __syncthreads();
#pragma unroll 8
            for (int q = 0; q < RT; ++q) acc = fmaf(a[threadIdx.y][q], b[threadIdx.x][q], acc);
            __syncthreads();
        }
    if (i < n && m < n) M[(size_t)i * n + m] = acc;
}

// B' from M~ and the loss terms (block partials: f/2, kappa, varpi).
__global__ void k_rx_coef(const float* M, const uint32_t* adj, int adj_words, int n, float alpha, float beta,
                          float cA, float cB, int bonus_diag, float* Bp, float* part) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float f = 0.f, ka = 0.f, va = 0.f;
    if (e < (long long)n * n) {
        const int i = (int)(e / n), m = (int)(e % n);
        const float x = M[e];
        const bool edge = (adj[(size_t)i * adj_words + (m >> 5)] >> (m & 31)) & 1u;
        float b = 0.f;
        if (edge) {
            f = 0.5f * x;
            ka = powf(x, alpha);
            b = 1.0f + cA * 2.0f * alpha * powf(x, alpha - 1.0f);
        } else if (m != i || bonus_diag) {
            va = powf(x, beta);
            b = -cB * 2.0f * beta * powf(x, beta - 1.0f);
        }
        Bp[e] = b;
    }
    __shared__ float sh[3][32];
    for (int o = 16; o > 0; o >>= 1) {
        f += __shfl_xor_sync(0xffffffffu, f, o);
        ka += __shfl_xor_sync(0xffffffffu, ka, o);
        va += __shfl_xor_sync(0xffffffffu, va, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = f;
        sh[1][threadIdx.x >> 5] = ka;
        sh[2][threadIdx.x >> 5] = va;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a0 += sh[0][w];
            a1 += sh[1][w];
            a2 += sh[2][w];
        }
        part[3 * blockIdx.x] = a0;
        part[3 * blockIdx.x + 1] = a1;
        part[3 * blockIdx.x + 2] = a2;
    }
}

// loss[0..3] = L, kappa, varpi, f_color (fixed-order reduction of partials).
__global__ void k_rx_loss(const float* part, int nparts, float cA, float cB, float* loss) {
    __shared__ float sh[3][32];
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
        a0 += part[3 * b];
        a1 += part[3 * b + 1];
        a2 += part[3 * b + 2];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = a0;
        sh[1][threadIdx.x >> 5] = a1;
        sh[2][threadIdx.x >> 5] = a2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float f = 0.f, ka = 0.f, va = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            f += sh[0][w];
            ka += sh[1][w];
            va += sh[2][w];
        }
        loss[0] = f + cA * ka - cB * va;
        loss[1] = ka;
        loss[2] = va;
        loss[3] = f;
    }
}

// G[d][i][:] = sum_m B'[i][m] S[d][m][:], then dL/dW for the row: block per
// (32-row tile, d), k <= 128 columns, B' and S tiles through shared memory.
__global__ void k_rx_grad(const float* Bp, const float* S, int n, int k, float inv_tau, float* gradW) {
    __shared__ float bs[RT][RT + 1];
    __shared__ float ss[RT][128 + 1];
    __shared__ float gs[RT][128 + 1];
    const int d = blockIdx.y, i0 = blockIdx.x * RT;
    const int tid = threadIdx.x;  // 256 threads
    for (int e = tid; e < RT * k; e += blockDim.x) gs[e / k][e % k] = 0.f;
    for (int m0 = 0; m0 < n; m0 += RT) {
        __syncthreads();
        for (int e = tid; e < RT * RT; e += blockDim.x) {
            const int r = e / RT, c = e % RT;
            bs[r][c] = (i0 + r < n && m0 + c < n) ? Bp[(size_t)(i0 + r) * n + m0 + c] : 0.f;
        }
        for (int e = tid; e < RT * k; e += blockDim.x) {
            const int r = e / k, j = e % k;
            ss[r][j] = (m0 + r < n) ? S[((size_t)d * n + m0 + r) * k + j] : 0.f;
        }
        __syncthreads();
        for (int e = tid; e < RT * k; e += blockDim.x) {
            const int r = e / k, j = e % k;
            float acc = gs[r][j];
#pragma unroll 8
            for (int q = 0; q < RT; ++q) acc = fmaf(bs[r][q], ss[q][j], acc);
            gs[r][j] = acc;
        }
    }
    __syncthreads();
    // one warp per row: dL/dW = (1/tau) S (.) (G - <S, G>)
    const int warp = tid >> 5, lane = tid & 31;
    for (int r = warp; r < RT; r += blockDim.x >> 5) {
        const int i = i0 + r;
        if (i >= n) continue;
        const float* srow = S + ((size_t)d * n + i) * k;
        float dot = 0.f;
        for (int j = lane; j < k; j += 32) dot += srow[j] * gs[r][j];
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        for (int j = lane; j < k; j += 32)
            gradW[((size_t)d * n + i) * k + j] = inv_tau * srow[j] * (gs[r][j] - dot);
    }
}

}  // namespace

int tc_relaxed_run(const tc_kparams& P, const float* W, float tau, long long t, float* loss, float* gradW,
                   float* S, float* M, float* Bp, float* part, cudaStream_t s) {
    const int n = P.n, D = P.D, k = P.k;
    if (k > 128) return TC_ERR_UNSUPPORTED;
    const long long rows = (long long)D * n;
    const float cA = (float)((double)P.lambda_ * (double)t), cB = (float)((double)P.mu * (double)t);
    k_rx_softmax<<<(unsigned)((rows + 7) / 8), 256, 0, s>>>(W, S, rows, k, 1.0f / tau);
    dim3 gm((n + RT - 1) / RT, (n + RT - 1) / RT);
    k_rx_mtilde<<<gm, dim3(RT, RT), 0, s>>>(S, M, n, D, k);
    const long long nn = (long long)n * n;
    const int cb = (int)((nn + 255) / 256);
    k_rx_coef<<<cb, 256, 0, s>>>(M, P.adj, P.adj_words, n, P.alpha, P.beta, cA, cB, P.bonus_diag, Bp, part);
    k_rx_loss<<<1, 256, 0, s>>>(part, cb, cA, cB, loss);
    dim3 gg((n + RT - 1) / RT, D);
    k_rx_grad<<<gg, 256, 0, s>>>(Bp, S, n, k, 1.0f / tau, gradW);
    return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

int tc_relaxed_partials(int n) { return (int)(((long long)n * n + 255) / 256); }
