// Pair terms of a population without any device allocation.
//
// Some callers cannot allocate device memory at all: a host process that
// shares a GPU whose memory another framework's pool manages, a
// latency-critical loop that must not call cudaMalloc / cudaFree (both can
// synchronise the whole device), or an embedding whose device memory budget
// is fixed at start-up.  For them this file offers one entry point that takes
// its inputs and output from the caller and keeps its scratch (the per-tile
// partial sums and a completion ticket) in a file-scope device array.  The
// array is part of the library image: every GPU that loads the library holds
// it until the process exits.
#include <math.h>
#include <mutex>

#include "tc_internal.cuh"

namespace {

constexpr int NT = 32;                    // vertex tile edge
constexpr int NA_THREADS = 256;           // 16 x 16 threads, 2 x 2 pairs each
constexpr int NA_DCHUNK = 128;            // individuals staged per pass
constexpr int kMaxTiles = (TC_NOALLOC_MAX_N / NT) * (TC_NOALLOC_MAX_N / NT + 1) / 2;
constexpr size_t kScratchBytes = 256 + sizeof(float) * 2 * (size_t)kMaxTiles;
static_assert(kScratchBytes <= TC_NOALLOC_SCRATCH_BYTES, "scratch size");

// [0, 4): completion ticket; [256, ...): 2 floats per tile (kappa, varpi)
static __device__ __align__(256) unsigned char g_scratch[TC_NOALLOC_SCRATCH_BYTES];

__global__ void __launch_bounds__(NA_THREADS) k_pairs_noalloc(int n, int D, const uint16_t* colors,
                                                              const uint8_t* adj, float alpha, float beta,
                                                              int bonus_diag, float* out, unsigned char* scratch) {
    __shared__ uint16_t s_ci[NA_DCHUNK][NT + 1];
    __shared__ uint16_t s_cm[NA_DCHUNK][NT + 1];
    __shared__ float s_red[2][NA_THREADS / 32];
    __shared__ int s_last;
    unsigned* ticket = reinterpret_cast<unsigned*>(scratch);
    float* part = reinterpret_cast<float*>(scratch + 256);
    const int T = (n + NT - 1) / NT;
    // tile (I, M), I <= M, from the block index (row-major upper triangle)
    int I = 0, rem = blockIdx.x;
    while (rem >= T - I) {
        rem -= T - I;
        ++I;
    }
    const int M = I + rem;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    int cnt[2][2] = {{0, 0}, {0, 0}};
    for (int d0 = 0; d0 < D; d0 += NA_DCHUNK) {
        const int dc = min(NA_DCHUNK, D - d0);
        __syncthreads();
        for (int e = tid; e < dc * NT; e += NA_THREADS) {
            const int dd = e / NT, r = e % NT;
            const int i = I * NT + r, m = M * NT + r;
            s_ci[dd][r] = i < n ? colors[(size_t)(d0 + dd) * n + i] : 0xFFFFu;
            s_cm[dd][r] = m < n ? colors[(size_t)(d0 + dd) * n + m] : 0xFFFEu;
        }
        __syncthreads();
        for (int dd = 0; dd < dc; ++dd)
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b) cnt[a][b] += s_ci[dd][ty + 16 * a] == s_cm[dd][tx + 16 * b];
    }
    float kap = 0.f, var = 0.f;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int il = ty + 16 * a, ml = tx + 16 * b;
            const int i = I * NT + il, m = M * NT + ml;
            if (i >= n || m >= n || (I == M && ml < il)) continue;
            const float x = (float)cnt[a][b];
            if (m == i) {
                if (bonus_diag) var += powf((float)D, beta);
            } else if (adj[(size_t)i * n + m]) {
                kap += 2.0f * powf(x, alpha);  // ordered pairs: (i, m) and (m, i)
            } else {
                var += 2.0f * powf(x, beta);
            }
        }
    for (int o = 16; o > 0; o >>= 1) {
        kap += __shfl_xor_sync(0xffffffffu, kap, o);
        var += __shfl_xor_sync(0xffffffffu, var, o);
    }
    if ((tid & 31) == 0) {
        s_red[0][tid >> 5] = kap;
        s_red[1][tid >> 5] = var;
    }
    __syncthreads();
    if (tid == 0) {
        float ka = 0.f, va = 0.f;
        for (int w = 0; w < NA_THREADS / 32; ++w) {
            ka += s_red[0][w];
            va += s_red[1][w];
        }
        part[2 * blockIdx.x] = ka;
        part[2 * blockIdx.x + 1] = va;
        __threadfence();
        s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    // the last block sums the tile partials in a fixed order
    __threadfence();
    float ka = 0.f, va = 0.f;
    for (int b = tid; b < (int)gridDim.x; b += NA_THREADS) {
        ka += __ldcg(part + 2 * b);
        va += __ldcg(part + 2 * b + 1);
    }
    for (int o = 16; o > 0; o >>= 1) {
        ka += __shfl_xor_sync(0xffffffffu, ka, o);
        va += __shfl_xor_sync(0xffffffffu, va, o);
    }
    __syncthreads();
    if ((tid & 31) == 0) {
        s_red[0][tid >> 5] = ka;
        s_red[1][tid >> 5] = va;
    }
    __syncthreads();
    if (tid == 0) {
        float k2 = 0.f, v2 = 0.f;
        for (int w = 0; w < NA_THREADS / 32; ++w) {
            k2 += s_red[0][w];
            v2 += s_red[1][w];
        }
        out[0] = k2;
        out[1] = v2;
        *ticket = 0u;
    }
}

std::mutex g_mu;
// Device address of g_scratch per device, valid for the CUDA context it was
// looked up in: a reset of the device's primary context (cudaDeviceReset)
// makes a new context in which the array may live elsewhere.
unsigned char* g_addr[256] = {nullptr};
CUcontext g_addr_ctx[256] = {nullptr};

// The calling thread's current driver context (cuCtxGetCurrent, reached
// through the runtime's driver entry-point query), or nullptr on failure.
CUcontext current_context() {
    typedef CUresult (*get_fn)(CUcontext*);
    static get_fn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p) {
            (void)cudaGetLastError();
            return nullptr;
        }
        fn = (get_fn)p;
    }
    CUcontext c = nullptr;
    return fn(&c) == CUDA_SUCCESS ? c : nullptr;
}

}  // namespace

extern "C" int tc_pair_terms_noalloc(int n, int D, const uint16_t* colors_dev, const uint8_t* adj_dev,
                                     float alpha, float beta, int bonus_diag, float* out_dev, void* stream) {
    if (n < 1 || n > TC_NOALLOC_MAX_N || D < 1 || D > TC_MAX_D || !colors_dev || !adj_dev || !out_dev)
        return TC_ERR_ARG;
    if (!(alpha > 1.f) || !(beta > 1.f)) return TC_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        (void)cudaGetLastError();
        return TC_ERR_CUDA;
    }
    unsigned char* scratch;
    {
        // first call on a device (or in a new context of it): look up where
        // the array lives there (the host-side symbol is only a stand-in, not
        // a device address); cudaGetSymbolAddress also makes the context
        // current, so the context is read after it
        std::lock_guard<std::mutex> lock(g_mu);
        const CUcontext now = current_context();
        if (!g_addr[dev] || !now || now != g_addr_ctx[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
                (void)cudaGetLastError();
                return TC_ERR_CUDA;
            }
            g_addr[dev] = static_cast<unsigned char*>(p);
            g_addr_ctx[dev] = current_context();
        }
        scratch = g_addr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the array keeps the previous call's contents: the ticket must start at 0
    if (cudaMemsetAsync(scratch, 0, sizeof(unsigned), s) != cudaSuccess) {
        (void)cudaGetLastError();
        return TC_ERR_CUDA;
    }
    const int T = (n + NT - 1) / NT;
    k_pairs_noalloc<<<T * (T + 1) / 2, NA_THREADS, 0, s>>>(n, D, colors_dev, adj_dev, alpha, beta, bonus_diag,
                                                           out_dev, scratch);
    if (cudaGetLastError() != cudaSuccess) return TC_ERR_CUDA;
    return TC_OK;
}
