// Dense forms of the two contractions of the TensCol iteration (Goudet,
// Duval, Hao, Algorithm 1):
//   Gamma = A . S_cat        Step 2 / first term of eq. 13 (the gamma matrix)
//   M~    = S_cat . S_cat^T  Step 3-i, eq. 4
// with S_cat (n x D k) the one-hot population side by side.  Both are
// C[M x N] = X[M x K] . Y[N x K]^T with X and Y holding only 0 and 1, which
// FP8 E4M3 represents exactly; FP32 accumulation is exact below 2^24, so the
// results are the exact integer counts.
//
//   k_gemm_tc    tcgen05.mma (kind::f8f6f4, K = 32) on the 5th-generation
//                tensor cores: persistent CTA per SM, warp 0 streams
//                128B-swizzled K-major tiles with TMA into a shared-memory
//                ring of ~192 KB, warp 1 issues the MMAs into one of two TMEM
//                accumulators, eight epilogue warps drain the other
//                (tcgen05.ld) and store it with TMA, each its own 32 rows of
//                half the columns, without handshakes.  Units of 128
//                rows run on one CTA (M = 128, N = 128 / 256, clusters
//                sharing the B tile by multicast) or units of 256 rows on a
//                CTA pair (cta_group::2, M = 256: each CTA loads half of the
//                B tile, so a CTA moves a third fewer operand bytes per MMA).
//   k_gemm_simt  the same contraction with FP32 FFMA on the CUDA cores (the
//                plain FP32 comparator), same work units and epilogues.
//
// Work is a host-built list of units (tile row, tile column, first and last
// K block); the M~ units cover only tiles touching the upper triangle and may
// split K, their partial sums being added in L2 by TMA reduce-adds (FP32
// atomics in the comparator; exact either way: integer values).  Every mbarrier wait is bounded by one second of wall
// time; on expiry the kernel records TC_ERR_TIMEOUT, drains its MMAs, frees
// TMEM and returns.
#include <cuda_fp8.h>
#include <stdint.h>

#include "tc_internal.cuh"

namespace {

constexpr int BM = 128, BK = 128;  // BK in bytes = FP8 elements
constexpr int BN = 256;            // column tile of the FP32 comparator and the padding unit
// Epilogue warps: two per TMEM lane quarter, each draining half of the
// accumulator's columns (one warp per quarter could not keep up with the
// MMAs of the short-K Gamma tiles).
constexpr int EPI_WARPS = 8;
constexpr int TC_THREADS = 32 * (2 + EPI_WARPS);  // producer, MMA, epilogue warps
// Output staging of the tensor-core epilogue: 32 KB after the operand ring,
// 4 KB per epilogue warp, which stages and sends its own 32 rows without
// waiting for the other warps: two 2 KB buffers of [32 columns][32 rows]
// uint16 for Gamma (one TMA store each), or one 4 KB buffer of [32 rows][32
// floats], 128-byte swizzled, for M~ (one TMA reduce-add each: the split-K
// partial sums add up in L2).
constexpr int STG_BYTES = 32768;
constexpr int STG_WARP = STG_BYTES / EPI_WARPS;

// Tile shapes of the tensor-core GEMM (the column tile BN_ is tuned per
// context).  PAIR: the two CTAs of a cluster pair run one 256-row MMA
// (cta_group::2): each holds its 128 rows of A and half of the B tile, and
// its 128 rows of the accumulator.  The stage ring keeps about 192 KB of
// operands in flight.
template <int BN_, bool PAIR = false>
struct TcShape {
    static constexpr int B_ROWS = PAIR ? BN_ / 2 : BN_;  // B rows held per CTA
    static constexpr int A_BYTES = BM * BK, B_BYTES = B_ROWS * BK, STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int STAGES = 196608 / STAGE_BYTES;
    static constexpr int TM = PAIR ? 2 * BM : BM;  // output rows of a unit
    static constexpr int TMEM_COLS = 2 * BN_;      // two BN_-column FP32 accumulators
    // instruction descriptor: D = F32, A = B = E4M3, both K-major, M = TM, N = BN_
    static constexpr uint32_t IDESC =
        (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(BN_ >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
    static constexpr int SMEM = STAGES * STAGE_BYTES + STG_BYTES + 1024;  // + output staging, alignment
};

__device__ __forceinline__ uint32_t su32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long gns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void bar_init(uint64_t* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count));
}

__device__ __forceinline__ void bar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}

__device__ __forceinline__ void bar_expect_tx(uint64_t* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool bar_try(uint64_t* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false after one second or once another role aborted.
__device__ __forceinline__ bool bar_wait(uint64_t* b, unsigned parity, volatile int* abort_flag,
                                         int* err) {
    if (bar_try(b, parity)) return true;
    const unsigned long long t0 = gns();
    for (unsigned it = 1;; ++it) {
        if (bar_try(b, parity)) return true;
        if ((it & 255u) == 0) {
            if (*abort_flag) return false;
            if (gns() - t0 > 1000000000ull) {
                *abort_flag = 1;
                atomicCAS(err, 0, TC_ERR_TIMEOUT);
                return false;
            }
        }
    }
}

__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// TMA load of one box delivered to the same shared-memory offset of every CTA
// in `mask` of the cluster, completing bytes on each CTA's own barrier there.
__device__ __forceinline__ void tma_load_2d_mc(void* dst, const CUtensorMap* map, int x, int y, uint64_t* b,
                                               uint16_t mask) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.multicast::cluster"
        " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(su32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(su32(b)), "h"(mask)
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* b) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(su32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(su32(b))
        : "memory");
}

// Shared::cluster address of the same variable in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t peer_addr(const void* p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(su32(p)), "r"(rank));
    return r;
}

// TMA load into this CTA's shared memory whose bytes complete on a barrier
// of either CTA of the pair (`bar`: shared::cluster address).
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(su32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Arrive on a barrier of another CTA of the cluster (shared::cluster address).
__device__ __forceinline__ void bar_arrive_remote(uint32_t bar) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile written by TMA
// with 128-byte swizzling: rows of 128 bytes, 8-row atoms 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);  // start address
    d |= (uint64_t)1u << 16;                  // leading byte offset (unused here)
    d |= (uint64_t)(1024u >> 4) << 32;        // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1u << 46;                  // descriptor version of sm_100 family
    d |= (uint64_t)2u << 61;                  // 128-byte swizzle
    return d;
}

// One MMA of the CTA (PAIR = false) or of the CTA pair (PAIR = true, issued
// by the even CTA; the descriptors name the same offsets in both CTAs).
template <bool PAIR>
__device__ __forceinline__ void mma_f8(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       int accumulate) {
    if constexpr (PAIR)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
}

// Arrives on the barrier at the same offset in every CTA of `mask` once the
// MMAs issued so far have completed.
template <bool PAIR>
__device__ __forceinline__ void mma_commit_mc(uint64_t* b, uint16_t mask) {
    if constexpr (PAIR)
        asm volatile(
            "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
                su32(b)),
            "h"(mask)
            : "memory");
    else
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
                su32(b)),
            "h"(mask)
            : "memory");
}

template <bool PAIR>
__device__ __forceinline__ void mma_commit(uint64_t* b) {
    if constexpr (PAIR)
        asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b))
                     : "memory");
    else
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b))
                     : "memory");
}

template <bool PAIR>
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t cols) {
    if constexpr (PAIR) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)), "r"(cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
    } else {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)), "r"(cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
}

template <bool PAIR>
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t cols) {
    if constexpr (PAIR)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols));
    else
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols));
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 lanes x 32 columns of FP32 from TMEM into v (asynchronous: the values
// are valid after tmem_wait, which names the registers so that no use of
// them moves above it).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
        "%30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
          "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
          "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait(uint32_t* v) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]),
                   "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]),
                   "+r"(v[14]), "+r"(v[15]), "+r"(v[16]), "+r"(v[17]), "+r"(v[18]), "+r"(v[19]), "+r"(v[20]),
                   "+r"(v[21]), "+r"(v[22]), "+r"(v[23]), "+r"(v[24]), "+r"(v[25]), "+r"(v[26]), "+r"(v[27]),
                   "+r"(v[28]), "+r"(v[29]), "+r"(v[30]), "+r"(v[31])
                 :
                 : "memory");
}

// Gamma entry (row i, column d k + j) in the transposed layout: column-major
// over the padded rows (used by the FP32 comparator's direct stores).
__device__ __forceinline__ uint16_t* gamma_at(const tc_gemm_args& g, int row, int col) {
    return reinterpret_cast<uint16_t*>(g.C) + (size_t)col * g.rows_alloc + row;
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(su32(src))
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

__device__ __forceinline__ void tma_reduce_add_2d(const CUtensorMap* map, int x, int y, const void* src) {
    asm volatile("cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(su32(src))
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void st_shared_u16(uint32_t a, uint16_t v) {
    asm volatile("st.shared.u16 [%0], %1;" ::"r"(a), "h"(v) : "memory");
}

__device__ __forceinline__ void st_shared_v4(uint32_t a, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(x), "r"(y), "r"(z), "r"(w) : "memory");
}

// PAIR = false, CL > 1: the CL CTAs of a cluster take CL units that share the
// column tile and K range (consecutive in the unit list); each loads 1/CL of
// the B tile and multicasts it to all, so B crosses L2 once per cluster.
// PAIR = true (CL = 2): the CTA pair takes one 256-row unit; the even CTA
// waits for both CTAs' operand bytes on its own barriers and issues the
// cta_group::2 MMAs, whose completion is multicast to the barriers of both;
// each CTA drains and stores its own 128 rows.
template <int BN_, int CL, bool PAIR>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY,
              const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmX2,
              const __grid_constant__ CUtensorMap tmY2, const __grid_constant__ CUtensorMap tmC2, tc_gemm_args g) {
    static_assert(!PAIR || CL == 2, "a CTA pair is a cluster of two");
    using Sh = TcShape<BN_, PAIR>;
    constexpr int STAGES = Sh::STAGES, A_BYTES = Sh::A_BYTES, B_BYTES = Sh::B_BYTES,
                  STAGE_BYTES = Sh::STAGE_BYTES, TMEM_COLS = Sh::TMEM_COLS, TM = Sh::TM;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 128-byte swizzled tiles need 1024-byte aligned bases
    uint8_t* smem = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], tfull[2], tempty[2], drain;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    const uint32_t crank = CL > 1 ? cluster_ctarank() : 0u;
    const uint16_t cmask = (uint16_t)((1u << CL) - 1u);
    const int group = blockIdx.x / CL, ngroups = gridDim.x / CL;
    // units of this CTA: PAIR, one per cluster; else one per CTA
    const int u_first = PAIR ? group : group * CL + (int)crank, u_step = PAIR ? ngroups : ngroups * CL;
    const bool leader = !PAIR || crank == 0u;
    const int row_half = PAIR ? (int)crank * BM : 0;  // this CTA's rows inside a unit
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            bar_init(&full[s], 1);
            bar_init(&empty[s], PAIR ? 1 : CL);  // one MMA commit from every CTA issuing into the stage
        }
        for (int a = 0; a < 2; ++a) {
            bar_init(&tfull[a], 1);
            bar_init(&tempty[a], PAIR ? 2 * EPI_WARPS : EPI_WARPS);  // the epilogue warps of every CTA holding it
        }
        bar_init(&drain, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) tmem_alloc<PAIR>(&tmem_slot, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    if (CL > 1) cluster_sync_all();  // peers' barriers initialised before any multicast
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    // launched as a programmatic dependent of the previous kernel of the
    // step: the set-up above overlaps its tail; the operands it wrote (and
    // the outputs it read) are only touched after it has completed
    pdl_trigger();
    pdl_wait();

    if (warp == 0) {
        if (lane == 0) {  // TMA producer
            unsigned gk = 0;
            bool ok = true;
            for (int u = u_first; u < g.n_units && ok; u += u_step) {
                int4 w = g.units[u];
                const bool second = (w.y & TC_UNIT_SECOND) != 0;  // a unit of the other contraction
                w.y &= ~TC_UNIT_SECOND;
                const CUtensorMap* mX = second ? &tmX2 : &tmX;
                const CUtensorMap* mY = second ? &tmY2 : &tmY;
                for (int kb = w.z; kb < w.w; ++kb, ++gk) {
                    const int s = gk % STAGES;
                    const unsigned r = gk / STAGES;
                    if (!(ok = bar_wait(&empty[s], (r & 1u) ^ 1u, &abort_flag, g.err))) break;
                    uint8_t* sa = smem + s * STAGE_BYTES;
                    if constexpr (PAIR) {
                        // both CTAs' bytes complete on the even CTA's barrier
                        const uint32_t fb = peer_addr(&full[s], 0u);
                        if (leader) bar_expect_tx(&full[s], 2 * STAGE_BYTES);
                        tma_load_2d_pair(sa, mX, kb * BK, w.x * TM + row_half, fb);
                        tma_load_2d_pair(sa + A_BYTES, mY, kb * BK, w.y * BN_ + (int)crank * (BN_ / 2), fb);
                    } else {
                        bar_expect_tx(&full[s], STAGE_BYTES);
                        tma_load_2d(sa, mX, kb * BK, w.x * BM, &full[s]);
                        if (CL == 1)
                            tma_load_2d(sa + A_BYTES, mY, kb * BK, w.y * BN_, &full[s]);
                        else  // my slice of the shared B tile, to every CTA of the cluster
                            tma_load_2d_mc(sa + A_BYTES + crank * (B_BYTES / CL), mY, kb * BK,
                                           w.y * BN_ + (int)crank * (BN_ / CL), &full[s], cmask);
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && leader) {  // MMA issuer
            unsigned gk = 0, ui = 0;
            bool ok = true;
            for (int u = u_first; u < g.n_units && ok; u += u_step, ++ui) {
                const int4 w = g.units[u];
                const int a = ui & 1;
                const unsigned ua = ui >> 1;
                if (!(ok = bar_wait(&tempty[a], (ua & 1u) ^ 1u, &abort_flag, g.err))) break;
                tc_fence_after();
                const uint32_t dt = tmem + (uint32_t)(a * BN_);
                for (int kb = w.z; kb < w.w; ++kb, ++gk) {
                    const int s = gk % STAGES;
                    const unsigned r = gk / STAGES;
                    if (!(ok = bar_wait(&full[s], r & 1u, &abort_flag, g.err))) break;
                    tc_fence_after();
                    const uint32_t sa = su32(smem + s * STAGE_BYTES);
                    const uint64_t ad = sw128_desc(sa), bd = sw128_desc(sa + A_BYTES);
#pragma unroll
                    for (int kk = 0; kk < BK / 32; ++kk)  // +32 bytes = +2 in the address field
                        mma_f8<PAIR>(dt, ad + 2 * kk, bd + 2 * kk, Sh::IDESC, (kb > w.z || kk > 0) ? 1 : 0);
                    if (CL == 1)
                        mma_commit<PAIR>(&empty[s]);  // stage s is free once these MMAs finish
                    else
                        mma_commit_mc<PAIR>(&empty[s], cmask);  // ... in every CTA that holds part of it
                }
                if (ok) {
                    if (PAIR)
                        mma_commit_mc<PAIR>(&tfull[a], cmask);  // both CTAs hold rows of the accumulator
                    else
                        mma_commit<PAIR>(&tfull[a]);
                }
            }
            // drain: every issued MMA completes before TMEM is released
            mma_commit<PAIR>(&drain);
            const unsigned long long t0 = gns();
            while (!bar_try(&drain, 0)) {
                if (gns() - t0 > 1000000000ull) {
                    atomicCAS(g.err, 0, TC_ERR_TIMEOUT);
                    break;
                }
            }
        }
    } else {  // epilogue warps: TMEM lanes 32 (warp % 4) ... 32 (warp % 4) + 31
        // Each warp drains its 32 rows of the accumulator, in its share of
        // the columns, 32 columns at a time (the next chunk's TMEM load in
        // flight while the current one is staged) and sends every chunk with
        // its own TMA store (Gamma) or reduce-add (M~) from a private buffer:
        // no warp waits for another.  A buffer is reused once the bulk group
        // that read it is done (bulk groups are per thread: lane 0 issues and
        // waits for them all).
        const int q = warp & 3, ew = warp - 2;
        // [32 cols][32 rows] u16 (2 KB, Gamma) | [32 rows][32 f32] (4 KB, M~); a
        // launch of both contractions gives every chunk the 4 KB buffer
        const uint32_t bytes_b = (g.fused || g.mode != TC_GEMM_GAMMA) ? 4096u : 2048u;
        const unsigned nb = STG_WARP / bytes_b;            // buffers per warp (1, 2 or 4)
        const uint32_t stg = su32(smem + STAGES * STAGE_BYTES) + (uint32_t)ew * STG_WARP;
        uint8_t* stg_gen = smem + STAGES * STAGE_BYTES + ew * STG_WARP;
        unsigned ui = 0, gc = 0;  // unit and chunk counters
        constexpr int NCH = BN_ / 32 / (EPI_WARPS / 4);  // chunks per warp per unit (even)
        static_assert(NCH >= 2 && NCH % 2 == 0, "each epilogue warp takes an even number of chunks");
        const int cbase = (ew >> 2) * NCH;                 // its first chunk
        for (int u = u_first; u < g.n_units; u += u_step, ++ui) {
            int4 w = g.units[u];
            const bool second = (w.y & TC_UNIT_SECOND) != 0;
            w.y &= ~TC_UNIT_SECOND;
            const bool gamma = (second ? g.mode2 : g.mode) == TC_GEMM_GAMMA;
            const CUtensorMap* mC = second ? &tmC2 : &tmC;
            const int cols_alloc = second ? g.cols_alloc2 : g.cols_alloc;
            const int a = ui & 1;
            const unsigned ua = ui >> 1;
            if (!bar_wait(&tfull[a], ua & 1u, &abort_flag, g.err)) break;
            tc_fence_after();
            const int row0 = w.x * TM + row_half + 32 * q;
            const uint32_t tbase = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(a * BN_);
            // stage chunk c from v into its buffer and send it
            auto emit = [&](const uint32_t* v, int c) {
                const uint32_t b = gc % nb;
                if (gc >= nb) {  // the group that last read buffer b is nb chunks back
                    if (lane == 0) {
                        if (nb >= 4)
                            asm volatile("cp.async.bulk.wait_group.read 3;" ::: "memory");
                        else if (nb == 2)
                            asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
                        else
                            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                    }
                    __syncwarp();
                }
                if (gamma) {  // element (column e, row lane) at 2 (32 e + lane)
                    const uint32_t base = stg + b * bytes_b + 2u * (uint32_t)lane;
#pragma unroll
                    for (int e = 0; e < 32; ++e)
                        st_shared_u16(base + 64u * (uint32_t)e, (uint16_t)__float2uint_rn(__uint_as_float(v[e])));
                } else {  // row lane: 128 bytes, 16-byte chunks swizzled by row mod 8
                    const uint32_t base = stg + b * bytes_b + 128u * (uint32_t)lane;
#pragma unroll
                    for (int h = 0; h < 8; ++h)
                        st_shared_v4(base + 16u * (uint32_t)(h ^ (lane & 7)), v[4 * h], v[4 * h + 1], v[4 * h + 2],
                                     v[4 * h + 3]);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the TMA unit
                __syncwarp();
                if (lane == 0) {
                    const int col0 = w.y * BN_ + 32 * c;
                    if (!gamma)
                        tma_reduce_add_2d(mC, col0, row0, stg_gen + b * bytes_b);
                    else if (col0 < cols_alloc)  // columns past D k are padding: not stored
                        tma_store_2d(mC, row0, col0, stg_gen + b * bytes_b);
                    else
                        asm volatile("cp.async.bulk.commit_group;" ::: "memory");  // an empty group keeps the count
                }
                __syncwarp();  // converged for the next tcgen05.ld / wait
                ++gc;
            };
            uint32_t v0[32], v1[32];
            tmem_ld32(tbase + (uint32_t)(32 * cbase), v0);
#pragma unroll 1
            for (int c = cbase; c < cbase + NCH; c += 2) {
                tmem_wait(v0);
                tmem_ld32(tbase + (uint32_t)(32 * (c + 1)), v1);  // NCH is even
                emit(v0, c);
                tmem_wait(v1);
                if (c + 2 < cbase + NCH) tmem_ld32(tbase + (uint32_t)(32 * (c + 2)), v0);
                emit(v1, c + 1);
            }
            // every TMEM load of this accumulator has completed (waited above)
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                if (PAIR)  // the accumulator is free once both CTAs drained it
                    bar_arrive_remote(peer_addr(&tempty[a], 0u));
                else
                    bar_arrive(&tempty[a]);
            }
        }
        if (lane == 0) bulk_wait_all();  // the output is in global memory before the CTA exits
    }
    tc_fence_before();
    __syncthreads();
    if (CL > 1) cluster_sync_all();  // no CTA leaves while peers may still write into it
    if (warp == 1) {
        tc_fence_after();
        tmem_free<PAIR>(tmem, TMEM_COLS);
    }
}

// ---------------------------------------------------------------------------
// FP32 CUDA-core GEMM over the same operands (FP8 bytes decoded to FP32) and
// the same work units: 128 x 256 tile, 256 threads, 8 x 16 outputs each.
// ---------------------------------------------------------------------------
constexpr int SK = 32;  // K elements per shared-memory stage

__global__ void __launch_bounds__(256, 1) k_gemm_simt(const uint8_t* X, const uint8_t* Y, int ldk,
                                                    tc_gemm_args g) {
    __shared__ __align__(16) float As[SK][BM];
    __shared__ __align__(16) float Bs[SK][BN];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    for (int u = blockIdx.x; u < g.n_units; u += gridDim.x) {
        const int4 w = g.units[u];
        float acc[8][16];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 16; ++b) acc[a][b] = 0.f;
        for (int kb = w.z * (BK / SK); kb < w.w * (BK / SK); ++kb) {
            const int k0 = kb * SK;
            __syncthreads();
            {  // X tile: 128 rows x 32 bytes, one 16-byte vector per thread
                const int r = tid >> 1, h = tid & 1;
                const uint4 v = *reinterpret_cast<const uint4*>(X + (size_t)(w.x * BM + r) * ldk + k0 + 16 * h);
                const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const __half2_raw h2 = __nv_cvt_fp8x2_to_halfraw2(
                        (__nv_fp8x2_storage_t)((wv[q >> 1] >> (16 * (q & 1))) & 0xFFFFu), __NV_E4M3);
                    const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&h2));
                    As[16 * h + 2 * q][r] = f.x;
                    As[16 * h + 2 * q + 1][r] = f.y;
                }
            }
#pragma unroll
            for (int p = 0; p < 2; ++p) {  // Y tile: 256 rows x 32 bytes
                const int e = tid + 256 * p;
                const int r = e >> 1, h = e & 1;
                const uint4 v = *reinterpret_cast<const uint4*>(Y + (size_t)(w.y * BN + r) * ldk + k0 + 16 * h);
                const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const __half2_raw h2 = __nv_cvt_fp8x2_to_halfraw2(
                        (__nv_fp8x2_storage_t)((wv[q >> 1] >> (16 * (q & 1))) & 0xFFFFu), __NV_E4M3);
                    const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&h2));
                    Bs[16 * h + 2 * q][r] = f.x;
                    Bs[16 * h + 2 * q + 1][r] = f.y;
                }
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < SK; ++kk) {
                float av[8], bv[16];
                const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * 8]);
                const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][ty * 8 + 4]);
                av[0] = a0.x; av[1] = a0.y; av[2] = a0.z; av[3] = a0.w;
                av[4] = a1.x; av[5] = a1.y; av[6] = a1.z; av[7] = a1.w;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 b4 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4 + 64 * q]);
                    bv[4 * q] = b4.x; bv[4 * q + 1] = b4.y; bv[4 * q + 2] = b4.z; bv[4 * q + 3] = b4.w;
                }
#pragma unroll
                for (int a = 0; a < 8; ++a)
#pragma unroll
                    for (int b = 0; b < 16; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
            }
        }
        // outputs: rows ty*8 + a, columns tx*4 + 64*qq + r
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const int row = w.x * BM + ty * 8 + a;
            if (row >= g.rows_alloc) continue;
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                const int col = w.y * BN + tx * 4 + 64 * qq;
                if (g.mode == TC_GEMM_GAMMA) {
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        if (col + r < g.cols_alloc)
                            *gamma_at(g, row, col + r) = (uint16_t)__float2uint_rn(acc[a][4 * qq + r]);
                } else {
                    if (col + 4 > g.cols_alloc) continue;
                    float* dst = reinterpret_cast<float*>(g.C) + (size_t)row * g.ldc + col;
                    atomicAdd(reinterpret_cast<float4*>(dst),
                              make_float4(acc[a][4 * qq], acc[a][4 * qq + 1], acc[a][4 * qq + 2],
                                          acc[a][4 * qq + 3]));
                }
            }
        }
    }
}

// S_cat / S_cat^T as FP8 one-hot operands from the colours (zeroed first).
__global__ void k_onehot_build(tc_kparams P) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (long long)P.D * P.n) return;
    const int d = (int)(r / P.n), i = (int)(r % P.n);
    const int col = d * P.k + P.c[r];
    P.S8[(size_t)i * P.ldg + col] = 0x38;  // E4M3 1.0
    P.S8T[(size_t)col * P.n_pad + i] = 0x38;
}

}  // namespace

cudaError_t tc_launch_onehot_build(const tc_kparams& P, cudaStream_t s) {
    const long long rows = (long long)P.D * P.n;
    k_onehot_build<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(P);
    return cudaGetLastError();
}

int tc_gemm_tile_m() { return BM; }
int tc_gemm_tile_n() { return BN; }
int tc_gemm_tile_k() { return BK; }

template <int BN_, int CL, bool PAIR>
static cudaLaunchConfig_t tc_config(int groups, cudaStream_t s, cudaLaunchAttribute* attr, bool pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(groups * CL);
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = TcShape<BN_, PAIR>::SMEM;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 2 : 1;
    return cfg;
}

// The shared-memory opt-in of a kernel variant, set once per device (a host
// call per launch would sit between the launches of a step).
template <int BN_, int CL, bool PAIR>
static cudaError_t smem_opt_in() {
    static int done_dev = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev == done_dev) return e;
    e = cudaFuncSetAttribute(k_gemm_tc<BN_, CL, PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             TcShape<BN_, PAIR>::SMEM);
    if (e == cudaSuccess) done_dev = dev;
    return e;
}

template <int BN_, int CL, bool PAIR>
static cudaError_t launch_tc(const CUtensorMap& tmX, const CUtensorMap& tmY, const CUtensorMap& tmC,
                             const CUtensorMap& tmX2, const CUtensorMap& tmY2, const CUtensorMap& tmC2,
                             const tc_gemm_args& g, int slots, bool pdl, cudaStream_t s) {
    cudaError_t e = smem_opt_in<BN_, CL, PAIR>();
    if (e != cudaSuccess) return e;
    const int per_cluster = PAIR ? 1 : CL;  // units a cluster takes per round
    int groups = slots < g.n_units / per_cluster ? slots : g.n_units / per_cluster;
    if (groups < 1) groups = 1;
    cudaLaunchAttribute attr[2];
    cudaLaunchConfig_t cfg = tc_config<BN_, CL, PAIR>(groups, s, attr, pdl);
    return cudaLaunchKernelEx(&cfg, k_gemm_tc<BN_, CL, PAIR>, tmX, tmY, tmC, tmX2, tmY2, tmC2, g);
}

template <int BN_, int CL, bool PAIR>
static int slots_tc(int num_sms) {
    // clusters must sit inside one GPC, so fewer than num_sms / CL of them
    // may be resident at once: a grid sized past that runs a second wave
    if (smem_opt_in<BN_, CL, PAIR>() != cudaSuccess) {
        (void)cudaGetLastError();
        return num_sms / CL;
    }
    cudaLaunchAttribute attr[2];
    cudaLaunchConfig_t cfg = tc_config<BN_, CL, PAIR>(num_sms / CL, nullptr, attr, false);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_gemm_tc<BN_, CL, PAIR>, &cfg) != cudaSuccess || n < 1) {
        (void)cudaGetLastError();
        return num_sms / CL;
    }
    return n < num_sms / CL ? n : num_sms / CL;
}

int tc_gemm_cluster_slots(int tm, int cluster, int bn, int num_sms) {
    if (tm == 2 * BM) return bn == 128 ? slots_tc<128, 2, true>(num_sms) : slots_tc<256, 2, true>(num_sms);
    if (bn == 128) {
        switch (cluster) {
            case 4: return slots_tc<128, 4, false>(num_sms);
            case 2: return slots_tc<128, 2, false>(num_sms);
            default: return slots_tc<128, 1, false>(num_sms);
        }
    }
    switch (cluster) {
        case 4: return slots_tc<256, 4, false>(num_sms);
        case 2: return slots_tc<256, 2, false>(num_sms);
        default: return slots_tc<256, 1, false>(num_sms);
    }
}

// `tm`: rows of a unit, 128 (one CTA per unit) or 256 (a CTA pair per unit,
// cta_group::2 MMAs; cluster 2).  `cluster` (tm = 128): CTAs sharing each B
// tile (1, 2 or 4); the unit list must come in groups of that many units
// with equal column tile and K range.  tmY's box holds bn / cluster rows
// (tm = 128) or bn / 2 rows (tm = 256).  `bn`: the column tile (128 or 256)
// the units were cut with.  `slots`: clusters launched at most (one wave,
// from tc_gemm_cluster_slots).  tmC: the output, Gamma transposed
// [D k][n_pad] uint16, or M~ [n_pad][n_pad] f32 128-byte swizzled, both with
// 32 x 32 boxes (one warp's rows of one 32-column chunk).  `pdl`: launched as
// a programmatic dependent of the stream's previous kernel.
cudaError_t tc_launch_gemm_tc(const CUtensorMap& tmX, const CUtensorMap& tmY, const CUtensorMap& tmC,
                              const tc_gemm_args& g, int slots, int tm, int cluster, int bn, bool pdl,
                              cudaStream_t s) {
    return tc_launch_gemm_tc2(tmX, tmY, tmC, tmX, tmY, tmC, g, slots, tm, cluster, bn, pdl, s);
}

cudaError_t tc_launch_gemm_tc2(const CUtensorMap& tmX, const CUtensorMap& tmY, const CUtensorMap& tmC,
                               const CUtensorMap& tmX2, const CUtensorMap& tmY2, const CUtensorMap& tmC2,
                               const tc_gemm_args& g, int slots, int tm, int cluster, int bn, bool pdl,
                               cudaStream_t s) {
    if (tm == 2 * BM)
        return bn == 128 ? launch_tc<128, 2, true>(tmX, tmY, tmC, tmX2, tmY2, tmC2, g, slots, pdl, s)
                         : launch_tc<256, 2, true>(tmX, tmY, tmC, tmX2, tmY2, tmC2, g, slots, pdl, s);
    if (bn == 128) {
        switch (cluster) {
            case 4: return launch_tc<128, 4, false>(tmX, tmY, tmC, tmX2, tmY2, tmC2, g, slots, pdl, s);
            case 2: return launch_tc<128, 2, false>(tmX, tmY, tmC, tmX2, tmY2, tmC2, g, slots, pdl, s);
            default: return launch_tc<128, 1, false>(tmX, tmY, tmC, tmX2, tmY2, tmC2, g, slots, pdl, s);
        }
    }
    switch (cluster) {
        case 4: return launch_tc<256, 4, false>(tmX, tmY, tmC, tmX2, tmY2, tmC2, g, slots, pdl, s);
        case 2: return launch_tc<256, 2, false>(tmX, tmY, tmC, tmX2, tmY2, tmC2, g, slots, pdl, s);
        default: return launch_tc<256, 1, false>(tmX, tmY, tmC, tmX2, tmY2, tmC2, g, slots, pdl, s);
    }
}

cudaError_t tc_launch_gemm_simt(const uint8_t* X, const uint8_t* Y, int ldk, const tc_gemm_args& g,
                                int num_sms, cudaStream_t s) {
    int grid = 2 * num_sms < g.n_units ? 2 * num_sms : g.n_units;
    if (grid < 1) grid = 1;
    k_gemm_simt<<<grid, 256, 0, s>>>(X, Y, ldk, g);
    return cudaGetLastError();
}
