// FP64 product on the BF16 tensor cores: D = alpha X Y^T + beta C + gamma I_blocks for FP64
// X (M x K) and Y (N x K), by the error-free slicing of Ozaki et al. in the integer
// accumulation form of Mukunoki, Ozaki, Ogita and Imamura ("DGEMM using Tensor Cores, and Its
// Accurate and Reproducible Versions", ISC 2020). The CUDA-core DFMA rate of this part is
// about 1.2 TFLOP/s; this engine replaces it for the FP64 precision.
//
// Slicing (k_oz64_slice). Row i of an operand gets the power of two 2^e_i just above its
// largest magnitude, and x_ij becomes the 55-bit integer T = round(x_ij 2^(55 - e_i)), cut by
// round-to-nearest into ND = 7 signed digits of at most 8 bits,
//   T = sum_p s_p 2^(8 (6 - p)),   |s_p| <= 128,   p = 0 .. 6,
// so x_ij = 2^e_i sum_p s_p 2^(-7 - 8 p) to within 2^(e_i - 56). Every digit is exact in BF16.
//
// Product. The digit pairs (p, q) with p + q = g share the weight 2^(e_i + f_j - 14 - 8 g);
// the 28 pairs with g <= 6 are formed (the dropped ones weigh 2^-56 of the leading term and
// less), one TMEM accumulator per group. A digit product is at most 2^14 and group g has
// g + 1 pairs, so over a chunk of 128 k the sums of the groups g <= 3 are integers below 2^23,
// exact in the FP32 accumulator; they restart every chunk and the epilogue adds them in 32-bit
// integers (K <= 16384 keeps those below 2^31). The groups g = 4, 5, 6 weigh 2^-32 and less
// of the leading one and accumulate over the whole K in TMEM; the truncating FP32 accumulation
// leaves them an error near 2^-47 of the leading term at K = 8192. The epilogue forms
//   2^(e_i + f_j - 38) [G_0 2^24 + G_1 2^16 + G_2 2^8 + G_3 + g_4 2^-8 + g_5 2^-16 + g_6 2^-24]
// from the 64-bit integer part and the FP32 tail in FP64, then the epilogue of the other
// engines (alpha, beta C, gamma on the diagonal blocks, transposed placement, fused dot).
//
// Kernel (k_gemm_oz64): a cluster of two CTAs per 256 x 64 output tile
// (tcgen05.mma.cta_group::2.kind::f16, M = 256, N = 64: seven 64-column accumulators fit the
// 512 TMEM columns), persistent over the tiles. K runs in blocks of 32 BF16 (64-byte rows,
// 64-byte swizzle) so that three stages of the 14 digit tiles (70 KB) fit in shared memory.
// Warp 0 issues the TMA copies of both CTAs (completing on CTA 0's full barrier), warp 1 of
// CTA 0 the MMAs (per k-block: the whole-K groups' 36, then the exact groups' 20, waiting for
// the previous chunk's drain only before the latter), warps 2..9 drain the accumulators: warp
// w reads TMEM lanes 32 (w % 4), columns 32 ((w - 2) / 4) ... of each group.
//
// Every mbarrier wait is bounded by %globaltimer; on timeout the error is recorded and both
// CTAs leave through the cluster barrier after freeing TMEM, as in the other tcgen05 kernels.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdlib>
#include <cstring>
#include <string>

#include "epilogue.cuh"
#include "internal.cuh"
#include "tc_ptx.cuh"

namespace cdmpt {

namespace {

using namespace tc;

constexpr int Z_ND = 7;            // digits per operand
constexpr int Z_NG = 7;            // groups g = p + q = 0 .. 6
constexpr int Z_NX = 4;            // exact groups (restarted every chunk)
constexpr int Z_NP = 28;           // digit pairs with p + q <= 6
constexpr int Z_NPX = 10;          // pairs of the exact groups
constexpr int Z_KB = 32;           // BF16 elements per 64-byte row
constexpr int Z_KCB = 4;           // k-blocks per exact chunk (K = 128)
constexpr int Z_STAGES = 3;
constexpr int Z_BN = 64;           // tile columns (N of the MMA)
constexpr int Z_CW = Z_BN / 2;     // columns per epilogue warp
constexpr int Z_THREADS = 320;     // producer, MMA, eight epilogue warps
constexpr int Z_A_BYTES = BM * Z_KB * 2;            // one digit, 128 rows: 8 KB
constexpr int Z_B_BYTES = (Z_BN / 2) * Z_KB * 2;    // one digit, 32 rows: 2 KB
constexpr int Z_STAGE_BYTES = Z_ND * (Z_A_BYTES + Z_B_BYTES);
constexpr int Z_SMEM = Z_STAGES * Z_STAGE_BYTES + 256 + 1024;
constexpr uint32_t Z_TMEM_COLS = 512;
static_assert(Z_NG * Z_BN <= 512, "TMEM");
static_assert(Z_SMEM <= 227 * 1024, "shared memory");
static_assert(Z_A_BYTES % 512 == 0 && Z_B_BYTES % 512 == 0, "64-byte swizzle atoms");

struct Oz64Maps {
    CUtensorMap x[Z_ND];
    CUtensorMap y[Z_ND];
};

// Digit pair i, ordered by group g = p + q and then p; group g holds pairs g (g + 1) / 2 ..
__host__ __device__ constexpr int zpair_p(int i) {
    int g = 0;
    while ((g + 1) * (g + 2) / 2 <= i) ++g;
    return i - g * (g + 1) / 2;
}
__host__ __device__ constexpr int zpair_g(int i) {
    int g = 0;
    while ((g + 1) * (g + 2) / 2 <= i) ++g;
    return g;
}
__host__ __device__ constexpr int zpair_q(int i) { return zpair_g(i) - zpair_p(i); }
__host__ __device__ constexpr int zgroup_first(int g) { return g * (g + 1) / 2; }

__device__ __forceinline__ uint32_t mapa_u32(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}

__device__ __forceinline__ uint32_t ld_cluster_u32(uint32_t caddr) {
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(caddr) : "memory");
    return v;
}

// Arrival on the peer's barrier (plain .release.cta form: it orders tcgen05 loads, completed
// by tcgen05.wait::ld and fenced before the thread sync).
__device__ __forceinline__ void arrive_remote(uint32_t caddr) {
    asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(caddr) : "memory");
}

__device__ __forceinline__ bool try_wait_cl(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool wait_cl(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                        int* err, int code) {
    if (try_wait_cl(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (true) {
        if (try_wait_cl(bar, parity)) return true;
        if (*abort_flag) return false;
        if (globaltimer() - t0 > kWaitNs) {
            *abort_flag = 1;
            if (err) atomicCAS(err, 0, code);
            return false;
        }
    }
}

__device__ __forceinline__ void tma_pair(void* dst, const CUtensorMap* map, int x, int y,
                                         uint32_t bar_c) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(bar_c)
        : "memory");
}

__device__ __forceinline__ void tmem_alloc2(uint32_t* holder, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(holder)),
                 "r"(cols)
                 : "memory");
}

__device__ __forceinline__ void tmem_dealloc2(uint32_t taddr, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols)
                 : "memory");
}

__device__ __forceinline__ void mma_bf16_2(uint32_t tmem_d, uint64_t a, uint64_t b,
                                           uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// kind::f16, D = F32 (bits 4-5 = 1), A = B = BF16 (bits 7-9, 10-12 = 1), K-major,
// N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__device__ __forceinline__ constexpr uint32_t idesc_oz64() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(Z_BN >> 3) << 17) |
           ((uint32_t)((2 * BM) >> 4) << 24);
}

// Shared-memory matrix descriptor of a K-major tile with 64-byte swizzle: rows of 64 bytes,
// 8-row core groups 512 bytes apart (stride byte offset), descriptor version 1 at bits 46-47,
// swizzle mode 4 (64 B) at bits 61-63.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}

__device__ __forceinline__ void commit_both(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
        " [%0], %1;" ::"r"(smem_u32(bar)),
        "h"((uint16_t)0x3)
        : "memory");
}

__device__ __forceinline__ void commit_local2(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void ld8(uint32_t ta, uint32_t (&a)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]),
                   "=r"(a[6]), "=r"(a[7])
                 : "r"(ta));
}
__device__ __forceinline__ void tmem_ld_wait() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void st8(uint32_t ta, const int* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(ta),
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]),
                 "r"(v[7])
                 : "memory");
}

__global__ void __launch_bounds__(Z_THREADS, 1)
    k_gemm_oz64(const __grid_constant__ Oz64Maps maps, const __grid_constant__ EpiParams<double> p,
                const int* __restrict__ ex_, const int* __restrict__ ey_, int K, int num_mt,
                int total_tiles, const double* skip, int* err) {
    if (skip != nullptr && *skip != 0.0) return;   // both CTAs of a pair read the same flag
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + Z_STAGES * Z_STAGE_BYTES);   // CTA 0
    uint64_t* empty = full + Z_STAGES;                                 // both CTAs
    uint64_t* tfull = empty + Z_STAGES;     // exact groups of a chunk ready (both CTAs)
    uint64_t* tempty = tfull + 1;           // exact groups drained (CTA 0, 16 warps)
    uint64_t* tfin = tempty + 1;            // whole-K groups of a tile ready (both CTAs)
    uint64_t* tfin_empty = tfin + 1;        // whole-K groups drained (CTA 0, 16 warps)
    uint64_t* drain = tfin_empty + 1;
    uint32_t* tmem_holder = (uint32_t*)(drain + 1);
    volatile int* abort_flag = (volatile int*)(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const int cid = (int)(blockIdx.x >> 1), ncl = (int)(gridDim.x >> 1);
    const int num_k = (K + Z_KB - 1) / Z_KB;
    auto stage_a = [&](int s, int d) { return smem + s * Z_STAGE_BYTES + d * Z_A_BYTES; };
    auto stage_b = [&](int s, int d) {
        return smem + s * Z_STAGE_BYTES + Z_ND * Z_A_BYTES + d * Z_B_BYTES;
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < Z_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(tfull, 1);
        mbar_init(tempty, 16);
        mbar_init(tfin, 1);
        mbar_init(tfin_empty, 16);
        mbar_init(drain, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 1) tmem_alloc2(tmem_holder, Z_TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    cluster_sync();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_holder;
    const bool bad = ld_cluster_u32(mapa_u32(smem_u32(tmem_holder), rank ^ 1u)) != tmem_base;
    if (bad && threadIdx.x == 0) atomicCAS(err, 0, DEV_TMEM_MISMATCH);

    if (bad) {
        // fall through to the final barrier
    } else if (warp == 0) {
        // ------------------------------------------------ TMA producer (both CTAs)
        if (lane == 0) {
            for (int d = 0; d < Z_ND; ++d) {
                prefetch_map(&maps.x[d]);
                prefetch_map(&maps.y[d]);
            }
            const uint32_t full0 = mapa_u32(smem_u32(full), 0);
            uint32_t it = 0;
            bool ok = true;
            for (int t = cid; t < total_tiles && ok; t += ncl) {
                const int mt = t % num_mt, nt = t / num_mt;
                const int m0 = mt * (2 * BM) + (int)rank * BM;
                const int y0 = nt * Z_BN + (int)rank * (Z_BN / 2);
                for (int kb = 0; kb < num_k; ++kb, ++it) {
                    const int s = it % Z_STAGES;
                    const uint32_t ph = (it / Z_STAGES) & 1;
                    if (!wait_cl(&empty[s], ph ^ 1, abort_flag, err, DEV_TIMEOUT_EMPTY)) {
                        ok = false;
                        break;
                    }
                    if (rank == 0) mbar_expect_tx(&full[s], 2 * Z_STAGE_BYTES);
                    const uint32_t fb = full0 + (uint32_t)s * 8u;
#pragma unroll
                    for (int d = 0; d < Z_ND; ++d) {
                        tma_pair(stage_a(s, d), &maps.x[d], kb * Z_KB, m0, fb);
                        tma_pair(stage_b(s, d), &maps.y[d], kb * Z_KB, y0, fb);
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer (CTA 0)
        if (lane == 0 && rank == 0) {
            constexpr uint32_t idesc = idesc_oz64();
            uint32_t it = 0, gc = 0, tc = 0;
            bool ok = true, issued = false;
            for (int t = cid; t < total_tiles && ok; t += ncl, ++tc) {
                // the whole-K groups restart with the tile: the previous tile's must be drained
                if (!wait_cl(tfin_empty, (tc & 1) ^ 1, abort_flag, err, DEV_TIMEOUT_ACCUM)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int kb = 0; kb < num_k && ok; ++kb, ++it) {
                    const int s = it % Z_STAGES;
                    const uint32_t ph = (it / Z_STAGES) & 1;
                    if (!wait_cl(&full[s], ph, abort_flag, err, DEV_TIMEOUT_FULL)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const bool chunk_first = (kb % Z_KCB) == 0;
                    // whole-K groups first (they never wait for a drain)
#pragma unroll
                    for (int kk = 0; kk < Z_KB / 16; ++kk) {
#pragma unroll
                        for (int q = Z_NPX; q < Z_NP; ++q) {
                            const int g = zpair_g(q);
                            const bool first = kb == 0 && kk == 0 && q == zgroup_first(g);
                            const uint64_t a = sw64_desc(smem_u32(stage_a(s, zpair_p(q))) + kk * 32);
                            const uint64_t b = sw64_desc(smem_u32(stage_b(s, zpair_q(q))) + kk * 32);
                            mma_bf16_2(tmem_base + (uint32_t)(g * Z_BN), a, b, idesc,
                                       first ? 0u : 1u);
                        }
                    }
                    if (chunk_first) {
                        // the exact groups restart: the previous chunk's must be drained
                        if (!wait_cl(tempty, (gc & 1) ^ 1, abort_flag, err, DEV_TIMEOUT_ACCUM)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                    }
#pragma unroll
                    for (int kk = 0; kk < Z_KB / 16; ++kk) {
#pragma unroll
                        for (int q = 0; q < Z_NPX; ++q) {
                            const int g = zpair_g(q);
                            const bool first = chunk_first && kk == 0 && q == zgroup_first(g);
                            const uint64_t a = sw64_desc(smem_u32(stage_a(s, zpair_p(q))) + kk * 32);
                            const uint64_t b = sw64_desc(smem_u32(stage_b(s, zpair_q(q))) + kk * 32);
                            mma_bf16_2(tmem_base + (uint32_t)(g * Z_BN), a, b, idesc,
                                       first ? 0u : 1u);
                        }
                    }
                    issued = true;
                    commit_both(&empty[s]);
                    if ((kb % Z_KCB) == Z_KCB - 1 || kb == num_k - 1) {
                        commit_both(tfull);
                        ++gc;
                    }
                }
                if (!ok) break;
                commit_both(tfin);
            }
            if (!ok && issued) {
                commit_local2(drain);
                mbar_drain(drain, 0);
            }
        }
    } else {
        // ------------------------------------------------ epilogue (both CTAs)
        const int q = warp & 3;                 // TMEM lane quarter
        const int h = (warp - 2) >> 2;          // column half
        const uint32_t lane_base =
            tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(Z_CW * h);
        const uint32_t tempty0 = mapa_u32(smem_u32(tempty), 0);
        const uint32_t tfin_empty0 = mapa_u32(smem_u32(tfin_empty), 0);
        const int nch = (num_k + Z_KCB - 1) / Z_KCB;
        uint32_t gc = 0, tc = 0;
        double dsum = 0.0;
        for (int t = cid; t < total_tiles; t += ncl, ++tc) {
            const int mt = t % num_mt, nt = t / num_mt;
            const int m = mt * (2 * BM) + (int)rank * BM + 32 * q + lane;
            const int n0 = nt * Z_BN + Z_CW * h;
            int G[Z_NX][Z_CW];
#pragma unroll
            for (int g = 0; g < Z_NX; ++g)
#pragma unroll
                for (int j = 0; j < Z_CW; ++j) G[g][j] = 0;
            bool ok = true;
            for (int c = 0; c < nch; ++c, ++gc) {
                int w = 1;
                if (lane == 0) w = wait_cl(tfull, gc & 1, abort_flag, err, DEV_TIMEOUT_ACCUM);
                w = __shfl_sync(0xffffffffu, w, 0);
                if (!w) {
                    ok = false;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int c0 = 0; c0 < Z_CW; c0 += 8) {
                    uint32_t r[Z_NX][8];
#pragma unroll
                    for (int g = 0; g < Z_NX; ++g) ld8(lane_base + (uint32_t)(g * Z_BN + c0), r[g]);
                    tmem_ld_wait();
#pragma unroll
                    for (int g = 0; g < Z_NX; ++g)
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            G[g][c0 + j] += __float2int_rn(__uint_as_float(r[g][j]));
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) arrive_remote(tempty0);
            }
            if (!ok) break;
            int w = 1;
            if (lane == 0) w = wait_cl(tfin, tc & 1, abort_flag, err, DEV_TIMEOUT_ACCUM);
            w = __shfl_sync(0xffffffffu, w, 0);
            if (!w) break;
            tc_fence_after();
            // park the exact sums in this warp's drained exact-group columns (the issuer leaves
            // them alone until this tile's final arrival below), then combine 8 columns at a time
#pragma unroll
            for (int g = 0; g < Z_NX; ++g)
#pragma unroll
                for (int c0 = 0; c0 < Z_CW; c0 += 8)
                    st8(lane_base + (uint32_t)(g * Z_BN + c0), &G[g][c0]);
            tmem_wait_st();
            const bool row_ok = m < p.M;
            const int ex = row_ok ? ex_[m] : 0;
#pragma unroll 1
            for (int c0 = 0; c0 < Z_CW; c0 += 8) {
                uint32_t r[Z_NG][8];
#pragma unroll
                for (int g = 0; g < Z_NG; ++g) ld8(lane_base + (uint32_t)(g * Z_BN + c0), r[g]);
                tmem_ld_wait();
                if (row_ok) {
                    // the chunk's loads first (column exponents, C and E), then the arithmetic
                    // of epi_apply and the stores: one memory latency per chunk, not per element
                    int eyv[8];
                    double cv[8], ev[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int n = n0 + c0 + j;
                        const bool ok = n < p.N;
                        size_t rr, cc;
                        epi_position(p, m, n, rr, cc);
                        eyv[j] = ok ? ey_[n] : 0;
                        cv[j] = (ok && p.beta != 0.0) ? p.C[rr * p.ldc + cc] : 0.0;
                        ev[j] = (ok && p.dot && p.E) ? p.E[rr * p.lde + cc] : 0.0;
                    }
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int n = n0 + c0 + j;
                        if (n < p.N) {
                            long long I = 0;
#pragma unroll
                            for (int g = 0; g < Z_NX; ++g) I = I * 256 + (long long)(int)r[g][j];
                            const double tail =
                                (double)__uint_as_float(r[Z_NX][j]) * (1.0 / 256.0) +
                                (double)__uint_as_float(r[Z_NX + 1][j]) * (1.0 / 65536.0) +
                                (double)__uint_as_float(r[Z_NX + 2][j]) * (1.0 / 16777216.0);
                            const double acc =
                                ldexp((double)I + tail, ex + eyv[j] - 14 - 8 * (Z_NX - 1));
                            size_t rr, cc;
                            epi_position(p, m, n, rr, cc);
                            double v = p.alpha * acc;
                            if (p.beta != 0.0) v = fma(p.beta, cv[j], v);
                            if (p.gamma != 0.0 && (m % p.diag_block) == n) v += p.gamma;
                            p.D[rr * p.ldd + cc] = v;
                            if (p.dot) dsum += v * (p.E ? ev[j] : v);
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) arrive_remote(tfin_empty0);
        }
        if (p.dot) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xffffffffu, dsum, o);
            if (lane == 0 && dsum != 0.0) atomicAdd(p.dot, dsum);
        }
    }

    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) {
        const unsigned long long t0 = globaltimer();
        while (globaltimer() - t0 < 100000ull) {
        }
    }
    __syncthreads();
    cluster_sync();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc2(tmem_base, Z_TMEM_COLS);
    }
}

// One warp per row: the row's power of two and the seven BF16 digits of every element
// (zeros in the padding columns cols .. ld - 1).
__global__ void k_oz64_slice(const double* __restrict__ x, int rows, int cols, int ld,
                             Oz64Operand out, const double* skip) {
    if (skip != nullptr && *skip != 0.0) return;
    constexpr int BITS = 8 * Z_ND - 1;   // 55
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    for (int r = blockIdx.x * wpb + (threadIdx.x >> 5); r < rows; r += gridDim.x * wpb) {
        const double* xr = x + (size_t)r * ld;
        double mx = 0.0;
        for (int j = lane; j < cols; j += 32) mx = fmax(mx, fabs(xr[j]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        int e = 0;
        if (mx > 0.0) (void)frexp(mx, &e);   // mx = m 2^e, m in [0.5, 1): |x| 2^-e < 1
        if (lane == 0) out.e[r] = e;
        const size_t off = (size_t)r * out.ld;
        for (int j = lane; j < out.ld; j += 32) {
            int dg[Z_ND];
#pragma unroll
            for (int d = 0; d < Z_ND; ++d) dg[d] = 0;
            if (j < cols && mx > 0.0) {
                // T = round(x 2^(55 - e)), |T| <= 2^55; digits by round-to-nearest
                long long T = __double2ll_rn(ldexp(xr[j], BITS - e));
#pragma unroll
                for (int d = 0; d < Z_ND - 1; ++d) {
                    const int sh = 8 * (Z_ND - 1 - d);
                    const long long a = (T + (1ll << (sh - 1))) >> sh;
                    dg[d] = (int)a;
                    T -= a << sh;
                }
                dg[Z_ND - 1] = (int)T;
            }
#pragma unroll
            for (int d = 0; d < Z_ND; ++d)
                ((__nv_bfloat16*)out.s[d])[off + j] = __float2bfloat16_rn((float)dg[d]);
        }
    }
}

bool make_map_oz64(CUtensorMap* map, const void* base, int rows, int cols, int ld, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)Z_KB, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box,
                    estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

cdmpt_status oz64_slice(const double* x, int rows, int cols, int ld, const Oz64Operand& out,
                        const double* skip, cudaStream_t s) {
    if (rows <= 0) return CDMPT_OK;
    if (cols > 16384 || cols > ld || cols > out.ld || (out.ld & 7) || !x) {
        set_error("FP64 Ozaki slicing: cols <= 16384, cols <= ld, digit ld a multiple of 8");
        return CDMPT_ERR_ARG;
    }
    for (int d = 0; d < Z_ND; ++d)
        if (!out.s[d] || !out.e) {
            set_error("FP64 Ozaki slicing: digit arrays missing");
            return CDMPT_ERR_ARG;
        }
    const int wpb = 8;
    int grid = (rows + wpb - 1) / wpb;
    if (grid > 152 * 16) grid = 152 * 16;
    k_oz64_slice<<<grid, 32 * wpb, 0, s>>>(x, rows, cols, ld, out, skip);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("FP64 Ozaki slicing launch: ") + cudaGetErrorString(e));
        return CDMPT_ERR_CUDA;
    }
    return CDMPT_OK;
}

cdmpt_status gemm_oz64(int M, int N, int K, const Oz64Operand& X, const Oz64Operand& Y,
                       double* D, int ldd, const Epilogue<double>& ep, const double* skip,
                       cudaStream_t s) {
    if (M <= 0 || N <= 0) return CDMPT_OK;
    if (!tc_supported()) {
        set_error("tcgen05 GEMM needs an sm_103 device");
        return CDMPT_ERR_UNSUPPORTED;
    }
    if (K < 1 || K > 16384 || (X.ld & 7) || (Y.ld & 7) || !D || ldd < N) {
        set_error("FP64 Ozaki GEMM: 1 <= K <= 16384, digit ld a multiple of 8, D given");
        return CDMPT_ERR_ARG;
    }
    auto kern = k_gemm_oz64;
    static int max_clusters = 0;
    if (max_clusters == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             Z_SMEM);
        cudaLaunchConfig_t q = {};
        q.gridDim = dim3(2 * (sm_count() / 2));
        q.blockDim = dim3(Z_THREADS);
        q.dynamicSmemBytes = Z_SMEM;
        cudaLaunchAttribute a;
        a.id = cudaLaunchAttributeClusterDimension;
        a.val.clusterDim.x = 2;
        a.val.clusterDim.y = 1;
        a.val.clusterDim.z = 1;
        q.attrs = &a;
        q.numAttrs = 1;
        int n = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(&n, kern, &q);
        if (e != cudaSuccess || n < 1) {
            cudaGetLastError();
            set_error("FP64 Ozaki GEMM: no resident cluster of two");
            return CDMPT_ERR_UNSUPPORTED;
        }
        max_clusters = n;
    }
    Oz64Maps maps;
    for (int d = 0; d < Z_ND; ++d) {
        if (!X.s[d] || !Y.s[d] || !make_map_oz64(&maps.x[d], X.s[d], M, K, X.ld, BM) ||
            !make_map_oz64(&maps.y[d], Y.s[d], N, K, Y.ld, Z_BN / 2)) {
            set_error("FP64 Ozaki GEMM: cuTensorMapEncodeTiled failed (digit arrays aligned?)");
            return CDMPT_ERR_ARG;
        }
    }
    EpiParams<double> p;
    p.alpha = ep.alpha;
    p.beta = ep.beta;
    p.gamma = ep.gamma;
    p.C = ep.C;
    p.ldc = ep.ldc;
    p.D = D;
    p.ldd = ldd;
    p.M = M;
    p.N = N;
    p.diag_block = ep.diag_block > 0 ? ep.diag_block : M;
    p.trans_block = ep.trans_block > 0 ? ep.trans_block : 0;
    p.dot = ep.dot;
    p.E = ep.E;
    p.lde = ep.lde;
    p.Dhi = nullptr;
    p.Dlo = nullptr;
    p.sym = 0;   // full tiles: every element computed
    const int num_mt = (M + 2 * BM - 1) / (2 * BM);
    const int tiles = num_mt * ((N + Z_BN - 1) / Z_BN);
    const int clusters = tiles < max_clusters ? tiles : max_clusters;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * clusters);
    cfg.blockDim = dim3(Z_THREADS);
    cfg.dynamicSmemBytes = Z_SMEM;
    cfg.stream = s;
    cudaLaunchAttribute a;
    a.id = cudaLaunchAttributeClusterDimension;
    a.val.clusterDim.x = 2;
    a.val.clusterDim.y = 1;
    a.val.clusterDim.z = 1;
    cfg.attrs = &a;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, maps, p, (const int*)X.e, (const int*)Y.e, K,
                                       num_mt, tiles, skip, device_error_word());
    count_launch();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("FP64 Ozaki GEMM launch: ") + cudaGetErrorString(e));
        return CDMPT_ERR_CUDA;
    }
    return CDMPT_OK;
}

}  // namespace cdmpt
