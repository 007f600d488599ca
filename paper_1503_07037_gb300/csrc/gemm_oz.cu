// Product of pair-stored FP32 matrices to FP64-class accuracy, X Y^T with X = xh + xl and
// Y = yh + yl, on the BF16 tensor cores: the error-free slicing of Ozaki et al. in the
// tensor-core form of Mukunoki, Ozaki, Ogita and Imamura ("DGEMM using Tensor Cores, and
// Its Accurate and Reproducible Versions", ISC 2020), written for tcgen05.
//
// Slicing (k_oz_slice). Row i of an operand gets the power of two 2^e_i just above its
// largest magnitude, and x_ij 2^-e_i in (-1, 1) becomes the (8 ND - 1)-bit fixed-point
// integer T = round(x_ij 2^(8 ND - 1 - e_i)), cut into ND signed digits by round-to-nearest,
//   T = sum_p s_p 2^(8 (ND - p)),   |s_p| <= 128,   p = 1 .. ND,
// so x_ij = 2^e_i sum_p s_p 2^(-7 - 8 (p - 1)) to within 2^(e_i - 8 ND). Every digit is an
// integer of at most 8 bits and is exact in BF16. ND = 5 (39 bits) is the default: the error
// is relative to the row's largest element, and in the late recursion steps the rows of Z_k
// decay away from O(1) entries near the diagonal, so four digits (31 bits) left the step
// residuals near 1e-7 of ||Z|| at N = 1728.
//
// Product. With the digits s_p of X and t_q of Y, X Y^T = sum_{p,q} 2^(e_i + f_j) w_p w_q S_p T_q^T.
// The pairs with p + q = g share the weight 2^(e_i + f_j - 14 - 8 (g - 2)), so one TMEM
// accumulator serves each group g = 2 .. ND + 1 (the ND (ND + 1) / 2 pairs with p + q <= ND + 1;
// the dropped ones weigh 2^(-8 ND) and less). A digit product is at most 2^14, so the sums of
// the groups g <= ND - 1 (at most ND - 2 pairs) over a chunk of 256 k are integers below
// 3 2^22 < 2^24, exact in the FP32 accumulator. They restart every chunk, and the epilogue
// converts each chunk's sums to int32 and adds them exactly (no overflow for K <= 32768). The
// last two groups weigh 2^(-8 (ND - 2)) and less of the leading term; they accumulate over the
// whole K in TMEM. The result,
//   2^(e_i + f_j - 14) [sum_{g exact} 2^(-8 (g - 2)) G_g + sum_{g last two} 2^(-8 (g - 2)) g_g],
// is formed as an exact 64-bit integer plus a float tail, i.e. a pair, and the epilogue
// combines it with pair-stored C terms in double-float arithmetic.
//
// Kernel (k_gemm_oz): a cluster of two CTAs (tcgen05.mma.cta_group::2, M = 256, N = BN: 128 for
// four digits, 96 for five, so that the ND accumulators fit the 512 TMEM columns) per 256 x BN
// output tile, persistent over tiles. Per k-block of 64 each CTA stages its 128 rows of the
// X digits and BN/2 rows of the Y digits (128-byte swizzle, two stages). Warp 0 issues the TMA
// copies of both CTAs (completing on CTA 0's full barrier), warp 1 of CTA 0 the MMAs of a
// k-block (four k-steps of K = 16 times the digit pairs), warps 2..9 drain the accumulators:
// warp w reads TMEM lanes 32 (w % 4) and columns (BN / 2) ((w - 2) / 4) ... At a chunk boundary
// the issuer first issues the whole-K groups' MMAs of the next k-block, and waits for the drain
// of the exact groups only before their first MMA of the new chunk.
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

#include "dd.cuh"
#include "internal.cuh"
#include "tc_ptx.cuh"

namespace cdmpt {

namespace {

using namespace tc;

constexpr int OZ_KB = 64;         // BF16 elements per 128-byte row
constexpr int OZ_KCB = 4;         // k-blocks per exact chunk (K = 256)
constexpr int OZ_STAGES = 2;
constexpr int OZ_THREADS = 320;   // producer, MMA, eight epilogue warps
constexpr int OZ_A_BYTES = BM * OZ_KB * 2;   // one digit, 128 rows: 16 KB

template <int ND>
struct OzCfg {
    static constexpr int BN = ND == 4 ? 128 : 96;          // tile columns (N of the MMA)
    static constexpr int CW = BN / 2;                      // columns per epilogue warp
    static constexpr int NG = ND;                          // accumulator groups g = 2 .. ND + 1
    static constexpr int NX = ND - 2;                      // exact groups (restart per chunk)
    static constexpr int NP = ND * (ND + 1) / 2;           // digit pairs
    static constexpr int NPX = NX * (NX + 1) / 2;          // pairs of the exact groups
    static constexpr int B_BYTES = (BN / 2) * OZ_KB * 2;   // one digit, BN/2 rows
    static constexpr int STAGE_BYTES = ND * (OZ_A_BYTES + B_BYTES);
    static constexpr int SMEM = OZ_STAGES * STAGE_BYTES + 256 + 1024;
    static constexpr uint32_t TMEM_COLS = 512;
    static_assert(NG * BN <= 512, "TMEM");
    static_assert(SMEM <= 227 * 1024, "shared memory");
    static_assert(B_BYTES % 1024 == 0, "1024-byte tiles");
    static_assert(CW % 8 == 0, "epilogue columns");
};

template <int ND>
struct OzMaps {
    CUtensorMap x[ND];
    CUtensorMap y[ND];
};

// Digit pair i (ordered by group g = p + q, then p), 0-based digits; and its group index
// g - 2. Group gi holds pairs gi (gi + 1) / 2 .. (gi + 1) (gi + 2) / 2 - 1.
template <int ND>
__host__ __device__ constexpr int pair_digit(int i, bool first) {
    int idx = 0;
    for (int g = 2; g <= ND + 1; ++g)
        for (int p = 1; p < g; ++p) {
            const int q = g - p;
            if (p > ND || q > ND) continue;
            if (idx == i) return first ? p - 1 : q - 1;
            ++idx;
        }
    return 0;
}
__host__ __device__ constexpr int pair_group(int i) {
    int g = 0;
    while ((g + 1) * (g + 2) / 2 <= i) ++g;
    return g;
}
__host__ __device__ constexpr int group_first(int gi) { return gi * (gi + 1) / 2; }

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

// Arrival on the peer's barrier with the plain (.release.cta) form: the drained-accumulator
// signals order tcgen05 loads (completed by tcgen05.wait::ld and fenced before the thread
// sync); a cluster-scope release would also wait for the warp's earlier global stores.
__device__ __forceinline__ void mbar_arrive_remote(uint32_t caddr) {
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
template <int N>
__device__ __forceinline__ constexpr uint32_t idesc_oz() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)((2 * BM) >> 4) << 24);
}

// commit to the mbarrier at the same offset in both CTAs of the pair
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

// 8 consecutive columns of this warp's 32 TMEM lanes (issue only; tmem_ld_wait() completes)
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

// x 2^sh by two exact power-of-two factors (|sh| <= 252 stays in range; the result may
// round only when it falls below the normal range)
__device__ __forceinline__ float scale2(float x, int sh) {
    sh = max(-252, min(252, sh));
    const int a = sh / 2, b = sh - a;
    return __fmul_rn(__fmul_rn(x, __int_as_float((a + 127) << 23)), __int_as_float((b + 127) << 23));
}


// Output tile t of the launch: M-fastest over all tiles, or, for a symmetric result, over
// the tiles that meet the upper triangle only (column tile nt holds the row tiles mt with
// 256 mt <= the tile's last column).
__host__ __device__ __forceinline__ int oz_sym_count(int nt, int num_mt, int bn) {
    const int c = (nt * bn + bn - 1) / (2 * BM) + 1;
    return c < num_mt ? c : num_mt;
}
__device__ __forceinline__ void oz_tile(int t, int num_mt, int bn, bool sym, int* mt, int* nt) {
    if (!sym) {
        *mt = t % num_mt;
        *nt = t / num_mt;
        return;
    }
    int j = 0;
    while (true) {
        const int c = oz_sym_count(j, num_mt, bn);
        if (t < c) break;
        t -= c;
        ++j;
    }
    *mt = t;
    *nt = j;
}

template <int ND>
__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_gemm_oz(const __grid_constant__ OzMaps<ND> maps, const __grid_constant__ OzEpi p, int K,
              int num_mt, int total_tiles, int* err) {
    using C = OzCfg<ND>;
    constexpr int BN = C::BN, CW = C::CW, NX = C::NX;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + OZ_STAGES * C::STAGE_BYTES);   // CTA 0
    uint64_t* empty = full + OZ_STAGES;                                 // both CTAs
    uint64_t* tfull = empty + OZ_STAGES;    // exact groups of a chunk ready (both CTAs)
    uint64_t* tempty = tfull + 1;           // exact groups drained (CTA 0, 16 warps)
    uint64_t* tfin = tempty + 1;            // whole-K groups of a tile ready (both CTAs)
    uint64_t* tfin_empty = tfin + 1;        // whole-K groups drained (CTA 0, 16 warps)
    uint64_t* drain = tfin_empty + 1;
    uint32_t* tmem_holder = (uint32_t*)(drain + 1);
    volatile int* abort_flag = (volatile int*)(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const int cid = (int)(blockIdx.x >> 1), ncl = (int)(gridDim.x >> 1);
    const int num_k = (K + OZ_KB - 1) / OZ_KB;
    auto stage_a = [&](int s, int d) { return smem + s * C::STAGE_BYTES + d * OZ_A_BYTES; };
    auto stage_b = [&](int s, int d) {
        return smem + s * C::STAGE_BYTES + ND * OZ_A_BYTES + d * C::B_BYTES;
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < OZ_STAGES; ++s) {
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
    if (warp == 1) tmem_alloc2(tmem_holder, C::TMEM_COLS);
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
            for (int d = 0; d < ND; ++d) {
                prefetch_map(&maps.x[d]);
                prefetch_map(&maps.y[d]);
            }
            const uint32_t full0 = mapa_u32(smem_u32(full), 0);
            uint32_t it = 0;
            bool ok = true;
            for (int t = cid; t < total_tiles && ok; t += ncl) {
                int mt = 0, nt = 0;
                oz_tile(t, num_mt, BN, p.sym != 0, &mt, &nt);
                const int m0 = mt * (2 * BM) + (int)rank * BM;
                const int y0 = nt * BN + (int)rank * (BN / 2);
                for (int kb = 0; kb < num_k; ++kb, ++it) {
                    const int s = it % OZ_STAGES;
                    const uint32_t ph = (it / OZ_STAGES) & 1;
                    if (!wait_cl(&empty[s], ph ^ 1, abort_flag, err, DEV_TIMEOUT_EMPTY)) {
                        ok = false;
                        break;
                    }
                    if (rank == 0) mbar_expect_tx(&full[s], 2 * C::STAGE_BYTES);
                    const uint32_t fb = full0 + (uint32_t)s * 8u;
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        tma_pair(stage_a(s, d), &maps.x[d], kb * OZ_KB, m0, fb);
                        tma_pair(stage_b(s, d), &maps.y[d], kb * OZ_KB, y0, fb);
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer (CTA 0)
        if (lane == 0 && rank == 0) {
            constexpr uint32_t idesc = idesc_oz<BN>();
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
                    const int s = it % OZ_STAGES;
                    const uint32_t ph = (it / OZ_STAGES) & 1;
                    if (!wait_cl(&full[s], ph, abort_flag, err, DEV_TIMEOUT_FULL)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const bool chunk_first = (kb % OZ_KCB) == 0;
                    // whole-K groups first (they never wait for a drain)
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
                        for (int q = C::NPX; q < C::NP; ++q) {
                            const int g = pair_group(q);
                            const bool first = kb == 0 && kk == 0 && q == group_first(g);
                            const uint64_t a =
                                sw128_desc(smem_u32(stage_a(s, pair_digit<ND>(q, true))) + kk * 32);
                            const uint64_t b =
                                sw128_desc(smem_u32(stage_b(s, pair_digit<ND>(q, false))) + kk * 32);
                            mma_bf16_2(tmem_base + (uint32_t)(g * BN), a, b, idesc, first ? 0u : 1u);
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
                    for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
                        for (int q = 0; q < C::NPX; ++q) {
                            const int g = pair_group(q);
                            const bool first = chunk_first && kk == 0 && q == group_first(g);
                            const uint64_t a =
                                sw128_desc(smem_u32(stage_a(s, pair_digit<ND>(q, true))) + kk * 32);
                            const uint64_t b =
                                sw128_desc(smem_u32(stage_b(s, pair_digit<ND>(q, false))) + kk * 32);
                            mma_bf16_2(tmem_base + (uint32_t)(g * BN), a, b, idesc, first ? 0u : 1u);
                        }
                    }
                    issued = true;
                    commit_both(&empty[s]);
                    if ((kb % OZ_KCB) == OZ_KCB - 1 || kb == num_k - 1) {
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
        const uint32_t lane_base = tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(CW * h);
        const uint32_t tempty0 = mapa_u32(smem_u32(tempty), 0);
        const uint32_t tfin_empty0 = mapa_u32(smem_u32(tfin_empty), 0);
        const int nch = (num_k + OZ_KCB - 1) / OZ_KCB;
        uint32_t gc = 0, tc = 0;
        double dsum = 0.0;
        for (int t = cid; t < total_tiles; t += ncl, ++tc) {
            int mt = 0, nt = 0;
            oz_tile(t, num_mt, BN, p.sym != 0, &mt, &nt);
            const int m = mt * (2 * BM) + (int)rank * BM + 32 * q + lane;
            const int n0 = nt * BN + CW * h;
            int G[NX][CW];
#pragma unroll
            for (int g = 0; g < NX; ++g)
#pragma unroll
                for (int j = 0; j < CW; ++j) G[g][j] = 0;
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
                for (int c0 = 0; c0 < CW; c0 += 8) {
                    uint32_t r[NX][8];
#pragma unroll
                    for (int g = 0; g < NX; ++g) ld8(lane_base + (uint32_t)(g * BN + c0), r[g]);
                    tmem_ld_wait();
#pragma unroll
                    for (int g = 0; g < NX; ++g)
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            G[g][c0 + j] += __float2int_rn(__uint_as_float(r[g][j]));
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_remote(tempty0);
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
            for (int g = 0; g < NX; ++g)
#pragma unroll
                for (int c0 = 0; c0 < CW; c0 += 8)
                    st8(lane_base + (uint32_t)(g * BN + c0), &G[g][c0]);
            tmem_wait_st();
            const bool row_ok = m < p.M;
            const int ex = row_ok ? p.ex[m] : 0;
            // every field the loop uses, read once: the stores below may alias p's memory
            // for all the compiler knows, which would make it reload them after each store
            const int PN = p.N, ldc = p.ldc, ldd = p.ldd;
            const bool sym = p.sym != 0;
            const float alpha = p.alpha, b1 = p.b1, b2 = p.b2, gamma = p.gamma;
            const float* c1h = p.c1h;
            const float* c1l = p.c1l;
            const float* c2h = p.c2h;
            const float* c2l = p.c2l;
            const int* ey = p.ey;
            float* const Dp = p.D;
            float* const Dlp = p.Dl;
            float* const Dth = p.Dthi;
            float* const Dtl = p.Dtlo;
#pragma unroll 1
            for (int c0 = 0; c0 < CW; c0 += 8) {
                uint32_t r[ND][8];
#pragma unroll
                for (int g = 0; g < ND; ++g) ld8(lane_base + (uint32_t)(g * BN + c0), r[g]);
                tmem_ld_wait();
                if (row_ok) {
                    const size_t rowc = (size_t)m * ldc, rowd = (size_t)m * ldd;
                    // the chunk's loads first (column exponents and C terms), then its
                    // arithmetic and stores: one memory latency per chunk, not per element
                    int eyv[8];
                    float ch1[8], cl1[8], ch2[8], cl2[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int n = n0 + c0 + j;
                        const bool ok = n < PN && !(sym && n < m);
                        eyv[j] = ok ? ey[n] : 0;
                        ch1[j] = (ok && c1h) ? c1h[rowc + n] : 0.f;
                        cl1[j] = (ok && c1l) ? c1l[rowc + n] : 0.f;
                        ch2[j] = (ok && c2h) ? c2h[rowc + n] : 0.f;
                        cl2[j] = (ok && c2l) ? c2l[rowc + n] : 0.f;
                    }
                    float local = 0.f;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int n = n0 + c0 + j;
                        if (n < PN && !(sym && n < m)) {
                            // exact integer part of the exact groups, then the float tail of the
                            // whole-K groups, in units of the last exact group's weight
                            long long I = 0;
#pragma unroll
                            for (int g = 0; g < NX; ++g) I = I * 256 + (long long)(int)r[g][j];
                            float vh = (float)I;
                            float vl = (float)(I - (long long)vh);
                            vl = __fadd_rn(vl, __fadd_rn(__uint_as_float(r[NX][j]) * (1.f / 256.f),
                                                         __uint_as_float(r[NX + 1][j]) * (1.f / 65536.f)));
                            const int sh = ex + eyv[j] - 14 - 8 * (NX - 1);
                            vh = scale2(vh, sh);
                            vl = scale2(vl, sh);
                            // D = alpha X Y^T + b1 C1 + b2 C2 + gamma I in double-float
                            float dh = __fmul_rn(alpha, vh), dl = __fmul_rn(alpha, vl);
                            if (c1h) {
                                const float ch = __fmul_rn(b1, ch1[j]);
                                const float cl = c1l ? __fmul_rn(b1, cl1[j]) : 0.f;
                                dd::add(dh, dl, ch, cl, dh, dl);
                            }
                            if (c2h) {
                                const float ch = __fmul_rn(b2, ch2[j]);
                                const float cl = c2l ? __fmul_rn(b2, cl2[j]) : 0.f;
                                dd::add(dh, dl, ch, cl, dh, dl);
                            }
                            if (gamma != 0.f && n == m) dd::add1(dh, dl, gamma, dh, dl);
                            float o, ol;
                            dd::fast_two_sum(dh, dl, o, ol);
                            // symmetric result: the mirror (n, m) too (the lanes hold
                            // consecutive rows m, so these stores coalesce)
                            const bool mir = sym && n > m;
                            const size_t mirror = (size_t)n * ldd + m;
                            Dp[rowd + n] = o;
                            if (mir) Dp[mirror] = o;
                            if (Dlp) {
                                Dlp[rowd + n] = ol;
                                if (mir) Dlp[mirror] = ol;
                            }
                            if (Dth) {
                                float th, tl;
                                dd::tf32_split(o, th, tl);
                                Dth[rowd + n] = th;
                                if (mir) Dth[mirror] = th;
                                if (Dtl) {
                                    Dtl[rowd + n] = tl;
                                    if (mir) Dtl[mirror] = tl;
                                }
                            }
                            local = __fmaf_rn(mir ? 2.f * o : o, o, local);
                        }
                    }
                    dsum += (double)local;
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_remote(tfin_empty0);
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
        tmem_dealloc2(tmem_base, C::TMEM_COLS);
    }
}

// One warp per row: the row's power of two and the ND BF16 digits of every element.
template <int ND>
__global__ void k_oz_slice(const float* __restrict__ xh, const float* __restrict__ xl, int rows,
                           int cols, int ld, OzOperand out) {
    constexpr int BITS = 8 * ND - 1;
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    for (int r = blockIdx.x * wpb + (threadIdx.x >> 5); r < rows; r += gridDim.x * wpb) {
        const float* hr = xh + (size_t)r * ld;
        const float* lr = xl ? xl + (size_t)r * ld : nullptr;
        float mx = 0.f;
        for (int j = lane; j < cols; j += 32) mx = fmaxf(mx, fabsf(hr[j]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        int e = 0;
        if (mx > 0.f) (void)frexpf(mx, &e);   // mx = m 2^e, m in [0.5, 1): |x| 2^-e < 1
        if (lane == 0) out.e[r] = e;
        const size_t off = (size_t)r * ld;
        for (int j = lane; j < ld; j += 32) {
            int dg[ND];
#pragma unroll
            for (int d = 0; d < ND; ++d) dg[d] = 0;
            if (j < cols && mx > 0.f) {
                // T = round((xh + xl) 2^(BITS - e)), |T| <= 2^BITS; digits by round-to-nearest
                long long T = __float2ll_rn(scale2(hr[j], BITS - e));
                if (lr) T += __float2ll_rn(scale2(lr[j], BITS - e));
#pragma unroll
                for (int d = 0; d < ND - 1; ++d) {
                    const int sh = 8 * (ND - 1 - d);
                    const long long a = (T + (1ll << (sh - 1))) >> sh;
                    dg[d] = (int)a;
                    T -= a << sh;
                }
                dg[ND - 1] = (int)T;
            }
#pragma unroll
            for (int d = 0; d < ND; ++d)
                ((__nv_bfloat16*)out.s[d])[off + j] = __float2bfloat16_rn((float)dg[d]);
        }
    }
}

bool make_map_oz(CUtensorMap* map, const void* base, int rows, int cols, int ld, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)OZ_KB, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box,
                    estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int ND>
cdmpt_status launch_oz(int M, int N, int K, const OzOperand& X, const OzOperand& Y,
                       const OzEpi& ep, cudaStream_t s) {
    using C = OzCfg<ND>;
    auto kern = k_gemm_oz<ND>;
    static int max_clusters = 0;
    if (max_clusters == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             C::SMEM);
        cudaLaunchConfig_t q = {};
        q.gridDim = dim3(2 * (sm_count() / 2));
        q.blockDim = dim3(OZ_THREADS);
        q.dynamicSmemBytes = C::SMEM;
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
            set_error("Ozaki GEMM: no resident cluster of two");
            return CDMPT_ERR_UNSUPPORTED;
        }
        max_clusters = n;
    }
    OzMaps<ND> maps;
    for (int d = 0; d < ND; ++d) {
        if (!X.s[d] || !Y.s[d] || !make_map_oz(&maps.x[d], X.s[d], M, K, X.ld, BM) ||
            !make_map_oz(&maps.y[d], Y.s[d], N, K, Y.ld, C::BN / 2)) {
            set_error("Ozaki GEMM: cuTensorMapEncodeTiled failed (digit arrays 16-byte aligned?)");
            return CDMPT_ERR_ARG;
        }
    }
    OzEpi p = ep;
    p.M = M;
    p.N = N;
    p.ex = X.e;
    p.ey = Y.e;
    const int num_mt = (M + 2 * BM - 1) / (2 * BM);
    const int num_nt = (N + C::BN - 1) / C::BN;
    p.sym = (ep.sym && M == N && X.s[0] == Y.s[0]) ? 1 : 0;
    int tiles = 0;
    if (p.sym)
        for (int j = 0; j < num_nt; ++j) tiles += oz_sym_count(j, num_mt, C::BN);
    else
        tiles = num_mt * num_nt;
    const int clusters = tiles < max_clusters ? tiles : max_clusters;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * clusters);
    cfg.blockDim = dim3(OZ_THREADS);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = s;
    cudaLaunchAttribute a;
    a.id = cudaLaunchAttributeClusterDimension;
    a.val.clusterDim.x = 2;
    a.val.clusterDim.y = 1;
    a.val.clusterDim.z = 1;
    cfg.attrs = &a;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, maps, p, K, num_mt, tiles, device_error_word());
    count_launch();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("Ozaki GEMM launch: ") + cudaGetErrorString(e));
        return CDMPT_ERR_CUDA;
    }
    return CDMPT_OK;
}

}  // namespace

cdmpt_status oz_slice(const float* xh, const float* xl, int rows, int cols, int ld,
                      const OzOperand& out, cudaStream_t s, int nd) {
    if (rows <= 0) return CDMPT_OK;
    if ((nd != 4 && nd != 5) || cols > 32768 || cols > ld || (ld & 7)) {
        set_error("Ozaki slicing: 4 or 5 digits, cols <= 32768, cols <= ld, ld a multiple of 8");
        return CDMPT_ERR_ARG;
    }
    const int wpb = 8;
    int grid = (rows + wpb - 1) / wpb;
    if (grid > 152 * 16) grid = 152 * 16;
    if (nd == 5)
        k_oz_slice<5><<<grid, 32 * wpb, 0, s>>>(xh, xl, rows, cols, ld, out);
    else
        k_oz_slice<4><<<grid, 32 * wpb, 0, s>>>(xh, xl, rows, cols, ld, out);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("Ozaki slicing launch: ") + cudaGetErrorString(e));
        return CDMPT_ERR_CUDA;
    }
    return CDMPT_OK;
}

cdmpt_status gemm_oz(int M, int N, int K, const OzOperand& X, const OzOperand& Y,
                     const OzEpi& ep, cudaStream_t s, int nd) {
    if (M <= 0 || N <= 0) return CDMPT_OK;
    if (!tc_supported()) {
        set_error("tcgen05 GEMM needs an sm_103 device");
        return CDMPT_ERR_UNSUPPORTED;
    }
    if ((nd != 4 && nd != 5) || K < 1 || K > 32768 || (X.ld & 7) || (Y.ld & 7) || !ep.D) {
        set_error("Ozaki GEMM: 4 or 5 digits, 1 <= K <= 32768, ld a multiple of 8, D given");
        return CDMPT_ERR_ARG;
    }
    return nd == 5 ? launch_oz<5>(M, N, K, X, Y, ep, s) : launch_oz<4>(M, N, K, X, Y, ep, s);
}

}  // namespace cdmpt
