// Two-SM tcgen05 GEMM for sm_103a: the same product as k_gemm_tc,
// D = alpha X Y^T + beta C + gamma I, with each MMA spanning a pair of SMs
// (tcgen05.mma.cta_group::2, M = 256).
//
// A cluster of two CTAs owns a 256 x BN output tile. CTA r of the pair keeps
// rows 128 r .. 128 r + 127 of the X tile and rows r BN/2 .. r BN/2 + BN/2 - 1
// of the Y tile in its own shared memory. The MMA, issued by one thread of
// CTA 0, reads both halves of both operands and writes accumulator rows
// 128 r .. 128 r + 127 into CTA r's tensor memory. Each SM thus stages half of
// the Y tile instead of all of it: per flop it receives fewer bytes, so the
// same shared memory holds more k-blocks of lookahead.
//
// Roles per CTA (320 threads):
//   warp 0      TMA producer in both CTAs, each loading its own halves. The
//               copies of both CTAs complete on CTA 0's full barrier (the
//               .cta_group::2 form of the copy may signal the peer's barrier),
//               whose expected byte count covers both CTAs;
//   warp 1      collective TMEM allocation of the pair; in CTA 0, lane 0
//               issues the MMAs and commits them to the empty and
//               accumulator-full barriers of both CTAs (multicast);
//   warps 2..9  epilogue of this CTA's 128 rows, two warps per TMEM lane
//               quarter, each with half of the columns, stored in 32 x 32
//               blocks through a shared-memory transpose (tc_store.cuh); after
//               draining an accumulator each warp arrives on CTA 0's
//               accumulator-empty barrier, which counts the 16 warps of the
//               pair. The whole K goes into one of two accumulators, so one
//               tile's stores overlap the next tile's MMAs.
// All tcgen05 instructions of the kernel use .cta_group::2.
//
// Every mbarrier wait is bounded by %globaltimer. On timeout the waiting
// thread records the error and raises its CTA's abort flag; the peer's waits
// then run out as well. Both CTAs meet at a cluster barrier before freeing
// tensor memory, so neither leaves while the other may still signal it.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdlib>
#include <cstring>
#include <string>

#include "epilogue.cuh"
#include "gemm_problem.cuh"
#include "internal.cuh"
#include "tc_store.cuh"
#include "tc_ptx.cuh"

namespace cdmpt {

namespace {

using namespace tc;

template <int BN, int STAGES, int PASSES>
struct Cfg2 {
    static constexpr int A_BYTES = BM * BK * 4;          // this CTA's 128 rows of X
    static constexpr int B_BYTES = (BN / 2) * BK * 4;    // this CTA's half of the Y tile
    static constexpr int PAIR_BYTES = A_BYTES + B_BYTES;
    static constexpr int STAGE_BYTES = PAIR_BYTES * (PASSES == 3 ? 2 : 1);
    static constexpr int BAR_BYTES = 256;
    // eight epilogue warps, each with a transpose buffer (tc_store.cuh)
    static constexpr int XPOSE_BYTES = 8 * kXposeWords * 4;
    static constexpr int SMEM = STAGES * STAGE_BYTES + BAR_BYTES + XPOSE_BYTES + 1024;
    static constexpr int THREADS = 320;
    static_assert(BN % 64 == 0 && BN >= 64 && BN <= 256, "BN");
    static_assert(A_BYTES % 1024 == 0 && B_BYTES % 1024 == 0, "1024-byte alignment of tiles");
    static_assert(SMEM <= 227 * 1024, "shared memory");
    static_assert((2 * STAGES + 8) * 8 + 8 <= BAR_BYTES, "barrier area");
};

__device__ __forceinline__ uint32_t mapa_u32(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}

// Arrive on an mbarrier given by its shared::cluster address with the default .release.cta
// semantics. The epilogue's per-chunk "accumulator drained" signal orders only tcgen05 loads
// (completed by tcgen05.wait::ld and tcgen05.fence::before_thread_sync) against the peer's MMA;
// a .release.cluster arrive would also wait, every chunk, for the warp's earlier global stores
// (the previous tile's epilogue) to become visible cluster-wide.
__device__ __forceinline__ void mbar_arrive_remote(uint32_t caddr) {
    asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(caddr) : "memory");
}

__device__ __forceinline__ uint32_t ld_cluster_u32(uint32_t caddr) {
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(caddr) : "memory");
    return v;
}

// Arrive on an mbarrier given by its shared::cluster address (either CTA).
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t caddr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(caddr)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait_cl(uint64_t* bar, uint32_t parity) {
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

// Bounded wait with cluster-scope acquire (barriers that the peer CTA signals).
__device__ __forceinline__ bool mbar_wait_cl(uint64_t* bar, uint32_t parity,
                                             volatile int* abort_flag, int* err, int code) {
    if (mbar_try_wait_cl(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (true) {
        if (mbar_try_wait_cl(bar, parity)) return true;
        if (*abort_flag) return false;
        if (globaltimer() - t0 > kWaitNs) {
            *abort_flag = 1;
            if (err) atomicCAS(err, 0, code);
            return false;
        }
    }
}

// TMA tile load into this CTA's shared memory whose completion is counted on
// the mbarrier at cluster address bar_c, which may belong to the peer CTA.
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* map, int x, int y,
                                                 uint32_t bar_c) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(bar_c)
        : "memory");
}

__device__ __forceinline__ void tmem_alloc_pair(uint32_t* holder, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(holder)),
                 "r"(cols)
                 : "memory");
}

__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols)
                 : "memory");
}

__device__ __forceinline__ void mma_tf32_pair(uint32_t tmem_d, uint64_t a, uint64_t b,
                                              uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// kind::f16 with both operands BF16 (K = 16 per instruction), FP32 accumulation.
__device__ __forceinline__ void mma_bf16_pair(uint32_t tmem_d, uint64_t a, uint64_t b,
                                              uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16 (bits 7-9 and
// 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
template <int M, int N>
__device__ __forceinline__ constexpr uint32_t idesc_bf16() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// Arrive on the mbarrier at the same offset in both CTAs of the pair once the
// MMAs issued so far by this thread complete.
__device__ __forceinline__ void mma_commit_pair(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
        " [%0], %1;" ::"r"(smem_u32(bar)),
        "h"((uint16_t)0x3)
        : "memory");
}

__device__ __forceinline__ void mma_commit_local_pair(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// BF16: operands are BF16 (64 elements per 128-byte row, kind::f16); else FP32
// read as TF32. The shared-memory layout is the same: 128-byte swizzled rows,
// four 32-byte k-steps per k-block.
template <int BN, int STAGES, int PASSES, int KCH, bool BF16 = false>
__global__ void __launch_bounds__(Cfg2<BN, STAGES, PASSES>::THREADS, 1)
    k_gemm_tc2sm(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY,
                 const __grid_constant__ CUtensorMap tmXl, const __grid_constant__ CUtensorMap tmYl,
                 const __grid_constant__ EpiParams<float> p, int K, int num_mt, int total_tiles,
                 const double* skip, int* err) {
    using C = Cfg2<BN, STAGES, PASSES>;
    // two accumulators; the chunked engine adds a sum buffer (power-of-two allocation)
    static_assert(KCH == 0, "the whole K in one of two accumulators");
    constexpr uint32_t kTmemCols = KCH > 0 ? 4 * BN : 2 * BN;
    static_assert(kTmemCols <= 512, "TMEM columns");
    // both CTAs of a pair read the same flag, so both return or neither does
    if (skip != nullptr && *skip != 0.0) return;

    extern __shared__ uint8_t smem_raw[];
    // the same offsets in both CTAs: the MMA addresses the peer's tiles by ours
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + STAGES * C::STAGE_BYTES);   // used in CTA 0
    uint64_t* empty = full + STAGES;
    // TMEM accumulators: two, or three for the chunked engine
    constexpr int NB = KCH > 0 ? 3 : 2;
    uint64_t* tfull = empty + STAGES;   // [NB]
    uint64_t* tempty = tfull + 3;       // [NB], used in CTA 0
    uint64_t* drain = tempty + 3;       // [1]
    uint32_t* tmem_holder = (uint32_t*)(drain + 1);
    volatile int* abort_flag = (volatile int*)(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const int cid = (int)(blockIdx.x >> 1), ncl = (int)(gridDim.x >> 1);
    constexpr int KB = BF16 ? 2 * BK : BK;   // K elements per 128-byte k-block
    static_assert(!BF16 || PASSES == 1, "BF16 is one pass");
    const int num_k = (K + KB - 1) / KB;
    // symmetric result with square 256 x 256 tiles: upper-triangular tiles only
    const bool sym = p.sym && BN == 2 * BM;
    auto tile_of = [&](int t, int* mt, int* nt) {
        if (sym) {
            tri_tile(t, num_mt, mt, nt);
        } else {
            *mt = t % num_mt;
            *nt = t / num_mt;
        }
    };
    auto chunks = [&](int* kc) {
        *kc = KCH > 0 ? KCH : num_k;
        return (num_k + *kc - 1) / *kc;
    };
    auto stage_a = [&](int s) { return smem + s * C::STAGE_BYTES; };
    auto stage_b = [&](int s) { return smem + s * C::STAGE_BYTES + C::A_BYTES; };
    auto stage_alo = [&](int s) { return smem + s * C::STAGE_BYTES + C::PAIR_BYTES; };
    auto stage_blo = [&](int s) {
        return smem + s * C::STAGE_BYTES + C::PAIR_BYTES + C::A_BYTES;
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < NB; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], 16);   // the eight epilogue warps of both CTAs
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 1) tmem_alloc_pair(tmem_holder, kTmemCols);
    tc_fence_before();
    __syncthreads();
    cluster_sync();   // barriers of both CTAs initialised, TMEM of the pair allocated
    tc_fence_after();
    const uint32_t tmem_base = *tmem_holder;
    // the pair's accumulators must sit at the same TMEM address in both CTAs
    const bool bad = ld_cluster_u32(mapa_u32(smem_u32(tmem_holder), rank ^ 1u)) != tmem_base;
    if (bad && threadIdx.x == 0) atomicCAS(err, 0, DEV_TMEM_MISMATCH);

    if (bad) {
        // fall through to the final barrier and free the allocation
    } else if (warp == 0) {
        // ------------------------------------------------ TMA producer (both CTAs)
        if (lane == 0) {
            prefetch_map(&tmX);
            prefetch_map(&tmY);
            if constexpr (PASSES == 3) {
                prefetch_map(&tmXl);
                prefetch_map(&tmYl);
            }
            const uint32_t full0 = mapa_u32(smem_u32(full), 0);   // CTA 0's full[0]
            uint32_t it = 0;
            bool ok = true;
            for (int t = cid; t < total_tiles && ok; t += ncl) {
                int mt = 0, nt = 0;
                tile_of(t, &mt, &nt);
                const int m0 = mt * (2 * BM) + (int)rank * BM;
                const int y0 = nt * BN + (int)rank * (BN / 2);
                for (int kb = 0; kb < num_k; ++kb, ++it) {
                    const int s = it % STAGES;
                    const uint32_t ph = (it / STAGES) & 1;
                    if (!mbar_wait_cl(&empty[s], ph ^ 1, abort_flag, err, DEV_TIMEOUT_EMPTY)) {
                        ok = false;
                        break;
                    }
                    if (rank == 0) mbar_expect_tx(&full[s], 2 * C::STAGE_BYTES);
                    const uint32_t fb = full0 + (uint32_t)s * 8u;
                    tma_load_2d_pair(stage_a(s), &tmX, kb * KB, m0, fb);
                    tma_load_2d_pair(stage_b(s), &tmY, kb * KB, y0, fb);
                    if constexpr (PASSES == 3) {
                        tma_load_2d_pair(stage_alo(s), &tmXl, kb * KB, m0, fb);
                        tma_load_2d_pair(stage_blo(s), &tmYl, kb * KB, y0, fb);
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer (CTA 0)
        if (lane == 0 && rank == 0) {
            constexpr uint32_t idesc = BF16 ? idesc_bf16<2 * BM, BN>() : idesc_tf32<2 * BM, BN>();
            uint32_t it = 0, g = 0;
            bool ok = true, issued = false;
            for (int t = cid; t < total_tiles && ok; t += ncl) {
                int kc = 0;
                const int nch = chunks(&kc);
                for (int c = 0; c < nch && ok; ++c, ++g) {
                    const int b = g % NB;
                    if (!mbar_wait_cl(&tempty[b], ((g / NB) & 1) ^ 1, abort_flag, err,
                                      DEV_TIMEOUT_ACCUM)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t tmem_d = tmem_base + (uint32_t)(b * BN);
                    const int kb0 = c * kc, kb1 = min(num_k, kb0 + kc);
                    for (int kb = kb0; kb < kb1; ++kb, ++it) {
                        const int s = it % STAGES;
                        const uint32_t ph = (it / STAGES) & 1;
                        if (!mbar_wait_cl(&full[s], ph, abort_flag, err, DEV_TIMEOUT_FULL)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a0 = smem_u32(stage_a(s)), b0 = smem_u32(stage_b(s));
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {   // 32-byte k-steps of the 128-byte row
                            const uint32_t off = kk * 32;
                            const uint64_t ah = sw128_desc(a0 + off), bh = sw128_desc(b0 + off);
                            const uint32_t first = ((kb - kb0) | kk) != 0 ? 1u : 0u;
                            if constexpr (PASSES == 3) {
                                const uint64_t al = sw128_desc(smem_u32(stage_alo(s)) + off);
                                const uint64_t bl = sw128_desc(smem_u32(stage_blo(s)) + off);
                                mma_tf32_pair(tmem_d, al, bh, idesc, first);
                                mma_tf32_pair(tmem_d, ah, bl, idesc, 1u);
                                mma_tf32_pair(tmem_d, ah, bh, idesc, 1u);
                            } else if constexpr (BF16) {
                                mma_bf16_pair(tmem_d, ah, bh, idesc, first);
                            } else {
                                mma_tf32_pair(tmem_d, ah, bh, idesc, first);
                            }
                        }
                        issued = true;
                        mma_commit_pair(&empty[s]);
                    }
                    if (!ok) break;
                    mma_commit_pair(&tfull[b]);
                }
            }
            if (!ok && issued) {
                mma_commit_local_pair(drain);
                mbar_drain(drain, 0);
            }
        }
    } else {
        // ------------------------------------------------ epilogue (both CTAs, warps 2 .. 9)
        // two warps per TMEM lane quarter, each with half of the tile's columns, stored in
        // 32 x 32 blocks through its transpose buffer
        const int ew = warp - 2;
        const int q = warp & 3;     // TMEM lane quarter this warp may read
        const int h = ew >> 2;      // column half
        const uint32_t lane_base = tmem_base + ((uint32_t)(32 * q) << 16);
        const uint32_t tempty0 = mapa_u32(smem_u32(tempty), 0);   // CTA 0's tempty[0]
        float* xbuf = (float*)(smem + STAGES * C::STAGE_BYTES + C::BAR_BYTES) + ew * kXposeWords;
        double dsum = 0.0;
        uint32_t g = 0;
        for (int t = cid; t < total_tiles; t += ncl) {
            int mt = 0, nt = 0;
            tile_of(t, &mt, &nt);
            const bool diag = sym && mt == nt;
            const int m0 = mt * (2 * BM) + (int)rank * BM + 32 * q;
            const int col0 = h * (BN / 2);
            const int b = g & 1;
            int w = 1;
            if (lane == 0)
                w = mbar_wait_cl(&tfull[b], (g >> 1) & 1, abort_flag, err, DEV_TIMEOUT_ACCUM);
            if (!__shfl_sync(0xffffffffu, w, 0)) break;
            tc_fence_after();
#pragma unroll 1
            for (int c0 = 0; c0 < BN / 2; c0 += 32) {
                uint32_t rr[32];
                tmem_ld32(lane_base + (uint32_t)(b * BN + col0 + c0), rr);
                float a[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) a[j] = __uint_as_float(rr[j]);
                dsum += (double)epi_block32(p, m0, nt * BN + col0 + c0, diag, a, xbuf, lane);
            }
            // the loads are complete (tcgen05.wait::ld); the plain arrive orders them before
            // the peer's next MMA without waiting for this tile's global stores
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_remote(tempty0 + (uint32_t)b * 8u);
            ++g;
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
        // after an abort, give copies still in flight time to land
        const unsigned long long t0 = globaltimer();
        while (globaltimer() - t0 < 100000ull) {
        }
    }
    __syncthreads();
    cluster_sync();   // no CTA frees TMEM or leaves while its peer may still signal it
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc_pair(tmem_base, kTmemCols);
    }
}

// ------------------------------------------------------------------ split TF32, wide tiles
// Split-TF32 product (lo*hi + hi*lo + hi*hi per k-step) on 256 x 256 output tiles of an SM
// pair. Order of the MMAs: each MMA truncates its FP32 result, an error of up to one unit in
// the last place of the accumulator. Within a k-block the eight cross-term MMAs (about 2^-11
// of the result) come first and the four hi*hi MMAs last, so on the first k-block of a chunk
// the cross terms are truncated at the scale of a small accumulator: a one-k-block chunk
// carries four truncations at the scale of the result instead of eleven. Against the 128 x 128 one-SM tile, every SM stages 128 rows of X and 128 rows of Y
// per k-block for twice the flops, so the shared-memory fill per flop (the L2 -> SM traffic,
// which bounds the narrow tile) halves. The accumulation restarts every KCH k-blocks (the
// truncating FP32 accumulation of the tensor cores; KCH = 0: whole K) into one of two
// 256-column TMEM accumulators, so the MMA of one chunk overlaps the drain of the other.
// EW = 8 epilogue warps per CTA: warp w drains TMEM lanes 32 (w % 4) of column group
// (w - 2) / 4, CW = 1024 / EW columns, and keeps its lane's CW running sums in registers
// (IEEE round-to-nearest adds). The drain of a chunk must keep pace with the chunk's MMAs
// (about 0.9 us at the TF32 rate); its arrival on the peer's barrier uses the plain
// (.release.cta) form, since a cluster-scope release made every drain wait for the previous
// tile's global stores (ncu: membar stalls dominated, 232 TF/s at N = 8192 against 344
// without). A finished tile is stored from the registers in 32 x 32 blocks through the warp's
// shared-memory transpose buffer (tc_store.cuh); the MMA meanwhile fills the other accumulator. Tiles run in groups of eight M-tiles (grouped raster), or over the
// upper triangle for symmetric results.
constexpr int SPLIT_BN = 256;
constexpr int SPLIT_GROUP = 8;
constexpr int split_threads(int ew) { return 32 * (2 + ew); }

// 16 consecutive columns of this warp's 32 TMEM lanes, completed before return (the
// 128 running sums and the 168-register budget of 320 threads leave room for 16 at a time)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int STAGES>
struct CfgS {
    static constexpr int A_BYTES = BM * BK * 4;                // this CTA's 128 rows of X
    static constexpr int B_BYTES = (SPLIT_BN / 2) * BK * 4;    // this CTA's 128 rows of Y
    static constexpr int PAIR_BYTES = A_BYTES + B_BYTES;
    static constexpr int STAGE_BYTES = 2 * PAIR_BYTES;         // hi and lo
    static constexpr int BAR_BYTES = 256;
    // eight epilogue warps, each with a transpose buffer (tc_store.cuh)
    static constexpr int XPOSE_BYTES = 8 * kXposeWords * 4;
    static constexpr int SMEM = STAGES * STAGE_BYTES + BAR_BYTES + XPOSE_BYTES + 1024;
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

// One output tile of the wide kernel: its problem's tensor maps, epilogue and K, and its
// position. Single launches take the kernel's own maps and parameters; grouped launches (the
// batched solve: one launch over the products of all systems) find the problem by binary search
// over the problems' first tiles.
struct WideTile {
    const CUtensorMap* mx;
    const CUtensorMap* my;
    const CUtensorMap* mxl;
    const CUtensorMap* myl;
    const EpiParams<float>* p;
    int mt, nt, num_k;
    bool sym, skip;
    int g;   // problem index (0 for single launches)
};

// Tile t of a problem with num_mt x num_nt tiles: the upper triangle for symmetric results,
// else groups of SPLIT_GROUP M-tiles (grouped raster).
__device__ __forceinline__ void wide_tile_pos(int t, int num_mt, int num_nt, bool sym, int* mt,
                                              int* nt) {
    if (sym) {
        tri_tile(t, num_mt, mt, nt);
    } else {
        const int grp = t / (SPLIT_GROUP * num_nt);
        const int first = grp * SPLIT_GROUP;
        const int gsize = min(SPLIT_GROUP, num_mt - first);
        const int r = t - grp * SPLIT_GROUP * num_nt;
        *mt = first + r % gsize;
        *nt = r / gsize;
    }
}

template <int STAGES, int KCH, int EW, bool GROUPED>
__global__ void __launch_bounds__(split_threads(EW), 1)
    k_gemm_split2sm(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY,
                    const __grid_constant__ CUtensorMap tmXl,
                    const __grid_constant__ CUtensorMap tmYl,
                    const __grid_constant__ EpiParams<float> p, int K, int num_mt, int num_nt,
                    int total_tiles, const double* skip, int* err, const GemmProblem* groups,
                    int G) {
    using C = CfgS<STAGES>;
    static_assert(EW == 8, "epilogue warps");
    constexpr int BN = SPLIT_BN, NB = 2, CW = 4 * BN / EW;
    constexpr int LW = CW >= 128 ? 32 : 16;   // columns per TMEM load
    constexpr uint32_t kTmemCols = NB * BN;
    if (!GROUPED && skip != nullptr && *skip != 0.0) return;

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + STAGES * C::STAGE_BYTES);   // used in CTA 0
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;   // [NB]
    uint64_t* tempty = tfull + NB;      // [NB], used in CTA 0
    uint64_t* drain = tempty + NB;
    uint32_t* tmem_holder = (uint32_t*)(drain + 1);
    volatile int* abort_flag = (volatile int*)(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const int cid = (int)(blockIdx.x >> 1), ncl = (int)(gridDim.x >> 1);
    auto tile = [&](int t) {
        WideTile w;
        if constexpr (GROUPED) {
            int lo = 0, hi = G - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (groups[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
            }
            const GemmProblem* pr = &groups[lo];
            w.g = lo;
            w.mx = pr->maps;
            w.my = pr->maps + 1;
            w.mxl = pr->maps + 2;
            w.myl = pr->maps + 3;
            w.p = &pr->p;
            w.sym = pr->p.sym != 0;
            w.num_k = (pr->K + BK - 1) / BK;
            w.skip = pr->skip != nullptr && *pr->skip != 0.0;
            wide_tile_pos(t - pr->tile_begin, pr->num_mt, (pr->p.N + BN - 1) / BN, w.sym, &w.mt,
                          &w.nt);
        } else {
            w.g = 0;
            w.mx = &tmX;
            w.my = &tmY;
            w.mxl = &tmXl;
            w.myl = &tmYl;
            w.p = &p;
            w.sym = p.sym != 0;
            w.num_k = (K + BK - 1) / BK;
            w.skip = false;
            wide_tile_pos(t, num_mt, num_nt, w.sym, &w.mt, &w.nt);
        }
        return w;
    };
    auto chunks = [&](int num_k, int* kc) {
        *kc = KCH > 0 ? KCH : num_k;
        return (num_k + *kc - 1) / *kc;
    };
    auto stage_a = [&](int s) { return smem + s * C::STAGE_BYTES; };
    auto stage_b = [&](int s) { return smem + s * C::STAGE_BYTES + C::A_BYTES; };
    auto stage_alo = [&](int s) { return smem + s * C::STAGE_BYTES + C::PAIR_BYTES; };
    auto stage_blo = [&](int s) {
        return smem + s * C::STAGE_BYTES + C::PAIR_BYTES + C::A_BYTES;
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < NB; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], 2 * EW);   // the epilogue warps of both CTAs
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 1) tmem_alloc_pair(tmem_holder, kTmemCols);
    tc_fence_before();
    __syncthreads();
    cluster_sync();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_holder;
    const bool bad = ld_cluster_u32(mapa_u32(smem_u32(tmem_holder), rank ^ 1u)) != tmem_base;
    if (bad && threadIdx.x == 0) atomicCAS(err, 0, DEV_TMEM_MISMATCH);

    if (bad) {
        // fall through to the final barrier and free the allocation
    } else if (warp == 0) {
        // ------------------------------------------------ TMA producer (both CTAs)
        if (lane == 0) {
            if constexpr (!GROUPED) {
                prefetch_map(&tmX);
                prefetch_map(&tmY);
                prefetch_map(&tmXl);
                prefetch_map(&tmYl);
            }
            const uint32_t full0 = mapa_u32(smem_u32(full), 0);
            uint32_t it = 0;
            bool ok = true;
            int last = -1;
            for (int t = cid; t < total_tiles && ok; t += ncl) {
                const WideTile w = tile(t);
                if (w.skip) continue;
                if constexpr (GROUPED) {
                    if (w.g != last) {   // maps written by the host: fence before first use
                        acquire_map(w.mx);
                        acquire_map(w.my);
                        acquire_map(w.mxl);
                        acquire_map(w.myl);
                        last = w.g;
                    }
                }
                const int m0 = w.mt * (2 * BM) + (int)rank * BM;
                const int y0 = w.nt * BN + (int)rank * (BN / 2);
                for (int kb = 0; kb < w.num_k; ++kb, ++it) {
                    const int s = it % STAGES;
                    const uint32_t ph = (it / STAGES) & 1;
                    if (!mbar_wait_cl(&empty[s], ph ^ 1, abort_flag, err, DEV_TIMEOUT_EMPTY)) {
                        ok = false;
                        break;
                    }
                    if (rank == 0) mbar_expect_tx(&full[s], 2 * C::STAGE_BYTES);
                    const uint32_t fb = full0 + (uint32_t)s * 8u;
                    tma_load_2d_pair(stage_a(s), w.mx, kb * BK, m0, fb);
                    tma_load_2d_pair(stage_b(s), w.my, kb * BK, y0, fb);
                    tma_load_2d_pair(stage_alo(s), w.mxl, kb * BK, m0, fb);
                    tma_load_2d_pair(stage_blo(s), w.myl, kb * BK, y0, fb);
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer (CTA 0)
        if (lane == 0 && rank == 0) {
            constexpr uint32_t idesc = idesc_tf32<2 * BM, BN>();
            uint32_t it = 0, g = 0;
            bool ok = true, issued = false;
            for (int t = cid; t < total_tiles && ok; t += ncl) {
                const WideTile w = tile(t);
                if (w.skip) continue;
                int kc = 0;
                const int nch = chunks(w.num_k, &kc);
                for (int c = 0; c < nch && ok; ++c, ++g) {
                    const int b = g % NB;
                    if (!mbar_wait_cl(&tempty[b], ((g / NB) & 1) ^ 1, abort_flag, err,
                                      DEV_TIMEOUT_ACCUM)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t tmem_d = tmem_base + (uint32_t)(b * BN);
                    const int kb0 = c * kc, kb1 = min(w.num_k, kb0 + kc);
                    for (int kb = kb0; kb < kb1; ++kb, ++it) {
                        const int s = it % STAGES;
                        const uint32_t ph = (it / STAGES) & 1;
                        if (!mbar_wait_cl(&full[s], ph, abort_flag, err, DEV_TIMEOUT_FULL)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a0 = smem_u32(stage_a(s)), b0 = smem_u32(stage_b(s));
                        const uint32_t al0 = smem_u32(stage_alo(s)), bl0 = smem_u32(stage_blo(s));
                        // cross terms of the k-block first, then its hi*hi terms
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint32_t off = kk * 32;
                            const uint32_t first = ((kb - kb0) | kk) != 0 ? 1u : 0u;
                            mma_tf32_pair(tmem_d, sw128_desc(al0 + off), sw128_desc(b0 + off),
                                          idesc, first);
                            mma_tf32_pair(tmem_d, sw128_desc(a0 + off), sw128_desc(bl0 + off),
                                          idesc, 1u);
                        }
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint32_t off = kk * 32;
                            mma_tf32_pair(tmem_d, sw128_desc(a0 + off), sw128_desc(b0 + off),
                                          idesc, 1u);
                        }
                        issued = true;
                        mma_commit_pair(&empty[s]);
                    }
                    if (!ok) break;
                    mma_commit_pair(&tfull[b]);
                }
            }
            if (!ok && issued) {
                mma_commit_local_pair(drain);
                mbar_drain(drain, 0);
            }
        }
    } else {
        // ------------------------------------------------ epilogue (both CTAs)
        const int q = warp & 3;            // TMEM lane quarter this warp may read
        const int h = (warp - 2) >> 2;     // column group
        const uint32_t lane_base = tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(CW * h);
        const uint32_t tempty0 = mapa_u32(smem_u32(tempty), 0);
        float* xbuf = (float*)(smem + STAGES * C::STAGE_BYTES + C::BAR_BYTES) +
                      (warp - 2) * kXposeWords;
        double dsum = 0.0;
        uint32_t g = 0;
        for (int t = cid; t < total_tiles; t += ncl) {
            const WideTile w = tile(t);
            if (w.skip) continue;
            const EpiParams<float>& P = *w.p;   // kernel parameter or problem descriptor
            const bool diag = w.sym && w.mt == w.nt;
            const int m = w.mt * (2 * BM) + (int)rank * BM + 32 * q + lane;
            const int n0 = w.nt * BN + CW * h;
            int kc = 0;
            const int nch = chunks(w.num_k, &kc);
            float acc[CW];
#pragma unroll
            for (int j = 0; j < CW; ++j) acc[j] = 0.f;
            bool ok = true;
            for (int c = 0; c < nch; ++c, ++g) {
                const int b = g % NB;
                int wt = 1;
                if (lane == 0)
                    wt = mbar_wait_cl(&tfull[b], (g / NB) & 1, abort_flag, err, DEV_TIMEOUT_ACCUM);
                if (!__shfl_sync(0xffffffffu, wt, 0)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int c0 = 0; c0 < CW; c0 += LW) {
                    uint32_t rr[LW];
                    if constexpr (LW == 32)
                        tmem_ld32(lane_base + (uint32_t)(b * BN + c0), rr);
                    else
                        tmem_ld16(lane_base + (uint32_t)(b * BN + c0), rr);
#pragma unroll
                    for (int j = 0; j < LW; ++j) acc[c0 + j] += __uint_as_float(rr[j]);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_remote(tempty0 + (uint32_t)b * 8u);
            }
            if (!ok) break;
#pragma unroll
            for (int c0 = 0; c0 < CW; c0 += 32) {
                float a[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) a[j] = acc[c0 + j];
                dsum += (double)epi_block32(P, m - lane, n0 + c0, diag, a, xbuf, lane);
            }
            if constexpr (GROUPED) {
                // each problem has its own dot target: flush per tile
                if (P.dot) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xffffffffu, dsum, o);
                    if (lane == 0 && dsum != 0.0) atomicAdd(P.dot, dsum);
                }
                dsum = 0.0;
            }
        }
        if constexpr (!GROUPED) {
            if (p.dot) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xffffffffu, dsum, o);
                if (lane == 0 && dsum != 0.0) atomicAdd(p.dot, dsum);
            }
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
        tmem_dealloc_pair(tmem_base, kTmemCols);
    }
}

// Tensor map of a BF16 operand (rows x cols, leading dimension ld elements).
bool make_map_bf16(CUtensorMap* map, const void* base, int rows, int cols, int ld, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)(2 * BK), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box,
                    estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int BN, int STAGES, int PASSES, int KCH, bool BF16 = false>
cdmpt_status launch_2sm(int M, int N, int K, const void* X, const void* Xl, int ldx,
                        const void* Y, const void* Yl, int ldy, const EpiParams<float>& p,
                        const double* skip, cudaStream_t s) {
    using C = Cfg2<BN, STAGES, PASSES>;
    auto kern = k_gemm_tc2sm<BN, STAGES, PASSES, KCH, BF16>;
    static int max_clusters = 0;
    if (max_clusters == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             C::SMEM);
        cudaLaunchConfig_t q = {};
        q.gridDim = dim3(2 * (sm_count() / 2));
        q.blockDim = dim3(C::THREADS);
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
            set_error("tcgen05 two-SM GEMM: no resident cluster of two");
            return CDMPT_ERR_UNSUPPORTED;
        }
        max_clusters = n;
    }
    CUtensorMap mx, my, mxl, myl;
    bool ok;
    if constexpr (BF16) {
        ok = make_map_bf16(&mx, X, M, K, ldx, BM) && make_map_bf16(&my, Y, N, K, ldy, BN / 2);
        mxl = mx;
        myl = my;
    } else {
        ok = make_map(&mx, (const float*)X, M, K, ldx, BM) &&
             make_map(&my, (const float*)Y, N, K, ldy, BN / 2) &&
             make_map(&mxl, (const float*)Xl, M, K, ldx, BM) &&
             make_map(&myl, (const float*)Yl, N, K, ldy, BN / 2);
    }
    if (!ok) {
        set_error("cuTensorMapEncodeTiled failed (alignment of X/Y or ld not a multiple of 4?)");
        return CDMPT_ERR_ARG;
    }
    const int num_mt = (M + 2 * BM - 1) / (2 * BM);
    const bool sym = p.sym && BN == 2 * BM && M == N;
    const int tiles = sym ? num_mt * (num_mt + 1) / 2 : num_mt * ((N + BN - 1) / BN);
    EpiParams<float> pk = p;
    pk.sym = sym ? 1 : 0;
    const int clusters = tiles < max_clusters ? tiles : max_clusters;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * clusters);
    cfg.blockDim = dim3(C::THREADS);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = s;
    cudaLaunchAttribute a;
    a.id = cudaLaunchAttributeClusterDimension;
    a.val.clusterDim.x = 2;
    a.val.clusterDim.y = 1;
    a.val.clusterDim.z = 1;
    cfg.attrs = &a;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, mx, my, mxl, myl, pk, K, num_mt, tiles, skip,
                                       device_error_word());
    count_launch();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("tcgen05 two-SM GEMM launch: ") + cudaGetErrorString(e));
        return CDMPT_ERR_CUDA;
    }
    return CDMPT_OK;
}



// Resident clusters of two of an instantiation of the wide kernel (0 with the error set when
// none fits), queried once per instantiation.
template <int STAGES, int KCH, int EW, bool GROUPED>
int split2sm_clusters() {
    using C = CfgS<STAGES>;
    auto kern = k_gemm_split2sm<STAGES, KCH, EW, GROUPED>;
    static int max_clusters = 0;
    if (max_clusters == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             C::SMEM);
        cudaLaunchConfig_t q = {};
        q.gridDim = dim3(2 * (sm_count() / 2));
        q.blockDim = dim3(split_threads(EW));
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
            set_error("split-TF32 two-SM GEMM: no resident cluster of two");
            return 0;
        }
        max_clusters = n;
    }
    return max_clusters;
}

template <int STAGES, int KCH, int EW, bool GROUPED>
cdmpt_status launch_wide(int clusters, const CUtensorMap& mx, const CUtensorMap& my,
                         const CUtensorMap& mxl, const CUtensorMap& myl, const EpiParams<float>& p,
                         int K, int num_mt, int num_nt, int tiles, const double* skip,
                         const GemmProblem* groups, int G, cudaStream_t s) {
    using C = CfgS<STAGES>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * clusters);
    cfg.blockDim = dim3(split_threads(EW));
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = s;
    cudaLaunchAttribute a;
    a.id = cudaLaunchAttributeClusterDimension;
    a.val.clusterDim.x = 2;
    a.val.clusterDim.y = 1;
    a.val.clusterDim.z = 1;
    cfg.attrs = &a;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_gemm_split2sm<STAGES, KCH, EW, GROUPED>, mx, my, mxl,
                                       myl, p, K, num_mt, num_nt, tiles, skip,
                                       device_error_word(), groups, G);
    count_launch();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("split-TF32 two-SM GEMM launch: ") + cudaGetErrorString(e));
        return CDMPT_ERR_CUDA;
    }
    return CDMPT_OK;
}

template <int STAGES, int KCH, int EW>
cdmpt_status launch_split2sm(int M, int N, int K, const float* X, const float* Xl, int ldx,
                             const float* Y, const float* Yl, int ldy, const EpiParams<float>& p,
                             const double* skip, cudaStream_t s) {
    const int max_clusters = split2sm_clusters<STAGES, KCH, EW, false>();
    if (max_clusters == 0) return CDMPT_ERR_UNSUPPORTED;
    CUtensorMap mx, my, mxl, myl;
    if (!make_map(&mx, X, M, K, ldx, BM) || !make_map(&my, Y, N, K, ldy, SPLIT_BN / 2) ||
        !make_map(&mxl, Xl, M, K, ldx, BM) || !make_map(&myl, Yl, N, K, ldy, SPLIT_BN / 2)) {
        set_error("cuTensorMapEncodeTiled failed (alignment of X/Y or ld not a multiple of 4?)");
        return CDMPT_ERR_ARG;
    }
    const int num_mt = (M + 2 * BM - 1) / (2 * BM);
    const int num_nt = (N + SPLIT_BN - 1) / SPLIT_BN;
    const bool sym = p.sym && M == N;
    const int tiles = sym ? num_mt * (num_mt + 1) / 2 : num_mt * num_nt;
    EpiParams<float> pk = p;
    pk.sym = sym ? 1 : 0;
    const int clusters = tiles < max_clusters ? tiles : max_clusters;
    return launch_wide<STAGES, KCH, EW, false>(clusters, mx, my, mxl, myl, pk, K, num_mt, num_nt,
                                               tiles, skip, nullptr, 0, s);
}

// Grouped launch over the problems of a batch (tiles numbered problem by problem, tensor maps
// in device memory, boxes of 128 rows for both operands).
template <int STAGES, int KCH, int EW>
cdmpt_status launch_split2sm_grouped(const GemmProblem* problems, int G, int total_tiles,
                                     cudaStream_t s) {
    const int max_clusters = split2sm_clusters<STAGES, KCH, EW, true>();
    if (max_clusters == 0) return CDMPT_ERR_UNSUPPORTED;
    CUtensorMap dummy;
    std::memset(&dummy, 0, sizeof(dummy));
    EpiParams<float> none;
    std::memset(&none, 0, sizeof(none));
    const int clusters = total_tiles < max_clusters ? total_tiles : max_clusters;
    return launch_wide<STAGES, KCH, EW, true>(clusters, dummy, dummy, dummy, dummy, none, 0, 0, 0,
                                              total_tiles, nullptr, problems, G, s);
}

}  // namespace

cdmpt_status gemm_tc_2sm(bool three, int kch, int M, int N, int K, const float* X,
                         const float* Xl, int ldx, const float* Y, const float* Yl, int ldy,
                         const EpiParams<float>& p, const double* skip, cudaStream_t s) {
    if (!three) return launch_2sm<256, 6, 1, 0>(M, N, K, X, X, ldx, Y, Y, ldy, p, skip, s);
    switch (kch) {
        case 0: return launch_split2sm<3, 0, 8>(M, N, K, X, Xl, ldx, Y, Yl, ldy, p, skip, s);
        case 2: return launch_split2sm<3, 2, 8>(M, N, K, X, Xl, ldx, Y, Yl, ldy, p, skip, s);
        case 4: return launch_split2sm<3, 4, 8>(M, N, K, X, Xl, ldx, Y, Yl, ldy, p, skip, s);
        default: return launch_split2sm<3, 1, 8>(M, N, K, X, Xl, ldx, Y, Yl, ldy, p, skip, s);
    }
}

cdmpt_status gemm_split2sm_grouped(int kch, const GemmProblem* problems, int G,
                                   int total_tiles, cudaStream_t s) {
    if (G <= 0 || total_tiles <= 0) return CDMPT_OK;
    switch (kch) {
        case 0: return launch_split2sm_grouped<3, 0, 8>(problems, G, total_tiles, s);
        case 2: return launch_split2sm_grouped<3, 2, 8>(problems, G, total_tiles, s);
        case 4: return launch_split2sm_grouped<3, 4, 8>(problems, G, total_tiles, s);
        default: return launch_split2sm_grouped<3, 1, 8>(problems, G, total_tiles, s);
    }
}

cdmpt_status gemm_tc_bf16(int M, int N, int K, const void* X, int ldx, const void* Y, int ldy,
                         const EpiParams<float>& p, const double* skip, cudaStream_t s) {
    return launch_2sm<256, 6, 1, 0, true>(M, N, K, X, X, ldx, Y, Y, ldy, p, skip, s);
}

}  // namespace cdmpt
