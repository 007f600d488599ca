// Persistent tcgen05 GEMM for sm_103a: D = alpha X Y^T + beta C + gamma I.
//
// Every product of the recursion has the form X Y^T with Y symmetric (the
// right factor is Z_k, A_k = I + Z_k^2, or the symmetrised response), so both
// operands are read K-major straight from row-major storage.
//
// Roles per CTA (one CTA per SM, persistent over output tiles):
//   warp 0      TMA producer: 128 x 32 and BN x 32 FP32 tiles, 128-byte
//               swizzle, into a STAGES-deep shared-memory ring;
//   warp 1      TMEM allocator and single-thread tcgen05.mma issuer
//               (kind::tf32, M = 128, N = BN, K = 8 per instruction) into
//               one of two TMEM accumulators (2 x BN columns);
//   warps 2..5  epilogue: tcgen05.ld of the accumulator (warp w reads TMEM
//               lanes 32 (w % 4) ...), alpha/beta/gamma, transposed
//               placement, fused Frobenius dot, global stores;
// For 3xTF32 the operands arrive already split in HBM (hi = rna_tf32(x),
// lo = rna_tf32(x - hi), written once by the kernel that produced x) and TMA
// loads the hi and lo tiles of both operands, so the MMA forms
// lo*hi + hi*lo + hi*hi (Ootomo & Yokota's split-TF32 scheme) with FP32
// accumulation in TMEM, restarted every KCH k-blocks and summed in registers.
//
// Every mbarrier wait is bounded (about 2 s of %globaltimer). On timeout a
// thread records the error, raises a shared abort flag that ends the other
// roles' loops, in-flight TMA/MMA work is drained with bounded waits, and the
// CTA frees its TMEM before returning.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>

#include "epilogue.cuh"
#include "gemm_problem.cuh"
#include "internal.cuh"

namespace cdmpt {

namespace {

constexpr int BM = 128;
constexpr int BK = 32;        // FP32 elements per 128-byte swizzle row
constexpr int UMMA_K = 8;     // K of one kind::tf32 instruction
constexpr unsigned long long kWaitNs = 2000000000ull;
// k-blocks (of 32) accumulated in TMEM before the partial sum moves to registers
// in the 3xTF32 engine. The tensor-core FP32 accumulation is not round-to-
// nearest; short chunks keep its bias at the level of FP32 rounding. The
// environment variable CDMPT_SPLIT_CHUNK (1, 2, 4 or 0 = whole K) overrides
// the default of 2 for tuning.
int split_chunk() {
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("CDMPT_SPLIT_CHUNK");
        v = e ? atoi(e) : 2;
        if (v != 0 && v != 1 && v != 2 && v != 4) v = 2;
    }
    return v;
}


template <int BN, int STAGES, int PASSES>
struct Cfg {
    static constexpr int A_BYTES = BM * BK * 4;
    static constexpr int B_BYTES = BN * BK * 4;
    static constexpr int PAIR_BYTES = A_BYTES + B_BYTES;
    // one pass: the A and B tiles; three passes: their hi and lo tiles
    static constexpr int STAGE_BYTES = PAIR_BYTES * (PASSES == 3 ? 2 : 1);
    static constexpr int BAR_BYTES = 256;
    static constexpr int SMEM = STAGES * STAGE_BYTES + BAR_BYTES + 1024;
    static constexpr int TMEM_COLS = 2 * BN;
    static constexpr int THREADS = 192;
    static_assert(BN % 32 == 0 && BN >= 64 && BN <= 256, "BN");
    static_assert(TMEM_COLS <= 512, "TMEM");
    static_assert(A_BYTES % 1024 == 0 && B_BYTES % 1024 == 0, "1024-byte alignment of tiles");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

// ---------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: true when the phase of the given parity completed; false when
// the abort flag is raised or the time limit passed (then the flag is raised
// and the error recorded).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          volatile int* abort_flag, int* err, int code) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (globaltimer() - t0 > kWaitNs) {
            *abort_flag = 1;
            if (err) atomicCAS(err, 0, code);
            return false;
        }
    }
}

// Bounded wait that ignores the abort flag (used while draining).
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity) {
    const unsigned long long t0 = globaltimer();
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer() - t0 > kWaitNs / 4) return;
    }
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// All threads of both CTAs of a cluster pair.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" :::
                     "memory");
}

// TMA load of one box into the same shared-memory offset of every CTA in
// mask, each CTA's mbarrier at the same offset receiving the transaction bytes.
__device__ __forceinline__ void tma_load_2d_mc(void* dst, const CUtensorMap* map, int x, int y,
                                               uint64_t* bar, uint16_t mask) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        ".multicast::cluster [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar)), "h"(mask)
        : "memory");
}

// Orders the tensormap proxy after the generic writes (a host copy) that put a
// tensor map into global memory, before TMA first reads it.
__device__ __forceinline__ void acquire_map(const CUtensorMap* map) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}

__device__ __forceinline__ void prefetch_map(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(map) : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* holder, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(holder)),
                 "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols)
                 : "memory");
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle:
// rows of 128 bytes, 8-row core groups 1024 bytes apart (stride byte offset),
// descriptor version 1 at bits 46-47, swizzle mode 2 (128 B) at bits 61-63.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor, kind::tf32: D = F32 (bits 4-5 = 1), A = B = TF32
// (bits 7-9 and 10-12 = 2), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28.
template <int BN>
__device__ __forceinline__ constexpr uint32_t idesc_tf32() {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
           ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// Arrives on the mbarrier at the same offset in every CTA of mask once this
// thread's prior tcgen05 operations complete.
__device__ __forceinline__ void mma_commit_mc(uint64_t* bar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
        " [%0], %1;" ::"r"(smem_u32(bar)),
        "h"(mask)
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t rna_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// ---------------------------------------------------------------- kernel

// Where one output tile lives: its problem, its corner and its tensor maps.
struct TileRef {
    const GemmProblem* pr;
    const CUtensorMap *mx, *my, *mxl, *myl;
    int m0, n0, num_k;
    bool skip;
};

// Tile t of the launch. A single problem uses the __grid_constant__ maps; a
// grouped launch finds the problem by binary search over tile_begin and reads
// its maps from global memory. A problem whose skip flag is set (its CG has
// converged) contributes no work; every role sees the same flags, so all roles
// walk the same sequence of tiles.
template <bool GROUPED>
__device__ __forceinline__ TileRef tile_ref(int t, const GemmProblem& single,
                                            const GemmProblem* groups, int G,
                                            const CUtensorMap* sx, const CUtensorMap* sy,
                                            const CUtensorMap* sxl, const CUtensorMap* syl) {
    TileRef r;
    const GemmProblem* pr;
    if constexpr (GROUPED) {
        int lo = 0, hi = G - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (groups[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
        }
        pr = &groups[lo];
        r.mx = pr->maps;
        r.my = pr->maps + 1;
        r.mxl = pr->maps + 2;
        r.myl = pr->maps + 3;
        r.skip = pr->skip != nullptr && *pr->skip != 0.0;
    } else {
        pr = &single;
        r.mx = sx;
        r.my = sy;
        r.mxl = sxl;
        r.myl = syl;
        r.skip = false;
    }
    const int lt = t - pr->tile_begin;
    r.pr = pr;
    r.m0 = (lt % pr->num_mt) * BM;
    r.n0 = 0;   // set by the caller, which knows BN
    r.num_k = (pr->K + BK - 1) / BK;
    return r;
}

// PAIR: a cluster of two CTAs works on vertically adjacent tiles (same B
// columns); each CTA loads its own A tile and half of the B tile, multicast to
// both, so each SM fetches half as many B bytes. Stage reuse then waits for
// both CTAs' MMAs (empty barriers count two commits).
template <int BN, int STAGES, int PASSES, int KCH, bool GROUPED, bool PAIR = false>
__global__ void __launch_bounds__(Cfg<BN, STAGES, PASSES>::THREADS, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY,
              const __grid_constant__ CUtensorMap tmXl, const __grid_constant__ CUtensorMap tmYl,
              const __grid_constant__ GemmProblem single, const GemmProblem* groups, int G,
              int total_tiles, int* err) {
    using C = Cfg<BN, STAGES, PASSES>;
    if (!GROUPED && single.skip != nullptr && *single.skip != 0.0) return;

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + STAGES * C::STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;   // [2]
    uint64_t* tempty = tfull + 2;       // [2]
    uint64_t* drain = tempty + 2;       // [1]
    uint32_t* tmem_holder = (uint32_t*)(drain + 1);
    volatile int* abort_flag = (volatile int*)(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    auto tile = [&](int t) {
        TileRef r = tile_ref<GROUPED>(t, single, groups, G, &tmX, &tmY, &tmXl, &tmYl);
        const int lt = t - r.pr->tile_begin;
        r.n0 = (lt / r.pr->num_mt) * BN;
        return r;
    };
    // K is accumulated in TMEM in chunks of kc k-blocks (KCH = 0: the whole K)
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

    const uint32_t rank = PAIR ? cluster_rank() : 0;
    // tile t of this CTA: single CTAs stride over tiles, pairs over tile pairs
    const int t_first = PAIR ? (int)(blockIdx.x / 2) * 2 + (int)rank : (int)blockIdx.x;
    const int t_step = PAIR ? (int)gridDim.x : (int)gridDim.x;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], PAIR ? 2 : 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], 128);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        fence_barrier_init();
        fence_proxy_async();
    }
    if (warp == 1) tmem_alloc(tmem_holder, C::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    if constexpr (PAIR) cluster_sync();   // peer barriers initialised before any multicast
    tc_fence_after();
    const uint32_t tmem_base = *tmem_holder;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            if constexpr (!GROUPED) {
                prefetch_map(&tmX);
                prefetch_map(&tmY);
                if constexpr (PASSES == 3) {
                    prefetch_map(&tmXl);
                    prefetch_map(&tmYl);
                }
            }
            uint32_t it = 0;
            bool ok = true;
            const GemmProblem* last = nullptr;
            for (int t = t_first; t < total_tiles && ok; t += t_step) {
                const TileRef r = tile(t);
                if (r.skip) continue;
                if constexpr (GROUPED) {
                    if (r.pr != last) {
                        acquire_map(r.mx);
                        acquire_map(r.my);
                        if constexpr (PASSES == 3) {
                            acquire_map(r.mxl);
                            acquire_map(r.myl);
                        }
                        last = r.pr;
                    }
                }
                for (int kb = 0; kb < r.num_k; ++kb, ++it) {
                    const int s = it % STAGES;
                    const uint32_t ph = (it / STAGES) & 1;
                    if (!mbar_wait(&empty[s], ph ^ 1, abort_flag, err, DEV_TIMEOUT_EMPTY)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&full[s], C::STAGE_BYTES);
                    tma_load_2d(stage_a(s), r.mx, kb * BK, r.m0, &full[s]);
                    if constexpr (PASSES == 3)
                        tma_load_2d(stage_alo(s), r.mxl, kb * BK, r.m0, &full[s]);
                    if constexpr (PAIR) {
                        // this CTA's half of the B box, into both CTAs
                        const int half = BN / 2;
                        const uint32_t off = rank * (uint32_t)(C::B_BYTES / 2);
                        tma_load_2d_mc(stage_b(s) + off, r.my, kb * BK, r.n0 + (int)rank * half,
                                       &full[s], (uint16_t)0x3);
                        if constexpr (PASSES == 3)
                            tma_load_2d_mc(stage_blo(s) + off, r.myl, kb * BK,
                                           r.n0 + (int)rank * half, &full[s], (uint16_t)0x3);
                    } else {
                        tma_load_2d(stage_b(s), r.my, kb * BK, r.n0, &full[s]);
                        if constexpr (PASSES == 3)
                            tma_load_2d(stage_blo(s), r.myl, kb * BK, r.n0, &full[s]);
                    }
                }
            }
            if (!ok) {
                // let the copies already issued land before the CTA exits
                const uint32_t first = it > (uint32_t)STAGES ? it - STAGES : 0;
                for (uint32_t j = first; j < it; ++j) mbar_drain(&full[j % STAGES], (j / STAGES) & 1);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_tf32<BN>();
            uint32_t it = 0, g = 0;
            bool ok = true, issued = false;
            for (int t = t_first; t < total_tiles && ok; t += t_step) {
                const TileRef r = tile(t);
                if (r.skip) continue;
                int kc = 0;
                const int nch = chunks(r.num_k, &kc);
                for (int c = 0; c < nch && ok; ++c, ++g) {
                    const int b = g & 1;
                    if (!mbar_wait(&tempty[b], ((g >> 1) & 1) ^ 1, abort_flag, err,
                                   DEV_TIMEOUT_ACCUM)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t tmem_d = tmem_base + (uint32_t)(b * BN);
                    const int kb0 = c * kc, kb1 = min(r.num_k, kb0 + kc);
                    for (int kb = kb0; kb < kb1; ++kb, ++it) {
                        const int s = it % STAGES;
                        const uint32_t ph = (it / STAGES) & 1;
                        if (!mbar_wait(&full[s], ph, abort_flag, err, DEV_TIMEOUT_FULL)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a0 = smem_u32(stage_a(s)), b0 = smem_u32(stage_b(s));
#pragma unroll
                        for (int kk = 0; kk < BK / UMMA_K; ++kk) {
                            const uint32_t off = kk * UMMA_K * 4;
                            const uint64_t ah = sw128_desc(a0 + off), bh = sw128_desc(b0 + off);
                            const uint32_t first = ((kb - kb0) | kk) != 0 ? 1u : 0u;
                            if constexpr (PASSES == 3) {
                                const uint64_t al = sw128_desc(smem_u32(stage_alo(s)) + off);
                                const uint64_t bl = sw128_desc(smem_u32(stage_blo(s)) + off);
                                mma_tf32(tmem_d, al, bh, idesc, first);
                                mma_tf32(tmem_d, ah, bl, idesc, 1u);
                                mma_tf32(tmem_d, ah, bh, idesc, 1u);
                            } else {
                                mma_tf32(tmem_d, ah, bh, idesc, first);
                            }
                        }
                        issued = true;
                        if constexpr (PAIR)
                            mma_commit_mc(&empty[s], (uint16_t)0x3);
                        else
                            mma_commit(&empty[s]);
                    }
                    if (!ok) break;
                    mma_commit(&tfull[b]);
                }
            }
            if (!ok && issued) {
                mma_commit(drain);
                mbar_drain(drain, 0);
            }
        }
    } else {
        // ------------------------------------------------ epilogue
        const int q = warp & 3;     // TMEM lane quarter this warp may read
        const uint32_t lane_base = tmem_base + ((uint32_t)(32 * q) << 16);
        double dsum = 0.0;
        uint32_t g = 0;
        for (int t = t_first; t < total_tiles; t += t_step) {
            const TileRef r = tile(t);
            if (r.skip) continue;
            const EpiParams<float> p = r.pr->p;
            const int m = r.m0 + 32 * q + lane;
            int kc = 0;
            const int nch = chunks(r.num_k, &kc);
            bool ok = true;
            if constexpr (KCH > 0) {
                // sum the short TMEM partial sums in registers (IEEE round-to-nearest)
                float acc[BN];
#pragma unroll
                for (int j = 0; j < BN; ++j) acc[j] = 0.f;
                for (int c = 0; c < nch; ++c, ++g) {
                    const int b = g & 1;
                    int w = 1;
                    if (lane == 0)
                        w = mbar_wait(&tfull[b], (g >> 1) & 1, abort_flag, err, DEV_TIMEOUT_ACCUM);
                    w = __shfl_sync(0xffffffffu, w, 0);
                    if (!w) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int c0 = 0; c0 < BN; c0 += 32) {
                        uint32_t rr[32];
                        tmem_ld32(lane_base + (uint32_t)(b * BN + c0), rr);
#pragma unroll
                        for (int j = 0; j < 32; ++j) acc[c0 + j] += __uint_as_float(rr[j]);
                    }
                    tc_fence_before();
                    mbar_arrive(&tempty[b]);
                }
                if (!ok) break;
                if (m < p.M) {
                    float local = 0.f;
#pragma unroll
                    for (int j = 0; j < BN; ++j) {
                        const int n = r.n0 + j;
                        if (n < p.N) local += epi_apply(p, m, n, acc[j]);
                    }
                    dsum += (double)local;
                }
            } else {
                (void)nch;
                const int b = g & 1;
                int w = 1;
                if (lane == 0)
                    w = mbar_wait(&tfull[b], (g >> 1) & 1, abort_flag, err, DEV_TIMEOUT_ACCUM);
                w = __shfl_sync(0xffffffffu, w, 0);
                if (!w) break;
                tc_fence_after();
#pragma unroll 1
                for (int c0 = 0; c0 < BN; c0 += 32) {
                    uint32_t rr[32];
                    tmem_ld32(lane_base + (uint32_t)(b * BN + c0), rr);
                    if (m < p.M) {
                        float local = 0.f;
                        const int nb = r.n0 + c0;
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const int n = nb + j;
                            if (n < p.N) local += epi_apply(p, m, n, __uint_as_float(rr[j]));
                        }
                        dsum += (double)local;
                    }
                }
                tc_fence_before();
                mbar_arrive(&tempty[b]);
                ++g;
            }
            if constexpr (GROUPED) {
                // each problem has its own dot target: flush per tile
                if (p.dot) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xffffffffu, dsum, o);
                    if (lane == 0 && dsum != 0.0) atomicAdd(p.dot, dsum);
                }
                dsum = 0.0;
            }
        }
        if constexpr (!GROUPED) {
            if (single.p.dot) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xffffffffu, dsum, o);
                if (lane == 0 && dsum != 0.0) atomicAdd(single.p.dot, dsum);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if constexpr (PAIR) cluster_sync();   // no CTA leaves while its peer may still signal it
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem_base, C::TMEM_COLS);
    }
}

// ---------------------------------------------------------------- host side

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
    });
    return fn;
}

bool make_map(CUtensorMap* map, const float* base, int rows, int cols, int ld, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 152;
    }
    return n;
}

template <int BN, int STAGES, int PASSES, int KCH, bool GROUPED>
cdmpt_status set_smem_attr() {
    using C = Cfg<BN, STAGES, PASSES>;
    static bool done = false;
    if (!done) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<BN, STAGES, PASSES, KCH, GROUPED>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (e != cudaSuccess) {
            set_error(std::string("tcgen05 GEMM smem attribute: ") + cudaGetErrorString(e));
            return CDMPT_ERR_CUDA;
        }
        done = true;
    }
    return CDMPT_OK;
}

template <int BN, int STAGES, int PASSES, int KCH>
cdmpt_status launch(int M, int N, int K, const float* X, const float* Xl, int ldx, const float* Y,
                    const float* Yl, int ldy, const EpiParams<float>& p, const double* skip,
                    cudaStream_t s) {
    using C = Cfg<BN, STAGES, PASSES>;
    {
        const cdmpt_status st = set_smem_attr<BN, STAGES, PASSES, KCH, false>();
        if (st != CDMPT_OK) return st;
    }
    CUtensorMap mx, my, mxl, myl;
    if (!make_map(&mx, X, M, K, ldx, BM) || !make_map(&my, Y, N, K, ldy, BN) ||
        !make_map(&mxl, Xl, M, K, ldx, BM) || !make_map(&myl, Yl, N, K, ldy, BN)) {
        set_error("cuTensorMapEncodeTiled failed (alignment of X/Y or ld not a multiple of 4?)");
        return CDMPT_ERR_ARG;
    }
    GemmProblem pr;
    pr.p = p;
    pr.K = K;
    pr.tile_begin = 0;
    pr.num_mt = (M + BM - 1) / BM;
    pr.skip = skip;
    pr.maps = nullptr;
    const int tiles = pr.num_mt * ((N + BN - 1) / BN);
    const int grid = tiles < sm_count() ? tiles : sm_count();
    k_gemm_tc<BN, STAGES, PASSES, KCH, false><<<grid, C::THREADS, C::SMEM, s>>>(
        mx, my, mxl, myl, pr, nullptr, 1, tiles, device_error_word());
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("tcgen05 GEMM launch: ") + cudaGetErrorString(e));
        return CDMPT_ERR_CUDA;
    }
    return CDMPT_OK;
}

// Cluster-pair launch (B multicast); needs an even number of M tiles.
template <int BN, int STAGES, int PASSES, int KCH>
cdmpt_status launch_pair(int M, int N, int K, const float* X, const float* Xl, int ldx,
                         const float* Y, const float* Yl, int ldy, const EpiParams<float>& p,
                         const double* skip, cudaStream_t s) {
    using C = Cfg<BN, STAGES, PASSES>;
    auto kern = k_gemm_tc<BN, STAGES, PASSES, KCH, false, true>;
    static int max_clusters = 0;
    if (max_clusters == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             C::SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 0);
        cudaLaunchConfig_t q = {};
        q.gridDim = dim3(2 * sm_count() / 2);
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
            set_error("tcgen05 pair GEMM: no resident cluster of two");
            return CDMPT_ERR_UNSUPPORTED;
        }
        max_clusters = n;
    }
    CUtensorMap mx, my, mxl, myl;
    if (!make_map(&mx, X, M, K, ldx, BM) || !make_map(&my, Y, N, K, ldy, BN / 2) ||
        !make_map(&mxl, Xl, M, K, ldx, BM) || !make_map(&myl, Yl, N, K, ldy, BN / 2)) {
        set_error("cuTensorMapEncodeTiled failed (alignment of X/Y or ld not a multiple of 4?)");
        return CDMPT_ERR_ARG;
    }
    GemmProblem pr;
    pr.p = p;
    pr.K = K;
    pr.tile_begin = 0;
    pr.num_mt = (M + BM - 1) / BM;
    pr.skip = skip;
    pr.maps = nullptr;
    const int tiles = pr.num_mt * ((N + BN - 1) / BN);
    const int pairs = tiles / 2;
    const int clusters = pairs < max_clusters ? pairs : max_clusters;
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
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, mx, my, mxl, myl, pr,
                                       (const GemmProblem*)nullptr, 1, tiles, device_error_word());
    count_launch();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("tcgen05 pair GEMM launch: ") + cudaGetErrorString(e));
        return CDMPT_ERR_CUDA;
    }
    return CDMPT_OK;
}

bool pair_enabled() {
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("CDMPT_PAIR");
        v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

template <int BN, int STAGES, int PASSES, int KCH>
cdmpt_status launch_grouped(const GemmProblem* problems, int G, int total_tiles, cudaStream_t s) {
    using C = Cfg<BN, STAGES, PASSES>;
    {
        const cdmpt_status st = set_smem_attr<BN, STAGES, PASSES, KCH, true>();
        if (st != CDMPT_OK) return st;
    }
    CUtensorMap dummy;
    std::memset(&dummy, 0, sizeof(dummy));
    GemmProblem none;
    std::memset(&none, 0, sizeof(none));
    const int grid = total_tiles < sm_count() ? total_tiles : sm_count();
    k_gemm_tc<BN, STAGES, PASSES, KCH, true><<<grid, C::THREADS, C::SMEM, s>>>(
        dummy, dummy, dummy, dummy, none, problems, G, total_tiles, device_error_word());
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("grouped tcgen05 GEMM launch: ") + cudaGetErrorString(e));
        return CDMPT_ERR_CUDA;
    }
    return CDMPT_OK;
}

}  // namespace

int tc_tile_n(int engine) { return engine == CDMPT_GEMM_TC_TF32 ? 256 : 128; }
int tc_tile_m() { return BM; }

bool tc_encode_operand(CUtensorMap* map, const float* base, int rows, int cols, int ld,
                       bool as_y, int engine) {
    // as X: box of 128 rows (BM); as Y: box of the engine's BN rows
    return make_map(map, base, rows, cols, ld, as_y ? tc_tile_n(engine) : BM);
}

cdmpt_status gemm_tc_grouped(int engine, const GemmProblem* problems, int G, int total_tiles,
                             cudaStream_t s) {
    if (G <= 0 || total_tiles <= 0) return CDMPT_OK;
    if (!tc_supported()) {
        set_error("tcgen05 GEMM needs an sm_103 device");
        return CDMPT_ERR_UNSUPPORTED;
    }
    if (engine == CDMPT_GEMM_TC_TF32) return launch_grouped<256, 4, 1, 0>(problems, G, total_tiles, s);
    switch (split_chunk()) {
        case 1: return launch_grouped<128, 3, 3, 1>(problems, G, total_tiles, s);
        case 4: return launch_grouped<128, 3, 3, 4>(problems, G, total_tiles, s);
        case 0: return launch_grouped<128, 3, 3, 0>(problems, G, total_tiles, s);
        default: return launch_grouped<128, 3, 3, 2>(problems, G, total_tiles, s);
    }
}

bool tc_supported() {
    static int cached = -1;
    if (cached < 0) {
        int dev = 0, major = 0, minor = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
        cached = (major == 10 && minor == 3) ? 1 : 0;
    }
    return cached == 1;
}

cdmpt_status gemm_tc_f32(int engine, int M, int N, int K, const Operand<float>& X, int ldx,
                         const Operand<float>& Y, int ldy, float* D, int ldd,
                         const Epilogue<float>& ep, const double* skip, cudaStream_t s) {
    if (M <= 0 || N <= 0) return CDMPT_OK;
    if (!tc_supported()) {
        set_error("tcgen05 GEMM needs an sm_103 device");
        return CDMPT_ERR_UNSUPPORTED;
    }
    const bool three = engine != CDMPT_GEMM_TC_TF32;
    const float* xh = X.hi ? X.hi : X.x;
    const float* yh = Y.hi ? Y.hi : Y.x;
    if (three && (!X.hi || !X.lo || !Y.hi || !Y.lo)) {
        set_error("3xTF32 GEMM needs the hi/lo split of both operands");
        return CDMPT_ERR_ARG;
    }
    auto misaligned = [](const float* q) { return q && (((uintptr_t)q) & 15); };
    if ((ldx & 3) || (ldy & 3) || !xh || !yh || misaligned(xh) || misaligned(yh) ||
        misaligned(X.lo) || misaligned(Y.lo) || K < 1) {
        set_error("tcgen05 GEMM: X/Y must be 16-byte aligned with ld a multiple of 4, K >= 1");
        return CDMPT_ERR_ARG;
    }
    EpiParams<float> p;
    p.alpha = (float)ep.alpha;
    p.beta = (float)ep.beta;
    p.gamma = (float)ep.gamma;
    p.C = ep.C;
    p.ldc = ep.ldc;
    p.D = D;
    p.ldd = ldd;
    p.M = M;
    p.N = N;
    p.diag_block = ep.diag_block > 0 ? ep.diag_block : M;
    p.trans_block = ep.trans_block;
    p.dot = ep.dot;
    p.E = ep.E;
    p.lde = ep.lde;
    p.Dhi = ep.Dhi;
    p.Dlo = ep.Dlo;
    const bool pair = pair_enabled() && ((M + BM - 1) / BM) % 2 == 0;
    if (!three) {
        if (pair) return launch_pair<256, 4, 1, 0>(M, N, K, xh, xh, ldx, yh, yh, ldy, p, skip, s);
        return launch<256, 4, 1, 0>(M, N, K, xh, xh, ldx, yh, yh, ldy, p, skip, s);
    }
    if (pair && split_chunk() == 2)
        return launch_pair<128, 3, 3, 2>(M, N, K, xh, X.lo, ldx, yh, Y.lo, ldy, p, skip, s);
    switch (split_chunk()) {
        case 1: return launch<128, 3, 3, 1>(M, N, K, xh, X.lo, ldx, yh, Y.lo, ldy, p, skip, s);
        case 4: return launch<128, 3, 3, 4>(M, N, K, xh, X.lo, ldx, yh, Y.lo, ldy, p, skip, s);
        case 0: return launch<128, 3, 3, 0>(M, N, K, xh, X.lo, ldx, yh, Y.lo, ldy, p, skip, s);
        default: return launch<128, 3, 3, 2>(M, N, K, xh, X.lo, ldx, yh, Y.lo, ldy, p, skip, s);
    }
}

}  // namespace cdmpt
