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
//   warps 2..9  epilogue: tcgen05.ld of the accumulator (warp w reads TMEM
//               lanes 32 (w % 4) ...), alpha/beta/gamma, transposed
//               placement, fused Frobenius dot, global stores in 32 x 32
//               blocks through a per-warp shared-memory transpose
//               (tc_store.cuh), so that every access is a row segment;
// For 3xTF32 the operands arrive already split in HBM (hi = rna_tf32(x),
// lo = rna_tf32(x - hi), written once by the kernel that produced x) and TMA
// loads the hi and lo tiles of both operands, so the MMA forms
// lo*hi + hi*lo + hi*hi (Ootomo & Yokota's split-TF32 scheme) with FP32
// accumulation in TMEM, restarted every KCH k-blocks and summed in registers.
// Each MMA truncates its FP32 result (an error of up to one unit in the last
// place of the accumulator), so within a k-block the eight cross-term MMAs,
// about 2^-11 of the result, are issued before the four hi*hi ones: on the
// first k-block of a chunk they are truncated at the scale of a small
// accumulator.
// Warps 2..9 (two per TMEM lane quarter, each with half of the columns) sum the
// chunks of a tile and park the finished sums in a TMEM sum buffer; warps 10..13
// (one per quarter) store the parked tile while the chunk warps drain the next
// tile's chunks, so the global stores overlap the MMAs. With the whole K in one
// accumulator (one pass, or KCH = 0) warps 2..9 drain it and store it themselves.
//
// Block-norm screening (single launches with a GemmProblem::mask): k-slice kb of
// an output tile is skipped when the product of the Frobenius norms of its X and Y
// tiles is at most tau, as recorded in a per-tile bit mask built before the launch
// (screen_mask). Producer, MMA issuer and epilogue read the same mask words, so
// they walk the same sequence of slices; a tile with no slice left is written by the
// epilogue as beta C + gamma I with coalesced stores (epi_fill_zero_tile), without
// touching TMEM or a barrier, and chunks group the remaining slices.
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
#include "tc_store.cuh"
#include "tc_ptx.cuh"

namespace cdmpt {

namespace {

using namespace tc;

// k-blocks (of 32) accumulated in TMEM before the partial sum moves to registers
// in the 3xTF32 engine. The tensor-core FP32 accumulation truncates rather than
// rounds, so its error has a bias that grows with the chunk; one k-block per chunk
// halves the mixed-precision P1 error against two (measured) for about 5 % of the
// solve time. The environment variable CDMPT_SPLIT_CHUNK (1, 2, 4 or 0 = whole K)
// overrides the default of 1 for tuning.
int split_chunk() {
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("CDMPT_SPLIT_CHUNK");
        v = e ? atoi(e) : 1;
        if (v != 0 && v != 1 && v != 2 && v != 4) v = 1;
    }
    return v;
}


// Threads of the kernel: producer and MMA warps, eight warps that drain the accumulators and,
// in the chunked engine, four store warps.
constexpr int tc_threads(int kch) { return kch > 0 ? 448 : 320; }

template <int BN, int STAGES, int PASSES>
struct Cfg {
    static constexpr int A_BYTES = BM * BK * 4;
    static constexpr int B_BYTES = BN * BK * 4;
    static constexpr int PAIR_BYTES = A_BYTES + B_BYTES;
    // one pass: the A and B tiles; three passes: their hi and lo tiles
    static constexpr int STAGE_BYTES = PAIR_BYTES * (PASSES == 3 ? 2 : 1);
    // mbarriers (256 bytes), then the grouped launches' tile cache (kTileCache entries)
    static constexpr int BAR_BYTES = 1024;
    // eight epilogue warps, each with a transpose buffer (tc_store.cuh)
    static constexpr int XPOSE_BYTES = 8 * kXposeWords * 4;
    static constexpr int SMEM = STAGES * STAGE_BYTES + BAR_BYTES + XPOSE_BYTES + 1024;
    static constexpr int TMEM_COLS = 2 * BN;
    static_assert(BN % 32 == 0 && BN >= 64 && BN <= 256, "BN");
    static_assert(TMEM_COLS <= 512, "TMEM");
    static_assert(A_BYTES % 1024 == 0 && B_BYTES % 1024 == 0, "1024-byte alignment of tiles");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

// ---------------------------------------------------------------- kernel

// Where one output tile lives: its problem, its corner and its tensor maps.
struct TileRef {
    const GemmProblem* pr;
    const CUtensorMap *mx, *my, *mxl, *myl;
    int m0, n0, num_k;
    bool skip;
    bool diag;   // symmetric result: a tile on the block diagonal
};

// Tile t of the launch. A single problem uses the __grid_constant__ maps; a
// grouped launch finds the problem by binary search over tile_begin and reads
// its maps from global memory. A problem whose skip flag is set (its CG has
// converged) contributes no work; every role sees the same flags, so all roles
// walk the same sequence of tiles.
// Problem of launch-wide tile t: binary search over tile_begin.
__device__ __forceinline__ int find_problem(int t, const GemmProblem* groups, int G) {
    int lo = 0, hi = G - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (groups[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Tiles of a grouped launch whose problem, K and skip flag each CTA looks up once, in
// parallel, when it starts (entry i: the CTA's i-th tile): the MMA issuer then starts a
// tile without a chain of dependent global loads. Later tiles use find_problem.
constexpr int kTileCache = 96;

template <bool GROUPED>
__device__ __forceinline__ TileRef tile_ref(int t, const GemmProblem& single,
                                            const GemmProblem* groups, int G,
                                            const CUtensorMap* sx, const CUtensorMap* sy,
                                            const CUtensorMap* sxl, const CUtensorMap* syl,
                                            const int2* cached = nullptr) {
    TileRef r;
    const GemmProblem* pr;
    if constexpr (GROUPED) {
        if (cached) {   // {problem, num_k or -1 when skipped}
            const int2 e = *cached;
            pr = &groups[e.x];
            r.skip = e.y < 0;
            r.num_k = e.y < 0 ? 0 : e.y;
        } else {
            pr = &groups[find_problem(t, groups, G)];
            r.skip = pr->skip != nullptr && *pr->skip != 0.0;
            r.num_k = (pr->K + BK - 1) / BK;
        }
        r.mx = pr->maps;
        r.my = pr->maps + 1;
        r.mxl = pr->maps + 2;
        r.myl = pr->maps + 3;
    } else {
        pr = &single;
        r.mx = sx;
        r.my = sy;
        r.mxl = sxl;
        r.myl = syl;
        r.skip = false;
        r.num_k = (pr->K + BK - 1) / BK;
    }
    const int lt = t - pr->tile_begin;
    r.pr = pr;
    r.m0 = (lt % pr->num_mt) * BM;
    r.n0 = 0;   // set by the caller, which knows BN
    return r;
}

// Epilogue of a tile whose product is zero (every k-slice screened out): D = beta C + gamma I
// over the tile and, for a symmetric result off the diagonal, over its mirror. Without TMEM
// the lanes need not own rows: warps take rows and lanes 16-byte column groups, so every
// store is coalesced (the mirror gets its own row-major pass, C and E being symmetric). With
// transposed placement the lanes take rows instead, which the placement turns into
// consecutive columns. Warp q of nq takes every nq-th row (column). Returns the D * E
// contribution of the lane's elements.
template <int BN>
__device__ double epi_fill_zero_tile(const EpiParams<float>& p, int m0, int n0, bool diag, int q,
                                     int nq, int lane) {
    double dsum = 0.0;
    if (p.trans_block > 0) {
        for (int j = q; j < BN && n0 + j < p.N; j += nq)
            for (int i = lane; i < BM && m0 + i < p.M; i += 32)
                dsum += (double)epi_apply(p, m0 + i, n0 + j, 0.f);
        return dsum;
    }
    EpiParams<float> f = p;
    f.sym = 0;
    const bool vec4 = epi_vec4_ok(f);
    auto pass = [&](int r0, int c0, int rows, int cols) {
        for (int i = q; i < rows && r0 + i < f.M; i += nq) {
            const int m = r0 + i;
            for (int c = lane * 4; c < cols; c += 128) {
                const int n = c0 + c;
                if (vec4 && n + 4 <= f.N) {
                    dsum += (double)epi_apply4(f, m, n, 0.f, 0.f, 0.f, 0.f);
                } else {
                    for (int t = 0; t < 4 && n + t < f.N; ++t)
                        dsum += (double)epi_apply(f, m, n + t, 0.f);
                }
            }
        }
    };
    pass(m0, n0, BM, BN);
    if (p.sym && !diag) pass(n0, m0, BN, BM);
    return dsum;
}

// Every CTA loads its own A and B tiles (no cluster, no multicast).
template <int BN, int STAGES, int PASSES, int KCH, bool GROUPED, bool SCREEN = false>
__global__ void __launch_bounds__(tc_threads(KCH), 1)
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
    // TMEM accumulators: two, or three for the chunked engine (the MMA may then
    // run two chunks ahead of the epilogue)
    constexpr int NB = KCH > 0 ? 3 : 2;
    uint64_t* tfull = empty + STAGES;   // [NB]
    uint64_t* tempty = tfull + 3;       // [NB]
    uint64_t* drain = tempty + 3;       // [1]
    uint64_t* parked = drain + 1;       // chunked engine: a finished tile is in the sum buffer
    uint64_t* pfree = parked + 1;       // ... and has been read by the store warps
    uint32_t* tmem_holder = (uint32_t*)(pfree + 1);
    volatile int* abort_flag = (volatile int*)(tmem_holder + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // symmetric results (p.sym, square tiles) enumerate the upper-triangular tiles only
    const int2* tcache = (const int2*)(smem + STAGES * C::STAGE_BYTES + 256);
    auto tile = [&](int t) {
        const int li = (t - (int)blockIdx.x) / (int)gridDim.x;
        TileRef r = tile_ref<GROUPED>(t, single, groups, G, &tmX, &tmY, &tmXl, &tmYl,
                                      GROUPED && li < kTileCache ? tcache + li : nullptr);
        const int lt = t - r.pr->tile_begin;
        r.diag = false;
        if (BN == BM && r.pr->p.sym) {
            int mi = 0, ni = 0;
            tri_tile(lt, r.pr->num_mt, &mi, &ni);
            r.m0 = mi * BM;
            r.n0 = ni * BN;
            r.diag = mi == ni;
        } else {
            r.n0 = (lt / r.pr->num_mt) * BN;
        }
        return r;
    };
    // K is accumulated in TMEM in chunks of kc k-blocks (KCH = 0: the whole K)
    auto chunks = [&](int num_k, int* kc) {
        *kc = KCH > 0 ? KCH : num_k;
        return (num_k + *kc - 1) / *kc;
    };
    // block-norm screening (compiled in only for the screened instantiations): the mask
    // words of tile r (BN = BM = 128 when screened)
    constexpr bool screen = SCREEN && !GROUPED;
    auto mask_of = [&](const TileRef& r) -> const uint32_t* {
        return single.mask + ((size_t)(r.m0 / BM) * single.nnt + r.n0 / BM) * single.nmw;
    };
    auto count_active = [&](const TileRef& r) -> int {
        if constexpr (!screen) {
            return r.num_k;
        } else {
            const uint32_t* w = mask_of(r);
            int c = 0;
            for (int i = 0; i < single.nmw; ++i) c += __popc(w[i]);
            return c;
        }
    };

    auto stage_a = [&](int s) { return smem + s * C::STAGE_BYTES; };
    auto stage_b = [&](int s) { return smem + s * C::STAGE_BYTES + C::A_BYTES; };
    auto stage_alo = [&](int s) { return smem + s * C::STAGE_BYTES + C::PAIR_BYTES; };
    auto stage_blo = [&](int s) {
        return smem + s * C::STAGE_BYTES + C::PAIR_BYTES + C::A_BYTES;
    };

    // tile t of this CTA: CTAs stride over the tiles
    const int t_first = (int)blockIdx.x;
    const int t_step = (int)gridDim.x;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < NB; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], 8);   // one arrival per draining warp
        }
        mbar_init(drain, 1);
        mbar_init(parked, 8);   // the eight chunk warps
        mbar_init(pfree, 4);    // the four store warps
        *abort_flag = 0;
        fence_barrier_init();
        fence_proxy_async();
    }
    // chunked engine: three chunk accumulators and a sum buffer (power-of-two allocation)
    constexpr uint32_t kTmemCols = KCH > 0 ? 4 * BN : C::TMEM_COLS;
    static_assert(kTmemCols <= 512, "TMEM columns");
    if (warp == 1) tmem_alloc(tmem_holder, kTmemCols);
    if constexpr (GROUPED) {
        // the tile cache: one lookup per thread, all in parallel
        int2* fill = (int2*)(smem + STAGES * C::STAGE_BYTES + 256);
        for (int i = (int)threadIdx.x; i < kTileCache; i += (int)blockDim.x) {
            const int t = t_first + i * t_step;
            int2 e = make_int2(0, -1);
            if (t < total_tiles) {
                const int g = find_problem(t, groups, G);
                const GemmProblem* pr = &groups[g];
                const bool sk = pr->skip != nullptr && *pr->skip != 0.0;
                e = make_int2(g, sk ? -1 : (pr->K + BK - 1) / BK);
            }
            fill[i] = e;
        }
    }
    tc_fence_before();
    __syncthreads();
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
                const uint32_t* mw = screen ? mask_of(r) : nullptr;
                uint32_t word = 0xffffffffu;
                for (int kb = 0; kb < r.num_k; ++kb) {
                    if constexpr (screen) {
                        if ((kb & 31) == 0) word = mw[kb >> 5];
                        if (!((word >> (kb & 31)) & 1u)) continue;
                    }
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
                    tma_load_2d(stage_b(s), r.my, kb * BK, r.n0, &full[s]);
                    if constexpr (PASSES == 3)
                        tma_load_2d(stage_blo(s), r.myl, kb * BK, r.n0, &full[s]);
                    ++it;
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
            constexpr uint32_t idesc = idesc_tf32<BM, BN>();
            uint32_t it = 0, g = 0;
            unsigned long long computed = 0, examined = 0;
            bool ok = true, issued = false;
            for (int t = t_first; t < total_tiles && ok; t += t_step) {
                const TileRef r = tile(t);
                if (r.skip) continue;
                const int na = count_active(r);
                computed += (unsigned long long)na;
                examined += (unsigned long long)r.num_k;
                if (na == 0) continue;   // the epilogue writes this tile from zero
                // the producer issues the computed slices in order, so the issuer only
                // needs their number
                int kc = 0;
                const int nch = chunks(na, &kc);
                for (int c = 0; c < nch && ok; ++c, ++g) {
                    const int b = g % NB;
                    if (!mbar_wait(&tempty[b], ((g / NB) & 1) ^ 1, abort_flag, err,
                                   DEV_TIMEOUT_ACCUM)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t tmem_d = tmem_base + (uint32_t)(b * BN);
                    // positions kb0 .. kb1 - 1 of the sequence of computed k-slices (all of
                    // them when dense)
                    const int kb0 = c * kc, kb1 = min(na, kb0 + kc);
                    for (int q = kb0; q < kb1; ++q, ++it) {
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
                            const uint32_t first = ((q - kb0) | kk) != 0 ? 1u : 0u;
                            if constexpr (PASSES == 3) {
                                // the two cross terms of the k-block come first, while the
                                // chunk's accumulator is small (see the note on the order)
                                const uint64_t al = sw128_desc(smem_u32(stage_alo(s)) + off);
                                const uint64_t bl = sw128_desc(smem_u32(stage_blo(s)) + off);
                                mma_tf32(tmem_d, al, bh, idesc, first);
                                mma_tf32(tmem_d, ah, bl, idesc, 1u);
                            } else {
                                mma_tf32(tmem_d, ah, bh, idesc, first);
                            }
                        }
                        if constexpr (PASSES == 3) {
#pragma unroll
                            for (int kk = 0; kk < BK / UMMA_K; ++kk) {
                                const uint32_t off = kk * UMMA_K * 4;
                                mma_tf32(tmem_d, sw128_desc(a0 + off), sw128_desc(b0 + off), idesc,
                                         1u);
                            }
                        }
                        issued = true;
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
            if constexpr (screen) {
                if (single.counts) {
                    atomicAdd(single.counts, computed);
                    atomicAdd(single.counts + 1, examined);
                }
            }
        }
    } else {
        // ------------------------------------------------ epilogue (warps 2 .. 9, 10 .. 13)
        const int ew = warp - 2;
        const int q = warp & 3;     // TMEM lane quarter this warp may read
        const uint32_t lane_base = tmem_base + ((uint32_t)(32 * q) << 16);
        float* xbuf = (float*)(smem + STAGES * C::STAGE_BYTES + C::BAR_BYTES) + (ew & 7) * kXposeWords;
        double dsum = 0.0;
        // each problem of a grouped launch has its own dot target: flush per tile
        auto flush_tile_dot = [&](double* dot) {
            if constexpr (GROUPED) {
                if (dot) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xffffffffu, dsum, o);
                    if (lane == 0 && dsum != 0.0) atomicAdd(dot, dsum);
                }
                dsum = 0.0;
            }
        };
        // computed k-slices of a tile, the same count as the MMA issuer's (from lane 0)
        auto active_of = [&](const TileRef& r) {
            int na = r.num_k;
            if constexpr (screen) {
                if (lane == 0) na = count_active(r);
                na = __shfl_sync(0xffffffffu, na, 0);
            }
            return na;
        };
        auto wait_bar = [&](uint64_t* bar, uint32_t parity, int code) {
            int w = 1;
            if (lane == 0) w = mbar_wait(bar, parity, abort_flag, err, code);
            return __shfl_sync(0xffffffffu, w, 0) != 0;
        };
        if constexpr (KCH > 0) {
            if (ew < 8) {
                // chunk warps, two per lane quarter, each with half of the columns: sum the
                // short TMEM partial sums of a tile in registers (IEEE round-to-nearest) and
                // park the finished sums in the sum buffer (TMEM columns NB BN ..)
                constexpr int HW = BN / 2;
                const int col0 = (ew >> 2) * HW;
                uint32_t g = 0, j = 0;
                for (int t = t_first; t < total_tiles; t += t_step) {
                    const TileRef r = tile(t);
                    if (r.skip) continue;
                    const int na = active_of(r);
                    if (screen && na == 0) {   // every slice screened out: no TMEM, no barrier
                        dsum += epi_fill_zero_tile<BN>(r.pr->p, r.m0, r.n0, r.diag, ew, 8, lane);
                        flush_tile_dot(r.pr->p.dot);
                        continue;
                    }
                    int kc = 0;
                    const int nch = chunks(na, &kc);
                    float acc[HW];
#pragma unroll
                    for (int i = 0; i < HW; ++i) acc[i] = 0.f;
                    bool ok = true;
                    for (int c = 0; c < nch; ++c, ++g) {
                        const int b = g % NB;
                        if (!wait_bar(&tfull[b], (g / NB) & 1, DEV_TIMEOUT_ACCUM)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
#pragma unroll
                        for (int c0 = 0; c0 < HW; c0 += 32) {
                            uint32_t rr[32];
                            tmem_ld32(lane_base + (uint32_t)(b * BN + col0 + c0), rr);
#pragma unroll
                            for (int i = 0; i < 32; ++i) acc[c0 + i] += __uint_as_float(rr[i]);
                        }
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&tempty[b]);
                    }
                    if (!ok) break;
                    // the store warps must have read the previous parked tile
                    if (!wait_bar(pfree, (j & 1) ^ 1, DEV_TIMEOUT_ACCUM)) break;
                    tc_fence_after();
#pragma unroll
                    for (int c0 = 0; c0 < HW; c0 += 32)
                        tmem_st32(lane_base + (uint32_t)(NB * BN + col0 + c0), acc + c0);
                    tmem_wait_st();
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(parked);
                    ++j;
                }
            } else {
                // store warps, one per lane quarter: the epilogue of each parked tile in
                // 32 x 32 blocks through the transpose buffer, then the sum buffer goes back
                uint32_t j = 0;
                for (int t = t_first; t < total_tiles; t += t_step) {
                    const TileRef r = tile(t);
                    if (r.skip) continue;
                    if (screen && active_of(r) == 0) continue;   // written by the chunk warps
                    const EpiParams<float> p = r.pr->p;
                    if (!wait_bar(parked, j & 1, DEV_TIMEOUT_ACCUM)) break;
                    tc_fence_after();
#pragma unroll 1
                    for (int c0 = 0; c0 < BN; c0 += 32) {
                        uint32_t rr[32];
                        tmem_ld32(lane_base + (uint32_t)(NB * BN + c0), rr);
                        float a[32];
#pragma unroll
                        for (int i = 0; i < 32; ++i) a[i] = __uint_as_float(rr[i]);
                        dsum += (double)epi_block32(p, r.m0 + 32 * q, r.n0 + c0, r.diag, a, xbuf,
                                                    lane);
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(pfree);
                    ++j;
                    flush_tile_dot(p.dot);
                }
            }
        } else {
            // the whole K in one accumulator: eight warps drain it, two per lane quarter,
            // each taking half of the columns
            const int h = ew >> 2;
            uint32_t g = 0;
            for (int t = t_first; t < total_tiles; t += t_step) {
                const TileRef r = tile(t);
                if (r.skip) continue;
                const EpiParams<float> p = r.pr->p;
                if (screen && active_of(r) == 0) {   // every slice screened out
                    dsum += epi_fill_zero_tile<BN>(p, r.m0, r.n0, r.diag, ew, 8, lane);
                    flush_tile_dot(p.dot);
                    continue;
                }
                const int b = g & 1;
                if (!wait_bar(&tfull[b], (g >> 1) & 1, DEV_TIMEOUT_ACCUM)) break;
                tc_fence_after();
#pragma unroll 1
                for (int c0 = h * (BN / 2); c0 < (h + 1) * (BN / 2); c0 += 32) {
                    uint32_t rr[32];
                    tmem_ld32(lane_base + (uint32_t)(b * BN + c0), rr);
                    float a[32];
#pragma unroll
                    for (int i = 0; i < 32; ++i) a[i] = __uint_as_float(rr[i]);
                    dsum += (double)epi_block32(p, r.m0 + 32 * q, r.n0 + c0, r.diag, a, xbuf, lane);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[b]);
                ++g;
                flush_tile_dot(p.dot);
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
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem_base, kTmemCols);
    }
}

template <int BN, int STAGES, int PASSES, int KCH, bool GROUPED, bool SCREEN = false>
cdmpt_status set_smem_attr() {
    using C = Cfg<BN, STAGES, PASSES>;
    static bool done = false;
    if (!done) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<BN, STAGES, PASSES, KCH, GROUPED, SCREEN>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (e != cudaSuccess) {
            set_error(std::string("tcgen05 GEMM smem attribute: ") + cudaGetErrorString(e));
            return CDMPT_ERR_CUDA;
        }
        done = true;
    }
    return CDMPT_OK;
}

template <int BN, int STAGES, int PASSES, int KCH, bool SCREEN = false>
cdmpt_status launch(int M, int N, int K, const float* X, const float* Xl, int ldx, const float* Y,
                    const float* Yl, int ldy, const EpiParams<float>& p, const double* skip,
                    cudaStream_t s, const GemmScreen* sc = nullptr) {
    using C = Cfg<BN, STAGES, PASSES>;
    static_assert(!SCREEN || BN == BM, "screened products use square tiles");
    if (SCREEN && !(sc && sc->mask)) {
        set_error("screened tcgen05 GEMM without a mask");
        return CDMPT_ERR_ARG;
    }
    {
        const cdmpt_status st = set_smem_attr<BN, STAGES, PASSES, KCH, false, SCREEN>();
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
    pr.mask = SCREEN ? sc->mask : nullptr;
    pr.nnt = SCREEN ? (N + BM - 1) / BM : 0;
    pr.nmw = SCREEN ? sc->nmw : 0;
    pr.counts = SCREEN ? sc->counts : nullptr;
    // symmetric results need square tiles: upper-triangular tiles only
    const bool sym = p.sym && BN == BM && M == N;
    pr.p.sym = sym ? 1 : 0;
    const int tiles = sym ? pr.num_mt * (pr.num_mt + 1) / 2 : pr.num_mt * ((N + BN - 1) / BN);
    const int grid = tiles < sm_count() ? tiles : sm_count();
    k_gemm_tc<BN, STAGES, PASSES, KCH, false, SCREEN><<<grid, tc_threads(KCH), C::SMEM, s>>>(
        mx, my, mxl, myl, pr, nullptr, 1, tiles, device_error_word());
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("tcgen05 GEMM launch: ") + cudaGetErrorString(e));
        return CDMPT_ERR_CUDA;
    }
    return CDMPT_OK;
}

// Kernel family for single (non-grouped) products with more than 128 rows: one SM per
// tile or the two-SM MMA (cta_group::2, 256 x 256 tiles; for split TF32 the wide kernel
// k_gemm_split2sm). Default: two-SM for both; CDMPT_TC_MODE=1sm|2sm forces one family.
bool use_2sm(bool /*three*/) {
    static int v = -2;
    if (v == -2) {
        const char* e = getenv("CDMPT_TC_MODE");
        v = !e ? -1 : (std::strcmp(e, "2sm") == 0 ? 1 : 0);
    }
    return v != 0;
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
    k_gemm_tc<BN, STAGES, PASSES, KCH, true><<<grid, tc_threads(KCH), C::SMEM, s>>>(
        dummy, dummy, dummy, dummy, none, problems, G, total_tiles, device_error_word());
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("grouped tcgen05 GEMM launch: ") + cudaGetErrorString(e));
        return CDMPT_ERR_CUDA;
    }
    return CDMPT_OK;
}

// One CTA waits, through the bounded wait of the tcgen05 kernels with a limit of limit_ns, on an
// mbarrier that nothing arrives on. No copy or MMA is in flight: the wait gives up, records
// DEV_TIMEOUT_FULL and the kernel returns.
__global__ void k_wait_probe(unsigned long long limit_ns, int* err) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        (void)mbar_wait(&bar, 0, (volatile int*)&abort_flag, err, DEV_TIMEOUT_FULL, limit_ns);
    __syncthreads();
}

}  // namespace

cdmpt_status bounded_wait_probe(double limit_ms, cudaStream_t s) {
    if (!(limit_ms > 0.0 && limit_ms <= 1000.0)) {
        set_error("bounded wait check: limit_ms must lie in (0, 1000]");
        return CDMPT_ERR_ARG;
    }
    k_wait_probe<<<1, 32, 0, s>>>((unsigned long long)(limit_ms * 1e6), device_error_word());
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("bounded wait check launch: ") + cudaGetErrorString(e));
        return CDMPT_ERR_CUDA;
    }
    return check_device_error(s);
}

int tc_tile_n(int engine) { return engine == CDMPT_GEMM_TC_TF32 ? 256 : 128; }
int tc_tile_m() { return BM; }

bool tc_encode_operand(CUtensorMap* map, const float* base, int rows, int cols, int ld,
                       bool as_y, int engine, int bn) {
    // as X: box of 128 rows (BM); as Y: box of BN rows (bn, else the engine's default)
    return make_map(map, base, rows, cols, ld, as_y ? (bn > 0 ? bn : tc_tile_n(engine)) : BM);
}

cdmpt_status gemm_tc_grouped(int engine, const GemmProblem* problems, int G, int total_tiles,
                             cudaStream_t s, int bn) {
    if (G <= 0 || total_tiles <= 0) return CDMPT_OK;
    if (!tc_supported()) {
        set_error("tcgen05 GEMM needs an sm_103 device");
        return CDMPT_ERR_UNSUPPORTED;
    }
    if (engine == CDMPT_GEMM_TC_TF32) {
        // one pass over the hi arrays; 128- and 64-column tiles share the tensor maps
        // of the split-TF32 engine with the same tile width (batched mixed precision)
        if (bn == 128 || bn == 256) return launch_grouped<128, 6, 1, 0>(problems, G, total_tiles, s);
        if (bn == 64) return launch_grouped<64, 8, 1, 0>(problems, G, total_tiles, s);
        return launch_grouped<256, 4, 1, 0>(problems, G, total_tiles, s);
    }
    if (bn == 256)   // the wide two-SM split kernel
        return gemm_split2sm_grouped(split_chunk(), problems, G, total_tiles, s);
    if (bn == 64)   // the same chunk as the 128-column kernel, so the same sums
        return split_chunk() == 2 ? launch_grouped<64, 4, 3, 2>(problems, G, total_tiles, s)
                                  : launch_grouped<64, 4, 3, 1>(problems, G, total_tiles, s);
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
                         const Epilogue<float>& ep, const double* skip, cudaStream_t s,
                         const GemmScreen* screen) {
    if (M <= 0 || N <= 0) return CDMPT_OK;
    if (!tc_supported()) {
        set_error("tcgen05 GEMM needs an sm_103 device");
        return CDMPT_ERR_UNSUPPORTED;
    }
    if (engine == CDMPT_GEMM_TC_BF16) {
        // operands rounded to BF16 in stream-ordered scratch (one copy when X is Y)
        if ((ldx & 7) || (ldy & 7) || !X.x || !Y.x || K < 1) {
            set_error("BF16 GEMM: X/Y needed, ld a multiple of 8, K >= 1");
            return CDMPT_ERR_ARG;
        }
        const bool same = X.x == Y.x && ldx == ldy && M == N;
        const size_t nx = (size_t)M * ldx, ny = same ? 0 : (size_t)N * ldy;
        void* buf = nullptr;
        if (cudaMallocAsync(&buf, (nx + ny) * 2 + 256, s) != cudaSuccess) {
            cudaGetLastError();
            set_error("BF16 GEMM: scratch allocation failed");
            return CDMPT_ERR_OOM;
        }
        char* xb = (char*)buf;
        char* yb = same ? xb : xb + ((nx * 2 + 255) & ~(size_t)255);
        cdmpt_status st = to_bf16(X.x, nx, xb, skip, s);
        if (st == CDMPT_OK && !same) st = to_bf16(Y.x, ny, yb, skip, s);
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
        p.sym = (ep.sym && M == N && ep.trans_block <= 0) ? 1 : 0;
        if (st == CDMPT_OK) st = gemm_tc_bf16(M, N, K, xb, ldx, yb, ldy, p, skip, s);
        cudaFreeAsync(buf, s);
        return st;
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
    p.sym = (ep.sym && M == N && ep.trans_block <= 0) ? 1 : 0;
    if (screen && screen->mask) {
        // screened: one-SM kernel with 128 x 128 tiles (the mask's granularity),
        // symmetric results on the upper triangle
        if (screen->nmw != ((K + BK - 1) / BK + 31) / 32) {
            set_error("screened tcgen05 GEMM: the mask does not match the product");
            return CDMPT_ERR_ARG;
        }
        if (!three)
            return launch<128, 6, 1, 0, true>(M, N, K, xh, xh, ldx, yh, yh, ldy, p, skip, s,
                                              screen);
        switch (split_chunk()) {
            case 1: return launch<128, 3, 3, 1, true>(M, N, K, xh, X.lo, ldx, yh, Y.lo, ldy, p, skip, s, screen);
            case 4: return launch<128, 3, 3, 4, true>(M, N, K, xh, X.lo, ldx, yh, Y.lo, ldy, p, skip, s, screen);
            case 0: return launch<128, 3, 3, 0, true>(M, N, K, xh, X.lo, ldx, yh, Y.lo, ldy, p, skip, s, screen);
            default: return launch<128, 3, 3, 2, true>(M, N, K, xh, X.lo, ldx, yh, Y.lo, ldy, p, skip, s, screen);
        }
    }
    if (p.sym) {
        // symmetric result: square tiles, upper triangle only (256 x 256 two-SM tiles; split
        // TF32 on one-SM 128 x 128 tiles when M <= 128 or the one-SM family is forced)
        if (!three)
            return gemm_tc_2sm(false, 0, M, N, K, xh, xh, ldx, yh, yh, ldy, p, skip, s);
        if (use_2sm(true) && M > BM)
            return gemm_tc_2sm(true, split_chunk(), M, N, K, xh, X.lo, ldx, yh, Y.lo, ldy, p,
                               skip, s);
        switch (split_chunk()) {
            case 1: return launch<128, 3, 3, 1>(M, N, K, xh, X.lo, ldx, yh, Y.lo, ldy, p, skip, s);
            case 4: return launch<128, 3, 3, 4>(M, N, K, xh, X.lo, ldx, yh, Y.lo, ldy, p, skip, s);
            case 0: return launch<128, 3, 3, 0>(M, N, K, xh, X.lo, ldx, yh, Y.lo, ldy, p, skip, s);
            default: return launch<128, 3, 3, 2>(M, N, K, xh, X.lo, ldx, yh, Y.lo, ldy, p, skip, s);
        }
    }
    if (use_2sm(three) && M > BM)
        return gemm_tc_2sm(three, split_chunk(), M, N, K, xh, three ? X.lo : xh, ldx, yh, three ? Y.lo : yh,
                           ldy, p, skip, s);
    if (!three) return launch<256, 4, 1, 0>(M, N, K, xh, xh, ldx, yh, yh, ldy, p, skip, s);
    switch (split_chunk()) {
        case 1: return launch<128, 3, 3, 1>(M, N, K, xh, X.lo, ldx, yh, Y.lo, ldy, p, skip, s);
        case 4: return launch<128, 3, 3, 4>(M, N, K, xh, X.lo, ldx, yh, Y.lo, ldy, p, skip, s);
        case 0: return launch<128, 3, 3, 0>(M, N, K, xh, X.lo, ldx, yh, Y.lo, ldy, p, skip, s);
        default: return launch<128, 3, 3, 2>(M, N, K, xh, X.lo, ldx, yh, Y.lo, ldy, p, skip, s);
    }
}

}  // namespace cdmpt
