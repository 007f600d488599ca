// Batched canonical solves: B Hamiltonians of uneven size N_b, each with D
// perturbation directions, advanced in lockstep (Algorithm 1 per system).
//
// Every product of a step is ONE grouped persistent tcgen05 launch over all
// systems (k_gemm_tc<..., GROUPED> walking a descriptor array of per-system
// problems), and every vector operation is one grouped elementwise launch.
// Each system keeps its own CG scalars, convergence flag and chemical
// potential on the device; a converged system is skipped through its flag
// (its GEMM tiles and elementwise blocks return at once). Storage is FP32 with
// split-TF32 (3xTF32) products, as in the single-system FP32 mode; with
// CDMPT_MIXED_TF32 the occupation sweeps use one-pass TF32 products and the
// trajectories are then refined (split-TF32 residuals, TF32 corrections,
// Newton steps on each system's mu), as in the single-system mixed mode.
//
// Tile autotuner: before the first product of a batch, each candidate tile
// width of the grouped kernel (128 and 64 columns, same accumulation chunk, so
// the same rounding) is timed on that product over all systems, which is
// idempotent (W_0 = Z_0 Z_0 and its split), and the fastest is kept for the
// batch's lifetime. CUDA graph: one CG iteration over all systems (grouped
// product, update, direction, scalar step) is captured once per launch shape
// from dedicated descriptor arrays and replayed for every iteration.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <cstdlib>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "cdmpt.h"
#include "batch_kernels.cuh"
#include "gemm_problem.cuh"
#include "internal.cuh"
#include "solver.cuh"

namespace cdmpt {

namespace {

constexpr int kEngine = CDMPT_GEMM_TC_3XTF32;
constexpr int kSlots = 64;

// When a system of a mixed-precision batch switches from split-TF32 refinement passes to
// passes with FP64-class late-step residuals: once its occupation error after a split pass
// is within this value times sqrt(N), so that the Newton steps on mu it still needs run on
// the cheaper split passes (default 1e-4; CDMPT_BATCH_HP_SWITCH overrides it, and a value of
// 0 or below switches every system right after its first split pass). On the 96-cluster
// workload, 1e-4 against switching at once: refinement 486 against 507 ms per batch.
double batch_hp_switch() {
    static double v = -2.0;
    if (v < -1.5) {
        const char* e = getenv("CDMPT_BATCH_HP_SWITCH");
        v = e ? atof(e) : 1e-4;
        if (!(v > 0)) v = -1.0;
    }
    return v;
}

struct Mat {   // FP32 matrix stack with TF32 split
    float* x = nullptr;
    float* hi = nullptr;
    float* lo = nullptr;
    float* xl = nullptr;   // mixed-precision trajectory: low FP32 part of a pair, value = x + xl
};

struct Sys {
    int N = 0, ld = 0;
    size_t blk = 0;
    double* H0 = nullptr;     // N x ld FP64
    double* H1 = nullptr;     // D x N x ld FP64
    std::vector<Mat> Z, W;
    Mat R, P, Q, S, A1, RHS, Z1a, Z1b, Qmu;
    double* sc = nullptr;     // kSlots doubles
    double gmin = 0, gmax = 0, trH0 = 0;
    // host-side state of the current solve
    double beta = 0, nocc = 0, s2 = 0, mu = 0, lo = 0, hi = 0;
    double e_lo = 0, e_hi = 0;   // occupation errors at lo and hi once a sweep set them
    bool converged = false;
    // mixed refinement: first step of the FP64-class residuals (n: none), whether this
    // system's passes form them yet, and how many such passes it has had
    int khp = 0;
    bool hp = false;
    int hp_passes = 0;
};

enum BSlot { B_TRZ = 8, B_ZZ = 9, B_TRQ = 10, B_TRZ1 = 16, B_ALPHA = 32 };

}  // namespace

}  // namespace cdmpt

using namespace cdmpt;

struct cdmpt_batch {
    cdmpt_opts opts;
    int B = 0, D = 0, n_alloc = -1;
    std::vector<Sys> sys;
    std::vector<void*> allocs;
    double* inactive = nullptr;   // device flag per system: 1 while skipped
    // tensor-map cache: (X hi, rows of X, Y hi) -> first of four maps in the device table
    std::map<std::tuple<const void*, int, const void*>, int> map_index;
    std::vector<CUtensorMap> maps_host;
    CUtensorMap* maps_dev = nullptr;
    int maps_uploaded = 0, maps_cap = 0;
    // staging ring for per-launch descriptor arrays
    char* stage_host = nullptr;
    char* stage_dev = nullptr;
    size_t stage_slot = 0, stage_slots = 0, slot_bytes = 0;
    double* pinned = nullptr;     // scalar readback, B x kSlots
    // tile autotuner: chosen tile width (0 = not tuned yet) and the timings
    int tile_bn = 0;
    double tune_ms[3] = {0.0, 0.0, 0.0};   // per launch, tile widths 128, 64 and 256
    // CUDA graph of one CG iteration: dedicated descriptors, graphs by shape
    GemmProblem* it_gemm = nullptr;   // B problems
    GrpEw* it_ew = nullptr;           // 3 B: update, direction, scalar step
    std::map<std::tuple<int, long long, int>, cudaGraphExec_t> it_graphs;   // (tiles, block, engine)
    bool graphs = true;
    // capture runs on a private stream (the caller's may be the legacy default
    // stream, which cannot be captured); replays go to the caller's stream
    cudaStream_t cap_stream = nullptr;
    Context cx;                   // stream, profile events, statistics hookup
    cdmpt_stats st;
    std::string err;
    bool have_H = false;
    // mixed precision: Ozaki digits of three operands (sized for the largest system) and the
    // low part of an Ozaki-formed W_k, one set per lane; the systems' FP64-class residuals run
    // on hp_nlanes side streams (at most kHpLanes; CDMPT_BATCH_HP_LANES, default 8: on the
    // 96-cluster workload the refinement took 617, 531 and 507 ms with 2, 4 and 8 lanes),
    // system i on lane i % hp_nlanes, so the small products of different systems share the
    // GPU (lane 0's set also serves the dP0/dmu right side)
    static constexpr int kHpLanes = 8;
    int hp_nlanes = 4;
    OzOperand oz[kHpLanes][3];
    float* oz_wl[kHpLanes] = {};
    cudaStream_t hp_st[kHpLanes] = {};
    cudaEvent_t hp_fork = nullptr;
    cudaEvent_t hp_join[kHpLanes] = {};
    int hp_lanes = 0;   // lanes forked by the last residual_batch_hp, not yet joined
};

namespace {

cdmpt_status bfail(cdmpt_batch* b, cdmpt_status s) {
    if (b) b->err = get_error();
    return s;
}

cdmpt_status bfail_msg(cdmpt_batch* b, cdmpt_status s, const std::string& m) {
    set_error(m);
    return bfail(b, s);
}

cdmpt_status grab(cdmpt_batch* b, size_t bytes, void** out) {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        set_error("batch: device allocation of " + std::to_string(bytes) + " bytes failed");
        return CDMPT_ERR_OOM;
    }
    if (cudaMemset(p, 0, bytes) != cudaSuccess) return CDMPT_ERR_CUDA;
    b->allocs.push_back(p);
    *out = p;
    return CDMPT_OK;
}

cdmpt_status grab_mat(cdmpt_batch* b, size_t elems, Mat* m, bool split) {
    CDMPT_TRY(grab(b, elems * sizeof(float), (void**)&m->x));
    if (split) {
        CDMPT_TRY(grab(b, elems * sizeof(float), (void**)&m->hi));
        CDMPT_TRY(grab(b, elems * sizeof(float), (void**)&m->lo));
    }
    return CDMPT_OK;
}

// Copies a descriptor array into the next staging slot; returns its device address.
template <typename T>
cdmpt_status stage(cdmpt_batch* b, const std::vector<T>& v, const T** dev) {
    const size_t bytes = v.size() * sizeof(T);
    if (bytes > b->slot_bytes) {
        set_error("batch: descriptor array exceeds the staging slot");
        return CDMPT_ERR_ARG;
    }
    if (b->stage_slot == b->stage_slots) {
        // every slot has been handed to the stream: wait before reusing them
        CDMPT_CUDA_TRY(cudaStreamSynchronize(b->cx.stream));
        b->stage_slot = 0;
    }
    char* h = b->stage_host + b->stage_slot * b->slot_bytes;
    char* d = b->stage_dev + b->stage_slot * b->slot_bytes;
    ++b->stage_slot;
    std::memcpy(h, v.data(), bytes);
    CDMPT_CUDA_TRY(cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, b->cx.stream));
    *dev = (const T*)d;
    return CDMPT_OK;
}

// Index of the first of four consecutive tensor maps (X hi, Y hi, X lo, Y lo)
// of one operand pair; encoded and uploaded on first use, never rewritten.
cdmpt_status quad_of(cdmpt_batch* b, const Mat* X, int rows, const Mat* Y, int N, int ld,
                     int* idx) {
    const auto key = std::make_tuple((const void*)X->hi, rows, (const void*)Y->hi);
    auto it = b->map_index.find(key);
    if (it != b->map_index.end()) {
        *idx = it->second;
        return CDMPT_OK;
    }
    if ((int)b->maps_host.size() + 4 > b->maps_cap) {
        set_error("batch: tensor-map table full");
        return CDMPT_ERR_OOM;
    }
    CUtensorMap m[4];
    // the wide two-SM kernel (tile width 256) loads boxes of 128 rows of both operands, as
    // does the one-pass 128-column kernel that shares these maps
    const int bn = b->tile_bn == 256 ? 128 : b->tile_bn;
    if (!tc_encode_operand(&m[0], X->hi, rows, N, ld, false, kEngine, bn) ||
        !tc_encode_operand(&m[1], Y->hi, N, N, ld, true, kEngine, bn) ||
        !tc_encode_operand(&m[2], X->lo, rows, N, ld, false, kEngine, bn) ||
        !tc_encode_operand(&m[3], Y->lo, N, N, ld, true, kEngine, bn)) {
        set_error("batch: tensor map encoding failed");
        return CDMPT_ERR_ARG;
    }
    *idx = (int)b->maps_host.size();
    for (int q = 0; q < 4; ++q) b->maps_host.push_back(m[q]);
    b->map_index[key] = *idx;
    return CDMPT_OK;
}

cdmpt_status flush_maps(cdmpt_batch* b) {
    const int n = (int)b->maps_host.size();
    if (n > b->maps_uploaded) {
        CDMPT_CUDA_TRY(cudaMemcpyAsync(b->maps_dev + b->maps_uploaded,
                                       b->maps_host.data() + b->maps_uploaded,
                                       (n - b->maps_uploaded) * sizeof(CUtensorMap),
                                       cudaMemcpyHostToDevice, b->cx.stream));
        // the host vector may reallocate later: wait for the copy before it can
        CDMPT_CUDA_TRY(cudaStreamSynchronize(b->cx.stream));
        b->maps_uploaded = n;
    }
    return CDMPT_OK;
}

// One problem of a grouped GEMM: D = alpha X Y^T + beta C + gamma I (rows x N_b, K = N_b).
void add_flops(cdmpt_batch* b, double f, int engine = kEngine) {
    if (b->cx.st) {
        b->cx.st->gemm_flops += f;
        b->cx.st->tensor_flops += (engine == CDMPT_GEMM_TC_3XTF32 ? 3.0 : 1.0) * f;
    }
}

// Flops of one symmetric N x N x N product: the upper-triangular tiles only
// when the grouped kernel's tiles are square (tile width 128 or 256), else all.
double sym_flops(const cdmpt_batch* b, int N) {
    const double n = N;
    return b->tile_bn != 64 ? n * (n + 1) * n : 2.0 * n * n * n;
}

struct GemmSpec {
    const Mat* X;
    int rows;
    const Mat* Y;
    EpiParams<float> p;
    const double* skip;
};

EpiParams<float> epi(float* D, int M, int N, int ld, float alpha = 1.f, float beta = 0.f,
                     const float* C = nullptr, float gamma = 0.f) {
    EpiParams<float> p;
    std::memset(&p, 0, sizeof(p));
    p.alpha = alpha;
    p.beta = beta;
    p.gamma = gamma;
    p.C = C;
    p.ldc = ld;
    p.D = D;
    p.ldd = ld;
    p.M = M;
    p.N = N;
    p.diag_block = N;
    p.lde = ld;
    return p;
}

// Problem descriptors of one grouped product (tensor maps resolved and uploaded). Tiles
// are 128 x tile_bn, except at tile width 256: 256 x 256 for split-TF32 products (the
// wide two-SM kernel) and 128 x 128 for one-pass TF32 products.
cdmpt_status prepare_grouped(cdmpt_batch* b, const std::vector<GemmSpec>& specs,
                             std::vector<GemmProblem>* probs, int* tiles_out,
                             int engine = kEngine) {
    std::vector<int> quad;
    probs->clear();
    probs->reserve(specs.size());
    int tiles = 0;
    int bm = tc_tile_m(), bn = b->tile_bn > 0 ? b->tile_bn : tc_tile_n(kEngine);
    if (bn == 256) {
        if (engine == kEngine)
            bm = 256;
        else
            bn = 128;
    }
    // tiles are numbered problem by problem and CTAs stride over them: the largest K
    // first, so that each stride takes tiles of about the same length and the last
    // ones to finish are the shortest (longest-processing-time order)
    std::vector<int> order(specs.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return specs[x].p.N > specs[y].p.N; });
    for (int oi : order) {
        const GemmSpec& g = specs[oi];
        const int N = g.p.N;
        int q = 0;
        CDMPT_TRY(quad_of(b, g.X, g.rows, g.Y, N, g.p.ldd, &q));
        GemmProblem pr;
        pr.p = g.p;
        pr.K = N;
        pr.tile_begin = tiles;
        pr.num_mt = (g.p.M + bm - 1) / bm;
        pr.skip = g.skip;
        pr.maps = nullptr;
        pr.mask = nullptr;   // grouped launches are never screened
        pr.nnt = pr.nmw = 0;
        pr.counts = nullptr;
        // symmetric results need square tiles: the upper triangle only
        pr.p.sym = (g.p.sym && bn == bm && g.p.M == N) ? 1 : 0;
        probs->push_back(pr);
        quad.push_back(q);
        tiles += pr.p.sym ? pr.num_mt * (pr.num_mt + 1) / 2 : pr.num_mt * ((N + bn - 1) / bn);
    }
    CDMPT_TRY(flush_maps(b));
    for (size_t i = 0; i < probs->size(); ++i) (*probs)[i].maps = b->maps_dev + quad[i];
    *tiles_out = tiles;
    return CDMPT_OK;
}

// engine: split TF32 (default) or one-pass TF32 (the occupation sweeps of mixed precision)
cdmpt_status grouped_gemm(cdmpt_batch* b, const std::vector<GemmSpec>& specs,
                          int engine = kEngine) {
    std::vector<GemmProblem> probs;
    int tiles = 0;
    CDMPT_TRY(prepare_grouped(b, specs, &probs, &tiles, engine));
    if (probs.empty()) return CDMPT_OK;
    const GemmProblem* dev = nullptr;
    CDMPT_TRY(stage(b, probs, &dev));
    if (b->cx.st) b->cx.st->gemm_launches += 1;
    return gemm_tc_grouped(engine, dev, (int)probs.size(), tiles, b->cx.stream, b->tile_bn);
}

void clear_maps(cdmpt_batch* b) {
    b->map_index.clear();
    b->maps_host.clear();
    b->maps_uploaded = 0;
}

// Times each candidate tile width on one grouped product (which must be
// idempotent) and keeps the fastest. CDMPT_BATCH_TILE=64|128 fixes the choice.
cdmpt_status tune_tiles(cdmpt_batch* b, const std::vector<GemmSpec>& specs) {
    const char* env = getenv("CDMPT_BATCH_TILE");
    if (env && (atoi(env) == 64 || atoi(env) == 128 || atoi(env) == 256)) {
        clear_maps(b);
        b->tile_bn = atoi(env);
        return CDMPT_OK;
    }
    const int cand[3] = {128, 64, 256};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CDMPT_CUDA_TRY(cudaEventCreate(&e0));
    CDMPT_CUDA_TRY(cudaEventCreate(&e1));
    cdmpt_stats* keep = b->cx.st;
    b->cx.st = nullptr;   // tuning launches are not part of the solve's statistics
    int best = 128;
    double best_ms = 1e300;
    cdmpt_status st = CDMPT_OK;
    for (int c = 0; c < 3 && st == CDMPT_OK; ++c) {
        clear_maps(b);
        b->tile_bn = cand[c];
        st = grouped_gemm(b, specs);   // warm-up (kernel attributes, maps)
        if (st != CDMPT_OK) break;
        cudaEventRecord(e0, b->cx.stream);
        for (int r = 0; r < 3 && st == CDMPT_OK; ++r) st = grouped_gemm(b, specs);
        cudaEventRecord(e1, b->cx.stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = CDMPT_ERR_CUDA;
        float ms = 0.f;
        if (st == CDMPT_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
            b->tune_ms[c] = ms / 3.0;
            if (ms / 3.0 < best_ms) {
                best_ms = ms / 3.0;
                best = cand[c];
            }
        }
    }
    b->cx.st = keep;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    clear_maps(b);
    b->tile_bn = best;
    if (st == CDMPT_OK) st = check_device_error(b->cx.stream);
    return st;
}

// Graph of one CG iteration over all systems for this launch shape (tiles of
// the grouped product, elements of the largest system's block); null when
// capture is unavailable (the caller then launches the kernels one by one).
cudaGraphExec_t iteration_graph(cdmpt_batch* b, int tiles, long long maxc, int engine) {
    const auto key = std::make_tuple(tiles, maxc, engine);
    auto it = b->it_graphs.find(key);
    if (it != b->it_graphs.end()) return it->second;
    if (!b->cap_stream &&
        cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        b->graphs = false;
        return nullptr;
    }
    cudaStream_t s = b->cap_stream;
    const int G = b->B;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        b->graphs = false;
        return nullptr;
    }
    cdmpt_status st = gemm_tc_grouped(engine, b->it_gemm, G, tiles, s, b->tile_bn);
    if (st == CDMPT_OK) st = grouped_ew(G_CG_UPDATE, b->it_ew, G, maxc, s);
    if (st == CDMPT_OK) st = grouped_ew(G_CG_DIR, b->it_ew + G, G, maxc, s);
    if (st == CDMPT_OK) st = grouped_cg_step(b->it_ew + 2 * G, G, s);
    count_launch(-4);   // captured, not run: replays are counted instead
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    cudaGraphExec_t exec = nullptr;
    if (st == CDMPT_OK && e == cudaSuccess && g) e = cudaGraphInstantiate(&exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (st != CDMPT_OK || e != cudaSuccess || !exec) {
        cudaGetLastError();
        b->graphs = false;
        return nullptr;
    }
    b->it_graphs[key] = exec;
    return exec;
}

void drop_graphs(cdmpt_batch* b) {
    for (auto& kv : b->it_graphs) cudaGraphExecDestroy(kv.second);
    b->it_graphs.clear();
}

}  // namespace

namespace {

GrpEw ewd(float* p0, float* p1 = nullptr, float* p2 = nullptr, float* p3 = nullptr) {
    GrpEw d;
    std::memset(&d, 0, sizeof(d));
    d.p0 = p0;
    d.p1 = p1;
    d.p2 = p2;
    d.p3 = p3;
    return d;
}

cdmpt_status run_ew(cdmpt_batch* b, int op, const std::vector<GrpEw>& d) {
    if (d.empty()) return CDMPT_OK;
    long long maxc = 0;
    for (const GrpEw& e : d) maxc = std::max(maxc, (long long)e.rows * e.ld);
    const GrpEw* dev = nullptr;
    CDMPT_TRY(stage(b, d, &dev));
    return grouped_ew(op, dev, (int)d.size(), maxc, b->cx.stream);
}

// Runs a tiled op (symmetrize / transpose-add / trace) over every system.
template <typename F>
cdmpt_status run_tiles(cdmpt_batch* b, const std::vector<GrpEw>& d, int blocks, F launch) {
    int maxN = 0;
    for (const GrpEw& e : d) maxN = std::max(maxN, e.N);
    const GrpEw* dev = nullptr;
    CDMPT_TRY(stage(b, d, &dev));
    return launch(dev, (int)d.size(), maxN, blocks, b->cx.stream);
}

double* scal_base(cdmpt_batch* b) { return b->sys[0].sc; }

cdmpt_status zero_slots(cdmpt_batch* b, int first, int count) {
    CDMPT_CUDA_TRY(cudaMemset2DAsync(scal_base(b) + first, kSlots * sizeof(double), 0,
                                     count * sizeof(double), b->B, b->cx.stream));
    return CDMPT_OK;
}

cdmpt_status read_all(cdmpt_batch* b) {
    CDMPT_CUDA_TRY(cudaMemcpyAsync(b->pinned, scal_base(b), (size_t)b->B * kSlots * sizeof(double),
                                   cudaMemcpyDeviceToHost, b->cx.stream));
    CDMPT_CUDA_TRY(cudaStreamSynchronize(b->cx.stream));
    return check_device_error(b->cx.stream);
}

// Per-system arguments of one grouped CG solve: X (s I + t W) = rhs_scale rhs.
struct BCg {
    float* X;
    const Mat* x0;        // warm start (scale 1) or null for zero
    const float* rhs;
    const Mat* W;
    int rows;
    // absolute tolerance on the scale of the updated quantity: stop also once
    // ||R|| <= tol_ref ref_scale ||ref|| (ref: rows x ld like X; null: none)
    const float* ref = nullptr;
    double ref_scale = 1.0;
};

// sym: every system's iterates are symmetric (0th-order solves), so the
// products run on upper-triangular tiles.
// init_engine (>= 0) computes the initial residual of warm-started systems with another
// engine than the iterations; tol_r0 > 0 also stops a system once ||R|| <= tol_r0 ||R_0||;
// rel0 (optional) receives the largest ||R_0|| / ||RHS|| over the systems.
cdmpt_status cg_batch(cdmpt_batch* b, const std::vector<BCg>& a, double s, double t, double tol,
                      const std::vector<const double*>& skip, int hint, int* iters,
                      bool sym = false, int engine = kEngine, int init_engine = -1,
                      double tol_r0 = 0.0, double* rel0 = nullptr, double tol_ref = 0.0,
                      bool* met_all = nullptr) {
    if (init_engine < 0) init_engine = engine;
    const int G = b->B;
    CDMPT_TRY(zero_slots(b, 0, CG_NSLOTS));
    bool use_ref = tol_ref > 0.0;
    for (const BCg& c : a) use_ref = use_ref && c.ref != nullptr;
    if (use_ref) {   // ||ref||^2 of every system into its reference slot
        CDMPT_TRY(zero_slots(b, kCgRefSlot, 1));
        std::vector<GrpEw> dref;
        for (int i = 0; i < G; ++i) {
            Sys& sy = b->sys[i];
            GrpEw q = ewd((float*)a[i].ref, (float*)a[i].ref);
            q.rows = a[i].rows; q.ld = sy.ld; q.N = sy.N;
            q.count = (long long)a[i].rows * sy.ld;
            q.sc = sy.sc;
            q.s0 = kCgRefSlot;
            q.skip = skip[i];
            dref.push_back(q);
        }
        CDMPT_TRY(run_ew(b, G_DOT, dref));
    }
    std::vector<GrpEw> dx, dr, drr, dbb, dp;
    std::vector<GemmSpec> g0;
    for (int i = 0; i < G; ++i) {
        Sys& sy = b->sys[i];
        const BCg& c = a[i];
        GrpEw e = ewd(c.X);
        e.rows = c.rows; e.ld = sy.ld; e.N = sy.N; e.count = (long long)c.rows * sy.ld;
        e.skip = skip[i];
        if (c.x0) {
            GrpEw x = e;                 // X = x0
            x.p1 = c.x0->x;
            x.s0 = 1.0;
            x.s1 = 0.0;
            dx.push_back(x);
            GrpEw r = e;                 // R = rhs - s x0
            r.p0 = sy.R.x;
            r.p1 = (float*)c.rhs;
            r.p2 = c.x0->x;
            r.s0 = 1.0;
            r.s1 = -s;
            dr.push_back(r);
            GemmSpec gs;                 // R += -t x0 W, <R,R>
            gs.X = c.x0;
            gs.rows = c.rows;
            gs.Y = c.W;
            gs.p = epi(sy.R.x, c.rows, sy.N, sy.ld, (float)-t, 1.f, sy.R.x);
            gs.p.sym = sym && c.rows == sy.N;
            gs.p.dot = sy.sc + CG_RR;
            gs.skip = skip[i];
            g0.push_back(gs);
        } else {
            GrpEw x = e;                 // X = 0
            dx.push_back(x);
            GrpEw r = e;                 // R = rhs
            r.p0 = sy.R.x;
            r.p1 = (float*)c.rhs;
            r.p2 = (float*)c.rhs;
            r.s0 = 1.0;
            r.s1 = 0.0;
            dr.push_back(r);
            GrpEw q = e;                 // <R,R>
            q.p0 = sy.R.x;
            q.p1 = sy.R.x;
            q.sc = sy.sc;
            q.s0 = CG_RR;
            drr.push_back(q);
        }
        GrpEw bb = e;
        bb.p0 = (float*)c.rhs;
        bb.p1 = (float*)c.rhs;
        bb.sc = sy.sc;
        bb.s0 = CG_BB;
        dbb.push_back(bb);
        GrpEw p = e;                     // P = R (split), unless done
        p.p0 = sy.P.x;
        p.p1 = sy.R.x;
        p.p2 = sy.P.hi;
        p.p3 = sy.P.lo;
        p.s0 = 1.0;
        p.s1 = 0.0;
        p.sc = sy.sc;
        dp.push_back(p);
    }
    if (!g0.empty()) {
        CDMPT_TRY(run_ew(b, G_AXPBY, dx));
        CDMPT_TRY(run_ew(b, G_LINCOMB, dr));
        CDMPT_TRY(grouped_gemm(b, g0, init_engine));
    } else {
        CDMPT_TRY(run_ew(b, G_ZERO, dx));
        CDMPT_TRY(run_ew(b, G_LINCOMB, dr));
        CDMPT_TRY(run_ew(b, G_DOT, drr));
    }
    CDMPT_TRY(run_ew(b, G_DOT, dbb));
    {
        std::vector<GrpEw> di(G);
        for (int i = 0; i < G; ++i) {
            di[i] = ewd(nullptr);
            di[i].sc = b->sys[i].sc;
            di[i].s0 = tol * tol;
            di[i].s1 = tol_r0 * tol_r0;
            di[i].s2 = use_ref ? tol_ref * tol_ref * a[i].ref_scale * a[i].ref_scale : 0.0;
            di[i].skip = skip[i];
        }
        const GrpEw* dev = nullptr;
        CDMPT_TRY(stage(b, di, &dev));
        CDMPT_TRY(grouped_cg_init(dev, G, b->cx.stream));
    }
    for (GrpEw& e : dp) e.skip = e.sc + CG_DONE;
    CDMPT_TRY(run_ew(b, G_AXPBY, dp));

    // iteration descriptors (constant over iterations)
    std::vector<GemmSpec> gi;
    std::vector<GrpEw> du, dd, ds;
    for (int i = 0; i < G; ++i) {
        Sys& sy = b->sys[i];
        const BCg& c = a[i];
        GemmSpec gs;
        gs.X = &sy.P;
        gs.rows = c.rows;
        gs.Y = c.W;
        gs.p = epi(sy.Q.x, c.rows, sy.N, sy.ld, (float)t, (float)s, sy.P.x);
        gs.p.sym = sym && c.rows == sy.N;
        gs.p.dot = sy.sc + CG_PQ;
        gs.p.E = sy.P.x;
        gs.skip = sy.sc + CG_DONE;
        gi.push_back(gs);
        GrpEw u = ewd(c.X, sy.R.x, sy.P.x, sy.Q.x);
        u.rows = c.rows; u.ld = sy.ld; u.N = sy.N; u.count = (long long)c.rows * sy.ld;
        u.sc = sy.sc;
        du.push_back(u);
        GrpEw dv = ewd(sy.P.x, sy.R.x, sy.P.hi, sy.P.lo);
        dv.rows = c.rows; dv.ld = sy.ld; dv.N = sy.N; dv.count = (long long)c.rows * sy.ld;
        dv.sc = sy.sc;
        dd.push_back(dv);
        GrpEw st = ewd(nullptr);
        st.sc = sy.sc;
        ds.push_back(st);
    }
    // the iteration as a CUDA graph: descriptors into the dedicated arrays
    cudaGraphExec_t graph = nullptr;
    if (b->graphs) {
        std::vector<GemmProblem> probs;
        int tiles = 0;
        CDMPT_TRY(prepare_grouped(b, gi, &probs, &tiles, engine));
        long long maxc = 0;
        for (const GrpEw& e : du) maxc = std::max(maxc, (long long)e.rows * e.ld);
        std::vector<GrpEw> ew(du);
        ew.insert(ew.end(), dd.begin(), dd.end());
        ew.insert(ew.end(), ds.begin(), ds.end());
        CDMPT_CUDA_TRY(cudaMemcpyAsync(b->it_gemm, probs.data(), probs.size() * sizeof(GemmProblem),
                                       cudaMemcpyHostToDevice, b->cx.stream));
        CDMPT_CUDA_TRY(cudaMemcpyAsync(b->it_ew, ew.data(), ew.size() * sizeof(GrpEw),
                                       cudaMemcpyHostToDevice, b->cx.stream));
        graph = iteration_graph(b, tiles, maxc, engine);
    }
    int chunk = std::max(1, hint), done_iters = 0;
    while (true) {
        for (int c = 0; c < chunk; ++c) {
            if (graph) {
                CDMPT_CUDA_TRY(cudaGraphLaunch(graph, b->cx.stream));
                count_launch(4);
                if (b->cx.st) b->cx.st->gemm_launches += 1;
                continue;
            }
            CDMPT_TRY(grouped_gemm(b, gi, engine));
            CDMPT_TRY(run_ew(b, G_CG_UPDATE, du));
            CDMPT_TRY(run_ew(b, G_CG_DIR, dd));
            const GrpEw* dev = nullptr;
            CDMPT_TRY(stage(b, ds, &dev));
            CDMPT_TRY(grouped_cg_step(dev, G, b->cx.stream));
        }
        done_iters += chunk;
        CDMPT_TRY(read_all(b));
        bool all = true;
        int most = 0;
        for (int i = 0; i < G; ++i) {
            all = all && b->pinned[i * kSlots + CG_DONE] != 0.0;
            most = std::max(most, (int)b->pinned[i * kSlots + CG_ITERS]);
        }
        if (all) {
            *iters = most;
            double worst = 0.0;
            for (int i = 0; i < G; ++i) {
                const Sys& sy = b->sys[i];
                const double f = (sym && a[i].rows == sy.N) ? sym_flops(b, sy.N)
                                                             : 2.0 * a[i].rows * (double)sy.N * sy.N;
                add_flops(b, f * b->pinned[i * kSlots + CG_ITERS], engine);
                if (a[i].x0 && !(skip[i] && b->sys[i].converged)) add_flops(b, f, init_engine);
                const double bb = b->pinned[i * kSlots + CG_BB];
                if (bb > 0) worst = std::max(worst, std::sqrt(b->pinned[i * kSlots + CG_RR0] / bb));
            }
            if (rel0) *rel0 = worst;
            if (met_all) {
                // every system's final residual meets the solve's own tolerance (relative to
                // its right side or the absolute reference), not only the tol_r0 reduction
                bool met = true;
                for (int i = 0; i < G; ++i) {
                    if (skip[i] && b->sys[i].converged) continue;   // skipped system
                    const double* q = b->pinned + (size_t)i * kSlots;
                    double lim = tol * tol * q[CG_BB];
                    if (use_ref)
                        lim = std::max(lim, tol_ref * tol_ref * a[i].ref_scale * a[i].ref_scale *
                                                q[kCgRefSlot]);
                    met = met && q[CG_RR] <= lim;
                }
                *met_all = met;
            }
            return CDMPT_OK;
        }
        if (done_iters >= b->opts.cg_maxit) {
            set_error("batch: CG did not converge in " + std::to_string(b->opts.cg_maxit) +
                      " iterations");
            return CDMPT_ERR_CG_MAXITER;
        }
        chunk = 2;
    }
}

// Z_0 = -s2 (H0 - mu I) of every active system (pair-stored in mixed precision).
cdmpt_status init_z0_batch(cdmpt_batch* b, const std::vector<const double*>& skip,
                           const std::vector<char>* only = nullptr) {
    std::vector<GrpEw> d, dp;
    for (int i = 0; i < b->B; ++i) {
        if (only && !(*only)[i]) continue;
        Sys& sy = b->sys[i];
        GrpEw e = sy.Z[0].xl ? ewd(sy.Z[0].x, sy.Z[0].xl, sy.Z[0].hi, sy.Z[0].lo)
                             : ewd(sy.Z[0].x, nullptr, sy.Z[0].hi, sy.Z[0].lo);
        e.h = sy.H0;
        e.rows = sy.N; e.ld = sy.ld; e.N = sy.N;
        e.s0 = -sy.s2;
        e.s1 = sy.mu;
        e.skip = skip[i];
        (sy.Z[0].xl ? dp : d).push_back(e);
    }
    CDMPT_TRY(run_ew(b, G_INIT_Z, d));
    return run_ew(b, G_PAIR_INIT, dp);
}

// One 0th-order pass for the systems whose inactive flag is 0, with products on
// engine and CG to relative residual tol.
cdmpt_status sweep_batch(cdmpt_batch* b, int n, int* iters_out, int engine, double tol) {
    const int G = b->B;
    std::vector<const double*> skip(G);
    for (int i = 0; i < G; ++i) skip[i] = b->inactive + i;
    CDMPT_TRY(init_z0_batch(b, skip));
    int total = 0, hint = 1;
    for (int k = 0; k < n; ++k) {
        std::vector<GemmSpec> gw, gr;
        std::vector<BCg> cg(G);
        std::vector<GrpEw> dz, dsym, dzl;
        for (int i = 0; i < G; ++i) {
            Sys& sy = b->sys[i];
            GemmSpec w;                  // W_k = Z_k Z_k
            w.X = &sy.Z[k];
            w.rows = sy.N;
            w.Y = &sy.Z[k];
            w.p = epi(sy.W[k].x, sy.N, sy.N, sy.ld);
            w.p.sym = 1;
            w.p.Dhi = sy.W[k].hi;
            w.p.Dlo = sy.W[k].lo;
            w.skip = skip[i];
            gw.push_back(w);
            GemmSpec r;                  // RHS = -2 Z_k W_k
            r.X = &sy.Z[k];
            r.rows = sy.N;
            r.Y = &sy.W[k];
            r.p = epi(sy.RHS.x, sy.N, sy.N, sy.ld, -2.f);
            r.p.sym = 1;
            r.skip = skip[i];
            gr.push_back(r);
            cg[i] = BCg{sy.Z[k + 1].x, nullptr, sy.RHS.x, &sy.W[k], sy.N};
            cg[i].ref = sy.Z[k].x;     // accurate sweeps: also relative to 2 Z_k (as cdmpt_solve)
            cg[i].ref_scale = 2.0;
            GrpEw z = ewd(sy.Z[k + 1].x, sy.Z[k].x);   // Z_{k+1} = 2 Z_k + d
            z.rows = sy.N; z.ld = sy.ld; z.N = sy.N; z.count = (long long)sy.N * sy.ld;
            z.s0 = 2.0;
            z.s1 = 1.0;
            z.skip = skip[i];
            dz.push_back(z);
            GrpEw y = ewd(sy.Z[k + 1].x, nullptr, sy.Z[k + 1].hi, sy.Z[k + 1].lo);
            y.rows = sy.N; y.ld = sy.ld; y.N = sy.N;
            y.skip = skip[i];
            dsym.push_back(y);
            if (sy.Z[k + 1].xl) {   // a sweep step leaves an FP32 iterate: zero low part
                GrpEw zl = ewd(sy.Z[k + 1].xl);
                zl.rows = sy.N; zl.ld = sy.ld; zl.N = sy.N; zl.count = (long long)sy.blk;
                zl.skip = skip[i];
                dzl.push_back(zl);
            }
        }
        if (b->tile_bn == 0) CDMPT_TRY(tune_tiles(b, gw));   // first product of the batch
        CDMPT_TRY(grouped_gemm(b, gw, engine));
        CDMPT_TRY(grouped_gemm(b, gr, engine));
        for (int i = 0; i < G; ++i)
            if (!b->sys[i].converged) add_flops(b, 2.0 * sym_flops(b, b->sys[i].N), engine);
        int it = 0;
        // mirrored CG products only in the one-pass sweeps of mixed precision (refined later);
        // the accurate sweeps (tol <= 1e-6) also stop relative to the new iterate
        CDMPT_TRY(cg_batch(b, cg, 1.0, 1.0, tol, skip, hint, &it, engine != kEngine, engine, -1,
                           0.0, nullptr, tol <= 1e-6 ? tol : 0.0));
        total += it;
        hint = std::max(1, it);
        CDMPT_TRY(run_ew(b, G_AXPBY, dz));
        CDMPT_TRY(run_tiles(b, dsym, 1, grouped_symmetrize));
        CDMPT_TRY(run_ew(b, G_ZERO, dzl));
    }
    *iters_out = total;
    return CDMPT_OK;
}

// The batch's stream continues after the lanes forked by residual_batch_hp.
cdmpt_status hp_join_lanes(cdmpt_batch* b) {
    cudaStream_t s = b->cx.stream;
    for (int l = 0; l < b->hp_lanes; ++l) {
        CDMPT_CUDA_TRY(cudaEventRecord(b->hp_join[l], b->hp_st[l]));
        CDMPT_CUDA_TRY(cudaStreamWaitEvent(s, b->hp_join[l], 0));
    }
    b->hp_lanes = 0;
    return CDMPT_OK;
}

// W_k and the residual 2 Z_k - Z_{k+1} - Z_{k+1} W_k of step k from Ozaki-sliced products of
// the pair-stored trajectory, for every active system one after another (they share the
// digit buffers); W_k's FP32 part and split replace the stored W_k, the residual goes to RHS.
// The work goes to side lanes forked from the batch's stream; join: the batch's stream waits
// for them before returning (else hp_join_lanes does, after more work on the batch's stream).
cdmpt_status residual_batch_hp(cdmpt_batch* b, int k, const std::vector<char>& active,
                               bool join = true) {
    cudaStream_t s = b->cx.stream;
    int nact = 0;
    for (int i = 0; i < b->B; ++i) nact += active[i] ? 1 : 0;
    if (nact == 0) return CDMPT_OK;
    const int L = std::min(nact, b->hp_nlanes);
    if (!b->hp_fork) {
        CDMPT_CUDA_TRY(cudaEventCreateWithFlags(&b->hp_fork, cudaEventDisableTiming));
        for (int l = 0; l < cdmpt_batch::kHpLanes; ++l) {
            CDMPT_CUDA_TRY(cudaStreamCreateWithFlags(&b->hp_st[l], cudaStreamNonBlocking));
            CDMPT_CUDA_TRY(cudaEventCreateWithFlags(&b->hp_join[l], cudaEventDisableTiming));
        }
    }
    // the lanes start after everything queued on the batch's stream
    CDMPT_CUDA_TRY(cudaEventRecord(b->hp_fork, s));
    for (int l = 0; l < L; ++l) CDMPT_CUDA_TRY(cudaStreamWaitEvent(b->hp_st[l], b->hp_fork, 0));
    int j = 0;
    for (int i = 0; i < b->B; ++i) {
        if (!active[i]) continue;
        const int l = j++ % L;
        cudaStream_t ls = b->hp_st[l];
        OzOperand* oz = b->oz[l];
        float* wl = b->oz_wl[l];
        Sys& sy = b->sys[i];
        for (int a = 0; a < 3; ++a) oz[a].ld = sy.ld;
        CDMPT_TRY(oz_slice(sy.Z[k].x, sy.Z[k].xl, sy.N, sy.N, sy.ld, oz[0], ls));
        OzEpi w;
        w.sym = 1;   // W_k = Z_k Z_k: upper-triangle tiles, mirrored
        w.D = sy.W[k].x;
        w.Dl = wl;
        w.Dthi = sy.W[k].hi;
        w.Dtlo = sy.W[k].lo;
        w.ldd = sy.ld;
        CDMPT_TRY(gemm_oz(sy.N, sy.N, sy.N, oz[0], oz[0], w, ls));
        CDMPT_TRY(oz_slice(sy.W[k].x, wl, sy.N, sy.N, sy.ld, oz[1], ls));
        CDMPT_TRY(oz_slice(sy.Z[k + 1].x, sy.Z[k + 1].xl, sy.N, sy.N, sy.ld, oz[2], ls));
        OzEpi r;
        r.D = sy.RHS.x;
        r.ldd = sy.ld;
        r.alpha = -1.f;
        r.b1 = 2.f;
        r.c1h = sy.Z[k].x;
        r.c1l = sy.Z[k].xl;
        r.b2 = -1.f;
        r.c2h = sy.Z[k + 1].x;
        r.c2l = sy.Z[k + 1].xl;
        r.ldc = sy.ld;
        CDMPT_TRY(gemm_oz(sy.N, sy.N, sy.N, oz[2], oz[1], r, ls));
        if (b->cx.st) {
            const double f = 2.0 * sy.N * (double)sy.N * sy.N;
            b->cx.st->gemm_launches += 2;
            b->cx.st->gemm_flops += 2.0 * f;
            b->cx.st->tensor_flops += 2.0 * oz_products(kOzDigits) * f;
        }
    }
    b->hp_lanes = L;
    return join ? hp_join_lanes(b) : CDMPT_OK;
}

// One refinement pass of the stored trajectories (mixed precision), for the systems whose
// inactive flag is 0 (active[i] on the host): per step, W_k = Z_k Z_k and the residual
// 2 Z_k - Z_{k+1} - Z_{k+1} W_k, then the correction d (I + W_k) = residual by CG with
// one-pass TF32 products (relative residual 1e-3), Z_{k+1} += d added to the pair,
// symmetrised. A system's steps form W_k and the residual with grouped split-TF32 products
// (full tiles for the residual: the stored Z_{k+1} does not commute with W_k to first order
// in its error), except, once the system is in its FP64-class passes (Sys::hp), the steps
// k >= Sys::khp, which use Ozaki-sliced products.
cdmpt_status refine_batch(cdmpt_batch* b, int n, const std::vector<char>& active,
                          int* iters_out) {
    const int G = b->B;
    std::vector<const double*> skip(G);
    for (int i = 0; i < G; ++i) skip[i] = b->inactive + i;
    int total = 0;
    for (int k = 0; k < n; ++k) {
        std::vector<GemmSpec> gw, gr;
        std::vector<BCg> cg(G);
        std::vector<GrpEw> ds, dz, dsym;
        std::vector<char> act_hp(G, 0), act_split(G, 0);
        bool any_hp = false, any_split = false;
        for (int i = 0; i < G; ++i) {
            const bool hp = b->sys[i].hp && k >= b->sys[i].khp;
            act_hp[i] = active[i] && hp;
            act_split[i] = active[i] && !hp;
            any_hp = any_hp || act_hp[i];
            any_split = any_split || act_split[i];
        }
        for (int i = 0; i < G; ++i) {
            Sys& sy = b->sys[i];
            cg[i] = BCg{sy.A1.x, nullptr, sy.RHS.x, &sy.W[k], sy.N};
            GrpEw z = ewd(sy.Z[k + 1].x, sy.Z[k + 1].xl, sy.A1.x);   // Z_{k+1} += d, to the pair
            z.rows = sy.N; z.ld = sy.ld; z.N = sy.N; z.count = (long long)sy.N * sy.ld;
            z.skip = skip[i];
            dz.push_back(z);
            GrpEw y = ewd(sy.Z[k + 1].x, sy.Z[k + 1].xl, sy.Z[k + 1].hi, sy.Z[k + 1].lo);
            y.rows = sy.N; y.ld = sy.ld; y.N = sy.N;
            y.skip = skip[i];
            dsym.push_back(y);
            if (!act_split[i]) continue;
            GemmSpec w;                  // W_k = Z_k Z_k, split-TF32
            w.X = &sy.Z[k];
            w.rows = sy.N;
            w.Y = &sy.Z[k];
            w.p = epi(sy.W[k].x, sy.N, sy.N, sy.ld);
            w.p.sym = 1;
            w.p.Dhi = sy.W[k].hi;
            w.p.Dlo = sy.W[k].lo;
            w.skip = skip[i];
            gw.push_back(w);
            // S = 2 Z_k - Z_{k+1} from the pairs
            GrpEw e = ewd(sy.S.x, sy.Z[k].x, sy.Z[k].xl, sy.Z[k + 1].x);
            e.p4 = sy.Z[k + 1].xl;
            e.rows = sy.N; e.ld = sy.ld; e.N = sy.N; e.count = (long long)sy.N * sy.ld;
            e.s0 = 2.0;
            e.s1 = -1.0;
            e.skip = skip[i];
            ds.push_back(e);
            GemmSpec r;                  // RHS = S - Z_{k+1} W_k, full tiles
            r.X = &sy.Z[k + 1];
            r.rows = sy.N;
            r.Y = &sy.W[k];
            r.p = epi(sy.RHS.x, sy.N, sy.N, sy.ld, -1.f, 1.f, sy.S.x);
            r.skip = skip[i];
            gr.push_back(r);
        }
        // the FP64-class residuals run on side lanes while the split products of the other
        // systems run on the batch's stream
        if (any_hp) CDMPT_TRY(residual_batch_hp(b, k, act_hp, false));
        if (any_split) {
            CDMPT_TRY(grouped_gemm(b, gw));
            CDMPT_TRY(run_ew(b, G_PAIR_LINCOMB, ds));
            CDMPT_TRY(grouped_gemm(b, gr));
            for (int i = 0; i < G; ++i) {
                if (!act_split[i]) continue;
                const double nn = b->sys[i].N;
                add_flops(b, sym_flops(b, b->sys[i].N) + 2.0 * nn * nn * nn);
            }
        }
        CDMPT_TRY(hp_join_lanes(b));
        int it = 0;
        CDMPT_TRY(cg_batch(b, cg, 1.0, 1.0, 1e-3, skip, 2, &it, false, CDMPT_GEMM_TC_TF32));
        total += it;
        CDMPT_TRY(run_ew(b, G_PAIR_ADD, dz));
        CDMPT_TRY(run_tiles(b, dsym, 1, grouped_pair_symmetrize));
    }
    *iters_out = total;
    return CDMPT_OK;
}

// Tr P0 and ||Z_n||_F^2 of every active system into its scalar slots (host copy in pinned).
cdmpt_status occupations(cdmpt_batch* b, int n) {
    const int G = b->B;
    CDMPT_TRY(zero_slots(b, B_TRZ, 2));
    std::vector<GrpEw> dt, dd;
    for (int i = 0; i < G; ++i) {
        Sys& sy = b->sys[i];
        GrpEw e = ewd(sy.Z[n].x, sy.Z[n].x);
        e.rows = sy.N; e.ld = sy.ld; e.N = sy.N; e.count = (long long)sy.blk;
        e.sc = sy.sc;
        e.skip = b->inactive + i;
        e.s0 = B_TRZ;
        dt.push_back(e);
        if (sy.Z[n].xl) {   // Tr of the pair's low part into the same slot
            GrpEw l = e;
            l.p0 = sy.Z[n].xl;
            dt.push_back(l);
        }
        e.s0 = B_ZZ;
        dd.push_back(e);
    }
    CDMPT_TRY(run_tiles(b, dt, 1, grouped_trace));
    CDMPT_TRY(run_ew(b, G_DOT, dd));
    return read_all(b);
}

cdmpt_status alloc_batch(cdmpt_batch* b, int n) {
    if (b->n_alloc >= n) return CDMPT_OK;
    drop_graphs(b);
    for (void* p : b->allocs) cudaFree(p);
    b->allocs.clear();
    b->map_index.clear();
    b->maps_host.clear();
    b->maps_uploaded = 0;
    const int B = b->B, D = b->D;
    double* scal = nullptr;
    CDMPT_TRY(grab(b, (size_t)B * kSlots * sizeof(double), (void**)&scal));
    CDMPT_TRY(grab(b, (size_t)B * sizeof(double), (void**)&b->inactive));
    b->maps_cap = B * (8 * n + 16) * 4;
    CDMPT_TRY(grab(b, (size_t)b->maps_cap * sizeof(CUtensorMap), (void**)&b->maps_dev));
    CDMPT_TRY(grab(b, (size_t)B * sizeof(GemmProblem), (void**)&b->it_gemm));
    CDMPT_TRY(grab(b, (size_t)3 * B * sizeof(GrpEw), (void**)&b->it_ew));
    b->maps_host.reserve(b->maps_cap);
    for (int i = 0; i < B; ++i) {
        Sys& sy = b->sys[i];
        sy.sc = scal + (size_t)i * kSlots;
        const size_t blk = sy.blk;
        const size_t big = (size_t)std::max(1, D) * blk;
        CDMPT_TRY(grab(b, blk * sizeof(double), (void**)&sy.H0));
        if (D > 0) CDMPT_TRY(grab(b, D * blk * sizeof(double), (void**)&sy.H1));
        sy.Z.assign(n + 1, Mat());
        sy.W.assign(n, Mat());
        for (int k = 0; k <= n; ++k) {
            CDMPT_TRY(grab_mat(b, blk, &sy.Z[k], true));
            if (b->opts.precision == CDMPT_MIXED_TF32)
                CDMPT_TRY(grab(b, blk * sizeof(float), (void**)&sy.Z[k].xl));
        }
        for (int k = 0; k < n; ++k) CDMPT_TRY(grab_mat(b, blk, &sy.W[k], true));
        CDMPT_TRY(grab_mat(b, big, &sy.R, false));
        CDMPT_TRY(grab_mat(b, big, &sy.P, true));
        CDMPT_TRY(grab_mat(b, big, &sy.Q, false));
        CDMPT_TRY(grab_mat(b, big, &sy.S, false));
        CDMPT_TRY(grab_mat(b, big, &sy.A1, true));
        CDMPT_TRY(grab_mat(b, big, &sy.RHS, true));
        CDMPT_TRY(grab_mat(b, big, &sy.Z1a, true));
        CDMPT_TRY(grab_mat(b, big, &sy.Z1b, true));
        CDMPT_TRY(grab_mat(b, blk, &sy.Qmu, false));
    }
    if (b->opts.precision == CDMPT_MIXED_TF32) {
        size_t mblk = 0;
        int mN = 0;
        for (const Sys& sy : b->sys) {
            mblk = std::max(mblk, sy.blk);
            mN = std::max(mN, sy.N);
        }
        const char* env = getenv("CDMPT_BATCH_HP_LANES");
        b->hp_nlanes = env ? std::min(std::max(atoi(env), 1), (int)cdmpt_batch::kHpLanes) : 8;
        for (int l = 0; l < b->hp_nlanes; ++l) {
            CDMPT_TRY(grab(b, mblk * sizeof(float), (void**)&b->oz_wl[l]));
            for (auto& o : b->oz[l]) {
                for (int d = 0; d < kOzDigits; ++d) CDMPT_TRY(grab(b, mblk * 2, &o.s[d]));
                CDMPT_TRY(grab(b, (size_t)mN * sizeof(int), (void**)&o.e));
            }
        }
    }
    b->n_alloc = n;
    b->have_H = false;
    return CDMPT_OK;
}

}  // namespace

extern "C" {

cdmpt_status cdmpt_batch_create(const cdmpt_opts* opts, int B, const int* N, int D,
                                cdmpt_batch** out) {
    if (!out || B < 1 || !N || D < 0 || D > 16) return CDMPT_ERR_ARG;
    *out = nullptr;
    for (int i = 0; i < B; ++i)
        if (N[i] < 1) return CDMPT_ERR_ARG;
    cdmpt_batch* b = new (std::nothrow) cdmpt_batch();
    if (!b) return CDMPT_ERR_OOM;
    if (opts)
        b->opts = *opts;
    else
        cdmpt_default_opts(&b->opts);
    if (!(b->opts.cg_tol > 0)) b->opts.cg_tol = 1e-7;
    if (b->opts.precision != CDMPT_FP32 && b->opts.precision != CDMPT_MIXED_TF32) {
        delete b;
        set_error("batch: CDMPT_FP32 (split-TF32 products) or CDMPT_MIXED_TF32 only");
        return CDMPT_ERR_UNSUPPORTED;
    }
    if (b->opts.fd_exact || b->opts.grand_canonical || b->opts.screen_tau != 0.0) {
        delete b;
        set_error("batch: canonical dense solves from the linear start of Eq. Rec_F_2 only "
                  "(no fd_exact, grand_canonical or screen_tau)");
        return CDMPT_ERR_UNSUPPORTED;
    }
    if (!tc_supported()) {
        delete b;
        set_error("batch: needs an sm_103 GPU (tcgen05)");
        return CDMPT_ERR_UNSUPPORTED;
    }
    std::memset(&b->st, 0, sizeof(b->st));
    {
        const char* g = getenv("CDMPT_BATCH_GRAPH");
        b->graphs = !(g && g[0] == '0');
    }
    b->B = B;
    b->D = D;
    b->sys.resize(B);
    for (int i = 0; i < B; ++i) {
        b->sys[i].N = N[i];
        b->sys[i].ld = (N[i] + 31) / 32 * 32;
        b->sys[i].blk = (size_t)N[i] * b->sys[i].ld;
    }
    b->cx.stream = (cudaStream_t)b->opts.stream;
    b->cx.profile = b->opts.profile != 0;   // phase boundaries of the solve (statistics)
    b->slot_bytes = std::max<size_t>(64 * 1024, (size_t)B * 16 * sizeof(GrpEw));
    b->slot_bytes = std::max<size_t>(b->slot_bytes, (size_t)B * D * sizeof(GrpEw) + 1024);
    b->slot_bytes = std::max<size_t>(b->slot_bytes, (size_t)B * sizeof(GemmProblem) + 1024);
    b->stage_slots = 512;
    if (cudaMallocHost((void**)&b->stage_host, b->slot_bytes * b->stage_slots) != cudaSuccess ||
        cudaMalloc((void**)&b->stage_dev, b->slot_bytes * b->stage_slots) != cudaSuccess ||
        cudaMallocHost((void**)&b->pinned, (size_t)B * kSlots * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        cdmpt_batch_destroy(b);
        set_error("batch: staging allocation failed");
        return CDMPT_ERR_OOM;
    }
    *out = b;
    return CDMPT_OK;
}

cdmpt_status cdmpt_batch_set_H(cdmpt_batch* b, const double* const* H0, const double* const* H1,
                               int n, int on_device) {
    if (!b || !H0 || (b->D > 0 && !H1) || n < 1 || n > 60) return CDMPT_ERR_ARG;
    cdmpt_status s = alloc_batch(b, n);
    if (s != CDMPT_OK) return bfail(b, s);
    cudaStream_t st = b->cx.stream;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    double* tmp = nullptr;
    CDMPT_CUDA_TRY(cudaMallocAsync((void**)&tmp, 4 * sizeof(double), st));
    for (int i = 0; i < b->B; ++i) {
        Sys& sy = b->sys[i];
        if (!H0[i] || (b->D > 0 && !H1[i])) return bfail_msg(b, CDMPT_ERR_ARG, "batch: NULL H");
        CDMPT_CUDA_TRY(cudaMemcpy2DAsync(sy.H0, sy.ld * sizeof(double), H0[i],
                                         sy.N * sizeof(double), sy.N * sizeof(double), sy.N,
                                         kind, st));
        if (b->D > 0)
            CDMPT_CUDA_TRY(cudaMemcpy2DAsync(sy.H1, sy.ld * sizeof(double), H1[i],
                                             sy.N * sizeof(double), sy.N * sizeof(double),
                                             (size_t)b->D * sy.N, kind, st));
        CDMPT_CUDA_TRY(cudaMemsetAsync(tmp, 0, 4 * sizeof(double), st));
        s = gershgorin(sy.H0, sy.N, sy.ld, tmp, st);
        if (s != CDMPT_OK) return bfail(b, s);
        s = Ew<double>::trace(sy.H0, sy.N, sy.ld, 1, tmp + 2, st);
        if (s != CDMPT_OK) return bfail(b, s);
        double host[3];
        CDMPT_CUDA_TRY(cudaMemcpyAsync(host, tmp, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
        CDMPT_CUDA_TRY(cudaStreamSynchronize(st));
        sy.gmin = host[0];
        sy.gmax = host[1];
        sy.trH0 = host[2];
    }
    CDMPT_CUDA_TRY(cudaFreeAsync(tmp, st));
    b->have_H = true;
    return CDMPT_OK;
}

cdmpt_status cdmpt_batch_solve(cdmpt_batch* b, const double* beta, const double* nocc, int n,
                               double* const* P0, double* const* P1, double* mu, double* mu1,
                               double* alpha, int out_on_device) {
    if (!b || !beta || !nocc) return CDMPT_ERR_ARG;
    if (!b->have_H || n > b->n_alloc)
        return bfail_msg(b, CDMPT_ERR_ARG, "batch: call cdmpt_batch_set_H with this n first");
    const auto t0 = std::chrono::steady_clock::now();
    const long long launches0 = launch_count();
    std::memset(&b->st, 0, sizeof(b->st));
    b->cx.st = &b->st;
    const int G = b->B, D = b->D;
    cudaStream_t st = b->cx.stream;
    std::vector<double> inact(G, 0.0);
    for (int i = 0; i < G; ++i) {
        Sys& sy = b->sys[i];
        if (!(beta[i] > 0) || !(nocc[i] > 0) || !(nocc[i] < sy.N))
            return bfail_msg(b, CDMPT_ERR_ARG, "batch: need beta > 0 and 0 < nocc < N");
        sy.beta = beta[i];
        sy.nocc = nocc[i];
        sy.s2 = std::ldexp(beta[i], -(n + 1));
        const double width = sy.gmax - sy.gmin;
        if (!(sy.s2 * width < 1.0))
            return bfail_msg(b, CDMPT_ERR_RANGE, "batch: beta (lambda_max - lambda_min) / 2^(n+1) "
                                                 ">= 1 for system " + std::to_string(i));
        const double pad = std::min(40.0 / sy.beta, 0.45 * (1.0 / sy.s2 - width));
        sy.lo = sy.gmin - pad;
        sy.hi = sy.gmax + pad;
        sy.mu = std::min(std::max(sy.trH0 / sy.N, sy.lo + 1e-3 * pad), sy.hi - 1e-3 * pad);
        sy.e_lo = sy.e_hi = 0.0;
        sy.converged = false;
    }
    // mixed precision: one-pass TF32 sweeps, then split-TF32 refinement (as in cdmpt_solve)
    const bool mixed = b->opts.precision == CDMPT_MIXED_TF32;
    const int sweep_engine = mixed ? (int)CDMPT_GEMM_TC_TF32 : kEngine;
    const double sweep_tol = mixed ? 1e-4 : b->opts.cg_tol;
    for (bool& f : b->cx.ph_set) f = false;
    b->cx.mark(0);
    // -------------------------------------------------- occupation loops, in lockstep
    int sweeps = 0;
    for (; sweeps < b->opts.mu_maxit; ++sweeps) {
        for (int i = 0; i < G; ++i) inact[i] = b->sys[i].converged ? 1.0 : 0.0;
        CDMPT_CUDA_TRY(cudaMemcpyAsync(b->inactive, inact.data(), G * sizeof(double),
                                       cudaMemcpyHostToDevice, st));
        int iters = 0;
        cdmpt_status s = sweep_batch(b, n, &iters, sweep_engine, sweep_tol);
        if (s != CDMPT_OK) return bfail(b, s);
        b->st.cg_iterations_sweeps += iters;
        CDMPT_TRY(zero_slots(b, B_TRZ, 2));
        {
            std::vector<GrpEw> dt, dd;
            for (int i = 0; i < G; ++i) {
                Sys& sy = b->sys[i];
                GrpEw e = ewd(sy.Z[n].x, sy.Z[n].x);
                e.rows = sy.N; e.ld = sy.ld; e.N = sy.N; e.count = (long long)sy.blk;
                e.sc = sy.sc;
                e.skip = b->inactive + i;
                e.s0 = B_TRZ;
                dt.push_back(e);
                e.s0 = B_ZZ;
                dd.push_back(e);
            }
            s = run_tiles(b, dt, 1, grouped_trace);
            if (s != CDMPT_OK) return bfail(b, s);
            s = run_ew(b, G_DOT, dd);
            if (s != CDMPT_OK) return bfail(b, s);
        }
        CDMPT_TRY(read_all(b));
        bool all = true;
        for (int i = 0; i < G; ++i) {
            Sys& sy = b->sys[i];
            if (sy.converged) continue;
            const double trP = 0.5 * (sy.N + b->pinned[i * kSlots + B_TRZ]);
            const double zz = b->pinned[i * kSlots + B_ZZ];
            const double err = trP - sy.nocc;
            double tol = b->opts.occ_tol > 0 ? b->opts.occ_tol : 1e-7 * sy.N;
            // one-pass TF32 traces are good to about 1e-4, and their per-level rounding adds
            // noise of about 5e-4 sqrt(N), which dominates for small N; the refinement
            // finishes mu
            if (mixed) tol = std::max({tol, 1e-5 * sy.N, 5e-4 * std::sqrt((double)sy.N)});
            if (std::fabs(err) <= tol) {
                sy.converged = true;
                continue;
            }
            all = false;
            if (err > 0) {
                sy.hi = sy.mu;
                sy.e_hi = err;
            } else {
                sy.lo = sy.mu;
                sy.e_lo = err;
            }
            const double slope = 0.25 * sy.beta * (sy.N - zz);
            double mnew = slope > 0 ? sy.mu - err / slope : sy.lo - 1.0;
            if (!(mnew > sy.lo && mnew < sy.hi))
                mnew = next_mu_outside_newton(sy.lo, sy.hi, sy.e_lo, sy.e_hi);
            sy.mu = mnew;
        }
        if (all) {
            ++sweeps;
            break;
        }
    }
    b->st.mu_iterations = sweeps;
    for (int i = 0; i < G; ++i)
        if (!b->sys[i].converged)
            return bfail_msg(b, CDMPT_ERR_NO_CONVERGENCE,
                             "batch: occupation of system " + std::to_string(i) + " not reached");
    b->cx.mark(1);
    // -------------------------------------------------- refinement (mixed), in lockstep
    if (mixed) {
        const int min_pass = std::max(1, b->opts.refine_rounds);
        for (int i = 0; i < G; ++i) b->sys[i].converged = false;
        // first step of each system's FP64-class residuals: every step, or the steps whose
        // spectral bound tanh(2^k atanh rho) exceeds hp_bound(), or none
        int k_first = n;
        for (int i = 0; i < G; ++i) {
            Sys& sy = b->sys[i];
            sy.hp = false;
            sy.hp_passes = 0;
            sy.khp = n;
            if (b->opts.fp64_residual > 0) {
                sy.khp = 0;
            } else if (b->opts.fp64_residual == 0) {
                const double a0 = std::atanh(
                    std::min(sy.s2 * std::max(sy.gmax - sy.mu, sy.mu - sy.gmin), 0.999999));
                int k = 0;
                while (k < n && std::tanh(std::ldexp(a0, k)) <= hp_bound()) ++k;
                sy.khp = k;
            }
            k_first = std::min(k_first, sy.khp);
        }
        b->st.fp64_residual_first_step = k_first;
        const double hp_occ = batch_hp_switch();
        // Each system runs split-TF32 passes until it switches to passes whose late-step
        // residuals are FP64-class (by default after its first split pass; with a switch
        // threshold, once its occupation error after a split pass is within the threshold,
        // so that the Newton steps on mu it still needs run on the cheaper split passes). It
        // finishes only in an FP64-class pass (or, without any, in a split pass that did not
        // follow a Newton step), so that no occupation is accepted on a trajectory carrying
        // the split products' bias.
        std::vector<char> shifted(G, 1);
        bool all = false;
        for (int pass = 0; pass < min_pass + 12 && !all; ++pass) {
            std::vector<char> active(G, 0);
            bool any_hp = false;
            for (int i = 0; i < G; ++i) {
                active[i] = b->sys[i].converged ? 0 : 1;
                inact[i] = active[i] ? 0.0 : 1.0;
                any_hp = any_hp || (active[i] && b->sys[i].hp && b->sys[i].khp < n);
            }
            CDMPT_CUDA_TRY(cudaMemcpyAsync(b->inactive, inact.data(), G * sizeof(double),
                                           cudaMemcpyHostToDevice, st));
            int iters = 0;
            cdmpt_status s = refine_batch(b, n, active, &iters);
            if (s != CDMPT_OK) return bfail(b, s);
            b->st.cg_iterations_refine += iters;
            b->st.refine_passes += 1;
            if (any_hp) b->st.fp64_residual_passes += 1;
            s = occupations(b, n);
            if (s != CDMPT_OK) return bfail(b, s);
            all = true;
            bool stuck = false;
            std::vector<char> reinit(G, 0);
            for (int i = 0; i < G; ++i) {
                Sys& sy = b->sys[i];
                if (sy.converged) continue;
                const double trP = 0.5 * (sy.N + b->pinned[i * kSlots + B_TRZ]);
                const double zz = b->pinned[i * kSlots + B_ZZ];
                const double err = trP - sy.nocc;
                // finish mu to 1e-9 N, or to 1e-7 sqrt(N) once the minimum passes are done
                const double tol = b->opts.occ_tol > 0
                                       ? b->opts.occ_tol
                                       : std::max(1e-9 * sy.N, pass + 1 >= min_pass
                                                                   ? 1e-7 * std::sqrt((double)sy.N)
                                                                   : 0.0);
                const bool occ_ok = std::fabs(err) <= tol;
                const bool final_phase = sy.hp || sy.khp >= n;
                if (final_phase && occ_ok && pass + 1 >= min_pass && (sy.hp || !shifted[i])) {
                    sy.converged = true;
                    continue;
                }
                all = false;
                shifted[i] = 0;
                if (sy.hp) {
                    if (++sy.hp_passes >= 4) stuck = true;
                } else if (sy.khp < n) {
                    // switch to the FP64-class passes: at once (hp_occ < 0), or once the
                    // occupation is within the threshold
                    if (hp_occ < 0 || std::fabs(err) <= std::max(tol, hp_occ * std::sqrt((double)sy.N)))
                        sy.hp = true;
                }
                if (!occ_ok) {   // Newton step on mu; Z_0 = -s2 (H0 - mu I) is rebuilt
                    const double slope = 0.25 * sy.beta * (sy.N - zz);
                    if (slope > 0) sy.mu -= err / slope;
                    reinit[i] = 1;
                    shifted[i] = 1;
                }
            }
            bool any_re = false;
            for (int i = 0; i < G; ++i) any_re = any_re || reinit[i];
            if (any_re) {
                std::vector<const double*> none_skip(G, nullptr);
                CDMPT_TRY(init_z0_batch(b, none_skip, &reinit));
            }
            if (stuck) break;
        }
        if (!all)
            return bfail_msg(b, CDMPT_ERR_NO_CONVERGENCE,
                             "batch: mixed-precision refinement did not converge");
    }
    if (mu)
        for (int i = 0; i < G; ++i) mu[i] = b->sys[i].mu;
    std::fill(inact.begin(), inact.end(), 0.0);
    CDMPT_CUDA_TRY(cudaMemcpyAsync(b->inactive, inact.data(), G * sizeof(double),
                                   cudaMemcpyHostToDevice, st));
    std::vector<const double*> none(G, nullptr);

    b->cx.mark(2);
    // -------------------------------------------------- response (all systems, D directions)
    if (D > 0) {
        std::vector<GrpEw> d;
        for (int i = 0; i < G; ++i) {
            Sys& sy = b->sys[i];
            GrpEw e = ewd(sy.Z1a.x, nullptr, sy.Z1a.hi, sy.Z1a.lo);
            e.h = sy.H1;
            e.rows = D * sy.N; e.ld = sy.ld; e.N = sy.N;
            e.s0 = -sy.s2;
            e.s1 = 0.0;
            d.push_back(e);
        }
        CDMPT_TRY(run_ew(b, G_INIT_Z, d));
        int total = 0, hint = 1;
        for (int k = 0; k < n; ++k) {
            std::vector<GemmSpec> gs, g1, g2;
            std::vector<GrpEw> dta, dz, dsym;
            std::vector<BCg> cg(G);
            for (int i = 0; i < G; ++i) {
                Sys& sy = b->sys[i];
                Mat* Z1 = (k % 2 == 0) ? &sy.Z1a : &sy.Z1b;
                Mat* Z1n = (k % 2 == 0) ? &sy.Z1b : &sy.Z1a;
                const int rows = D * sy.N;
                GemmSpec a;              // S^T = Z1 Z_k
                a.X = Z1;
                a.rows = rows;
                a.Y = &sy.Z[k];
                a.p = epi(sy.S.x, rows, sy.N, sy.ld);
                a.skip = nullptr;
                gs.push_back(a);
                GrpEw t = ewd(sy.A1.x, sy.S.x, sy.A1.hi, sy.A1.lo);
                t.rows = rows; t.ld = sy.ld; t.N = sy.N;
                dta.push_back(t);
                GemmSpec r1;             // RHS = -(A1 Z_{k+1})^T
                r1.X = &sy.A1;
                r1.rows = rows;
                r1.Y = &sy.Z[k + 1];
                r1.p = epi(sy.RHS.x, rows, sy.N, sy.ld, -1.f);
                r1.p.trans_block = sy.N;
                r1.skip = nullptr;
                g1.push_back(r1);
                GemmSpec r2;             // RHS -= 2 Z1 W_k
                r2.X = Z1;
                r2.rows = rows;
                r2.Y = &sy.W[k];
                r2.p = epi(sy.RHS.x, rows, sy.N, sy.ld, -2.f, 1.f, sy.RHS.x);
                r2.skip = nullptr;
                g2.push_back(r2);
                cg[i] = BCg{Z1n->x, nullptr, sy.RHS.x, &sy.W[k], rows};
                cg[i].ref = Z1->x;     // tolerance also relative to 2 Z1_k (as cdmpt_solve)
                cg[i].ref_scale = 2.0;
                GrpEw z = ewd(Z1n->x, Z1->x);
                z.rows = rows; z.ld = sy.ld; z.N = sy.N; z.count = (long long)rows * sy.ld;
                z.s0 = 2.0;
                z.s1 = 1.0;
                dz.push_back(z);
                GrpEw y = ewd(Z1n->x, nullptr, Z1n->hi, Z1n->lo);
                y.rows = rows; y.ld = sy.ld; y.N = sy.N;
                dsym.push_back(y);
            }
            CDMPT_TRY(grouped_gemm(b, gs));
            CDMPT_TRY(run_tiles(b, dta, D, grouped_transpose_add));
            CDMPT_TRY(grouped_gemm(b, g1));
            CDMPT_TRY(grouped_gemm(b, g2));
            for (int i = 0; i < G; ++i)
                add_flops(b, 6.0 * D * (double)b->sys[i].N * b->sys[i].N * b->sys[i].N);
            int it = 0;
            cdmpt_status s = CDMPT_OK;
            if (mixed) {
                // mixed-precision iterative refinement of each step's system, as in
                // cdmpt_solve: one-pass TF32 cycles that cut the residual about three digits,
                // restarted from the split-TF32 residual of the current solution
                std::vector<GrpEw> dsplit;   // hi/lo of the current solution for the restart
                for (int i = 0; i < G; ++i) {
                    Sys& sy = b->sys[i];
                    Mat* Z1n = (k % 2 == 0) ? &sy.Z1b : &sy.Z1a;
                    GrpEw e = ewd(Z1n->x, Z1n->x, Z1n->hi, Z1n->lo);
                    e.rows = D * sy.N; e.ld = sy.ld; e.N = sy.N;
                    e.count = (long long)D * sy.N * sy.ld;
                    e.s0 = 1.0;
                    e.s1 = 0.0;
                    dsplit.push_back(e);
                }
                int h = hint;
                for (int cyc = 0; cyc < 8 && s == CDMPT_OK; ++cyc) {
                    if (cyc > 0) {
                        for (int i = 0; i < G; ++i)
                            cg[i].x0 = (k % 2 == 0) ? &b->sys[i].Z1b : &b->sys[i].Z1a;
                        CDMPT_TRY(run_ew(b, G_AXPBY, dsplit));
                    }
                    int itc = 0;
                    double r0 = 0.0;
                    bool met = false;
                    s = cg_batch(b, cg, 1.0, 1.0, b->opts.cg_tol, none, h, &itc, false,
                                 CDMPT_GEMM_TC_TF32, kEngine, 1e-3, &r0, b->opts.cg_tol, &met);
                    it += itc;
                    h = std::max(1, itc);
                    if (itc == 0 || met || r0 * 1e-3 <= b->opts.cg_tol) break;
                }
            } else {
                s = cg_batch(b, cg, 1.0, 1.0, b->opts.cg_tol, none, hint, &it, false, kEngine, -1,
                             0.0, nullptr, b->opts.cg_tol);
            }
            if (s != CDMPT_OK) return bfail(b, s);
            total += it;
            hint = std::max(1, it);
            CDMPT_TRY(run_ew(b, G_AXPBY, dz));
            CDMPT_TRY(run_tiles(b, dsym, D, grouped_symmetrize));
        }
        b->st.cg_iterations_response = total;
        b->cx.mark(3);
        // Q' = (I - Z_n^2)(I - W_0)^-1; dP0/dmu = beta/4 Q'
        {
            std::vector<GemmSpec> gq;
            std::vector<BCg> cg(G);
            std::vector<GrpEw> dsym;
            for (int i = 0; i < G; ++i) {
                Sys& sy = b->sys[i];
                GemmSpec q;
                q.X = &sy.Z[n];
                q.rows = sy.N;
                q.Y = &sy.Z[n];
                q.p = epi(sy.RHS.x, sy.N, sy.N, sy.ld, -1.f, 0.f, nullptr, 1.f);
                q.p.sym = 1;
                q.p.Dhi = sy.RHS.hi;
                q.p.Dlo = sy.RHS.lo;
                q.skip = nullptr;
                gq.push_back(q);
                cg[i] = BCg{sy.Qmu.x, &sy.RHS, sy.RHS.x, &sy.W[0], sy.N};
                GrpEw y = ewd(sy.Qmu.x);
                y.rows = sy.N; y.ld = sy.ld; y.N = sy.N;
                dsym.push_back(y);
            }
            if (mixed) {
                // I - Z_n^2 cancels for saturated levels: form it from the pair-stored Z_n with
                // the Ozaki-sliced product, system by system
                for (int i = 0; i < G; ++i) {
                    Sys& sy = b->sys[i];
                    for (auto& o : b->oz[0]) o.ld = sy.ld;
                    CDMPT_TRY(oz_slice(sy.Z[n].x, sy.Z[n].xl, sy.N, sy.N, sy.ld, b->oz[0][0], st));
                    OzEpi q;
                    q.sym = 1;   // I - Z_n Z_n: upper-triangle tiles, mirrored
                    q.D = sy.RHS.x;
                    q.Dthi = sy.RHS.hi;
                    q.Dtlo = sy.RHS.lo;
                    q.ldd = sy.ld;
                    q.alpha = -1.f;
                    q.gamma = 1.f;
                    CDMPT_TRY(gemm_oz(sy.N, sy.N, sy.N, b->oz[0][0], b->oz[0][0], q, st));
                    if (b->cx.st) {
                        const double f = 2.0 * sy.N * (double)sy.N * sy.N;
                        b->cx.st->gemm_launches += 1;
                        b->cx.st->gemm_flops += f;
                        b->cx.st->tensor_flops += oz_products(kOzDigits) * f;
                    }
                }
            } else {
                CDMPT_TRY(grouped_gemm(b, gq));
                for (int i = 0; i < G; ++i) add_flops(b, sym_flops(b, b->sys[i].N));
            }
            int it = 0;
            cdmpt_status s = cg_batch(b, cg, 1.0, -1.0, b->opts.cg_tol, none, 1, &it, true);
            if (s != CDMPT_OK) return bfail(b, s);
            b->st.cg_iterations_q = it;
            CDMPT_TRY(run_tiles(b, dsym, 1, grouped_symmetrize));
        }
        // traces, mu1, P1 = Z1/2 + mu1 Q, alpha = -sum Z1 H1
        Mat* Z1f = (n % 2 == 0) ? nullptr : nullptr;
        (void)Z1f;
        CDMPT_TRY(zero_slots(b, B_TRQ, 1));
        CDMPT_TRY(zero_slots(b, B_TRZ1, 32));
        {
            std::vector<GrpEw> dq, dz;
            for (int i = 0; i < G; ++i) {
                Sys& sy = b->sys[i];
                Mat* Z1 = (n % 2 == 0) ? &sy.Z1a : &sy.Z1b;
                GrpEw q = ewd(sy.Qmu.x);
                q.rows = sy.N; q.ld = sy.ld; q.N = sy.N;
                q.sc = sy.sc;
                q.s0 = B_TRQ;
                dq.push_back(q);
                GrpEw z = ewd(Z1->x);
                z.rows = D * sy.N; z.ld = sy.ld; z.N = sy.N;
                z.sc = sy.sc;
                z.s0 = B_TRZ1;
                dz.push_back(z);
            }
            CDMPT_TRY(run_tiles(b, dq, 1, grouped_trace));
            CDMPT_TRY(run_tiles(b, dz, D, grouped_trace));
        }
        CDMPT_TRY(read_all(b));
        {
            std::vector<GrpEw> da, dh;
            for (int i = 0; i < G; ++i) {
                Sys& sy = b->sys[i];
                Mat* Z1 = (n % 2 == 0) ? &sy.Z1a : &sy.Z1b;
                const double trQ = 0.25 * sy.beta * b->pinned[i * kSlots + B_TRQ];
                for (int dd = 0; dd < D; ++dd) {
                    const double trP1 = 0.5 * b->pinned[i * kSlots + B_TRZ1 + dd];
                    const double m1 = trQ > 0 ? -trP1 / trQ : 0.0;
                    if (mu1) mu1[i * D + dd] = m1;
                    GrpEw a = ewd(Z1->x + (size_t)dd * sy.blk, sy.Qmu.x);
                    a.rows = sy.N; a.ld = sy.ld; a.N = sy.N; a.count = (long long)sy.blk;
                    a.s0 = 2.0 * m1 * 0.25 * sy.beta;
                    a.s1 = 1.0;
                    da.push_back(a);
                    GrpEw h = ewd(Z1->x + (size_t)dd * sy.blk);
                    h.h = sy.H1 + (size_t)dd * sy.blk;
                    h.rows = sy.N; h.ld = sy.ld; h.N = sy.N;
                    h.sc = sy.sc;
                    h.s0 = B_ALPHA + dd;
                    dh.push_back(h);
                }
            }
            CDMPT_TRY(zero_slots(b, B_ALPHA, 16));
            CDMPT_TRY(run_ew(b, G_AXPBY, da));
            CDMPT_TRY(run_ew(b, G_DOT_H, dh));
        }
        CDMPT_TRY(read_all(b));
        for (int i = 0; i < G; ++i)
            for (int dd = 0; dd < D; ++dd)
                if (alpha) alpha[i * D + dd] = -b->pinned[i * kSlots + B_ALPHA + dd];
    }
    b->cx.mark(4);
    // -------------------------------------------------- outputs
    for (int i = 0; i < G; ++i) {
        Sys& sy = b->sys[i];
        const size_t e0 = (size_t)sy.N * sy.N;
        if (P0 && P0[i]) {
            auto p0_out = [&](double* out) -> cdmpt_status {
                if (sy.Z[n].xl)
                    return pair::to_f64(out, sy.N, sy.Z[n].x, sy.Z[n].xl, sy.ld, sy.N, sy.N, 0.5,
                                        0.5, st);
                return Ew<float>::to_f64(out, sy.N, sy.Z[n].x, sy.ld, sy.N, sy.N, 0.5, 0.5, st);
            };
            if (out_on_device) {
                CDMPT_TRY(p0_out(P0[i]));
            } else {
                double* tmp = nullptr;
                CDMPT_CUDA_TRY(cudaMallocAsync((void**)&tmp, e0 * sizeof(double), st));
                CDMPT_TRY(p0_out(tmp));
                CDMPT_CUDA_TRY(cudaMemcpyAsync(P0[i], tmp, e0 * sizeof(double),
                                               cudaMemcpyDeviceToHost, st));
                CDMPT_CUDA_TRY(cudaFreeAsync(tmp, st));
            }
        }
        if (D > 0 && P1 && P1[i]) {
            Mat* Z1 = (n % 2 == 0) ? &sy.Z1a : &sy.Z1b;
            const int rows = D * sy.N;
            if (out_on_device) {
                CDMPT_TRY(Ew<float>::to_f64(P1[i], sy.N, Z1->x, sy.ld, sy.N, rows, 0.5, 0.0, st));
            } else {
                double* tmp = nullptr;
                CDMPT_CUDA_TRY(cudaMallocAsync((void**)&tmp, D * e0 * sizeof(double), st));
                CDMPT_TRY(Ew<float>::to_f64(tmp, sy.N, Z1->x, sy.ld, sy.N, rows, 0.5, 0.0, st));
                CDMPT_CUDA_TRY(cudaMemcpyAsync(P1[i], tmp, D * e0 * sizeof(double),
                                               cudaMemcpyDeviceToHost, st));
                CDMPT_CUDA_TRY(cudaFreeAsync(tmp, st));
            }
        }
    }
    b->cx.mark(5);
    CDMPT_CUDA_TRY(cudaStreamSynchronize(st));
    b->st.kernel_launches = (int)(launch_count() - launches0);
    b->st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int i = 0; i < 5 && b->cx.profile; ++i) {
        if (!b->cx.ph_set[i]) continue;
        int j = i + 1;
        while (j < 6 && !b->cx.ph_set[j]) ++j;
        float e = 0;
        if (j < 6 && cudaEventElapsedTime(&e, b->cx.ph[i], b->cx.ph[j]) == cudaSuccess)
            b->st.phase_ms[i] = e;
    }
    b->st.n = n;
    b->st.D = D;
    b->st.N = G;
    cdmpt_status s = check_device_error(st);
    if (s != CDMPT_OK) return bfail(b, s);
    return CDMPT_OK;
}

cdmpt_status cdmpt_batch_get_stats(const cdmpt_batch* b, cdmpt_stats* st) {
    if (!b || !st) return CDMPT_ERR_ARG;
    *st = b->st;
    return CDMPT_OK;
}

const char* cdmpt_batch_last_error(const cdmpt_batch* b) {
    if (!b) return get_error().c_str();
    return b->err.c_str();
}

cdmpt_status cdmpt_batch_get_tuning(const cdmpt_batch* b, int* tile_n, double* ms, int* graphs) {
    if (!b) return CDMPT_ERR_ARG;
    if (tile_n) *tile_n = b->tile_bn;
    if (ms) {
        ms[0] = b->tune_ms[0];
        ms[1] = b->tune_ms[1];
        ms[2] = b->tune_ms[2];
    }
    if (graphs) *graphs = (b->graphs && !b->it_graphs.empty()) ? 1 : 0;
    return CDMPT_OK;
}

void cdmpt_batch_destroy(cdmpt_batch* b) {
    if (!b) return;
    drop_graphs(b);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (cudaEvent_t e : b->cx.ph)
        if (e) cudaEventDestroy(e);
    for (int l = 0; l < cdmpt_batch::kHpLanes; ++l) {
        if (b->hp_st[l]) cudaStreamDestroy(b->hp_st[l]);
        if (b->hp_join[l]) cudaEventDestroy(b->hp_join[l]);
    }
    if (b->hp_fork) cudaEventDestroy(b->hp_fork);
    for (void* p : b->allocs) cudaFree(p);
    if (b->stage_host) cudaFreeHost(b->stage_host);
    if (b->stage_dev) cudaFree(b->stage_dev);
    if (b->pinned) cudaFreeHost(b->pinned);
    delete b;
}

}  // extern "C"
