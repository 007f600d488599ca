// Canonical DMPT solve on the device, in the deviation form Z = 2X - I.
//
// Paper (Eq. Rec_F_2, Algorithm 1) -> this code:
//   X_0 = I/2 - 2^-(n+2) beta (H - mu I)        Z_0 = -s2 (H - mu I), s2 = beta / 2^(n+1)
//   T_{k} = 2 X_k (X_k - I) + I                  T_k = (I + Z_k^2) / 2 = A_k / 2
//   T_k X_{k+1} = X_k^2                          Z_{k+1} A_k = 2 Z_k
//   T_k X^(1)_{k+1} = C^(1)_k + B^(1)_k X_{k+1}  Z1_{k+1} A_k = 2 Z1_k - Z_{k+1} (Z_k Z1_k + Z1_k Z_k)
//   P0 = X_n, P1 = X^(1)_n                       P0 = (I + Z_n)/2, P1 = Z1_n / 2
// Every linear system is solved with right multiplication X -> X A_k (A_k is
// symmetric), so all products are X Y^T with Y symmetric. Solutions are
// symmetric in exact arithmetic and are symmetrised after every solve.
// A_k is kept as W_k = Z_k^2 and applied as X + X W_k, and the 0th-order step
// solves for the correction d = Z_{k+1} - 2 Z_k from d A_k = -2 Z_k W_k: in
// FP32 this keeps the small quantities (Z^2 in early steps, the correction)
// in their own exponent range instead of rounding them against I or 2 Z_k,
// which makes the CG result about three times more accurate than solving for
// Z_{k+1} against A_k = I + Z_k^2 directly.
//
// Chemical potential: Newton on Tr P0 = N_occ with the paper's slope
// Tr P_mu = beta Tr[P0 (I - P0)] = beta/4 (N - ||Z_n||_F^2) (Eq. NewtRaphs),
// safeguarded by a bisection bracket. mu1: P1 is linear in mu1 with slope
// Q = dP0/dmu, which at finite n is exactly beta P0 (I - P0) (I - Z_0^2)^-1;
// the response runs once with mu1 = 0 and mu1 = -Tr P1|_0 / Tr Q follows in
// closed form (the fixed point of the mu1 update of Algorithm 1).
//
// Mixed precision (CDMPT_MIXED_TF32): the occupation sweeps run with one-pass
// TF32 products. The converged trajectory is then refined step by step: with
// Z_k already refined, A_k = I + Z_k^2 and the residual 2 Z_k - Z_{k+1} A_k
// are formed with split-TF32 (FP32-accurate) products, and the correction of
// Z_{k+1} is found by CG whose iterations use one-pass TF32 products (mixed-
// precision iterative refinement of each step's linear system). Between
// passes a Newton step on mu shifts Z_0 by s2 dmu I. The response then uses
// split-TF32 products throughout. CDMPT_MIXED_BF16 is the same with the
// occupation sweeps on BF16-rounded operands (kind::f16, FP32 accumulation).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <cmath>
#include <string>

#include "solver.cuh"

namespace cdmpt {

namespace {
enum Slot {
    S_TRZ = 8,      // Tr Z_n
    S_ZZ = 9,       // ||Z_n||_F^2
    S_TRQ = 10,     // Tr Q
    S_REF = 11,     // ||ref||_F^2 of the running CG solve's absolute tolerance
    S_TRZ1 = 16,    // Tr Z1_d (d < 16)
    S_ALPHA = 32,   // sum P1_d * H1_d (d < 16)
    S_FE = 48,      // free energy and Omega terms: traces and dots (5 slots)
    S_NSLOTS = 64
};
constexpr int kMaxD = 16;
}  // namespace

template <typename T>
Solver<T>::~Solver() {
    for (void* p : allocs_) cudaFree(p);
}

template <typename T>
cdmpt_status Solver<T>::reserve(int N, int D, int n, int ckpt, bool pairs) {
    const int ld_new = (N + 31) / 32 * 32;
    const int rows_needed = std::max(1, D) * N;
    pairs = pairs && sizeof(T) == 4 && ckpt == 0;
    seg_ = -1;
    // with checkpoints the trajectory views are laid out for exactly n steps
    if (N == N_ && D <= D_ && (ckpt == 0 ? n <= n_ : n == n_) && ckpt == ck_ && ld == ld_new &&
        rows_cap_ >= rows_needed && pairs == pairs_)
        return CDMPT_OK;
    for (void* p : allocs_) cudaFree(p);
    allocs_.clear();
    Z_.clear();
    W_.clear();
    orders_ready_ = false;
    oz64_ready_ = false;
    ck_ = ckpt;
    pairs_ = pairs;
    N_ = N;
    D_ = D;
    n_ = n;
    ld = ld_new;
    blk_ = (size_t)N * ld;
    rows_cap_ = rows_needed;
    auto grab = [&](size_t elems, T** out) -> cdmpt_status {
        void* p = nullptr;
        if (cudaMalloc(&p, elems * sizeof(T)) != cudaSuccess) {
            cudaGetLastError();
            set_error("device allocation of " + std::to_string(elems * sizeof(T)) + " bytes failed");
            return CDMPT_ERR_OOM;
        }
        if (cudaMemset(p, 0, elems * sizeof(T)) != cudaSuccess) return CDMPT_ERR_CUDA;
        allocs_.push_back(p);
        *out = (T*)p;
        return CDMPT_OK;
    };
    // split = true: also the TF32 hi/lo arrays (float storage only)
    auto buf = [&](size_t elems, Buf<T>* b, bool split) -> cdmpt_status {
        *b = Buf<T>();
        CDMPT_TRY(grab(elems, &b->x));
        if (split && sizeof(T) == 4) {
            CDMPT_TRY(grab(elems, &b->hi));
            CDMPT_TRY(grab(elems, &b->lo));
        }
        return CDMPT_OK;
    };
    Z_.resize(n + 1);
    W_.resize(n);
    if (ck_ == 0) {
        for (int k = 0; k <= n; ++k) {
            CDMPT_TRY(buf(blk_, &Z_[k], true));
            if (pairs_) CDMPT_TRY(grab(blk_, &Z_[k].xl));
        }
        for (int k = 0; k < n; ++k) CDMPT_TRY(buf(blk_, &W_[k], true));
    } else {
        std::vector<Buf<T>> zseg(std::max(0, ck_ - 1)), wseg(ck_);
        for (auto& b : zseg) CDMPT_TRY(buf(blk_, &b, true));
        for (auto& b : wseg) CDMPT_TRY(buf(blk_, &b, true));
        for (int k = 0; k < n; ++k) {
            if (k % ck_ == 0)
                CDMPT_TRY(buf(blk_, &Z_[k], true));   // checkpoint
            else
                Z_[k] = zseg[k % ck_ - 1];
        }
        CDMPT_TRY(buf(blk_, &Z_[n], true));
        CDMPT_TRY(buf(blk_, &W_[0], true));
        for (int k = 1; k < n; ++k) W_[k] = wseg[k % ck_];
    }
    const size_t big = (size_t)rows_needed * ld;
    CDMPT_TRY(buf(big, &R_, false));
    CDMPT_TRY(buf(big, &P_, true));
    CDMPT_TRY(buf(big, &Q_, false));
    CDMPT_TRY(buf(big, &S_, false));
    CDMPT_TRY(buf(big, &A1_, true));
    CDMPT_TRY(buf(big, &RHS_, true));
    CDMPT_TRY(buf(big, &Z1a_, true));
    CDMPT_TRY(buf(big, &Z1b_, true));
    CDMPT_TRY(buf(blk_, &Qmu_, false));
    CDMPT_TRY(buf(blk_, &Zh_, false));
    wl_ = nullptr;
    for (auto& o : oz_) o = OzOperand();
    if (pairs_) {
        // Ozaki digits of three N x N operands: kOzDigits BF16 arrays and N row exponents each
        CDMPT_TRY(grab(blk_, &wl_));
        for (auto& o : oz_) {
            o.ld = ld;
            for (int d = 0; d < kOzDigits; ++d) {
                void* q = nullptr;
                if (cudaMalloc(&q, blk_ * 2) != cudaSuccess) {
                    cudaGetLastError();
                    set_error("device allocation of the Ozaki digits failed");
                    return CDMPT_ERR_OOM;
                }
                allocs_.push_back(q);
                o.s[d] = q;
            }
            void* q = nullptr;
            if (cudaMalloc(&q, (size_t)N * sizeof(int)) != cudaSuccess) {
                cudaGetLastError();
                set_error("device allocation of the Ozaki exponents failed");
                return CDMPT_ERR_OOM;
            }
            allocs_.push_back(q);
            o.e = (int*)q;
        }
    }
    tnx_ = tny_ = tnw_ = nullptr;
    wnorm_src_ = nullptr;
    tmask_ = nullptr;
    tcnt_ = nullptr;
    if (sizeof(T) == 4) {
        // screening: norm tables of 128-row blocks x 32-column slices, the slice mask of
        // 128 x 128 output tiles, and two counters
        const size_t rb = (size_t)(rows_needed + 127) / 128, nkb = (size_t)(N + 31) / 32;
        const size_t words = rb * ((size_t)(N + 127) / 128) * ((nkb + 31) / 32);
        void* q[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
        const size_t bytes[5] = {rb * nkb * sizeof(float), rb * nkb * sizeof(float),
                                 words * sizeof(uint32_t), 2 * sizeof(unsigned long long),
                                 rb * nkb * sizeof(float)};
        for (int i = 0; i < 5; ++i) {
            if (cudaMalloc(&q[i], bytes[i]) != cudaSuccess) {
                cudaGetLastError();
                set_error("device allocation of the screening tables failed");
                return CDMPT_ERR_OOM;
            }
            allocs_.push_back(q[i]);
        }
        tnx_ = (float*)q[0];
        tny_ = (float*)q[1];
        tmask_ = (uint32_t*)q[2];
        tcnt_ = (unsigned long long*)q[3];
        tnw_ = (float*)q[4];
    }
    traj_valid_ = q_valid_ = false;
    void* p = nullptr;
    if (cudaMalloc(&p, S_NSLOTS * sizeof(double)) != cudaSuccess) return CDMPT_ERR_OOM;
    allocs_.push_back(p);
    sc_ = (double*)p;
    return CDMPT_OK;
}

template <typename T>
cdmpt_status Solver<T>::read_scalars(Context& cx, const double* dev, int count) {
    CDMPT_CUDA_TRY(cudaMemcpyAsync(cx.pinned, dev, count * sizeof(double), cudaMemcpyDeviceToHost,
                                   cx.stream));
    CDMPT_CUDA_TRY(cudaStreamSynchronize(cx.stream));
    return check_device_error(cx.stream);
}

// The mu step of the occupation loop when Newton's step (Eq. NewtRaphs: slope beta Tr[P (I -
// P)], exact only as n -> infinity) leaves the bracket [lo, hi]: false position between the
// bracket's ends once sweeps have measured both occupation errors (e_lo < 0 < e_hi), else
// bisection. Where mu sits in a gap of the spectrum the slope nearly vanishes, Newton leaves
// the bracket, and bisection alone would halve a bracket of several hoppings each sweep.
double next_mu_outside_newton(double lo, double hi, double e_lo, double e_hi) {
    if (e_lo < 0.0 && e_hi > 0.0) {
        const double m = lo - e_lo * (hi - lo) / (e_hi - e_lo);
        // stay away from the ends, where false position stalls
        const double w = hi - lo;
        if (m > lo + 0.05 * w && m < hi - 0.05 * w) return m;
    }
    return 0.5 * (lo + hi);
}

// FP64 storage: products on the tensor cores by the FP64 Ozaki engine (seven BF16 digits)
// unless CUDA-core DFMA is asked for; CDMPT_FP64_ENGINE=simt forces DFMA for comparison.
static bool fp64_on_tc() {
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("CDMPT_FP64_ENGINE");
        v = (e && std::strcmp(e, "simt") == 0) ? 0 : (tc_supported() ? 1 : 0);
    }
    return v == 1;
}

template <typename T>
int Solver<T>::engine_of(const Context& cx, int override_engine) const {
    if constexpr (sizeof(T) == 8) {
        const int e = override_engine ? override_engine : cx.engine;
        if (e == CDMPT_GEMM_SIMT) return CDMPT_GEMM_SIMT;
        return fp64_on_tc() ? CDMPT_GEMM_TC_OZAKI : CDMPT_GEMM_SIMT;
    } else {
        const int e = override_engine ? override_engine : cx.engine;
        return e == CDMPT_GEMM_AUTO ? CDMPT_GEMM_TC_3XTF32 : e;
    }
}

template <typename T>
cdmpt_status Solver<T>::oz64_prepare() {
    if (oz64_ready_) return CDMPT_OK;
    const size_t rows[2] = {(size_t)rows_cap_, (size_t)N_};
    Oz64Operand* ops[2] = {&ox64_, &oy64_};
    for (int i = 0; i < 2; ++i) {
        *ops[i] = Oz64Operand();
        ops[i]->ld = ld;
        for (int d = 0; d < 7; ++d) {
            void* q = nullptr;
            if (cudaMalloc(&q, rows[i] * ld * 2) != cudaSuccess) {
                cudaGetLastError();
                set_error("device allocation of the FP64 Ozaki digits failed");
                return CDMPT_ERR_OOM;
            }
            allocs_.push_back(q);
            ops[i]->s[d] = q;
        }
        void* q = nullptr;
        if (cudaMalloc(&q, rows[i] * sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            set_error("device allocation of the FP64 Ozaki exponents failed");
            return CDMPT_ERR_OOM;
        }
        allocs_.push_back(q);
        ops[i]->e = (int*)q;
    }
    oz64_ready_ = true;
    return CDMPT_OK;
}

// CDMPT_RESPONSE_IR=0 turns off the iterative-refinement CG of the mixed first-order
// response (every iteration then uses the FP32-accurate engine).
static bool response_ir() {
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("CDMPT_RESPONSE_IR");
        v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

// Largest relative step residual, measured at the start of a split-TF32 refinement pass, at
// which the refinement moves to the FP64-class residuals of the late steps: the correction
// CG gains three digits, so a pass that starts below 1e-3 leaves the residuals near 1e-6 and
// the FP64-class pass that follows takes them to about 1e-9. Measured on the 20^3 lattice and
// the N = 8192 banded system: one split pass and one FP64-class pass instead of two and one,
// a 13 % shorter solve, errors unchanged. The Newton step on mu that the first pass calls for
// precedes the first FP64-class pass. CDMPT_REFINE_SETTLE overrides the threshold and
// CDMPT_REFINE_EARLY_HP=0 restores the switch only after the occupation has settled on split
// residuals too (for comparison).
double refine_settle() {
    static double v = -1.0;
    if (v < 0) {
        const char* e = getenv("CDMPT_REFINE_SETTLE");
        v = e ? atof(e) : 1e-3;
        if (!(v > 0 && v < 1)) v = 1e-3;
    }
    return v;
}

bool refine_early_hp() {
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("CDMPT_REFINE_EARLY_HP");
        v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

// First step of the FP64-class residuals: the first k whose spectral bound tanh(2^k atanh rho)
// exceeds this value (default 1/2; CDMPT_HP_BOUND overrides it). Before that step the error
// of a split-TF32 residual, relative to Z_k, carries the factor ||W_k|| <= bound^2.
double hp_bound() {
    static double v = -1.0;
    if (v < 0) {
        const char* e = getenv("CDMPT_HP_BOUND");
        v = e ? atof(e) : 0.5;
        if (!(v > 0 && v < 1)) v = 0.5;
    }
    return v;
}

static double tensor_factor(int engine) {
    return engine == CDMPT_GEMM_TC_3XTF32 ? 3.0
           : (engine == CDMPT_GEMM_TC_TF32 || engine == CDMPT_GEMM_TC_BF16) ? 1.0
           : engine == CDMPT_GEMM_TC_OZAKI ? 28.0   // FP64 storage: 28 BF16 digit products
                                           : 0.0;
}

template <typename T>
cdmpt_status Solver<T>::gemm(Context& cx, int M, int Nc, int K, const Operand<T>& X,
                             const Operand<T>& Y, T* D, const Epilogue<T>& ep, const double* skip,
                             int engine_override) {
    const int engine = engine_of(cx, engine_override);
    // flops the product needs: a symmetric result on the tensor-core engines is
    // computed on its upper-triangular tiles only, N (N + 1) K instead of 2 N^2 K
    const bool sym_tc = ep.sym && M == Nc && (engine == CDMPT_GEMM_TC_TF32 ||
                                              engine == CDMPT_GEMM_TC_3XTF32 ||
                                              engine == CDMPT_GEMM_TC_BF16);
    const double flops = sym_tc ? (double)M * (M + 1) * K : 2.0 * M * (double)Nc * K;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cx.profile) {
        while (cx.ev.size() < 2 * (cx.ev_used + 1)) {
            cudaEvent_t e;
            CDMPT_CUDA_TRY(cudaEventCreate(&e));
            cx.ev.push_back(e);
        }
        if (cx.ev_ok.size() < cx.ev_used + 1) {
            cx.ev_ok.resize(cx.ev_used + 1);
            cx.ev_engine.resize(cx.ev_used + 1);
            cx.ev_flops.resize(cx.ev_used + 1);
        }
        cx.ev_ok[cx.ev_used] = 1;
        cx.ev_engine[cx.ev_used] = engine;
        cx.ev_flops[cx.ev_used] = flops;
        e0 = cx.ev[2 * cx.ev_used];
        e1 = cx.ev[2 * cx.ev_used + 1];
        CDMPT_CUDA_TRY(cudaEventRecord(e0, cx.stream));
    }
    cdmpt_status s;
    if constexpr (sizeof(T) == 4) {
        if (engine == CDMPT_GEMM_SIMT) {
            s = gemm_simt<float>(M, Nc, K, X.x, ld, Y.x, ld, D, ld, ep, skip, cx.stream);
        } else {
            // block-norm screening: tile norms of both operands, then the screened kernel
            GemmScreen sc;
            const GemmScreen* psc = nullptr;
            const bool tf32 = engine == CDMPT_GEMM_TC_TF32 || engine == CDMPT_GEMM_TC_3XTF32;
            if (screen_tau_ > 0.f && tf32 && tnx_ && M <= rows_cap_ && Nc <= N_ && K <= N_) {
                const float* xs = X.x ? X.x : X.hi;
                const float* ys = Y.x ? Y.x : Y.hi;
                CDMPT_TRY(tile_norms(xs, M, K, ld, tnx_, skip, cx.stream));
                const float* ny = tnx_;
                if (ys == wnorm_src_ && Nc == N_ && K == N_) {
                    ny = tnw_;   // the CG operator's factor: norms taken once per solve
                } else if (!(ys == xs && Nc == M)) {
                    CDMPT_TRY(tile_norms(ys, Nc, K, ld, tny_, skip, cx.stream));
                    ny = tny_;
                }
                const int nkb = (K + 31) / 32;
                CDMPT_TRY(screen_mask(tnx_, ny, M, Nc, nkb, screen_tau_, tmask_, skip, cx.stream));
                sc.mask = tmask_;
                sc.nmw = (nkb + 31) / 32;
                sc.counts = tcnt_;
                psc = &sc;
            }
            s = gemm_tc_f32(engine, M, Nc, K, X, ld, Y, ld, D, ld, ep, skip, cx.stream, psc);
        }
    } else {
        if (engine == CDMPT_GEMM_TC_OZAKI && M <= rows_cap_ && Nc <= N_ && K <= N_ &&
            K <= 16384) {
            // slice both operands (once when X is Y), then the digit product
            CDMPT_TRY(oz64_prepare());
            CDMPT_TRY(oz64_slice(X.x, M, K, ld, ox64_, skip, cx.stream));
            const Oz64Operand* oy = &ox64_;
            if (!(Y.x == X.x && Nc == M)) {
                CDMPT_TRY(oz64_slice(Y.x, Nc, K, ld, oy64_, skip, cx.stream));
                oy = &oy64_;
            }
            s = gemm_oz64(M, Nc, K, ox64_, *oy, D, ld, ep, skip, cx.stream);
        } else {
            s = gemm_simt<double>(M, Nc, K, X.x, ld, Y.x, ld, D, ld, ep, skip, cx.stream);
        }
    }
    if (s != CDMPT_OK) return s;
    if (cx.profile) {
        CDMPT_CUDA_TRY(cudaEventRecord(e1, cx.stream));
        ++cx.ev_used;
    }
    if (cx.st && skip == nullptr) {
        const double f = flops;
        cx.st->gemm_launches += 1;
        cx.st->gemm_flops += f;
        cx.st->tensor_flops += tensor_factor(engine) * f;
    }
    return CDMPT_OK;
}

// Solve X A = rhs_scale * rhs for X (rows x N) by global CG in the Frobenius
// inner product, starting from x0_scale * x0 (or zero). A is SPD (spectrum in
// [1, 2] for the recursion, Sec. II). The initial residual and the iterations
// may use different GEMM engines (accurate residual, cheap iterations: one
// step of mixed-precision iterative refinement). Scalars stay on the device;
// the host reads the convergence flag once per chunk of iterations, and
// iterations launched after convergence return at once.
template <typename T>
cdmpt_status Solver<T>::cg(Context& cx, T* X, const CgArgs& a, int* iters_out,
                           double* rel_res0, bool* met_tol) {
    const size_t count = (size_t)a.rows * ld;
    double* sc = sc_;
    const int init_engine = engine_of(cx, a.init_engine);
    const int iter_engine = engine_of(cx, a.iter_engine);
    // screened products: the operator's right factor W is fixed for the whole solve, so its
    // tile norms are taken once here and reused by every product with it
    struct NormCache {
        const float** src;
        ~NormCache() { *src = nullptr; }
    } norm_cache{&wnorm_src_};
    if constexpr (sizeof(T) == 4) {
        if (screen_tau_ > 0.f && tnw_ && a.W) {
            const float* w = a.W->x ? a.W->x : a.W->hi;
            CDMPT_TRY(tile_norms(w, N_, N_, ld, tnw_, nullptr, cx.stream));
            wnorm_src_ = w;
        }
    }
    CDMPT_CUDA_TRY(cudaMemsetAsync(sc, 0, CG_NSLOTS * sizeof(double), cx.stream));
    if (a.x0) {
        if (X != a.x0->x || a.x0_scale != 1.0)
            CDMPT_TRY(Ew<T>::axpby(X, a.x0->x, count, a.x0_scale, 0.0, nullptr, cx.stream));
        // R = rhs_scale rhs - x0_scale (s x0 + t x0 W), <R,R>
        CDMPT_TRY(Ew<T>::lincomb(R_.x, a.rhs, a.rhs_scale, a.x0->x, -a.x0_scale * a.s, count,
                                 cx.stream));
        Epilogue<T> ep;
        ep.alpha = -a.x0_scale * a.t;
        ep.beta = 1.0;
        ep.C = R_.x;
        ep.ldc = ld;
        ep.dot = sc + CG_RR;
        ep.sym = a.sym && a.rows == N_;
        CDMPT_TRY(gemm(cx, a.rows, N_, N_, a.x0->op(), a.W->op(), R_.x, ep, nullptr, init_engine));
    } else {
        CDMPT_CUDA_TRY(cudaMemsetAsync(X, 0, count * sizeof(T), cx.stream));
        CDMPT_TRY(Ew<T>::axpby(R_.x, a.rhs, count, a.rhs_scale, 0.0, nullptr, cx.stream));
        CDMPT_TRY(Ew<T>::dot(R_.x, R_.x, count, sc + CG_RR, nullptr, cx.stream));
    }
    CDMPT_TRY(Ew<T>::dot(a.rhs, a.rhs, count, sc + CG_BB, nullptr, cx.stream));
    const bool use_ref = a.ref != nullptr && a.tol_ref > 0.0;
    if (use_ref) {
        CDMPT_CUDA_TRY(cudaMemsetAsync(sc + S_REF, 0, sizeof(double), cx.stream));
        CDMPT_TRY(Ew<T>::dot(a.ref, a.ref, count, sc + S_REF, nullptr, cx.stream));
    }
    CDMPT_TRY(cg_scalar_init(sc, a.tol * a.tol * a.rhs_scale * a.rhs_scale, a.tol_r0 * a.tol_r0,
                             cx.stream, use_ref ? sc + S_REF : nullptr,
                             a.tol_ref * a.tol_ref * a.ref_scale * a.ref_scale));
    // the split of the direction P: both halves for the split-TF32 iterations, hi alone for
    // one-pass TF32, none for the engines that read P itself
    T* p_hi = (iter_engine == CDMPT_GEMM_TC_3XTF32 || iter_engine == CDMPT_GEMM_TC_TF32) ? P_.hi
                                                                                        : nullptr;
    T* p_lo = iter_engine == CDMPT_GEMM_TC_3XTF32 ? P_.lo : nullptr;
    CDMPT_TRY(Ew<T>::axpby(P_.x, R_.x, count, 1.0, 0.0, sc + CG_DONE, cx.stream, p_hi, p_lo));

    int chunk = std::max(1, a.hint);
    int iters = 0;
    while (true) {
        const size_t ev_first = cx.ev_used;
        for (int c = 0; c < chunk; ++c) {
            Epilogue<T> ep;   // Q = s P + t P W, <P,Q>
            ep.alpha = a.t;
            ep.beta = a.s;
            ep.C = P_.x;
            ep.ldc = ld;
            ep.dot = sc + CG_PQ;
            ep.E = P_.x;
            ep.lde = ld;
            ep.sym = a.sym && a.rows == N_;
            CDMPT_TRY(gemm(cx, a.rows, N_, N_, P_.op(), a.W->op(), Q_.x, ep, sc + CG_DONE,
                           iter_engine));
            CDMPT_TRY(Ew<T>::cg_update(X, R_.x, P_.x, Q_.x, count, sc, cx.stream));
            CDMPT_TRY(Ew<T>::cg_direction(P_.x, R_.x, count, sc, cx.stream, p_hi, p_lo));
            CDMPT_TRY(cg_scalar_step(sc, cx.stream));
        }
        CDMPT_TRY(read_scalars(cx, sc, S_REF + 1));
        const int now = (int)cx.pinned[CG_ITERS];
        const int ran = now - iters;
        iters = now;
        if (cx.profile) {
            // event pairs of GEMMs that returned at once are dropped
            for (size_t e = ev_first + ran; e < cx.ev_used; ++e) cx.ev_ok[e] = 0;
        }
        if (cx.st) {
            const bool sym_tc = a.sym && a.rows == N_ && iter_engine != CDMPT_GEMM_SIMT;
            const double f =
                sym_tc ? (double)N_ * (N_ + 1) * N_ : 2.0 * a.rows * (double)N_ * N_;
            cx.st->gemm_launches += ran;
            cx.st->gemm_flops += ran * f;
            cx.st->tensor_flops += ran * tensor_factor(iter_engine) * f;
        }
        if (cx.pinned[CG_DONE] != 0.0) break;
        if (iters >= a.maxit) {
            *iters_out = iters;
            set_error("CG did not reach the tolerance in " + std::to_string(a.maxit) +
                      " iterations (relative residual " +
                      std::to_string(std::sqrt(cx.pinned[CG_RRNEW] /
                                               std::max(1e-300, cx.pinned[CG_BB] * a.rhs_scale *
                                                                    a.rhs_scale))) +
                      ")");
            return CDMPT_ERR_CG_MAXITER;
        }
        chunk = 2;
    }
    *iters_out = iters;
    if (rel_res0) {
        const double bb = cx.pinned[CG_BB] * a.rhs_scale * a.rhs_scale;
        *rel_res0 = bb > 0 ? std::sqrt(cx.pinned[CG_RR0] / bb) : 0.0;
    }
    if (met_tol) {
        // the final residual meets the tolerance of the solve itself (relative to the right
        // side or the absolute reference), not only the tol_r0 reduction of this call
        const double bb = cx.pinned[CG_BB] * a.rhs_scale * a.rhs_scale;
        double lim = a.tol * a.tol * bb;
        if (use_ref)
            lim = std::max(lim, a.tol_ref * a.tol_ref * a.ref_scale * a.ref_scale *
                                    cx.pinned[S_REF]);
        *met_tol = cx.pinned[CG_RR] <= lim;
    }
    return CDMPT_OK;
}

// Fermi-Dirac-exact start (opts.fd_exact). With Y = -s2 (H0 - mu I), the n-step recursion
// maps Z_0 to Z_n = tanh(2^n atanh Z_0) (Appendix A), so Z_0 = tanh(Y) gives
// Z_n = tanh(-beta (H0 - mu I) / 2), i.e. P0 = the Fermi-Dirac function itself instead of the
// n-step function of the linear X_0 of Eq. Rec_F_2. tanh(Y) = Y h(U), U = Y^2,
// h(u) = sum_k a_k u^k, with the Taylor coefficients of tanh from tanh' = 1 - tanh^2:
// a_0 = 1, (2k + 1) a_k = -sum_{i+j=k-1} a_i a_j. The series converges for |y| < pi/2 and
// |y| <= rho < 1 here; it is cut where |a_k| rho^(2k) falls below eps.
static int tanh_terms(double rho, double eps, std::vector<double>* a) {
    a->assign(1, 1.0);
    for (int k = 1; k < 64; ++k) {
        double s = 0.0;
        for (int i = 0; i <= k - 1; ++i) s += (*a)[i] * (*a)[k - 1 - i];
        a->push_back(-s / (2 * k + 1));
        if (std::fabs(a->back()) * std::pow(rho, 2 * k) < eps) break;
    }
    return (int)a->size() - 1;   // highest power of U
}

template <typename T>
double Solver<T>::fdx_eps() const {
    return sizeof(T) == 8 ? 1e-17 : 1e-12;
}

template <typename T>
cdmpt_status Solver<T>::init_z0(Context& cx, const double* H0, double mu, double s2, double rho,
                                int engine) {
    if (!fdx_) {
        if constexpr (sizeof(T) == 4) {
            if (Z_[0].xl)   // pair storage: Z_0 to about 48 bits from the FP64 Hamiltonian
                return pair::init(Z_[0].x, Z_[0].xl, H0, N_, ld, ld, 1, -s2, mu, cx.stream,
                                  Z_[0].hi, Z_[0].lo);
        }
        return Ew<T>::init_z(Z_[0].x, H0, N_, ld, ld, 1, -s2, mu, cx.stream, Z_[0].hi, Z_[0].lo);
    }
    std::vector<double> a;
    const int K = tanh_terms(rho, fdx_eps(), &a);
    // Y and U = Y^2 stay for the tangents of the start; Horner scratch outside the
    // trajectory (the mixed refinement rebuilds Z_0 while the stored Z_1 .. Z_n are needed)
    CDMPT_TRY(reserve_orders());
    Buf<T>& Y = Yfd_;
    Buf<T>& U = Ufd_;
    CDMPT_TRY(Ew<T>::init_z(Y.x, H0, N_, ld, ld, 1, -s2, mu, cx.stream, Y.hi, Y.lo));
    {
        Epilogue<T> ep;
        ep.Dhi = U.hi;
        ep.Dlo = U.lo;
        ep.sym = true;
        CDMPT_TRY(gemm(cx, N_, N_, N_, Y.op(), Y.op(), U.x, ep, nullptr, engine));
    }
    Buf<T>* hc = &zo_[1][0];
    Buf<T>* hn = &zo_[1][1];
    CDMPT_CUDA_TRY(cudaMemsetAsync(hc->x, 0, blk_ * sizeof(T), cx.stream));
    if (hc->hi) CDMPT_CUDA_TRY(cudaMemsetAsync(hc->hi, 0, blk_ * sizeof(T), cx.stream));
    if (hc->lo) CDMPT_CUDA_TRY(cudaMemsetAsync(hc->lo, 0, blk_ * sizeof(T), cx.stream));
    // pair storage: Z_0 = Y + Y (h - I), the FP64 Y exactly as a pair and the small
    // correction Y (h - I) = O(rho^2) Y from the products (h - I: the constant term dropped)
    const bool pr = Z_[0].xl != nullptr;
    CDMPT_TRY(Ew<T>::add_diag(hc->x, N_, ld, 1, (pr && K == 0) ? 0.0 : a[K], cx.stream, hc->hi,
                              hc->lo));
    for (int k = K - 1; k >= 0; --k) {   // h <- U h + a_k I
        Epilogue<T> ep;
        ep.gamma = (pr && k == 0) ? 0.0 : a[k];
        ep.Dhi = hn->hi;
        ep.Dlo = hn->lo;
        CDMPT_TRY(gemm(cx, N_, N_, N_, U.op(), hc->op(), hn->x, ep, nullptr, engine));
        std::swap(hc, hn);
    }
    if constexpr (sizeof(T) == 4) {
        if (pr) {
            CDMPT_TRY(pair::init(Z_[0].x, Z_[0].xl, H0, N_, ld, ld, 1, -s2, mu, cx.stream));
            if (K > 0) {
                Epilogue<T> ep;   // E = Y (h - I)
                CDMPT_TRY(gemm(cx, N_, N_, N_, Y.op(), hc->op(), S_.x, ep, nullptr, engine));
                CDMPT_TRY(pair::add(Z_[0].x, Z_[0].xl, S_.x, blk_, cx.stream));
            }
            return pair::symmetrize(Z_[0].x, Z_[0].xl, N_, ld, 1, cx.stream, Z_[0].hi, Z_[0].lo);
        }
    }
    Epilogue<T> ep;   // Z_0 = Y h
    ep.Dhi = Z_[0].hi;
    ep.Dlo = Z_[0].lo;
    CDMPT_TRY(gemm(cx, N_, N_, N_, Y.op(), hc->op(), Z_[0].x, ep, nullptr, engine));
    return Ew<T>::symmetrize(Z_[0].x, N_, ld, 1, cx.stream, Z_[0].hi, Z_[0].lo);
}

// First-order start of the Fermi-Dirac-exact variant: Z1_0 = Dtanh(Y)[Y1] for the stacked
// directions Y1_d = -s2 H1_d (mu1 = 0; the mu1 term is added through Q afterwards).
template <typename T>
cdmpt_status Solver<T>::init_z1(Context& cx, const double* H1, int D, T* out, T* out_hi,
                                T* out_lo) {
    CDMPT_TRY(Ew<T>::init_z(Z1b_.x, H1, N_, ld, ld, D, -last_s2_, 0.0, cx.stream, Z1b_.hi,
                            Z1b_.lo));
    return tanh_tangent(cx, D, out, out_hi, out_lo);
}

// out_d = Dtanh(Y)[E_d] for the stacked symmetric directions E_d held in Z1b_ (with its TF32
// split in FP32), Y = -s2 (H0 - mu I) at the trajectory's mu, by the tangent of the Horner
// scheme of tanh(Y) = Y h(Y^2): with U1 = Y E + E Y, h1 <- U1 h + U h1 alongside h <- U h +
// a_k I, and out = E h + Y h1. Left products with the symmetric N x N factors use the
// transposed epilogue, (X_d F)^T = F X_d. The Frechet derivative of a polynomial of a
// symmetric matrix is self-adjoint in the Frobenius product, so the same map also carries an
// adjoint of Z_0 back to one of Y. Scratch: zo_[0..1], A1_, RHS_, P_, S_.
template <typename T>
cdmpt_status Solver<T>::tanh_tangent(Context& cx, int D, T* out, T* out_hi, T* out_lo) {
    const int N = N_;
    const int rows = D * N;
    const size_t count = (size_t)rows * ld;
    const int acc = last_acc_;
    std::vector<double> a;
    const int K = tanh_terms(last_rho_, fdx_eps(), &a);
    CDMPT_TRY(reserve_orders());
    Buf<T>& Y = Yfd_;
    Buf<T>& U = Ufd_;
    Buf<T>* hc = &zo_[1][0];
    Buf<T>* hn = &zo_[1][1];
    Buf<T>& Y1 = Z1b_;
    Buf<T>& U1 = A1_;
    Buf<T>* gc = &RHS_;
    Buf<T>* gn = &P_;
    auto zero = [&](Buf<T>& b, size_t c) -> cdmpt_status {
        CDMPT_CUDA_TRY(cudaMemsetAsync(b.x, 0, c * sizeof(T), cx.stream));
        if (b.hi) CDMPT_CUDA_TRY(cudaMemsetAsync(b.hi, 0, c * sizeof(T), cx.stream));
        if (b.lo) CDMPT_CUDA_TRY(cudaMemsetAsync(b.lo, 0, c * sizeof(T), cx.stream));
        return CDMPT_OK;
    };
    {
        Epilogue<T> ep;   // S = Y1_d Y, then U1_d = S + S^T
        CDMPT_TRY(gemm(cx, rows, N, N, Y1.op(), Y.op(), S_.x, ep, nullptr, acc));
        CDMPT_TRY(Ew<T>::transpose_add(U1.x, S_.x, N, ld, D, cx.stream, U1.hi, U1.lo));
    }
    CDMPT_TRY(zero(*hc, blk_));
    CDMPT_TRY(Ew<T>::add_diag(hc->x, N, ld, 1, a[K], cx.stream, hc->hi, hc->lo));
    CDMPT_TRY(zero(*gc, count));
    for (int k = K - 1; k >= 0; --k) {
        {   // h1 <- U1 h + U h1  (U h1_d = (h1_d U)^T)
            Epilogue<T> ep;
            ep.Dhi = gn->hi;
            ep.Dlo = gn->lo;
            CDMPT_TRY(gemm(cx, rows, N, N, U1.op(), hc->op(), gn->x, ep, nullptr, acc));
            Epilogue<T> e2;
            e2.beta = 1.0;
            e2.C = gn->x;
            e2.ldc = ld;
            e2.trans_block = N;
            e2.Dhi = gn->hi;
            e2.Dlo = gn->lo;
            CDMPT_TRY(gemm(cx, rows, N, N, gc->op(), U.op(), gn->x, e2, nullptr, acc));
        }
        {   // h <- U h + a_k I
            Epilogue<T> ep;
            ep.gamma = a[k];
            ep.Dhi = hn->hi;
            ep.Dlo = hn->lo;
            CDMPT_TRY(gemm(cx, N, N, N, U.op(), hc->op(), hn->x, ep, nullptr, acc));
        }
        std::swap(hc, hn);
        std::swap(gc, gn);
    }
    {   // Z1_0 = Y1 h + Y h1  (Y h1_d = (h1_d Y)^T)
        Epilogue<T> ep;
        CDMPT_TRY(gemm(cx, rows, N, N, Y1.op(), hc->op(), out, ep, nullptr, acc));
        Epilogue<T> e2;
        e2.beta = 1.0;
        e2.C = out;
        e2.ldc = ld;
        e2.trans_block = N;
        CDMPT_TRY(gemm(cx, rows, N, N, gc->op(), Y.op(), out, e2, nullptr, acc));
    }
    return Ew<T>::symmetrize(out, N, ld, D, cx.stream, out_hi, out_lo);
}

// Higher-order starts of the Fermi-Dirac-exact variant. With Y(lambda) = sum_q lambda^q Y^(q)
// (Y^(0) = Y, Y^(q) = -s2 (H^(q) - mu^(q) I)) the order-q Taylor coefficient of tanh Y(lambda) =
// Y(lambda) h(U(lambda)), U(lambda) = Y(lambda)^2, follows from the Horner scheme run on
// truncated power series in lambda: U^(q) = sum_{i+j=q} Y^(i) Y^(j),
//   h^(q) <- sum_{i+j=q} U^(i) h^(j) (+ a_k I for q = 0),
// and Z^(q)_0 = sum_{i+j=q} Y^(i) h^(j). Each coefficient of h is symmetric (h(lambda) is a
// polynomial of the symmetric U(lambda)), so h^(j) serves as a transposed right factor. The
// orders are updated from the top down, each into one spare buffer that then takes the old
// coefficient's place. Scratch: ao_ (U^(1..m)), P_, A1_, RHS_, Z1a_, Z1b_ (h and the spare).
template <typename T>
cdmpt_status Solver<T>::tanh_taylor(Context& cx, int m) {
    const int N = N_;
    const int acc = last_acc_;
    std::vector<double> a;
    const int K = tanh_terms(last_rho_, fdx_eps(), &a);
    Buf<T>* Yq[4] = {&Yfd_, &zo_[0][1], &zo_[1][1], &zo_[2][1]};
    Buf<T>* Uq[4] = {&Ufd_, &ao_[0], &ao_[1], &ao_[2]};
    Buf<T>* h[4] = {&P_, &A1_, &RHS_, &Z1a_};
    Buf<T>* spare = &Z1b_;
    for (int q = 1; q <= m; ++q) {   // U^(q) = S + S^T (+ Y^(q/2)^2), S = sum_{i<q-i} Y^(i) Y^(q-i)
        for (int i = 0; i < q - i; ++i) {
            Epilogue<T> ep;
            if (i > 0) {
                ep.beta = 1.0;
                ep.C = S_.x;
                ep.ldc = ld;
            }
            CDMPT_TRY(gemm(cx, N, N, N, Yq[i]->op(), Yq[q - i]->op(), S_.x, ep, nullptr, acc));
        }
        Buf<T>& U = *Uq[q];
        const bool middle = q % 2 == 0;
        CDMPT_TRY(Ew<T>::transpose_add(U.x, S_.x, N, ld, 1, cx.stream, middle ? nullptr : U.hi,
                                       middle ? nullptr : U.lo));
        if (middle) {
            Epilogue<T> ep;
            ep.beta = 1.0;
            ep.C = U.x;
            ep.ldc = ld;
            ep.Dhi = U.hi;
            ep.Dlo = U.lo;
            CDMPT_TRY(gemm(cx, N, N, N, Yq[q / 2]->op(), Yq[q / 2]->op(), U.x, ep, nullptr, acc));
        }
    }
    for (int q = 0; q <= m; ++q) {   // h = a_K I
        Buf<T>& b = *h[q];
        CDMPT_CUDA_TRY(cudaMemsetAsync(b.x, 0, blk_ * sizeof(T), cx.stream));
        if (b.hi) CDMPT_CUDA_TRY(cudaMemsetAsync(b.hi, 0, blk_ * sizeof(T), cx.stream));
        if (b.lo) CDMPT_CUDA_TRY(cudaMemsetAsync(b.lo, 0, blk_ * sizeof(T), cx.stream));
        if (q == 0) CDMPT_TRY(Ew<T>::add_diag(b.x, N, ld, 1, a[K], cx.stream, b.hi, b.lo));
    }
    for (int k = K - 1; k >= 0; --k) {
        for (int q = m; q >= 0; --q) {
            for (int i = 0; i <= q; ++i) {
                Epilogue<T> ep;
                if (i > 0) {
                    ep.beta = 1.0;
                    ep.C = spare->x;
                    ep.ldc = ld;
                }
                if (i == q) {   // the last term also rounds the split and adds a_k I (q = 0)
                    ep.gamma = q == 0 ? a[k] : 0.0;
                    ep.Dhi = spare->hi;
                    ep.Dlo = spare->lo;
                }
                CDMPT_TRY(gemm(cx, N, N, N, Uq[i]->op(), h[q - i]->op(), spare->x, ep, nullptr,
                               acc));
            }
            std::swap(h[q], spare);
        }
    }
    for (int q = 1; q <= m; ++q) {   // Z^(q)_0 = sum_{i+j=q} Y^(i) h^(j)
        Buf<T>& out = zo_[q - 1][0];
        for (int i = 0; i <= q; ++i) {
            Epilogue<T> ep;
            if (i > 0) {
                ep.beta = 1.0;
                ep.C = out.x;
                ep.ldc = ld;
            }
            CDMPT_TRY(gemm(cx, N, N, N, Yq[i]->op(), h[q - i]->op(), out.x, ep, nullptr, acc));
        }
        CDMPT_TRY(Ew<T>::symmetrize(out.x, N, ld, 1, cx.stream, out.hi, out.lo));
    }
    return CDMPT_OK;
}

// One step of the 0th-order recursion: W_k = Z_k Z_k and the correction d of
// d (I + W_k) = -2 Z_k W_k, then Z_{k+1} = sym(2 Z_k + d) with its TF32 split.
template <typename T>
cdmpt_status Solver<T>::step0(Context& cx, int k, int engine, double tol, int maxit,
                              bool make_w, bool solve, int* hint, int* iters) {
    if (make_w) {   // W_k = Z_k Z_k (symmetric)
        Epilogue<T> ep;
        ep.Dhi = W_[k].hi;
        ep.Dlo = W_[k].lo;
        ep.sym = true;
        CDMPT_TRY(gemm(cx, N_, N_, N_, Z_[k].op(), Z_[k].op(), W_[k].x, ep, nullptr, engine));
    }
    if (!solve) return CDMPT_OK;
    {   // right side of the correction: -2 Z_k W_k = -2 Z_k^3 (symmetric)
        Epilogue<T> ep;
        ep.alpha = -2.0;
        ep.sym = true;
        CDMPT_TRY(gemm(cx, N_, N_, N_, Z_[k].op(), W_[k].op(), RHS_.x, ep, nullptr, engine));
    }
    CgArgs a;
    a.W = &W_[k];
    a.rhs = RHS_.x;
    a.rows = N_;
    a.tol = tol;
    a.maxit = maxit;
    a.init_engine = a.iter_engine = engine;
    a.hint = *hint;
    // accurate solves (FP32, FP64): tolerance relative to the new iterate Z_{k+1} = 2 Z_k + d
    // as well: in the early steps the right side -2 Z_k W_k is far below Z_k, and its own
    // relative tolerance would solve d to digits that Z_{k+1} cannot hold. The one-pass sweeps
    // of the mixed precisions keep theirs: their traces steer mu before the refinement.
    if (tol <= 1e-6) {
        a.ref = Z_[k].x;
        a.ref_scale = 2.0;
        a.tol_ref = tol;
    }
    // mirrored CG products only in the one-pass sweeps that are refined afterwards:
    // the iterates drift from commuting with W_k at rounding level, and the mirrored
    // operator is then not self-adjoint (measured: FP32-mode P1 errors doubled)
    a.sym = engine == CDMPT_GEMM_TC_TF32 || engine == CDMPT_GEMM_TC_BF16;
    int it = 0;
    CDMPT_TRY(cg(cx, Z_[k + 1].x, a, &it, nullptr));   // d, in the Z_{k+1} buffer
    *iters += it;
    *hint = std::max(1, it);
    CDMPT_TRY(Ew<T>::axpby(Z_[k + 1].x, Z_[k].x, blk_, 2.0, 1.0, nullptr, cx.stream));
    CDMPT_TRY(Ew<T>::symmetrize(Z_[k + 1].x, N_, ld, 1, cx.stream, Z_[k + 1].hi, Z_[k + 1].lo));
    // a sweep step leaves an FP32 iterate: the low part of a pair-stored one is zero
    if (Z_[k + 1].xl) CDMPT_CUDA_TRY(cudaMemsetAsync(Z_[k + 1].xl, 0, blk_ * sizeof(T), cx.stream));
    return CDMPT_OK;
}

// One 0th-order pass of Algorithm 1 at chemical potential mu: Z_0 .. Z_n, A_0 .. A_{n-1}.
// With checkpointing the segment buffers end up holding the last segment.
template <typename T>
cdmpt_status Solver<T>::sweep(Context& cx, const double* H0, double mu, double s2,
                              const cdmpt_opts& o, int n, int engine, double tol,
                              int* cg_iters) {
    CDMPT_TRY(init_z0(cx, H0, mu, s2, s2 * std::max(gmax_ - mu, mu - gmin_), acc_cur_));
    int total = 0, hint = 1;
    for (int k = 0; k < n; ++k)
        CDMPT_TRY(step0(cx, k, engine, tol, o.cg_maxit, true, true, &hint, &total));
    seg_ = ck_ ? (n - 1) / ck_ : -1;
    *cg_iters = total;
    return CDMPT_OK;
}

// Checkpointed trajectory: recompute segment j = k / ck_ from its checkpoint
// Z_{j ck_} at the final mu, with the engine and tolerance of the final sweep
// (the CG runs the same iterations on the same data, so the recomputed Z_k
// equal the sweep's up to the summation order of the device reductions). W_0
// is kept; the segment's last step ends on the next checkpoint (or Z_n), so it
// needs W only.
template <typename T>
cdmpt_status Solver<T>::need(Context& cx, int k) {
    if (ck_ == 0) return CDMPT_OK;
    const int j = k / ck_;
    if (j == seg_) return CDMPT_OK;
    const int k0 = j * ck_, k1 = std::min(k0 + ck_, last_n_);
    int hint = 1, iters = 0;
    seg_ = -1;   // invalid while being rewritten
    for (int i = k0; i < k1; ++i)
        CDMPT_TRY(step0(cx, i, last_acc_, last_sweep_tol_, last_opts_.cg_maxit, i > 0, i + 1 < k1,
                        &hint, &iters));
    replay_iters_ += iters;
    seg_ = j;
    return CDMPT_OK;
}

// Z_k += d and symmetrise; a pair-stored Z_k takes the correction without rounding the sum
// to FP32.
template <typename T>
cdmpt_status Solver<T>::correct(Context& cx, int k, const T* d) {
    if constexpr (sizeof(T) == 4) {
        if (Z_[k].xl) {
            CDMPT_TRY(pair::add(Z_[k].x, Z_[k].xl, d, blk_, cx.stream));
            return pair::symmetrize(Z_[k].x, Z_[k].xl, N_, ld, 1, cx.stream, Z_[k].hi, Z_[k].lo);
        }
    }
    CDMPT_TRY(Ew<T>::axpby(Z_[k].x, d, blk_, 1.0, 1.0, nullptr, cx.stream));
    return Ew<T>::symmetrize(Z_[k].x, N_, ld, 1, cx.stream, Z_[k].hi, Z_[k].lo);
}

// One refinement pass over the stored trajectory (mixed precision). For each step, with
// Z_k already refined: the step matrix A_k = I + W_k from the refined Z_k and the residual
// r = 2 Z_k - Z_{k+1} - Z_{k+1} W_k of the stored Z_{k+1} (Algorithm 1's per-step system in
// the deviation form), then the correction d (I + W_k) = r by CG with one-pass TF32 products,
// added to Z_{k+1}. Steps k < k_hp form W_k and r with split-TF32 products (with pair
// storage the linear part 2 Z_k - Z_{k+1} comes from the pairs; both carry an error of
// about 2^-22 ||Z_k||^2 relative to Z_k, small while ||Z_k|| is); steps k >= k_hp with the
// Ozaki-sliced products of the pair-stored trajectory (FP64-class: about 2^-31, and free of
// the truncation bias of FP32 tensor-core accumulation).
template <typename T>
cdmpt_status Solver<T>::refine(Context& cx, const cdmpt_opts& o, int n, int k_hp, int* cg_iters,
                               double* max_rel_res) {
    int total = 0;
    double worst = 0.0;
    for (int k = 0; k < n; ++k) {
        if (k >= k_hp) {
            CDMPT_TRY(residual_hp(cx, k));
        } else {
            {   // W_k from the refined Z_k
                Epilogue<T> ep;
                ep.Dhi = W_[k].hi;
                ep.Dlo = W_[k].lo;
                ep.sym = true;
                CDMPT_TRY(gemm(cx, N_, N_, N_, Z_[k].op(), Z_[k].op(), W_[k].x, ep, nullptr,
                               CDMPT_GEMM_TC_3XTF32));
            }
            // linear part 2 Z_k - Z_{k+1}: it is small, of the size of Z_{k+1} W_k, so its
            // FP32 rounding is at the level of the product's
            if constexpr (sizeof(T) == 4) {
                if (Z_[k].xl)
                    CDMPT_TRY(pair::lincomb(S_.x, 2.0, Z_[k].x, Z_[k].xl, -1.0, Z_[k + 1].x,
                                            Z_[k + 1].xl, blk_, cx.stream));
                else
                    CDMPT_TRY(Ew<T>::lincomb(S_.x, Z_[k].x, 2.0, Z_[k + 1].x, -1.0, blk_,
                                             cx.stream));
            } else {
                CDMPT_TRY(Ew<T>::lincomb(S_.x, Z_[k].x, 2.0, Z_[k + 1].x, -1.0, blk_, cx.stream));
            }
            {   // full tiles: the stored Z_{k+1} differs from the exact one by an error that
                // does not commute with W_k, so Z_{k+1} W_k is not symmetric and its upper
                // triangle alone would change the correction at first order
                Epilogue<T> ep;
                ep.alpha = -1.0;
                ep.beta = 1.0;
                ep.C = S_.x;
                ep.ldc = ld;
                CDMPT_TRY(gemm(cx, N_, N_, N_, Z_[k + 1].op(), W_[k].op(), RHS_.x, ep, nullptr,
                               CDMPT_GEMM_TC_3XTF32));
            }
        }
        // correction d (I + W_k) = r with one-pass TF32 iterations
        CgArgs a;
        a.W = &W_[k];
        a.rhs = RHS_.x;
        a.rows = N_;
        a.tol = 1e-3;      // one-pass TF32 iterations gain about three digits
        a.maxit = o.cg_maxit;
        a.init_engine = a.iter_engine = CDMPT_GEMM_TC_TF32;
        a.hint = 2;
        int it = 0;
        CDMPT_TRY(cg(cx, A1_.x, a, &it, nullptr));
        total += it;
        // relative size of the residual: |r| / |2 Z_k| (host-side from CG scalars)
        const double bb = cx.pinned[CG_BB];
        CDMPT_CUDA_TRY(cudaMemsetAsync(sc_ + S_ZZ, 0, sizeof(double), cx.stream));
        CDMPT_TRY(Ew<T>::dot(Z_[k].x, Z_[k].x, blk_, sc_ + S_ZZ, nullptr, cx.stream));
        CDMPT_TRY(read_scalars(cx, sc_, S_NSLOTS));
        const double zz = cx.pinned[S_ZZ];
        if (zz > 0) worst = std::max(worst, std::sqrt(bb / (4.0 * zz)));
        CDMPT_TRY(correct(cx, k + 1, A1_.x));
    }
    *cg_iters = total;
    *max_rel_res = worst;
    return CDMPT_OK;
}

// Z_0 += shift I (a Newton step on mu moves Z_0 = -s2 (H0 - mu I) by s2 dmu I)
template <typename T>
cdmpt_status Solver<T>::shift_z0(Context& cx, double shift) {
    if constexpr (sizeof(T) == 4) {
        if (Z_[0].xl)
            return pair::add_diag(Z_[0].x, Z_[0].xl, N_, ld, 1, shift, cx.stream, Z_[0].hi,
                                  Z_[0].lo);
    }
    return Ew<T>::add_diag(Z_[0].x, N_, ld, 1, shift, cx.stream, Z_[0].hi, Z_[0].lo);
}

// P0 = (I + Z_n) / 2 in FP64 (device array, leading dimension ldo)
template <typename T>
cdmpt_status Solver<T>::p0_out(Context& cx, double* out, int ldo) {
    const int n = last_n_;
    if constexpr (sizeof(T) == 4) {
        if (Z_[n].xl)
            return pair::to_f64(out, ldo, Z_[n].x, Z_[n].xl, ld, N_, N_, 0.5, 0.5, cx.stream);
    }
    return Ew<T>::to_f64(out, ldo, Z_[n].x, ld, N_, N_, 0.5, 0.5, cx.stream);
}

template <typename T>
cdmpt_status Solver<T>::gemm_hp(Context& cx, const OzOperand& X, const OzOperand& Y,
                                const OzEpi& ep) {
    // a symmetric result computes the tiles of the upper triangle: N (N + 1) N, as for the
    // symmetric TF32 products
    const double flops = ep.sym ? (double)N_ * (N_ + 1) * N_ : 2.0 * N_ * (double)N_ * N_;
    cudaEvent_t e1 = nullptr;
    if (cx.profile) {
        while (cx.ev.size() < 2 * (cx.ev_used + 1)) {
            cudaEvent_t e;
            CDMPT_CUDA_TRY(cudaEventCreate(&e));
            cx.ev.push_back(e);
        }
        if (cx.ev_ok.size() < cx.ev_used + 1) {
            cx.ev_ok.resize(cx.ev_used + 1);
            cx.ev_engine.resize(cx.ev_used + 1);
            cx.ev_flops.resize(cx.ev_used + 1);
        }
        cx.ev_ok[cx.ev_used] = 1;
        cx.ev_engine[cx.ev_used] = CDMPT_GEMM_TC_OZAKI;
        cx.ev_flops[cx.ev_used] = flops;
        e1 = cx.ev[2 * cx.ev_used + 1];
        CDMPT_CUDA_TRY(cudaEventRecord(cx.ev[2 * cx.ev_used], cx.stream));
    }
    CDMPT_TRY(gemm_oz(N_, N_, N_, X, Y, ep, cx.stream));
    if (cx.profile) {
        CDMPT_CUDA_TRY(cudaEventRecord(e1, cx.stream));
        ++cx.ev_used;
    }
    if (cx.st) {
        cx.st->gemm_launches += 1;
        cx.st->gemm_flops += flops;
        cx.st->tensor_flops += (double)oz_products(kOzDigits) * flops;   // BF16 digit products
    }
    return CDMPT_OK;
}

// W_k = Z_k Z_k and r = 2 Z_k - Z_{k+1} - Z_{k+1} W_k (into RHS_) from Ozaki-sliced products
// of the pair-stored trajectory: the FP32 part and TF32 split of W_k replace the stored W_k, its
// low part goes to wl_, and the linear part of r is formed in double-float in the epilogue.
template <typename T>
cdmpt_status Solver<T>::residual_hp(Context& cx, int k) {
    if constexpr (sizeof(T) != 4) {
        set_error("FP64-class residuals need the pair-stored FP32 trajectory");
        return CDMPT_ERR_UNSUPPORTED;
    } else {
        if (!pairs_ || !Z_[k].xl) {
            set_error("FP64-class residuals need the pair-stored FP32 trajectory");
            return CDMPT_ERR_UNSUPPORTED;
        }
        CDMPT_TRY(oz_slice(Z_[k].x, Z_[k].xl, N_, N_, ld, oz_[0], cx.stream));
        {
            OzEpi ep;
            ep.sym = 1;   // W_k = Z_k Z_k: upper-triangle tiles, mirrored
            ep.D = W_[k].x;
            ep.Dl = wl_;
            ep.Dthi = W_[k].hi;
            ep.Dtlo = W_[k].lo;
            ep.ldd = ld;
            CDMPT_TRY(gemm_hp(cx, oz_[0], oz_[0], ep));
        }
        CDMPT_TRY(oz_slice(W_[k].x, wl_, N_, N_, ld, oz_[1], cx.stream));
        CDMPT_TRY(oz_slice(Z_[k + 1].x, Z_[k + 1].xl, N_, N_, ld, oz_[2], cx.stream));
        OzEpi ep;
        ep.D = RHS_.x;
        ep.ldd = ld;
        ep.alpha = -1.f;
        ep.b1 = 2.f;
        ep.c1h = Z_[k].x;
        ep.c1l = Z_[k].xl;
        ep.b2 = -1.f;
        ep.c2h = Z_[k + 1].x;
        ep.c2l = Z_[k + 1].xl;
        ep.ldc = ld;
        return gemm_hp(cx, oz_[2], oz_[1], ep);
    }
}

template <typename T>
cdmpt_status Solver<T>::occupation(Context& cx, int n, double* trP, double* zz) {
    CDMPT_CUDA_TRY(cudaMemsetAsync(sc_ + S_TRZ, 0, 2 * sizeof(double), cx.stream));
    CDMPT_TRY(Ew<T>::trace(Z_[n].x, N_, ld, 1, sc_ + S_TRZ, cx.stream));
    if (Z_[n].xl) CDMPT_TRY(Ew<T>::trace(Z_[n].xl, N_, ld, 1, sc_ + S_TRZ, cx.stream));
    CDMPT_TRY(Ew<T>::dot(Z_[n].x, Z_[n].x, blk_, sc_ + S_ZZ, nullptr, cx.stream));
    CDMPT_TRY(read_scalars(cx, sc_, S_NSLOTS));
    *trP = 0.5 * (N_ + cx.pinned[S_TRZ]);
    *zz = cx.pinned[S_ZZ];
    return CDMPT_OK;
}

// Q = dP0/dmu = beta/4 (I - Z_n^2)(I - Z_0^2)^-1 for the stored trajectory,
// by CG with the operator X - X W_0.
template <typename T>
cdmpt_status Solver<T>::compute_q(Context& cx) {
    const int n = last_n_, N = N_;
    const double beta = last_beta_;
    const int acc = last_acc_;
    const cdmpt_opts& o = last_opts_;
    cdmpt_stats& st = *cx.st;
    // right side beta/4 (I - Z_n^2): for saturated levels 1 - z^2 cancels to a small value, so
    // the pair-stored trajectory forms I - Z_n^2 with the Ozaki-sliced product (an FP32-class
    // product's error, relative to the O(1) terms, would dominate Tr Q and hence mu1)
    double rhs_scale = 1.0;
    bool hp_rhs = false;
    if constexpr (sizeof(T) == 4) {
        if (pairs_ && Z_[n].xl) {
            CDMPT_TRY(oz_slice(Z_[n].x, Z_[n].xl, N_, N_, ld, oz_[0], cx.stream));
            OzEpi ep;
            ep.sym = 1;   // I - Z_n Z_n: upper-triangle tiles, mirrored
            ep.D = RHS_.x;
            ep.Dthi = RHS_.hi;
            ep.Dtlo = RHS_.lo;
            ep.ldd = ld;
            ep.alpha = -1.f;
            ep.gamma = 1.f;
            CDMPT_TRY(gemm_hp(cx, oz_[0], oz_[0], ep));
            rhs_scale = 0.25 * beta;
            hp_rhs = true;
        }
    }
    if (!hp_rhs) {
        Epilogue<T> ep;
        ep.alpha = -0.25 * beta;
        ep.gamma = 0.25 * beta;
        ep.Dhi = RHS_.hi;
        ep.Dlo = RHS_.lo;
        ep.sym = true;
        CDMPT_TRY(gemm(cx, N, N, N, Z_[n].op(), Z_[n].op(), RHS_.x, ep, nullptr, acc));
    }
    if (fdx_) {   // Z_0 = tanh(Y): dZ_0/dmu = s2 (I - Z_0^2), so Q = beta/4 (I - Z_n^2) = beta P0 (I - P0)
        CDMPT_TRY(Ew<T>::axpby(Qmu_.x, RHS_.x, blk_, rhs_scale, 0.0, nullptr, cx.stream));
        st.cg_iterations_q = 0;
        q_valid_ = true;
        return CDMPT_OK;
    }
    CgArgs a;   // (I - W_0) Q = beta/4 (I - Z_n^2), i.e. operator X - X W_0
    a.W = &W_[0];
    a.s = 1.0;
    a.t = -1.0;
    a.x0 = &RHS_;
    a.x0_scale = rhs_scale;
    a.rhs = RHS_.x;
    a.rhs_scale = rhs_scale;
    a.rows = N;
    a.tol = o.cg_tol;
    a.maxit = o.cg_maxit;
    a.init_engine = a.iter_engine = acc;
    a.sym = true;
    int it = 0;
    CDMPT_TRY(cg(cx, Qmu_.x, a, &it, nullptr));
    st.cg_iterations_q = it;
    CDMPT_TRY(Ew<T>::symmetrize(Qmu_.x, N, ld, 1, cx.stream));
    q_valid_ = true;
    return CDMPT_OK;
}

// Reverse sweep. With Zh_{k+1} the (symmetric) adjoint of Z_{k+1}, the step
// Z_{k+1} = 2 A_k^-1 Z_k, whose tangent is A_k dZ_{k+1} = 2 dZ_k - (Z_k dZ_k +
// dZ_k Z_k) Z_{k+1}, gives with V = Zh_{k+1} A_k^-1 (one CG solve)
//   Zh_k = sym(2 V - Z_{k+1} V Z_k - Z_k Z_{k+1} V).
// Left products use the TN kernel with transposed right factors:
// Z_k V^T = gemm(Z_k, V), Z_{k+1} V Z_k = gemm(Z_{k+1}, Z_k V^T), B V = gemm(B, V^T).
// Z_0 = -s2 (H0 - mu I) and the canonical dmu = Tr(Q dH0) / Tr Q give
//   grad = -s2 Zh_0 + s2 Tr(Zh_0) Q / Tr Q.
// With the Fermi-Dirac-exact start Z_0 = tanh(Y), Y = -s2 (H0 - mu I), the adjoint of Y is
// Yh = Dtanh(Y)[Zh_0] (the derivative is self-adjoint), and the same formula holds with Yh
// for Zh_0: Tr Yh = <Zh_0, Dtanh(Y)[I]> is the mu-sensitivity through the start.
template <typename T>
cdmpt_status Solver<T>::vjp_p0(Context& cx, const double* G0, double* grad, double p0_weight) {
    if (!traj_valid_) {
        set_error("vjp: no completed solve on this handle");
        return CDMPT_ERR_ARG;
    }
    const int n = last_n_, N = N_;
    const int acc = last_acc_;
    const cdmpt_opts& o = last_opts_;
    // Zh_n = 1/2 sym(G0)   (P0 = (I + Z_n) / 2)
    CDMPT_TRY(Ew<T>::init_z(Zh_.x, G0, N, ld, N, 1, 0.5, 0.0, cx.stream));
    CDMPT_TRY(Ew<T>::symmetrize(Zh_.x, N, ld, 1, cx.stream));
    Buf<T>& V = Z1a_;
    Buf<T>& VT = Z1b_;
    Buf<T>& M1T = A1_;
    Buf<T>& B = RHS_;
    for (int k = n - 1; k >= 0; --k) {
        CDMPT_TRY(need(cx, k));   // checkpointing: each segment recomputed once, last first
        CgArgs a;
        a.W = &W_[k];
        a.rhs = Zh_.x;
        a.rows = N;
        a.tol = o.cg_tol;
        a.maxit = o.cg_maxit;
        a.init_engine = a.iter_engine = acc;
        a.hint = 2;
        int it = 0;
        CDMPT_TRY(cg(cx, V.x, a, &it, nullptr));
        if constexpr (sizeof(T) == 4) CDMPT_TRY(split_tf32(V.x, blk_, V.hi, V.lo, cx.stream));
        CDMPT_TRY(Ew<T>::transpose(VT.x, V.x, N, ld, 1, cx.stream, VT.hi, VT.lo));
        {
            Epilogue<T> ep;   // Z_k V^T
            ep.Dhi = M1T.hi;
            ep.Dlo = M1T.lo;
            CDMPT_TRY(gemm(cx, N, N, N, Z_[k].op(), V.op(), M1T.x, ep, nullptr, acc));
        }
        {
            Epilogue<T> ep;   // Z_{k+1} V Z_k
            CDMPT_TRY(gemm(cx, N, N, N, Z_[k + 1].op(), M1T.op(), S_.x, ep, nullptr, acc));
        }
        {
            Epilogue<T> ep;   // B = Z_k Z_{k+1}
            ep.Dhi = B.hi;
            ep.Dlo = B.lo;
            CDMPT_TRY(gemm(cx, N, N, N, Z_[k].op(), Z_[k + 1].op(), B.x, ep, nullptr, acc));
        }
        CDMPT_TRY(Ew<T>::lincomb(S_.x, V.x, 2.0, S_.x, -1.0, blk_, cx.stream));   // 2V - Z'VZ
        {
            Epilogue<T> ep;   // Zh_k = 2V - Z'VZ - B V
            ep.alpha = -1.0;
            ep.beta = 1.0;
            ep.C = S_.x;
            ep.ldc = ld;
            CDMPT_TRY(gemm(cx, N, N, N, B.op(), VT.op(), Zh_.x, ep, nullptr, acc));
        }
        CDMPT_TRY(Ew<T>::symmetrize(Zh_.x, N, ld, 1, cx.stream));
    }
    if (fdx_) {   // Zh_0 -> Yh = Dtanh(Y)[Zh_0]
        CDMPT_CUDA_TRY(cudaMemcpyAsync(Z1b_.x, Zh_.x, blk_ * sizeof(T),
                                       cudaMemcpyDeviceToDevice, cx.stream));
        if constexpr (sizeof(T) == 4)
            CDMPT_TRY(split_tf32(Z1b_.x, blk_, Z1b_.hi, Z1b_.lo, cx.stream));
        CDMPT_TRY(tanh_tangent(cx, 1, Zh_.x, nullptr, nullptr));
    }
    // canonical: mu follows H0 through Tr P0 = N_occ (the Q term); grand canonical: fixed mu
    const bool gc = o.grand_canonical != 0;
    if (!q_valid_ && !gc) CDMPT_TRY(compute_q(cx));
    CDMPT_CUDA_TRY(cudaMemsetAsync(sc_ + S_TRQ, 0, 2 * sizeof(double), cx.stream));
    if (!gc) CDMPT_TRY(Ew<T>::trace(Qmu_.x, N, ld, 1, sc_ + S_TRQ, cx.stream));
    CDMPT_TRY(Ew<T>::trace(Zh_.x, N, ld, 1, sc_ + S_TRQ + 1, cx.stream));
    CDMPT_TRY(read_scalars(cx, sc_, S_NSLOTS));
    const double trQ = cx.pinned[S_TRQ], trZh = cx.pinned[S_TRQ + 1];
    const double c = (!gc && trQ > 0) ? last_s2_ * trZh / trQ : 0.0;
    CDMPT_TRY(Ew<T>::lincomb(Zh_.x, Zh_.x, -last_s2_, Qmu_.x, c, blk_, cx.stream));
    // optional + p0_weight P0 = p0_weight (I + Z_n) / 2, added in the padded buffer (the
    // identity part through the diagonal shift of the FP64 conversion)
    if (p0_weight != 0.0)
        CDMPT_TRY(Ew<T>::axpby(Zh_.x, Z_[n].x, blk_, 0.5 * p0_weight, 1.0, nullptr, cx.stream));
    CDMPT_TRY(Ew<T>::to_f64(grad, N, Zh_.x, ld, N, N, 1.0, 0.5 * p0_weight, cx.stream));
    CDMPT_CUDA_TRY(cudaStreamSynchronize(cx.stream));
    return check_device_error(cx.stream);
}

template <typename T>
cdmpt_status Solver<T>::reserve_orders() {
    if (orders_ready_) return CDMPT_OK;
    auto buf = [&](Buf<T>* b) -> cdmpt_status {
        *b = Buf<T>();
        const int parts = sizeof(T) == 4 ? 3 : 1;
        T* q[3] = {nullptr, nullptr, nullptr};
        for (int i = 0; i < parts; ++i) {
            void* p = nullptr;
            if (cudaMalloc(&p, blk_ * sizeof(T)) != cudaSuccess) {
                cudaGetLastError();
                set_error("device allocation for the higher-order response failed");
                return CDMPT_ERR_OOM;
            }
            if (cudaMemset(p, 0, blk_ * sizeof(T)) != cudaSuccess) return CDMPT_ERR_CUDA;
            allocs_.push_back(p);
            q[i] = (T*)p;
        }
        b->x = q[0];
        b->hi = q[1];
        b->lo = q[2];
        return CDMPT_OK;
    };
    for (int q = 0; q < 3; ++q) {
        CDMPT_TRY(buf(&zo_[q][0]));
        CDMPT_TRY(buf(&zo_[q][1]));
        CDMPT_TRY(buf(&ao_[q]));
    }
    CDMPT_TRY(buf(&G_));
    CDMPT_TRY(buf(&Yfd_));
    CDMPT_TRY(buf(&Ufd_));
    orders_ready_ = true;
    return CDMPT_OK;
}

// Joint forward sweep of the perturbation orders 1..m (the inner loop of
// Algorithm 1 to third order, with H^(q) = 0 for q >= 2) in the deviation form.
// With Z(lambda) = sum_q lambda^q Z^(q) and A = I + Z^2, the order-q part of
// A_k Z_{k+1} = 2 Z_k reads
//   A_k Z^(q)_{k+1} = 2 Z^(q)_k - sum_{j=1..q} A^(j)_k Z^(q-j)_{k+1},
//   A^(j)_k = sum_{i=0..j} Z^(i)_k Z^(j-i)_k   (Z^(0) = Z, the trajectory),
// the deviation-form image of the paper's C^(m) and B^(m) terms. Each order is
// solved in correction form d (I + W_k) = -sum_j Z^(q-j)_{k+1} A^(j)_k -
// 2 Z^(q)_k W_k, Z^(q)_{k+1} = sym(2 Z^(q)_k + d), lower orders first, all with
// the same step matrix. Start: Z^(1)_0 = -s2 (H1 - mu1 I), Z^(q)_0 = s2 mu^(q) I
// for q >= 2 (minus s2 H^(q) where given); with the Fermi-Dirac-exact start these are the
// Y^(q) of tanh_taylor. Only the current and next iterate of each order are kept.
template <typename T>
cdmpt_status Solver<T>::orders(Context& cx, const double* H1d, const double* H2d,
                               const double* H3d, int m, const double* mus) {
    const int n = last_n_, N = N_;
    const int acc = last_acc_;
    const cdmpt_opts& o = last_opts_;
    auto cur = [&](int q) -> Buf<T>& { return zo_[q - 1][cur_[q - 1]]; };
    auto nxt = [&](int q) -> Buf<T>& { return zo_[q - 1][1 - cur_[q - 1]]; };
    auto mu_of = [&](int q) { return q < m ? mus[q - 1] : 0.0; };
    for (int q = 1; q <= m; ++q) cur_[q - 1] = 0;
    // the linear starts Y^(q) = -s2 (H^(q) - mu^(q) I); the Fermi-Dirac-exact start keeps them
    // in the next-iterate buffers and maps them through the Taylor coefficients of tanh
    auto start = [&](int q) -> Buf<T>& { return fdx_ ? nxt(q) : cur(q); };
    CDMPT_TRY(Ew<T>::init_z(start(1).x, H1d, N, ld, ld, 1, -last_s2_, mu_of(1), cx.stream,
                            start(1).hi, start(1).lo));
    for (int q = 2; q <= m; ++q) {
        Buf<T>& b = start(q);
        const double* Hq = q == 2 ? H2d : H3d;
        if (Hq) {   // Z^(q)_0 = -s2 (H^(q) - mu^(q) I)
            CDMPT_TRY(Ew<T>::init_z(b.x, Hq, N, ld, ld, 1, -last_s2_, mu_of(q), cx.stream, b.hi,
                                    b.lo));
            continue;
        }
        CDMPT_CUDA_TRY(cudaMemsetAsync(b.x, 0, blk_ * sizeof(T), cx.stream));
        if (b.hi) CDMPT_CUDA_TRY(cudaMemsetAsync(b.hi, 0, blk_ * sizeof(T), cx.stream));
        if (b.lo) CDMPT_CUDA_TRY(cudaMemsetAsync(b.lo, 0, blk_ * sizeof(T), cx.stream));
        if (mu_of(q) != 0.0)
            CDMPT_TRY(Ew<T>::add_diag(b.x, N, ld, 1, last_s2_ * mu_of(q), cx.stream, b.hi, b.lo));
    }
    if (fdx_) CDMPT_TRY(tanh_taylor(cx, m));
    int hint[3] = {1, 1, 1};
    for (int k = 0; k < n; ++k) {
        CDMPT_TRY(need(cx, k));
        // A^(q)_k from the step-k iterates: S = Z^(q) Z + sum_{1 <= i < q-i} Z^(q-i) Z^(i)
        // (products X Y^T with Y symmetric), A^(q) = S + S^T, plus Z^(q/2) Z^(q/2) for even q
        for (int q = 1; q <= m; ++q) {
            {
                Epilogue<T> ep;
                CDMPT_TRY(gemm(cx, N, N, N, cur(q).op(), Z_[k].op(), S_.x, ep, nullptr, acc));
            }
            for (int i = 1; i < q - i; ++i) {
                Epilogue<T> ep;
                ep.beta = 1.0;
                ep.C = S_.x;
                ep.ldc = ld;
                CDMPT_TRY(gemm(cx, N, N, N, cur(q - i).op(), cur(i).op(), S_.x, ep, nullptr, acc));
            }
            Buf<T>& A = ao_[q - 1];
            const bool middle = q % 2 == 0;
            CDMPT_TRY(Ew<T>::transpose_add(A.x, S_.x, N, ld, 1, cx.stream, middle ? nullptr : A.hi,
                                           middle ? nullptr : A.lo));
            if (middle) {   // += Z^(q/2) Z^(q/2), with the split for A's use as a left factor
                Epilogue<T> ep;
                ep.beta = 1.0;
                ep.C = A.x;
                ep.ldc = ld;
                ep.Dhi = A.hi;
                ep.Dlo = A.lo;
                CDMPT_TRY(gemm(cx, N, N, N, cur(q / 2).op(), cur(q / 2).op(), A.x, ep, nullptr,
                               acc));
            }
        }
        for (int q = 1; q <= m; ++q) {
            // RHS = -sum_{j=1..q} Z^(q-j)_{k+1} A^(j)_k = -sum_j (A^(j)_k Z^(q-j)_{k+1})^T
            for (int j = 1; j <= q; ++j) {
                const Buf<T>& Zn = j == q ? Z_[k + 1] : nxt(q - j);
                Epilogue<T> ep;
                ep.alpha = -1.0;
                if (j > 1) {
                    ep.beta = 1.0;
                    ep.C = RHS_.x;
                    ep.ldc = ld;
                }
                ep.trans_block = N;
                CDMPT_TRY(gemm(cx, N, N, N, ao_[j - 1].op(), Zn.op(), RHS_.x, ep, nullptr, acc));
            }
            {   // -= 2 Z^(q)_k W_k
                Epilogue<T> ep;
                ep.alpha = -2.0;
                ep.beta = 1.0;
                ep.C = RHS_.x;
                ep.ldc = ld;
                CDMPT_TRY(gemm(cx, N, N, N, cur(q).op(), W_[k].op(), RHS_.x, ep, nullptr, acc));
            }
            CgArgs a;
            a.W = &W_[k];
            a.rhs = RHS_.x;
            a.rows = N;
            a.tol = o.cg_tol;
            a.maxit = o.cg_maxit;
            a.init_engine = a.iter_engine = acc;
            a.hint = hint[q - 1];
            int it = 0;
            Buf<T>& Zq = nxt(q);
            CDMPT_TRY(cg(cx, Zq.x, a, &it, nullptr));
            hint[q - 1] = std::max(1, it);
            CDMPT_TRY(Ew<T>::axpby(Zq.x, cur(q).x, blk_, 2.0, 1.0, nullptr, cx.stream));
            CDMPT_TRY(Ew<T>::symmetrize(Zq.x, N, ld, 1, cx.stream, Zq.hi, Zq.lo));
        }
        for (int q = 1; q <= m; ++q) cur_[q - 1] ^= 1;
    }
    return CDMPT_OK;
}

// Canonical response of order m = 1, 2 or 3 per direction (m = 1: a first-order pass for
// perturbations other than the solve's, on the stored trajectory). P^(m) is linear in
// mu^(m) with slope Q = dP0/dmu (Z^(m)_0 = s2 mu^(m) I enters through the same
// tangent map as a uniform shift of Z_0), so one sweep with mu^(m) = 0 gives
// mu^(m) = -Tr P^(m)|_0 / Tr Q and P^(m) = Z^(m)_n / 2 + mu^(m) Q. Order 3 needs
// mu2 first, from an order-2 sweep. Omega^(m+1) = 1/(m+1) Tr[H1 P^(m)] (Eq.
// Resp_0 with H^(1) = H1 only).
template <typename T>
cdmpt_status Solver<T>::higher(Context& cx, const double* H1, int D, int m, const double* w,
                               double* Pm, double* mu_out, double* omega, double* grad,
                               const double* H2, const double* H3, const double* mu1s) {
    if (grad && (H2 || H3)) {
        set_error("the polarizability gradient is d alpha / d H0 for H^(2) = H^(3) = 0: clear "
                  "the higher perturbation terms first");
        return CDMPT_ERR_ARG;
    }
    if (!traj_valid_ || D < 1 || (m > 1 && !mu1s && (int)last_mu1_.size() < D)) {
        set_error("higher-order response: no completed solve with perturbations on this handle");
        return CDMPT_ERR_ARG;
    }
    const int N = N_;
    const cdmpt_opts& o = last_opts_;
    CDMPT_TRY(reserve_orders());
    const bool gc = o.grand_canonical != 0;   // fixed mu: mu^(m) = 0, no Q term
    if (!q_valid_ && !gc) CDMPT_TRY(compute_q(cx));
    CDMPT_CUDA_TRY(cudaMemsetAsync(sc_ + S_TRQ, 0, sizeof(double), cx.stream));
    if (!gc) CDMPT_TRY(Ew<T>::trace(Qmu_.x, N, ld, 1, sc_ + S_TRQ, cx.stream));
    CDMPT_TRY(read_scalars(cx, sc_, S_NSLOTS));
    const double trQ = cx.pinned[S_TRQ];
    if (!gc && !(trQ > 0)) {
        set_error("higher-order response: Tr dP0/dmu is not positive");
        return CDMPT_ERR_NO_CONVERGENCE;
    }
    if (grad) CDMPT_CUDA_TRY(cudaMemsetAsync(G_.x, 0, blk_ * sizeof(T), cx.stream));
    for (int d = 0; d < D; ++d) {
        const double* H1d = H1 + (size_t)d * blk_;
        const double* H2d = H2 ? H2 + (size_t)d * blk_ : nullptr;
        const double* H3d = H3 ? H3 + (size_t)d * blk_ : nullptr;
        double mus[2] = {m > 1 ? (mu1s ? mu1s[d] : last_mu1_[d]) : 0.0, 0.0};
        for (int q = std::min(m, 2); q <= m; ++q) {
            CDMPT_TRY(orders(cx, H1d, H2d, H3d, q, mus));
            Buf<T>& Zq = zo_[q - 1][cur_[q - 1]];
            CDMPT_CUDA_TRY(cudaMemsetAsync(sc_ + S_TRQ + 1, 0, sizeof(double), cx.stream));
            CDMPT_TRY(Ew<T>::trace(Zq.x, N, ld, 1, sc_ + S_TRQ + 1, cx.stream));
            CDMPT_TRY(read_scalars(cx, sc_, S_NSLOTS));
            const double muq = gc ? 0.0 : -0.5 * cx.pinned[S_TRQ + 1] / trQ;
            if (q < m) {
                mus[q - 1] = muq;
                continue;
            }
            if (mu_out) mu_out[d] = muq;
            // Z^(m) += 2 mu^(m) Q  (P^(m) = Z^(m) / 2)
            if (!gc) CDMPT_TRY(Ew<T>::axpby(Zq.x, Qmu_.x, blk_, 2.0 * muq, 1.0, nullptr, cx.stream));
            if (omega) {
                // Eq. Resp_0: Omega^(m+1) = 1/(m+1) sum_k k Tr[H^(k) P^(m+1-k)], with
                // P^(q) = Z^(q)_n / 2 (q >= 1, canonical shifts included) and P0 = (I + Z_n)/2
                CDMPT_CUDA_TRY(cudaMemsetAsync(sc_ + S_FE, 0, 5 * sizeof(double), cx.stream));
                CDMPT_TRY(Ew<T>::dot_h(Zq.x, H1d, N, ld, ld, sc_ + S_FE, cx.stream));
                if (m == 1 && H2d) {
                    CDMPT_TRY(Ew<T>::dot_h(Z_[last_n_].x, H2d, N, ld, ld, sc_ + S_FE + 1, cx.stream));
                    CDMPT_TRY(Ew<double>::trace(H2d, N, ld, 1, sc_ + S_FE + 2, cx.stream));
                }
                if (m >= 2 && H2d)
                    CDMPT_TRY(Ew<T>::dot_h(zo_[m - 2][cur_[m - 2]].x, H2d, N, ld, ld,
                                           sc_ + S_FE + 1, cx.stream));
                const double* H3k = m == 2 ? H3d : nullptr;   // Tr[H3 P0] enters Omega^(3)
                if (H3k) {
                    CDMPT_TRY(Ew<T>::dot_h(Z_[last_n_].x, H3k, N, ld, ld, sc_ + S_FE + 3,
                                           cx.stream));
                    CDMPT_TRY(Ew<double>::trace(H3k, N, ld, 1, sc_ + S_FE + 4, cx.stream));
                }
                if (m == 3 && H3d)   // 3 Tr[H3 P1] enters Omega^(4)
                    CDMPT_TRY(Ew<T>::dot_h(zo_[0][cur_[0]].x, H3d, N, ld, ld, sc_ + S_FE + 3,
                                           cx.stream));
                CDMPT_TRY(read_scalars(cx, sc_, S_NSLOTS));
                const double* v = cx.pinned + S_FE;
                double sum = 0.5 * v[0];                 // Tr[H1 P^(m)]
                if (m == 1) {
                    sum += 2.0 * 0.5 * (v[2] + v[1]);   // 2 Tr[H2 P0]
                } else {
                    sum += 2.0 * 0.5 * v[1];            // 2 Tr[H2 P^(m-1)]
                    if (m == 2) sum += 3.0 * 0.5 * (v[4] + v[3]);   // 3 Tr[H3 P0]
                    else sum += 3.0 * 0.5 * v[3];                   // 3 Tr[H3 P1]
                }
                omega[d] = sum / (m + 1);
            }
            if (Pm)
                CDMPT_TRY(Ew<T>::to_f64(Pm + (size_t)d * N * N, N, Zq.x, ld, N, N, 0.5, 0.0,
                                        cx.stream));
            if (grad) {   // -4 w_d P2_d = -2 w_d Z2
                const double wd = w ? w[d] : 1.0;
                CDMPT_TRY(Ew<T>::axpby(G_.x, Zq.x, blk_, -2.0 * wd, 1.0, nullptr, cx.stream));
            }
        }
    }
    if (grad) {
        CDMPT_TRY(Ew<T>::symmetrize(G_.x, N, ld, 1, cx.stream));
        CDMPT_TRY(Ew<T>::to_f64(grad, N, G_.x, ld, N, N, 1.0, 0.0, cx.stream));
    }
    CDMPT_CUDA_TRY(cudaStreamSynchronize(cx.stream));
    return check_device_error(cx.stream);
}

// Second order (H^(2) = 0). The polarizability gradient follows from the
// symmetry of the third derivatives of the canonical free energy (whose gradient
// in H0 is P0): d alpha_d / d H0 = -2 d^2 P / d lambda_d^2 = -4 P2_d.
template <typename T>
cdmpt_status Solver<T>::response2(Context& cx, const double* H1, int D, const double* w,
                                  double* P2, double* mu2_out, double* omega3, double* grad,
                                  const double* H2, const double* H3) {
    return higher(cx, H1, D, 2, w, P2, mu2_out, omega3, grad, H2, H3);
}

template <typename T>
cdmpt_status Solver<T>::response1(Context& cx, const double* H1, int D, double* P1,
                                  double* mu1_out, double* omega2) {
    return higher(cx, H1, D, 1, nullptr, P1, mu1_out, omega2, nullptr);
}

template <typename T>
cdmpt_status Solver<T>::response2_at(Context& cx, const double* H1, const double* H2, int D,
                                     const double* mu1s, double* P2, double* mu2) {
    return higher(cx, H1, D, 2, nullptr, P2, mu2, nullptr, nullptr, H2, nullptr, mu1s);
}

template <typename T>
cdmpt_status Solver<T>::response3(Context& cx, const double* H1, int D, double* P3,
                                  double* mu3_out, double* omega4, const double* H2,
                                  const double* H3) {
    return higher(cx, H1, D, 3, nullptr, P3, mu3_out, omega4, nullptr, H2, H3);
}

template <typename T>
cdmpt_status Solver<T>::logdet(Context& cx, const Buf<T>& M, double a, double b, double lo,
                               double hi, double eps, double* out) {
    const int N = N_;
    const cdmpt_opts& o = last_opts_;
    const int acc = last_acc_;
    const double c = std::sqrt(lo * hi);
    const double r = (std::sqrt(hi) - std::sqrt(lo)) / (std::sqrt(hi) + std::sqrt(lo));
    // terms j = 0..J of sum Tr(Y^(2j+1)) / (2j+1), |y| <= r: remainder below eps per level
    int J = 0;
    while (J < 64 && std::pow(r, 2 * J + 3) / ((2 * J + 3) * (1.0 - r * r)) > eps) ++J;
    Buf<T>& Y = zo_[0][0];
    Buf<T>& Y2 = zo_[0][1];
    Buf<T>* Pw = &zo_[1][0];
    Buf<T>* Pn = &zo_[1][1];
    // Y (A + c I) = A - c I with A = a I + b M: operator X -> (a + c) X + b X M
    CDMPT_TRY(Ew<T>::axpby(RHS_.x, M.x, blk_, b, 0.0, nullptr, cx.stream));
    CDMPT_TRY(Ew<T>::add_diag(RHS_.x, N, ld, 1, a - c, cx.stream));
    CgArgs g;
    g.W = &M;
    g.s = a + c;
    g.t = b;
    g.rhs = RHS_.x;
    g.rows = N;
    g.tol = o.cg_tol;
    g.maxit = o.cg_maxit;
    g.init_engine = g.iter_engine = acc;
    g.hint = 4;
    int it = 0;
    CDMPT_TRY(cg(cx, Y.x, g, &it, nullptr));
    CDMPT_TRY(Ew<T>::symmetrize(Y.x, N, ld, 1, cx.stream, Y.hi, Y.lo));
    auto trace_of = [&](const Buf<T>& B, double* v) -> cdmpt_status {
        CDMPT_CUDA_TRY(cudaMemsetAsync(sc_ + S_FE, 0, sizeof(double), cx.stream));
        CDMPT_TRY(Ew<T>::trace(B.x, N, ld, 1, sc_ + S_FE, cx.stream));
        CDMPT_TRY(read_scalars(cx, sc_, S_NSLOTS));
        *v = cx.pinned[S_FE];
        return CDMPT_OK;
    };
    double sum = 0.0, t = 0.0;
    CDMPT_TRY(trace_of(Y, &t));
    sum = t;
    if (J > 0) {
        Epilogue<T> ep;   // Y^2 (symmetric)
        ep.Dhi = Y2.hi;
        ep.Dlo = Y2.lo;
        ep.sym = true;
        CDMPT_TRY(gemm(cx, N, N, N, Y.op(), Y.op(), Y2.x, ep, nullptr, acc));
    }
    const Buf<T>* odd = &Y;
    for (int j = 1; j <= J; ++j) {   // Y^(2j+1) = Y^(2j-1) Y^2
        Epilogue<T> ep;
        ep.Dhi = Pn->hi;
        ep.Dlo = Pn->lo;
        CDMPT_TRY(gemm(cx, N, N, N, odd->op(), Y2.op(), Pn->x, ep, nullptr, acc));
        CDMPT_TRY(trace_of(*Pn, &t));
        sum += t / (2 * j + 1);
        odd = Pn;
        std::swap(Pw, Pn);
    }
    *out = N * std::log(c) + 2.0 * sum;
    return CDMPT_OK;
}

// Free energy without eigenvalues. For P = X_n of the recursion,
// 1 - x_{k+1} = (1 - x_k)^2 / t_k with t_k = x_k^2 + (1 - x_k)^2 = (1 + z_k^2)/2
// per level, so
//   ln det(I - P) = 2^n ln det(I - X_0) - sum_k 2^(n-1-k) ln det(A_k / 2)
//                 = 2^n ln det(I - Z_0) - sum_k 2^(n-1-k) ln det A_k - N ln 2,
// every determinant of a matrix with spectrum well inside (0, 2]. With
// ln(P (I - P)^-1) = 2^(n+1) atanh(Z_0) (the closed form of n steps, Appendix A)
// and H0 - mu I = -T 2^(n+1) Z_0, the functional of Eqs. (FreeE), (SED) becomes
//   Omega = mu Tr P + T ln det(I - P) + T 2^(n+1) Tr[P R],  R = atanh(Z_0) - Z_0,
// with R = Z_0 W_0 sum_j W_0^j / (2j + 3) by Horner in W_0 = Z_0^2. dOmega/dP =
// H0 + T ln(P (I - P)^-1) = mu I + T 2^(n+1) R, so the gradient is P0 plus the
// adjoint of the recursion applied to that matrix (vjp_p0 carries the
// canonical or fixed-mu constraint of the solve).
// With the Fermi-Dirac-exact start Z_0 = tanh(Y), atanh(Z_0) = Y = -(H0 - mu I) / (T 2^(n+1))
// to the series cut, so R = 0: Omega = mu Tr P + T ln det(I - P), dOmega/dP = mu I, and the
// canonical gradient is P0 itself (Tr dP0 = 0); at fixed mu it is P0 + vjp(mu I).
template <typename T>
cdmpt_status Solver<T>::free_energy(Context& cx, double* omega, double* grad) {
    if (!traj_valid_) {
        set_error("free energy: no completed solve on this handle");
        return CDMPT_ERR_ARG;
    }
    const int n = last_n_, N = N_;
    const int acc = last_acc_;
    // |Z_0| <= rho: the bound on |Y| for the linear start, tanh of it for the exact one
    const double rho = std::min(fdx_ ? std::tanh(last_rho_) : last_rho_, 1.0 - 1e-12);
    const double beta = last_beta_, mu = last_mu_;
    const double Te = 1.0 / beta;
    const double eps = sizeof(T) == 8 ? 1e-17 : 1e-12;
    CDMPT_TRY(reserve_orders());
    // ln det(I - Z_0): spectrum of I - Z_0 in [1 - rho, 1 + rho]
    double ld0 = 0.0;
    CDMPT_TRY(logdet(cx, Z_[0], 1.0, -1.0, 1.0 - rho, 1.0 + rho, eps, &ld0));
    // ln det A_k, A_k = I + W_k with W_k in [0, tanh(2^k atanh rho)^2]
    double lda = 0.0;
    const double u0 = std::atanh(rho);
    for (int k = 0; k < n; ++k) {
        CDMPT_TRY(need(cx, k));
        const double zk = std::tanh(std::ldexp(u0, k));
        double v = 0.0;
        CDMPT_TRY(logdet(cx, W_[k], 1.0, 1.0, 1.0, 1.0 + zk * zk, eps, &v));
        lda += std::ldexp(v, n - 1 - k);
    }
    const double logdet_1mp = std::ldexp(ld0, n) - lda - N * std::log(2.0);
    if (fdx_) {
        CDMPT_CUDA_TRY(cudaMemsetAsync(sc_ + S_FE, 0, sizeof(double), cx.stream));
        CDMPT_TRY(Ew<T>::trace(Z_[n].x, N, ld, 1, sc_ + S_FE, cx.stream));
        if (Z_[n].xl) CDMPT_TRY(Ew<T>::trace(Z_[n].xl, N, ld, 1, sc_ + S_FE, cx.stream));
        CDMPT_TRY(read_scalars(cx, sc_, S_NSLOTS));
        if (omega) *omega = mu * 0.5 * (N + cx.pinned[S_FE]) + Te * logdet_1mp;
        if (grad && last_opts_.grand_canonical == 0) {   // P0 = (I + Z_n) / 2
            CDMPT_TRY(p0_out(cx, grad, N));
        } else if (grad) {
            double* G0 = nullptr;
            CDMPT_CUDA_TRY(cudaMallocAsync((void**)&G0, (size_t)N * N * sizeof(double),
                                           cx.stream));
            CDMPT_CUDA_TRY(cudaMemsetAsync(G0, 0, (size_t)N * N * sizeof(double), cx.stream));
            CDMPT_TRY(Ew<double>::add_diag(G0, N, N, 1, mu, cx.stream));
            const cdmpt_status s = vjp_p0(cx, G0, grad, 1.0);
            cudaFreeAsync(G0, cx.stream);
            CDMPT_TRY(s);
        }
        CDMPT_CUDA_TRY(cudaStreamSynchronize(cx.stream));
        return check_device_error(cx.stream);
    }
    // R = Z_0 W_0 h(W_0), h = sum_{j=0..J} W_0^j / (2j + 3), Horner from the top
    int J = 0;
    while (J < 200 && std::pow(rho, 2 * J + 2) > eps * (2 * J + 5) / 3.0) ++J;
    Buf<T>* Hc = &ao_[0];
    Buf<T>* Hn = &ao_[1];
    Buf<T>& R = ao_[2];
    CDMPT_CUDA_TRY(cudaMemsetAsync(Hc->x, 0, blk_ * sizeof(T), cx.stream));
    if (Hc->hi) CDMPT_CUDA_TRY(cudaMemsetAsync(Hc->hi, 0, blk_ * sizeof(T), cx.stream));
    if (Hc->lo) CDMPT_CUDA_TRY(cudaMemsetAsync(Hc->lo, 0, blk_ * sizeof(T), cx.stream));
    CDMPT_TRY(Ew<T>::add_diag(Hc->x, N, ld, 1, 1.0 / (2 * J + 3), cx.stream, Hc->hi, Hc->lo));
    for (int j = J - 1; j >= -1; --j) {   // j >= 0: h <- W_0 h + I/(2j+3); j = -1: W_0 h
        Epilogue<T> ep;
        ep.gamma = j >= 0 ? 1.0 / (2 * j + 3) : 0.0;
        ep.Dhi = Hn->hi;
        ep.Dlo = Hn->lo;
        CDMPT_TRY(gemm(cx, N, N, N, W_[0].op(), Hc->op(), Hn->x, ep, nullptr, acc));
        std::swap(Hc, Hn);
    }
    {
        Epilogue<T> ep;   // R = Z_0 (W_0 h)
        ep.Dhi = R.hi;
        ep.Dlo = R.lo;
        CDMPT_TRY(gemm(cx, N, N, N, Z_[0].op(), Hc->op(), R.x, ep, nullptr, acc));
    }
    // Tr P0 = (N + Tr Z_n)/2 and Tr[P0 R] = (Tr R + <Z_n, R>)/2
    CDMPT_CUDA_TRY(cudaMemsetAsync(sc_ + S_FE, 0, 3 * sizeof(double), cx.stream));
    CDMPT_TRY(Ew<T>::trace(Z_[n].x, N, ld, 1, sc_ + S_FE, cx.stream));
    if (Z_[n].xl) CDMPT_TRY(Ew<T>::trace(Z_[n].xl, N, ld, 1, sc_ + S_FE, cx.stream));
    CDMPT_TRY(Ew<T>::trace(R.x, N, ld, 1, sc_ + S_FE + 1, cx.stream));
    CDMPT_TRY(Ew<T>::dot(Z_[n].x, R.x, blk_, sc_ + S_FE + 2, nullptr, cx.stream));
    CDMPT_TRY(read_scalars(cx, sc_, S_NSLOTS));
    const double trP = 0.5 * (N + cx.pinned[S_FE]);
    const double trPR = 0.5 * (cx.pinned[S_FE + 1] + cx.pinned[S_FE + 2]);
    const double scale = std::ldexp(Te, n + 1);   // T 2^(n+1)
    if (omega) *omega = mu * trP + Te * logdet_1mp + scale * trPR;
    if (grad) {   // grad = vjp(mu I + T 2^(n+1) R) + P0
        double* G0 = nullptr;
        CDMPT_CUDA_TRY(cudaMallocAsync((void**)&G0, (size_t)N * N * sizeof(double), cx.stream));
        CDMPT_TRY(Ew<T>::to_f64(G0, N, R.x, ld, N, N, scale, mu, cx.stream));
        const cdmpt_status s = vjp_p0(cx, G0, grad, 1.0);
        cudaFreeAsync(G0, cx.stream);
        CDMPT_TRY(s);
    }
    CDMPT_CUDA_TRY(cudaStreamSynchronize(cx.stream));
    return check_device_error(cx.stream);
}

template <typename T>
cdmpt_status Solver<T>::solve(Context& cx, const double* H0, const double* H1, int N, int D,
                              double gmin, double gmax, double trH0, const cdmpt_opts& o,
                              double beta, double nocc, int n, double* P0, double* P1,
                              double* mu_out, double* mu1_out, int out_on_device,
                              double* alpha_out) {
    if (D > kMaxD) {
        set_error("at most 16 perturbation directions per solve");
        return CDMPT_ERR_ARG;
    }
    const bool bf16 = sizeof(T) == 4 && o.precision == CDMPT_MIXED_BF16;
    const bool mixed = sizeof(T) == 4 && (o.precision == CDMPT_MIXED_TF32 || bf16);
    if (mixed && cx.engine == CDMPT_GEMM_SIMT) {
        set_error("mixed precision needs the tcgen05 engines");
        return CDMPT_ERR_ARG;
    }
    // trajectory checkpoints: every ck-th Z_k (ckpt_stride < 0: ck = ceil(sqrt(n)))
    int ck = 0;
    if (o.ckpt_stride != 0) {
        if (mixed) {
            set_error("checkpointing needs the FP64 or FP32 precision: the mixed-precision "
                      "refinement revisits every stored step");
            return CDMPT_ERR_ARG;
        }
        ck = o.ckpt_stride < 0 ? (int)std::ceil(std::sqrt((double)n) - 1e-9)
                               : std::min(o.ckpt_stride, n);
    }
    CDMPT_TRY(reserve(N, D, n, ck, mixed));
    traj_valid_ = q_valid_ = false;
    fdx_ = o.fd_exact != 0;
    screen_tau_ = (sizeof(T) == 4 && tcnt_) ? (float)o.screen_tau : 0.f;
    if (screen_tau_ > 0.f)
        CDMPT_CUDA_TRY(cudaMemsetAsync(tcnt_, 0, 2 * sizeof(unsigned long long), cx.stream));
    gmin_ = gmin;
    gmax_ = gmax;
    replay_iters_ = 0;
    last_mu1_.assign(std::max(D, 0), 0.0);
    cdmpt_stats& st = *cx.st;
    const double s2 = std::ldexp(beta, -(n + 1));
    const double width = gmax - gmin;
    if (!(s2 * width < 1.0)) {
        set_error("beta * (lambda_max - lambda_min) / 2^(n+1) = " + std::to_string(s2 * width) +
                  " >= 1: X_0 leaves [0, 1]; use more recursion steps");
        return CDMPT_ERR_RANGE;
    }
    // engines: "acc" for FP32-accurate products, "fast" for the occupation sweeps
    const int acc = mixed ? (int)CDMPT_GEMM_TC_3XTF32 : engine_of(cx, 0);
    const int fast = mixed ? (bf16 ? (int)CDMPT_GEMM_TC_BF16 : (int)CDMPT_GEMM_TC_TF32) : acc;
    acc_cur_ = acc;
    const double pad = std::min(40.0 / beta, 0.45 * (1.0 / s2 - width));
    double lo = gmin - pad, hi = gmax + pad;
    const bool gc = o.grand_canonical != 0;   // fixed mu: no occupation loop, mu1 = 0
    double mu = o.have_mu_guess ? o.mu_guess : trH0 / N;
    if (gc) {
        // X_0 keeps its spectrum in [0, 1] iff |eps - mu| < 2^(n+1) / beta over the spectrum
        if (!(gmax - mu < 1.0 / s2 && mu - gmin < 1.0 / s2)) {
            set_error("grand canonical: mu = " + std::to_string(mu) +
                      " puts X_0 outside [0, 1]; use more recursion steps");
            return CDMPT_ERR_RANGE;
        }
    } else {
        mu = std::min(std::max(mu, lo + 1e-3 * pad), hi - 1e-3 * pad);
    }
    const double occ_tol = o.occ_tol > 0 ? o.occ_tol : N * (sizeof(T) == 8 ? 1e-12 : 1e-7);
    // one-pass TF32 traces are good to about 1e-4 relative, BF16 ones to about 1e-2, and
    // their per-level rounding (2^-11, 2^-8) adds noise of about that times sqrt(N), which
    // dominates for small N; the refinement finishes mu
    const double occ_tol_sweep =
        mixed ? std::max({occ_tol, (bf16 ? 1e-3 : 1e-5) * N,
                          (bf16 ? 1e-2 : 5e-4) * std::sqrt((double)N)})
              : occ_tol;
    const double sweep_tol = mixed ? (bf16 ? 1e-3 : 1e-4) : o.cg_tol;

    // -------------------------------------------------- occupation loop
    cx.mark(0);
    bool converged = false;
    double trP = 0, zz = 0;
    double e_lo = 0.0, e_hi = 0.0;   // occupation errors at lo and hi once a sweep set them
    for (int it = 0; it < o.mu_maxit; ++it) {
        int iters = 0;
        CDMPT_TRY(sweep(cx, H0, mu, s2, o, n, fast, sweep_tol, &iters));
        st.mu_iterations += 1;
        st.cg_iterations_sweeps += iters;
        st.cg_iterations_last_sweep = iters;
        CDMPT_TRY(occupation(cx, n, &trP, &zz));
        const double err = gc ? 0.0 : trP - nocc;
        st.mu = mu;
        st.trace_P0 = trP;
        st.occupation_error = std::fabs(err);
        if (std::fabs(err) <= occ_tol_sweep) {
            converged = true;
            break;
        }
        if (err > 0) {
            hi = mu;
            e_hi = err;
        } else {
            lo = mu;
            e_lo = err;
        }
        const double slope = 0.25 * beta * (N - zz);
        double mu_new = slope > 0 ? mu - err / slope : lo - 1.0;
        if (!(mu_new > lo && mu_new < hi))
            mu_new = next_mu_outside_newton(lo, hi, e_lo, e_hi);
        if (mu_new == mu) break;
        mu = mu_new;
    }
    if (!converged) {
        set_error("occupation did not converge: |Tr P0 - N_occ| = " +
                  std::to_string(st.occupation_error) + " after " +
                  std::to_string(st.mu_iterations) + " sweeps");
        return CDMPT_ERR_NO_CONVERGENCE;
    }

    // -------------------------------------------------- refinement (mixed)
    cx.mark(1);
    if (mixed) {
        const int min_pass = std::max(1, o.refine_rounds);
        // first step of the FP64-class pass: every step, or the steps whose spectral bound
        // tanh(2^k atanh rho) exceeds hp_bound() (before them the error of a split-TF32
        // residual, relative to Z_k, carries the factor ||W_k|| <= tanh(2^k atanh rho)^2)
        int k_hp = n;
        if (o.fp64_residual >= 0) {
            k_hp = 0;
            if (o.fp64_residual == 0) {
                const double a0 = std::atanh(std::min(s2 * std::max(gmax - mu, mu - gmin), 0.999999));
                while (k_hp < n && std::tanh(std::ldexp(a0, k_hp)) <= hp_bound()) ++k_hp;
            }
        }
        st.fp64_residual_first_step = k_hp;
        // split-TF32 passes until the step residuals settle (one pass from the sweep's
        // trajectory, see refine_settle); from then on (including the Newton steps that
        // follow) every pass forms the residuals of steps k >= k_hp with Ozaki-sliced
        // products, so that no occupation is measured on a trajectory carrying the split
        // products' bias
        bool done = false, hp_phase = false;
        int hp_passes = 0;
        for (int pass = 0; pass < min_pass + (bf16 ? 10 : 6) + 4 && !done; ++pass) {
            int iters = 0;
            double worst = 0.0;
            CDMPT_TRY(refine(cx, o, n, hp_phase ? k_hp : n, &iters, &worst));
            st.cg_iterations_refine += iters;
            st.refine_passes += 1;
            if (hp_phase) st.fp64_residual_passes += 1;
            CDMPT_TRY(occupation(cx, n, &trP, &zz));
            const double err = gc ? 0.0 : trP - nocc;
            st.trace_P0 = trP;
            st.occupation_error = std::fabs(err);
            // finish mu to 1e-9 N, or to 1e-7 sqrt(N) once the minimum passes are done
            const double tol_ref =
                o.occ_tol > 0 ? occ_tol
                              : std::max(1e-9 * N, pass + 1 >= min_pass ? 1e-7 * std::sqrt((double)N)
                                                                         : 0.0);
            const bool occ_ok = std::fabs(err) <= tol_ref;
            if (hp_phase) {
                if (occ_ok && pass + 1 >= min_pass) {
                    done = true;
                    break;
                }
                if (++hp_passes >= 4) break;
            } else {
                // the pass started from relative step residuals below 1e-6, so it left them
                // at about 1e-9 or at the split-TF32 floor (or, after three extra passes,
                // below 1e-4)
                if (k_hp >= n) {
                    // split residuals only: finish once the pass started below 1e-6 (it left
                    // the residuals near 1e-9 or at the split floor), or below 1e-4 after three
                    // extra passes
                    const bool settled =
                        worst < 1e-6 || (pass + 1 >= min_pass + 3 && worst < 1e-4);
                    if (occ_ok && pass + 1 >= min_pass && settled) {
                        done = true;
                        break;
                    }
                } else {
                    const bool settled =
                        worst < (refine_early_hp() ? refine_settle() : 1e-6) ||
                        (pass + 1 >= min_pass + 3 && worst < 1e-4);
                    if (settled && (refine_early_hp() || (occ_ok && pass + 1 >= min_pass))) {
                        hp_phase = true;
                        if (occ_ok) continue;
                    }
                }
            }
            if (!occ_ok) {   // Newton step on mu; Z_0 = -s2 (H - mu I) moves by s2 dmu I
                const double slope = 0.25 * beta * (N - zz);
                const double dmu = slope > 0 ? -err / slope : 0.0;
                mu += dmu;
                if (fdx_)   // Z_0 = tanh(Y) is not shifted by a multiple of I: rebuild it
                    CDMPT_TRY(init_z0(cx, H0, mu, s2, s2 * std::max(gmax - mu, mu - gmin), acc));
                else
                    CDMPT_TRY(shift_z0(cx, s2 * dmu));
            }
        }
        if (!done) {
            set_error("mixed-precision refinement did not converge: |Tr P0 - N_occ| = " +
                      std::to_string(st.occupation_error));
            return CDMPT_ERR_NO_CONVERGENCE;
        }
    }
    st.mu = mu;
    if (mu_out) *mu_out = mu;
    cx.mark(2);
    traj_valid_ = true;
    last_beta_ = beta;
    last_mu_ = mu;
    last_rho_ = s2 * std::max(gmax - mu, mu - gmin);
    last_s2_ = s2;
    last_n_ = n;
    last_acc_ = acc;
    last_sweep_tol_ = sweep_tol;
    last_opts_ = o;

    // -------------------------------------------------- first-order response
    if (D > 0) {
        const int rows = D * N;
        const size_t count = (size_t)rows * ld;
        Buf<T>* Z1 = &Z1a_;
        Buf<T>* Z1n = &Z1b_;
        if (fdx_)
            CDMPT_TRY(init_z1(cx, H1, D, Z1->x, Z1->hi, Z1->lo));
        else
            CDMPT_TRY(Ew<T>::init_z(Z1->x, H1, N, ld, ld, D, -s2, 0.0, cx.stream, Z1->hi,
                                    Z1->lo));
        int total = 0, hint = 1;
        for (int k = 0; k < n; ++k) {
            CDMPT_TRY(need(cx, k));
            {   // S^T = Z1 Z_k (stacked over directions)
                Epilogue<T> ep;
                CDMPT_TRY(gemm(cx, rows, N, N, Z1->op(), Z_[k].op(), S_.x, ep, nullptr, acc));
            }
            // A1 = Z_k Z1 + Z1 Z_k, block by block
            CDMPT_TRY(Ew<T>::transpose_add(A1_.x, S_.x, N, ld, D, cx.stream, A1_.hi, A1_.lo));
            // correction form: Z1_{k+1} = 2 Z1_k + d1 with
            //   d1 (I + W_k) = -Z_{k+1} A1 - 2 Z1_k W_k
            // (both terms carry the same sign for saturated levels, so no cancellation)
            {   // -Z_{k+1} A1 = -(A1 Z_{k+1})^T per block
                Epilogue<T> ep;
                ep.alpha = -1.0;
                ep.trans_block = N;
                CDMPT_TRY(gemm(cx, rows, N, N, A1_.op(), Z_[k + 1].op(), RHS_.x, ep, nullptr, acc));
            }
            {   // -= 2 Z1_k W_k
                Epilogue<T> ep;
                ep.alpha = -2.0;
                ep.beta = 1.0;
                ep.C = RHS_.x;
                ep.ldc = ld;
                CDMPT_TRY(gemm(cx, rows, N, N, Z1->op(), W_[k].op(), RHS_.x, ep, nullptr, acc));
            }
            CgArgs a;
            a.W = &W_[k];
            a.rhs = RHS_.x;
            a.rows = rows;
            a.tol = o.cg_tol;
            a.maxit = o.cg_maxit;
            a.init_engine = a.iter_engine = acc;
            a.hint = hint;
            // the correction d1 needs the tolerance relative to the new iterate
            // Z1_{k+1} = 2 Z1_k + d1, not to its own right side: in the early steps that side
            // is of the size of W_k Z1_k, far below Z1_k, and a tolerance relative to it
            // would ask for digits the stored response never keeps
            a.ref = Z1->x;
            a.ref_scale = 2.0;
            a.tol_ref = o.cg_tol;
            int it = 0;
            if (mixed && response_ir()) {
                // mixed-precision iterative refinement of the step's system: one-pass TF32
                // CG iterations, each cycle stopped after about three digits, restarted from
                // an FP32-accurate (split-TF32) residual of the current solution
                a.iter_engine = fast == (int)CDMPT_GEMM_TC_BF16 ? (int)CDMPT_GEMM_TC_TF32 : fast;
                a.tol_r0 = 1e-3;
                for (int cyc = 0; cyc < 8; ++cyc) {
                    if (cyc > 0) {
                        a.x0 = Z1n;
                        if constexpr (sizeof(T) == 4)
                            CDMPT_TRY(split_tf32(Z1n->x, count, Z1n->hi, Z1n->lo, cx.stream));
                    }
                    int itc = 0;
                    double rel0 = 0.0;
                    bool met = false;
                    CDMPT_TRY(cg(cx, Z1n->x, a, &itc, &rel0, &met));
                    it += itc;
                    a.hint = std::max(1, itc);
                    // done when the accurate residual already met the tolerance, or when this
                    // cycle's three digits reached it
                    if (itc == 0 || met || rel0 * a.tol_r0 <= o.cg_tol) break;
                }
            } else {
                CDMPT_TRY(cg(cx, Z1n->x, a, &it, nullptr));
            }
            total += it;
            hint = std::max(1, it);
            CDMPT_TRY(Ew<T>::axpby(Z1n->x, Z1->x, count, 2.0, 1.0, nullptr, cx.stream));
            CDMPT_TRY(Ew<T>::symmetrize(Z1n->x, N, ld, D, cx.stream, Z1n->hi, Z1n->lo));
            std::swap(Z1, Z1n);
        }
        st.cg_iterations_response = total;
        cx.mark(3);

        if (!gc) CDMPT_TRY(compute_q(cx));
        CDMPT_CUDA_TRY(cudaMemsetAsync(sc_ + S_TRQ, 0, (S_NSLOTS - S_TRQ) * sizeof(double),
                                       cx.stream));
        if (!gc) CDMPT_TRY(Ew<T>::trace(Qmu_.x, N, ld, 1, sc_ + S_TRQ, cx.stream));
        CDMPT_TRY(Ew<T>::trace(Z1->x, N, ld, D, sc_ + S_TRZ1, cx.stream));
        CDMPT_TRY(read_scalars(cx, sc_, S_NSLOTS));
        const double trQ = cx.pinned[S_TRQ];
        st.trace_Q = trQ;
        for (int d = 0; d < D; ++d) {
            const double trP1 = 0.5 * cx.pinned[S_TRZ1 + d];
            // grand canonical: mu stays fixed, so mu1 = 0 and P1 = Z1 / 2
            const double mu1 = (!gc && trQ > 0) ? -trP1 / trQ : 0.0;
            if (mu1_out) mu1_out[d] = mu1;
            last_mu1_[d] = mu1;
            // P1 = Z1/2 + mu1 Q  <=>  Z1 += 2 mu1 Q
            if (!gc)
                CDMPT_TRY(Ew<T>::axpby(Z1->x + (size_t)d * blk_, Qmu_.x, blk_, 2.0 * mu1, 1.0,
                                       nullptr, cx.stream));
            CDMPT_TRY(Ew<T>::dot_h(Z1->x + (size_t)d * blk_, H1 + (size_t)d * blk_, N, ld, ld,
                                      sc_ + S_ALPHA + d, cx.stream));
        }
        CDMPT_CUDA_TRY(cudaMemsetAsync(sc_ + S_TRZ1, 0, kMaxD * sizeof(double), cx.stream));
        CDMPT_TRY(Ew<T>::trace(Z1->x, N, ld, D, sc_ + S_TRZ1, cx.stream));
        if (P1) {
            if (out_on_device) {
                CDMPT_TRY(Ew<T>::to_f64(P1, N, Z1->x, ld, N, rows, 0.5, 0.0, cx.stream));
            } else {
                double* tmp = nullptr;
                CDMPT_CUDA_TRY(cudaMallocAsync((void**)&tmp, (size_t)rows * N * sizeof(double),
                                               cx.stream));
                CDMPT_TRY(Ew<T>::to_f64(tmp, N, Z1->x, ld, N, rows, 0.5, 0.0, cx.stream));
                CDMPT_CUDA_TRY(cudaMemcpyAsync(P1, tmp, (size_t)rows * N * sizeof(double),
                                               cudaMemcpyDeviceToHost, cx.stream));
                CDMPT_CUDA_TRY(cudaFreeAsync(tmp, cx.stream));
            }
        }
        CDMPT_TRY(read_scalars(cx, sc_, S_NSLOTS));
        double occ1 = 0;
        for (int d = 0; d < D; ++d) {
            occ1 += std::fabs(0.5 * cx.pinned[S_TRZ1 + d]);
            // alpha_d = -2 Tr[P1 H1] = -2 * (1/2) sum Z1 * H1
            if (alpha_out) alpha_out[d] = -cx.pinned[S_ALPHA + d];
        }
        st.occupation_error += occ1;
    }
    cx.mark(4);

    if (P0) {
        if (out_on_device) {
            CDMPT_TRY(p0_out(cx, P0, N));
        } else {
            double* tmp = nullptr;
            CDMPT_CUDA_TRY(cudaMallocAsync((void**)&tmp, (size_t)N * N * sizeof(double), cx.stream));
            CDMPT_TRY(p0_out(cx, tmp, N));
            CDMPT_CUDA_TRY(cudaMemcpyAsync(P0, tmp, (size_t)N * N * sizeof(double),
                                           cudaMemcpyDeviceToHost, cx.stream));
            CDMPT_CUDA_TRY(cudaFreeAsync(tmp, cx.stream));
        }
    }
    st.cg_iterations_recompute = replay_iters_;
    st.checkpoint_stride = ck_;
    st.screen_slices_computed = st.screen_slices_examined = 0.0;
    if (screen_tau_ > 0.f) {
        unsigned long long c[2] = {0, 0};
        CDMPT_CUDA_TRY(cudaMemcpyAsync(c, tcnt_, sizeof(c), cudaMemcpyDeviceToHost, cx.stream));
        CDMPT_CUDA_TRY(cudaStreamSynchronize(cx.stream));
        st.screen_slices_computed = (double)c[0];
        st.screen_slices_examined = (double)c[1];
    }
    cx.mark(5);
    CDMPT_CUDA_TRY(cudaStreamSynchronize(cx.stream));
    return check_device_error(cx.stream);
}

template class Solver<float>;
template class Solver<double>;

}  // namespace cdmpt
