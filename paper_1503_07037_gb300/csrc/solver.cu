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
//
// Chemical potential: Newton on Tr P0 = N_occ with the paper's slope
// Tr P_mu = beta Tr[P0 (I - P0)] = beta/4 (N - ||Z_n||_F^2) (Eq. NewtRaphs),
// safeguarded by a bisection bracket. mu1: P1 is linear in mu1 with slope
// Q = dP0/dmu, which at finite n is exactly beta P0 (I - P0) (I - Z_0^2)^-1;
// the response runs once with mu1 = 0 and mu1 = -Tr P1|_0 / Tr Q follows in
// closed form (the fixed point of the mu1 update of Algorithm 1).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>

#include "solver.cuh"

namespace cdmpt {

namespace {
enum Slot {
    S_TRZ = 8,      // Tr Z_n
    S_ZZ = 9,       // ||Z_n||_F^2
    S_TRQ = 10,     // Tr Q
    S_TRZ1 = 16,    // Tr Z1_d (d < 16)
    S_ALPHA = 32,   // sum P1_d * H1_d (d < 16)
    S_NSLOTS = 64
};
constexpr int kMaxD = 16;
}  // namespace

template <typename T>
Solver<T>::~Solver() {
    for (void* p : allocs_) cudaFree(p);
}

template <typename T>
cdmpt_status Solver<T>::reserve(int N, int D, int n) {
    const int ld_new = (N + 31) / 32 * 32;
    const int rows_needed = std::max(1, D) * N;
    if (N == N_ && D <= D_ && n <= n_ && ld == ld_new && rows_cap_ >= rows_needed) return CDMPT_OK;
    for (void* p : allocs_) cudaFree(p);
    allocs_.clear();
    Z_.clear();
    A_.clear();
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
    Z_.resize(n + 1);
    A_.resize(n);
    for (int k = 0; k <= n; ++k) CDMPT_TRY(grab(blk_, &Z_[k]));
    for (int k = 0; k < n; ++k) CDMPT_TRY(grab(blk_, &A_[k]));
    const size_t big = (size_t)rows_needed * ld;
    CDMPT_TRY(grab(big, &R_));
    CDMPT_TRY(grab(big, &P_));
    CDMPT_TRY(grab(big, &Q_));
    CDMPT_TRY(grab(big, &S_));
    CDMPT_TRY(grab(big, &A1_));
    CDMPT_TRY(grab(big, &RHS_));
    CDMPT_TRY(grab(big, &Z1a_));
    CDMPT_TRY(grab(big, &Z1b_));
    CDMPT_TRY(grab(blk_, &Qmu_));
    CDMPT_TRY(grab(blk_, &Mq_));
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

template <typename T>
cdmpt_status Solver<T>::gemm(Context& cx, int M, int Nc, int K, const T* X, const T* Y, T* D,
                             const Epilogue<T>& ep, const double* skip, int engine_override) {
    int engine = CDMPT_GEMM_SIMT;
    if constexpr (sizeof(T) == 4) {
        engine = engine_override ? engine_override : cx.engine;
        if (engine == CDMPT_GEMM_AUTO) engine = CDMPT_GEMM_TC_3XTF32;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cx.profile) {
        while (cx.ev.size() < 2 * (cx.ev_used + 1)) {
            cudaEvent_t e;
            CDMPT_CUDA_TRY(cudaEventCreate(&e));
            cx.ev.push_back(e);
        }
        if (cx.ev_ok.size() < cx.ev_used + 1) cx.ev_ok.resize(cx.ev_used + 1);
        cx.ev_ok[cx.ev_used] = 1;
        e0 = cx.ev[2 * cx.ev_used];
        e1 = cx.ev[2 * cx.ev_used + 1];
        CDMPT_CUDA_TRY(cudaEventRecord(e0, cx.stream));
    }
    cdmpt_status s;
    if constexpr (sizeof(T) == 4) {
        if (engine == CDMPT_GEMM_SIMT)
            s = gemm_simt<float>(M, Nc, K, X, ld, Y, ld, D, ld, ep, skip, cx.stream);
        else
            s = gemm_tc_f32(engine, M, Nc, K, X, ld, Y, ld, D, ld, ep, skip, cx.stream);
    } else {
        s = gemm_simt<double>(M, Nc, K, X, ld, Y, ld, D, ld, ep, skip, cx.stream);
    }
    if (s != CDMPT_OK) return s;
    if (cx.profile) {
        CDMPT_CUDA_TRY(cudaEventRecord(e1, cx.stream));
        ++cx.ev_used;
    }
    if (cx.st && skip == nullptr) {
        const double f = 2.0 * M * (double)Nc * K;
        cx.st->gemm_launches += 1;
        cx.st->gemm_flops += f;
        cx.st->tensor_flops += engine == CDMPT_GEMM_TC_3XTF32 ? 3 * f
                               : engine == CDMPT_GEMM_TC_TF32 ? f
                                                              : 0.0;
    }
    return CDMPT_OK;
}

// Solve X A = rhs_scale * rhs_base for X (rows x N), warm start in X.
// Global CG in the Frobenius inner product; A is SPD (spectrum in [1, 2] for
// the recursion, Sec. II). Scalars stay on the device; the host reads the
// convergence flag once per chunk of iterations, and iterations launched
// after convergence return at once.
template <typename T>
cdmpt_status Solver<T>::cg(Context& cx, T* X, const T* A, const T* rhs_base, double rhs_scale,
                           int rows, double tol, int maxit, int* iters_out, int engine_override) {
    const size_t count = (size_t)rows * ld;
    double* sc = sc_;
    CDMPT_CUDA_TRY(cudaMemsetAsync(sc, 0, CG_NSLOTS * sizeof(double), cx.stream));
    {   // R = s B - X A, <R,R>
        Epilogue<T> ep;
        ep.alpha = -1.0;
        ep.beta = rhs_scale;
        ep.C = rhs_base;
        ep.ldc = ld;
        ep.dot = sc + CG_RR;
        CDMPT_TRY(gemm(cx, rows, N_, N_, X, A, R_, ep, nullptr, engine_override));
    }
    CDMPT_TRY(Ew<T>::dot(rhs_base, rhs_base, count, sc + CG_BB, nullptr, cx.stream));
    CDMPT_TRY(cg_scalar_init(sc, tol * tol * rhs_scale * rhs_scale, cx.stream));
    CDMPT_TRY(Ew<T>::axpby(P_, R_, count, 1.0, 0.0, sc + CG_DONE, cx.stream));

    int chunk = std::max(1, *iters_out);
    int launched = 0, iters = 0;
    while (true) {
        const size_t ev_first = cx.ev_used;
        for (int c = 0; c < chunk; ++c) {
            Epilogue<T> ep;
            ep.dot = sc + CG_PQ;
            ep.E = P_;
            ep.lde = ld;
            CDMPT_TRY(gemm(cx, rows, N_, N_, P_, A, Q_, ep, sc + CG_DONE, engine_override));
            CDMPT_TRY(Ew<T>::cg_update(X, R_, P_, Q_, count, sc, cx.stream));
            CDMPT_TRY(Ew<T>::cg_direction(P_, R_, count, sc, cx.stream));
            CDMPT_TRY(cg_scalar_step(sc, cx.stream));
        }
        launched += chunk;
        CDMPT_TRY(read_scalars(cx, sc, CG_NSLOTS));
        const int now = (int)cx.pinned[CG_ITERS];
        const int ran = now - iters;
        iters = now;
        if (cx.profile) {
            // event pairs of GEMMs that returned at once are dropped
            for (size_t e = ev_first + ran; e < cx.ev_used; ++e) cx.ev_ok[e] = 0;
        }
        if (cx.st) {
            const double f = 2.0 * rows * (double)N_ * N_;
            int engine = CDMPT_GEMM_SIMT;
            if constexpr (sizeof(T) == 4) {
                engine = engine_override ? engine_override : cx.engine;
                if (engine == CDMPT_GEMM_AUTO) engine = CDMPT_GEMM_TC_3XTF32;
            }
            cx.st->gemm_launches += ran;
            cx.st->gemm_flops += ran * f;
            cx.st->tensor_flops += ran * (engine == CDMPT_GEMM_TC_3XTF32 ? 3 * f
                                          : engine == CDMPT_GEMM_TC_TF32 ? f
                                                                         : 0.0);
        }
        if (cx.pinned[CG_DONE] != 0.0) break;
        if (iters >= maxit) {
            *iters_out = iters;
            set_error("CG did not reach the tolerance in " + std::to_string(maxit) +
                      " iterations (relative residual " +
                      std::to_string(std::sqrt(cx.pinned[CG_RRNEW] /
                                               std::max(1e-300, cx.pinned[CG_BB] * rhs_scale *
                                                                    rhs_scale))) +
                      ")");
            return CDMPT_ERR_CG_MAXITER;
        }
        chunk = 2;
    }
    *iters_out = iters;
    return CDMPT_OK;
}

// One 0th-order pass of Algorithm 1 at chemical potential mu: Z_0 .. Z_n, A_0 .. A_{n-1}.
template <typename T>
cdmpt_status Solver<T>::sweep(Context& cx, const double* H0, double mu, double s2,
                              const cdmpt_opts& o, int n, int* cg_iters, int engine_override) {
    CDMPT_TRY(Ew<T>::init_z(Z_[0], H0, N_, ld, ld, 1, -s2, mu, cx.stream));
    int total = 0, hint = 1;
    for (int k = 0; k < n; ++k) {
        Epilogue<T> ep;
        ep.gamma = 1.0;   // A_k = I + Z_k Z_k
        CDMPT_TRY(gemm(cx, N_, N_, N_, Z_[k], Z_[k], A_[k], ep, nullptr, engine_override));
        CDMPT_TRY(Ew<T>::axpby(Z_[k + 1], Z_[k], blk_, 2.0, 0.0, nullptr, cx.stream));
        int it = hint;
        CDMPT_TRY(cg(cx, Z_[k + 1], A_[k], Z_[k], 2.0, N_, o.cg_tol, o.cg_maxit, &it,
                     engine_override));
        total += it;
        hint = std::max(1, it);
        CDMPT_TRY(Ew<T>::symmetrize(Z_[k + 1], N_, ld, 1, cx.stream));
    }
    *cg_iters = total;
    return CDMPT_OK;
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
    CDMPT_TRY(reserve(N, D, n));
    cdmpt_stats& st = *cx.st;
    const double s2 = std::ldexp(beta, -(n + 1));
    const double width = gmax - gmin;
    if (!(s2 * width < 1.0)) {
        set_error("beta * (lambda_max - lambda_min) / 2^(n+1) = " + std::to_string(s2 * width) +
                  " >= 1: X_0 leaves [0, 1]; use more recursion steps");
        return CDMPT_ERR_RANGE;
    }
    const double pad = std::min(40.0 / beta, 0.45 * (1.0 / s2 - width));
    double lo = gmin - pad, hi = gmax + pad;
    double mu = o.have_mu_guess ? o.mu_guess : trH0 / N;
    mu = std::min(std::max(mu, lo + 1e-3 * pad), hi - 1e-3 * pad);
    const double occ_tol =
        o.occ_tol > 0 ? o.occ_tol : N * (sizeof(T) == 8 ? 1e-12 : 1e-7);

    // -------------------------------------------------- occupation loop
    bool converged = false;
    double trP = 0, zz = 0;
    for (int it = 0; it < o.mu_maxit; ++it) {
        int iters = 0;
        CDMPT_TRY(sweep(cx, H0, mu, s2, o, n, &iters, 0));
        st.mu_iterations += 1;
        st.cg_iterations_sweeps += iters;
        st.cg_iterations_last_sweep = iters;
        CDMPT_CUDA_TRY(cudaMemsetAsync(sc_ + S_TRZ, 0, 2 * sizeof(double), cx.stream));
        CDMPT_TRY(Ew<T>::trace(Z_[n], N, ld, 1, sc_ + S_TRZ, cx.stream));
        CDMPT_TRY(Ew<T>::dot(Z_[n], Z_[n], blk_, sc_ + S_ZZ, nullptr, cx.stream));
        CDMPT_TRY(read_scalars(cx, sc_, S_NSLOTS));
        trP = 0.5 * (N + cx.pinned[S_TRZ]);
        zz = cx.pinned[S_ZZ];
        const double err = trP - nocc;
        st.mu = mu;
        st.trace_P0 = trP;
        st.occupation_error = std::fabs(err);
        if (std::fabs(err) <= occ_tol) {
            converged = true;
            break;
        }
        if (err > 0)
            hi = mu;
        else
            lo = mu;
        const double slope = 0.25 * beta * (N - zz);
        double mu_new = slope > 0 ? mu - err / slope : 0.5 * (lo + hi);
        if (!(mu_new > lo && mu_new < hi)) mu_new = 0.5 * (lo + hi);
        if (mu_new == mu) break;
        mu = mu_new;
    }
    if (!converged) {
        set_error("occupation did not converge: |Tr P0 - N_occ| = " +
                  std::to_string(st.occupation_error) + " after " +
                  std::to_string(st.mu_iterations) + " sweeps");
        return CDMPT_ERR_NO_CONVERGENCE;
    }
    if (mu_out) *mu_out = mu;

    // -------------------------------------------------- first-order response
    if (D > 0) {
        const int rows = D * N;
        const size_t count = (size_t)rows * ld;
        T* Z1 = Z1a_;
        T* Z1n = Z1b_;
        CDMPT_TRY(Ew<T>::init_z(Z1, H1, N, ld, ld, D, -s2, 0.0, cx.stream));
        int total = 0, hint = 1;
        for (int k = 0; k < n; ++k) {
            {   // S^T = Z1 Z_k (stacked over directions)
                Epilogue<T> ep;
                CDMPT_TRY(gemm(cx, rows, N, N, Z1, Z_[k], S_, ep, nullptr));
            }
            // A1 = Z_k Z1 + Z1 Z_k, block by block
            CDMPT_TRY(Ew<T>::transpose_add(A1_, S_, N, ld, D, cx.stream));
            {   // RHS = 2 Z1 - Z_{k+1} A1 = (2 Z1 - A1 Z_{k+1})^T per block
                Epilogue<T> ep;
                ep.alpha = -1.0;
                ep.beta = 2.0;
                ep.C = Z1;
                ep.ldc = ld;
                ep.trans_block = N;
                CDMPT_TRY(gemm(cx, rows, N, N, A1_, Z_[k + 1], RHS_, ep, nullptr));
            }
            CDMPT_TRY(Ew<T>::axpby(Z1n, Z1, count, 2.0, 0.0, nullptr, cx.stream));
            int it = hint;
            CDMPT_TRY(cg(cx, Z1n, A_[k], RHS_, 1.0, rows, o.cg_tol, o.cg_maxit, &it));
            total += it;
            hint = std::max(1, it);
            CDMPT_TRY(Ew<T>::symmetrize(Z1n, N, ld, D, cx.stream));
            std::swap(Z1, Z1n);
        }
        st.cg_iterations_response = total;

        // Q = dP0/dmu = beta/4 (I - Z_n^2)(I - Z_0^2)^-1
        {
            Epilogue<T> ep;
            ep.alpha = -0.25 * beta;
            ep.gamma = 0.25 * beta;
            CDMPT_TRY(gemm(cx, N, N, N, Z_[n], Z_[n], RHS_, ep, nullptr));
            Epilogue<T> em;
            em.alpha = -1.0;
            em.gamma = 1.0;
            CDMPT_TRY(gemm(cx, N, N, N, Z_[0], Z_[0], Mq_, em, nullptr));
            CDMPT_TRY(Ew<T>::axpby(Qmu_, RHS_, blk_, 1.0, 0.0, nullptr, cx.stream));
            int it = 1;
            CDMPT_TRY(cg(cx, Qmu_, Mq_, RHS_, 1.0, N, o.cg_tol, o.cg_maxit, &it));
            st.cg_iterations_q = it;
            CDMPT_TRY(Ew<T>::symmetrize(Qmu_, N, ld, 1, cx.stream));
        }
        CDMPT_CUDA_TRY(cudaMemsetAsync(sc_ + S_TRQ, 0, (S_NSLOTS - S_TRQ) * sizeof(double),
                                       cx.stream));
        CDMPT_TRY(Ew<T>::trace(Qmu_, N, ld, 1, sc_ + S_TRQ, cx.stream));
        CDMPT_TRY(Ew<T>::trace(Z1, N, ld, D, sc_ + S_TRZ1, cx.stream));
        CDMPT_TRY(read_scalars(cx, sc_, S_NSLOTS));
        const double trQ = cx.pinned[S_TRQ];
        st.trace_Q = trQ;
        for (int d = 0; d < D; ++d) {
            const double trP1 = 0.5 * cx.pinned[S_TRZ1 + d];
            const double mu1 = trQ > 0 ? -trP1 / trQ : 0.0;
            if (mu1_out) mu1_out[d] = mu1;
            // P1 = Z1/2 + mu1 Q  <=>  Z1 += 2 mu1 Q
            CDMPT_TRY(Ew<T>::axpby(Z1 + (size_t)d * blk_, Qmu_, blk_, 2.0 * mu1, 1.0, nullptr,
                                   cx.stream));
            CDMPT_TRY(Ew<T>::diag_dot(Z1 + (size_t)d * blk_, H1 + (size_t)d * blk_, N, ld, ld,
                                      sc_ + S_ALPHA + d, cx.stream));
        }
        CDMPT_CUDA_TRY(cudaMemsetAsync(sc_ + S_TRZ1, 0, kMaxD * sizeof(double), cx.stream));
        CDMPT_TRY(Ew<T>::trace(Z1, N, ld, D, sc_ + S_TRZ1, cx.stream));
        if (P1) {
            if (out_on_device) {
                CDMPT_TRY(Ew<T>::to_f64(P1, N, Z1, ld, N, rows, 0.5, 0.0, cx.stream));
            } else {
                double* tmp = nullptr;
                CDMPT_CUDA_TRY(cudaMallocAsync((void**)&tmp, (size_t)rows * N * sizeof(double),
                                               cx.stream));
                CDMPT_TRY(Ew<T>::to_f64(tmp, N, Z1, ld, N, rows, 0.5, 0.0, cx.stream));
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

    if (P0) {
        if (out_on_device) {
            CDMPT_TRY(Ew<T>::to_f64(P0, N, Z_[n], ld, N, N, 0.5, 0.5, cx.stream));
        } else {
            double* tmp = nullptr;
            CDMPT_CUDA_TRY(cudaMallocAsync((void**)&tmp, (size_t)N * N * sizeof(double), cx.stream));
            CDMPT_TRY(Ew<T>::to_f64(tmp, N, Z_[n], ld, N, N, 0.5, 0.5, cx.stream));
            CDMPT_CUDA_TRY(cudaMemcpyAsync(P0, tmp, (size_t)N * N * sizeof(double),
                                           cudaMemcpyDeviceToHost, cx.stream));
            CDMPT_CUDA_TRY(cudaFreeAsync(tmp, cx.stream));
        }
    }
    CDMPT_CUDA_TRY(cudaStreamSynchronize(cx.stream));
    return check_device_error(cx.stream);
}

template class Solver<float>;
template class Solver<double>;

}  // namespace cdmpt
