// C ABI of libcdmpt.so (declared in include/cdmpt.h).
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "cdmpt.h"
#include "overlap.cuh"
#include "scc.cuh"
#include "solver.cuh"

namespace cdmpt {

namespace {
thread_local std::string g_err;
std::mutex g_err_word_mu;
int* g_err_word[64] = {nullptr};
}  // namespace

void set_error(const std::string& msg) { g_err = msg; }
const std::string& get_error() { return g_err; }

int* device_error_word() {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_err_word_mu);
    if (!g_err_word[dev]) {
        int* p = nullptr;
        if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        cudaMemset(p, 0, sizeof(int));
        cudaDeviceSynchronize();
        g_err_word[dev] = p;
    }
    return g_err_word[dev];
}

cdmpt_status check_device_error(cudaStream_t s) {
    int* w = device_error_word();
    if (!w) return CDMPT_OK;
    int host = 0;
    CDMPT_CUDA_TRY(cudaMemcpyAsync(&host, w, sizeof(int), cudaMemcpyDeviceToHost, s));
    CDMPT_CUDA_TRY(cudaStreamSynchronize(s));
    if (host != DEV_OK) {
        CDMPT_CUDA_TRY(cudaMemsetAsync(w, 0, sizeof(int), s));
        set_error("a bounded device wait gave up (code " + std::to_string(host) + ")");
        return CDMPT_ERR_TIMEOUT;
    }
    return CDMPT_OK;
}

}  // namespace cdmpt

using namespace cdmpt;

struct cdmpt_handle {
    cdmpt_opts opts;
    int device = 0;
    int N = 0, D = 0, ld = 0;
    double* H0 = nullptr;     // N x ld, FP64, zero padding
    double* H1 = nullptr;     // D x N x ld
    double* H2 = nullptr;     // D x N x ld higher perturbation terms (cdmpt_set_H_orders), or null
    double* H3 = nullptr;
    double* dscal = nullptr;  // device scalars for set_H (bounds, trace)
    double gmin = 0, gmax = 0, trH0 = 0;
    Solver<float>* sf = nullptr;
    Solver<double>* sd = nullptr;
    Context cx;
    cdmpt_stats st;
    std::string err;
    bool solved = false;
    std::vector<double> alpha;
    // non-orthogonal basis (cdmpt_set_overlap): Loewdin factor Z = S^(-1/2), N x ld FP64,
    // and 2 N x ld doubles of scratch for the congruences X -> Z X Z
    double* Zov = nullptr;
    double* Sov = nullptr;     // S itself (N x ld), for the Mulliken charges of the SCC layer
    double* ovtmp = nullptr;
    int ovN = 0, ov_iters = 0;
    double ov_resid = 0;
};

namespace {

cdmpt_status fail(cdmpt_handle* h, cdmpt_status s) {
    if (h) h->err = get_error();
    return s;
}

cdmpt_status fail_msg(cdmpt_handle* h, cdmpt_status s, const std::string& m) {
    set_error(m);
    return fail(h, s);
}

// Non-orthogonal mode: dst_b = Z src_b Z for `blocks` FP64 N x N matrices (leading
// dimension N) held on the device, written to device or host memory.
cdmpt_status ov_map(cdmpt_handle* h, const double* src, double* dst, int blocks,
                    int dst_on_device) {
    const int N = h->N, ld = h->ld;
    const size_t nn = (size_t)N * N, blk = (size_t)N * ld;
    cudaStream_t s = h->cx.stream;
    for (int b = 0; b < blocks; ++b) {
        double* out = dst_on_device ? dst + b * nn : h->ovtmp + blk;
        CDMPT_TRY(congruence(h->Zov, ld, N, src + b * nn, N, out, N, h->ovtmp, s));
        if (!dst_on_device) {
            CDMPT_CUDA_TRY(cudaMemcpyAsync(dst + b * nn, out, nn * sizeof(double),
                                           cudaMemcpyDeviceToHost, s));
            CDMPT_CUDA_TRY(cudaStreamSynchronize(s));
        }
    }
    return CDMPT_OK;
}

bool valid_opts(const cdmpt_opts* o) {
    if (o->precision < CDMPT_FP64 || o->precision > CDMPT_MIXED_BF16) return false;
    if (o->gemm_engine < CDMPT_GEMM_AUTO || o->gemm_engine > CDMPT_GEMM_TC_OZAKI) return false;
    // the Ozaki engine is a choice of the FP64 precision only
    if (o->gemm_engine == CDMPT_GEMM_TC_OZAKI && o->precision != CDMPT_FP64) return false;
    if (o->cg_maxit < 1 || o->mu_maxit < 1 || o->refine_rounds < 0) return false;
    if (o->grand_canonical && !o->have_mu_guess) return false;
    if (o->ckpt_stride < -1) return false;
    if (o->fp64_residual < -1 || o->fp64_residual > 1) return false;
    if (o->ckpt_stride != 0 &&
        (o->precision == CDMPT_MIXED_TF32 || o->precision == CDMPT_MIXED_BF16))
        return false;
    // screened products run on the tcgen05 TF32 engines only
    if (!(o->screen_tau >= 0.0) || o->screen_tau > 1e30) return false;
    if (o->screen_tau > 0.0 &&
        ((o->precision != CDMPT_FP32 && o->precision != CDMPT_MIXED_TF32) ||
         (o->gemm_engine != CDMPT_GEMM_AUTO && o->gemm_engine != CDMPT_GEMM_TC_TF32 &&
          o->gemm_engine != CDMPT_GEMM_TC_3XTF32)))
        return false;
    return true;
}

void normalise(cdmpt_opts* o) {
    if (!(o->cg_tol > 0)) o->cg_tol = o->precision == CDMPT_FP64 ? 1e-13 : 1e-7;
}

}  // namespace

extern "C" {

int cdmpt_version(void) { return (CDMPT_VERSION_MAJOR << 16) | CDMPT_VERSION_MINOR; }

cdmpt_status cdmpt_default_opts(cdmpt_opts* o) {
    if (!o) return CDMPT_ERR_ARG;
    std::memset(o, 0, sizeof(*o));
    o->precision = CDMPT_FP32;
    o->gemm_engine = CDMPT_GEMM_AUTO;
    o->cg_tol = 0.0;
    o->cg_maxit = 200;
    o->refine_rounds = 2;
    o->occ_tol = 0.0;
    o->mu_maxit = 60;
    o->have_mu_guess = 0;
    o->mu_guess = 0.0;
    o->profile = 0;
    o->stream = nullptr;
    o->grand_canonical = 0;
    o->ckpt_stride = 0;
    o->fd_exact = 0;
    o->screen_tau = 0.0;
    o->fp64_residual = 0;
    return CDMPT_OK;
}

cdmpt_status cdmpt_set_opts(cdmpt_handle* h, const cdmpt_opts* opts) {
    if (!h || !opts) return CDMPT_ERR_ARG;
    if (!valid_opts(opts)) return fail_msg(h, CDMPT_ERR_ARG, "invalid options");
    const bool needs_tc =
        opts->precision != CDMPT_FP64 &&
        (opts->gemm_engine == CDMPT_GEMM_AUTO || opts->gemm_engine >= CDMPT_GEMM_TC_TF32);
    if (needs_tc && !tc_supported())
        return fail_msg(h, CDMPT_ERR_UNSUPPORTED,
                        "tcgen05 engines need an sm_103 GPU; choose CDMPT_GEMM_SIMT or FP64");
    h->opts = *opts;
    normalise(&h->opts);
    h->cx.stream = (cudaStream_t)h->opts.stream;
    h->cx.engine = h->opts.gemm_engine;
    h->cx.profile = h->opts.profile != 0;
    return CDMPT_OK;
}

cdmpt_status cdmpt_create(const cdmpt_opts* opts, cdmpt_handle** out) {
    if (!out) return CDMPT_ERR_ARG;
    *out = nullptr;
    cdmpt_opts o;
    if (opts)
        o = *opts;
    else
        cdmpt_default_opts(&o);
    if (!valid_opts(&o)) {   // host-side check before any device call
        set_error("invalid options");
        return CDMPT_ERR_ARG;
    }
    cdmpt_handle* h = new (std::nothrow) cdmpt_handle();
    if (!h) return CDMPT_ERR_OOM;
    std::memset(&h->st, 0, sizeof(h->st));
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        set_error("no CUDA device");
        return CDMPT_ERR_CUDA;
    }
    cdmpt_status s = cdmpt_set_opts(h, &o);
    if (s != CDMPT_OK) {
        delete h;
        return s;
    }
    if (cudaMallocHost((void**)&h->cx.pinned, 64 * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&h->dscal, 8 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        set_error("allocation of handle scalars failed");
        cdmpt_destroy(h);
        return CDMPT_ERR_OOM;
    }
    *out = h;
    return CDMPT_OK;
}

cdmpt_status cdmpt_set_overlap(cdmpt_handle* h, int N, const double* S, int on_device) {
    if (!h) return CDMPT_ERR_ARG;
    cudaStream_t s = h->cx.stream;
    // the stored Hamiltonian belongs to the previous basis: cdmpt_set_H must follow
    cudaFree(h->H0);
    cudaFree(h->H1);
    cudaFree(h->H2);
    cudaFree(h->H3);
    h->H0 = h->H1 = h->H2 = h->H3 = nullptr;
    h->N = h->D = h->ld = 0;
    h->solved = false;
    cudaFree(h->Zov);
    cudaFree(h->Sov);
    cudaFree(h->ovtmp);
    h->Zov = h->Sov = h->ovtmp = nullptr;
    h->ovN = 0;
    if (!S) return CDMPT_OK;
    if (N < 1) return fail_msg(h, CDMPT_ERR_ARG, "set_overlap: need N >= 1");
    const int ld = (N + 31) / 32 * 32;
    const size_t blk = (size_t)N * ld;
    double* work = nullptr;   // four Newton-Schulz iterates
    if (cudaMalloc((void**)&work, 4 * blk * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&h->Zov, blk * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&h->Sov, blk * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&h->ovtmp, 2 * blk * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(work);
        cudaFree(h->Zov);
        cudaFree(h->Sov);
        cudaFree(h->ovtmp);
        h->Zov = h->Sov = h->ovtmp = nullptr;
        return fail_msg(h, CDMPT_ERR_OOM, "set_overlap: device allocation failed");
    }
    double* Sd = h->Sov;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cdmpt_status st = CDMPT_OK;
    double host[2] = {0, 0};
    if (cudaMemsetAsync(Sd, 0, blk * sizeof(double), s) != cudaSuccess ||
        cudaMemsetAsync(h->Zov, 0, blk * sizeof(double), s) != cudaSuccess ||
        cudaMemcpy2DAsync(Sd, ld * sizeof(double), S, N * sizeof(double), N * sizeof(double), N,
                          kind, s) != cudaSuccess ||
        cudaMemsetAsync(h->dscal, 0, 8 * sizeof(double), s) != cudaSuccess) {
        set_error("set_overlap: copy of S failed");
        st = CDMPT_ERR_CUDA;
    }
    if (st == CDMPT_OK) st = gershgorin(Sd, N, ld, h->dscal, s);
    if (st == CDMPT_OK &&
        (cudaMemcpyAsync(host, h->dscal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s) !=
             cudaSuccess ||
         cudaStreamSynchronize(s) != cudaSuccess)) {
        set_error("set_overlap: reading the bounds of S failed");
        st = CDMPT_ERR_CUDA;
    }
    if (st == CDMPT_OK && !(host[1] > 0)) {
        set_error("set_overlap: S has no positive Gershgorin bound");
        st = CDMPT_ERR_ARG;
    }
    int it = 0;
    double res = 0;
    if (st == CDMPT_OK)
        st = lowdin_factor(Sd, N, ld, host[1], h->Zov, work, h->dscal + 4, 200, 1e-12, &it, &res,
                           s);
    cudaStreamSynchronize(s);
    cudaFree(work);
    if (st != CDMPT_OK) {
        cudaFree(h->Zov);
        cudaFree(h->Sov);
        cudaFree(h->ovtmp);
        h->Zov = h->Sov = h->ovtmp = nullptr;
        return fail(h, st);
    }
    h->ovN = N;
    h->ov_iters = it;
    h->ov_resid = res;
    return CDMPT_OK;
}

cdmpt_status cdmpt_get_overlap_info(const cdmpt_handle* h, int* iterations, double* residual) {
    if (!h) return CDMPT_ERR_ARG;
    if (iterations) *iterations = h->ovN ? h->ov_iters : 0;
    if (residual) *residual = h->ovN ? h->ov_resid : 0.0;
    return CDMPT_OK;
}

cdmpt_status cdmpt_set_H(cdmpt_handle* h, int N, const double* H0, int D, const double* H1,
                         int on_device) {
    if (!h) return CDMPT_ERR_ARG;
    if (N < 1 || D < 0 || !H0 || (D > 0 && !H1))
        return fail_msg(h, CDMPT_ERR_ARG, "set_H: need N >= 1, D >= 0, H0 and (D > 0) H1");
    if (D > 16) return fail_msg(h, CDMPT_ERR_ARG, "set_H: at most 16 perturbation directions");
    cudaStream_t s = h->cx.stream;
    const int ld = (N + 31) / 32 * 32;
    const size_t blk = (size_t)N * ld;
    cudaFree(h->H2);   // higher perturbation terms belong to the previous H1
    cudaFree(h->H3);
    h->H2 = h->H3 = nullptr;
    if (N != h->N || D != h->D || ld != h->ld) {
        cudaFree(h->H0);
        cudaFree(h->H1);
        h->H0 = h->H1 = nullptr;
        if (cudaMalloc((void**)&h->H0, blk * sizeof(double)) != cudaSuccess ||
            (D > 0 && cudaMalloc((void**)&h->H1, D * blk * sizeof(double)) != cudaSuccess)) {
            cudaGetLastError();
            h->N = 0;
            return fail_msg(h, CDMPT_ERR_OOM, "set_H: device allocation failed");
        }
        h->N = N;
        h->D = D;
        h->ld = ld;
    }
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CDMPT_CUDA_TRY(cudaMemsetAsync(h->H0, 0, blk * sizeof(double), s));
    CDMPT_CUDA_TRY(cudaMemcpy2DAsync(h->H0, ld * sizeof(double), H0, N * sizeof(double),
                                     N * sizeof(double), N, kind, s));
    if (D > 0) {
        CDMPT_CUDA_TRY(cudaMemsetAsync(h->H1, 0, D * blk * sizeof(double), s));
        CDMPT_CUDA_TRY(cudaMemcpy2DAsync(h->H1, ld * sizeof(double), H1, N * sizeof(double),
                                         N * sizeof(double), (size_t)D * N, kind, s));
    }
    if (h->ovN) {   // non-orthogonal input: F_perp = Z F Z, h1_perp = Z h1 Z (Eq. Fermi_D)
        if (N != h->ovN)
            return fail_msg(h, CDMPT_ERR_ARG, "set_H: N differs from the overlap's size");
        cdmpt_status st = congruence(h->Zov, ld, N, h->H0, ld, h->H0, ld, h->ovtmp, s);
        for (int d = 0; d < D && st == CDMPT_OK; ++d)
            st = congruence(h->Zov, ld, N, h->H1 + d * blk, ld, h->H1 + d * blk, ld, h->ovtmp, s);
        if (st != CDMPT_OK) return fail(h, st);
    }
    CDMPT_CUDA_TRY(cudaMemsetAsync(h->dscal, 0, 8 * sizeof(double), s));
    cdmpt_status st = gershgorin(h->H0, N, ld, h->dscal, s);
    if (st != CDMPT_OK) return fail(h, st);
    st = Ew<double>::trace(h->H0, N, ld, 1, h->dscal + 2, s);
    if (st != CDMPT_OK) return fail(h, st);
    double host[3];
    CDMPT_CUDA_TRY(cudaMemcpyAsync(host, h->dscal, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CDMPT_CUDA_TRY(cudaStreamSynchronize(s));
    h->gmin = host[0];
    h->gmax = host[1];
    h->trH0 = host[2];
    h->solved = false;
    return CDMPT_OK;
}

cdmpt_status cdmpt_set_H_orders(cdmpt_handle* h, const double* H2, const double* H3,
                                int on_device) {
    if (!h) return CDMPT_ERR_ARG;
    if (h->N < 1 || h->D < 1)
        return fail_msg(h, CDMPT_ERR_ARG, "set_H_orders: call cdmpt_set_H with directions first");
    cudaStream_t s = h->cx.stream;
    const int N = h->N, D = h->D, ld = h->ld;
    const size_t blk = (size_t)N * ld;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const double* src[2] = {H2, H3};
    double** dst[2] = {&h->H2, &h->H3};
    for (int t = 0; t < 2; ++t) {
        cudaFree(*dst[t]);
        *dst[t] = nullptr;
        if (!src[t]) continue;
        if (cudaMalloc((void**)dst[t], D * blk * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return fail_msg(h, CDMPT_ERR_OOM, "set_H_orders: device allocation failed");
        }
        CDMPT_CUDA_TRY(cudaMemsetAsync(*dst[t], 0, D * blk * sizeof(double), s));
        CDMPT_CUDA_TRY(cudaMemcpy2DAsync(*dst[t], ld * sizeof(double), src[t], N * sizeof(double),
                                         N * sizeof(double), (size_t)D * N, kind, s));
        for (int d = 0; d < D && h->ovN; ++d) {   // non-orthogonal input: Z H Z
            const cdmpt_status st = congruence(h->Zov, ld, N, *dst[t] + d * blk, ld,
                                               *dst[t] + d * blk, ld, h->ovtmp, s);
            if (st != CDMPT_OK) return fail(h, st);
        }
    }
    CDMPT_CUDA_TRY(cudaStreamSynchronize(s));
    return CDMPT_OK;
}

cdmpt_status cdmpt_solve(cdmpt_handle* h, double beta, double nocc, int n, double* P0,
                         double* P1, double* mu, double* mu1, int out_on_device) {
    if (!h) return CDMPT_ERR_ARG;
    if (h->N < 1) return fail_msg(h, CDMPT_ERR_ARG, "solve: call cdmpt_set_H first");
    const bool gc = h->opts.grand_canonical != 0;   // nocc unused at fixed mu
    if (!(beta > 0) || (!gc && (!(nocc > 0) || !(nocc < h->N))) || n < 1 || n > 60)
        return fail_msg(h, CDMPT_ERR_ARG, "solve: need beta > 0, 0 < nocc < N, 1 <= n <= 60");
    std::memset(&h->st, 0, sizeof(h->st));
    h->st.N = h->N;
    h->st.D = h->D;
    h->st.n = n;
    h->cx.st = &h->st;
    h->cx.ev_used = 0;
    for (bool& b : h->cx.ph_set) b = false;
    h->solved = false;
    h->alpha.assign(h->D, 0.0);
    const long long launches0 = launch_count();
    const auto t0 = std::chrono::steady_clock::now();
    // non-orthogonal mode: the solver writes P_perp to device scratch, mapped to D = Z P Z below
    double* P0u = P0;
    double* P1u = (h->D > 0) ? P1 : nullptr;
    int od = out_on_device;
    double* scratch = nullptr;
    const size_t nn = (size_t)h->N * h->N;
    if (h->ovN && (P0u || P1u)) {
        const size_t elems = (P0u ? nn : 0) + (P1u ? (size_t)h->D * nn : 0);
        CDMPT_CUDA_TRY(cudaMallocAsync((void**)&scratch, elems * sizeof(double), h->cx.stream));
        P0u = P0 ? scratch : nullptr;
        P1u = P1u ? scratch + (P0 ? nn : 0) : nullptr;
        od = 1;
    }
    cdmpt_status s;
    if (h->opts.precision == CDMPT_FP64) {
        if (!h->sd) h->sd = new (std::nothrow) Solver<double>();
        if (!h->sd) return fail_msg(h, CDMPT_ERR_OOM, "solver allocation");
        s = h->sd->solve(h->cx, h->H0, h->H1, h->N, h->D, h->gmin, h->gmax, h->trH0, h->opts,
                         beta, nocc, n, P0u, P1u, mu, mu1, od, h->alpha.data());
    } else {
        if (!h->sf) h->sf = new (std::nothrow) Solver<float>();
        if (!h->sf) return fail_msg(h, CDMPT_ERR_OOM, "solver allocation");
        s = h->sf->solve(h->cx, h->H0, h->H1, h->N, h->D, h->gmin, h->gmax, h->trH0, h->opts,
                         beta, nocc, n, P0u, P1u, mu, mu1, od, h->alpha.data());
    }
    if (scratch) {
        if (s == CDMPT_OK && P0u) s = ov_map(h, P0u, P0, 1, out_on_device);
        if (s == CDMPT_OK && P1u) s = ov_map(h, P1u, P1, h->D, out_on_device);
        cudaFreeAsync(scratch, h->cx.stream);
        cudaStreamSynchronize(h->cx.stream);
    }
    h->st.kernel_launches = (int)(launch_count() - launches0);
    h->st.seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (h->cx.profile && s == CDMPT_OK) {
        double ms = 0;
        int timed = 0;
        for (size_t i = 0; i < h->cx.ev_used; ++i) {
            if (!h->cx.ev_ok[i]) continue;
            float e = 0;
            if (cudaEventElapsedTime(&e, h->cx.ev[2 * i], h->cx.ev[2 * i + 1]) == cudaSuccess) {
                ms += e;
                ++timed;
                const int eng = h->cx.ev_engine[i];
                if (eng < 0 || eng > 5) continue;
                h->st.engine_ms[eng] += e;
                h->st.engine_launches[eng] += 1;
                h->st.engine_flops[eng] += h->cx.ev_flops[i];
            }
        }
        h->st.gemm_ms = ms;
        h->st.gemm_timed = timed;
        // phases: the span from each recorded boundary to the next recorded one
        for (int i = 0; i < 5; ++i) {
            if (!h->cx.ph_set[i]) continue;
            int j = i + 1;
            while (j < 6 && !h->cx.ph_set[j]) ++j;
            float e = 0;
            if (j < 6 && cudaEventElapsedTime(&e, h->cx.ph[i], h->cx.ph[j]) == cudaSuccess)
                h->st.phase_ms[i] = e;
        }
    }
    if (s != CDMPT_OK) return fail(h, s);
    h->solved = true;
    return CDMPT_OK;
}

cdmpt_status cdmpt_spectral_bounds(const double* H, int N, int ldh, double* bounds, void* stream) {
    if (!H || !bounds || N < 1 || ldh < N) {
        set_error("spectral_bounds: need H, bounds, N >= 1 and ldh >= N");
        return CDMPT_ERR_ARG;
    }
    return gershgorin(H, N, ldh, bounds, (cudaStream_t)stream);
}

cdmpt_status cdmpt_spectral_bounds_noalloc(const double* H, int N, int ldh, double* bounds,
                                           void* stream) {
    if (!H || !bounds || N < 1 || ldh < N) {
        set_error("spectral_bounds_noalloc: need H, bounds, N >= 1 and ldh >= N");
        return CDMPT_ERR_ARG;
    }
    return gershgorin_noalloc(H, N, ldh, bounds, (cudaStream_t)stream);
}

cdmpt_status cdmpt_vjp_P0(cdmpt_handle* h, const double* G0, double* gradH0, int on_device) {
    if (!h) return CDMPT_ERR_ARG;
    if (!G0 || !gradH0) return fail_msg(h, CDMPT_ERR_ARG, "vjp_P0: NULL pointer");
    if (!h->solved) return fail_msg(h, CDMPT_ERR_ARG, "vjp_P0: no completed solve on this handle");
    cudaStream_t s = h->cx.stream;
    const size_t nn = (size_t)h->N * h->N;
    const size_t bytes = nn * sizeof(double);
    const bool ov = h->ovN != 0;
    const double* g = G0;
    double* out = gradH0;
    double* tmp = nullptr;
    if (!on_device || ov) {   // [G0 on the device | Z G0 Z | gradient]
        CDMPT_CUDA_TRY(cudaMallocAsync((void**)&tmp, 3 * bytes, s));
        if (!on_device) {
            CDMPT_CUDA_TRY(cudaMemcpyAsync(tmp, G0, bytes, cudaMemcpyHostToDevice, s));
            g = tmp;
        }
        out = tmp + 2 * nn;
    }
    cdmpt_status st = CDMPT_OK;
    if (ov) {   // D = Z P_perp Z, so dL/dP_perp = Z G0 Z
        st = ov_map(h, g, tmp + nn, 1, 1);
        g = tmp + nn;
    }
    cdmpt_stats keep = h->st;
    h->cx.st = &h->st;
    if (st == CDMPT_OK) {
        if (h->opts.precision == CDMPT_FP64)
            st = h->sd ? h->sd->vjp_p0(h->cx, g, out) : CDMPT_ERR_ARG;
        else
            st = h->sf ? h->sf->vjp_p0(h->cx, g, out) : CDMPT_ERR_ARG;
    }
    h->st = keep;
    if (st == CDMPT_OK && ov) {   // F_perp = Z F Z, so dL/dF = Z (dL/dF_perp) Z
        st = ov_map(h, out, gradH0, 1, on_device);
    } else if (st == CDMPT_OK && !on_device) {
        CDMPT_CUDA_TRY(cudaMemcpyAsync(gradH0, out, bytes, cudaMemcpyDeviceToHost, s));
        CDMPT_CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (tmp) cudaFreeAsync(tmp, s);
    if (st != CDMPT_OK) return fail(h, st);
    return CDMPT_OK;
}

cdmpt_status cdmpt_free_energy(cdmpt_handle* h, double* omega, double* gradH0, int on_device) {
    if (!h) return CDMPT_ERR_ARG;
    if (!h->solved)
        return fail_msg(h, CDMPT_ERR_ARG, "free_energy: no completed solve on this handle");
    cudaStream_t s = h->cx.stream;
    const size_t bytes = (size_t)h->N * h->N * sizeof(double);
    double* g = gradH0;
    double* tmp = nullptr;
    const bool ov = h->ovN != 0;
    if (gradH0 && (!on_device || ov)) {
        CDMPT_CUDA_TRY(cudaMallocAsync((void**)&tmp, bytes, s));
        g = tmp;
    }
    cdmpt_stats keep = h->st;
    h->cx.st = &h->st;
    double om = 0.0;
    cdmpt_status st;
    if (h->opts.precision == CDMPT_FP64)
        st = h->sd ? h->sd->free_energy(h->cx, &om, g) : CDMPT_ERR_ARG;
    else
        st = h->sf ? h->sf->free_energy(h->cx, &om, g) : CDMPT_ERR_ARG;
    h->st = keep;
    if (st == CDMPT_OK && gradH0 && ov) {
        st = ov_map(h, g, gradH0, 1, on_device);   // dOmega/dF = Z (dOmega/dF_perp) Z
    } else if (st == CDMPT_OK && gradH0 && !on_device) {
        CDMPT_CUDA_TRY(cudaMemcpyAsync(gradH0, g, bytes, cudaMemcpyDeviceToHost, s));
        CDMPT_CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (tmp) cudaFreeAsync(tmp, s);
    if (st != CDMPT_OK) return fail(h, st);
    if (omega) *omega = om;
    return CDMPT_OK;
}

// Self-consistent charge layer (Sec. IV with a synthetic G(D)); see cdmpt_scc_solve in cdmpt.h.
cdmpt_status cdmpt_scc_solve2(cdmpt_handle* h, const cdmpt_scc_model* m, int N,
                              const double* hcore, int D, const double* h1, double beta,
                              double nocc, int n, double* D0, double* D1, double* mu, double* mu1,
                              double* omega1, double* omega2, double* D2, double* mu2,
                              double* omega3, int* iters, int on_device) {
    const bool second = D2 || mu2 || omega3;
    if (!h) return CDMPT_ERR_ARG;
    if (!m || !m->gamma || !hcore || N < 1 || D < 0 || D > 16 || (D > 0 && !h1))
        return fail_msg(h, CDMPT_ERR_ARG,
                        "scc_solve: need the model (gamma), hcore, N >= 1, 0 <= D <= 16 and h1");
    if (h->ovN && h->ovN != N)
        return fail_msg(h, CDMPT_ERR_ARG, "scc_solve: N differs from the overlap's size");
    if (h->opts.grand_canonical)
        return fail_msg(h, CDMPT_ERR_ARG, "scc_solve: the self-consistent layer is canonical");
    cudaStream_t s = h->cx.stream;
    const int ld = (N + 31) / 32 * 32;
    const size_t nn = (size_t)N * N, blk = (size_t)N * ld;
    const double tol = m->tol > 0 ? m->tol : (h->opts.precision == CDMPT_FP64 ? 1e-10 : 1e-6);
    const int maxit = m->maxit > 0 ? m->maxit : 200;
    const int depth = m->history > 0 ? m->history : 6;
    const double mix = m->mix > 0 ? m->mix : 0.3;
    // device work: hcore, gamma, F, D, D1 (orthogonal), D1 (caller's basis), h1, F1 (padded),
    // q0, dq, V; for the second order also F2 (padded) and a zero matrix
    double* w = nullptr;
    const size_t elems = 6 * nn + (size_t)D * nn + blk + 3 * (size_t)N + (second ? blk + nn : 0);
    if (cudaMalloc((void**)&w, elems * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail_msg(h, CDMPT_ERR_OOM, "scc_solve: device allocation failed");
    }
    double *hc = w, *gam = hc + nn, *F = gam + nn, *Dd = F + nn, *D1p = Dd + nn, *D1d = D1p + nn;
    double *h1d = D1d + nn, *F1 = h1d + (size_t)D * nn, *q0d = F1 + blk, *dq = q0d + N,
           *V = dq + N;
    double* F2 = second ? V + N : nullptr;
    double* zero = second ? F2 + blk : nullptr;
    const double* Sg = h->ovN ? h->Sov : nullptr;
    const cdmpt_opts saved = h->opts;
    cdmpt_status st = CDMPT_OK;
    int scf_it = 0, cp_it = 0;
    double mu_last = 0.0;
    auto cuda_ok = [&](cudaError_t e, const char* what) {
        if (e != cudaSuccess && st == CDMPT_OK) {
            set_error(std::string("scc_solve: ") + what + ": " + cudaGetErrorString(e));
            st = CDMPT_ERR_CUDA;
        }
    };
    const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cuda_ok(cudaMemcpyAsync(hc, hcore, nn * sizeof(double), kin, s), "copy hcore");
    cuda_ok(cudaMemcpyAsync(gam, m->gamma, nn * sizeof(double), kin, s), "copy gamma");
    if (D > 0) cuda_ok(cudaMemcpyAsync(h1d, h1, D * nn * sizeof(double), kin, s), "copy h1");
    cuda_ok(cudaMemsetAsync(q0d, 0, N * sizeof(double), s), "zero q0");
    if (m->q0) cuda_ok(cudaMemcpyAsync(q0d, m->q0, N * sizeof(double), kin, s), "copy q0");
    cuda_ok(cudaMemsetAsync(F1, 0, blk * sizeof(double), s), "zero F1");
    if (second) {
        cuda_ok(cudaMemsetAsync(F2, 0, blk * sizeof(double), s), "zero F2");
        cuda_ok(cudaMemsetAsync(zero, 0, nn * sizeof(double), s), "zero matrix");
    }
    std::vector<double> x(N, 0.0), y(N), r(N);
    // ---- SCF on the charges: F = h + G(D(F)) (a fixed point in dq)
    bool conv = false;
    {
        Anderson mixer(N, depth, mix);
        for (; st == CDMPT_OK && scf_it < maxit; ++scf_it) {
            cuda_ok(cudaMemcpyAsync(dq, x.data(), N * sizeof(double), cudaMemcpyHostToDevice, s),
                    "charges to device");
            if (st == CDMPT_OK) st = scc_gemv(gam, N, dq, N, V, s);
            if (st == CDMPT_OK) st = scc_fock(hc, N, Sg, ld, V, N, F, N, s);
            if (st == CDMPT_OK) st = cdmpt_set_H(h, N, F, 0, nullptr, 1);
            if (st == CDMPT_OK && scf_it > 0) {   // warm start mu from the previous iteration
                h->opts.have_mu_guess = 1;
                h->opts.mu_guess = mu_last;
            }
            if (st == CDMPT_OK) st = cdmpt_solve(h, beta, nocc, n, Dd, nullptr, &mu_last, nullptr, 1);
            if (st == CDMPT_OK) st = scc_charges(Dd, N, Sg, ld, q0d, N, dq, s);
            cuda_ok(cudaMemcpyAsync(y.data(), dq, N * sizeof(double), cudaMemcpyDeviceToHost, s),
                    "charges to host");
            cuda_ok(cudaStreamSynchronize(s), "synchronize");
            if (st != CDMPT_OK) break;
            double res = 0.0;
            for (int i = 0; i < N; ++i) {
                r[i] = y[i] - x[i];
                res = std::max(res, std::fabs(r[i]));
            }
            if (res < tol) {
                conv = true;
                break;
            }
            mixer.next(x, r);
        }
    }
    h->opts = saved;
    if (st == CDMPT_OK && !conv) {
        set_error("scc_solve: the charges did not converge in " + std::to_string(maxit) +
                  " iterations");
        st = CDMPT_ERR_NO_CONVERGENCE;
    }
    // ---- coupled-perturbed SCF per direction: D1 = R(h1 + G(D1)) (linear fixed point in dq1)
    std::vector<double> om1(D, 0.0), om2(D, 0.0), m1(D, 0.0), om3(D, 0.0), m2v(D, 0.0);
    Solver<float>* sf = h->sf;
    Solver<double>* sd = h->sd;
    for (int d = 0; d < D && st == CDMPT_OK; ++d) {
        std::vector<double> x1(N, 0.0), y1(N);
        Anderson mixer(N, depth, mix);
        bool c1 = false;
        for (int it = 0; st == CDMPT_OK && it < maxit; ++it, ++cp_it) {
            cuda_ok(cudaMemcpyAsync(dq, x1.data(), N * sizeof(double), cudaMemcpyHostToDevice, s),
                    "response charges to device");
            if (st == CDMPT_OK) st = scc_gemv(gam, N, dq, N, V, s);
            if (st == CDMPT_OK) st = scc_fock(h1d + d * nn, N, Sg, ld, V, N, F1, ld, s);
            if (st == CDMPT_OK && h->ovN)
                st = congruence(h->Zov, ld, N, F1, ld, F1, ld, h->ovtmp, s);
            double mud = 0.0;
            cdmpt_stats keep = h->st;
            h->cx.st = &h->st;
            if (st == CDMPT_OK)
                st = h->opts.precision == CDMPT_FP64 ? sd->response1(h->cx, F1, 1, D1p, &mud, nullptr)
                                                     : sf->response1(h->cx, F1, 1, D1p, &mud, nullptr);
            h->st = keep;
            const double* D1c = D1p;
            if (st == CDMPT_OK && h->ovN) {
                st = ov_map(h, D1p, D1d, 1, 1);
                D1c = D1d;
            }
            if (st == CDMPT_OK) st = scc_charges(D1c, N, Sg, ld, nullptr, N, dq, s);
            cuda_ok(cudaMemcpyAsync(y1.data(), dq, N * sizeof(double), cudaMemcpyDeviceToHost, s),
                    "response charges to host");
            cuda_ok(cudaStreamSynchronize(s), "synchronize");
            if (st != CDMPT_OK) break;
            double res = 0.0;
            for (int i = 0; i < N; ++i) {
                r[i] = y1[i] - x1[i];
                res = std::max(res, std::fabs(r[i]));
            }
            m1[d] = mud;
            if (res < tol) {
                c1 = true;
                if (D1c != D1d) cuda_ok(cudaMemcpyAsync(D1d, D1c, nn * sizeof(double),
                                                        cudaMemcpyDeviceToDevice, s), "keep D1");
                break;
            }
            mixer.next(x1, r);
        }
        if (st == CDMPT_OK && !c1) {
            set_error("scc_solve: the response charges of direction " + std::to_string(d) +
                      " did not converge");
            st = CDMPT_ERR_NO_CONVERGENCE;
        }
        // Omega_SCF^(m) = (2/m) Tr[h1 D^(m-1)] (Eq. Resp_Omega): m = 1 with D0, m = 2 with D1
        if (st == CDMPT_OK) {
            cuda_ok(cudaMemsetAsync(h->dscal, 0, 2 * sizeof(double), s), "zero dots");
            if (st == CDMPT_OK) st = scc_dot(h1d + d * nn, Dd, nn, h->dscal, s);
            if (st == CDMPT_OK) st = scc_dot(h1d + d * nn, D1d, nn, h->dscal + 1, s);
            double dots[2] = {0, 0};
            cuda_ok(cudaMemcpyAsync(dots, h->dscal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s),
                    "dots to host");
            cuda_ok(cudaStreamSynchronize(s), "synchronize");
            om1[d] = 2.0 * dots[0];
            om2[d] = dots[1];
        }
        if (st == CDMPT_OK && D1) {
            const cudaMemcpyKind ko = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
            cuda_ok(cudaMemcpyAsync(D1 + d * nn, D1d, nn * sizeof(double), ko, s), "copy D1");
        }
        // second order: D2 = R2(F^(1) = h1 + G(D1), F^(2) = G(D2)), a linear fixed point in the
        // second-order charges; F1 still holds the converged F^(1) (mapped to the orthogonal
        // basis), and D1p / D1d are free again
        if (st == CDMPT_OK && second) {
            cuda_ok(cudaStreamSynchronize(s), "synchronize");
            std::vector<double> x2(N, 0.0), y2(N);
            Anderson mixer2(N, depth, mix);
            bool c2 = false;
            for (int it = 0; st == CDMPT_OK && it < maxit; ++it, ++cp_it) {
                cuda_ok(cudaMemcpyAsync(dq, x2.data(), N * sizeof(double), cudaMemcpyHostToDevice,
                                        s), "second-order charges to device");
                if (st == CDMPT_OK) st = scc_gemv(gam, N, dq, N, V, s);
                if (st == CDMPT_OK) st = scc_fock(zero, N, Sg, ld, V, N, F2, ld, s);
                if (st == CDMPT_OK && h->ovN)
                    st = congruence(h->Zov, ld, N, F2, ld, F2, ld, h->ovtmp, s);
                double m2d = 0.0;
                cdmpt_stats keep = h->st;
                h->cx.st = &h->st;
                if (st == CDMPT_OK)
                    st = h->opts.precision == CDMPT_FP64
                             ? sd->response2_at(h->cx, F1, F2, 1, &m1[d], D1p, &m2d)
                             : sf->response2_at(h->cx, F1, F2, 1, &m1[d], D1p, &m2d);
                h->st = keep;
                const double* D2c = D1p;
                if (st == CDMPT_OK && h->ovN) {
                    st = ov_map(h, D1p, D1d, 1, 1);
                    D2c = D1d;
                }
                if (st == CDMPT_OK) st = scc_charges(D2c, N, Sg, ld, nullptr, N, dq, s);
                cuda_ok(cudaMemcpyAsync(y2.data(), dq, N * sizeof(double), cudaMemcpyDeviceToHost,
                                        s), "second-order charges to host");
                cuda_ok(cudaStreamSynchronize(s), "synchronize");
                if (st != CDMPT_OK) break;
                double res = 0.0;
                for (int i = 0; i < N; ++i) {
                    r[i] = y2[i] - x2[i];
                    res = std::max(res, std::fabs(r[i]));
                }
                m2v[d] = m2d;
                if (res < tol) {
                    c2 = true;
                    if (D2c != D1d)
                        cuda_ok(cudaMemcpyAsync(D1d, D2c, nn * sizeof(double),
                                                cudaMemcpyDeviceToDevice, s), "keep D2");
                    break;
                }
                mixer2.next(x2, r);
            }
            if (st == CDMPT_OK && !c2) {
                set_error("scc_solve: the second-order charges of direction " +
                          std::to_string(d) + " did not converge");
                st = CDMPT_ERR_NO_CONVERGENCE;
            }
            if (st == CDMPT_OK) {   // Omega_SCF^(3) = (2/3) Tr[h1 D2] (Eq. Resp_Omega)
                cuda_ok(cudaMemsetAsync(h->dscal, 0, sizeof(double), s), "zero dot");
                if (st == CDMPT_OK) st = scc_dot(h1d + d * nn, D1d, nn, h->dscal, s);
                double dot3 = 0.0;
                cuda_ok(cudaMemcpyAsync(&dot3, h->dscal, sizeof(double), cudaMemcpyDeviceToHost,
                                        s), "dot to host");
                cuda_ok(cudaStreamSynchronize(s), "synchronize");
                om3[d] = 2.0 / 3.0 * dot3;
            }
            if (st == CDMPT_OK && D2) {
                const cudaMemcpyKind ko =
                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
                cuda_ok(cudaMemcpyAsync(D2 + d * nn, D1d, nn * sizeof(double), ko, s), "copy D2");
            }
        }
    }
    if (st == CDMPT_OK && D0) {
        const cudaMemcpyKind ko = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        cuda_ok(cudaMemcpyAsync(D0, Dd, nn * sizeof(double), ko, s), "copy D0");
    }
    cuda_ok(cudaStreamSynchronize(s), "synchronize");
    cudaFree(w);
    if (iters) {
        iters[0] = scf_it + 1;
        iters[1] = cp_it;
    }
    if (st != CDMPT_OK) return fail(h, st);
    if (mu) *mu = mu_last;
    for (int d = 0; d < D; ++d) {
        if (mu1) mu1[d] = m1[d];
        if (omega1) omega1[d] = om1[d];
        if (omega2) omega2[d] = om2[d];
        if (mu2) mu2[d] = m2v[d];
        if (omega3) omega3[d] = om3[d];
    }
    return CDMPT_OK;
}

cdmpt_status cdmpt_scc_solve(cdmpt_handle* h, const cdmpt_scc_model* m, int N, const double* hcore,
                             int D, const double* h1, double beta, double nocc, int n, double* D0,
                             double* D1, double* mu, double* mu1, double* omega1, double* omega2,
                             int* iters, int on_device) {
    return cdmpt_scc_solve2(h, m, N, hcore, D, h1, beta, nocc, n, D0, D1, mu, mu1, omega1, omega2,
                            nullptr, nullptr, nullptr, iters, on_device);
}

cdmpt_status cdmpt_response1(cdmpt_handle* h, int D, const double* H1, double* P1, double* mu1,
                             double* omega2, double* alpha, int on_device) {
    if (!h) return CDMPT_ERR_ARG;
    if (!h->solved)
        return fail_msg(h, CDMPT_ERR_ARG, "response1: no completed solve on this handle");
    if (D < 1 || D > 16 || !H1)
        return fail_msg(h, CDMPT_ERR_ARG, "response1: need 1 <= D <= 16 and H1");
    cudaStream_t s = h->cx.stream;
    const int N = h->N, ld = h->ld;
    const size_t nn = (size_t)N * N, blk = (size_t)N * ld;
    const bool ov = h->ovN != 0;
    // padded FP64 copy of the perturbations (and of P1 when it needs mapping or a host copy)
    const bool via = P1 && (!on_device || ov);
    double* w = nullptr;
    const size_t elems = (size_t)D * blk + (via ? (size_t)D * nn : 0);
    CDMPT_CUDA_TRY(cudaMallocAsync((void**)&w, elems * sizeof(double), s));
    double* h1p = w;
    double* pout = via ? w + (size_t)D * blk : P1;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cdmpt_status st = CDMPT_OK;
    if (cudaMemsetAsync(h1p, 0, (size_t)D * blk * sizeof(double), s) != cudaSuccess ||
        cudaMemcpy2DAsync(h1p, ld * sizeof(double), H1, N * sizeof(double), N * sizeof(double),
                          (size_t)D * N, kind, s) != cudaSuccess) {
        set_error("response1: copy of H1 failed");
        st = CDMPT_ERR_CUDA;
    }
    for (int d = 0; d < D && st == CDMPT_OK && ov; ++d)   // h1_perp = Z h1 Z
        st = congruence(h->Zov, ld, N, h1p + d * blk, ld, h1p + d * blk, ld, h->ovtmp, s);
    std::vector<double> m1(D, 0.0), om(D, 0.0);
    cdmpt_stats keep = h->st;
    h->cx.st = &h->st;
    if (st == CDMPT_OK) {
        if (h->opts.precision == CDMPT_FP64)
            st = h->sd ? h->sd->response1(h->cx, h1p, D, pout, m1.data(), om.data())
                       : CDMPT_ERR_ARG;
        else
            st = h->sf ? h->sf->response1(h->cx, h1p, D, pout, m1.data(), om.data())
                       : CDMPT_ERR_ARG;
    }
    h->st = keep;
    if (st == CDMPT_OK && P1 && ov) {
        st = ov_map(h, pout, P1, D, on_device);   // D1 = Z P1 Z
    } else if (st == CDMPT_OK && via) {
        if (cudaMemcpyAsync(P1, pout, (size_t)D * nn * sizeof(double), cudaMemcpyDeviceToHost,
                            s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            set_error("response1: copy of P1 failed");
            st = CDMPT_ERR_CUDA;
        }
    }
    cudaFreeAsync(w, s);
    cudaStreamSynchronize(s);
    if (st != CDMPT_OK) return fail(h, st);
    for (int d = 0; d < D; ++d) {
        if (mu1) mu1[d] = m1[d];
        if (omega2) omega2[d] = om[d];
        if (alpha) alpha[d] = -4.0 * om[d];   // alpha_d = -2 Tr[H1_d P1_d] = -4 Omega^(2)_d
    }
    return CDMPT_OK;
}

// Orders 2 and 3 share the marshalling: P^(m) (and the gradient) through a
// device scratch when the caller's buffers are on the host.
static cdmpt_status respond(cdmpt_handle* h, int m, const double* w, double* Pm, double* mu,
                            double* omega, double* gradH0, int on_device) {
    const char* name = m == 2 ? "response2" : "response3";
    if (!h) return CDMPT_ERR_ARG;
    if (!h->solved)
        return fail_msg(h, CDMPT_ERR_ARG, std::string(name) + ": no completed solve on this handle");
    if (h->D < 1)
        return fail_msg(h, CDMPT_ERR_ARG,
                        std::string(name) + ": the handle has no perturbation directions");
    cudaStream_t s = h->cx.stream;
    const int D = h->D;
    const size_t nn = (size_t)h->N * h->N;
    double* pm = Pm;
    double* g = gradH0;
    double* tmp = nullptr;
    const bool ov = h->ovN != 0;
    if ((!on_device || ov) && (Pm || gradH0)) {
        const size_t elems = (Pm ? (size_t)D * nn : 0) + (gradH0 ? nn : 0);
        CDMPT_CUDA_TRY(cudaMallocAsync((void**)&tmp, elems * sizeof(double), s));
        pm = Pm ? tmp : nullptr;
        g = gradH0 ? tmp + (Pm ? (size_t)D * nn : 0) : nullptr;
    }
    std::vector<double> mus(D, 0.0), om(D, 0.0);
    cdmpt_stats keep = h->st;
    h->cx.st = &h->st;
    cdmpt_status st;
    if (h->opts.precision == CDMPT_FP64) {
        if (!h->sd)
            st = CDMPT_ERR_ARG;
        else if (m == 2)
            st = h->sd->response2(h->cx, h->H1, D, w, pm, mus.data(), omega ? om.data() : nullptr, g,
                                  h->H2, h->H3);
        else
            st = h->sd->response3(h->cx, h->H1, D, pm, mus.data(), omega ? om.data() : nullptr,
                                  h->H2, h->H3);
    } else {
        if (!h->sf)
            st = CDMPT_ERR_ARG;
        else if (m == 2)
            st = h->sf->response2(h->cx, h->H1, D, w, pm, mus.data(), omega ? om.data() : nullptr, g,
                                  h->H2, h->H3);
        else
            st = h->sf->response3(h->cx, h->H1, D, pm, mus.data(), omega ? om.data() : nullptr,
                                  h->H2, h->H3);
    }
    h->st = keep;
    if (st == CDMPT_OK && ov) {   // D^(m) = Z P^(m) Z; d alpha / dF = Z (d alpha / dF_perp) Z
        if (Pm) st = ov_map(h, pm, Pm, D, on_device);
        if (st == CDMPT_OK && gradH0) st = ov_map(h, g, gradH0, 1, on_device);
    } else if (st == CDMPT_OK && !on_device) {
        if (Pm)
            CDMPT_CUDA_TRY(cudaMemcpyAsync(Pm, pm, (size_t)D * nn * sizeof(double),
                                           cudaMemcpyDeviceToHost, s));
        if (gradH0)
            CDMPT_CUDA_TRY(cudaMemcpyAsync(gradH0, g, nn * sizeof(double), cudaMemcpyDeviceToHost,
                                           s));
        CDMPT_CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (tmp) cudaFreeAsync(tmp, s);
    if (st != CDMPT_OK) return fail(h, st);
    if (mu)
        for (int d = 0; d < D; ++d) mu[d] = mus[d];
    if (omega)
        for (int d = 0; d < D; ++d) omega[d] = om[d];
    return CDMPT_OK;
}

cdmpt_status cdmpt_response2(cdmpt_handle* h, const double* w, double* P2, double* mu2,
                             double* omega3, double* gradH0, int on_device) {
    return respond(h, 2, w, P2, mu2, omega3, gradH0, on_device);
}

cdmpt_status cdmpt_response3(cdmpt_handle* h, double* P3, double* mu3, double* omega4,
                             int on_device) {
    return respond(h, 3, nullptr, P3, mu3, omega4, nullptr, on_device);
}

cdmpt_status cdmpt_polarizability(cdmpt_handle* h, double* alpha) {
    if (!h || !alpha) return CDMPT_ERR_ARG;
    if (!h->solved) return fail_msg(h, CDMPT_ERR_ARG, "polarizability: no completed solve");
    for (int d = 0; d < h->D; ++d) alpha[d] = h->alpha[d];
    return CDMPT_OK;
}

cdmpt_status cdmpt_get_stats(const cdmpt_handle* h, cdmpt_stats* st) {
    if (!h || !st) return CDMPT_ERR_ARG;
    *st = h->st;
    return CDMPT_OK;
}

const char* cdmpt_last_error(const cdmpt_handle* h) {
    if (!h) return get_error().c_str();
    return h->err.c_str();
}

void cdmpt_destroy(cdmpt_handle* h) {
    if (!h) return;
    delete h->sf;
    delete h->sd;
    for (cudaEvent_t e : h->cx.ev) cudaEventDestroy(e);
    for (cudaEvent_t e : h->cx.ph)
        if (e) cudaEventDestroy(e);
    cudaFree(h->H0);
    cudaFree(h->H1);
    cudaFree(h->H2);
    cudaFree(h->H3);
    cudaFree(h->dscal);
    cudaFree(h->Zov);
    cudaFree(h->Sov);
    cudaFree(h->ovtmp);
    if (h->cx.pinned) cudaFreeHost(h->cx.pinned);
    delete h;
}

cdmpt_status cdmpt_gemm_f32(int engine, int M, int Ncols, int K, const float* X, int ldx,
                            const float* Y, int ldy, float* D, int ldd, double alpha,
                            double beta, const float* C, int ldc, double gamma, int diag_block,
                            int trans_block, double* dot, const float* E, int lde,
                            void* stream) {
    if (M < 0 || Ncols < 0 || K < 0 || !X || !Y || !D || (beta != 0.0 && !C)) {
        set_error("gemm_f32: bad arguments");
        return CDMPT_ERR_ARG;
    }
    if (trans_block > 0 && (Ncols != trans_block || M % trans_block)) {
        set_error("gemm_f32: trans_block needs Ncols == trans_block and M a multiple of it");
        return CDMPT_ERR_ARG;
    }
    Epilogue<float> ep;
    ep.alpha = alpha;
    ep.beta = beta;
    ep.C = C;
    ep.ldc = ldc;
    ep.gamma = gamma;
    ep.diag_block = diag_block;
    ep.trans_block = trans_block > 0 ? trans_block : 0;
    ep.sym = trans_block < 0;
    ep.dot = dot;
    ep.E = E;
    ep.lde = lde;
    cudaStream_t s = (cudaStream_t)stream;
    if (engine == CDMPT_GEMM_SIMT) return gemm_simt<float>(M, Ncols, K, X, ldx, Y, ldy, D, ldd, ep,
                                                           nullptr, s);
    if (engine == CDMPT_GEMM_TC_BF16) {
        Operand<float> ox, oy;
        ox.x = X;
        oy.x = Y;
        return gemm_tc_f32(engine, M, Ncols, K, ox, ldx, oy, ldy, D, ldd, ep, nullptr, s);
    }
    if (engine != CDMPT_GEMM_AUTO && engine != CDMPT_GEMM_TC_TF32 && engine != CDMPT_GEMM_TC_3XTF32) {
        set_error("gemm_f32: unknown engine");
        return CDMPT_ERR_ARG;
    }
    if ((ldx & 3) || (ldy & 3) || (((uintptr_t)X) & 15) || (((uintptr_t)Y) & 15) || K < 1) {
        set_error("gemm_f32: tcgen05 engines need 16-byte aligned X, Y, ld a multiple of 4, K >= 1");
        return CDMPT_ERR_ARG;
    }
    // The tensor-core engines read TF32-split operands; split X and Y into
    // stream-ordered temporaries (the solver keeps splits resident instead).
    const size_t nx = (size_t)M * ldx, ny = (size_t)Ncols * ldy;
    const size_t px = (nx + 63) / 64 * 64, py = (ny + 63) / 64 * 64;
    float* tmp = nullptr;
    CDMPT_CUDA_TRY(cudaMallocAsync((void**)&tmp, (2 * px + 2 * py) * sizeof(float), s));
    Operand<float> ox, oy;
    ox.x = X;
    ox.hi = tmp;
    ox.lo = tmp + px;
    oy.x = Y;
    oy.hi = tmp + 2 * px;
    oy.lo = tmp + 2 * px + py;
    cdmpt_status st = split_tf32(X, (nx + 3) / 4 * 4, tmp, tmp + px, s);
    if (st == CDMPT_OK) st = split_tf32(Y, (ny + 3) / 4 * 4, tmp + 2 * px, tmp + 2 * px + py, s);
    if (st == CDMPT_OK)
        st = gemm_tc_f32(engine == CDMPT_GEMM_AUTO ? CDMPT_GEMM_TC_3XTF32 : engine, M, Ncols, K, ox,
                         ldx, oy, ldy, D, ldd, ep, nullptr, s);
    cudaFreeAsync(tmp, s);
    return st;
}

cdmpt_status cdmpt_split_tf32(const float* X, size_t count, float* hi, float* lo, void* stream) {
    if (!X || !hi || !lo || (count & 3)) {
        set_error("split_tf32: need X, hi, lo and count a multiple of 4");
        return CDMPT_ERR_ARG;
    }
    return split_tf32(X, count, hi, lo, (cudaStream_t)stream);
}

cdmpt_status cdmpt_gemm_f32_split(int engine, int M, int Ncols, int K, const float* Xhi,
                                  const float* Xlo, int ldx, const float* Yhi, const float* Ylo,
                                  int ldy, float* D, int ldd, double alpha, double beta,
                                  const float* C, int ldc, double gamma, int diag_block,
                                  int trans_block, double* dot, const float* E, int lde,
                                  void* stream) {
    if (M < 0 || Ncols < 0 || K < 1 || !Xhi || !Yhi || !D || (beta != 0.0 && !C) ||
        (engine != CDMPT_GEMM_TC_TF32 && (!Xlo || !Ylo))) {
        set_error("gemm_f32_split: bad arguments");
        return CDMPT_ERR_ARG;
    }
    if (engine != CDMPT_GEMM_AUTO && engine != CDMPT_GEMM_TC_TF32 && engine != CDMPT_GEMM_TC_3XTF32) {
        set_error("gemm_f32_split: engine must be AUTO, TC_TF32 or TC_3XTF32");
        return CDMPT_ERR_ARG;
    }
    if (trans_block > 0 && (Ncols != trans_block || M % trans_block)) {
        set_error("gemm_f32_split: trans_block needs Ncols == trans_block and M a multiple of it");
        return CDMPT_ERR_ARG;
    }
    Epilogue<float> ep;
    ep.alpha = alpha;
    ep.beta = beta;
    ep.C = C;
    ep.ldc = ldc;
    ep.gamma = gamma;
    ep.diag_block = diag_block;
    ep.trans_block = trans_block > 0 ? trans_block : 0;
    ep.sym = trans_block < 0;
    ep.dot = dot;
    ep.E = E;
    ep.lde = lde;
    Operand<float> ox, oy;
    ox.x = Xhi;
    ox.hi = Xhi;
    ox.lo = Xlo;
    oy.x = Yhi;
    oy.hi = Yhi;
    oy.lo = Ylo;
    return gemm_tc_f32(engine == CDMPT_GEMM_AUTO ? CDMPT_GEMM_TC_3XTF32 : engine, M, Ncols, K, ox,
                       ldx, oy, ldy, D, ldd, ep, nullptr, (cudaStream_t)stream);
}

cdmpt_status cdmpt_gemm_f64(int M, int Ncols, int K, const double* X, int ldx, const double* Y,
                            int ldy, double* D, int ldd, double alpha, double beta,
                            const double* C, int ldc, double gamma, int diag_block,
                            int trans_block, double* dot, const double* E, int lde,
                            void* stream) {
    if (M < 0 || Ncols < 0 || K < 0 || !X || !Y || !D || (beta != 0.0 && !C)) {
        set_error("gemm_f64: bad arguments");
        return CDMPT_ERR_ARG;
    }
    if (trans_block > 0 && (Ncols != trans_block || M % trans_block)) {
        set_error("gemm_f64: trans_block needs Ncols == trans_block and M a multiple of it");
        return CDMPT_ERR_ARG;
    }
    Epilogue<double> ep;
    ep.alpha = alpha;
    ep.beta = beta;
    ep.C = C;
    ep.ldc = ldc;
    ep.gamma = gamma;
    ep.diag_block = diag_block;
    ep.trans_block = trans_block > 0 ? trans_block : 0;
    ep.sym = trans_block < 0;
    ep.dot = dot;
    ep.E = E;
    ep.lde = lde;
    return gemm_simt<double>(M, Ncols, K, X, ldx, Y, ldy, D, ldd, ep, nullptr,
                             (cudaStream_t)stream);
}

cdmpt_status cdmpt_gemm_f64_tc(int M, int Ncols, int K, const double* X, int ldx,
                               const double* Y, int ldy, double* D, int ldd, double alpha,
                               double beta, const double* C, int ldc, double gamma,
                               int diag_block, int trans_block, double* dot, const double* E,
                               int lde, void* stream) {
    if (M < 0 || Ncols < 0 || K < 1 || K > 16384 || !X || !Y || !D || ldx < K || ldy < K ||
        ldd < (trans_block > 0 ? trans_block : Ncols) || (beta != 0.0 && !C)) {
        set_error("gemm_f64_tc: bad arguments (1 <= K <= 16384, ld >= K)");
        return CDMPT_ERR_ARG;
    }
    if (trans_block > 0 && (Ncols != trans_block || M % trans_block)) {
        set_error("gemm_f64_tc: trans_block needs Ncols == trans_block and M a multiple of it");
        return CDMPT_ERR_ARG;
    }
    if (M == 0 || Ncols == 0) return CDMPT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int ldq = (K + 7) / 8 * 8;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t dx = up((size_t)M * ldq * 2), dy = up((size_t)Ncols * ldq * 2);
    const size_t ex = up((size_t)M * 4), ey = up((size_t)Ncols * 4);
    char* buf = nullptr;
    if (cudaMallocAsync((void**)&buf, 7 * dx + 7 * dy + ex + ey, s) != cudaSuccess) {
        cudaGetLastError();
        set_error("gemm_f64_tc: scratch allocation failed");
        return CDMPT_ERR_OOM;
    }
    Oz64Operand ox, oy;
    for (int d = 0; d < 7; ++d) {
        ox.s[d] = buf + d * dx;
        oy.s[d] = buf + 7 * dx + d * dy;
    }
    ox.e = (int*)(buf + 7 * dx + 7 * dy);
    oy.e = (int*)(buf + 7 * dx + 7 * dy + ex);
    ox.ld = oy.ld = ldq;
    Epilogue<double> ep;
    ep.alpha = alpha;
    ep.beta = beta;
    ep.C = C;
    ep.ldc = ldc;
    ep.gamma = gamma;
    ep.diag_block = diag_block;
    ep.trans_block = trans_block > 0 ? trans_block : 0;
    ep.dot = dot;
    ep.E = E;
    ep.lde = lde;
    cdmpt_status st = oz64_slice(X, M, K, ldx, ox, nullptr, s);
    if (st == CDMPT_OK) st = oz64_slice(Y, Ncols, K, ldy, oy, nullptr, s);
    if (st == CDMPT_OK) st = gemm_oz64(M, Ncols, K, ox, oy, D, ldd, ep, nullptr, s);
    cudaFreeAsync(buf, s);
    return st;
}

}  // extern "C"

namespace {
bool pow2_or_zero(double a) {
    if (a == 0.0) return true;
    int e = 0;
    return std::frexp(std::fabs(a), &e) == 0.5;
}
}  // namespace

extern "C" cdmpt_status cdmpt_gemm_pair(int M, int Ncols, int K, const float* Xh, const float* Xl,
                                        int ldx, const float* Yh, const float* Yl, int ldy,
                                        float* D, float* Dl, int ldd, double alpha, double b1,
                                        const float* C1h, const float* C1l, double b2,
                                        const float* C2h, const float* C2l, int ldc, int sym,
                                        void* stream) {
    using namespace cdmpt;
    if (M < 0 || Ncols < 0 || K < 1 || K > 32768 || !Xh || !Yh || !D || ldx < K || ldy < K ||
        (ldx & 7) || (ldy & 7) || ldd < Ncols || ((C1h || C2h) && ldc < Ncols) ||
        !pow2_or_zero(alpha) || !pow2_or_zero(b1) || !pow2_or_zero(b2)) {
        set_error("gemm_pair: bad arguments (ld multiples of 8 and >= K, K <= 32768, alpha, b1, "
                  "b2 powers of two or zero)");
        return CDMPT_ERR_ARG;
    }
    if (M == 0 || Ncols == 0) return CDMPT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t dx = up((size_t)M * ldx * 2), dy = up((size_t)Ncols * ldy * 2);
    const size_t ex = up((size_t)M * 4), ey = up((size_t)Ncols * 4);
    char* buf = nullptr;
    const int nd = kOzDigits;
    if (cudaMallocAsync((void**)&buf, nd * dx + nd * dy + ex + ey, s) != cudaSuccess) {
        cudaGetLastError();
        set_error("gemm_pair: scratch allocation failed");
        return CDMPT_ERR_OOM;
    }
    OzOperand ox, oy;
    for (int d = 0; d < nd; ++d) {
        ox.s[d] = buf + d * dx;
        oy.s[d] = buf + nd * dx + d * dy;
    }
    ox.e = (int*)(buf + nd * dx + nd * dy);
    oy.e = (int*)(buf + nd * dx + nd * dy + ex);
    ox.ld = ldx;
    oy.ld = ldy;
    cdmpt_status st = oz_slice(Xh, Xl, M, K, ldx, ox, s);
    const bool same = Xh == Yh && Xl == Yl && M == Ncols && ldx == ldy;
    if (st == CDMPT_OK && !same) st = oz_slice(Yh, Yl, Ncols, K, ldy, oy, s);
    if (same) oy = ox;   // one set of digits for both operands (the symmetric mode needs it)
    OzEpi ep;
    ep.sym = (sym && M == Ncols && Xh == Yh && Xl == Yl) ? 1 : 0;
    ep.D = D;
    ep.Dl = Dl;
    ep.ldd = ldd;
    ep.c1h = C1h;
    ep.c1l = C1l;
    ep.c2h = C2h;
    ep.c2l = C2l;
    ep.ldc = ldc;
    ep.alpha = (float)alpha;
    ep.b1 = (float)b1;
    ep.b2 = (float)b2;
    if (st == CDMPT_OK) st = gemm_oz(M, Ncols, K, ox, oy, ep, s);
    cudaFreeAsync(buf, s);
    return st;
}

extern "C" cdmpt_status cdmpt_check_bounded_wait(double limit_ms, void* stream) {
    return cdmpt::bounded_wait_probe(limit_ms, (cudaStream_t)stream);
}
