// Non-orthogonal basis (Sec. IV, Eq. Fermi_D): D = Z [exp(beta (F_perp - mu I)) + I]^-1 Z^T
// with F_perp = Z^T F Z and Z^T S Z = I. Z is the Loewdin factor S^(-1/2) (symmetric, so
// Z^T = Z), found by the coupled Newton-Schulz iteration, which needs only products:
//   Y_0 = S / c, Z_0 = I, T_k = (3 I - Z_k Y_k) / 2, Y_{k+1} = Y_k T_k, Z_{k+1} = T_k Z_k,
// with Y_k -> (S/c)^(1/2) and Z_k -> (S/c)^(-1/2) while ||I - S/c|| < 1; c is the
// Gershgorin upper bound of S, so the spectrum of S / c lies in (0, 1]. Everything runs in
// FP64 on the CUDA-core product kernel (a set-up step, once per overlap).
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <utility>

#include "internal.cuh"
#include "overlap.cuh"

namespace cdmpt {

cdmpt_status lowdin_factor(const double* S, int N, int ld, double c, double* Z, double* work,
                           double* dscal, int maxit, double tol, int* iters, double* resid,
                           cudaStream_t s) {
    const size_t blk = (size_t)N * ld;
    double* Y = work;
    double* Zc = work + blk;
    double* E = work + 2 * blk;
    double* Yn = work + 3 * blk;
    double* Zn = Z;   // the output buffer doubles as the fourth iterate
    CDMPT_TRY(Ew<double>::axpby(Y, S, blk, 1.0 / c, 0.0, nullptr, s));
    CDMPT_CUDA_TRY(cudaMemsetAsync(Zc, 0, blk * sizeof(double), s));
    CDMPT_TRY(Ew<double>::add_diag(Zc, N, ld, 1, 1.0, s));
    double res = 1.0;
    int it = 0;
    bool polish = false;   // one more step after the tolerance is met (quadratic convergence)
    for (; it < maxit; ++it) {
        // E = Z_k Y_k - I (both symmetric), and ||E||_F^2
        CDMPT_CUDA_TRY(cudaMemsetAsync(dscal, 0, sizeof(double), s));
        Epilogue<double> ep;
        ep.gamma = -1.0;
        ep.dot = dscal;
        CDMPT_TRY(gemm_simt<double>(N, N, N, Zc, ld, Y, ld, E, ld, ep, nullptr, s));
        double rr = 0.0;
        CDMPT_CUDA_TRY(cudaMemcpyAsync(&rr, dscal, sizeof(double), cudaMemcpyDeviceToHost, s));
        CDMPT_CUDA_TRY(cudaStreamSynchronize(s));
        res = std::sqrt(rr / N);
        if (!(res == res)) break;   // NaN: report below
        if (res < tol) {
            if (polish) break;
            polish = true;
        }
        // T = I - E / 2 = (3 I - Z Y) / 2, in E
        CDMPT_TRY(Ew<double>::lincomb(E, E, -0.5, E, 0.0, blk, s));
        CDMPT_TRY(Ew<double>::add_diag(E, N, ld, 1, 1.0, s));
        Epilogue<double> e2;
        CDMPT_TRY(gemm_simt<double>(N, N, N, Y, ld, E, ld, Yn, ld, e2, nullptr, s));   // Y T
        CDMPT_TRY(gemm_simt<double>(N, N, N, E, ld, Zc, ld, Zn, ld, e2, nullptr, s));  // T Z
        CDMPT_TRY(Ew<double>::symmetrize(Yn, N, ld, 1, s));
        CDMPT_TRY(Ew<double>::symmetrize(Zn, N, ld, 1, s));
        std::swap(Y, Yn);
        std::swap(Zc, Zn);
    }
    *iters = it;
    *resid = res;
    if (!(res < tol)) {
        set_error("overlap: Newton-Schulz for S^(-1/2) did not converge (||Z S Z / c - I||_F / "
                  "sqrt(N) = " + std::to_string(res) + " after " + std::to_string(it) +
                  " iterations); is S symmetric positive definite?");
        return CDMPT_ERR_NO_CONVERGENCE;
    }
    // Z = Z_k / sqrt(c), written to the output buffer
    CDMPT_TRY(Ew<double>::axpby(Z, Zc, blk, 1.0 / std::sqrt(c), 0.0, nullptr, s));
    return check_device_error(s);
}

cdmpt_status congruence(const double* Z, int ldz, int N, const double* X, int ldx, double* out,
                        int ldo, double* tmp, cudaStream_t s) {
    Epilogue<double> ep;
    CDMPT_TRY(gemm_simt<double>(N, N, N, Z, ldz, X, ldx, tmp, ldz, ep, nullptr, s));   // Z X
    CDMPT_TRY(gemm_simt<double>(N, N, N, tmp, ldz, Z, ldz, out, ldo, ep, nullptr, s)); // Z X Z
    return CDMPT_OK;
}

}  // namespace cdmpt
