// Device-resident solver of one canonical DMPT problem (Algorithm 1, orders
// 0 to 3) for storage type T. Host code here only sequences kernel launches
// and reads back a handful of FP64 scalars (traces, CG status).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "internal.cuh"

namespace cdmpt {

struct Context {
    cudaStream_t stream = nullptr;
    int engine = CDMPT_GEMM_AUTO;   // float storage only
    bool profile = false;
    // statistics of the running solve
    cdmpt_stats* st = nullptr;
    // event pairs for GEMM timing (profile mode)
    std::vector<cudaEvent_t> ev;
    std::vector<char> ev_ok;        // pair i timed a GEMM that did its work
    std::vector<int> ev_engine;     // engine of pair i
    std::vector<double> ev_flops;   // algorithmic flops of pair i
    size_t ev_used = 0;
    double* pinned = nullptr;       // host scalar readback (64 doubles)
    // phase boundaries of a solve (profile mode): start, after the occupation sweeps,
    // after the refinement, after the response, after dP0/dmu, end
    cudaEvent_t ph[6] = {};
    bool ph_set[6] = {};
    void mark(int i) {
        if (!profile || i < 0 || i > 5) return;
        if (!ph[i] && cudaEventCreate(&ph[i]) != cudaSuccess) {
            cudaGetLastError();
            ph[i] = nullptr;
            return;
        }
        ph_set[i] = cudaEventRecord(ph[i], stream) == cudaSuccess;
    }
};

// A rows x ld matrix (or stack of N-row blocks) and, for float storage, its
// TF32 split written by whichever kernel produced it.
template <typename T>
struct Buf {
    T* x = nullptr;
    T* hi = nullptr;
    T* lo = nullptr;
    // mixed-precision trajectory only: the low FP32 part of a pair, value = x + xl
    T* xl = nullptr;
    Operand<T> op() const {
        Operand<T> o;
        o.x = x;
        o.hi = hi;
        o.lo = lo;
        return o;
    }
};

template <typename T>
class Solver {
public:
    ~Solver();
    // (Re)allocate for N x N problems with D directions and n steps. ckpt > 0
    // keeps only every ckpt-th Z_k of the trajectory (plus Z_n and W_0); the
    // other steps are recomputed one segment at a time when they are needed.
    // pairs: the trajectory Z_0..Z_n is stored as FP32 pairs (mixed precision).
    cdmpt_status reserve(int N, int D, int n, int ckpt, bool pairs = false);
    cdmpt_status solve(Context& cx, const double* H0, const double* H1, int N, int D,
                       double gmin, double gmax, double trH0, const cdmpt_opts& o, double beta,
                       double nocc, int n, double* P0, double* P1, double* mu_out,
                       double* mu1_out, int out_on_device, double* alpha_out);

    // Vector-Jacobian product of the last solve: grad = d Tr[G0 P0] / d H0 under
    // the canonical constraint, by a reverse sweep through the stored
    // trajectory. G0 and grad are N x N FP64 device arrays (leading dimension N).
    // p0_weight != 0 adds p0_weight P0 to the gradient.
    cdmpt_status vjp_p0(Context& cx, const double* G0, double* grad, double p0_weight = 0.0);

    // Second-order canonical response of the last solve (Algorithm 1, order 2,
    // H^(2) = 0) for each of the D directions of H1 (device, D x N x ld FP64):
    // P2_d = 1/2 d^2 P / d lambda_d^2 and mu2_d with Tr P2_d = 0. Optionally
    // grad = -4 sum_d w_d P2_d = d (sum_d w_d alpha_d) / d H0 (w null: all 1).
    // P2 (D x N x N) and grad (N x N) are FP64 device arrays with leading
    // dimension N, or null; mu2 is a host array of D doubles, or null.
    // omega3 (host, D doubles, or null): Omega^(3)_d = 1/3 Tr[H1_d P2_d] (Eq. Resp_0).
    // H2, H3 (device, D x N x ld FP64, or null): higher terms of the perturbation,
    // H(lambda) = H0 + lambda H1 + lambda^2 H2 + lambda^3 H3 (Eq. H_prt); Omega^(3) is then
    // (1/3)(Tr[H1 P2] + 2 Tr[H2 P1] + 3 Tr[H3 P0]), and grad (which is d alpha / d H0 for
    // H2 = 0) is refused.
    cdmpt_status response2(Context& cx, const double* H1, int D, const double* w, double* P2,
                           double* mu2, double* omega3, double* grad,
                           const double* H2 = nullptr, const double* H3 = nullptr);

    // First-order canonical response of the last solve to other perturbations H1 (device,
    // D x N x ld FP64), on the stored trajectory: P1 (D x N x N FP64 device, leading
    // dimension N, or null), mu1 and Omega^(2) = 1/2 Tr[H1 P1] (host arrays of D, or null).
    cdmpt_status response1(Context& cx, const double* H1, int D, double* P1, double* mu1,
                           double* omega2);

    // Second-order canonical response of the last solve to a perturbation series with
    // first-order term H1 (whose canonical mu1 per direction is given in mu1s, host) and
    // second-order term H2 (both device, D x N x ld FP64): P2 (device, D x N x N, leading
    // dimension N) and mu2 (host). Used by the self-consistent layer, whose H1 is h1 + G(D1).
    cdmpt_status response2_at(Context& cx, const double* H1, const double* H2, int D,
                              const double* mu1s, double* P2, double* mu2);

    // Third-order canonical response of the last solve (Algorithm 1, the order-3
    // line, H^(2) = H^(3) = 0): P3_d = 1/6 d^3 P / d lambda_d^3 with mu3_d from
    // Tr P3_d = 0 (mu2_d from an order-2 pass first), and Omega^(4)_d =
    // 1/4 Tr[H1_d P3_d] (Eq. Resp_0). P3: D x N x N FP64 device array (leading
    // dimension N) or null; mu3, omega4: host arrays of D doubles, or null.
    cdmpt_status response3(Context& cx, const double* H1, int D, double* P3, double* mu3,
                           double* omega4, const double* H2 = nullptr,
                           const double* H3 = nullptr);

    // Free energy of the last solve, Omega = Tr[P0 H0] - T_e S[P0] (Eqs. FreeE,
    // SED; k_B = 1, T_e = 1/beta) for the recursion's own P0, evaluated without
    // eigenvalues, and optionally grad = dOmega/dH0 under the solve's constraint
    // (N x N FP64 device array, leading dimension N). omega: host double or null.
    cdmpt_status free_energy(Context& cx, double* omega, double* grad);
    bool trajectory_valid() const { return traj_valid_; }

    int ld = 0;

private:
    struct CgArgs {
        // system operator X -> s X + t X W (W symmetric): the step matrix
        // A_k = I + Z_k^2 is applied as X + X W_k so that the small part
        // W_k = Z_k^2 keeps its own FP32 precision instead of sitting next to I
        const Buf<T>* W = nullptr;
        double s = 1.0, t = 1.0;
        const Buf<T>* x0 = nullptr;     // warm start (null: zero)
        double x0_scale = 1.0;
        const T* rhs = nullptr;         // right-hand side = rhs_scale * rhs
        double rhs_scale = 1.0;
        int rows = 0;
        double tol = 1e-7;              // ||R|| <= tol ||RHS||
        double tol_r0 = 0.0;            // or ||R|| <= tol_r0 ||R_0||
        int maxit = 200;
        int init_engine = 0;            // engine of the initial residual (0: context default)
        int iter_engine = 0;            // engine of the iterations
        int hint = 1;                   // iterations expected (first chunk size)
        // or ||R|| <= tol_ref ref_scale ||ref|| (ref: rows x ld, the same shape as X; null:
        // none): an absolute tolerance on the scale of the quantity the solve updates
        const T* ref = nullptr;
        double ref_scale = 1.0;
        double tol_ref = 0.0;
        // symmetric iterates: rhs and x0 symmetric and commuting with W (every
        // 0th-order solve), so each product is computed on upper-triangular tiles
        bool sym = false;
    };
    cdmpt_status gemm(Context& cx, int M, int Nc, int K, const Operand<T>& X,
                      const Operand<T>& Y, T* D, const Epilogue<T>& ep, const double* skip,
                      int engine_override = 0);
    cdmpt_status cg(Context& cx, T* X, const CgArgs& a, int* iters_out, double* rel_res0,
                    bool* met_tol = nullptr);
    cdmpt_status sweep(Context& cx, const double* H0, double mu, double s2, const cdmpt_opts& o,
                       int n, int engine, double tol, int* cg_iters);
    // One 0th-order step: W_k = Z_k^2 (unless make_w is false) and, if solve,
    // Z_{k+1} from the step's linear system. *hint carries the CG chunk size.
    cdmpt_status step0(Context& cx, int k, int engine, double tol, int maxit, bool make_w,
                       bool solve, int* hint, int* iters);
    // Z_0 at chemical potential mu: -s2 (H0 - mu I), or with fd_exact tanh of it (odd
    // Taylor series in Y, |Y| <= rho); and the matching first-order start for D stacked
    // directions of H1 (into out, with its TF32 split).
    cdmpt_status init_z0(Context& cx, const double* H0, double mu, double s2, double rho,
                         int engine);
    cdmpt_status init_z1(Context& cx, const double* H1, int D, T* out, T* out_hi, T* out_lo);
    // out_d = Dtanh(Y)[E_d] for D stacked directions E_d held in Z1b_ (Fermi-Dirac-exact
    // start; the map is self-adjoint, so it also serves the reverse sweep).
    cdmpt_status tanh_tangent(Context& cx, int D, T* out, T* out_hi, T* out_lo);
    // Taylor coefficients Z^(q)_0, q = 1..m (m <= 3), of tanh(Y + sum_q lambda^q Y^(q)) for
    // the Fermi-Dirac-exact start, with the Y^(q) held in zo_[q-1][1]; written to zo_[q-1][0].
    cdmpt_status tanh_taylor(Context& cx, int m);
    double fdx_eps() const;
    // Make Z_k, W_k and Z_{k+1} of step k valid (checkpointing: recompute the
    // segment of step k from its checkpoint unless the segment buffers hold it).
    cdmpt_status need(Context& cx, int k);
    // Joint forward sweep of the orders 1..m (m <= 3) for one direction H1d, with
    // mu^(1..m-1) = mus[0..m-2] known and mu^(m) = 0. Leaves Z^(o)_n in
    // zo_[o-1][cur_[o-1]].
    cdmpt_status orders(Context& cx, const double* H1d, const double* H2d, const double* H3d,
                        int m, const double* mus);
    cdmpt_status reserve_orders();
    // Tr ln(a I + b M) for symmetric M whose spectrum puts a I + b M inside
    // [lo, hi] (0 < lo <= hi), by the Cayley transform Y = (A - cI)(A + cI)^-1,
    // c = sqrt(lo hi), one CG solve and the odd series of 2 Tr atanh(Y),
    // truncated where the remainder falls below eps per level. Uses zo_ buffers.
    cdmpt_status logdet(Context& cx, const Buf<T>& M, double a, double b, double lo, double hi,
                        double eps, double* out);
    // Canonical response of order m (2 or 3) for every direction: P^(m), mu^(m),
    // Omega^(m+1), and for m = 2 the weighted polarizability gradient.
    cdmpt_status higher(Context& cx, const double* H1, int D, int m, const double* w,
                        double* Pm, double* mu_out, double* omega, double* grad,
                        const double* H2 = nullptr, const double* H3 = nullptr,
                        const double* mu1s = nullptr);
    // One refinement pass; steps k >= k_hp form their residuals with Ozaki-sliced products.
    cdmpt_status refine(Context& cx, const cdmpt_opts& o, int n, int k_hp, int* cg_iters,
                        double* max_rel_res);
    // W_k and the residual of step k (into RHS_) from Ozaki-sliced products of the
    // pair-stored trajectory (FP64-class residuals).
    cdmpt_status residual_hp(Context& cx, int k);
    // D = op(X Y^T) by gemm_oz, with the profile events and statistics of gemm()
    cdmpt_status gemm_hp(Context& cx, const OzOperand& X, const OzOperand& Y, const OzEpi& ep);
    // Z_k += d, symmetrised (pair storage: without rounding the sum to FP32)
    cdmpt_status correct(Context& cx, int k, const T* d);
    // Z_0 += shift I
    cdmpt_status shift_z0(Context& cx, double shift);
    // P0 = (I + Z_n)/2 of the last solve in FP64 (device, leading dimension ldo)
    cdmpt_status p0_out(Context& cx, double* out, int ldo);
    cdmpt_status occupation(Context& cx, int n, double* trP, double* zz);
    cdmpt_status compute_q(Context& cx);
    cdmpt_status read_scalars(Context& cx, const double* dev, int count);
    int engine_of(const Context& cx, int override_engine) const;

    int N_ = 0, D_ = 0, n_ = 0;
    size_t blk_ = 0;                 // N * ld elements
    // trajectory views Z_0..Z_n and W_k = Z_k^2 (k < n). Without checkpointing
    // each view has its own storage. With stride ck_ the views of Z at
    // multiples of ck_ and of Z_n own storage (checkpoints), W_0 owns storage,
    // and the interior views of every segment [j ck_, (j+1) ck_) alias the same
    // ck_ - 1 Z and ck_ W segment buffers; seg_ is the segment they hold.
    std::vector<Buf<T>> Z_, W_;
    int ck_ = 0, seg_ = -1;
    bool pairs_ = false;             // Z_k.xl allocated (mixed precision)
    OzOperand oz_[3];                // digit operands of the Ozaki-sliced products (pairs_)
    T* wl_ = nullptr;                // low part of the Ozaki-formed W_k (pairs_)
    // FP64 storage on the tensor cores: digits of a product's left (up to D N rows) and
    // right (N rows) operand, allocated at the first product of that engine
    Oz64Operand ox64_, oy64_;
    bool oz64_ready_ = false;
    cdmpt_status oz64_prepare();
    int replay_iters_ = 0;           // CG iterations spent recomputing segments
    Buf<T> R_, P_, Q_;               // CG work (D' * N rows)
    Buf<T> S_, A1_, RHS_;            // response work
    Buf<T> Z1a_, Z1b_;               // response iterates
    Buf<T> Qmu_;                     // dP/dmu
    Buf<T> Zh_;                      // adjoint of Z_k in the reverse sweep
    // orders 1..3 of the joint forward sweep: iterates Z^(o)_k, Z^(o)_{k+1}
    // (zo_[o-1][cur_[o-1]] is the current one), A^(o)_k = sum_{i+j=o} Z^(i)_k
    // Z^(j)_k, and the gradient accumulator
    Buf<T> zo_[3][2], ao_[3], G_;
    // Fermi-Dirac-exact start: Y = -s2 (H0 - mu I) at the trajectory's mu and U = Y^2
    Buf<T> Yfd_, Ufd_;
    // block-norm screening (opts.screen_tau, FP32 storage): tile-norm tables of the two
    // operands of the current product, and the [computed, examined] slice counters
    float* tnx_ = nullptr;
    float* tny_ = nullptr;
    uint32_t* tmask_ = nullptr;   // slice mask of the current product
    float* tnw_ = nullptr;        // norms of the fixed right factor of the running CG solve
    const float* wnorm_src_ = nullptr;   // that factor's data while tnw_ holds its norms
    unsigned long long* tcnt_ = nullptr;
    float screen_tau_ = 0.f;
    int cur_[3] = {0, 0, 0};
    bool orders_ready_ = false;
    std::vector<double> last_mu1_;
    // state of the last solve, for the response's Q and the adjoint
    bool traj_valid_ = false, q_valid_ = false;
    double last_beta_ = 0, last_s2_ = 0;
    double last_mu_ = 0, last_rho_ = 0;   // mu and max |z0| over the Gershgorin interval
    bool fdx_ = false;                    // Fermi-Dirac-exact start of the current solve
    double gmin_ = 0, gmax_ = 0;          // Gershgorin interval of H0
    int acc_cur_ = 0;                     // FP32-accurate engine of the current solve
    int last_n_ = 0, last_acc_ = 0;
    double last_sweep_tol_ = 0;
    cdmpt_opts last_opts_{};
    double* sc_ = nullptr;           // device scalars
    std::vector<void*> allocs_;
    int rows_cap_ = 0;               // row capacity of the CG work buffers
};

}  // namespace cdmpt
