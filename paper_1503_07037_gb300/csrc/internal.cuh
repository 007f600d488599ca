// Internal declarations shared by the translation units of libcdmpt.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "cdmpt.h"

namespace cdmpt {

// Status-returning CUDA check; records the failing call in the thread's last error.
void set_error(const std::string& msg);
const std::string& get_error();

#define CDMPT_CUDA_TRY(expr)                                                            \
    do {                                                                                \
        cudaError_t _e = (expr);                                                        \
        if (_e != cudaSuccess) {                                                        \
            ::cdmpt::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e) +     \
                               " (" __FILE__ ":" + std::to_string(__LINE__) + ")");     \
            return CDMPT_ERR_CUDA;                                                      \
        }                                                                               \
    } while (0)

#define CDMPT_TRY(expr)                   \
    do {                                  \
        cdmpt_status _s = (expr);         \
        if (_s != CDMPT_OK) return _s;    \
    } while (0)

// Epilogue of every GEMM: D = alpha * X Y^T + beta * C + gamma * I_blocks, with
// optional transposed placement inside row blocks and an optional fused dot.
template <typename T>
struct Epilogue {
    double alpha = 1.0;
    double beta = 0.0;
    const T* C = nullptr;
    int ldc = 0;
    double gamma = 0.0;
    int diag_block = 0;    // identity on (m % diag_block) == n; 0 -> diag_block = M
    int trans_block = 0;   // > 0: write at the transposed position inside row blocks
    double* dot = nullptr; // accumulate sum D * E
    const T* E = nullptr;  // nullptr with dot -> E = D
    int lde = 0;
    T* Dhi = nullptr;      // optional TF32 hi/lo split of D (float only)
    T* Dlo = nullptr;
    // symmetric result (M = N, C and E symmetric, no trans_block): the tcgen05
    // engines compute only the upper-triangular tiles and mirror them; the
    // other engines ignore the flag (they compute every element)
    bool sym = false;
};

// A GEMM operand: the values and, for float storage, their TF32 split
// (hi = rna_tf32(x), lo = rna_tf32(x - hi)); hi/lo may be null when unused.
template <typename T>
struct Operand {
    const T* x = nullptr;
    const T* hi = nullptr;
    const T* lo = nullptr;
};

// Device-side CG scalars (one block of doubles per solve).
enum CgSlot {
    CG_RR = 0,      // <R, R> of the current iterate
    CG_PQ = 1,      // <P, A P>
    CG_RRNEW = 2,   // <R, R> after the update
    CG_BB = 3,      // <RHS, RHS>
    CG_DONE = 4,    // 1.0 once converged (kernels then return at once)
    CG_ITERS = 5,   // iterations taken (as double)
    CG_THRESH = 6,  // stop when <R,R> <= this (absolute)
    CG_RR0 = 7,     // <R,R> of the initial residual
    CG_NSLOTS = 8
};

// Error word written by kernels whose bounded waits give up.
enum DeviceError {
    DEV_OK = 0,
    DEV_TIMEOUT_FULL = 1,
    DEV_TIMEOUT_EMPTY = 2,
    DEV_TIMEOUT_CONV = 3,
    DEV_TIMEOUT_ACCUM = 4,
    DEV_TMEM_MISMATCH = 5,   // the two CTAs of a pair got different TMEM addresses
};

int* device_error_word();   // per-device word, zeroed at first use
cdmpt_status check_device_error(cudaStream_t s);

// GEMM launchers (asynchronous).
template <typename T>
cdmpt_status gemm_simt(int M, int N, int K, const T* X, int ldx, const T* Y, int ldy, T* D,
                       int ldd, const Epilogue<T>& ep, const double* skip, cudaStream_t s);

// Block-norm screening of one tcgen05 product X Y^T (M x N, depth K): the bit mask of
// the k-slices each 128 x 128 output tile computes (see GemmProblem), nmw words per
// tile, ceil(N / 128) tiles per tile row. counts, if not null, receives
// += [slices computed, slices examined] (two device counters).
struct GemmScreen {
    const uint32_t* mask = nullptr;
    int nmw = 0;
    unsigned long long* counts = nullptr;
};
// Tile norms for screening: out[rb * nkb + kb] = || X[128 rb .., 32 kb ..] ||_F over
// the rows x cols matrix (leading dimension ld), nkb = ceil(cols / 32). The kernel
// returns at once while *skip != 0 (skip may be null).
cdmpt_status tile_norms(const float* X, int rows, int cols, int ld, float* out,
                        const double* skip, cudaStream_t s);
// Screening mask of the product of X (M rows) and Y (N rows) from their tile norms:
// bit kb of tile (I, J) is set when nx[I][kb] * ny[J][kb] > tau. mask holds
// ceil(M / 128) * ceil(N / 128) * ceil(nkb / 32) words.
cdmpt_status screen_mask(const float* nx, const float* ny, int M, int N, int nkb, float tau,
                         uint32_t* mask, const double* skip, cudaStream_t s);

// tcgen05 engines. TF32 reads X.hi / Y.hi when given (round-to-nearest
// operands), else X.x / Y.x; 3xTF32 requires the hi and lo arrays of both.
// screen (TF32 and 3xTF32 only; null or tau = 0: dense) skips negligible k-slices.
cdmpt_status gemm_tc_f32(int engine, int M, int N, int K, const Operand<float>& X, int ldx,
                         const Operand<float>& Y, int ldy, float* D, int ldd,
                         const Epilogue<float>& ep, const double* skip, cudaStream_t s,
                         const GemmScreen* screen = nullptr);
bool tc_supported();   // device is sm_103 (tcgen05 kernels built for sm_103a)
// One CTA waits on an mbarrier that nothing arrives on, through the kernels' bounded wait
// with the given limit; returns CDMPT_ERR_TIMEOUT (and clears the error word) when it gave up.
cdmpt_status bounded_wait_probe(double limit_ms, cudaStream_t s);
// Two-SM variant (tcgen05.mma.cta_group::2, 256-row tiles per CTA pair);
// X / Y are the hi operands (TF32) and Xl / Yl the lo operands (3xTF32).
template <typename T>
struct EpiParams;
// BF16 engine: operands already rounded to BF16 (row-major, ld a multiple of 8).
cdmpt_status gemm_tc_bf16(int M, int N, int K, const void* X, int ldx, const void* Y, int ldy,
                          const EpiParams<float>& p, const double* skip, cudaStream_t s);
// out[i] = BF16(x[i]) rounded to nearest even, count a multiple of 4; skipped while *skip != 0.
cdmpt_status to_bf16(const float* x, size_t count, void* out, const double* skip,
                     cudaStream_t s);
// kch: k-blocks per TMEM accumulation chunk of the 3xTF32 engine (0 = whole K).
cdmpt_status gemm_tc_2sm(bool three, int kch, int M, int N, int K, const float* X,
                         const float* Xl, int ldx, const float* Y, const float* Yl, int ldy,
                         const EpiParams<float>& p, const double* skip, cudaStream_t s);

// Grouped tcgen05 launches (batched solves). A GemmProblem holds one problem's
// epilogue, K, tile offset, skip flag and four tensor maps in device memory.
struct GemmProblem;
int tc_tile_n(int engine);
int tc_tile_m();
// bn: tile width of the split-TF32 grouped kernel (128, or 64 for many small
// problems); 0 = the engine's default. Tensor maps of Y operands must be
// encoded with the same bn (tc_encode_operand).
cdmpt_status gemm_tc_grouped(int engine, const GemmProblem* problems, int G, int total_tiles,
                             cudaStream_t s, int bn = 0);
// bn = 256 with the split engine: the grouped wide kernel, 256 x 256 two-SM tiles (problems'
// num_mt in 256-row tiles, tensor maps with 128-row boxes for both operands; kch as in
// gemm_tc_2sm).
cdmpt_status gemm_split2sm_grouped(int kch, const GemmProblem* problems, int G,
                                   int total_tiles, cudaStream_t s);

// Elementwise / reduction launchers (T = float or double). "count" is the
// number of elements of a contiguous rows x ld block; padding columns hold 0.
template <typename T>
struct Ew {
    // Kernels that produce GEMM operands optionally also write the hi/lo TF32
    // split of their output (float only; hi = lo = nullptr skips it).
    static cdmpt_status init_z(T* Z, const double* H, int N, int ld, int ldh, int blocks,
                               double scale, double shift, cudaStream_t s, T* hi = nullptr,
                               T* lo = nullptr);
    static cdmpt_status cg_update(T* X, T* R, const T* P, const T* Q, size_t count,
                                  double* sc, cudaStream_t s);
    static cdmpt_status cg_direction(T* P, const T* R, size_t count, const double* sc,
                                     cudaStream_t s, T* hi = nullptr, T* lo = nullptr);
    static cdmpt_status dot(const T* A, const T* B, size_t count, double* out, const double* skip,
                            cudaStream_t s);
    static cdmpt_status axpby(T* Y, const T* X, size_t count, double a, double b,
                              const double* skip, cudaStream_t s, T* hi = nullptr,
                              T* lo = nullptr);
    static cdmpt_status trace(const T* A, int N, int ld, int blocks, double* out, cudaStream_t s);
    static cdmpt_status transpose_add(T* out, const T* S, int N, int ld, int blocks,
                                      cudaStream_t s, T* hi = nullptr, T* lo = nullptr);
    static cdmpt_status symmetrize(T* Z, int N, int ld, int blocks, cudaStream_t s,
                                   T* hi = nullptr, T* lo = nullptr);
    static cdmpt_status add_diag(T* A, int N, int ld, int blocks, double shift, cudaStream_t s,
                                 T* hi = nullptr, T* lo = nullptr);
    static cdmpt_status lincomb(T* out, const T* X, double a, const T* Y, double b, size_t count,
                                cudaStream_t s);
    static cdmpt_status transpose(T* out, const T* in, int N, int ld, int blocks, cudaStream_t s,
                                  T* hi = nullptr, T* lo = nullptr);
    static cdmpt_status to_f64(double* out, int ldo, const T* in, int ldi, int N, int rows,
                               double a, double b_diag, cudaStream_t s);
    static cdmpt_status dot_h(const T* A, const double* H, int N, int ld, int ldh,
                                 double* out, cudaStream_t s);
};

// Ozaki-sliced product of pair-stored matrices (gemm_oz.cu). An operand is nd = 4 or 5 BF16
// digit arrays (rows x ld, row-major) and one power-of-two exponent per row, written by
// oz_slice from a pair (xh, xl; xl may be null): x = 2^e sum_p s_p 2^(-7 - 8 p), p = 0 .. nd-1.
struct OzOperand {
    void* s[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    int* e = nullptr;
    int ld = 0;
};
// Epilogue of gemm_oz, in double-float arithmetic:
//   D (+ Dl) = alpha X Y^T + b1 (c1h + c1l) + b2 (c2h + c2l) + gamma I,
// with alpha, b1, b2 powers of two (exact scalings). D receives the FP32 rounding, Dl (if
// given) the remainder, Dthi / Dtlo (if given) the TF32 split of D, and dot (if given)
// += sum D^2. C terms and outputs share the leading dimensions ldc and ldd.
struct OzEpi {
    int M = 0, N = 0;
    float* D = nullptr;
    float* Dl = nullptr;
    float* Dthi = nullptr;
    float* Dtlo = nullptr;
    int ldd = 0;
    const float* c1h = nullptr;
    const float* c1l = nullptr;
    const float* c2h = nullptr;
    const float* c2l = nullptr;
    int ldc = 0;
    float alpha = 1.f, b1 = 0.f, b2 = 0.f, gamma = 0.f;
    double* dot = nullptr;
    const int* ex = nullptr;   // set by gemm_oz from the operands
    const int* ey = nullptr;
    // symmetric result (X is Y, M = N, the C terms symmetric): only the tiles that meet the
    // upper triangle are computed, each element n >= m written at (m, n) and (n, m)
    int sym = 0;
};
constexpr int kOzDigits = 5;   // digits of the refinement products (39 bits of the row maximum)
// digit products per k-step: the pairs (p, q) with p + q <= nd + 1, i.e. nd (nd + 1) / 2
constexpr int oz_products(int nd) { return nd * (nd + 1) / 2; }
// Settings of the mixed-precision refinement shared by the single and the batched solve
// (environment overrides read once; see solver.cu): the split-residual level at which the
// FP64-class passes start, whether they start before the occupation has settled, and the
// spectral bound above which a step's residual is FP64-class.
double refine_settle();
bool refine_early_hp();
double hp_bound();
// mu step of the occupation loops when Newton's step leaves the bracket (see solver.cu)
double next_mu_outside_newton(double lo, double hi, double e_lo, double e_hi);

// Digits of an FP64 operand for the FP64 Ozaki engine: seven BF16 digit arrays (rows x ld)
// and the rows' powers of two.
struct Oz64Operand {
    void* s[7] = {};
    int* e = nullptr;
    int ld = 0;
};
// One warp per row: digits of x (rows x cols, leading dimension ld) into out (out.ld >= cols,
// zeros in the padding). Does nothing while *skip != 0 (skip may be null).
cdmpt_status oz64_slice(const double* x, int rows, int cols, int ld, const Oz64Operand& out,
                        const double* skip, cudaStream_t s);
// D = alpha X Y^T + beta C + gamma I_blocks in FP64 from the digits of X (M x K) and Y (N x K),
// K <= 16384; full tiles (ep.sym is ignored), transposed placement and fused dot as the other
// engines. Does nothing while *skip != 0.
cdmpt_status gemm_oz64(int M, int N, int K, const Oz64Operand& X, const Oz64Operand& Y,
                       double* D, int ldd, const Epilogue<double>& ep, const double* skip,
                       cudaStream_t s);
cdmpt_status oz_slice(const float* xh, const float* xl, int rows, int cols, int ld,
                      const OzOperand& out, cudaStream_t s, int nd = kOzDigits);
// D = op(X Y^T) for X (M x K) and Y (N x K) given as nd digits each; K <= 32768.
cdmpt_status gemm_oz(int M, int N, int K, const OzOperand& X, const OzOperand& Y,
                     const OzEpi& ep, cudaStream_t s, int nd = kOzDigits);

// Pair-stored FP32 matrices (value = hi + lo, double-float arithmetic; pair.cu). thi / tlo,
// when given, receive the TF32 split of the new hi for the split-TF32 engine.
namespace pair {
// (hi, lo) = scale (H - shift I) per N x N block, rounded from FP64 to a pair
cdmpt_status init(float* hi, float* lo, const double* H, int N, int ld, int ldh, int blocks,
                  double scale, double shift, cudaStream_t s, float* thi = nullptr,
                  float* tlo = nullptr);
// out = FP32(a x + b y), x and y pairs, a and b powers of two (exact scalings) or zero
cdmpt_status lincomb(float* out, double a, const float* xh, const float* xl, double b,
                     const float* yh, const float* yl, size_t count, cudaStream_t s);
// (hi, lo) += d without rounding the sum to FP32
cdmpt_status add(float* hi, float* lo, const float* d, size_t count, cudaStream_t s,
                 float* thi = nullptr, float* tlo = nullptr);
cdmpt_status symmetrize(float* hi, float* lo, int N, int ld, int blocks, cudaStream_t s,
                        float* thi = nullptr, float* tlo = nullptr);
cdmpt_status add_diag(float* hi, float* lo, int N, int ld, int blocks, double shift,
                      cudaStream_t s, float* thi = nullptr, float* tlo = nullptr);
// out = a (hi + lo) + b_diag I in FP64
cdmpt_status to_f64(double* out, int ldo, const float* hi, const float* lo, int ldi, int N,
                    int rows, double a, double b_diag, cudaStream_t s);
}  // namespace pair

cdmpt_status split_tf32(const float* X, size_t count, float* hi, float* lo, cudaStream_t s);
cdmpt_status cg_scalar_step(double* sc, cudaStream_t s);
// threshold = max(tol2 * <B,B>, tol2_r0 * <R0,R0>)
// Starts a CG solve's scalars: stop once <R,R> <= max(tol2 <RHS,RHS>, tol2_r0 <R0,R0>,
// tol2_ref *ref) (ref: a device scalar, or null).
cdmpt_status cg_scalar_init(double* sc, double tol2, double tol2_r0, cudaStream_t s,
                            const double* ref = nullptr, double tol2_ref = 0.0);
cdmpt_status gershgorin(const double* H, int N, int ld, double* out2, cudaStream_t s);
cdmpt_status gershgorin_noalloc(const double* H, int N, int ld, double* out2, cudaStream_t s);
// Count of kernel launches issued by this thread (for statistics).
void count_launch(int k = 1);
long long launch_count();

}  // namespace cdmpt
