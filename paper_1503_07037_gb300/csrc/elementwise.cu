// HBM-bound kernels of the recursion: initial deviation Z_0, the CG vector
// updates with their fused Frobenius dots, traces, symmetrisation, the
// transposed sum S + S^T of the response step, and conversions to FP64.
//
// All matrices are stored as consecutive N-row blocks with a leading
// dimension ld (a multiple of 32 elements); columns N..ld-1 hold zero and
// every kernel here maps zero padding to zero padding.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace cdmpt {

namespace {

constexpr int kThreads = 256;

int num_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 152;
    }
    return sms;
}

int grid_for(size_t work_items) {
    size_t want = (work_items + kThreads - 1) / kThreads;
    size_t cap = (size_t)num_sms() * 8;
    return (int)std::max<size_t>(1, std::min(want, cap));
}

template <typename T>
struct Vec;
template <>
struct Vec<float> {
    using type = float4;
    static constexpr int W = 4;
};
template <>
struct Vec<double> {
    using type = double2;
    static constexpr int W = 2;
};

template <typename T>
__device__ __forceinline__ void load16(const T* p, T (&v)[Vec<T>::W]) {
    typename Vec<T>::type t = *reinterpret_cast<const typename Vec<T>::type*>(p);
    const T* q = reinterpret_cast<const T*>(&t);
#pragma unroll
    for (int i = 0; i < Vec<T>::W; ++i) v[i] = q[i];
}

template <typename T>
__device__ __forceinline__ void store16(T* p, const T (&v)[Vec<T>::W]) {
    typename Vec<T>::type t;
    T* q = reinterpret_cast<T*>(&t);
#pragma unroll
    for (int i = 0; i < Vec<T>::W; ++i) q[i] = v[i];
    *reinterpret_cast<typename Vec<T>::type*>(p) = t;
}

// Block-wide sum of one double per thread; thread 0 adds the total to *out.
__device__ __forceinline__ void block_sum_atomic(double v, double* out) {
    __shared__ double part[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) part[warp] = v;
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        v = lane < nw ? part[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0 && v != 0.0) atomicAdd(out, v);
    }
}

// hi = rna_tf32(v), lo = rna_tf32(v - hi): the split operands of the 3xTF32
// tensor-core engine (both exactly representable in TF32). No-op for double.
template <typename T>
__device__ __forceinline__ void put_split(T* hi, T* lo, size_t i, T v) {
    if constexpr (sizeof(T) == 4) {
        if (hi) {
            uint32_t h, l;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
            const float hv = __uint_as_float(h);
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(v - hv));
            hi[i] = hv;
            lo[i] = __uint_as_float(l);
        }
    }
}

template <typename T>
__device__ __forceinline__ void put_split16(T* hi, T* lo, size_t i, const T (&v)[Vec<T>::W]) {
    if constexpr (sizeof(T) == 4) {
        if (hi) {
            float h[4], l[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                uint32_t a, b;
                asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(a) : "f"(v[k]));
                h[k] = __uint_as_float(a);
                asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(b) : "f"(v[k] - h[k]));
                l[k] = __uint_as_float(b);
            }
            store16(hi + i, h);
            if (lo) store16(lo + i, l);   // lo = null: the one-pass TF32 engine reads hi only
        }
    }
}

// Z[r][j] = scale * (H[r][j] - shift * [j == r mod N]) for j < N, 0 for j >= N.
template <typename T>
__global__ void k_init_z(T* __restrict__ Z, const double* __restrict__ H, int N, int ld, int ldh,
                         size_t rows, double scale, double shift, T* __restrict__ hi,
                         T* __restrict__ lo) {
    const size_t total = rows * (size_t)ld;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const size_t r = e / ld;
        const int j = (int)(e - r * ld);
        double v = 0.0;
        if (j < N) {
            v = H[r * ldh + j];
            if ((size_t)j == r % (size_t)N) v -= shift;
            v *= scale;
        }
        Z[e] = (T)v;
        put_split(hi, lo, e, (T)v);
    }
}

// alpha = <R,R>/<P,AP>;  X += alpha P;  R -= alpha Q;  sc[RRNEW] += <R,R>.
template <typename T>
__global__ void k_cg_update(T* __restrict__ X, T* __restrict__ R, const T* __restrict__ P,
                            const T* __restrict__ Q, size_t nvec, double* __restrict__ sc) {
    if (sc[CG_DONE] != 0.0) return;
    const T alpha = (T)(sc[CG_RR] / sc[CG_PQ]);
    constexpr int W = Vec<T>::W;
    double acc = 0.0;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < nvec;
         v += (size_t)gridDim.x * blockDim.x) {
        T x[W], r[W], p[W], q[W];
        load16(X + v * W, x);
        load16(R + v * W, r);
        load16(P + v * W, p);
        load16(Q + v * W, q);
        T s = 0;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            x[i] = fma(alpha, p[i], x[i]);
            r[i] = fma(-alpha, q[i], r[i]);
            s = fma(r[i], r[i], s);
        }
        acc += (double)s;
        store16(X + v * W, x);
        store16(R + v * W, r);
    }
    block_sum_atomic(acc, sc + CG_RRNEW);
}

// P = R + beta P with beta = rr_new / rr, unless converged.
template <typename T>
__global__ void k_cg_direction(T* __restrict__ P, const T* __restrict__ R, size_t nvec,
                               const double* __restrict__ sc, T* __restrict__ hi,
                               T* __restrict__ lo) {
    if (sc[CG_DONE] != 0.0) return;
    if (sc[CG_RRNEW] <= sc[CG_THRESH]) return;
    const T beta = (T)(sc[CG_RRNEW] / sc[CG_RR]);
    constexpr int W = Vec<T>::W;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < nvec;
         v += (size_t)gridDim.x * blockDim.x) {
        T p[W], r[W];
        load16(P + v * W, p);
        load16(R + v * W, r);
#pragma unroll
        for (int i = 0; i < W; ++i) p[i] = fma(beta, p[i], r[i]);
        store16(P + v * W, p);
        put_split16(hi, lo, v * W, p);
    }
}

__global__ void k_cg_scalar_step(double* sc) {
    if (sc[CG_DONE] != 0.0) return;
    sc[CG_ITERS] += 1.0;
    if (sc[CG_RRNEW] <= sc[CG_THRESH]) {
        sc[CG_DONE] = 1.0;
        sc[CG_RR] = sc[CG_RRNEW];
    } else {
        sc[CG_RR] = sc[CG_RRNEW];
        sc[CG_PQ] = 0.0;
        sc[CG_RRNEW] = 0.0;
    }
}

__global__ void k_cg_scalar_init(double* sc, double tol2, double tol2_r0, const double* ref,
                                 double tol2_ref) {
    double thresh = fmax(tol2 * sc[CG_BB], tol2_r0 * sc[CG_RR]);
    if (ref) thresh = fmax(thresh, tol2_ref * *ref);
    sc[CG_THRESH] = thresh;
    sc[CG_RR0] = sc[CG_RR];
    sc[CG_ITERS] = 0.0;
    sc[CG_PQ] = 0.0;
    sc[CG_RRNEW] = 0.0;
    sc[CG_DONE] = (sc[CG_RR] <= thresh) ? 1.0 : 0.0;
}

template <typename T>
__global__ void k_dot(const T* __restrict__ A, const T* __restrict__ B, size_t nvec,
                      double* __restrict__ out, const double* __restrict__ skip) {
    if (skip && *skip != 0.0) return;
    constexpr int W = Vec<T>::W;
    double acc = 0.0;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < nvec;
         v += (size_t)gridDim.x * blockDim.x) {
        T a[W], b[W];
        load16(A + v * W, a);
        load16(B + v * W, b);
        T s = 0;
#pragma unroll
        for (int i = 0; i < W; ++i) s = fma(a[i], b[i], s);
        acc += (double)s;
    }
    block_sum_atomic(acc, out);
}

template <typename T>
__global__ void k_axpby(T* __restrict__ Y, const T* __restrict__ X, size_t nvec, double a,
                        double b, const double* __restrict__ skip, T* __restrict__ hi,
                        T* __restrict__ lo) {
    if (skip && *skip != 0.0) return;
    constexpr int W = Vec<T>::W;
    const T ta = (T)a, tb = (T)b;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < nvec;
         v += (size_t)gridDim.x * blockDim.x) {
        T x[W], y[W];
        load16(X + v * W, x);
        if (b != 0.0) {
            load16(Y + v * W, y);
#pragma unroll
            for (int i = 0; i < W; ++i) y[i] = ta * x[i] + tb * y[i];
        } else {
#pragma unroll
            for (int i = 0; i < W; ++i) y[i] = ta * x[i];
        }
        store16(Y + v * W, y);
        put_split16(hi, lo, v * W, y);
    }
}

// out = a X + b Y (out may alias X or Y).
template <typename T>
__global__ void k_lincomb(T* __restrict__ out, const T* X, double a, const T* Y, double b,
                          size_t nvec) {
    constexpr int W = Vec<T>::W;
    const T ta = (T)a, tb = (T)b;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < nvec;
         v += (size_t)gridDim.x * blockDim.x) {
        T x[W], y[W];
        load16(X + v * W, x);
        load16(Y + v * W, y);
#pragma unroll
        for (int i = 0; i < W; ++i) x[i] = fma(ta, x[i], tb * y[i]);
        store16(out + v * W, x);
    }
}

// hi/lo split of a contiguous array (float only).
__global__ void k_split(const float* __restrict__ X, size_t nvec, float* __restrict__ hi,
                        float* __restrict__ lo) {
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < nvec;
         v += (size_t)gridDim.x * blockDim.x) {
        float x[4];
        load16(X + v * 4, x);
        put_split16<float>(hi, lo, v * 4, x);
    }
}

// BF16 copy (round to nearest even) of a contiguous array, four elements per
// thread; returns at once while *skip != 0.
__global__ void k_to_bf16(const float* __restrict__ X, size_t nvec, uint2* __restrict__ out,
                          const double* skip) {
    if (skip && *skip != 0.0) return;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < nvec;
         v += (size_t)gridDim.x * blockDim.x) {
        float x[4];
        load16(X + v * 4, x);
        uint32_t lo, hi;
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(x[1]), "f"(x[0]));
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(x[3]), "f"(x[2]));
        out[v] = make_uint2(lo, hi);
    }
}

// A[b N + i][i] += s for every block b (diagonal shift of a stack).
template <typename T>
__global__ void k_add_diag(T* __restrict__ A, int N, int ld, size_t rows, double s,
                           T* __restrict__ hi, T* __restrict__ lo) {
    for (size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x; r < rows;
         r += (size_t)gridDim.x * blockDim.x) {
        const size_t i = r * ld + (r % (size_t)N);
        const T v = A[i] + (T)s;
        A[i] = v;
        put_split(hi, lo, i, v);
    }
}

// out[b] += sum_i A[b N + i][i]
template <typename T>
__global__ void k_trace(const T* __restrict__ A, int N, int ld, double* __restrict__ out) {
    const int b = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (i < N) v = (double)A[((size_t)b * N + i) * ld + i];
    block_sum_atomic(v, out + b);
}

constexpr int TT = 32;  // transpose tile

// out_b = S_b + S_b^T for every N x N block b.
template <typename T>
__global__ void k_transpose_add(T* __restrict__ out, const T* __restrict__ S, int N, int ld,
                                T* __restrict__ hi, T* __restrict__ lo) {
    __shared__ T tile[TT][TT + 1];
    const size_t base = (size_t)blockIdx.z * N * ld;
    const int i0 = blockIdx.y * TT, j0 = blockIdx.x * TT;
    // load S[j0 + ty][i0 + tx] -> tile[ty][tx]
    for (int y = threadIdx.y; y < TT; y += blockDim.y) {
        const int r = j0 + y, c = i0 + threadIdx.x;
        tile[y][threadIdx.x] = (r < N && c < N) ? S[base + (size_t)r * ld + c] : T(0);
    }
    __syncthreads();
    for (int y = threadIdx.y; y < TT; y += blockDim.y) {
        const int r = i0 + y, c = j0 + threadIdx.x;
        if (r < N && c < N) {
            const size_t i = base + (size_t)r * ld + c;
            const T v = S[i] + tile[threadIdx.x][y];
            out[i] = v;
            put_split(hi, lo, i, v);
        }
    }
}

// out_b = in_b^T for every N x N block b (out-of-place), with optional split.
template <typename T>
__global__ void k_transpose(T* __restrict__ out, const T* __restrict__ in, int N, int ld,
                            T* __restrict__ hi, T* __restrict__ lo) {
    __shared__ T tile[TT][TT + 1];
    const size_t base = (size_t)blockIdx.z * N * ld;
    const int i0 = blockIdx.y * TT, j0 = blockIdx.x * TT;
    for (int y = threadIdx.y; y < TT; y += blockDim.y) {
        const int r = j0 + y, c = i0 + threadIdx.x;
        tile[y][threadIdx.x] = (r < N && c < N) ? in[base + (size_t)r * ld + c] : T(0);
    }
    __syncthreads();
    for (int y = threadIdx.y; y < TT; y += blockDim.y) {
        const int r = i0 + y, c = j0 + threadIdx.x;
        if (r < N && c < N) {
            const size_t i = base + (size_t)r * ld + c;
            const T v = tile[threadIdx.x][y];
            out[i] = v;
            put_split(hi, lo, i, v);
        }
    }
}

// Z_b = (Z_b + Z_b^T)/2 in place; block (bx, by) with bx < by exits, the
// other one owns the tile pair.
template <typename T>
__global__ void k_symmetrize(T* __restrict__ Z, int N, int ld, T* __restrict__ hi,
                             T* __restrict__ lo) {
    const int bi = blockIdx.y, bj = blockIdx.x;
    if (bi > bj) return;
    __shared__ T a[TT][TT + 1];
    __shared__ T b[TT][TT + 1];
    const size_t base = (size_t)blockIdx.z * N * ld;
    const int i0 = bi * TT, j0 = bj * TT;
    for (int y = threadIdx.y; y < TT; y += blockDim.y) {
        int r = i0 + y, c = j0 + threadIdx.x;
        a[y][threadIdx.x] = (r < N && c < N) ? Z[base + (size_t)r * ld + c] : T(0);
        r = j0 + y;
        c = i0 + threadIdx.x;
        b[y][threadIdx.x] = (r < N && c < N) ? Z[base + (size_t)r * ld + c] : T(0);
    }
    __syncthreads();
    // a[y][x] = Z[i0+y][j0+x], b[y][x] = Z[j0+y][i0+x]
    for (int y = threadIdx.y; y < TT; y += blockDim.y) {
        const int x = threadIdx.x;
        const T avg_ij = T(0.5) * (a[y][x] + b[x][y]);  // position (i0+y, j0+x)
        const T avg_ji = T(0.5) * (b[y][x] + a[x][y]);  // position (j0+y, i0+x)
        int r = i0 + y, c = j0 + x;
        if (r < N && c < N) {
            Z[base + (size_t)r * ld + c] = avg_ij;
            put_split(hi, lo, base + (size_t)r * ld + c, avg_ij);
        }
        if (bi != bj) {
            r = j0 + y;
            c = i0 + x;
            if (r < N && c < N) {
                Z[base + (size_t)r * ld + c] = avg_ji;
                put_split(hi, lo, base + (size_t)r * ld + c, avg_ji);
            }
        }
    }
}

template <typename T>
__global__ void k_to_f64(double* __restrict__ out, int ldo, const T* __restrict__ in, int ldi,
                         int N, size_t rows, double a, double bd) {
    const size_t total = rows * (size_t)N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const size_t r = e / N;
        const int j = (int)(e - r * N);
        double v = a * (double)in[r * ldi + j];
        if ((size_t)j == r % (size_t)N) v += bd;
        out[r * ldo + j] = v;
    }
}

// out += sum_{i,j < N} A[i][j] H[i][j]  (A in T with ld, H in FP64 with ldh)
template <typename T>
__global__ void k_dot_f64h(const T* __restrict__ A, const double* __restrict__ H, int N, int ld,
                           int ldh, double* __restrict__ out) {
    const size_t total = (size_t)N * N;
    double acc = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const size_t r = e / N;
        const int j = (int)(e - r * N);
        const double h = H[r * ldh + j];
        if (h != 0.0) acc += (double)A[r * ld + j] * h;
    }
    block_sum_atomic(acc, out);
}

// Gershgorin discs: one warp per row writes (center - radius, center + radius).
__global__ void k_gershgorin_rows(const double* __restrict__ H, int N, int ld,
                                  double* __restrict__ lohi) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= N) return;
    const double* row = H + (size_t)warp * ld;
    double rad = 0.0;
    for (int j = lane; j < N; j += 32)
        if (j != warp) rad += fabs(row[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rad += __shfl_down_sync(0xffffffffu, rad, o);
    if (lane == 0) {
        lohi[2 * (size_t)warp] = row[warp] - rad;
        lohi[2 * (size_t)warp + 1] = row[warp] + rad;
    }
}

__global__ void k_gershgorin_reduce(const double* __restrict__ lohi, int N, double* out2) {
    __shared__ double smin[32], smax[32];
    double lo = 1e300, hi = -1e300;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        lo = fmin(lo, lohi[2 * (size_t)i]);
        hi = fmax(hi, lohi[2 * (size_t)i + 1]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_down_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_down_sync(0xffffffffu, hi, o));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        smin[warp] = lo;
        smax[warp] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            lo = fmin(lo, smin[w]);
            hi = fmax(hi, smax[w]);
        }
        out2[0] = fmin(lo, smin[0]);
        out2[1] = fmax(hi, smax[0]);
    }
}

thread_local long long g_launches = 0;

// Scratch of cdmpt_spectral_bounds_noalloc: the two disc ends of every row,
// for at most kNoAllocMaxN rows (2 x 32768 doubles = 512 KiB). It lives in the
// module's static device memory, so every GPU that loads the library holds it
// until the process exits. The row pass writes entries 0 .. 2N-1 before the
// reduction reads them, so no entry has to start at zero.
constexpr int kNoAllocMaxN = 32768;
__device__ __align__(256) double g_bounds_scratch[2 * kNoAllocMaxN];

// Frobenius norms of the 128 x 32 tiles of a rows x cols FP32 matrix, one CTA of
// 128 threads per tile: each warp covers 32 rows, four rows per step with eight
// lanes (one float4 each) per 128-byte row segment, so every load is coalesced.
__global__ void k_tile_norms(const float* __restrict__ X, int rows, int cols, int ld, int nkb,
                             bool vec, float* __restrict__ out, const double* __restrict__ skip) {
    if (skip && *skip != 0.0) return;
    const int rb = blockIdx.x / nkb, kb = blockIdx.x - rb * nkb;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = kb * 32 + (lane & 7) * 4;
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int r = rb * 128 + warp * 32 + i * 4 + (lane >> 3);
        if (r >= rows) continue;
        const float* x = X + (size_t)r * ld + c;
        if (vec && c + 4 <= cols) {
            const float4 v = *reinterpret_cast<const float4*>(x);
            acc += v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w;
        } else {
            for (int j = 0; j < 4 && c + j < cols; ++j) acc += x[j] * x[j];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ float part[4];
    if (lane == 0) part[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) out[blockIdx.x] = sqrtf(part[0] + part[1] + part[2] + part[3]);
}

// Screening mask of a product from the tile norms of its operands: bit kb of word w of
// output tile (I, J) is set unless nx[I][kb] * ny[J][kb] <= tau (a NaN norm keeps the
// slice, so non-finite values propagate as in the dense product).
__global__ void k_screen_mask(const float* __restrict__ nx, const float* __restrict__ ny,
                              int mt, int nt, int nkb, int nmw, float tau,
                              uint32_t* __restrict__ mask, const double* __restrict__ skip) {
    if (skip && *skip != 0.0) return;
    const size_t total = (size_t)mt * nt * nmw;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int w = (int)(e % nmw);
        const size_t tile = e / nmw;
        const int J = (int)(tile % nt), I = (int)(tile / nt);
        const int k0 = w * 32, k1 = min(nkb, k0 + 32);
        uint32_t bits = 0u;
        for (int kb = k0; kb < k1; ++kb)
            if (!(nx[(size_t)I * nkb + kb] * ny[(size_t)J * nkb + kb] <= tau))
                bits |= 1u << (kb - k0);
        mask[e] = bits;
    }
}

}  // namespace

void count_launch(int k) { g_launches += k; }
long long launch_count() { return g_launches; }

#define LAUNCH_CHECK()                                                                   \
    do {                                                                                 \
        count_launch();                                                                  \
        cudaError_t _e = cudaGetLastError();                                             \
        if (_e != cudaSuccess) {                                                         \
            set_error(std::string("kernel launch: ") + cudaGetErrorString(_e) + " (" +   \
                      __FILE__ + ":" + std::to_string(__LINE__) + ")");                  \
            return CDMPT_ERR_CUDA;                                                       \
        }                                                                                \
    } while (0)

template <typename T>
cdmpt_status Ew<T>::init_z(T* Z, const double* H, int N, int ld, int ldh, int blocks,
                           double scale, double shift, cudaStream_t s, T* hi, T* lo) {
    const size_t rows = (size_t)blocks * N;
    k_init_z<T><<<grid_for(rows * ld), kThreads, 0, s>>>(Z, H, N, ld, ldh, rows, scale, shift, hi,
                                                          lo);
    LAUNCH_CHECK();
    return CDMPT_OK;
}

template <typename T>
cdmpt_status Ew<T>::cg_update(T* X, T* R, const T* P, const T* Q, size_t count, double* sc,
                              cudaStream_t s) {
    const size_t nvec = count / Vec<T>::W;
    k_cg_update<T><<<grid_for(nvec), kThreads, 0, s>>>(X, R, P, Q, nvec, sc);
    LAUNCH_CHECK();
    return CDMPT_OK;
}

template <typename T>
cdmpt_status Ew<T>::cg_direction(T* P, const T* R, size_t count, const double* sc,
                                 cudaStream_t s, T* hi, T* lo) {
    const size_t nvec = count / Vec<T>::W;
    k_cg_direction<T><<<grid_for(nvec), kThreads, 0, s>>>(P, R, nvec, sc, hi, lo);
    LAUNCH_CHECK();
    return CDMPT_OK;
}

template <typename T>
cdmpt_status Ew<T>::dot(const T* A, const T* B, size_t count, double* out, const double* skip,
                        cudaStream_t s) {
    const size_t nvec = count / Vec<T>::W;
    k_dot<T><<<grid_for(nvec), kThreads, 0, s>>>(A, B, nvec, out, skip);
    LAUNCH_CHECK();
    return CDMPT_OK;
}

template <typename T>
cdmpt_status Ew<T>::axpby(T* Y, const T* X, size_t count, double a, double b,
                          const double* skip, cudaStream_t s, T* hi, T* lo) {
    const size_t nvec = count / Vec<T>::W;
    k_axpby<T><<<grid_for(nvec), kThreads, 0, s>>>(Y, X, nvec, a, b, skip, hi, lo);
    LAUNCH_CHECK();
    return CDMPT_OK;
}

template <typename T>
cdmpt_status Ew<T>::trace(const T* A, int N, int ld, int blocks, double* out, cudaStream_t s) {
    dim3 grid((N + kThreads - 1) / kThreads, blocks);
    k_trace<T><<<grid, kThreads, 0, s>>>(A, N, ld, out);
    LAUNCH_CHECK();
    return CDMPT_OK;
}

template <typename T>
cdmpt_status Ew<T>::transpose_add(T* out, const T* S, int N, int ld, int blocks,
                                  cudaStream_t s, T* hi, T* lo) {
    const int nt = (N + TT - 1) / TT;
    dim3 grid(nt, nt, blocks), block(TT, 8);
    k_transpose_add<T><<<grid, block, 0, s>>>(out, S, N, ld, hi, lo);
    LAUNCH_CHECK();
    return CDMPT_OK;
}

template <typename T>
cdmpt_status Ew<T>::symmetrize(T* Z, int N, int ld, int blocks, cudaStream_t s, T* hi, T* lo) {
    const int nt = (N + TT - 1) / TT;
    dim3 grid(nt, nt, blocks), block(TT, 8);
    k_symmetrize<T><<<grid, block, 0, s>>>(Z, N, ld, hi, lo);
    LAUNCH_CHECK();
    return CDMPT_OK;
}

template <typename T>
cdmpt_status Ew<T>::to_f64(double* out, int ldo, const T* in, int ldi, int N, int rows, double a,
                           double b_diag, cudaStream_t s) {
    k_to_f64<T><<<grid_for((size_t)rows * N), kThreads, 0, s>>>(out, ldo, in, ldi, N,
                                                                 (size_t)rows, a, b_diag);
    LAUNCH_CHECK();
    return CDMPT_OK;
}

template <typename T>
cdmpt_status Ew<T>::dot_h(const T* A, const double* H, int N, int ld, int ldh, double* out,
                             cudaStream_t s) {
    k_dot_f64h<T><<<grid_for((size_t)N * N), kThreads, 0, s>>>(A, H, N, ld, ldh, out);
    LAUNCH_CHECK();
    return CDMPT_OK;
}

template <typename T>
cdmpt_status Ew<T>::transpose(T* out, const T* in, int N, int ld, int blocks, cudaStream_t s,
                              T* hi, T* lo) {
    const int nt = (N + TT - 1) / TT;
    dim3 grid(nt, nt, blocks), block(TT, 8);
    k_transpose<T><<<grid, block, 0, s>>>(out, in, N, ld, hi, lo);
    LAUNCH_CHECK();
    return CDMPT_OK;
}

template <typename T>
cdmpt_status Ew<T>::lincomb(T* out, const T* X, double a, const T* Y, double b, size_t count,
                            cudaStream_t s) {
    const size_t nvec = count / Vec<T>::W;
    k_lincomb<T><<<grid_for(nvec), kThreads, 0, s>>>(out, X, a, Y, b, nvec);
    LAUNCH_CHECK();
    return CDMPT_OK;
}

template <typename T>
cdmpt_status Ew<T>::add_diag(T* A, int N, int ld, int blocks, double shift, cudaStream_t s, T* hi,
                             T* lo) {
    const size_t rows = (size_t)blocks * N;
    k_add_diag<T><<<grid_for(rows), kThreads, 0, s>>>(A, N, ld, rows, shift, hi, lo);
    LAUNCH_CHECK();
    return CDMPT_OK;
}

cdmpt_status to_bf16(const float* x, size_t count, void* out, const double* skip,
                     cudaStream_t s) {
    const size_t nvec = count / 4;
    if (!nvec) return CDMPT_OK;
    k_to_bf16<<<grid_for(nvec), kThreads, 0, s>>>(x, nvec, (uint2*)out, skip);
    LAUNCH_CHECK();
    return CDMPT_OK;
}

cdmpt_status tile_norms(const float* X, int rows, int cols, int ld, float* out,
                        const double* skip, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return CDMPT_OK;
    const int nrb = (rows + 127) / 128, nkb = (cols + 31) / 32;
    const bool vec = (ld % 4) == 0 && (((uintptr_t)X) & 15) == 0;
    k_tile_norms<<<(unsigned)((size_t)nrb * nkb), 128, 0, s>>>(X, rows, cols, ld, nkb, vec, out,
                                                               skip);
    LAUNCH_CHECK();
    return CDMPT_OK;
}

cdmpt_status screen_mask(const float* nx, const float* ny, int M, int N, int nkb, float tau,
                         uint32_t* mask, const double* skip, cudaStream_t s) {
    const int mt = (M + 127) / 128, nt = (N + 127) / 128, nmw = (nkb + 31) / 32;
    if (mt <= 0 || nt <= 0 || nmw <= 0) return CDMPT_OK;
    k_screen_mask<<<grid_for((size_t)mt * nt * nmw), kThreads, 0, s>>>(nx, ny, mt, nt, nkb, nmw,
                                                                        tau, mask, skip);
    LAUNCH_CHECK();
    return CDMPT_OK;
}

cdmpt_status split_tf32(const float* X, size_t count, float* hi, float* lo, cudaStream_t s) {
    const size_t nvec = count / 4;
    k_split<<<grid_for(nvec), kThreads, 0, s>>>(X, nvec, hi, lo);
    LAUNCH_CHECK();
    return CDMPT_OK;
}

template struct Ew<float>;
template struct Ew<double>;

cdmpt_status cg_scalar_step(double* sc, cudaStream_t s) {
    k_cg_scalar_step<<<1, 1, 0, s>>>(sc);
    LAUNCH_CHECK();
    return CDMPT_OK;
}

cdmpt_status cg_scalar_init(double* sc, double tol2, double tol2_r0, cudaStream_t s,
                            const double* ref, double tol2_ref) {
    k_cg_scalar_init<<<1, 1, 0, s>>>(sc, tol2, tol2_r0, ref, tol2_ref);
    LAUNCH_CHECK();
    return CDMPT_OK;
}

cdmpt_status gershgorin(const double* H, int N, int ld, double* out2, cudaStream_t s) {
    double* lohi = nullptr;
    CDMPT_CUDA_TRY(cudaMallocAsync((void**)&lohi, sizeof(double) * 2 * (size_t)N, s));
    const int warps_per_block = kThreads / 32;
    k_gershgorin_rows<<<(N + warps_per_block - 1) / warps_per_block, kThreads, 0, s>>>(H, N, ld,
                                                                                        lohi);
    LAUNCH_CHECK();
    k_gershgorin_reduce<<<1, 1024, 0, s>>>(lohi, N, out2);
    LAUNCH_CHECK();
    CDMPT_CUDA_TRY(cudaFreeAsync(lohi, s));
    return CDMPT_OK;
}

// Allocation-free variant of gershgorin(): same two kernels, with the per-row
// scratch in g_bounds_scratch instead of a stream-ordered allocation.
// Host code cannot pass g_bounds_scratch itself to a kernel (on the host the
// name is a stand-in, not a device address); the device address is looked up
// with cudaGetSymbolAddress once per device, with that device current, on the
// first call made on it.
cdmpt_status gershgorin_noalloc(const double* H, int N, int ld, double* out2, cudaStream_t s) {
    if (N > kNoAllocMaxN) {
        set_error("spectral_bounds_noalloc: N = " + std::to_string(N) +
                  " exceeds the static scratch limit of " + std::to_string(kNoAllocMaxN) +
                  " rows; use cdmpt_spectral_bounds");
        return CDMPT_ERR_ARG;
    }
    static std::mutex mu;
    static double* addr[64] = {nullptr};
    int dev = 0;
    CDMPT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("spectral_bounds_noalloc: device ordinal out of range");
        return CDMPT_ERR_ARG;
    }
    double* lohi = nullptr;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!addr[dev]) {
            void* p = nullptr;
            CDMPT_CUDA_TRY(cudaGetSymbolAddress(&p, g_bounds_scratch));
            addr[dev] = (double*)p;
        }
        lohi = addr[dev];
    }
    const int warps_per_block = kThreads / 32;
    k_gershgorin_rows<<<(N + warps_per_block - 1) / warps_per_block, kThreads, 0, s>>>(H, N, ld,
                                                                                        lohi);
    LAUNCH_CHECK();
    k_gershgorin_reduce<<<1, 1024, 0, s>>>(lohi, N, out2);
    LAUNCH_CHECK();
    return CDMPT_OK;
}

}  // namespace cdmpt
