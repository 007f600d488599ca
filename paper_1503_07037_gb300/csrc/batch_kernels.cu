// Grouped elementwise kernels of the batched solve (FP32 storage).
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "batch_kernels.cuh"
#include "dd.cuh"
#include "internal.cuh"

namespace cdmpt {

namespace {

constexpr int kT = 256;
constexpr int TT = 32;

__device__ __forceinline__ void split1(float v, float* hi, float* lo, size_t i) {
    uint32_t h, l;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
    const float hv = __uint_as_float(h);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(v - hv));
    hi[i] = hv;
    lo[i] = __uint_as_float(l);
}

__device__ __forceinline__ void block_add(double v, double* out) {
    __shared__ double part[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) part[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < (int)(blockDim.x >> 5) ? part[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0 && v != 0.0) atomicAdd(out, v);
    }
}

template <int OP>
__global__ void k_grouped(const GrpEw* __restrict__ desc) {
    const GrpEw d = desc[blockIdx.y];
    if (d.skip && *d.skip != 0.0) return;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t first = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if constexpr (OP == G_CG_UPDATE || OP == G_CG_DIR) {
        if (d.sc[CG_DONE] != 0.0) return;
    }
    if constexpr (OP == G_CG_DIR) {
        if (d.sc[CG_RRNEW] <= d.sc[CG_THRESH]) return;
    }
    double acc = 0.0;
    if constexpr (OP == G_PAIR_INIT) {
        const size_t total = (size_t)d.rows * d.ld;
        for (size_t e = first; e < total; e += stride) {
            const size_t r = e / d.ld;
            const int j = (int)(e - r * d.ld);
            double v = 0.0;
            if (j < d.N) {
                v = d.h[r * d.ld + j];
                if ((size_t)j == r % (size_t)d.N) v -= d.s1;
                v *= d.s0;
            }
            const float h = (float)v;
            d.p0[e] = h;
            d.p1[e] = (float)(v - (double)h);
            if (d.p2) split1(h, d.p2, d.p3, e);
        }
    } else if constexpr (OP == G_PAIR_LINCOMB || OP == G_PAIR_ADD) {
        const float a0 = (float)d.s0, a1 = (float)d.s1;
        const size_t nv = (size_t)d.count / 4;
        for (size_t v = first; v < nv; v += stride) {
            const size_t i = v * 4;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float h, l;
                if constexpr (OP == G_PAIR_LINCOMB) {
                    dd::add(__fmul_rn(a0, d.p1[i + k]), __fmul_rn(a0, d.p2[i + k]),
                            __fmul_rn(a1, d.p3[i + k]), __fmul_rn(a1, d.p4[i + k]), h, l);
                    d.p0[i + k] = __fadd_rn(h, l);
                } else {
                    dd::add1(d.p0[i + k], d.p1[i + k], d.p2[i + k], h, l);
                    d.p0[i + k] = h;
                    d.p1[i + k] = l;
                    if (d.p3) split1(h, d.p3, d.p4, i + k);
                }
            }
        }
    } else if constexpr (OP == G_INIT_Z || OP == G_DOT_H) {
        const size_t total = (size_t)d.rows * d.ld;
        for (size_t e = first; e < total; e += stride) {
            const size_t r = e / d.ld;
            const int j = (int)(e - r * d.ld);
            if constexpr (OP == G_INIT_Z) {
                double v = 0.0;
                if (j < d.N) {
                    v = d.h[r * d.ld + j];
                    if ((size_t)j == r % (size_t)d.N) v -= d.s1;
                    v *= d.s0;
                }
                d.p0[e] = (float)v;
                if (d.p2) split1((float)v, d.p2, d.p3, e);
            } else {
                if (j < d.N) acc += (double)d.p0[e] * d.h[r * d.ld + j];
            }
        }
    } else {
        const float a0 = (float)d.s0, a1 = (float)d.s1;
        float alpha = 0.f, beta = 0.f;
        if constexpr (OP == G_CG_UPDATE) alpha = (float)(d.sc[CG_RR] / d.sc[CG_PQ]);
        if constexpr (OP == G_CG_DIR) beta = (float)(d.sc[CG_RRNEW] / d.sc[CG_RR]);
        const size_t nv = (size_t)d.count / 4;
        for (size_t v = first; v < nv; v += stride) {
            const size_t i = v * 4;
            if constexpr (OP == G_AXPBY) {
                float4 x = *(const float4*)(d.p1 + i);
                float4 y = a1 != 0.f ? *(const float4*)(d.p0 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
                y.x = a0 * x.x + a1 * y.x;
                y.y = a0 * x.y + a1 * y.y;
                y.z = a0 * x.z + a1 * y.z;
                y.w = a0 * x.w + a1 * y.w;
                *(float4*)(d.p0 + i) = y;
                if (d.p2) {
                    split1(y.x, d.p2, d.p3, i);
                    split1(y.y, d.p2, d.p3, i + 1);
                    split1(y.z, d.p2, d.p3, i + 2);
                    split1(y.w, d.p2, d.p3, i + 3);
                }
            } else if constexpr (OP == G_LINCOMB) {
                float4 x = *(const float4*)(d.p1 + i), y = *(const float4*)(d.p2 + i);
                x.x = a0 * x.x + a1 * y.x;
                x.y = a0 * x.y + a1 * y.y;
                x.z = a0 * x.z + a1 * y.z;
                x.w = a0 * x.w + a1 * y.w;
                *(float4*)(d.p0 + i) = x;
            } else if constexpr (OP == G_CG_UPDATE) {
                float4 x = *(float4*)(d.p0 + i), r = *(float4*)(d.p1 + i);
                const float4 p = *(const float4*)(d.p2 + i), q = *(const float4*)(d.p3 + i);
                x.x = fmaf(alpha, p.x, x.x);
                x.y = fmaf(alpha, p.y, x.y);
                x.z = fmaf(alpha, p.z, x.z);
                x.w = fmaf(alpha, p.w, x.w);
                r.x = fmaf(-alpha, q.x, r.x);
                r.y = fmaf(-alpha, q.y, r.y);
                r.z = fmaf(-alpha, q.z, r.z);
                r.w = fmaf(-alpha, q.w, r.w);
                *(float4*)(d.p0 + i) = x;
                *(float4*)(d.p1 + i) = r;
                acc += (double)(r.x * r.x + r.y * r.y + r.z * r.z + r.w * r.w);
            } else if constexpr (OP == G_CG_DIR) {
                float4 p = *(float4*)(d.p0 + i);
                const float4 r = *(const float4*)(d.p1 + i);
                p.x = fmaf(beta, p.x, r.x);
                p.y = fmaf(beta, p.y, r.y);
                p.z = fmaf(beta, p.z, r.z);
                p.w = fmaf(beta, p.w, r.w);
                *(float4*)(d.p0 + i) = p;
                if (d.p2) {
                    split1(p.x, d.p2, d.p3, i);
                    split1(p.y, d.p2, d.p3, i + 1);
                    split1(p.z, d.p2, d.p3, i + 2);
                    split1(p.w, d.p2, d.p3, i + 3);
                }
            } else if constexpr (OP == G_DOT) {
                const float4 x = *(const float4*)(d.p0 + i), y = *(const float4*)(d.p1 + i);
                acc += (double)(x.x * y.x + x.y * y.y + x.z * y.z + x.w * y.w);
            } else if constexpr (OP == G_SPLIT) {
                const float4 x = *(const float4*)(d.p0 + i);
                split1(x.x, d.p2, d.p3, i);
                split1(x.y, d.p2, d.p3, i + 1);
                split1(x.z, d.p2, d.p3, i + 2);
                split1(x.w, d.p2, d.p3, i + 3);
            } else if constexpr (OP == G_ZERO) {
                *(float4*)(d.p0 + i) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    }
    if constexpr (OP == G_CG_UPDATE) block_add(acc, d.sc + CG_RRNEW);
    if constexpr (OP == G_DOT || OP == G_DOT_H) block_add(acc, d.sc + (int)d.s0);
}

// blockIdx.z = system * max_blocks + block; tiles beyond a system's N exit
template <int OP>
__global__ void k_grouped_tiles(const GrpEw* __restrict__ desc, int max_blocks) {
    const int sys = blockIdx.z / max_blocks, blk = blockIdx.z % max_blocks;
    const GrpEw d = desc[sys];
    if (d.skip && *d.skip != 0.0) return;
    const int N = d.N, ld = d.ld;
    if (blk >= d.rows / N) return;
    const int bi = blockIdx.y, bj = blockIdx.x;
    const int i0 = bi * TT, j0 = bj * TT;
    if (i0 >= N || j0 >= N) return;
    const size_t base = (size_t)blk * N * ld;
    __shared__ float a[TT][TT + 1];
    __shared__ float b[TT][TT + 1];
    if constexpr (OP == 0) {   // symmetrise p0 in place
        if (bi > bj) return;
        for (int y = threadIdx.y; y < TT; y += blockDim.y) {
            int r = i0 + y, c = j0 + threadIdx.x;
            a[y][threadIdx.x] = (r < N && c < N) ? d.p0[base + (size_t)r * ld + c] : 0.f;
            r = j0 + y;
            c = i0 + threadIdx.x;
            b[y][threadIdx.x] = (r < N && c < N) ? d.p0[base + (size_t)r * ld + c] : 0.f;
        }
        __syncthreads();
        for (int y = threadIdx.y; y < TT; y += blockDim.y) {
            const int x = threadIdx.x;
            const float vij = 0.5f * (a[y][x] + b[x][y]);
            const float vji = 0.5f * (b[y][x] + a[x][y]);
            int r = i0 + y, c = j0 + x;
            if (r < N && c < N) {
                const size_t i = base + (size_t)r * ld + c;
                d.p0[i] = vij;
                if (d.p2) split1(vij, d.p2, d.p3, i);
            }
            if (bi != bj) {
                r = j0 + y;
                c = i0 + x;
                if (r < N && c < N) {
                    const size_t i = base + (size_t)r * ld + c;
                    d.p0[i] = vji;
                    if (d.p2) split1(vji, d.p2, d.p3, i);
                }
            }
        }
    } else if constexpr (OP == 2) {   // pair (p0, p1) symmetrised in double-float
        if (bi > bj) return;
        __shared__ float al[TT][TT + 1];
        __shared__ float bl[TT][TT + 1];
        for (int y = threadIdx.y; y < TT; y += blockDim.y) {
            int r = i0 + y, c = j0 + threadIdx.x;
            bool in = r < N && c < N;
            a[y][threadIdx.x] = in ? d.p0[base + (size_t)r * ld + c] : 0.f;
            al[y][threadIdx.x] = in ? d.p1[base + (size_t)r * ld + c] : 0.f;
            r = j0 + y;
            c = i0 + threadIdx.x;
            in = r < N && c < N;
            b[y][threadIdx.x] = in ? d.p0[base + (size_t)r * ld + c] : 0.f;
            bl[y][threadIdx.x] = in ? d.p1[base + (size_t)r * ld + c] : 0.f;
        }
        __syncthreads();
        for (int y = threadIdx.y; y < TT; y += blockDim.y) {
            const int x = threadIdx.x;
            float h1, l1, h2, l2;
            dd::add(a[y][x], al[y][x], b[x][y], bl[x][y], h1, l1);
            dd::add(b[y][x], bl[y][x], a[x][y], al[x][y], h2, l2);
            h1 *= 0.5f;
            l1 *= 0.5f;
            h2 *= 0.5f;
            l2 *= 0.5f;
            int r = i0 + y, c = j0 + x;
            if (r < N && c < N) {
                const size_t i = base + (size_t)r * ld + c;
                d.p0[i] = h1;
                d.p1[i] = l1;
                if (d.p2) split1(h1, d.p2, d.p3, i);
            }
            if (bi != bj) {
                r = j0 + y;
                c = i0 + x;
                if (r < N && c < N) {
                    const size_t i = base + (size_t)r * ld + c;
                    d.p0[i] = h2;
                    d.p1[i] = l2;
                    if (d.p2) split1(h2, d.p2, d.p3, i);
                }
            }
        }
    } else {                   // p0 = p1 + p1^T
        for (int y = threadIdx.y; y < TT; y += blockDim.y) {
            const int r = j0 + y, c = i0 + threadIdx.x;
            a[y][threadIdx.x] = (r < N && c < N) ? d.p1[base + (size_t)r * ld + c] : 0.f;
        }
        __syncthreads();
        for (int y = threadIdx.y; y < TT; y += blockDim.y) {
            const int r = i0 + y, c = j0 + threadIdx.x;
            if (r < N && c < N) {
                const size_t i = base + (size_t)r * ld + c;
                const float v = d.p1[i] + a[threadIdx.x][y];
                d.p0[i] = v;
                if (d.p2) split1(v, d.p2, d.p3, i);
            }
        }
    }
}

__global__ void k_grouped_trace(const GrpEw* __restrict__ desc, int max_blocks) {
    const int sys = blockIdx.y / max_blocks, blk = blockIdx.y % max_blocks;
    const GrpEw d = desc[sys];
    double v = 0.0;
    const bool live = !(d.skip && *d.skip != 0.0) && blk < d.rows / d.N;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (live && i < d.N) v = (double)d.p0[((size_t)blk * d.N + i) * d.ld + i];
    if (!live) return;
    block_add(v, d.sc + (int)d.s0 + blk);
}

__global__ void k_grouped_cg_init(const GrpEw* __restrict__ desc, int G) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const GrpEw d = desc[g];
    double* sc = d.sc;
    double thresh = fmax(d.s0 * sc[CG_BB], d.s1 * sc[CG_RR]);
    if (d.s2 > 0.0) thresh = fmax(thresh, d.s2 * sc[kCgRefSlot]);
    sc[CG_THRESH] = thresh;
    sc[CG_RR0] = sc[CG_RR];
    sc[CG_ITERS] = 0.0;
    sc[CG_PQ] = 0.0;
    sc[CG_RRNEW] = 0.0;
    const bool skipped = d.skip && *d.skip != 0.0;
    sc[CG_DONE] = (skipped || sc[CG_RR] <= thresh) ? 1.0 : 0.0;
}

__global__ void k_grouped_cg_step(const GrpEw* __restrict__ desc, int G) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    double* sc = desc[g].sc;
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

cdmpt_status check(const char* what) {
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string(what) + ": " + cudaGetErrorString(e));
        return CDMPT_ERR_CUDA;
    }
    return CDMPT_OK;
}

}  // namespace

cdmpt_status grouped_ew(int op, const GrpEw* dev_desc, int G, long long max_count,
                        cudaStream_t s) {
    if (G <= 0) return CDMPT_OK;
    const long long work = std::max<long long>(1, max_count / 4);
    dim3 grid((unsigned)std::min<long long>(64, (work + kT - 1) / kT), G);
    switch (op) {
        case G_AXPBY: k_grouped<G_AXPBY><<<grid, kT, 0, s>>>(dev_desc); break;
        case G_LINCOMB: k_grouped<G_LINCOMB><<<grid, kT, 0, s>>>(dev_desc); break;
        case G_CG_UPDATE: k_grouped<G_CG_UPDATE><<<grid, kT, 0, s>>>(dev_desc); break;
        case G_CG_DIR: k_grouped<G_CG_DIR><<<grid, kT, 0, s>>>(dev_desc); break;
        case G_DOT: k_grouped<G_DOT><<<grid, kT, 0, s>>>(dev_desc); break;
        case G_SPLIT: k_grouped<G_SPLIT><<<grid, kT, 0, s>>>(dev_desc); break;
        case G_ZERO: k_grouped<G_ZERO><<<grid, kT, 0, s>>>(dev_desc); break;
        case G_INIT_Z: k_grouped<G_INIT_Z><<<grid, kT, 0, s>>>(dev_desc); break;
        case G_DOT_H: k_grouped<G_DOT_H><<<grid, kT, 0, s>>>(dev_desc); break;
        case G_PAIR_INIT: k_grouped<G_PAIR_INIT><<<grid, kT, 0, s>>>(dev_desc); break;
        case G_PAIR_LINCOMB: k_grouped<G_PAIR_LINCOMB><<<grid, kT, 0, s>>>(dev_desc); break;
        case G_PAIR_ADD: k_grouped<G_PAIR_ADD><<<grid, kT, 0, s>>>(dev_desc); break;
        default: set_error("grouped_ew: unknown op"); return CDMPT_ERR_ARG;
    }
    return check("grouped elementwise launch");
}

cdmpt_status grouped_symmetrize(const GrpEw* dev_desc, int G, int max_N, int max_blocks,
                                cudaStream_t s) {
    const int nt = (max_N + TT - 1) / TT;
    dim3 grid(nt, nt, G * max_blocks), block(TT, 8);
    k_grouped_tiles<0><<<grid, block, 0, s>>>(dev_desc, max_blocks);
    return check("grouped symmetrize launch");
}

cdmpt_status grouped_transpose_add(const GrpEw* dev_desc, int G, int max_N, int max_blocks,
                                   cudaStream_t s) {
    const int nt = (max_N + TT - 1) / TT;
    dim3 grid(nt, nt, G * max_blocks), block(TT, 8);
    k_grouped_tiles<1><<<grid, block, 0, s>>>(dev_desc, max_blocks);
    return check("grouped transpose-add launch");
}

cdmpt_status grouped_pair_symmetrize(const GrpEw* dev_desc, int G, int max_N, int max_blocks,
                                     cudaStream_t s) {
    const int nt = (max_N + TT - 1) / TT;
    dim3 grid(nt, nt, G * max_blocks), block(TT, 8);
    k_grouped_tiles<2><<<grid, block, 0, s>>>(dev_desc, max_blocks);
    return check("grouped pair symmetrize launch");
}

cdmpt_status grouped_trace(const GrpEw* dev_desc, int G, int max_N, int max_blocks,
                           cudaStream_t s) {
    dim3 grid((max_N + kT - 1) / kT, G * max_blocks);
    k_grouped_trace<<<grid, kT, 0, s>>>(dev_desc, max_blocks);
    return check("grouped trace launch");
}

cdmpt_status grouped_cg_init(const GrpEw* dev_desc, int G, cudaStream_t s) {
    k_grouped_cg_init<<<(G + 127) / 128, 128, 0, s>>>(dev_desc, G);
    return check("grouped CG init launch");
}

cdmpt_status grouped_cg_step(const GrpEw* dev_desc, int G, cudaStream_t s) {
    k_grouped_cg_step<<<(G + 127) / 128, 128, 0, s>>>(dev_desc, G);
    return check("grouped CG step launch");
}

}  // namespace cdmpt
