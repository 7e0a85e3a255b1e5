// Plain FP32 form of the two DFT products (FFMA on the CUDA cores).
//
// Forward (Eq. 1 in separable form):
//   Z_c = A_x B_c with B_c = S_c . X         ([nk x nx] x [nx x ny])
//   y_c[k] = sum_j Z_c[k][j] A_y[k][j]        (row-sum of the Hadamard product)
// One block owns 64 samples of one coil and sweeps all j, so the row-sum
// completes inside the block.
//
// Adjoint:
//   W_c = A_x^H diag(y_c) conj(A_y)            ([nx x nk] x [nk x ny])
// split over `ksplit` contiguous ranges of samples; each range writes a
// partial image to part[c][j][ig][p][64] (the layout of the tensor-core
// adjoint, pixel i = 64 ig + (i % 64)) and launch_adj_reduce sums the partials
// in a fixed order and applies conj(S_c) (the paper's cross-core sum of
// partial images, done on chip).
//
// Both products accumulate in two levels: each 16-term stage of the K loop
// is summed into a fresh register block, which is then added to the running
// sum.  A single sequential FP32 sum over a k-space split (hundreds of
// samples, dominated by the large central ones of a radial trajectory)
// carries enough rounding to move the N=32 reconstruction by ~3e-3 NRMSE
// from the FP64 solver; with 16-sample blocks an emulation of the same
// arithmetic lands ~8e-5 from it, for one extra add per 16 FMAs.
#include "common.cuh"
#include "internal.h"

namespace mri {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;  // tile of the FP32 products, 256 threads, 4x4 per thread

// B_c[i][j] = S_c[i][j] * x[i][j]
__global__ void coil_product_kernel(const float2 *__restrict__ x, const float2 *__restrict__ maps,
                                    float2 *__restrict__ out, int npix, int nc,
                                    const DevScalars *sc, int skip) {
    if (should_skip(sc, skip)) return;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= npix) return;
    const float2 v = x[n];
    for (int c = 0; c < nc; ++c) out[(size_t)c * npix + n] = cmul(maps[(size_t)c * npix + n], v);
}

__global__ void __launch_bounds__(256) fwd_fp32_kernel(const float2 *__restrict__ ax, const float2 *__restrict__ ay,
                                                       const float2 *__restrict__ bsx, float2 *__restrict__ y,
                                                       int y_ld, int nx, int ny, int nk, int b_transposed,
                                                       const DevScalars *sc, int skip) {
    if (should_skip(sc, skip)) return;
    __shared__ __align__(16) float2 As[2][BK][BM];  // As[k][m] = A_x[k0+m][i0+k]
    __shared__ __align__(16) float2 Bs[2][BK][BN];  // Bs[k][n] = B_c[i0+k][j0+n]
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int c = blockIdx.y;
    const int k0 = blockIdx.x * BM;
    const float2 *B = bsx + (size_t)c * nx * ny;

    float2 yacc[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) yacc[m] = make_float2(0.f, 0.f);

    for (int j0 = 0; j0 < ny; j0 += BN) {
        float2 acc[4][4];
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[m][q] = make_float2(0.f, 0.f);

        // staging: A tile 64 rows x 16 cols, each thread 4 consecutive i of one row
        const int a_row = tid >> 2, a_col = (tid & 3) * 4;
        // B tile 16 rows (i) x 64 cols (j), each thread 4 elements contiguous
        // in memory: 4 consecutive j of one i (image layout [i][j]) or 4
        // consecutive i of one j (the solver's transposed layout [j][i])
        const int b_row = b_transposed ? (tid & 3) * 4 : tid >> 4;
        const int b_col = b_transposed ? tid >> 2 : (tid & 15) * 4;
        float2 ra[4], rb[4];
        auto load = [&](int i0) {
            const int kk = k0 + a_row, ii0 = i0 + a_col;
            if (kk < nk && ii0 + 3 < nx && (nx & 1) == 0) {  // two aligned 16-byte loads
                const float4 *src = reinterpret_cast<const float4 *>(ax + (size_t)kk * nx + ii0);
                const float4 u = src[0], v = src[1];
                ra[0] = make_float2(u.x, u.y);
                ra[1] = make_float2(u.z, u.w);
                ra[2] = make_float2(v.x, v.y);
                ra[3] = make_float2(v.z, v.w);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    ra[q] = (kk < nk && ii0 + q < nx) ? ax[(size_t)kk * nx + ii0 + q] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int bi = i0 + b_row + (b_transposed ? q : 0), bj = j0 + b_col + (b_transposed ? 0 : q);
                rb[q] = (bi < nx && bj < ny) ? B[b_transposed ? (size_t)bj * nx + bi : (size_t)bi * ny + bj]
                                             : make_float2(0.f, 0.f);
            }
        };
        auto store = [&](int buf) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                As[buf][a_col + q][a_row] = ra[q];
                if (b_transposed)
                    Bs[buf][b_row + q][b_col] = rb[q];
                else
                    Bs[buf][b_row][b_col + q] = rb[q];
            }
        };
        load(0);
        store(0);
        __syncthreads();
        int buf = 0;
        for (int i0 = 0; i0 < nx; i0 += BK) {
            const bool more = i0 + BK < nx;
            if (more) load(i0 + BK);
            float2 blk[4][4];  // this stage's 16 terms, added to acc below
#pragma unroll
            for (int m = 0; m < 4; ++m)
#pragma unroll
                for (int q = 0; q < 4; ++q) blk[m][q] = make_float2(0.f, 0.f);
#pragma unroll
            for (int kq = 0; kq < BK; ++kq) {
                const float4 a01 = *reinterpret_cast<const float4 *>(&As[buf][kq][ty * 4]);
                const float4 a23 = *reinterpret_cast<const float4 *>(&As[buf][kq][ty * 4 + 2]);
                const float4 b01 = *reinterpret_cast<const float4 *>(&Bs[buf][kq][tx * 4]);
                const float4 b23 = *reinterpret_cast<const float4 *>(&Bs[buf][kq][tx * 4 + 2]);
                const float2 a[4] = {make_float2(a01.x, a01.y), make_float2(a01.z, a01.w),
                                     make_float2(a23.x, a23.y), make_float2(a23.z, a23.w)};
                const float2 b[4] = {make_float2(b01.x, b01.y), make_float2(b01.z, b01.w),
                                     make_float2(b23.x, b23.y), make_float2(b23.z, b23.w)};
#pragma unroll
                for (int m = 0; m < 4; ++m)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        blk[m][q].x = fmaf(a[m].x, b[q].x, blk[m][q].x);
                        blk[m][q].x = fmaf(-a[m].y, b[q].y, blk[m][q].x);
                        blk[m][q].y = fmaf(a[m].x, b[q].y, blk[m][q].y);
                        blk[m][q].y = fmaf(a[m].y, b[q].x, blk[m][q].y);
                    }
            }
#pragma unroll
            for (int m = 0; m < 4; ++m)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[m][q] = cadd(acc[m][q], blk[m][q]);
            if (more) {
                store(buf ^ 1);
                __syncthreads();
                buf ^= 1;
            }
        }
        // epilogue: row-sum of Z .* A_y over this j tile
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int kk = k0 + ty * 4 + m;
            if (kk >= nk) continue;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int jj = j0 + tx * 4 + q;
                if (jj < ny) yacc[m] = cadd(yacc[m], cmul(acc[m][q], ay[(size_t)kk * ny + jj]));
            }
        }
        __syncthreads();
    }
    // reduce over the 16 threads (tx) that share ty: consecutive lanes
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        float re = yacc[m].x, im = yacc[m].y;
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
        }
        const int kk = k0 + ty * 4 + m;
        if (tx == 0 && kk < nk) y[(size_t)c * y_ld + kk] = make_float2(re, im);
    }
}

// part[c][j][i / 64][p][i % 64] = sum_{k in split p} conj(A_x[k][i]) y_c[k] conj(A_y[k][j])
__global__ void __launch_bounds__(256) adj_fp32_kernel(const float2 *__restrict__ ax, const float2 *__restrict__ ay,
                                                       const float2 *__restrict__ y, float2 *__restrict__ part,
                                                       int y_ld, int nx, int ny, int nk, int nc, int nx_pad,
                                                       int ksplit, int samples_per_split, const DevScalars *sc,
                                                       int skip) {
    if (should_skip(sc, skip)) return;
    __shared__ __align__(16) float2 Us[2][BK][BM];  // Us[k][m] = conj(A_x[k][i0+m]) y_c[k]
    __shared__ __align__(16) float2 Vs[2][BK][BN];  // Vs[k][n] = conj(A_y[k][j0+n])
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int tiles_i = (nx + BM - 1) / BM;
    const int i0 = (blockIdx.x % tiles_i) * BM, j0 = (blockIdx.x / tiles_i) * BN;
    const int c = blockIdx.y, p = blockIdx.z;
    const int kbeg = p * samples_per_split;
    const int kend = min(nk, kbeg + samples_per_split);
    const float2 *yc = y + (size_t)c * y_ld;

    float2 acc[4][4];
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[m][q] = make_float2(0.f, 0.f);

    // staging: 16 rows (samples) x 64 cols, each thread 4 consecutive columns of one row
    const int s_row = tid >> 4, s_col = (tid & 15) * 4;
    float2 ru[4], rv[4];
    auto load = [&](int kb) {
        const int kk = kb + s_row;
        const bool ok = kk < kend;
        const float2 yk = ok ? yc[kk] : make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int ii = i0 + s_col + q, jj = j0 + s_col + q;
            ru[q] = (ok && ii < nx) ? cmulc(ax[(size_t)kk * nx + ii], yk) : make_float2(0.f, 0.f);
            rv[q] = (ok && jj < ny) ? cconj(ay[(size_t)kk * ny + jj]) : make_float2(0.f, 0.f);
        }
    };
    auto store = [&](int buf) {
        *reinterpret_cast<float4 *>(&Us[buf][s_row][s_col]) = make_float4(ru[0].x, ru[0].y, ru[1].x, ru[1].y);
        *reinterpret_cast<float4 *>(&Us[buf][s_row][s_col + 2]) = make_float4(ru[2].x, ru[2].y, ru[3].x, ru[3].y);
        *reinterpret_cast<float4 *>(&Vs[buf][s_row][s_col]) = make_float4(rv[0].x, rv[0].y, rv[1].x, rv[1].y);
        *reinterpret_cast<float4 *>(&Vs[buf][s_row][s_col + 2]) = make_float4(rv[2].x, rv[2].y, rv[3].x, rv[3].y);
    };
    if (kbeg < kend) {
        load(kbeg);
        store(0);
    }
    __syncthreads();
    int buf = 0;
    for (int kb = kbeg; kb < kend; kb += BK) {
        const bool more = kb + BK < kend;
        if (more) load(kb + BK);
        float2 blk[4][4];  // this stage's 16 samples, added to acc below
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
            for (int q = 0; q < 4; ++q) blk[m][q] = make_float2(0.f, 0.f);
#pragma unroll
        for (int kq = 0; kq < BK; ++kq) {
            const float4 u01 = *reinterpret_cast<const float4 *>(&Us[buf][kq][ty * 4]);
            const float4 u23 = *reinterpret_cast<const float4 *>(&Us[buf][kq][ty * 4 + 2]);
            const float4 v01 = *reinterpret_cast<const float4 *>(&Vs[buf][kq][tx * 4]);
            const float4 v23 = *reinterpret_cast<const float4 *>(&Vs[buf][kq][tx * 4 + 2]);
            const float2 u[4] = {make_float2(u01.x, u01.y), make_float2(u01.z, u01.w),
                                 make_float2(u23.x, u23.y), make_float2(u23.z, u23.w)};
            const float2 v[4] = {make_float2(v01.x, v01.y), make_float2(v01.z, v01.w),
                                 make_float2(v23.x, v23.y), make_float2(v23.z, v23.w)};
#pragma unroll
            for (int m = 0; m < 4; ++m)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    blk[m][q].x = fmaf(u[m].x, v[q].x, blk[m][q].x);
                    blk[m][q].x = fmaf(-u[m].y, v[q].y, blk[m][q].x);
                    blk[m][q].y = fmaf(u[m].x, v[q].y, blk[m][q].y);
                    blk[m][q].y = fmaf(u[m].y, v[q].x, blk[m][q].y);
                }
        }
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[m][q] = cadd(acc[m][q], blk[m][q]);
        if (more) {
            store(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }
    // write the partial image: the tile's 64 rows i are one 64-pixel group
    const size_t js = (size_t)(nx_pad / 64) * ksplit * 64;
    float2 *dst = part + (size_t)c * ny * js + (size_t)(i0 >> 6) * ksplit * 64 + (size_t)p * 64;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int jj = j0 + tx * 4 + q;
        if (jj >= ny) continue;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int ii = i0 + ty * 4 + m;
            if (ii < nx) dst[(size_t)jj * js + (ii & 63)] = acc[m][q];
        }
    }
}

}  // namespace

// Blocks of the FP32 adjoint that the GPU holds at once (occupancy x SMs).
int adj_fp32_slots(int num_sms) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adj_fp32_kernel, 256, 0) != cudaSuccess ||
        per_sm <= 0) {
        cudaGetLastError();
        per_sm = 1;
    }
    return per_sm * num_sms;
}

cudaError_t launch_fwd_fp32(mri_plan *p, const float2 *image, const float2 *maps, float2 *kspace, int ld,
                            int skip, cudaStream_t s) {
    const int npix = p->nx * p->ny;
    if (image) {  // else the solver has written S_c . v to bsx, transposed
        coil_product_kernel<<<ceil_div(npix, 256), 256, 0, s>>>(image, maps, p->bsx, npix, p->nc, p->scal, skip);
        p->launches += 1;
    }
    dim3 grid(ceil_div(p->nk, BM), p->nc);
    timing_begin(p, s);
    fwd_fp32_kernel<<<grid, 256, 0, s>>>(p->ax, p->ay, p->bsx, kspace, ld, p->nx, p->ny, p->nk, image ? 0 : 1,
                                         p->scal, skip);
    timing_end(p, s);
    p->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_adj_fp32(mri_plan *p, int skip, cudaStream_t s) {
    dim3 grid(ceil_div(p->nx, BM) * ceil_div(p->ny, BN), p->nc, p->ksplit);
    timing_begin(p, s);
    adj_fp32_kernel<<<grid, 256, 0, s>>>(p->ax, p->ay, p->y, p->part, p->nk_pad, p->nx, p->ny, p->nk, p->nc,
                                         p->nx_pad, p->ksplit, p->ksplit_blocks, p->scal, skip);
    timing_end(p, s);
    p->launches += 1;
    return cudaGetLastError();
}

}  // namespace mri
