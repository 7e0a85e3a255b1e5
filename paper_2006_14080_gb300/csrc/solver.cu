// Image-space kernels of the operator entry points: the fixed-order
// reduction that finishes the adjoint (sum over k-space splits, coil
// combination, optional (beta/2) Theta^H Theta term and CG dot product), the
// finite-difference transform Theta and its transpose, and the soft
// threshold (Eq. 9).  All image-sized arrays are in the ABI layout [nx][ny]
// complex64; the TV fields are [2][nx][ny].  The reconstruction's own
// kernels (Alg. 2 and 4) are in admm.cu.
#include "common.cuh"
#include "internal.h"

namespace mri {

namespace {

constexpr int kEwThreads = 256;
constexpr int kEwMaxBlocks = 1024;  // grid-stride cap for element-wise reductions

__device__ __forceinline__ float2 ld(const float2 *a, int i, int j, int nx, int ny) {
    return (i >= 0 && i < nx && j >= 0 && j < ny) ? a[(size_t)i * ny + j] : make_float2(0.f, 0.f);
}

// Theta at (i, j): forward differences along x and y, zero past the last pixel.
__device__ __forceinline__ void theta_at(const float2 *x, int i, int j, int nx, int ny, float2 &gx, float2 &gy) {
    const float2 c = x[(size_t)i * ny + j];
    gx = csub(ld(x, i + 1, j, nx, ny), c);
    gy = csub(ld(x, i, j + 1, nx, ny), c);
}

// Theta^H at (i, j) of the field pair (g0, g1): g0[i-1][j] - g0[i][j] + g1[i][j-1] - g1[i][j].
__device__ __forceinline__ float2 theta_h_at(const float2 *g0, const float2 *g1, int i, int j, int nx, int ny) {
    float2 v = csub(ld(g0, i - 1, j, nx, ny), g0[(size_t)i * ny + j]);
    return cadd(v, csub(ld(g1, i, j - 1, nx, ny), g1[(size_t)i * ny + j]));
}

// (Theta^H Theta p)(i, j), written as the composition of the two stencils.
__device__ __forceinline__ float2 theta_h_theta_at(const float2 *p, int i, int j, int nx, int ny) {
    float2 gx_here, gy_here, gx_up = make_float2(0.f, 0.f), gy_left = make_float2(0.f, 0.f), dummy;
    theta_at(p, i, j, nx, ny, gx_here, gy_here);
    if (i > 0) theta_at(p, i - 1, j, nx, ny, gx_up, dummy);
    if (j > 0) theta_at(p, i, j - 1, nx, ny, dummy, gy_left);
    return cadd(csub(gx_up, gx_here), csub(gy_left, gy_here));
}

// out[i][j] = sum_c conj(S_c[i][j]) sum_p part[c][j][i / 64][p][i % 64]  (+ half_beta Theta^H Theta tv_src)
// and optionally Re<dot_src, out> -> alpha = tau / dot.  Block (32, G),
// G = min(nc, 16): it covers the 64 consecutive pixels i of one column j,
// two per lane (one 16-byte load of each partial row); thread row ty takes
// the coils c = ty, ty + G, ..., sums each coil's k-space splits (eight
// 16-byte loads in flight per lane, combined in a fixed order), applies conj(S_c)
// once per coil and pixel, and the G groups are added in a fixed order.
constexpr int kReduceGroups = 16;
__global__ void __launch_bounds__(32 * kReduceGroups, 2)
    adj_reduce_kernel(const float2 *__restrict__ part, int ksplit, int nc, int nx, int ny, int nx_pad,
                      const float2 *__restrict__ maps, float2 *__restrict__ out, const float2 *__restrict__ tv_src,
                      float half_beta, const float2 *__restrict__ dot_src, DevScalars *sc, double *partials,
                      int skip) {
    if (should_skip(sc, skip)) return;
    __shared__ float4 grp[kReduceGroups][32];
    __shared__ double red[32];
    const int tx = threadIdx.x, ty = threadIdx.y, G = blockDim.y;
    const int i0 = blockIdx.x * 64 + 2 * tx, j = blockIdx.y;
    const bool has1 = i0 + 1 < nx;  // i0 + 1 < nx_pad always (nx_pad is a multiple of 64)
    const size_t npix = (size_t)nx * ny;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i0 < nx) {
        const size_t pstride = 32;  // float4 units between k-space splits (64 pixels)
        const int n_ig = nx_pad / 64;
        for (int c = ty; c < nc; c += G) {
            const float4 *src = reinterpret_cast<const float4 *>(
                part + (((size_t)c * ny + j) * n_ig + blockIdx.x) * ksplit * 64 + 2 * tx);
            // w[e] sums the splits p = e (mod 4) in increasing order
            float4 w[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) w[e] = make_float4(0.f, 0.f, 0.f, 0.f);
            int p = 0;
            for (; p + 7 < ksplit; p += 8) {
                float4 v[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) v[e] = src[(size_t)(p + e) * pstride];
#pragma unroll
                for (int e = 0; e < 4; ++e) w[e] = f4add(f4add(w[e], v[e]), v[e + 4]);
            }
            for (; p < ksplit; ++p) w[p & 3] = f4add(w[p & 3], src[(size_t)p * pstride]);
            const float4 t = f4add(f4add(w[0], w[1]), f4add(w[2], w[3]));
            const float2 *s = maps + c * npix + (size_t)i0 * ny + j;
            const float2 a0 = cmulc(s[0], make_float2(t.x, t.y));
            const float2 a1 = has1 ? cmulc(s[ny], make_float2(t.z, t.w)) : make_float2(0.f, 0.f);
            acc = f4add(acc, make_float4(a0.x, a0.y, a1.x, a1.y));
        }
    }
    grp[ty][tx] = acc;
    __syncthreads();
    double dot = 0.0;
    // rows 0 and 1 finish pixels i0 and i0 + 1 (row 0 both when G = 1)
    for (int h = ty; h < 2; h += G) {
        const int i = i0 + h;
        if (i >= nx) continue;
        float4 g = grp[0][tx];
        for (int q = 1; q < G; ++q) g = f4add(g, grp[q][tx]);
        float2 v = h ? make_float2(g.z, g.w) : make_float2(g.x, g.y);
        if (tv_src) {
            const float2 tt = theta_h_theta_at(tv_src, i, j, nx, ny);
            v.x = fmaf(half_beta, tt.x, v.x);
            v.y = fmaf(half_beta, tt.y, v.y);
        }
        out[(size_t)i * ny + j] = v;
        if (dot_src) {
            const float2 dv = dot_src[(size_t)i * ny + j];
            dot += (double)dv.x * (double)v.x + (double)dv.y * (double)v.y;
        }
    }
    if (dot_src) {
        double sum = block_sum(dot, red);
        double part_s[1] = {sum};
        grid_reduce_last<1>(part_s, partials, &sc->counters[kCntDot],
                            [&](const double *tot) { sc->alpha = sc->tau / tot[0]; });
    }
}

__global__ void tv_forward_kernel(int nx, int ny, const float2 *__restrict__ x, float2 *__restrict__ g) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nx * ny) return;
    const int i = n / ny, j = n % ny;
    float2 gx, gy;
    theta_at(x, i, j, nx, ny, gx, gy);
    g[n] = gx;
    g[(size_t)nx * ny + n] = gy;
}

__global__ void tv_adjoint_kernel(int nx, int ny, const float2 *__restrict__ g, float2 *__restrict__ x) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nx * ny) return;
    x[n] = theta_h_at(g, g + (size_t)nx * ny, n / ny, n % ny, nx, ny);
}

__device__ __forceinline__ float2 soft_threshold(float2 a, float t) {
    const float mag = sqrtf(a.x * a.x + a.y * a.y);
    if (!(mag > t)) return make_float2(0.f, 0.f);
    const float s = 1.0f - t / mag;
    return make_float2(a.x * s, a.y * s);
}

__global__ void shrink_kernel(int n, float t, const float2 *in, float2 *out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) out[q] = soft_threshold(in[q], t);
}

int ew_blocks(int n) { return max(1, min(kEwMaxBlocks, ceil_div(n, kEwThreads))); }

}  // namespace

cudaError_t launch_adj_reduce(mri_plan *p, const float2 *maps, float2 *out, const ReduceEpilogue &e,
                              cudaStream_t s) {
    dim3 grid(ceil_div(p->nx, 64), p->ny);
    adj_reduce_kernel<<<grid, dim3(32, std::min(p->nc, kReduceGroups)), 0, s>>>(p->part, p->ksplit, p->nc, p->nx, p->ny, p->nx_pad, maps, out,
                                                   e.tv_src, e.half_beta, e.dot_src, p->scal, p->partials, e.skip);
    return cudaGetLastError();
}

cudaError_t launch_tv_forward(int nx, int ny, const float2 *x, float2 *g, cudaStream_t s) {
    tv_forward_kernel<<<ceil_div(nx * ny, kEwThreads), kEwThreads, 0, s>>>(nx, ny, x, g);
    return cudaGetLastError();
}

cudaError_t launch_tv_adjoint(int nx, int ny, const float2 *g, float2 *x, cudaStream_t s) {
    tv_adjoint_kernel<<<ceil_div(nx * ny, kEwThreads), kEwThreads, 0, s>>>(nx, ny, g, x);
    return cudaGetLastError();
}

cudaError_t launch_shrink(int n, float t, const float2 *in, float2 *out, cudaStream_t s) {
    shrink_kernel<<<ceil_div(n, kEwThreads), kEwThreads, 0, s>>>(n, t, in, out);
    return cudaGetLastError();
}

}  // namespace mri
