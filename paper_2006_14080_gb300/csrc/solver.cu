// Image-space kernels of the reconstruction: the fixed-order reduction that
// finishes the adjoint (sum over k-space splits, coil combination, optional
// (beta/2) Theta^H Theta term and CG dot product), the finite-difference
// transform Theta and its transpose, the soft threshold (Eq. 9), and the
// CG (Alg. 2) and ADMM (Alg. 4, Eq. 6-12) vector updates with FP64 scalar
// reductions.  All image-sized arrays are [nx][ny] complex64; the TV fields
// are [2][nx][ny].
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

// out[i][j] = sum_c conj(S_c[i][j]) sum_p part[p][c][j][i]  (+ half_beta Theta^H Theta tv_src)
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
        const size_t pstride = (size_t)nc * ny * nx_pad / 2;  // float4 units between k-space splits
        for (int c = ty; c < nc; c += G) {
            const float4 *src = reinterpret_cast<const float4 *>(part + ((size_t)c * ny + j) * nx_pad + i0);
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

// mu = S_t(Theta x + eta); xprev = x; opens a new x-update (cg_done = 0).
__global__ void admm_mu_kernel(int nx, int ny, const float2 *__restrict__ x, const float2 *__restrict__ eta,
                               float2 *__restrict__ mu, float2 *__restrict__ xprev, float t, DevScalars *sc) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (sc->admm_done) {
        if (n == 0) sc->step_active = 0;
        return;
    }
    if (n == 0) {
        sc->cg_done = 0;
        sc->step_active = 1;
    }
    if (n >= nx * ny) return;
    const size_t npix = (size_t)nx * ny;
    const int i = n / ny, j = n % ny;
    float2 gx, gy;
    theta_at(x, i, j, nx, ny, gx, gy);
    mu[n] = soft_threshold(cadd(gx, eta[n]), t);
    mu[npix + n] = soft_threshold(cadd(gy, eta[npix + n]), t);
    xprev[n] = x[n];
}

// b = F^H d + half_beta Theta^H (mu - eta)   (Eq. 12)
__global__ void admm_rhs_kernel(int nx, int ny, const float2 *__restrict__ fhd, const float2 *__restrict__ mu,
                                const float2 *__restrict__ eta, float2 *__restrict__ b, float half_beta,
                                const DevScalars *sc) {
    if (sc->admm_done) return;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nx * ny) return;
    const size_t npix = (size_t)nx * ny;
    const int i = n / ny, j = n % ny;
    // Theta^H of the field pair (mu - eta), evaluated from its four neighbours
    auto diff = [&](int f, int ii, int jj) -> float2 {
        if (ii < 0 || jj < 0) return make_float2(0.f, 0.f);
        const size_t q = (size_t)f * npix + (size_t)ii * ny + jj;
        return csub(mu[q], eta[q]);
    };
    float2 t = cadd(csub(diff(0, i - 1, j), diff(0, i, j)), csub(diff(1, i, j - 1), diff(1, i, j)));
    const float2 f = fhd[n];
    b[n] = make_float2(fmaf(half_beta, t.x, f.x), fmaf(half_beta, t.y, f.y));
}

// r = b - A x, d = r, tau = ||r||^2 (Alg. 2 start, A x already in ad)
__global__ void cg_init_kernel(int npix, const float2 *__restrict__ b, const float2 *__restrict__ ax,
                               float2 *__restrict__ r, float2 *__restrict__ d, DevScalars *sc, double *partials) {
    if (sc->admm_done) return;
    __shared__ double red[32];
    double s = 0.0;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < npix; n += gridDim.x * blockDim.x) {
        const float2 v = csub(b[n], ax[n]);
        r[n] = v;
        d[n] = v;
        s += (double)v.x * v.x + (double)v.y * v.y;
    }
    double part[1] = {block_sum(s, red)};
    grid_reduce_last<1>(part, partials, &sc->counters[kCntInit], [&](const double *tot) {
        sc->tau = tot[0];
        sc->cg_done = !(tot[0] > sc->atol2);
    });
}

// x += alpha d; r -= alpha A d; tau' = ||r||^2; beta_cg = tau'/tau; tau = tau'.
// The step length is applied in FP64 (Alg. 2 keeps its scalars in double):
// rounding alpha to FP32 alone moves the N=32 reconstruction by ~2.5e-3 NRMSE
// against the FP64 solver, while FP32 vectors with FP64 scalars move it by
// ~5e-5.  Each updated element is rounded to FP32 once.
__global__ void cg_update_kernel(int npix, float2 *__restrict__ x, float2 *__restrict__ r,
                                 const float2 *__restrict__ d, const float2 *__restrict__ ad, DevScalars *sc,
                                 double *partials) {
    if (sc->admm_done || sc->cg_done) return;
    __shared__ double red[32];
    const double alpha = sc->alpha;
    double s = 0.0;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < npix; n += gridDim.x * blockDim.x) {
        const float2 dv = d[n], adv = ad[n];
        float2 xv = x[n], rv = r[n];
        xv.x = (float)fma(alpha, (double)dv.x, (double)xv.x);
        xv.y = (float)fma(alpha, (double)dv.y, (double)xv.y);
        rv.x = (float)fma(-alpha, (double)adv.x, (double)rv.x);
        rv.y = (float)fma(-alpha, (double)adv.y, (double)rv.y);
        x[n] = xv;
        r[n] = rv;
        s += (double)rv.x * rv.x + (double)rv.y * rv.y;
    }
    double part[1] = {block_sum(s, red)};
    grid_reduce_last<1>(part, partials, &sc->counters[kCntTau], [&](const double *tot) {
        sc->beta_cg = tot[0] / sc->tau;
        sc->tau = tot[0];
        sc->cg_done = !(tot[0] > sc->atol2);
    });
}

// d = r + beta_cg d, with beta_cg applied in FP64 like alpha above
__global__ void cg_direction_kernel(int npix, const float2 *__restrict__ r, float2 *__restrict__ d,
                                    const DevScalars *sc) {
    if (sc->admm_done || sc->cg_done) return;
    const double bcg = sc->beta_cg;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < npix; n += gridDim.x * blockDim.x) {
        const float2 rv = r[n], dv = d[n];
        d[n] = make_float2((float)fma(bcg, (double)dv.x, (double)rv.x), (float)fma(bcg, (double)dv.y, (double)rv.y));
    }
}

// eta += Theta x - mu; alpha_admm = ||x - xprev||^2 / ||x||^2
__global__ void admm_dual_kernel(int nx, int ny, const float2 *__restrict__ x, const float2 *__restrict__ xprev,
                                 const float2 *__restrict__ mu, float2 *__restrict__ eta, DevScalars *sc,
                                 double *partials, double *alpha_hist, int m) {
    if (sc->admm_done) return;
    __shared__ double red[32];
    const int npix = nx * ny;
    double num = 0.0, den = 0.0;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < npix; n += gridDim.x * blockDim.x) {
        const int i = n / ny, j = n % ny;
        float2 gx, gy;
        theta_at(x, i, j, nx, ny, gx, gy);
        eta[n] = csub(cadd(eta[n], gx), mu[n]);
        eta[npix + n] = csub(cadd(eta[npix + n], gy), mu[npix + n]);
        const float2 xv = x[n], pv = xprev[n];
        const double dx = (double)xv.x - pv.x, dy = (double)xv.y - pv.y;
        num += dx * dx + dy * dy;
        den += (double)xv.x * xv.x + (double)xv.y * xv.y;
    }
    double part[2];
    part[0] = block_sum(num, red);
    part[1] = block_sum(den, red);
    grid_reduce_last<2>(part, partials, &sc->counters[kCntDual], [&](const double *tot) {
        const double a = tot[0] / (tot[1] > 1e-300 ? tot[1] : 1e-300);
        sc->admm_alpha = a;
        if (alpha_hist) alpha_hist[m] = a;
        sc->admm_done = !(a > sc->rtol2);
    });
}

// f = ||y - d||^2 + lambda sum |Theta x|  (Eq. 3), with y = F x already in
// yfx.  Recorded for every step that ran, including the one that met rtol.
__global__ void objective_kernel(int nx, int ny, int nk, int nkc, const float2 *__restrict__ yfx, int yfx_ld,
                                 const float2 *__restrict__ kspace, const float2 *__restrict__ x, float lambda,
                                 DevScalars *sc, double *partials, double *obj_hist, int m) {
    if (!sc->step_active) return;
    __shared__ double red[32];
    const int npix = nx * ny;
    double fid = 0.0, l1 = 0.0;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < nkc; n += gridDim.x * blockDim.x) {
        const float2 r = csub(yfx[(size_t)(n / nk) * yfx_ld + n % nk], kspace[n]);
        fid += (double)r.x * r.x + (double)r.y * r.y;
    }
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < npix; n += gridDim.x * blockDim.x) {
        float2 gx, gy;
        theta_at(x, n / ny, n % ny, nx, ny, gx, gy);
        l1 += sqrt((double)gx.x * gx.x + (double)gx.y * gx.y) + sqrt((double)gy.x * gy.x + (double)gy.y * gy.y);
    }
    double part[2];
    part[0] = block_sum(fid, red);
    part[1] = block_sum(l1, red);
    grid_reduce_last<2>(part, partials, &sc->counters[kCntObj],
                        [&](const double *tot) { obj_hist[m] = tot[0] + (double)lambda * tot[1]; });
}

__global__ void admm_reset_kernel(DevScalars *sc, double atol2, double rtol2) {
    sc->tau = 0.0;
    sc->alpha = 0.0;
    sc->beta_cg = 0.0;
    sc->admm_alpha = 1.0;
    sc->atol2 = atol2;
    sc->rtol2 = rtol2;
    sc->cg_done = 0;
    sc->admm_done = 0;
    sc->step_active = 0;
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

cudaError_t launch_admm_mu(mri_plan *p, float thresh, cudaStream_t s) {
    admm_mu_kernel<<<ceil_div(p->nx * p->ny, kEwThreads), kEwThreads, 0, s>>>(p->nx, p->ny, p->x, p->eta, p->mu,
                                                                              p->xprev, thresh, p->scal);
    return cudaGetLastError();
}

cudaError_t launch_admm_rhs(mri_plan *p, float half_beta, cudaStream_t s) {
    admm_rhs_kernel<<<ceil_div(p->nx * p->ny, kEwThreads), kEwThreads, 0, s>>>(p->nx, p->ny, p->fhd, p->mu, p->eta,
                                                                               p->b, half_beta, p->scal);
    return cudaGetLastError();
}

cudaError_t launch_cg_init(mri_plan *p, cudaStream_t s) {
    const int npix = p->nx * p->ny;
    cg_init_kernel<<<ew_blocks(npix), kEwThreads, 0, s>>>(npix, p->b, p->ad, p->r, p->d, p->scal, p->partials);
    return cudaGetLastError();
}

cudaError_t launch_cg_update(mri_plan *p, cudaStream_t s) {
    const int npix = p->nx * p->ny;
    cg_update_kernel<<<ew_blocks(npix), kEwThreads, 0, s>>>(npix, p->x, p->r, p->d, p->ad, p->scal, p->partials);
    return cudaGetLastError();
}

cudaError_t launch_cg_direction(mri_plan *p, cudaStream_t s) {
    const int npix = p->nx * p->ny;
    cg_direction_kernel<<<ew_blocks(npix), kEwThreads, 0, s>>>(npix, p->r, p->d, p->scal);
    return cudaGetLastError();
}

cudaError_t launch_admm_dual(mri_plan *p, double *alpha_hist, int m, cudaStream_t s) {
    const int npix = p->nx * p->ny;
    admm_dual_kernel<<<ew_blocks(npix), kEwThreads, 0, s>>>(p->nx, p->ny, p->x, p->xprev, p->mu, p->eta, p->scal,
                                                            p->partials, alpha_hist, m);
    return cudaGetLastError();
}

cudaError_t launch_objective(mri_plan *p, const float2 *kspace, float lambda, double *obj_hist, int m,
                             cudaStream_t s) {
    const int npix = p->nx * p->ny;
    const int nkc = p->nk * p->nc;
    objective_kernel<<<ew_blocks(max(npix, nkc)), kEwThreads, 0, s>>>(p->nx, p->ny, p->nk, nkc, p->y, p->nk_pad,
                                                                      kspace, p->x, lambda, p->scal, p->partials,
                                                                      obj_hist, m);
    return cudaGetLastError();
}

cudaError_t launch_admm_reset(mri_plan *p, double atol, double rtol, cudaStream_t s) {
    admm_reset_kernel<<<1, 1, 0, s>>>(p->scal, atol * atol, rtol * rtol);
    return cudaGetLastError();
}

}  // namespace mri
