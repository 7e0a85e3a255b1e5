// Generation of the separable DFT factors (Alg. 1, per axis):
//   A_x[k][i] = exp(-i 2 pi kx_k x_i),  A_y[k][j] = exp(-i 2 pi ky_k y_j),
// x_i = i - nx/2, y_j = j - ny/2.  The phase kx_k * x_i is formed in FP64
// (exact: a 24-bit mantissa times a small integer) and reduced to [-1/2, 1/2]
// by subtracting the nearest integer, also exact; only then is it rounded to
// FP32 for sincospif.  Besides the FP32 factors, the kernel writes the
// tensor-core operands: the real embedding of A_x (forward product) and of
// conj(A_y) (adjoint product), as BF16 hi/lo splits or as TF32-rounded FP32.
#include "common.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace mri {

namespace {

// exp(-i 2 pi k x) for an integer coordinate x
__device__ __forceinline__ float2 phasor_at(float k, int x) {
    const double t = (double)k * (double)x;
    const double f = t - rint(t);
    float s, c;
    sincospif(-2.0f * (float)f, &s, &c);
    return make_float2(c, s);
}

__device__ __forceinline__ float2 dft_phasor(float k, int idx, int n) { return phasor_at(k, idx - n / 2); }

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 a, __nv_bfloat16 b) {
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// hi = bf16(v), lo = bf16(v - hi) for the two halves of a pair.
__device__ __forceinline__ void split_pair(float a, float b, uint32_t &hi, uint32_t &lo) {
    __nv_bfloat16 ah = __float2bfloat16_rn(a), bh = __float2bfloat16_rn(b);
    __nv_bfloat16 al = __float2bfloat16_rn(a - __bfloat162float(ah));
    __nv_bfloat16 bl = __float2bfloat16_rn(b - __bfloat162float(bh));
    hi = pack_bf16(ah, bh);
    lo = pack_bf16(al, bl);
}

// TF32-rounded pair (a, b) as one 64-bit word (a first).
__device__ __forceinline__ uint2 tf32_pair(float a, float b) { return make_uint2(tc::tf32_bits(a), tc::tf32_bits(b)); }

// One 32 (samples) x 32 (pixel index) tile of one axis.  block = (32, 8).
// F [nk][n] and FT [n][nk] are the FP32 factor and its transpose (either may
// be null).  emb_hi/lo (nullable) receive the forward-product embedding
// rows 2k: (Re, -Im), 2k+1: (Im, Re) at columns 2*idx, leading dim ld_emb.
// cemb_hi/lo (nullable) receive the adjoint-product embedding of
// G = conj(F), leading dim ld_cemb: with one row per index, row idx holds
// (Re G, Im G) at columns 2k, 2k+1; with two rows per index (cemb_two_rows)
// row 2 idx holds (Re G, -Im G) and row 2 idx + 1 holds (Im G, Re G), the
// right operand of [Re U | Im U] G whose output columns 2 idx, 2 idx + 1
// are Re and Im of column idx.  emb_t and cemb_t (nullable) receive the
// same embeddings as TF32-rounded FP32.
__global__ void factor_tile_kernel(const float *__restrict__ traj, int axis, int n, int nk,
                                   float2 *__restrict__ F, float2 *__restrict__ FT, int ld_t,
                                   uint32_t *__restrict__ emb_hi, uint32_t *__restrict__ emb_lo,
                                   uint2 *__restrict__ emb_t, int ld_emb, uint32_t *__restrict__ cemb_hi,
                                   uint32_t *__restrict__ cemb_lo, uint2 *__restrict__ cemb_t, int ld_cemb,
                                   int cemb_two_rows) {
    __shared__ float2 tile[32][33];
    const int k0 = blockIdx.x * 32, p0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    // pass 1: threads along the pixel index (coalesced rows of F and of the forward embedding)
    for (int q = ty; q < 32; q += 8) {
        const int k = k0 + q, idx = p0 + tx;
        float2 v = make_float2(0.f, 0.f);
        if (k < nk && idx < n) {
            v = dft_phasor(traj[2 * k + axis], idx, n);
            if (F) F[(size_t)k * n + idx] = v;
            if (emb_hi) {
                uint32_t h, l;
                // row 2k: (Re, -Im)
                split_pair(v.x, -v.y, h, l);
                emb_hi[((size_t)(2 * k) * ld_emb) / 2 + idx] = h;
                emb_lo[((size_t)(2 * k) * ld_emb) / 2 + idx] = l;
                // row 2k+1: (Im, Re)
                split_pair(v.y, v.x, h, l);
                emb_hi[((size_t)(2 * k + 1) * ld_emb) / 2 + idx] = h;
                emb_lo[((size_t)(2 * k + 1) * ld_emb) / 2 + idx] = l;
            }
            if (emb_t) {
                emb_t[((size_t)(2 * k) * ld_emb) / 2 + idx] = tf32_pair(v.x, -v.y);
                emb_t[((size_t)(2 * k + 1) * ld_emb) / 2 + idx] = tf32_pair(v.y, v.x);
            }
        }
        tile[q][tx] = v;
    }
    __syncthreads();
    // pass 2: threads along the sample index (coalesced rows of FT and of the adjoint embedding)
    for (int q = ty; q < 32; q += 8) {
        const int idx = p0 + q, k = k0 + tx;
        if (k < nk && idx < n) {
            const float2 v = tile[tx][q];
            if (FT) FT[(size_t)idx * ld_t + k] = v;
            // G = conj(F) = (v.x, -v.y)
            if (cemb_two_rows) {
                const size_t r0 = ((size_t)(2 * idx) * ld_cemb) / 2 + k, r1 = r0 + (size_t)ld_cemb / 2;
                if (cemb_hi) {
                    uint32_t h, l;
                    split_pair(v.x, v.y, h, l);  // (Re G, -Im G)
                    cemb_hi[r0] = h;
                    cemb_lo[r0] = l;
                    split_pair(-v.y, v.x, h, l);  // (Im G, Re G)
                    cemb_hi[r1] = h;
                    cemb_lo[r1] = l;
                }
                if (cemb_t) {
                    cemb_t[r0] = tf32_pair(v.x, v.y);
                    cemb_t[r1] = tf32_pair(-v.y, v.x);
                }
            } else {
                if (cemb_hi) {
                    uint32_t h, l;
                    split_pair(v.x, -v.y, h, l);  // (Re G, Im G)
                    cemb_hi[((size_t)idx * ld_cemb) / 2 + k] = h;
                    cemb_lo[((size_t)idx * ld_cemb) / 2 + k] = l;
                }
                if (cemb_t) cemb_t[((size_t)idx * ld_cemb) / 2 + k] = tf32_pair(v.x, -v.y);
            }
        }
    }
}

// Phasor table of one axis: T[r][k] = exp(-i 2 pi k_k (x0 + step r)) for
// r < rows, k < nk, leading dim ld.  The adjoint's pixel-row form takes A_x as
// the product of two such tables (pixel i = 16 a + b: the row of 16 a - nx/2
// times the row of b), a few FP32 roundings from the direct phasor.
__global__ void phasor_table_kernel(const float *__restrict__ traj, int axis, int nk, int rows, int x0, int step,
                                    float2 *__restrict__ T, int ld) {
    const int k = blockIdx.x * 32 + threadIdx.x;
    if (k >= nk) return;
    const float kv = traj[2 * k + axis];
    for (int r = blockIdx.y * blockDim.y + threadIdx.y; r < rows; r += blockDim.y * gridDim.y)
        T[(size_t)r * ld + k] = phasor_at(kv, x0 + step * r);
}

}  // namespace

cudaError_t launch_factors(mri_plan *p, const float *traj, cudaStream_t s) {
    dim3 block(32, 8);
    {
        dim3 grid(ceil_div(p->nk, 32), ceil_div(p->nx, 32));
        factor_tile_kernel<<<grid, block, 0, s>>>(traj, 0, p->nx, p->nk, p->ax, p->axT, p->nk_pad,
                                                  (uint32_t *)p->afwd_hi, (uint32_t *)p->afwd_lo,
                                                  (uint2 *)p->afwd_t, p->kx, nullptr, nullptr, nullptr, 0, 0);
    }
    {
        dim3 grid(ceil_div(p->nk, 32), ceil_div(p->ny, 32));
        factor_tile_kernel<<<grid, block, 0, s>>>(traj, 1, p->ny, p->nk, p->ay, p->ayT, p->nk_pad, nullptr,
                                                  nullptr, nullptr, 0, (uint32_t *)p->badj_hi,
                                                  (uint32_t *)p->badj_lo, (uint2 *)p->badj_t, p->kk,
                                                  p->adj_tile_px == 128);
    }
    p->launches += 2;
    if (p->axP) {
        const int prow = p->nx_pad / 16;
        phasor_table_kernel<<<dim3(ceil_div(p->nk, 32), ceil_div(prow, 8)), block, 0, s>>>(
            traj, 0, p->nk, prow, -(p->nx / 2), 16, p->axP, p->nk_pad);
        phasor_table_kernel<<<dim3(ceil_div(p->nk, 32), 2), block, 0, s>>>(traj, 0, p->nk, 16, 0, 1, p->axQ,
                                                                           p->nk_pad);
        p->launches += 2;
    }
    return cudaGetLastError();
}

}  // namespace mri
