// Shared device helpers of the mrirecon library: complex arithmetic, warp and
// block reductions in FP64, and the deterministic "last block finishes the
// sum" pattern used by every scalar reduction of the solver.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "mrirecon.h"

namespace mri {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float4 f4add(float4 a, float4 b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 v) { return *reinterpret_cast<uint32_t *>(&v); }

// hi/lo split of a pair of FP32 values into packed bf16x2 words (a in the low
// half): hi = bf16(v), lo = bf16(v - hi), both rounded to nearest even.
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo) {
    const __nv_bfloat162 h = __float22bfloat162_rn(make_float2(a, b));
    const float2 hf = __bfloat1622float2(h);
    hi = bf2_bits(h);
    lo = bf2_bits(__float22bfloat162_rn(make_float2(a - hf.x, b - hf.y)));
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Flattened thread index for 2-D blocks.
__device__ __forceinline__ int flat_tid() { return threadIdx.y * blockDim.x + threadIdx.x; }

// Sum of v over the block (1-D or 2-D, a multiple of 32 threads, <= 1024),
// fixed order; the result is valid in flat thread 0.
__device__ __forceinline__ double block_sum(double v, double *scratch /* >= 32 doubles */) {
    const int tid = flat_tid();
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarp = (blockDim.x * blockDim.y + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (tid == 0)
        for (int w = 0; w < nwarp; ++w) s += scratch[w];
    return s;
}

// Deterministic grid reduction: every block deposits its partial sums
// (NV values) in partials[block][NV]; the last block to arrive adds them in
// block order and calls fin(sums) with thread 0 only.  counter must start at
// zero and is reset by the last block.  Returns true in the block that ran fin.
template <int NV, typename Fin>
__device__ __forceinline__ bool grid_reduce_last(const double (&part)[NV], double *partials,
                                                 unsigned *counter, Fin fin) {
    __shared__ bool is_last;
    const int nblocks = gridDim.x * gridDim.y * gridDim.z;
    const int bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    const int tid = flat_tid();
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) partials[(size_t)bid * NV + q] = part[q];
        __threadfence();
        unsigned t = atomicAdd(counter, 1u);
        is_last = (t == (unsigned)nblocks - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    // warp 0 of the last block adds the partials: lane l takes blocks l,
    // l + 32, ... in order, then the lanes are combined in a fixed order (the
    // other warps take no part: FP64 adds are slow on this GPU)
    double s[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) s[q] = 0.0;
    if (tid < 32) {
        for (int b = tid; b < nblocks; b += 32)
#pragma unroll
            for (int q = 0; q < NV; ++q) s[q] += __ldcg(&partials[(size_t)b * NV + q]);
#pragma unroll
        for (int q = 0; q < NV; ++q) s[q] = warp_sum(s[q]);
    }
    if (tid == 0) {
        fin(s);
        *counter = 0u;
        __threadfence();
    }
    return true;
}

}  // namespace mri
