// Allocation-free adjoint DFT entry point (mri_nudft_adjoint_noalloc).
//
// For callers that cannot allocate device memory: code that runs while
// allocation is forbidden or unsafe (inside a real-time loop or a
// host callback, in a process whose memory is fully reserved up front, or a
// plug-in that must not touch the CUDA allocator).  The call needs no plan:
// it computes the separable DFT factors on the fly from the trajectory and
// keeps its k-space-split partial images in a fixed, file-scope device
// buffer that every GPU which loads the library holds until the process exits.
//
// Limits and sharing rules:
//   - the scratch holds kNoallocScratchElems complex values (16 MiB);
//     nc * nx * ny must not exceed that, or the call returns MRI_ERR_INVALID.
//   - all calls on one device share the buffer and it keeps the last call's
//     contents.  Calls whose work overlaps on the GPU (different streams, no
//     ordering between them) race on it; serialise them.  Every element a
//     call reads is written earlier by the same call, so nothing needs
//     clearing between calls.
//   - nc must not exceed 65535 (one grid row per coil), else MRI_ERR_INVALID.
//   - the first call on a device looks up the buffer's device address (once
//     per device, with that device current); make that first call before any
//     stream capture.  The address is kept for the life of the process, so
//     calls after a cudaDeviceReset of that device are not supported.
//   - numerics follow the FP32 form of mri_nudft_adjoint: FP64 phase
//     reduction, FP32 sine/cosine and FFMA products, fixed-order two-level
//     sums (16-sample blocks, then the running sum).
#include <algorithm>
#include <mutex>
#include <string>

#include "common.cuh"
#include "internal.h"

namespace mri {

namespace {

constexpr size_t kNoallocScratchElems = (16u << 20) / sizeof(float2);  // 16 MiB of complex64
constexpr int kMaxDevices = 64;
constexpr int NBM = 64, NBN = 64, NBK = 16;

static __device__ __align__(256) float2 g_noalloc_scratch[kNoallocScratchElems];

std::mutex g_scratch_mutex;
float2 *g_scratch_ptr[kMaxDevices] = {};

__device__ __forceinline__ float2 phasor(float k, int idx, int n) {
    const double t = (double)k * (double)(idx - n / 2);
    const double f = t - rint(t);
    float s, c;
    sincospif(-2.0f * (float)f, &s, &c);
    return make_float2(c, s);
}

// part[p][c][i][j] = sum_{k in split p} conj(A_x[k][i]) y_c[k] conj(A_y[k][j]),
// factors formed on the fly while staging.  256 threads, 64 x 64 tile, 4 x 4 per thread.
__global__ void __launch_bounds__(256) noalloc_adj_partials(const float *__restrict__ traj,
                                                            const float2 *__restrict__ y, float2 *__restrict__ part,
                                                            int nx, int ny, int nk, int nc, int per_split) {
    __shared__ __align__(16) float2 Us[NBK][NBM];
    __shared__ __align__(16) float2 Vs[NBK][NBN];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int tiles_i = (nx + NBM - 1) / NBM;
    const int i0 = (blockIdx.x % tiles_i) * NBM, j0 = (blockIdx.x / tiles_i) * NBN;
    const int c = blockIdx.y, p = blockIdx.z;
    const int kbeg = p * per_split, kend = min(nk, kbeg + per_split);
    const float2 *yc = y + (size_t)c * nk;
    float2 acc[4][4];
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[m][q] = make_float2(0.f, 0.f);
    const int s_row = tid >> 4, s_col = (tid & 15) * 4;
    for (int kb = kbeg; kb < kend; kb += NBK) {
        const int kk = kb + s_row;
        const bool ok = kk < kend;
        const float2 yk = ok ? yc[kk] : make_float2(0.f, 0.f);
        const float kx = ok ? traj[2 * kk] : 0.f, ky = ok ? traj[2 * kk + 1] : 0.f;
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int ii = i0 + s_col + q, jj = j0 + s_col + q;
            Us[s_row][s_col + q] = (ok && ii < nx) ? cmulc(phasor(kx, ii, nx), yk) : make_float2(0.f, 0.f);
            Vs[s_row][s_col + q] = (ok && jj < ny) ? cconj(phasor(ky, jj, ny)) : make_float2(0.f, 0.f);
        }
        __syncthreads();
        float2 blk[4][4];  // this stage's NBK samples, added to acc below (two-level sum)
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
            for (int q = 0; q < 4; ++q) blk[m][q] = make_float2(0.f, 0.f);
#pragma unroll
        for (int kq = 0; kq < NBK; ++kq) {
            float2 u[4], v[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) u[m] = Us[kq][ty * 4 + m];
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = Vs[kq][tx * 4 + q];
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
    }
    // image layout (j fastest), so that the combine below reads it coalesced
    float2 *dst = part + (((size_t)p * nc + c) * nx) * ny;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int ii = i0 + ty * 4 + m;
        if (ii >= nx) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int jj = j0 + tx * 4 + q;
            if (jj < ny) dst[(size_t)ii * ny + jj] = acc[m][q];
        }
    }
}

// image[i][j] = sum_c conj(S_c[i][j]) sum_p part[p][c][i][j], fixed order;
// consecutive threads take consecutive pixels n = i ny + j of every array.
__global__ void noalloc_adj_combine(const float2 *__restrict__ part, const float2 *__restrict__ maps,
                                    float2 *__restrict__ image, int nx, int ny, int nc, int ksplit) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nx * ny) return;
    const size_t npix = (size_t)nx * ny;
    float2 acc = make_float2(0.f, 0.f);
    for (int c = 0; c < nc; ++c) {
        float2 w = make_float2(0.f, 0.f);
        for (int p = 0; p < ksplit; ++p) w = cadd(w, part[((size_t)p * nc + c) * npix + n]);
        acc = cadd(acc, cmulc(maps[c * npix + n], w));
    }
    image[n] = acc;
}

// Device address of the scratch buffer on the current device (looked up once per device).
int scratch_for_current_device(float2 **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return MRI_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device index out of range for the allocation-free entry point");
        return MRI_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || ptr == nullptr) {
            set_error(std::string("cudaGetSymbolAddress of the scratch buffer: ") + cudaGetErrorString(e));
            return MRI_ERR_CUDA;
        }
        g_scratch_ptr[dev] = (float2 *)ptr;
    }
    *out = g_scratch_ptr[dev];
    return MRI_OK;
}

}  // namespace

}  // namespace mri

using namespace mri;

extern "C" MRI_API int mri_nudft_adjoint_noalloc(int nx, int ny, int nk, int nc, const float *traj,
                                                 const mri_c64 *kspace, const mri_c64 *coil_maps, mri_c64 *image,
                                                 mri_stream_t stream) {
    if (nx <= 0 || ny <= 0 || nk <= 0 || nc <= 0) {
        set_error("dimensions must be positive");
        return MRI_ERR_INVALID;
    }
    if (!traj || !kspace || !coil_maps || !image) {
        set_error("null argument");
        return MRI_ERR_INVALID;
    }
    if (nc > 65535) {
        set_error("nc = " + std::to_string(nc) + " exceeds the 65535 coils of the allocation-free entry point");
        return MRI_ERR_INVALID;
    }
    const size_t per_split_elems = (size_t)nc * nx * ny;
    if (per_split_elems > kNoallocScratchElems) {
        set_error("nc * nx * ny = " + std::to_string(per_split_elems) +
                  " exceeds the allocation-free scratch capacity of " + std::to_string(kNoallocScratchElems) +
                  " complex values (16 MiB)");
        return MRI_ERR_INVALID;
    }
    float2 *scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc != MRI_OK) return rc;
    int num_sms = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
    // k-space splits: enough blocks for two waves, bounded by the scratch capacity
    const int tiles = ceil_div(nx, NBM) * ceil_div(ny, NBN) * nc;
    int split = std::max(1, std::min(ceil_div(2 * std::max(1, num_sms), tiles), ceil_div(nk, 256)));
    split = std::min<int>(split, (int)(kNoallocScratchElems / per_split_elems));
    const int per = round_up(ceil_div(nk, split), NBK);
    split = ceil_div(nk, per);
    cudaStream_t s = (cudaStream_t)stream;
    dim3 grid(ceil_div(nx, NBM) * ceil_div(ny, NBN), nc, split);
    noalloc_adj_partials<<<grid, 256, 0, s>>>(traj, (const float2 *)kspace, scratch, nx, ny, nk, nc, per);
    noalloc_adj_combine<<<ceil_div(nx * ny, 256), 256, 0, s>>>(scratch, (const float2 *)coil_maps, (float2 *)image,
                                                              nx, ny, nc, split);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("mri_nudft_adjoint_noalloc launch: ") + cudaGetErrorString(e));
        return MRI_ERR_CUDA;
    }
    return MRI_OK;
}
