// Image-space kernels of the reconstruction (Alg. 4 with Alg. 2 inside,
// Eq. 6-12), working on the solver's own copy of the image-sized state in
// the transposed layout v[j][i] (pixel (i, j) at j * nx + i).
//
// The adjoint product leaves its k-space-split partial images with the
// pixel index i fastest (part[c][j][ig][p][64]), and the forward product
// reads its operand S_c . v as rows (c, j) with i along K.  Keeping x, r, d,
// A d, b, F^H d, mu, eta and the coil maps with i fastest too makes every
// access of these kernels coalesced, lets the kernel that finishes the
// adjoint write the next forward operand directly, and removes the separate
// operand kernel from every CG step.  The caller's image, maps and saved
// states stay in the ABI layout [i][j]; they are transposed in and out once
// per reconstruction.
//
// One CG step of Alg. 2 after the two products is a single cooperative
// kernel (or, for reconstructions that share the GPU with others, the same
// arithmetic as two ordinary kernels split at the barrier): (1) the fixed-order sum of the partial images and the coil
// combination give A d (with the (beta/2) Theta^H Theta d term), and the
// dot products Re<d, A d>, Re<r, A d> and ||A d||^2; one grid barrier;
// (2) alpha = tau / Re<d, A d>, tau' = ||r - alpha A d||^2 from the expanded
// square, beta = tau' / tau; (3) x += alpha d, r -= alpha A d,
// d = r + beta d, and the forward operand S_c . d for the next step.  All
// scalars are FP64 and every sum runs in a fixed order (per-thread, then
// per-block in thread order, then over blocks in block order, the same in
// every block), so the result does not depend on scheduling.  The grid
// barriers are bounded waits: past the limit the kernel records
// kStatusTimeout in the plan's status word and runs on (its results are then
// invalid, never a hang).
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace mri {

namespace {

// Forms of the forward operand the solver writes (one per precision).
enum OperandMode : int { kOpBf16x3 = 0, kOpTf32 = 1, kOpFp32 = 2 };

constexpr int kRedThreadsX = 32;   // lanes: two pixels i each (64 per item)
constexpr int kRedGroups = 16;     // thread rows: coils c = ty, ty + 16, ...
constexpr int kRedThreads = kRedThreadsX * kRedGroups;
constexpr int kEwThreads = 256;
constexpr int kEwMaxBlocks = 1024;
constexpr uint64_t kBarrierLimitNs = 1000000000ull;  // 1 s per grid barrier

__device__ __forceinline__ float2 ldT(const float2 *a, int i, int j, int nx, int ny) {
    return (i >= 0 && i < nx && j >= 0 && j < ny) ? a[(size_t)j * nx + i] : make_float2(0.f, 0.f);
}

// Theta at (i, j) of a transposed image: differences along i (first field)
// and along j (second field), zero past the last pixel.
__device__ __forceinline__ void thetaT(const float2 *x, int i, int j, int nx, int ny, float2 &gx, float2 &gy) {
    const float2 c = x[(size_t)j * nx + i];
    gx = csub(ldT(x, i + 1, j, nx, ny), c);
    gy = csub(ldT(x, i, j + 1, nx, ny), c);
}

// (Theta^H Theta v)(i, j) of a transposed image, as the composition of the two stencils.
__device__ __forceinline__ float2 theta_h_thetaT(const float2 *v, int i, int j, int nx, int ny) {
    float2 gx_here, gy_here, gx_up = make_float2(0.f, 0.f), gy_left = make_float2(0.f, 0.f), dummy;
    thetaT(v, i, j, nx, ny, gx_here, gy_here);
    if (i > 0) thetaT(v, i - 1, j, nx, ny, gx_up, dummy);
    if (j > 0) thetaT(v, i, j - 1, nx, ny, dummy, gy_left);
    return cadd(csub(gx_up, gx_here), csub(gy_left, gy_here));
}

__device__ __forceinline__ float2 soft_threshold(float2 a, float t) {
    const float mag = sqrtf(a.x * a.x + a.y * a.y);
    if (!(mag > t)) return make_float2(0.f, 0.f);
    const float s = 1.0f - t / mag;
    return make_float2(a.x * s, a.y * s);
}

// Where the solver writes the forward operand S_c . v of pixel (i, j).
struct Operand {
    uint32_t *hi = nullptr, *lo = nullptr;  // BF16x3: packed (re, im) bf16 words [nc * ny_pad][kx / 2]
    uint2 *t32 = nullptr;                   // TF32: (re, im) TF32 words [nc * ny_pad][kx / 2]
    float2 *fp32 = nullptr;                 // FP32 form: [nc][ny][nx] (transposed)
    int ny_pad = 0, kx2 = 0;
};

// An FP64 scalar as a pair of FP32 values, s = hi + lo to about 2^-48.
struct Split {
    float hi, lo;
};
__device__ __forceinline__ Split split_scalar(double s) {
    const float hi = (float)s;
    return {hi, (float)(s - (double)hi)};
}
// acc + s v for an FP64 scalar s applied as its FP32 pair (two FP32 FMAs per
// component): the scalar keeps its FP64 value, and the result carries FP32
// rounding only, as one FP64 FMA rounded to FP32 would, without using the
// FP64 pipe (a small fraction of the FP32 rate on this GPU).
__device__ __forceinline__ float2 axpy(Split s, float2 v, float2 acc) {
    return make_float2(fmaf(s.lo, v.x, fmaf(s.hi, v.x, acc.x)), fmaf(s.lo, v.y, fmaf(s.hi, v.y, acc.y)));
}

// Forward operand entry of coil c at pixel n = j nx + i: S_c . v, with the
// maps in the plan's transposed copy mapsT[c][j][ldm] (rows padded to ldm).
// Callers loop over (coil, pixel) pairs e = c npix + n, one per thread, so
// that every coil's map entries and operand words are read and written
// coalesced and the coils proceed in parallel.
__device__ __forceinline__ float2 map_at(const float2 *__restrict__ mapsT, int ldm, int ny, int c, size_t n, int nx) {
    return mapsT[((size_t)c * ny + n / nx) * ldm + n % nx];
}
// ... with the map entry s = map_at(...) already loaded.
template <int kMode>
__device__ __forceinline__ void put_operand_w(const Operand &op, int c, size_t e, size_t n, int nx, float2 s, float2 v) {
    const int i = (int)(n % nx), j = (int)(n / nx);
    const float2 w = cmul(s, v);
    if constexpr (kMode == kOpFp32) {
        op.fp32[e] = w;
    } else {
        const size_t off = ((size_t)c * op.ny_pad + j) * op.kx2 + i;
        if constexpr (kMode == kOpTf32) {
            op.t32[off] = make_uint2(tc::tf32_bits(w.x), tc::tf32_bits(w.y));
        } else {
            uint32_t h, l;
            split2(w.x, w.y, h, l);
            op.hi[off] = h;
            op.lo[off] = l;
        }
    }
}
template <int kMode>
__device__ __forceinline__ void put_operand_one(const Operand &op, const float2 *__restrict__ mapsT, int ldm, int ny,
                                                size_t e, int c, size_t n, int nx, float2 v) {
    const int i = (int)(n % nx), j = (int)(n / nx);
    const float2 w = cmul(mapsT[((size_t)c * ny + j) * ldm + i], v);
    if constexpr (kMode == kOpFp32) {
        op.fp32[e] = w;
    } else {
        const size_t off = ((size_t)c * op.ny_pad + j) * op.kx2 + i;
        if constexpr (kMode == kOpTf32) {
            op.t32[off] = make_uint2(tc::tf32_bits(w.x), tc::tf32_bits(w.y));
        } else {
            uint32_t h, l;
            split2(w.x, w.y, h, l);
            op.hi[off] = h;
            op.lo[off] = l;
        }
    }
}

// The operand of a transposed image v that the kernel does not write, over
// the grid-stride loop e = e0, e0 + de, ... < nc npix.
template <int kMode>
__device__ __forceinline__ void put_operand_all(const Operand &op, const float2 *__restrict__ mapsT, int ldm,
                                                const float2 *__restrict__ v, int nc, int ny, size_t npix, int nx,
                                                size_t e0, size_t de) {
    for (size_t e = e0; e < npix * nc; e += de) {
        const int c = (int)(e / npix);
        const size_t n = e - (size_t)c * npix;
        put_operand_one<kMode>(op, mapsT, ldm, ny, e, c, n, nx, v[n]);
    }
}

// The partial images and what is needed to finish the adjoint at a pixel
// group: item (j, ig) is the 64 pixels i = 64 ig + [0, 64) of column j.
struct Partials {
    const float2 *part;
    int ksplit, nc, nx, ny, n_ig;
    const float2 *mapsT;  // [nc][ny][nx_pad]
    int cs, n_groups;     // coils per shared-memory stage; stages per item
    int chunk;            // complex values per coil in a stage: ksplit * 64 partials + 64 map entries
    int stage_elems;      // complex values per stage: cs * chunk, at least kMinStageElems
};

// A stage holds at least 1024 complex values: the CG step reuses the ring
// (2 x 1024 doubles) to stage its per-item partial triples.
constexpr int kMinStageElems = 1024;

constexpr int kRingStages = 2;
constexpr uint64_t kStageWaitNs = 1000000000ull;  // 1 s per stage wait

// Shared-memory ring of the staged partial sums: kRingStages stages of
// cs * chunk complex values each, and their mbarriers.
struct Ring {
    float2 *buf;
    uint64_t *full;
    int stage_elems;
    volatile int *abort;
};

// One unit of a block's sequence: group g (coils [g cs, g cs + cs)) of the
// block's item number u / n_groups.  Called by the lanes of warp 0: lane l
// stages coil g cs + l -- its ksplit contiguous 64-pixel partial rows and its
// 64 map entries, two bulk copies completing on the stage's mbarrier -- and
// lane 0 also arrives with the unit's byte count (a copy may land before
// that arrival: the phase completes only once both have happened).
__device__ __forceinline__ void issue_unit(const Partials &P, const Ring &R, int u) {
    const int lane = threadIdx.x & 31;
    const int k = u / P.n_groups, g = u - k * P.n_groups;
    const int item = blockIdx.x + k * gridDim.x;
    const int ig = item % P.n_ig, j = item / P.n_ig;
    const int c0 = g * P.cs, c1 = min(P.nc, c0 + P.cs);
    const int slot = u % kRingStages;
    float2 *stage = R.buf + (size_t)slot * R.stage_elems;
    const uint32_t bar = tc::smem_u32(R.full + slot);
    tc::fence_proxy_async_smem();  // the stage's previous contents were read through the generic proxy
    if (lane == 0) tc::mbar_arrive_expect_tx(bar, (uint32_t)((c1 - c0) * P.chunk * sizeof(float2)));
    for (int c = c0 + lane; c < c1; c += 32) {
        float2 *dst = stage + (size_t)(c - c0) * P.chunk;
        const float2 *src = P.part + (((size_t)c * P.ny + j) * P.n_ig + ig) * P.ksplit * 64;
        tc::bulk_load(tc::smem_u32(dst), src, (uint32_t)(P.ksplit * 64 * sizeof(float2)), bar);
        const float2 *msrc = P.mapsT + ((size_t)c * P.ny + j) * (P.n_ig * 64) + ig * 64;
        tc::bulk_load(tc::smem_u32(dst + P.ksplit * 64), msrc, 64 * sizeof(float2), bar);
    }
}

// sum_c conj(S_c) sum_p part over the block's items (item = blockIdx.x +
// k gridDim.x < n_items), staged through shared memory by TMA bulk copies
// (two stages in flight).  Every thread row takes part in each stage: the
// rpc = 16 / cs rows of coil slot q = ty / rpc each add the k-space splits
// p = s, s + rpc, s + 2 rpc, ... (s = ty % rpc, increasing order, two
// interleaved chains) for the lane's pixels 64 ig + 2 tx and + 1; row q rpc
// then adds the slot's rpc sums in pairs of increasing s, multiplies by conj(S_c)
// and adds that to its running value (coils in increasing order); the rows
// are finally added in increasing order.  The splits of a coil are summed
// completely before the multiplication: partial images over subsets of the
// splits are far larger than their sum (radial streaks that cancel), and a
// product rounded per subset would carry that larger size into the error.
// The order depends on the plan's shape only.  For each item, epi(item, j, ig,
// i, v) runs in thread rows 0 and 1 (pixel i = 64 ig + 2 tx + ty, v its
// value; i may lie past the image), then done(item) in every thread.
// Returns false if a stage wait ran out (kStatusTimeout is recorded).  All
// threads of the block must call it.
template <typename Epi, typename Done>
__device__ __forceinline__ bool staged_items(const Partials &P, const Ring &R, int n_items, int *status,
                                             float4 (*grp)[kRedThreadsX], Epi epi, Done done) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int my_items = n_items > (int)blockIdx.x ? (n_items - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int units = my_items * P.n_groups;
    int issued = 0;  // warp 0: units issued so far
    if (flat_tid() < 32)
        for (; issued < min(units, kRingStages); ++issued) issue_unit(P, R, issued);
    // this row's coil slot and first split (rows past cs * rpc stay idle)
    const int rpc = kRedGroups / P.cs, slot_q = ty / rpc, sub = ty - slot_q * rpc;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    bool ok = true;
    for (int u = 0; u < units; ++u) {
        const int k = u / P.n_groups, g = u - k * P.n_groups;
        const int slot = u % kRingStages;
        const uint32_t parity = (uint32_t)(u / kRingStages) & 1u;
        if (!tc::mbar_wait(tc::smem_u32(R.full + slot), parity, R.abort, kStageWaitNs)) ok = false;
        const int c = g * P.cs + slot_q;
        if (ok && slot_q < P.cs && c < P.nc) {
            const float2 *chunk = R.buf + (size_t)slot * R.stage_elems + (size_t)slot_q * P.chunk;
            const float4 *src = reinterpret_cast<const float4 *>(chunk) + tx;  // 32 float4 per 64-pixel row
            float4 w0 = make_float4(0.f, 0.f, 0.f, 0.f), w1 = w0;
            int p = sub;
            for (; p + rpc < P.ksplit; p += 2 * rpc) {
                w0 = f4add(w0, src[(size_t)p * 32]);
                w1 = f4add(w1, src[(size_t)(p + rpc) * 32]);
            }
            if (p < P.ksplit) w0 = f4add(w0, src[(size_t)p * 32]);
            grp[ty][tx] = f4add(w0, w1);
        }
        __syncthreads();  // the slots' split sums are in grp
        if (ok && sub == 0 && slot_q < P.cs && c < P.nc) {
            const float2 *chunk = R.buf + (size_t)slot * R.stage_elems + (size_t)slot_q * P.chunk;
            // pairs first: (t0 + t1) + (t2 + t3) + ..., a balanced tree for rpc = 2, 4
            float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
            int q = 0;
            for (; q + 1 < rpc; q += 2) t = f4add(t, f4add(grp[ty + q][tx], grp[ty + q + 1][tx]));
            if (q < rpc) t = f4add(t, grp[ty + q][tx]);
            const float4 m = reinterpret_cast<const float4 *>(chunk + (size_t)P.ksplit * 64)[tx];
            const float2 a0 = cmulc(make_float2(m.x, m.y), make_float2(t.x, t.y));
            const float2 a1 = cmulc(make_float2(m.z, m.w), make_float2(t.z, t.w));
            acc = f4add(acc, make_float4(a0.x, a0.y, a1.x, a1.y));
        }
        __syncthreads();  // the stage and grp have been read
        if (flat_tid() < 32 && ok && !*R.abort && u + kRingStages < units) issue_unit(P, R, issued++);
        if (g == P.n_groups - 1) {
            const int item = blockIdx.x + k * gridDim.x;
            grp[ty][tx] = acc;
            acc = make_float4(0.f, 0.f, 0.f, 0.f);
            __syncthreads();
            if (ty < 2) {
                float4 gs = grp[0][tx];
                for (int q = 1; q < kRedGroups; ++q) gs = f4add(gs, grp[q][tx]);
                const float2 v = ty ? make_float2(gs.z, gs.w) : make_float2(gs.x, gs.y);
                epi(item, item / P.n_ig, item % P.n_ig, (item % P.n_ig) * 64 + 2 * tx + ty, v);
            }
            __syncthreads();  // grp is free again
            done(item);       // all threads
        }
    }
    if (!ok && flat_tid() == 0) {
        atomicExch(status, kStatusTimeout);
        // let the copies that may still be in flight land before the block leaves
        for (int u = max(0, issued - kRingStages); u < issued; ++u) {
            volatile int local = 0;
            tc::mbar_wait(tc::smem_u32(R.full + (u % kRingStages)), (uint32_t)(u / kRingStages) & 1u, &local,
                          kStageWaitNs / 8);
        }
    }
    __syncthreads();
    return ok;
}

// Sets up the ring in dynamic shared memory (barrier init by thread 0).
__device__ __forceinline__ Ring make_ring(const Partials &P, uint8_t *smem, volatile int *abort_flag) {
    Ring R;
    R.stage_elems = P.stage_elems;
    R.buf = reinterpret_cast<float2 *>(smem);
    R.full = reinterpret_cast<uint64_t *>(smem + (size_t)kRingStages * R.stage_elems * sizeof(float2));
    R.abort = abort_flag;
    if (flat_tid() == 0) {
        for (int q = 0; q < kRingStages; ++q) tc::mbar_init(tc::smem_u32(R.full + q), 1);
        *abort_flag = 0;
        tc::fence_barrier_init();
    }
    __syncthreads();
    return R;
}

// Bounded grid-wide barrier of a cooperative launch.  bar[0] counts
// arrivals and only grows (reset to 0 once per reconstruction, a multiple
// of the grid size before every use): a block's ticket t names its barrier,
// which is complete when the count reaches the next multiple of the grid
// size past t.  Nobody resets anything, so the last block's arrival alone
// releases the others.  Returns false (and records kStatusTimeout) if the
// other blocks did not arrive within the limit.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, int *status) {
    __shared__ int ok_s;
    __syncthreads();
    if (flat_tid() == 0) {
        int ok = 1;
        const unsigned nblocks = gridDim.x * gridDim.y * gridDim.z;
        __threadfence();  // the block's writes (made visible to thread 0 by the barrier above) before the arrival
        const unsigned ticket = atomicAdd(bar, 1u);
        const unsigned target = ticket - ticket % nblocks + nblocks;
        volatile unsigned *vbar = bar;
        if ((int)(*vbar - target) < 0) {
            const uint64_t t0 = tc::global_timer_ns();
            while ((int)(*vbar - target) < 0) {
                if (tc::global_timer_ns() - t0 > kBarrierLimitNs) {
                    atomicExch(status, kStatusTimeout);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// Three sums over the warps of thread rows 0 and 1 of a (32, 16) block (the
// rows that hold the pixel values; FP64 adds are slow on this GPU, so the
// other warps take no part), in a fixed order; valid in flat thread 0.
__device__ __forceinline__ void rows01_sum3(double (&v)[3], double (*scratch)[2]) {
    if (threadIdx.y < 2) {
#pragma unroll
        for (int q = 0; q < 3; ++q) v[q] = warp_sum(v[q]);
        if (threadIdx.x == 0)
#pragma unroll
            for (int q = 0; q < 3; ++q) scratch[q][threadIdx.y] = v[q];
    }
    __syncthreads();
    if (flat_tid() == 0)
#pragma unroll
        for (int q = 0; q < 3; ++q) v[q] = scratch[q][0] + scratch[q][1];
}

// The per-item partial triples [0, n) summed in a fixed order that does not
// depend on the grid: warp 0 adds them, lane l taking items l, l + 32, ...
// in increasing order, then the lanes are combined.  They are staged through
// shared memory (cap doubles at a time, one load per thread, no chain of
// dependent global loads).  Valid in flat thread 0.
__device__ __forceinline__ void sum_partials3(const double *partials, int n, double *stage, int cap,
                                              double (&t)[3]) {
#pragma unroll
    for (int q = 0; q < 3; ++q) t[q] = 0.0;
    const int per = cap / 96 * 32;  // items per chunk, a multiple of 32
    for (int b0 = 0; b0 < n; b0 += per) {
        const int m = min(per, n - b0);
        __syncthreads();
        for (int q = flat_tid(); q < 3 * m; q += blockDim.x * blockDim.y) stage[q] = __ldcg(&partials[3 * b0 + q]);
        __syncthreads();
        if (flat_tid() < 32)
            for (int b = flat_tid(); b < m; b += 32)
#pragma unroll
                for (int q = 0; q < 3; ++q) t[q] += stage[3 * b + q];
    }
    if (flat_tid() < 32)
#pragma unroll
        for (int q = 0; q < 3; ++q) t[q] = warp_sum(t[q]);
}

struct CgArgs {
    Partials P;
    float2 *x, *ad;
    const float2 *r, *d;    // the current residual and direction
    float2 *r_next, *d_next;  // receive the next ones (the plan alternates two buffers of each)
    float half_beta;
    Operand op;
    DevScalars *sc;
    double *partials;  // 3 x gridDim.x
    unsigned *bar;
    int n_items;       // n_ig * ny
};

// alpha = tau / Re<d, A d>, tau' = ||r - alpha A d||^2 = tau - 2 alpha
// Re<r, A d> + alpha^2 ||A d||^2 (the square expanded, so that one
// grid-wide reduction serves alpha and beta) and beta = tau' / tau, from the
// per-item partial triples; out[0..2] = alpha, tau', beta in every thread.
// rtau = 1 / tau, formed by the caller before the reduction (off the
// critical path: beta = tau' rtau needs no division after it).  splits[0..2]
// receive alpha, -alpha and beta as FP32 pairs for the updates, formed once
// here: converting them in every thread would keep the SM's few FP64 lanes
// busy for microseconds.
__device__ __forceinline__ void cg_scalars(const double *partials, int n_items, double *stage, double tau,
                                           double rtau, double *out, Split *splits) {
    double t3[3];
    sum_partials3(partials, n_items, stage, 2 * kMinStageElems, t3);
    if (flat_tid() == 0) {
        const double alpha = tau / t3[0];
        const double tau_next = tau - 2.0 * alpha * t3[1] + alpha * alpha * t3[2];
        const double beta = tau_next * rtau;
        out[0] = alpha;
        out[1] = tau_next;
        out[2] = beta;
        splits[0] = split_scalar(alpha);
        splits[1] = split_scalar(-alpha);
        splits[2] = split_scalar(beta);
    }
    __syncthreads();
}

// The updates of a CG step over the grid-stride loop of (coil, pixel) pairs
// starting at gtid: r' = r - alpha A d and d' = r' + beta d at each pair's
// pixel (the same values for every coil) and the operand entry S_c d';
// coil 0 stores x += alpha d, r' and d' (r' and d' into the other buffers:
// r and d are still being read).
template <int kMode>
__device__ __forceinline__ void cg_updates(const CgArgs &A, Split sa, Split sna, Split sb, size_t gtid,
                                           size_t gstride) {
    const int nx = A.P.nx, ny = A.P.ny;
    const size_t npix = (size_t)nx * ny;
    const size_t total = npix * A.P.nc;
    for (size_t e0 = gtid; e0 < total; e0 += 2 * gstride) {
        // two pairs e0 and e0 + gstride per pass, loads of both issued first
        // every load of both pairs (r, d, A d, the map entry and, for coil 0,
        // x) is issued before the first store, so that one round trip to
        // memory serves the pass
        float2 rv[2], dv[2], adv[2], sv[2], xv[2];
        size_t n[2];
        int c[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const size_t e = e0 + h * gstride;
            c[h] = e < total ? (int)(e / npix) : -1;
            n[h] = e < total ? e - (size_t)c[h] * npix : 0;
            if (c[h] >= 0) {
                rv[h] = A.r[n[h]];
                dv[h] = A.d[n[h]];
                adv[h] = A.ad[n[h]];
                sv[h] = map_at(A.P.mapsT, A.P.n_ig * 64, ny, c[h], n[h], nx);
                if (c[h] == 0) xv[h] = A.x[n[h]];
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (c[h] < 0) continue;
            const float2 rn = axpy(sna, adv[h], rv[h]);
            const float2 nd = axpy(sb, dv[h], rn);
            if (c[h] == 0) {  // x is read and written by this thread only
                A.x[n[h]] = axpy(sa, dv[h], xv[h]);
                A.r_next[n[h]] = rn;
                A.d_next[n[h]] = nd;
            }
            put_operand_w<kMode>(A.op, c[h], e0 + h * gstride, n[h], nx, sv[h], nd);
        }
    }
}

// Step (1) of a CG step over the block's items: A d (written to ad) and the
// per-item partial triples Re<d, A d>, Re<r, A d>, ||A d||^2 (each item's 64
// pixels summed in thread order), so that the sums that follow do not
// depend on how items map to blocks.
template <int kMode>
__device__ __forceinline__ void cg_reduce_items(const CgArgs &A, const Ring &R, float4 (*grp)[kRedThreadsX],
                                                double (*red3)[2]) {
    const int nx = A.P.nx, ny = A.P.ny;
    double v3[3] = {0.0, 0.0, 0.0};
    staged_items(
        A.P, R, A.n_items, &A.sc->status, grp,
        [&](int, int j, int, int i, float2 v) {
            if (i >= nx) return;
            const size_t n = (size_t)j * nx + i;
            const float2 dv = A.d[n], rv = A.r[n];  // loaded with the stencil's, before the store
            const float2 tt = theta_h_thetaT(A.d, i, j, nx, ny);
            v.x = fmaf(A.half_beta, tt.x, v.x);
            v.y = fmaf(A.half_beta, tt.y, v.y);
            A.ad[n] = v;
            v3[0] = (double)dv.x * (double)v.x + (double)dv.y * (double)v.y;
            v3[1] = (double)rv.x * (double)v.x + (double)rv.y * (double)v.y;
            v3[2] = (double)v.x * (double)v.x + (double)v.y * (double)v.y;
        },
        [&](int item) {
            rows01_sum3(v3, red3);
            if (flat_tid() == 0)
                for (int q = 0; q < 3; ++q) A.partials[3 * item + q] = v3[q];
            v3[0] = v3[1] = v3[2] = 0.0;
        });
}

// Whether this block is the last of the grid to arrive (counter reset by it).
__device__ __forceinline__ bool last_block_arrives(unsigned *counter) {
    __shared__ int last_s;
    __syncthreads();
    if (flat_tid() == 0) {
        __threadfence();
        const unsigned nblocks = gridDim.x * gridDim.y * gridDim.z;
        const unsigned t = atomicAdd(counter, 1u);
        last_s = t == nblocks - 1;
        if (last_s) *counter = 0u;
        __threadfence();
    }
    __syncthreads();
    return last_s != 0;
}

// A whole CG step as one cooperative kernel: (1) over the items, one grid
// barrier, then every block forms the scalars and (3) the updates.
template <int kMode>
__global__ void __launch_bounds__(kRedThreads, 2) cg_step_kernel(const CgArgs A) {
    if (should_skip(A.sc, kSkipCg)) return;
    extern __shared__ __align__(128) uint8_t dyn_smem[];
    __shared__ float4 grp[kRedGroups][kRedThreadsX];
    __shared__ double red3[3][2];
    __shared__ double scal_s[3];
    __shared__ Split split_s[3];
    __shared__ int abort_s;
    const double tau = A.sc->tau;
    const double rtau = 1.0 / tau;
    const Ring R = make_ring(A.P, dyn_smem, &abort_s);
    cg_reduce_items<kMode>(A, R, grp, red3);
    if (!grid_barrier(A.bar, &A.sc->status)) return;
    // every block forms the same scalars (the ring now stages the partials)
    cg_scalars(A.partials, A.n_items, reinterpret_cast<double *>(R.buf), tau, rtau, scal_s, split_s);
    const double alpha = scal_s[0], tau_next = scal_s[1], beta = scal_s[2];
    cg_updates<kMode>(A, split_s[0], split_s[1], split_s[2], (size_t)blockIdx.x * kRedThreads + flat_tid(),
                      (size_t)gridDim.x * kRedThreads);
    if (blockIdx.x == 0 && flat_tid() == 0) {
        A.sc->alpha = alpha;
        A.sc->beta_cg = beta;
        A.sc->tau = tau_next;
        A.sc->cg_done = !(tau_next > A.sc->atol2);
    }
}

// The same CG step as two ordinary kernels.  The reduction: one item per
// block; the last block to finish forms the scalars from the same partials
// in the same order and hands them to the update kernel.
template <int kMode>
__global__ void __launch_bounds__(kRedThreads, 2) cg_reduce_kernel(const CgArgs A) {
    if (should_skip(A.sc, kSkipCg)) return;
    extern __shared__ __align__(128) uint8_t dyn_smem[];
    __shared__ float4 grp[kRedGroups][kRedThreadsX];
    __shared__ double red3[3][2];
    __shared__ double scal_s[3];
    __shared__ Split split_s[3];
    __shared__ int abort_s;
    const double tau = A.sc->tau;
    const double rtau = 1.0 / tau;
    const Ring R = make_ring(A.P, dyn_smem, &abort_s);
    cg_reduce_items<kMode>(A, R, grp, red3);
    if (!last_block_arrives(&A.sc->counters[kCntDot])) return;
    cg_scalars(A.partials, A.n_items, reinterpret_cast<double *>(R.buf), tau, rtau, scal_s, split_s);
    if (flat_tid() == 0) {
        A.sc->alpha = scal_s[0];
        A.sc->tau_next = scal_s[1];
        A.sc->beta_cg = scal_s[2];
        for (int q = 0; q < 3; ++q) {
            A.sc->cg_split[2 * q] = split_s[q].hi;
            A.sc->cg_split[2 * q + 1] = split_s[q].lo;
        }
        A.sc->step_pending = 1;
    }
}

// The updates of the two-kernel CG step, one (coil, pixel) pair per thread.
template <int kMode>
__global__ void cg_update_kernel(const CgArgs A) {
    if (A.sc->admm_done || !A.sc->step_pending) return;
    const float *f = A.sc->cg_split;  // alpha, -alpha, beta as FP32 pairs, formed once by the reduction
    cg_updates<kMode>(A, Split{f[0], f[1]}, Split{f[2], f[3]}, Split{f[4], f[5]},
                      (size_t)blockIdx.x * blockDim.x + threadIdx.x, (size_t)gridDim.x * blockDim.x);
    if (!last_block_arrives(&A.sc->counters[kCntTau])) return;
    if (threadIdx.x == 0) {
        const double tau_next = A.sc->tau_next;
        A.sc->tau = tau_next;
        A.sc->cg_done = !(tau_next > A.sc->atol2);
        A.sc->step_pending = 0;
    }
}

// The start of Alg. 2 after the products of A x0: r = b - A x0, d = r, the
// forward operand of d, tau = ||r||^2 (last block).  One item per block.
template <int kMode>
__global__ void __launch_bounds__(kRedThreads, 2)
    cg_init_kernel(const Partials P, const float2 *__restrict__ x, const float2 *__restrict__ b, float half_beta,
                   float2 *__restrict__ r, float2 *__restrict__ d, const Operand op, DevScalars *sc,
                   double *partials) {
    if (sc->admm_done) return;
    extern __shared__ __align__(128) uint8_t dyn_smem[];
    __shared__ float4 grp[kRedGroups][kRedThreadsX];
    __shared__ double red3[3][2];
    __shared__ float2 rs[64];
    __shared__ int abort_s;
    const Ring R = make_ring(P, dyn_smem, &abort_s);
    const size_t npix = (size_t)P.nx * P.ny;
    double s = 0.0;
    staged_items(P, R, gridDim.x, &sc->status, grp, [&](int, int j, int ig, int i, float2 v) {
        if (i >= P.nx) return;
        const float2 tt = theta_h_thetaT(x, i, j, P.nx, P.ny);
        v.x = fmaf(half_beta, tt.x, v.x);
        v.y = fmaf(half_beta, tt.y, v.y);
        const size_t n = (size_t)j * P.nx + i;
        const float2 rv = csub(b[n], v);
        r[n] = rv;
        d[n] = rv;
        rs[i - ig * 64] = rv;
        s = (double)rv.x * rv.x + (double)rv.y * rv.y;
    }, [](int) {});
    // the operand of d = r at the block's pixels, one (coil, pixel) pair per thread
    const int ig = blockIdx.x % P.n_ig, j = blockIdx.x / P.n_ig;
    const int npx = min(64, P.nx - ig * 64);
    for (int e = flat_tid(); e < npx * P.nc; e += kRedThreads) {
        const int c = e / npx, q = e - c * npx;
        const size_t n = (size_t)j * P.nx + ig * 64 + q;
        put_operand_one<kMode>(op, P.mapsT, P.n_ig * 64, P.ny, (size_t)c * npix + n, c, n, P.nx, rs[q]);
    }
    double v3[3] = {s, 0.0, 0.0};
    rows01_sum3(v3, red3);
    double part[1] = {v3[0]};
    grid_reduce_last<1>(part, partials, &sc->counters[kCntInit], [&](const double *tot) {
        sc->tau = tot[0];
        sc->cg_done = !(tot[0] > sc->atol2);
    });
}

// F^H d of the measurement (Eq. 12's fixed term), once per reconstruction.
__global__ void __launch_bounds__(kRedThreads, 2) fhd_kernel(const Partials P, float2 *__restrict__ out, int *status) {
    extern __shared__ __align__(128) uint8_t dyn_smem[];
    __shared__ float4 grp[kRedGroups][kRedThreadsX];
    __shared__ int abort_s;
    const Ring R = make_ring(P, dyn_smem, &abort_s);
    staged_items(
        P, R, gridDim.x, status, grp,
        [&](int, int j, int, int i, float2 v) {
            if (i < P.nx) out[(size_t)j * P.nx + i] = v;
        },
        [](int) {});
}

// Opens an ADMM step (Eq. 8 and 12): mu = S_t(Theta x + eta), b = F^H d +
// (beta/2) Theta^H (mu - eta), xprev = x, and the forward operand of x for
// A x0 (x is only read here).  The mu of the neighbours that Theta^H needs
// are recomputed from x and eta with the same arithmetic.
template <int kMode>
__global__ void mu_rhs_kernel(int nx, int ny, const float2 *__restrict__ x, const float2 *__restrict__ eta,
                              const float2 *__restrict__ fhd, float2 *__restrict__ mu, float2 *__restrict__ b,
                              float2 *__restrict__ xprev, float t, float half_beta, const float2 *__restrict__ mapsT,
                              int ldm, int nc, const Operand op, DevScalars *sc) {
    const size_t npix = (size_t)nx * ny;
    const size_t g0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x, dg = (size_t)gridDim.x * blockDim.x;
    if (sc->admm_done) {
        if (g0 == 0) sc->step_active = 0;
        return;
    }
    if (g0 == 0) {
        sc->cg_done = 0;
        sc->step_active = 1;
    }
    const float2 *ex = eta, *ey = eta + npix;
    for (size_t n = g0; n < npix; n += dg) {
        const int i = (int)(n % nx), j = (int)(n / nx);
        const float2 xv = x[n];
        float2 gx, gy;
        thetaT(x, i, j, nx, ny, gx, gy);
        const float2 mx = soft_threshold(cadd(gx, ex[n]), t), my = soft_threshold(cadd(gy, ey[n]), t);
        mu[n] = mx;
        mu[npix + n] = my;
        float2 w = csub(make_float2(0.f, 0.f), cadd(csub(mx, ex[n]), csub(my, ey[n])));
        if (i > 0) {
            const size_t q = n - 1;  // pixel (i - 1, j): its x-difference is x(i, j) - x(i - 1, j)
            w = cadd(w, csub(soft_threshold(cadd(csub(xv, x[q]), ex[q]), t), ex[q]));
        }
        if (j > 0) {
            const size_t q = n - nx;  // pixel (i, j - 1)
            w = cadd(w, csub(soft_threshold(cadd(csub(xv, x[q]), ey[q]), t), ey[q]));
        }
        const float2 f = fhd[n];
        b[n] = make_float2(fmaf(half_beta, w.x, f.x), fmaf(half_beta, w.y, f.y));
        xprev[n] = xv;
    }
    put_operand_all<kMode>(op, mapsT, ldm, x, nc, ny, npix, nx, g0, dg);
}

// eta += Theta x - mu; alpha_admm = ||x - xprev||^2 / ||x||^2 (Alg. 4); and,
// when the objective is recorded, the forward operand of x (only read here).
template <int kMode>
__global__ void dual_kernel(int nx, int ny, const float2 *__restrict__ x, const float2 *__restrict__ xprev,
                            const float2 *__restrict__ mu, float2 *__restrict__ eta, const float2 *__restrict__ mapsT,
                            int ldm, int nc, const Operand op, int operand, DevScalars *sc, double *partials,
                            double *alpha_hist, int m) {
    if (sc->admm_done) return;
    __shared__ double red[32];
    const size_t npix = (size_t)nx * ny;
    const size_t g0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x, dg = (size_t)gridDim.x * blockDim.x;
    double num = 0.0, den = 0.0;
    for (size_t n = g0; n < npix; n += dg) {
        const int i = (int)(n % nx), j = (int)(n / nx);
        float2 gx, gy;
        thetaT(x, i, j, nx, ny, gx, gy);
        eta[n] = csub(cadd(eta[n], gx), mu[n]);
        eta[npix + n] = csub(cadd(eta[npix + n], gy), mu[npix + n]);
        const float2 xv = x[n], pv = xprev[n];
        const double dx = (double)xv.x - pv.x, dy = (double)xv.y - pv.y;
        num += dx * dx + dy * dy;
        den += (double)xv.x * xv.x + (double)xv.y * xv.y;
    }
    if (operand) put_operand_all<kMode>(op, mapsT, ldm, x, nc, ny, npix, nx, g0, dg);
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

// f = ||y - d||^2 + lambda sum |Theta x| (Eq. 3), with y = F x in yfx.
// Recorded for every step that ran, including the one that met rtol.
__global__ void objective_kernel(int nx, int ny, int nk, int nkc, const float2 *__restrict__ yfx, int yfx_ld,
                                 const float2 *__restrict__ kspace, const float2 *__restrict__ x, float lambda,
                                 DevScalars *sc, double *partials, double *obj_hist, int m) {
    if (!sc->step_active) return;
    __shared__ double red[32];
    const size_t npix = (size_t)nx * ny;
    double fid = 0.0, l1 = 0.0;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < nkc; n += gridDim.x * blockDim.x) {
        const float2 r = csub(yfx[(size_t)(n / nk) * yfx_ld + n % nk], kspace[n]);
        fid += (double)r.x * r.x + (double)r.y * r.y;
    }
    for (size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x; n < npix; n += (size_t)gridDim.x * blockDim.x) {
        float2 gx, gy;
        thetaT(x, (int)(n % nx), (int)(n / nx), nx, ny, gx, gy);
        l1 += sqrt((double)gx.x * gx.x + (double)gx.y * gx.y) + sqrt((double)gy.x * gy.x + (double)gy.y * gy.y);
    }
    double part[2];
    part[0] = block_sum(fid, red);
    part[1] = block_sum(l1, red);
    grid_reduce_last<2>(part, partials, &sc->counters[kCntObj],
                        [&](const double *tot) { obj_hist[m] = tot[0] + (double)lambda * tot[1]; });
}

// dst[b][c][r] = src[b][r][c] for `planes` planes of rows x cols complex
// values; destination rows are ld_dst apart (>= rows), planes cols * ld_dst.
__global__ void transpose_kernel(const float2 *__restrict__ src, float2 *__restrict__ dst, int rows, int cols,
                                 int ld_dst) {
    __shared__ float2 t[32][33];
    const float2 *s = src + blockIdx.z * ((size_t)rows * cols);
    float2 *o = dst + blockIdx.z * ((size_t)cols * ld_dst);
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int r = r0 + threadIdx.y + 8 * q, c = c0 + threadIdx.x;
        if (r < rows && c < cols) t[threadIdx.y + 8 * q][threadIdx.x] = s[(size_t)r * cols + c];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c = c0 + threadIdx.y + 8 * q, r = r0 + threadIdx.x;
        if (r < rows && c < cols) o[(size_t)c * ld_dst + r] = t[threadIdx.x][threadIdx.y + 8 * q];
    }
}

__global__ void admm_reset_kernel(DevScalars *sc, unsigned *bar, double atol2, double rtol2) {
    sc->tau = 0.0;
    sc->alpha = 0.0;
    sc->beta_cg = 0.0;
    sc->admm_alpha = 1.0;
    sc->atol2 = atol2;
    sc->rtol2 = rtol2;
    sc->cg_done = 0;
    sc->admm_done = 0;
    sc->step_active = 0;
    sc->step_pending = 0;
    sc->tau_next = 0.0;
    bar[0] = 0u;  // a barrier that ran out of time may have left arrivals counted
}

int ew_blocks(size_t n) { return (int)std::max<size_t>(1, std::min<size_t>(kEwMaxBlocks, (n + kEwThreads - 1) / kEwThreads)); }

Operand operand_of(const mri_plan *p) {
    Operand op;
    op.hi = (uint32_t *)p->bfwd_hi;
    op.lo = (uint32_t *)p->bfwd_lo;
    op.t32 = (uint2 *)p->bfwd_t;
    op.fp32 = p->bsx;
    op.ny_pad = p->ny_pad;
    op.kx2 = p->kx / 2;
    return op;
}

constexpr int kStageBytes = 48 * 1024;  // target size of one shared-memory stage

Partials partials_of(const mri_plan *p) {
    Partials P;
    P.part = p->part;
    P.ksplit = p->ksplit;
    P.nc = p->nc;
    P.nx = p->nx;
    P.ny = p->ny;
    P.n_ig = p->nx_pad / 64;
    P.mapsT = p->mapsT;
    P.chunk = (p->ksplit + 1) * 64;
    P.cs = std::max(1, std::min(std::min(p->nc, kRedGroups), kStageBytes / (P.chunk * (int)sizeof(float2))));
    P.n_groups = ceil_div(p->nc, P.cs);
    P.stage_elems = std::max(P.cs * P.chunk, kMinStageElems);
    return P;
}

// Dynamic shared memory of the staged kernels: the ring and its barriers.
size_t ring_bytes(const Partials &P) {
    return (size_t)kRingStages * P.stage_elems * sizeof(float2) + kRingStages * sizeof(uint64_t);
}

template <typename Kern>
cudaError_t allow_smem(Kern kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

int operand_mode(const mri_plan *p) {
    return p->precision == MRI_BF16X3 ? kOpBf16x3 : p->precision == MRI_TF32 ? kOpTf32 : kOpFp32;
}

template <int kMode>
CgArgs cg_args(mri_plan *p, float half_beta, int it) {
    CgArgs A;
    A.P = partials_of(p);
    A.x = p->x;
    // cg_init leaves the first residual and direction in p->r and p->d
    A.r = (it & 1) ? p->r2 : p->r;
    A.r_next = (it & 1) ? p->r : p->r2;
    A.d = (it & 1) ? p->d2 : p->d;
    A.d_next = (it & 1) ? p->d : p->d2;
    A.ad = p->ad;
    A.half_beta = half_beta;
    A.op = operand_of(p);
    A.sc = p->scal;
    A.partials = p->partials;
    A.bar = p->grid_bar;
    A.n_items = A.P.n_ig * p->ny;
    return A;
}

template <int kMode>
cudaError_t launch_cg_step_t(mri_plan *p, float half_beta, int it, cudaStream_t s) {
    const CgArgs A = cg_args<kMode>(p, half_beta, it);
    const size_t smem = ring_bytes(A.P);
    cudaError_t e = allow_smem(cg_step_kernel<kMode>, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(p->cg_grid);
    cfg.blockDim = dim3(kRedThreadsX, kRedGroups);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, cg_step_kernel<kMode>, A);
}

template <int kMode>
cudaError_t launch_cg_step_split_t(mri_plan *p, float half_beta, int it, cudaStream_t s) {
    const CgArgs A = cg_args<kMode>(p, half_beta, it);
    const size_t smem = ring_bytes(A.P);
    cudaError_t e = allow_smem(cg_reduce_kernel<kMode>, smem);
    if (e != cudaSuccess) return e;
    cg_reduce_kernel<kMode><<<A.n_items, dim3(kRedThreadsX, kRedGroups), smem, s>>>(A);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cg_update_kernel<kMode><<<ew_blocks((size_t)p->nx * p->ny * p->nc), kEwThreads, 0, s>>>(A);
    return cudaGetLastError();
}

}  // namespace

int cg_step_grid(const mri_plan *p) {
    int per_sm = 0;
    const void *fn = p->precision == MRI_BF16X3  ? (const void *)cg_step_kernel<kOpBf16x3>
                     : p->precision == MRI_TF32 ? (const void *)cg_step_kernel<kOpTf32>
                                                : (const void *)cg_step_kernel<kOpFp32>;
    const size_t smem = ring_bytes(partials_of(p));
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kRedThreads, smem) != cudaSuccess || per_sm <= 0) {
        cudaGetLastError();
        per_sm = 1;
    }
    const long items = (long)(p->nx_pad / 64) * p->ny;
    const long pix_blocks = ((long)p->nx * p->ny + kRedThreads - 1) / kRedThreads;
    const long want = std::max(items, pix_blocks);
    return (int)std::max(1L, std::min<long>((long)per_sm * p->num_sms, want));
}

cudaError_t launch_transpose(const float2 *src, float2 *dst, int rows, int cols, int planes, cudaStream_t s,
                             int ld_dst) {
    dim3 grid(ceil_div(cols, 32), ceil_div(rows, 32), planes);
    transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(src, dst, rows, cols, ld_dst > 0 ? ld_dst : rows);
    return cudaGetLastError();
}

cudaError_t launch_admm_reset(mri_plan *p, double atol, double rtol, cudaStream_t s) {
    admm_reset_kernel<<<1, 1, 0, s>>>(p->scal, p->grid_bar, atol * atol, rtol * rtol);
    return cudaGetLastError();
}

cudaError_t launch_fhd(mri_plan *p, cudaStream_t s) {
    const Partials P = partials_of(p);
    const size_t smem = ring_bytes(P);
    cudaError_t e = allow_smem(fhd_kernel, smem);
    if (e != cudaSuccess) return e;
    fhd_kernel<<<(p->nx_pad / 64) * p->ny, dim3(kRedThreadsX, kRedGroups), smem, s>>>(P, p->fhd, &p->scal->status);
    return cudaGetLastError();
}

cudaError_t launch_mu_rhs(mri_plan *p, float thresh, float half_beta, cudaStream_t s) {
    const size_t npix = (size_t)p->nx * p->ny;
    const int grid = ew_blocks(npix * p->nc);
    const Operand op = operand_of(p);
    switch (operand_mode(p)) {
    case kOpBf16x3:
        mu_rhs_kernel<kOpBf16x3><<<grid, kEwThreads, 0, s>>>(p->nx, p->ny, p->x, p->eta, p->fhd, p->mu, p->b, p->xprev,
                                                              thresh, half_beta, p->mapsT, p->nx_pad, p->nc, op, p->scal);
        break;
    case kOpTf32:
        mu_rhs_kernel<kOpTf32><<<grid, kEwThreads, 0, s>>>(p->nx, p->ny, p->x, p->eta, p->fhd, p->mu, p->b, p->xprev,
                                                            thresh, half_beta, p->mapsT, p->nx_pad, p->nc, op, p->scal);
        break;
    default:
        mu_rhs_kernel<kOpFp32><<<grid, kEwThreads, 0, s>>>(p->nx, p->ny, p->x, p->eta, p->fhd, p->mu, p->b, p->xprev,
                                                            thresh, half_beta, p->mapsT, p->nx_pad, p->nc, op, p->scal);
    }
    return cudaGetLastError();
}

template <int kMode>
cudaError_t launch_cg_init_t(mri_plan *p, float half_beta, cudaStream_t s) {
    const Partials P = partials_of(p);
    const size_t smem = ring_bytes(P);
    cudaError_t e = allow_smem(cg_init_kernel<kMode>, smem);
    if (e != cudaSuccess) return e;
    cg_init_kernel<kMode><<<(p->nx_pad / 64) * p->ny, dim3(kRedThreadsX, kRedGroups), smem, s>>>(
        P, p->x, p->b, half_beta, p->r, p->d, operand_of(p), p->scal, p->partials);
    return cudaGetLastError();
}

cudaError_t launch_cg_init(mri_plan *p, float half_beta, cudaStream_t s) {
    switch (operand_mode(p)) {
    case kOpBf16x3:
        return launch_cg_init_t<kOpBf16x3>(p, half_beta, s);
    case kOpTf32:
        return launch_cg_init_t<kOpTf32>(p, half_beta, s);
    default:
        return launch_cg_init_t<kOpFp32>(p, half_beta, s);
    }
}

cudaError_t launch_cg_step(mri_plan *p, float half_beta, int it, cudaStream_t s) {
    switch (operand_mode(p)) {
    case kOpBf16x3:
        return launch_cg_step_t<kOpBf16x3>(p, half_beta, it, s);
    case kOpTf32:
        return launch_cg_step_t<kOpTf32>(p, half_beta, it, s);
    default:
        return launch_cg_step_t<kOpFp32>(p, half_beta, it, s);
    }
}

cudaError_t launch_cg_step_split(mri_plan *p, float half_beta, int it, cudaStream_t s) {
    switch (operand_mode(p)) {
    case kOpBf16x3:
        return launch_cg_step_split_t<kOpBf16x3>(p, half_beta, it, s);
    case kOpTf32:
        return launch_cg_step_split_t<kOpTf32>(p, half_beta, it, s);
    default:
        return launch_cg_step_split_t<kOpFp32>(p, half_beta, it, s);
    }
}

cudaError_t launch_dual(mri_plan *p, bool operand, double *alpha_hist, int m, cudaStream_t s) {
    const size_t npix = (size_t)p->nx * p->ny;
    const int grid = ew_blocks(operand ? npix * p->nc : npix);
    const Operand op = operand_of(p);
    switch (operand_mode(p)) {
    case kOpBf16x3:
        dual_kernel<kOpBf16x3><<<grid, kEwThreads, 0, s>>>(p->nx, p->ny, p->x, p->xprev, p->mu, p->eta, p->mapsT,
                                                           p->nx_pad, p->nc, op, operand ? 1 : 0, p->scal, p->partials, alpha_hist, m);
        break;
    case kOpTf32:
        dual_kernel<kOpTf32><<<grid, kEwThreads, 0, s>>>(p->nx, p->ny, p->x, p->xprev, p->mu, p->eta, p->mapsT, p->nx_pad,
                                                         p->nc, op, operand ? 1 : 0, p->scal, p->partials, alpha_hist, m);
        break;
    default:
        dual_kernel<kOpFp32><<<grid, kEwThreads, 0, s>>>(p->nx, p->ny, p->x, p->xprev, p->mu, p->eta, p->mapsT, p->nx_pad,
                                                         p->nc, op, operand ? 1 : 0, p->scal, p->partials, alpha_hist, m);
    }
    return cudaGetLastError();
}

cudaError_t launch_objective(mri_plan *p, const float2 *kspace, float lambda, double *obj_hist, int m,
                             cudaStream_t s) {
    const size_t npix = (size_t)p->nx * p->ny;
    const int nkc = p->nk * p->nc;
    objective_kernel<<<ew_blocks(std::max<size_t>(npix, (size_t)nkc)), kEwThreads, 0, s>>>(
        p->nx, p->ny, p->nk, nkc, p->y, p->nk_pad, kspace, p->x, lambda, p->scal, p->partials, obj_hist, m);
    return cudaGetLastError();
}

}  // namespace mri
