// C-ABI entry points of libmrirecon: argument checks, plan and workspace
// management, and the host-side sequencing of the reconstruction (Alg. 4 with
// Alg. 2 inside), all enqueued on the caller's stream without synchronising.
#include <atomic>
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <string>

#include "common.cuh"
#include "internal.h"

namespace mri {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

void invalidate_graph(mri_plan *p) {
    p->config_gen += 1;
    if (p->graph_exec) {
        cudaGraphExecDestroy(p->graph_exec);
        p->graph_exec = nullptr;
    }
    p->graph_launches = 0;
}

namespace {

int fail(int code, const std::string &msg) {
    set_error(msg);
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(MRI_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define MRI_CUDA_TRY(expr)                                  \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) return cuda_fail(_e, #expr); \
    } while (0)

template <typename T>
int dev_alloc(mri_plan *p, T **ptr, size_t count) {
    if (count == 0) {
        *ptr = nullptr;
        return MRI_OK;
    }
    cudaError_t e = p->pool ? cudaMallocFromPoolAsync((void **)ptr, count * sizeof(T), p->pool, p->pool_stream)
                            : cudaMalloc((void **)ptr, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return fail(MRI_ERR_NOMEM, std::string("device allocation of ") + std::to_string(count * sizeof(T)) +
                                       " bytes failed: " + cudaGetErrorString(e));
    }
    p->bytes += count * sizeof(T);
    return MRI_OK;
}

// Frees everything the plan owns; pool-allocated plans free stream-ordered on
// free_stream (the caller guarantees no work on the plan is still pending).
void free_plan(mri_plan *p, cudaStream_t free_stream = nullptr) {
    if (!p) return;
    invalidate_graph(p);
    void *bufs[] = {p->ax,      p->ay,      p->axT,     p->axP,    p->axQ,      p->ayT,  p->afwd_hi,
                    p->afwd_lo, p->badj_hi, p->badj_lo, p->bfwd_hi, p->bfwd_lo, p->afwd_t, p->badj_t,
                    p->bfwd_t,  p->bsx,     p->y,       p->part,   p->x,        p->xprev, p->r,
                    p->d,       p->ad,      p->b,       p->fhd,    p->mu,       p->eta,   p->partials,
                    p->scal,    p->mapsT,   p->grid_bar, p->d2,  p->r2};
    for (void *q : bufs)
        if (q) {
            if (p->pool)
                cudaFreeAsync(q, free_stream);
            else
                cudaFree(q);
        }
    for (cudaEvent_t e : p->ev_free) cudaEventDestroy(e);
    for (auto *list : {&p->ev_fwd, &p->ev_adj, &p->ev_red})
        for (auto &pr : *list) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
    delete p;
}

// Number of k-space splits of the adjoint product: enough independent work
// units to fill the GPU a few times, chosen from the problem's own shape and
// the SM count only (so a reconstruction is computed identically alone or
// alongside others).
int choose_ksplit_fp32(const mri_plan *p, int *samples_per_split) {
    const int tiles = ceil_div(p->nx, 64) * ceil_div(p->ny, 64) * p->nc;
    const int slots = adj_fp32_slots(p->num_sms);
    // at most 4096 samples summed in one FP32 run (rounding error of a
    // sequential FP32 sum of L random-phase terms grows like 2^-24 sqrt(L)),
    // at least 256 (or the whole trajectory) per split, at most 64 splits;
    // among those, the split count whose blocks take the fewest sample
    // sweeps in waves of `slots` blocks (makespan = waves x samples per
    // split), the smallest count on ties
    const int lo = std::min(64, std::max(1, ceil_div(p->nk, 4096)));
    const int hi = std::max(lo, std::min(64, ceil_div(p->nk, 256)));
    long best_cost = -1;
    int best = lo;
    for (int split = lo; split <= hi; ++split) {
        const int per = round_up(ceil_div(p->nk, split), 16);
        const int eff = ceil_div(p->nk, per);
        const long cost = (long)ceil_div(tiles * eff, slots) * per;
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = eff;
        }
    }
    const int per = round_up(ceil_div(p->nk, best), 16);
    *samples_per_split = per;
    return ceil_div(p->nk, per);
}

bool finite(float v) { return isfinite(v) != 0; }

}  // namespace

// ---------------------------------------------------------------------------
// operator sequences shared by the entry points
// ---------------------------------------------------------------------------
// Take a pair of timing events from the plan's pool (creating them as needed).
static bool timing_arm(mri_plan *p) {
    if (!p->timing) return false;
    cudaEvent_t ev[2];
    for (int q = 0; q < 2; ++q) {
        if (!p->ev_free.empty()) {
            ev[q] = p->ev_free.back();
            p->ev_free.pop_back();
        } else if (cudaEventCreate(&ev[q]) != cudaSuccess) {
            cudaGetLastError();
            if (q == 1) p->ev_free.push_back(ev[0]);
            return false;
        }
    }
    p->t_ev0 = ev[0];
    p->t_ev1 = ev[1];
    return true;
}

static void timing_disarm(mri_plan *p, std::vector<std::pair<cudaEvent_t, cudaEvent_t>> &list) {
    list.emplace_back(p->t_ev0, p->t_ev1);
    p->t_ev0 = p->t_ev1 = nullptr;
}

// out[c * ld + k] = (F image)_c[k]
static cudaError_t op_forward(mri_plan *p, const float2 *image, const float2 *maps, float2 *out, int ld, int skip,
                              cudaStream_t s) {
    const bool timed = timing_arm(p);
    cudaError_t e = is_tc_precision(p->precision) ? launch_fwd_tc(p, image, maps, out, ld, skip, s)
                                                  : launch_fwd_fp32(p, image, maps, out, ld, skip, s);
    if (timed) timing_disarm(p, p->ev_fwd);
    return e;
}

// Partial images of F^H kspace; kspace is [nc][nk] unless it is the plan's
// own padded workspace y, into which any other input is copied first.
static cudaError_t op_adjoint_partials(mri_plan *p, const float2 *kspace, int skip, cudaStream_t s) {
    if (kspace != p->y) {
        cudaError_t e = cudaMemcpy2DAsync(p->y, (size_t)p->nk_pad * sizeof(float2), kspace,
                                          (size_t)p->nk * sizeof(float2), (size_t)p->nk * sizeof(float2), p->nc,
                                          cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    const bool timed = timing_arm(p);
    cudaError_t e = is_tc_precision(p->precision) ? launch_adj_tc(p, skip, s) : launch_adj_fp32(p, skip, s);
    if (timed) timing_disarm(p, p->ev_adj);
    return e;
}

// out = F^H F src (+ half_beta Theta^H Theta src) (+ CG dot)
static cudaError_t op_normal(mri_plan *p, const float2 *src, const float2 *maps, float2 *out, float half_beta,
                             bool cg_dot, int skip, cudaStream_t s) {
    cudaError_t e = op_forward(p, src, maps, p->y, p->nk_pad, skip, s);
    if (e != cudaSuccess) return e;
    e = op_adjoint_partials(p, p->y, skip, s);
    if (e != cudaSuccess) return e;
    ReduceEpilogue ep;
    ep.tv_src = half_beta != 0.f ? src : nullptr;
    ep.half_beta = half_beta;
    ep.dot_src = cg_dot ? src : nullptr;
    ep.skip = skip;
    p->launches += 1;
    const bool timed = timing_arm(p);
    if (timed) cudaEventRecord(p->t_ev0, s);
    e = launch_adj_reduce(p, maps, out, ep, s);
    if (timed) {
        cudaEventRecord(p->t_ev1, s);
        timing_disarm(p, p->ev_red);
    }
    return e;
}

// The solver's forward product of the operand it has written (no operand kernel).
static cudaError_t solver_forward(mri_plan *p, int skip, cudaStream_t s) {
    const bool timed = timing_arm(p);
    cudaError_t e = is_tc_precision(p->precision) ? launch_fwd_tc(p, nullptr, nullptr, p->y, p->nk_pad, skip, s)
                                                  : launch_fwd_fp32(p, nullptr, nullptr, p->y, p->nk_pad, skip, s);
    if (timed) timing_disarm(p, p->ev_fwd);
    return e;
}

// One fused CG step (finishes the adjoint, then Alg. 2's updates); timed
// with the reductions.
static cudaError_t solver_cg_step(mri_plan *p, float half_beta, int it, cudaStream_t s) {
    const bool timed = timing_arm(p);
    if (timed) cudaEventRecord(p->t_ev0, s);
    cudaError_t e = launch_cg_step(p, half_beta, it, s);
    p->launches += 1;
    if (timed) {
        cudaEventRecord(p->t_ev1, s);
        timing_disarm(p, p->ev_red);
    }
    return e;
}

}  // namespace mri

using namespace mri;

extern "C" {

MRI_API const char *mri_last_error(void) { return g_last_error.c_str(); }

MRI_API int mri_version(void) { return 100; }

}  // extern "C"

namespace mri {

int plan_create(mri_plan **out, int nx, int ny, int nk, int nc, const float *traj, int precision,
                cudaStream_t stream, cudaMemPool_t pool) {
    if (!out) return fail(MRI_ERR_INVALID, "plan output pointer is null");
    *out = nullptr;
    if (nx <= 0 || ny <= 0 || nk <= 0 || nc <= 0) return fail(MRI_ERR_INVALID, "dimensions must be positive");
    if ((long long)nx * ny > (1LL << 26) || nk > (1 << 28) || nc > 4096)
        return fail(MRI_ERR_INVALID, "dimensions too large");
    if (!traj) return fail(MRI_ERR_INVALID, "trajectory pointer is null");
    if (precision != MRI_FP32 && !is_tc_precision(precision)) return fail(MRI_ERR_INVALID, "unknown precision");
    cudaStream_t s = (cudaStream_t)stream;

    static std::atomic<uint64_t> next_serial{1};
    mri_plan *p = new mri_plan();
    p->serial = next_serial.fetch_add(1);
    p->pool = pool;
    p->pool_stream = s;
    p->nx = nx;
    p->ny = ny;
    p->nk = nk;
    p->nc = nc;
    p->precision = precision;
    {
        cudaError_t e0 = cudaGetDevice(&p->device);
        if (e0 == cudaSuccess) e0 = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
        if (e0 != cudaSuccess) {
            delete p;
            return cuda_fail(e0, "device query");
        }
    }
    p->nx_pad = round_up(nx, 64);
    // UMMA N granularity; an image wider than one UMMA (256) is processed in
    // column parts of 256
    p->ny_pad = ny <= 256 ? round_up(ny, 16) : round_up(ny, 256);
    p->kx = round_up(2 * nx, 64);
    p->kk = round_up(2 * nk, 64);
    p->nk_pad = round_up(nk, 32);

    int rc = MRI_OK;
    const size_t npix = (size_t)nx * ny;
    if (is_tc_precision(precision)) {
        const std::string form = precision == MRI_TF32 ? "TF32" : "BF16x3";
        std::string why;
        if (!tc_supported(p, &why)) {
            delete p;
            return fail(MRI_ERR_UNSUPPORTED, form + " tensor-core path: " + why);
        }
        rc = tc_plan_tiling(p);
        if (rc != MRI_OK) {
            delete p;
            return fail(rc, form + " tensor-core path: shared-memory plan does not fit");
        }
        if (p->adj_tile_px == 128) {
            if (rc == MRI_OK) rc = dev_alloc(p, &p->axP, (size_t)(p->nx_pad / 16) * p->nk_pad);
            if (rc == MRI_OK) rc = dev_alloc(p, &p->axQ, (size_t)16 * p->nk_pad);
        } else {
            if (rc == MRI_OK) rc = dev_alloc(p, &p->axT, (size_t)nx * p->nk_pad);
        }
        if (rc == MRI_OK) rc = dev_alloc(p, &p->ayT, (size_t)ny * p->nk_pad);
        if (precision == MRI_TF32) {
            if (rc == MRI_OK) rc = dev_alloc(p, &p->afwd_t, (size_t)2 * nk * p->kx);
            if (rc == MRI_OK) rc = dev_alloc(p, &p->badj_t, (size_t)p->badj_rows * p->kk);
            if (rc == MRI_OK) rc = dev_alloc(p, &p->bfwd_t, (size_t)nc * p->ny_pad * p->kx);
        } else {
            if (rc == MRI_OK) rc = dev_alloc(p, &p->afwd_hi, (size_t)2 * nk * p->kx);
            if (rc == MRI_OK) rc = dev_alloc(p, &p->afwd_lo, (size_t)2 * nk * p->kx);
            if (rc == MRI_OK) rc = dev_alloc(p, &p->badj_hi, (size_t)p->badj_rows * p->kk);
            if (rc == MRI_OK) rc = dev_alloc(p, &p->badj_lo, (size_t)p->badj_rows * p->kk);
            if (rc == MRI_OK) rc = dev_alloc(p, &p->bfwd_hi, (size_t)nc * p->ny_pad * p->kx);
            if (rc == MRI_OK) rc = dev_alloc(p, &p->bfwd_lo, (size_t)nc * p->ny_pad * p->kx);
        }
    } else {
        int per = 0;
        p->ksplit = choose_ksplit_fp32(p, &per);
        p->ksplit_blocks = per;
        if (rc == MRI_OK) rc = dev_alloc(p, &p->ax, (size_t)nk * nx);
        if (rc == MRI_OK) rc = dev_alloc(p, &p->ay, (size_t)nk * ny);
        if (rc == MRI_OK) rc = dev_alloc(p, &p->bsx, (size_t)nc * npix);
    }
    if (rc == MRI_OK) rc = dev_alloc(p, &p->y, (size_t)nc * p->nk_pad);
    if (rc == MRI_OK) rc = dev_alloc(p, &p->part, (size_t)p->ksplit * nc * ny * p->nx_pad);
    float2 **img_bufs[] = {&p->x, &p->xprev, &p->r, &p->r2, &p->d, &p->d2, &p->ad, &p->b, &p->fhd};
    for (float2 **q : img_bufs)
        if (rc == MRI_OK) rc = dev_alloc(p, q, npix);
    if (rc == MRI_OK) rc = dev_alloc(p, &p->mu, 2 * npix);
    if (rc == MRI_OK) rc = dev_alloc(p, &p->eta, 2 * npix);
    if (rc == MRI_OK) rc = dev_alloc(p, &p->mapsT, (size_t)nc * ny * p->nx_pad);
    if (rc == MRI_OK) rc = dev_alloc(p, &p->grid_bar, 2);
    // one slot pair per block of the largest reducing grid (element-wise
    // kernels use at most 1024 blocks, the adjoint reduction one per 32x32 tile)
    p->partials_cap = 3 * std::max(1024, ceil_div(nx, 32) * ny);
    if (rc == MRI_OK) rc = dev_alloc(p, &p->partials, (size_t)p->partials_cap);
    if (rc == MRI_OK) rc = dev_alloc(p, &p->scal, 1);
    if (rc != MRI_OK) {
        free_plan(p);
        return rc;
    }
    // zero padding of the tensor-core operands must stay zero
    cudaError_t e = cudaSuccess;
    if (precision == MRI_BF16X3) {
        __nv_bfloat16 *zb[] = {p->afwd_hi, p->afwd_lo, p->badj_hi, p->badj_lo, p->bfwd_hi, p->bfwd_lo};
        size_t zn[] = {(size_t)2 * nk * p->kx, (size_t)2 * nk * p->kx, (size_t)p->badj_rows * p->kk,
                       (size_t)p->badj_rows * p->kk, (size_t)nc * p->ny_pad * p->kx, (size_t)nc * p->ny_pad * p->kx};
        for (int q = 0; q < 6 && e == cudaSuccess; ++q) e = cudaMemsetAsync(zb[q], 0, zn[q] * 2, s);
    } else if (precision == MRI_TF32) {
        float *zt[] = {p->afwd_t, p->badj_t, p->bfwd_t};
        size_t zn[] = {(size_t)2 * nk * p->kx, (size_t)p->badj_rows * p->kk, (size_t)nc * p->ny_pad * p->kx};
        for (int q = 0; q < 3 && e == cudaSuccess; ++q) e = cudaMemsetAsync(zt[q], 0, zn[q] * 4, s);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(p->part, 0, (size_t)p->ksplit * nc * ny * p->nx_pad * 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->y, 0, (size_t)nc * p->nk_pad * 8, s);
    if (e == cudaSuccess && p->axT) e = cudaMemsetAsync(p->axT, 0, (size_t)nx * p->nk_pad * 8, s);
    if (e == cudaSuccess && p->axP) e = cudaMemsetAsync(p->axP, 0, (size_t)(p->nx_pad / 16) * p->nk_pad * 8, s);
    if (e == cudaSuccess && p->axQ) e = cudaMemsetAsync(p->axQ, 0, (size_t)16 * p->nk_pad * 8, s);
    if (e == cudaSuccess && p->ayT) e = cudaMemsetAsync(p->ayT, 0, (size_t)ny * p->nk_pad * 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->scal, 0, sizeof(DevScalars), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->grid_bar, 0, 2 * sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->mapsT, 0, (size_t)nc * ny * p->nx_pad * sizeof(float2), s);
    p->cg_grid = cg_step_grid(p);
    if (e == cudaSuccess && is_tc_precision(precision)) {
        rc = tc_make_tensor_maps(p);
        int cpt = 0, fs = 0, as = 0;
        // the tile configuration an earlier autotune chose for this shape, if valid here
        if (rc == MRI_OK && tuning_lookup(p, &cpt, &fs, &as) && tc_tiles_valid(p, cpt, fs, as))
            rc = tc_set_tiles(p, cpt, fs, as);
        if (rc != MRI_OK) {
            free_plan(p);
            return rc;
        }
    }
    if (e == cudaSuccess) e = launch_factors(p, traj, s);
    if (e != cudaSuccess) {
        free_plan(p);
        return cuda_fail(e, "plan initialisation");
    }
    *out = p;
    return MRI_OK;
}

void plan_destroy_async(mri_plan *p, cudaStream_t s) { free_plan(p, s); }

}  // namespace mri

extern "C" {

MRI_API int mri_plan_create(mri_plan **out, int nx, int ny, int nk, int nc, const float *traj, int precision,
                            mri_stream_t stream) {
    NvtxRange range("mri_plan_create");
    return plan_create(out, nx, ny, nk, nc, traj, precision, (cudaStream_t)stream, nullptr);
}

MRI_API int mri_plan_set_trajectory(mri_plan *p, const float *traj, mri_stream_t stream) {
    if (!p || !traj) return fail(MRI_ERR_INVALID, "null plan or trajectory");
    cudaError_t e = launch_factors(p, traj, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "factor generation");
    return MRI_OK;
}

MRI_API int mri_plan_destroy(mri_plan *p) {
    if (!p) return MRI_OK;
    cudaDeviceSynchronize();
    free_plan(p);
    return MRI_OK;
}

MRI_API int mri_plan_sync_status(mri_plan *p, mri_stream_t stream) {
    if (!p) return fail(MRI_ERR_INVALID, "null plan");
    MRI_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    int status = 0;
    MRI_CUDA_TRY(cudaMemcpy(&status, &p->scal->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status != kStatusOk) {
        int zero = 0;
        MRI_CUDA_TRY(cudaMemcpy(&p->scal->status, &zero, sizeof(int), cudaMemcpyHostToDevice));
        return fail(MRI_ERR_TIMEOUT, "a bounded device-side wait gave up (status " + std::to_string(status) + ")");
    }
    return MRI_OK;
}

MRI_API size_t mri_plan_device_bytes(const mri_plan *p) { return p ? p->bytes : 0; }

// Mirrors the allocations of mri_plan_create without allocating.
MRI_API size_t mri_plan_estimate_bytes(int nx, int ny, int nk, int nc, int precision) {
    if (nx <= 0 || ny <= 0 || nk <= 0 || nc <= 0) return 0;
    if (precision != MRI_FP32 && !is_tc_precision(precision)) return 0;
    mri_plan t;
    t.nx = nx;
    t.ny = ny;
    t.nk = nk;
    t.nc = nc;
    t.precision = precision;
    if (cudaGetDevice(&t.device) != cudaSuccess ||
        cudaDeviceGetAttribute(&t.num_sms, cudaDevAttrMultiProcessorCount, t.device) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    t.nx_pad = round_up(nx, 64);
    t.ny_pad = ny <= 256 ? round_up(ny, 16) : round_up(ny, 256);
    t.kx = round_up(2 * nx, 64);
    t.kk = round_up(2 * nk, 64);
    t.nk_pad = round_up(nk, 32);
    const size_t npix = (size_t)nx * ny, c64 = sizeof(float2), bf = 2;
    size_t bytes = 0;
    if (is_tc_precision(precision)) {
        // BF16x3 hi + lo (2 + 2 bytes) and TF32 (4 bytes) operands take the same bytes
        if (tc_plan_tiling(&t) != MRI_OK) return 0;
        const size_t ax_rows = t.adj_tile_px == 128 ? (size_t)t.nx_pad / 16 + 16 : (size_t)nx;
        bytes += c64 * (ax_rows * t.nk_pad + (size_t)ny * t.nk_pad);
        bytes += bf * (2 * (size_t)2 * nk * t.kx + 2 * (size_t)t.badj_rows * t.kk + 2 * (size_t)nc * t.ny_pad * t.kx);
    } else {
        int per = 0;
        t.ksplit = choose_ksplit_fp32(&t, &per);
        bytes += c64 * ((size_t)nk * nx + (size_t)nk * ny + (size_t)nc * npix);
    }
    bytes += c64 * ((size_t)nc * t.nk_pad + (size_t)t.ksplit * nc * ny * t.nx_pad + 9 * npix + 4 * npix +
                    (size_t)nc * ny * t.nx_pad);
    bytes += 2 * sizeof(unsigned);
    bytes += sizeof(double) * (size_t)(3 * std::max(1024, ceil_div(nx, 32) * ny));
    bytes += sizeof(DevScalars);
    return bytes;
}

MRI_API int mri_nudft_forward(mri_plan *p, const mri_c64 *image, const mri_c64 *maps, mri_c64 *kspace,
                              mri_stream_t stream) {
    NvtxRange range("mri_nudft_forward");
    if (!p || !image || !maps || !kspace) return fail(MRI_ERR_INVALID, "null argument");
    cudaError_t e = op_forward(p, (const float2 *)image, (const float2 *)maps, (float2 *)kspace, p->nk, kSkipNever,
                               (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "forward operator");
    return MRI_OK;
}

MRI_API int mri_nudft_adjoint(mri_plan *p, const mri_c64 *kspace, const mri_c64 *maps, mri_c64 *image,
                              mri_stream_t stream) {
    NvtxRange range("mri_nudft_adjoint");
    if (!p || !image || !maps || !kspace) return fail(MRI_ERR_INVALID, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = op_adjoint_partials(p, (const float2 *)kspace, kSkipNever, s);
    if (e == cudaSuccess) e = launch_adj_reduce(p, (const float2 *)maps, (float2 *)image, ReduceEpilogue(), s);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint operator");
    return MRI_OK;
}

MRI_API int mri_normal_op(mri_plan *p, const mri_c64 *image, const mri_c64 *maps, float beta, mri_c64 *out,
                          mri_stream_t stream) {
    NvtxRange range("mri_normal_op");
    if (!p || !image || !maps || !out) return fail(MRI_ERR_INVALID, "null argument");
    if (!finite(beta) || beta < 0.f) return fail(MRI_ERR_INVALID, "beta must be finite and >= 0");
    if ((const void *)image == (const void *)out) return fail(MRI_ERR_INVALID, "image and out must differ");
    cudaError_t e = op_normal(p, (const float2 *)image, (const float2 *)maps, (float2 *)out, 0.5f * beta, false,
                              kSkipNever, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "normal operator");
    return MRI_OK;
}

MRI_API int mri_tv_forward(int nx, int ny, const mri_c64 *image, mri_c64 *grad, mri_stream_t stream) {
    if (nx <= 0 || ny <= 0 || !image || !grad) return fail(MRI_ERR_INVALID, "bad argument");
    cudaError_t e = launch_tv_forward(nx, ny, (const float2 *)image, (float2 *)grad, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "tv_forward");
    return MRI_OK;
}

MRI_API int mri_tv_adjoint(int nx, int ny, const mri_c64 *grad, mri_c64 *image, mri_stream_t stream) {
    if (nx <= 0 || ny <= 0 || !image || !grad) return fail(MRI_ERR_INVALID, "bad argument");
    cudaError_t e = launch_tv_adjoint(nx, ny, (const float2 *)grad, (float2 *)image, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "tv_adjoint");
    return MRI_OK;
}

MRI_API int mri_soft_threshold(int n, float t, const mri_c64 *in, mri_c64 *out, mri_stream_t stream) {
    if (n < 0 || !in || !out || !finite(t) || t < 0.f) return fail(MRI_ERR_INVALID, "bad argument");
    if (n == 0) return MRI_OK;
    cudaError_t e = launch_shrink(n, t, (const float2 *)in, (float2 *)out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "soft_threshold");
    return MRI_OK;
}

}  // extern "C"

// Enqueue the whole reconstruction (Alg. 4 with Alg. 2) on s.  The solver
// works on the plan's transposed copies of the image-sized state (admm.cu):
// the coil maps and any saved state are transposed in first, the image and
// the final dual variable out at the end.  Per CG step: the forward product
// (its operand written by the kernel before it), the adjoint product, and
// one cooperative kernel that finishes the adjoint and takes the CG step.
int mri::enqueue_admm(mri_plan *p, const mri_c64 *kspace_in, const mri_c64 *maps_in, const mri_admm_params *prm,
                      mri_c64 *image_out, double *objective_hist, double *alpha_hist, cudaStream_t s,
                      const AdmmWarm &warm, bool coop) {
    const float2 *kspace = (const float2 *)kspace_in;
    const float2 *maps = (const float2 *)maps_in;
    const size_t npix = (size_t)p->nx * p->ny;
    const float half_beta = 0.5f * prm->beta;
    const float thresh = prm->lambda / prm->beta;

#define STEP(expr)                                                  \
    do {                                                            \
        cudaError_t _e = (expr);                                    \
        if (_e != cudaSuccess) return cuda_fail(_e, "admm: " #expr); \
    } while (0)
#define KERNEL(expr)      \
    do {                  \
        STEP(expr);       \
        p->launches += 1; \
    } while (0)

    KERNEL(launch_admm_reset(p, prm->atol, prm->rtol, s));
    KERNEL(launch_transpose(maps, p->mapsT, p->nx, p->ny, p->nc, s, p->nx_pad));
    // x^0 = 0 and eta^0 = 0 (Alg. 4), or a saved state to resume from
    if (warm.x0)
        KERNEL(launch_transpose((const float2 *)warm.x0, p->x, p->nx, p->ny, 1, s));
    else
        STEP(cudaMemsetAsync(p->x, 0, npix * sizeof(float2), s));
    if (warm.eta0)
        KERNEL(launch_transpose((const float2 *)warm.eta0, p->eta, p->nx, p->ny, 2, s));
    else
        STEP(cudaMemsetAsync(p->eta, 0, 2 * npix * sizeof(float2), s));
    // F^H d, once per reconstruction (Section IV-C: the right-hand side stays
    // fixed through the CG iterations)
    STEP(op_adjoint_partials(p, kspace, kSkipNever, s));
    KERNEL(launch_fhd(p, s));
    for (int m = 0; m < prm->admm_iters; ++m) {
        KERNEL(launch_mu_rhs(p, thresh, half_beta, s));  // Eq. 8 (mu), Eq. 12 (b), operand of x
        // A x0 and the start of Alg. 2
        STEP(solver_forward(p, kSkipAdmm, s));
        STEP(op_adjoint_partials(p, p->y, kSkipAdmm, s));
        KERNEL(launch_cg_init(p, half_beta, s));
        for (int it = 0; it < prm->cg_iters; ++it) {
            STEP(solver_forward(p, kSkipCg, s));                // F d (operand written by the kernel before)
            STEP(op_adjoint_partials(p, p->y, kSkipCg, s));     // F^H F d, partial images
            // A d, alpha, x, r, beta, d, operand of d
            if (coop) {
                STEP(solver_cg_step(p, half_beta, it, s));
            } else {
                STEP(launch_cg_step_split(p, half_beta, it, s));
                p->launches += 2;
            }
        }
        const bool obj = objective_hist != nullptr;
        KERNEL(launch_dual(p, obj, alpha_hist, m, s));  // Eq. 8 (dual), Alg. 4 relative change
        if (obj) {
            STEP(solver_forward(p, kSkipStep, s));
            KERNEL(launch_objective(p, kspace, prm->lambda, objective_hist, m, s));
        }
    }
    KERNEL(launch_transpose(p->x, (float2 *)image_out, p->ny, p->nx, 1, s));
    if (warm.eta_out) KERNEL(launch_transpose(p->eta, (float2 *)warm.eta_out, p->ny, p->nx, 2, s));
#undef KERNEL
#undef STEP
    return MRI_OK;
}

int mri::check_admm_args(const mri_plan *p, const mri_c64 *kspace_in, const mri_c64 *maps_in,
                         const mri_admm_params *prm, const mri_c64 *image_out) {
    if (!p || !kspace_in || !maps_in || !prm || !image_out) return fail(MRI_ERR_INVALID, "null argument");
    if (!finite(prm->lambda) || prm->lambda < 0.f) return fail(MRI_ERR_INVALID, "lambda must be finite and >= 0");
    if (!finite(prm->beta) || !(prm->beta > 0.f)) return fail(MRI_ERR_INVALID, "beta must be finite and > 0");
    if (prm->admm_iters < 0 || prm->cg_iters < 0) return fail(MRI_ERR_INVALID, "iteration counts must be >= 0");
    if (!isfinite(prm->rtol) || prm->rtol < 0 || !isfinite(prm->atol) || prm->atol < 0)
        return fail(MRI_ERR_INVALID, "tolerances must be finite and >= 0");
    return MRI_OK;
}

extern "C" {

}  // extern "C"

// mri_admm_reconstruct, mri_admm_resume and served requests: direct
// launches, or the cached CUDA graph of the whole reconstruction while the
// arguments repeat.
int mri::run_admm(mri_plan *p, const mri_c64 *kspace_in, const mri_c64 *maps_in, const mri_admm_params *prm,
                  mri_c64 *image_out, double *objective_hist, double *alpha_hist, const AdmmWarm &warm,
                  cudaStream_t s, bool coop) {
    const int arc = check_admm_args(p, kspace_in, maps_in, prm, image_out);
    if (arc != MRI_OK) return arc;
    // per-kernel timing events cannot be read back from graph replays, so a
    // timed plan launches its kernels directly
    if (!p->use_graphs || s == nullptr || p->timing)
        return enqueue_admm(p, kspace_in, maps_in, prm, image_out, objective_hist, alpha_hist, s, warm, coop);
    const mri_plan::GraphKey key{kspace_in,  maps_in,   image_out,       objective_hist, alpha_hist,
                                 prm->lambda, prm->beta, prm->admm_iters, prm->cg_iters,  prm->rtol,
                                 prm->atol,   warm.x0,   warm.eta0,       warm.eta_out,   coop};
    if (p->graph_exec && p->graph_key == key) {
        cudaError_t e = cudaGraphLaunch(p->graph_exec, s);
        if (e != cudaSuccess) return cuda_fail(e, "graph launch");
        p->launches += p->graph_launches;
        p->graph_replays += 1;
        return MRI_OK;
    }
    invalidate_graph(p);
    const long long l0 = p->launches;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "graph capture");
    const int rc = enqueue_admm(p, kspace_in, maps_in, prm, image_out, objective_hist, alpha_hist, s, warm, coop);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(s, &graph);
    if (rc != MRI_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        p->launches = l0;
        return rc != MRI_OK ? rc : cuda_fail(e, "graph capture");
    }
    e = cudaGraphInstantiate(&p->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        p->graph_exec = nullptr;
        p->launches = l0;
        return cuda_fail(e, "graph instantiate");
    }
    p->graph_key = key;
    p->graph_launches = p->launches - l0;
    p->graph_captures += 1;
    e = cudaGraphLaunch(p->graph_exec, s);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    return MRI_OK;
}

extern "C" {

MRI_API int mri_admm_reconstruct(mri_plan *p, const mri_c64 *kspace_in, const mri_c64 *maps_in,
                                 const mri_admm_params *prm, mri_c64 *image_out, double *objective_hist,
                                 double *alpha_hist, mri_stream_t stream) {
    NvtxRange range("mri_admm_reconstruct");
    return run_admm(p, kspace_in, maps_in, prm, image_out, objective_hist, alpha_hist, AdmmWarm(),
                    (cudaStream_t)stream);
}

MRI_API int mri_admm_resume(mri_plan *p, const mri_c64 *kspace, const mri_c64 *maps, const mri_admm_params *prm,
                            const mri_c64 *x0, const mri_c64 *eta0, mri_c64 *image_out, mri_c64 *eta_out,
                            double *objective_hist, double *alpha_hist, mri_stream_t stream) {
    NvtxRange range("mri_admm_resume");
    AdmmWarm warm;
    warm.x0 = x0;
    warm.eta0 = eta0;
    warm.eta_out = eta_out;
    if (eta_out && (eta_out == eta0 || (const void *)eta_out == (const void *)x0))
        return fail(MRI_ERR_INVALID, "eta_out must not alias x0 or eta0");
    return run_admm(p, kspace, maps, prm, image_out, objective_hist, alpha_hist, warm, (cudaStream_t)stream);
}

MRI_API int mri_plan_set_graphs(mri_plan *p, int enable) {
    if (!p) return fail(MRI_ERR_INVALID, "null plan");
    p->use_graphs = enable != 0;
    if (!p->use_graphs) invalidate_graph(p);
    return MRI_OK;
}

MRI_API int mri_plan_set_timing(mri_plan *p, int enable) {
    if (!p) return fail(MRI_ERR_INVALID, "null plan");
    p->timing = enable != 0;
    return MRI_OK;
}

MRI_API int mri_plan_read_timing(mri_plan *p, double *fwd_ms, long long *fwd_launches, double *adj_ms,
                                 long long *adj_launches, double *red_ms, long long *red_launches) {
    if (!p) return fail(MRI_ERR_INVALID, "null plan");
    double sums[3] = {0.0, 0.0, 0.0};
    long long counts[3] = {0, 0, 0};
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> *lists[3] = {&p->ev_fwd, &p->ev_adj, &p->ev_red};
    for (int q = 0; q < 3; ++q) {
        for (auto &pr : *lists[q]) {
            float ms = 0.f;
            cudaError_t e = cudaEventSynchronize(pr.second);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, pr.first, pr.second);
            if (e != cudaSuccess) return cuda_fail(e, "read_timing");
            sums[q] += ms;
            counts[q] += 1;
            p->ev_free.push_back(pr.first);
            p->ev_free.push_back(pr.second);
        }
        lists[q]->clear();
    }
    if (fwd_ms) *fwd_ms = sums[0];
    if (fwd_launches) *fwd_launches = counts[0];
    if (adj_ms) *adj_ms = sums[1];
    if (adj_launches) *adj_launches = counts[1];
    if (red_ms) *red_ms = sums[2];
    if (red_launches) *red_launches = counts[2];
    return MRI_OK;
}

MRI_API long long mri_plan_launch_count(const mri_plan *p) { return p ? p->launches : 0; }

MRI_API int mri_plan_get_config(const mri_plan *p, int *fwd_coils_per_tile, int *fwd_stages, int *adj_stages,
                                int *adj_ksplit) {
    if (!p) return fail(MRI_ERR_INVALID, "null plan");
    if (fwd_coils_per_tile) *fwd_coils_per_tile = p->fwd_coils_per_tile;
    if (fwd_stages) *fwd_stages = p->fwd_stages;
    if (adj_stages) *adj_stages = p->adj_stages;
    if (adj_ksplit) *adj_ksplit = p->ksplit;
    return MRI_OK;
}

MRI_API int mri_plan_set_tiles(mri_plan *p, int fwd_coils_per_tile, int fwd_stages, int adj_stages) {
    if (!p) return fail(MRI_ERR_INVALID, "null plan");
    if (!is_tc_precision(p->precision))
        return fail(MRI_ERR_UNSUPPORTED, "tile configurations apply to the tensor-core forms");
    return tc_set_tiles(p, fwd_coils_per_tile, fwd_stages, adj_stages);
}

// Times every valid tile configuration of the two product kernels on this
// plan's shape (the data do not change the work, so the plan's zeroed
// workspace is used) and keeps the fastest: coils per forward N tile with
// the forward stage count, and the adjoint stage count.  The choice changes
// scheduling only, never the arithmetic or its order.  Allocates a temporary
// coil-map buffer and synchronises the stream.
MRI_API int mri_plan_autotune(mri_plan *p, int repeats, mri_stream_t stream) {
    if (!p) return fail(MRI_ERR_INVALID, "null plan");
    if (!is_tc_precision(p->precision)) return MRI_OK;  // the FP32 form has nothing to tune
    if (repeats <= 0) repeats = 3;
    cudaStream_t s = (cudaStream_t)stream;
    float2 *maps = nullptr;
    const size_t npix = (size_t)p->nx * p->ny;
    if (cudaMalloc(&maps, (size_t)p->nc * npix * sizeof(float2)) != cudaSuccess) {
        cudaGetLastError();
        return fail(MRI_ERR_NOMEM, "autotune: temporary coil maps");
    }
    cudaMemsetAsync(maps, 0, (size_t)p->nc * npix * sizeof(float2), s);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const bool was_timing = p->timing;
    p->timing = false;
    int best_cpt = p->fwd_coils_per_tile, best_fs = p->fwd_stages, best_as = p->adj_stages;
    float best_tf = 1e30f, best_ta = 1e30f;
    int rc = MRI_OK;
    // which = 0: forward (coils per tile x stages); which = 1: adjoint (stages)
    for (int which = 0; which < 2 && rc == MRI_OK; ++which) {
        const int cpt_max = which == 0 ? tc_max_coils_per_tile(p) : 1;
        for (int cpt = 1; cpt <= cpt_max && rc == MRI_OK; ++cpt) {
            for (int st = 2; st <= 4; ++st) {
                const int c = which == 0 ? cpt : best_cpt, fs = which == 0 ? st : best_fs;
                const int as = which == 0 ? best_as : st;
                if (!tc_tiles_valid(p, c, fs, as)) continue;
                rc = tc_set_tiles(p, c, fs, as);
                if (rc != MRI_OK) break;
                cudaError_t e = cudaSuccess;
                for (int it = 0; it <= repeats && e == cudaSuccess; ++it) {
                    if (it == 1) cudaEventRecord(e0, s);
                    e = which == 0 ? launch_fwd_tc(p, p->x, maps, p->y, p->nk_pad, kSkipNever, s)
                                   : launch_adj_tc(p, kSkipNever, s);
                }
                cudaEventRecord(e1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) {
                    rc = cuda_fail(e, "autotune");
                    break;
                }
                if (which == 0 && ms < best_tf) {
                    best_tf = ms;
                    best_cpt = cpt;
                    best_fs = st;
                }
                if (which == 1 && ms < best_ta) {
                    best_ta = ms;
                    best_as = st;
                }
            }
        }
    }
    if (rc == MRI_OK) rc = tc_set_tiles(p, best_cpt, best_fs, best_as);
    if (rc == MRI_OK) tuning_record(p);
    p->timing = was_timing;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(maps);
    return rc;
}

}  // extern "C"
