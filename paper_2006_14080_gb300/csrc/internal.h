// Internal declarations of the mrirecon library: the plan object and the
// launchers each translation unit provides.  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stddef.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "mrirecon.h"

namespace mri {

// Scalars of the solver, resident on the device so that no step of the
// reconstruction waits on the host.
struct DevScalars {
    double tau;         // ||r||^2 of the current CG iterate (Alg. 2)
    double alpha;       // CG step length tau / Re<d, A d>
    double beta_cg;     // CG direction coefficient tau' / tau
    double admm_alpha;  // relative change ||x'-x||^2 / ||x'||^2 (Alg. 4)
    double atol2;       // atol^2
    double rtol2;       // rtol^2
    int cg_done;        // CG has met its tolerance for the current x-update
    int admm_done;      // ADMM has met its tolerance
    int status;         // 0, or a device-side failure code (see kStatus*)
    int step_active;    // the current ADMM step runs (ADMM had not stopped when it began)
    double tau_next;    // two-kernel CG step: ||r'||^2, handed from the reduction to the update
    int step_pending;   // two-kernel CG step: the reduction ran and its update is due
    float cg_split[6];  // two-kernel CG step: alpha, -alpha, beta as FP32 (hi, lo) pairs
    unsigned counters[8];  // grid-reduction tickets, one per reduction site
};

enum : int { kStatusOk = 0, kStatusTimeout = 1 };
enum SkipMode : int { kSkipNever = 0, kSkipAdmm = 1, kSkipCg = 2, kSkipStep = 3 };

__device__ __forceinline__ bool should_skip(const DevScalars *s, int mode) {
    if (mode == kSkipNever || s == nullptr) return false;
    if (mode == kSkipStep) return !s->step_active;
    if (s->admm_done) return true;
    return mode == kSkipCg && s->cg_done;
}

enum Counter : int { kCntDot = 0, kCntTau = 1, kCntInit = 2, kCntDual = 3, kCntObj = 4 };

// Tile constants of the tensor-core kernels.
constexpr int kTcBlockM = 128;   // UMMA M (rows of the real-embedded operand)
constexpr int kTcBlockK = 64;    // bf16 elements per 128-byte swizzled row

// Host-side NVTX range around a library call (shown on Nsight timelines; ncu
// can select the kernels a call launched with --nvtx --nvtx-include).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

inline bool is_tc_precision(int precision) { return precision == MRI_BF16X3 || precision == MRI_TF32; }

inline int round_up(int a, int b) { return (a + b - 1) / b * b; }
inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

}  // namespace mri

struct mri_plan {
    int nx = 0, ny = 0, nk = 0, nc = 0, precision = 0;
    int device = 0, num_sms = 0;

    // FP32 factors (Alg. 1, separable): A_x[k][i], A_y[k][j]
    float2 *ax = nullptr;   // [nk][nx]
    float2 *ay = nullptr;   // [nk][ny]
    // transposed FP32 factors used by the tensor-core path
    float2 *axT = nullptr;  // [nx][nk] (adjoint row-pair form)
    // adjoint pixel-row form: A_x[k][i] = axP[i / 16][k] * axQ[i % 16][k] with
    // axP[a][k] = exp(-i 2 pi kx_k (16 a - nx/2)), axQ[b][k] = exp(-i 2 pi kx_k b)
    float2 *axP = nullptr;  // [nx_pad / 16][nk_pad]
    float2 *axQ = nullptr;  // [16][nk_pad]
    float2 *ayT = nullptr;  // [ny][nk]

    int nk_pad = 0;   // round_up(nk, 32): leading dimension of sample-indexed rows (axT, ayT, y)

    // BF16 hi/lo real-embedded operands (tensor-core path)
    int kx = 0;       // round_up(2*nx, 64): K of the forward product
    int kk = 0;       // round_up(2*nk, 64): K of the adjoint product
    int ny_pad = 0;   // round_up(ny, 16), or round_up(ny, 256) past 256: UMMA N granularity
    int nx_pad = 0;   // round_up(nx, 64): image rows per adjoint M tile group
    int fwd_coils_per_tile = 0, fwd_block_n = 0, fwd_n_tiles = 0, fwd_m_tiles = 0;
    int adj_m_tiles = 0, adj_block_n = 0;  // adjoint M tiles (coils x pixel tiles) and UMMA N
    // adjoint M tile: 64 pixels as Re/Im row pairs of the embedded U (B =
    // conj(A_y) with one row per image column), or 128 pixels with one row
    // each (B with two rows per column, UMMA N = 2 ny_pad; when ny <= 128
    // and nx_pad is a multiple of 128)
    int adj_tile_px = 64;
    int badj_rows = 0;  // rows of the adjoint B operand: ny_pad, or 2 ny_pad with 128-pixel tiles
    int fwd_stages = 0, adj_stages = 0;      // operand ring stages of the two products (0: as many as fit)
    int fwd_grid = 0, adj_grid = 0;          // persistent grid sizes (co-resident CTAs)
    __nv_bfloat16 *afwd_hi = nullptr, *afwd_lo = nullptr;  // [2*nk][kx]
    __nv_bfloat16 *badj_hi = nullptr, *badj_lo = nullptr;  // [badj_rows][kk]
    __nv_bfloat16 *bfwd_hi = nullptr, *bfwd_lo = nullptr;  // [nc*ny_pad][kx]
    // TF32 form: the same operands as single TF32-rounded FP32 matrices
    float *afwd_t = nullptr;  // [2*nk][kx]
    float *badj_t = nullptr;  // [badj_rows][kk]
    float *bfwd_t = nullptr;  // [nc*ny_pad][kx]
    // tensor maps of the operands; in the TF32 form the _hi and _lo maps are
    // the same map, and a K block's two 128-byte halves are its columns
    // [64 kb, 64 kb + 32) and [64 kb + 32, 64 kb + 64)
    CUtensorMap tm_afwd_hi, tm_afwd_lo, tm_bfwd_hi, tm_bfwd_lo, tm_badj_hi, tm_badj_lo;
    CUtensorMap tm_axT, tm_y, tm_ayT;  // FP32 views of axT, y, ayT for staged factor tiles
    CUtensorMap tm_axP, tm_axQ;        // FP32 views of axP, axQ (pixel-row form)

    // operator workspace
    float2 *bsx = nullptr;    // [nc][nx][ny] S_c . x (FP32 path)
    float2 *y = nullptr;      // [nc][nk_pad] k-space workspace (padding stays zero)
    // adjoint partial images part[c][j][ig][p][64]: pixel i = 64 ig + (i % 64)
    // fastest, then the k-space split p, the 64-pixel group ig (nx_pad / 64 of
    // them), the column j and the coil, so that the splits of one coil, column
    // and pixel group are contiguous for the fixed-order sum
    float2 *part = nullptr;
    int ksplit = 1;           // k-space splits of the adjoint product
    int ksplit_blocks = 0;    // K blocks per split (tensor path) or samples per split (FP32)

    // solver state, in the transposed layout v[j][i] (pixel (i, j) at j * nx + i)
    float2 *x = nullptr, *xprev = nullptr, *r = nullptr, *r2 = nullptr, *d = nullptr, *d2 = nullptr, *ad = nullptr;
    float2 *b = nullptr, *fhd = nullptr;                 // [ny][nx]
    float2 *mu = nullptr, *eta = nullptr;                // [2][ny][nx]
    float2 *mapsT = nullptr;                             // [nc][ny][nx_pad]: the coil maps of the reconstruction
    double *partials = nullptr;                          // grid-reduction partials
    int partials_cap = 0;                                // doubles
    unsigned *grid_bar = nullptr;                        // [2]: the CG step's grid barrier (count, generation)
    int cg_grid = 0;                                     // blocks of the cooperative CG step
    mri::DevScalars *scal = nullptr;

    size_t bytes = 0;
    // when set, every buffer comes from this stream-ordered pool (allocated on
    // pool_stream) and is freed stream-ordered (see plan_destroy_async)
    cudaMemPool_t pool = nullptr;
    cudaStream_t pool_stream = nullptr;

    // diagnostics: kernel launches issued on this plan, and optional CUDA-event
    // timing of the two product kernels (see mri_plan_set_timing)
    long long launches = 0;
    bool timing = false;
    cudaEvent_t t_ev0 = nullptr, t_ev1 = nullptr;  // set by the caller around one product launch
    std::vector<cudaEvent_t> ev_free;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_fwd, ev_adj, ev_red;

    // CUDA graph of one whole reconstruction, replayed while the arguments
    // (device pointers and parameters) stay the same
    bool use_graphs = true;
    struct GraphKey {
        const void *kspace, *maps, *image_out, *obj, *alpha;
        float lambda, beta;
        int admm_iters, cg_iters;
        double rtol, atol;
        const void *x0, *eta0, *eta_out;  // resumed reconstructions (else null)
        bool coop;                         // CG step as one cooperative kernel, or as two kernels
        bool operator==(const GraphKey &o) const {
            return kspace == o.kspace && maps == o.maps && image_out == o.image_out && obj == o.obj &&
                   alpha == o.alpha && lambda == o.lambda && beta == o.beta && admm_iters == o.admm_iters &&
                   cg_iters == o.cg_iters && rtol == o.rtol && atol == o.atol && x0 == o.x0 && eta0 == o.eta0 &&
                   eta_out == o.eta_out && coop == o.coop;
        }
    } graph_key{};
    cudaGraphExec_t graph_exec = nullptr;
    long long graph_launches = 0;  // kernels in one replay
    long long graph_captures = 0, graph_replays = 0;  // reconstructions captured, and replayed from a graph
    // Identity for graphs captured outside the plan (batches): unique per plan
    // in the process, so that a new plan at a freed plan's address never
    // matches, and a generation that grows whenever the plan's own graph is
    // dropped because its captured arguments went stale.
    uint64_t serial = 0;
    uint64_t config_gen = 0;
};

namespace mri {
// mri_plan_create with an optional stream-ordered pool for the plan's buffers.
int plan_create(mri_plan **out, int nx, int ny, int nk, int nc, const float *traj, int precision,
                cudaStream_t stream, cudaMemPool_t pool);
// Release a plan without synchronising: pool-allocated buffers are freed
// stream-ordered on s (no work on the plan may be pending elsewhere).
void plan_destroy_async(mri_plan *p, cudaStream_t s);
// Drop the cached reconstruction graph (its kernels' arguments are stale).
void invalidate_graph(mri_plan *p);
// Persistent autotuning table (tuning.cu): record a plan's tile configuration
// (forward coils per tile, forward and adjoint stages) / look up the one
// recorded for its precision, shape and SM count.
void tuning_record(const mri_plan *p);
bool tuning_lookup(const mri_plan *p, int *fwd_coils_per_tile, int *fwd_stages, int *adj_stages);
// Argument checks of mri_admm_reconstruct (MRI_* status, sets the error text).
int check_admm_args(const mri_plan *p, const mri_c64 *kspace, const mri_c64 *maps, const mri_admm_params *prm,
                    const mri_c64 *image_out);
// Saved ADMM state to start from (x0, eta0; null = zero) and where to leave
// the final dual variable (eta_out, nullable).
struct AdmmWarm {
    const mri_c64 *x0 = nullptr, *eta0 = nullptr;
    mri_c64 *eta_out = nullptr;
};
// Enqueue one whole reconstruction (Alg. 4 with Alg. 2) on s; MRI_* status.
// coop: each CG step as one cooperative kernel (a single reconstruction on
// the stream); else as two ordinary kernels with the same arithmetic and
// results, for reconstructions that run concurrently with others (batches,
// the server), where a cooperative grid would wait for the whole GPU.
int enqueue_admm(mri_plan *p, const mri_c64 *kspace, const mri_c64 *maps, const mri_admm_params *prm,
                 mri_c64 *image_out, double *objective_hist, double *alpha_hist, cudaStream_t s,
                 const AdmmWarm &warm = AdmmWarm(), bool coop = true);
// enqueue_admm through the plan's cached CUDA graph of the whole
// reconstruction: captured on the first call with these arguments (device
// pointers, parameters, coop), replayed while they repeat; direct launches
// when the plan's graphs are off, its timing is on, or s is the legacy stream.
int run_admm(mri_plan *p, const mri_c64 *kspace, const mri_c64 *maps, const mri_admm_params *prm,
             mri_c64 *image_out, double *objective_hist, double *alpha_hist, const AdmmWarm &warm, cudaStream_t s,
             bool coop = true);
}  // namespace mri

// Record the timing events (when set) immediately around a product kernel.
inline void timing_begin(mri_plan *p, cudaStream_t s) {
    if (p->t_ev0) cudaEventRecord(p->t_ev0, s);
}
inline void timing_end(mri_plan *p, cudaStream_t s) {
    if (p->t_ev1) cudaEventRecord(p->t_ev1, s);
}

namespace mri {

void set_error(const std::string &msg);

// factors.cu
cudaError_t launch_factors(mri_plan *p, const float *traj, cudaStream_t s);

// nudft_fp32.cu -- forward writes kspace[c * ld + k] (image == nullptr: the
// operand S_c . v is already in p->bsx, transposed, written by the solver);
// adjoint reads p->y
cudaError_t launch_fwd_fp32(mri_plan *p, const float2 *image, const float2 *maps, float2 *kspace, int ld,
                            int skip, cudaStream_t s);
cudaError_t launch_adj_fp32(mri_plan *p, int skip, cudaStream_t s);
// Blocks of the FP32 adjoint the GPU holds at once (its occupancy x num_sms).
int adj_fp32_slots(int num_sms);

// nudft_tc.cu -- same conventions (image == nullptr: the operand is already
// in bfwd_hi/lo or bfwd_t, written by the solver)
bool tc_supported(const mri_plan *p, std::string *why);
int tc_plan_tiling(mri_plan *p);       // tile shapes and k-space splits; MRI_* status
int tc_make_tensor_maps(mri_plan *p);  // TMA descriptors of the allocated operands; MRI_* status
// Tile configuration of the two products: coils per forward N tile
// (1..tc_max_coils_per_tile) and operand ring stages of each (2..4, as the
// shared memory and TMEM allow); 0 keeps the current value.  Rebuilds the
// tensor maps.  None of them changes the arithmetic or its order.
int tc_set_tiles(mri_plan *p, int fwd_coils_per_tile, int fwd_stages, int adj_stages);
bool tc_tiles_valid(const mri_plan *p, int fwd_coils_per_tile, int fwd_stages, int adj_stages);
int tc_max_coils_per_tile(const mri_plan *p);
cudaError_t launch_fwd_tc(mri_plan *p, const float2 *image, const float2 *maps, float2 *kspace, int ld,
                          int skip, cudaStream_t s);
cudaError_t launch_adj_tc(mri_plan *p, int skip, cudaStream_t s);

// solver.cu
struct ReduceEpilogue {
    const float2 *tv_src = nullptr;  // add half_beta * Theta^H Theta tv_src when non-null
    float half_beta = 0.f;
    const float2 *dot_src = nullptr; // when non-null: Re<dot_src, out> -> scal->alpha = tau / dot
    int skip = kSkipNever;
};
cudaError_t launch_adj_reduce(mri_plan *p, const float2 *maps, float2 *out, const ReduceEpilogue &e,
                              cudaStream_t s);
cudaError_t launch_tv_forward(int nx, int ny, const float2 *x, float2 *g, cudaStream_t s);
cudaError_t launch_tv_adjoint(int nx, int ny, const float2 *g, float2 *x, cudaStream_t s);
cudaError_t launch_shrink(int n, float t, const float2 *in, float2 *out, cudaStream_t s);

// admm.cu -- the reconstruction's kernels, on the plan's transposed state
// dst[b][c][r] = src[b][r][c] for `planes` planes of rows x cols complex
// values; destination rows ld_dst apart (0: rows)
cudaError_t launch_transpose(const float2 *src, float2 *dst, int rows, int cols, int planes, cudaStream_t s,
                             int ld_dst = 0);
cudaError_t launch_admm_reset(mri_plan *p, double atol, double rtol, cudaStream_t s);
cudaError_t launch_fhd(mri_plan *p, cudaStream_t s);  // fhd from the adjoint's partial images
cudaError_t launch_mu_rhs(mri_plan *p, float thresh, float half_beta, cudaStream_t s);
cudaError_t launch_cg_init(mri_plan *p, float half_beta, cudaStream_t s);
// cooperative; step `it` of a CG solve reads the residual and direction
// from r, d (it even) or r2, d2 (odd) and leaves the next ones in the others
cudaError_t launch_cg_step(mri_plan *p, float half_beta, int it, cudaStream_t s);
// the same CG step as two ordinary kernels (reduction, then the updates)
cudaError_t launch_cg_step_split(mri_plan *p, float half_beta, int it, cudaStream_t s);
cudaError_t launch_dual(mri_plan *p, bool operand, double *alpha_hist, int m, cudaStream_t s);
cudaError_t launch_objective(mri_plan *p, const float2 *kspace, float lambda, double *obj_hist, int m,
                             cudaStream_t s);
int cg_step_grid(const mri_plan *p);  // co-resident blocks of the cooperative CG step

}  // namespace mri
