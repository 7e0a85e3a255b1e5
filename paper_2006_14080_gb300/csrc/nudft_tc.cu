// BF16x3 tensor-core form of the two DFT products (tcgen05 + TMA, sm_103a).
//
// Complex products are real-embedded so that one real GEMM carries them:
// a complex row a of the left operand becomes two real rows (Re a, -Im a) and
// (Im a, Re a) interleaved along K, the right operand stores (Re b, Im b)
// interleaved along K, and output rows 2r, 2r+1 are Re and Im of row r.
// Every FP32 operand v is split into hi = bf16(v) and lo = bf16(v - hi); the
// product is accumulated in FP32 (TMEM) as hi*hi + hi*lo + lo*hi (the paper's
// "decomposition and accumulation" on bf16 multipliers, Section II-A).
//
// Forward  (Eq. 1):  Z = A_x (S_c . X) for all coils at once
//     A  = embedded A_x          [2 nk][kx]        static, TMA
//     B  = (S_c . X)^T per coil  [nc * ny_pad][kx] written by fwd_operand_kernel, TMA
//   tile: 128 rows (64 samples) x block_n columns (whole coils); the epilogue
//   forms y_c[k] = sum_j Z[k][j] A_y[k][j] from TMEM and writes y.
// Adjoint: W_c = U_c conj(A_y) with U_c[i][k] = conj(A_x[k][i]) y_c[k]
//     A  = embedded U_c          built in shared memory by producer warps
//     B  = conj(A_y)^T           [ny_pad][kk]      static, TMA
//   tile: 128 rows (64 pixels of one coil) x ny_pad columns, split over
//   contiguous k-space ranges; the epilogue writes partial images that
//   launch_adj_reduce sums in a fixed order (the paper's cross-core sum).
//
// Both kernels are persistent (one CTA per SM), warp-specialised, with a
// multi-stage mbarrier ring between the operand producers and the single
// UMMA-issuing thread and a double-buffered TMEM accumulator between the
// UMMA thread and the epilogue warps.  Every wait is bounded: on give-up the
// block raises a shared abort flag, drains its own copies and UMMAs, frees
// TMEM, records kStatusTimeout and returns.
#include <algorithm>
#include <string>

#include "common.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace mri {

namespace {

using namespace tc;

constexpr uint64_t kWaitLimitNs = 4000000000ull;  // 4 s per wait
constexpr uint64_t kDrainLimitNs = 200000000ull;  // 0.2 s per drain wait
constexpr int kTileBytesA = kTcBlockM * 128;      // 128 rows x 64 bf16
constexpr int kFwdThreads = 192;                  // w0 TMA, w1 UMMA, w2-5 epilogue
constexpr int kAdjThreads = 288;                  // w0-3 producers (+TMA), w4 UMMA, w5-8 epilogue
constexpr int kMaxSmem = 227 * 1024;

struct FwdParams {
    const float2 *ayT;  // [ny][nk]
    float2 *y;          // [nc][nk]
    int nk, ny, ny_pad, nc, cpt, block_n, n_tiles, num_tiles, num_kb, stages;
    uint32_t tmem_cols;
    const DevScalars *sc;
    int skip;
    int *status;
};

struct AdjParams {
    const float2 *axT;  // [nx][nk]
    const float2 *y;    // [nc][nk]
    float2 *part;       // [ksplit][nc][ny][nx_pad]
    int nx, nk, ny, ny_pad, nx_pad, nc, tiles_per_coil, m_tiles, kb_per_split, num_kb, num_units, stages;
    uint32_t tmem_cols;
    const DevScalars *sc;
    int skip;
    int *status;
};

__device__ __forceinline__ uint8_t *align1024(uint8_t *p) {
    return (uint8_t *)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
}

// Wait (bounded, independent of the abort flag) for a phase that may still
// have copies in flight; used only while shutting down after an abort.
__device__ __forceinline__ void drain_wait(uint32_t bar, uint32_t parity) {
    volatile int local = 0;
    mbar_wait(bar, parity, &local, kDrainLimitNs);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
}

// hi/lo split of a pair of FP32 values into packed bf16x2 words.
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo) {
    const __nv_bfloat16 ah = __float2bfloat16_rn(a), bh = __float2bfloat16_rn(b);
    hi = (uint32_t)__bfloat16_as_ushort(ah) | ((uint32_t)__bfloat16_as_ushort(bh) << 16);
    lo = pack_bf16x2(a - __bfloat162float(ah), b - __bfloat162float(bh));
}

// ---------------------------------------------------------------------------
// Forward operand: B[(c*ny_pad + j)][2i + {0,1}] = split(Re, Im of S_c[i][j] x[i][j])
// block (32, 8) over a 32 x 32 (i, j) tile, transposed through shared memory.
__global__ void fwd_operand_kernel(const float2 *__restrict__ x, const float2 *__restrict__ maps,
                                   uint32_t *__restrict__ hi, uint32_t *__restrict__ lo, int nx, int ny, int ny_pad,
                                   int kx, int nc, const DevScalars *sc, int skip) {
    if (should_skip(sc, skip)) return;
    __shared__ float2 xs[32][33];
    __shared__ float2 ss[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    const size_t npix = (size_t)nx * ny;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = i0 + ty + 8 * q, j = j0 + tx;
        xs[ty + 8 * q][tx] = (i < nx && j < ny) ? x[(size_t)i * ny + j] : make_float2(0.f, 0.f);
    }
    for (int c = 0; c < nc; ++c) {
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + ty + 8 * q, j = j0 + tx;
            ss[ty + 8 * q][tx] = (i < nx && j < ny) ? maps[c * npix + (size_t)i * ny + j] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = j0 + ty + 8 * q, i = i0 + tx;
            if (i < nx && j < ny) {
                const float2 v = cmul(ss[tx][ty + 8 * q], xs[tx][ty + 8 * q]);
                uint32_t h, l;
                split2(v.x, v.y, h, l);
                const size_t off = ((size_t)c * ny_pad + j) * (kx / 2) + i;
                hi[off] = h;
                lo[off] = l;
            }
        }
    }
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kFwdThreads, 1)
    fwd_tc_kernel(const __grid_constant__ CUtensorMap ta_hi, const __grid_constant__ CUtensorMap ta_lo,
                  const __grid_constant__ CUtensorMap tb_hi, const __grid_constant__ CUtensorMap tb_lo,
                  const FwdParams P) {
    if (should_skip(P.sc, P.skip)) return;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = align1024(smem_raw);
    const uint32_t b_bytes = (uint32_t)P.block_n * 128u;
    const uint32_t stage_bytes = 2u * kTileBytesA + 2u * b_bytes;
    const int S = P.stages;
    uint64_t *bars = (uint64_t *)(smem + (size_t)S * stage_bytes);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + S);
    const uint32_t tfull0 = smem_u32(bars + 2 * S), tempty0 = smem_u32(bars + 2 * S + 2);
    const uint32_t fin = smem_u32(bars + 2 * S + 4);
    uint32_t *tmem_slot = (uint32_t *)(bars + 2 * S + 5);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(tfull0 + 8 * a, 1);
            mbar_init(tempty0 + 8 * a, 128);
        }
        mbar_init(fin, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), P.tmem_cols);
        tmem_relinquish();
    }
    if (warp == 0 && lane == 0) {
        prefetch_tensormap(&ta_hi);
        prefetch_tensormap(&ta_lo);
        prefetch_tensormap(&tb_hi);
        prefetch_tensormap(&tb_lo);
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            uint32_t issued_phase[4] = {0, 0, 0, 0};
            int issued_mask = 0;
            for (int tile = blockIdx.x; tile < P.num_tiles && !*abort_flag; tile += gridDim.x) {
                const int m_blk = tile / P.n_tiles, n_blk = tile % P.n_tiles;
                for (int kb = 0; kb < P.num_kb; ++kb) {
                    if (!mbar_wait(empty0 + 8 * stage, phase ^ 1, abort_flag, kWaitLimitNs)) break;
                    const uint32_t sbase = smem_u32(smem + (size_t)stage * stage_bytes);
                    const uint32_t fb = full0 + 8 * stage;
                    mbar_arrive_expect_tx(fb, stage_bytes);
                    tma_load_2d(sbase, &ta_hi, fb, kb * kTcBlockK, m_blk * kTcBlockM);
                    tma_load_2d(sbase + kTileBytesA, &ta_lo, fb, kb * kTcBlockK, m_blk * kTcBlockM);
                    tma_load_2d(sbase + 2 * kTileBytesA, &tb_hi, fb, kb * kTcBlockK, n_blk * P.block_n);
                    tma_load_2d(sbase + 2 * kTileBytesA + b_bytes, &tb_lo, fb, kb * kTcBlockK, n_blk * P.block_n);
                    issued_phase[stage] = phase;
                    issued_mask |= 1 << stage;
                    if (++stage == S) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
            }
            if (*abort_flag)
                for (int s = 0; s < S; ++s)
                    if (issued_mask & (1 << s)) drain_wait(full0 + 8 * s, issued_phase[s]);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_f32(kTcBlockM, P.block_n);
            int stage = 0;
            uint32_t phase = 0;
            int lt = 0;
            bool issued_any = false;
            for (int tile = blockIdx.x; tile < P.num_tiles; tile += gridDim.x, ++lt) {
                const int a = lt & 1;
                const uint32_t ap = (lt >> 1) & 1;
                if (!mbar_wait(tempty0 + 8 * a, ap ^ 1, abort_flag, kWaitLimitNs)) break;
                fence_after_sync();
                const uint32_t d_tmem = tmem_base + (uint32_t)(a * P.block_n);
                bool ok = true;
                for (int kb = 0; kb < P.num_kb; ++kb) {
                    if (!mbar_wait(full0 + 8 * stage, phase, abort_flag, kWaitLimitNs)) {
                        ok = false;
                        break;
                    }
                    fence_after_sync();
                    const uint32_t sa_hi = smem_u32(smem + (size_t)stage * stage_bytes);
                    const uint32_t sa_lo = sa_hi + kTileBytesA;
                    const uint32_t sb_hi = sa_hi + 2 * kTileBytesA;
                    const uint32_t sb_lo = sb_hi + b_bytes;
#pragma unroll
                    for (int kk = 0; kk < kTcBlockK / 16; ++kk) {
                        const uint32_t off = kk * 32;
                        const uint64_t dah = sdesc_kmajor_sw128(sa_hi + off), dal = sdesc_kmajor_sw128(sa_lo + off);
                        const uint64_t dbh = sdesc_kmajor_sw128(sb_hi + off), dbl = sdesc_kmajor_sw128(sb_lo + off);
                        umma_f16(d_tmem, dah, dbh, idesc, (kb | kk) != 0);
                        umma_f16(d_tmem, dah, dbl, idesc, 1u);
                        umma_f16(d_tmem, dal, dbh, idesc, 1u);
                    }
                    issued_any = true;
                    umma_commit(empty0 + 8 * stage);
                    if (++stage == S) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
                if (!ok) break;
                umma_commit(tfull0 + 8 * a);
            }
            if (*abort_flag && issued_any) {
                umma_commit(fin);
                drain_wait(fin, 0);
            }
        }
    } else {
        // epilogue: warp (w % 4) reads TMEM lanes [32 (w % 4), 32 (w % 4) + 32)
        const int wq = warp & 3;
        const int row = wq * 32 + lane;
        const int o = row & 1;
        const uint32_t lane_base = (uint32_t)(wq * 32) << 16;
        int lt = 0;
        for (int tile = blockIdx.x; tile < P.num_tiles; tile += gridDim.x, ++lt) {
            const int a = lt & 1;
            const uint32_t ap = (lt >> 1) & 1;
            if (!mbar_wait(tfull0 + 8 * a, ap, abort_flag, kWaitLimitNs)) break;
            fence_after_sync();
            const int m_blk = tile / P.n_tiles, n_blk = tile % P.n_tiles;
            const int kappa = m_blk * (kTcBlockM / 2) + (row >> 1);
            const bool kv = kappa < P.nk;
            for (int cs = 0; cs < P.cpt; ++cs) {
                const int c = n_blk * P.cpt + cs;
                if (c >= P.nc) break;
                const uint32_t col0 = (uint32_t)(a * P.block_n + cs * P.ny_pad);
                float s0 = 0.f, s1 = 0.f;
                int jc = 0;
                for (; jc + 32 <= P.ny_pad; jc += 32) {
                    float v[32];
                    tmem_ld_32cols(tmem_base + lane_base + col0 + jc, v);
                    if (kv) {
#pragma unroll
                        for (int q = 0; q < 32; ++q) {
                            const int j = jc + q;
                            if (j < P.ny) {
                                const float2 ay = __ldg(&P.ayT[(size_t)j * P.nk + kappa]);
                                const float c0 = o ? -ay.y : ay.x, c1 = o ? ay.x : ay.y;
                                s0 = fmaf(v[q], c0, s0);
                                s1 = fmaf(v[q], c1, s1);
                            }
                        }
                    }
                }
                if (jc < P.ny_pad) {  // 16-column tail
                    float v[16];
                    tmem_ld_16cols(tmem_base + lane_base + col0 + jc, v);
                    if (kv) {
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const int j = jc + q;
                            if (j < P.ny) {
                                const float2 ay = __ldg(&P.ayT[(size_t)j * P.nk + kappa]);
                                const float c0 = o ? -ay.y : ay.x, c1 = o ? ay.x : ay.y;
                                s0 = fmaf(v[q], c0, s0);
                                s1 = fmaf(v[q], c1, s1);
                            }
                        }
                    }
                }
                s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
                s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
                if (o == 0 && kv) P.y[(size_t)c * P.nk + kappa] = make_float2(s0, s1);
            }
            fence_before_sync();
            mbar_arrive(tempty0 + 8 * a);
        }
    }

    fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        fence_after_sync();
        tmem_dealloc(tmem_base, P.tmem_cols);
    }
    if (threadIdx.x == 0 && *abort_flag) atomicExch(P.status, kStatusTimeout);
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kAdjThreads, 1)
    adj_tc_kernel(const __grid_constant__ CUtensorMap tb_hi, const __grid_constant__ CUtensorMap tb_lo,
                  const AdjParams P) {
    if (should_skip(P.sc, P.skip)) return;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = align1024(smem_raw);
    const uint32_t b_bytes = (uint32_t)P.ny_pad * 128u;
    const uint32_t stage_bytes = 2u * kTileBytesA + 2u * b_bytes;
    const int S = P.stages;
    uint64_t *bars = (uint64_t *)(smem + (size_t)S * stage_bytes);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + S);
    const uint32_t tfull0 = smem_u32(bars + 2 * S), tempty0 = smem_u32(bars + 2 * S + 2);
    const uint32_t fin = smem_u32(bars + 2 * S + 4);
    uint32_t *tmem_slot = (uint32_t *)(bars + 2 * S + 5);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full0 + 8 * s, 129);  // 128 producer threads + the TMA expect_tx arrival
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(tfull0 + 8 * a, 1);
            mbar_init(tempty0 + 8 * a, 128);
        }
        mbar_init(fin, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 4) {
        tmem_alloc(smem_u32(tmem_slot), P.tmem_cols);
        tmem_relinquish();
    }
    if (threadIdx.x == 0) {
        prefetch_tensormap(&tb_hi);
        prefetch_tensormap(&tb_lo);
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem_base = *tmem_slot;

    if (warp < 4) {
        // producers: thread t builds row (ii = t/2, o = t%2) of the embedded U tile
        const int t = threadIdx.x;
        const int ii = t >> 1, o = t & 1;
        int stage = 0;
        uint32_t phase = 0;
        uint32_t issued_phase[4] = {0, 0, 0, 0};
        int issued_mask = 0;
        for (int u = blockIdx.x; u < P.num_units && !*abort_flag; u += gridDim.x) {
            const int p = u / P.m_tiles, m = u % P.m_tiles;
            const int c = m / P.tiles_per_coil, ib = m % P.tiles_per_coil;
            const int i = ib * 64 + ii;
            const bool iv = i < P.nx;
            const int kb0 = p * P.kb_per_split, kb1 = min(P.num_kb, kb0 + P.kb_per_split);
            const float2 *arow = P.axT + (size_t)(iv ? i : 0) * P.nk;
            const float2 *yc = P.y + (size_t)c * P.nk;
            bool ok = true;
            for (int kb = kb0; kb < kb1; ++kb) {
                if (!mbar_wait(empty0 + 8 * stage, phase ^ 1, abort_flag, kWaitLimitNs)) {
                    ok = false;
                    break;
                }
                uint8_t *sbase = smem + (size_t)stage * stage_bytes;
                const uint32_t fb = full0 + 8 * stage;
                if (t == 0) {
                    const uint32_t sb = smem_u32(sbase + 2 * kTileBytesA);
                    mbar_arrive_expect_tx(fb, 2u * b_bytes);
                    tma_load_2d(sb, &tb_hi, fb, kb * kTcBlockK, 0);
                    tma_load_2d(sb + b_bytes, &tb_lo, fb, kb * kTcBlockK, 0);
                    issued_phase[stage] = phase;
                    issued_mask |= 1 << stage;
                }
                const int k0 = kb * (kTcBlockK / 2);  // 32 samples per K block
                uint32_t hi[32], lo[32];
                // vector path: rows of axT and y start 16-byte aligned only when nk is even
                if (iv && k0 + 32 <= P.nk && (P.nk & 1) == 0) {
#pragma unroll
                    for (int q = 0; q < 32; q += 2) {
                        const float4 av = __ldg(reinterpret_cast<const float4 *>(arow + k0 + q));
                        const float4 yv = __ldg(reinterpret_cast<const float4 *>(yc + k0 + q));
                        const float2 u0 = cmulc(make_float2(av.x, av.y), make_float2(yv.x, yv.y));
                        const float2 u1 = cmulc(make_float2(av.z, av.w), make_float2(yv.z, yv.w));
                        if (o == 0) {
                            split2(u0.x, -u0.y, hi[q], lo[q]);
                            split2(u1.x, -u1.y, hi[q + 1], lo[q + 1]);
                        } else {
                            split2(u0.y, u0.x, hi[q], lo[q]);
                            split2(u1.y, u1.x, hi[q + 1], lo[q + 1]);
                        }
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        const int kappa = k0 + q;
                        float2 uv = make_float2(0.f, 0.f);
                        if (iv && kappa < P.nk) uv = cmulc(arow[kappa], yc[kappa]);
                        if (o == 0)
                            split2(uv.x, -uv.y, hi[q], lo[q]);
                        else
                            split2(uv.y, uv.x, hi[q], lo[q]);
                    }
                }
                const int row = 2 * ii + o;
#pragma unroll
                for (int ch = 0; ch < 8; ++ch) {
                    const uint32_t off = sw128_offset(row, ch * 16);
                    *reinterpret_cast<uint4 *>(sbase + off) =
                        make_uint4(hi[4 * ch], hi[4 * ch + 1], hi[4 * ch + 2], hi[4 * ch + 3]);
                    *reinterpret_cast<uint4 *>(sbase + kTileBytesA + off) =
                        make_uint4(lo[4 * ch], lo[4 * ch + 1], lo[4 * ch + 2], lo[4 * ch + 3]);
                }
                fence_proxy_async_smem();
                mbar_arrive(fb);
                if (++stage == S) {
                    stage = 0;
                    phase ^= 1;
                }
            }
            if (!ok) break;
        }
        if (t == 0 && *abort_flag)
            for (int s = 0; s < S; ++s)
                if (issued_mask & (1 << s)) drain_wait(full0 + 8 * s, issued_phase[s]);
    } else if (warp == 4) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_f32(kTcBlockM, P.ny_pad);
            int stage = 0;
            uint32_t phase = 0;
            int lt = 0;
            bool issued_any = false;
            for (int u = blockIdx.x; u < P.num_units; u += gridDim.x, ++lt) {
                const int p = u / P.m_tiles;
                const int kb0 = p * P.kb_per_split, kb1 = min(P.num_kb, kb0 + P.kb_per_split);
                const int a = lt & 1;
                const uint32_t ap = (lt >> 1) & 1;
                if (!mbar_wait(tempty0 + 8 * a, ap ^ 1, abort_flag, kWaitLimitNs)) break;
                fence_after_sync();
                const uint32_t d_tmem = tmem_base + (uint32_t)(a * P.ny_pad);
                bool ok = true;
                for (int kb = kb0; kb < kb1; ++kb) {
                    if (!mbar_wait(full0 + 8 * stage, phase, abort_flag, kWaitLimitNs)) {
                        ok = false;
                        break;
                    }
                    fence_after_sync();
                    const uint32_t sa_hi = smem_u32(smem + (size_t)stage * stage_bytes);
                    const uint32_t sa_lo = sa_hi + kTileBytesA;
                    const uint32_t sb_hi = sa_hi + 2 * kTileBytesA;
                    const uint32_t sb_lo = sb_hi + b_bytes;
#pragma unroll
                    for (int kk = 0; kk < kTcBlockK / 16; ++kk) {
                        const uint32_t off = kk * 32;
                        const uint64_t dah = sdesc_kmajor_sw128(sa_hi + off), dal = sdesc_kmajor_sw128(sa_lo + off);
                        const uint64_t dbh = sdesc_kmajor_sw128(sb_hi + off), dbl = sdesc_kmajor_sw128(sb_lo + off);
                        umma_f16(d_tmem, dah, dbh, idesc, (kb != kb0 || kk != 0) ? 1u : 0u);
                        umma_f16(d_tmem, dah, dbl, idesc, 1u);
                        umma_f16(d_tmem, dal, dbh, idesc, 1u);
                    }
                    issued_any = true;
                    umma_commit(empty0 + 8 * stage);
                    if (++stage == S) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
                if (!ok) break;
                umma_commit(tfull0 + 8 * a);
            }
            if (*abort_flag && issued_any) {
                umma_commit(fin);
                drain_wait(fin, 0);
            }
        }
    } else {
        // epilogue: warps 5..8; TMEM lane quadrant = warp % 4
        const int wq = warp & 3;
        const int row = wq * 32 + lane;
        const int ii = row >> 1, o = row & 1;
        const uint32_t lane_base = (uint32_t)(wq * 32) << 16;
        int lt = 0;
        for (int u = blockIdx.x; u < P.num_units; u += gridDim.x, ++lt) {
            const int a = lt & 1;
            const uint32_t ap = (lt >> 1) & 1;
            if (!mbar_wait(tfull0 + 8 * a, ap, abort_flag, kWaitLimitNs)) break;
            fence_after_sync();
            const int p = u / P.m_tiles, m = u % P.m_tiles;
            const int c = m / P.tiles_per_coil, ib = m % P.tiles_per_coil;
            const int i = ib * 64 + ii;
            float *dst = reinterpret_cast<float *>(P.part + ((size_t)p * P.nc + c) * P.ny * P.nx_pad) + 2 * i + o;
            const size_t jstride = 2 * (size_t)P.nx_pad;
            const uint32_t col0 = (uint32_t)(a * P.ny_pad);
            int jc = 0;
            for (; jc + 32 <= P.ny_pad; jc += 32) {
                float v[32];
                tmem_ld_32cols(tmem_base + lane_base + col0 + jc, v);
#pragma unroll
                for (int q = 0; q < 32; ++q)
                    if (jc + q < P.ny) dst[(size_t)(jc + q) * jstride] = v[q];
            }
            if (jc < P.ny_pad) {
                float v[16];
                tmem_ld_16cols(tmem_base + lane_base + col0 + jc, v);
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    if (jc + q < P.ny) dst[(size_t)(jc + q) * jstride] = v[q];
            }
            fence_before_sync();
            mbar_arrive(tempty0 + 8 * a);
        }
    }

    fence_before_sync();
    __syncthreads();
    if (warp == 4) {
        fence_after_sync();
        tmem_dealloc(tmem_base, P.tmem_cols);
    }
    if (threadIdx.x == 0 && *abort_flag) atomicExch(P.status, kStatusTimeout);
}

// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)ptr;
    }
    return fn;
}

// 2-D bf16 tensor [rows][cols] (cols contiguous), box = 64 cols x box_rows, 128-byte swizzle.
bool make_map(CUtensorMap *m, void *base, uint64_t cols, uint64_t rows, uint32_t box_rows) {
    EncodeTiledFn fn = get_encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)kTcBlockK, box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int stages_for(uint32_t stage_bytes) {
    const int avail = kMaxSmem - 1024 - 256;
    return std::min(4, avail / (int)stage_bytes);
}

uint32_t tmem_cols_for(int cols) {
    uint32_t n = 32;
    while ((int)n < cols) n <<= 1;
    return n;
}

size_t fwd_smem_bytes(const mri_plan *p) {
    const uint32_t stage = 2u * kTileBytesA + 2u * (uint32_t)p->fwd_block_n * 128u;
    return 1024 + (size_t)stages_for(stage) * stage + 256;
}

size_t adj_smem_bytes(const mri_plan *p) {
    const uint32_t stage = 2u * kTileBytesA + 2u * (uint32_t)p->ny_pad * 128u;
    return 1024 + (size_t)stages_for(stage) * stage + 256;
}

}  // namespace

bool tc_supported(const mri_plan *p, std::string *why) {
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, p->device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, p->device);
    if (major != 10 || minor != 3) {
        *why = "needs an sm_103 GPU (found sm_" + std::to_string(major) + std::to_string(minor) + ")";
        return false;
    }
    if (round_up(p->ny, 16) > 256) {
        *why = "ny up to 256 is supported by the tensor-core kernels";
        return false;
    }
    if (!get_encode_fn()) {
        *why = "cuTensorMapEncodeTiled is not available from the driver";
        return false;
    }
    return true;
}

int tc_plan_tiling(mri_plan *p) {
    // forward: whole coils per N tile
    const int cpt_max = std::max(1, 256 / p->ny_pad);
    const int n_tiles = ceil_div(p->nc, cpt_max);
    p->fwd_coils_per_tile = ceil_div(p->nc, n_tiles);
    p->fwd_block_n = p->fwd_coils_per_tile * p->ny_pad;
    p->fwd_n_tiles = ceil_div(p->nc, p->fwd_coils_per_tile);
    p->fwd_m_tiles = ceil_div(2 * p->nk, kTcBlockM);
    // adjoint: 64 pixels (128 embedded rows) of one coil per M tile; split K
    // (k-space samples) so that the units fill the SMs evenly
    p->adj_m_tiles = p->nc * (p->nx_pad / 64);
    p->adj_block_n = p->ny_pad;
    const int num_kb = p->kk / kTcBlockK;
    long best_cost = -1;
    int best_split = 1;
    for (int split = 1; split <= std::min(num_kb, 128); ++split) {
        const int per = ceil_div(num_kb, split);
        const int eff = ceil_div(num_kb, per);
        const long waves = ceil_div(p->adj_m_tiles * eff, p->num_sms);
        const long cost = waves * per + (long)eff / 8;  // makespan in K blocks, small penalty per split
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best_split = eff;
        }
    }
    p->ksplit_blocks = ceil_div(num_kb, best_split);
    p->ksplit = ceil_div(num_kb, p->ksplit_blocks);
    if (fwd_smem_bytes(p) > (size_t)kMaxSmem || adj_smem_bytes(p) > (size_t)kMaxSmem) return MRI_ERR_UNSUPPORTED;
    return MRI_OK;
}

int tc_make_tensor_maps(mri_plan *p) {
    bool ok = make_map(&p->tm_afwd_hi, p->afwd_hi, p->kx, 2ull * p->nk, kTcBlockM) &&
              make_map(&p->tm_afwd_lo, p->afwd_lo, p->kx, 2ull * p->nk, kTcBlockM) &&
              make_map(&p->tm_bfwd_hi, p->bfwd_hi, p->kx, (uint64_t)p->nc * p->ny_pad, p->fwd_block_n) &&
              make_map(&p->tm_bfwd_lo, p->bfwd_lo, p->kx, (uint64_t)p->nc * p->ny_pad, p->fwd_block_n) &&
              make_map(&p->tm_badj_hi, p->badj_hi, p->kk, p->ny_pad, p->ny_pad) &&
              make_map(&p->tm_badj_lo, p->badj_lo, p->kk, p->ny_pad, p->ny_pad);
    if (!ok) {
        set_error("cuTensorMapEncodeTiled failed");
        return MRI_ERR_CUDA;
    }
    cudaError_t e = cudaFuncSetAttribute(fwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(adj_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    if (e != cudaSuccess) {
        set_error(std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
        return MRI_ERR_CUDA;
    }
    return MRI_OK;
}

cudaError_t launch_fwd_tc(mri_plan *p, const float2 *image, const float2 *maps, float2 *kspace, int skip,
                          cudaStream_t s) {
    dim3 og(ceil_div(p->nx, 32), ceil_div(p->ny, 32));
    fwd_operand_kernel<<<og, dim3(32, 8), 0, s>>>(image, maps, (uint32_t *)p->bfwd_hi, (uint32_t *)p->bfwd_lo, p->nx,
                                                  p->ny, p->ny_pad, p->kx, p->nc, p->scal, skip);
    FwdParams P;
    P.ayT = p->ayT;
    P.y = kspace;
    P.nk = p->nk;
    P.ny = p->ny;
    P.ny_pad = p->ny_pad;
    P.nc = p->nc;
    P.cpt = p->fwd_coils_per_tile;
    P.block_n = p->fwd_block_n;
    P.n_tiles = p->fwd_n_tiles;
    P.num_tiles = p->fwd_m_tiles * p->fwd_n_tiles;
    P.num_kb = p->kx / kTcBlockK;
    const uint32_t stage = 2u * kTileBytesA + 2u * (uint32_t)p->fwd_block_n * 128u;
    P.stages = stages_for(stage);
    P.tmem_cols = tmem_cols_for(2 * p->fwd_block_n);
    P.sc = p->scal;
    P.skip = skip;
    P.status = &p->scal->status;
    const int grid = std::min(P.num_tiles, p->num_sms);
    timing_begin(p, s);
    fwd_tc_kernel<<<grid, kFwdThreads, fwd_smem_bytes(p), s>>>(p->tm_afwd_hi, p->tm_afwd_lo, p->tm_bfwd_hi,
                                                               p->tm_bfwd_lo, P);
    timing_end(p, s);
    p->launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_adj_tc(mri_plan *p, const float2 *kspace, int skip, cudaStream_t s) {
    AdjParams P;
    P.axT = p->axT;
    P.y = kspace;
    P.part = p->part;
    P.nx = p->nx;
    P.nk = p->nk;
    P.ny = p->ny;
    P.ny_pad = p->ny_pad;
    P.nx_pad = p->nx_pad;
    P.nc = p->nc;
    P.tiles_per_coil = p->nx_pad / 64;
    P.m_tiles = p->adj_m_tiles;
    P.kb_per_split = p->ksplit_blocks;
    P.num_kb = p->kk / kTcBlockK;
    P.num_units = p->adj_m_tiles * p->ksplit;
    const uint32_t stage = 2u * kTileBytesA + 2u * (uint32_t)p->ny_pad * 128u;
    P.stages = stages_for(stage);
    P.tmem_cols = tmem_cols_for(2 * p->ny_pad);
    P.sc = p->scal;
    P.skip = skip;
    P.status = &p->scal->status;
    const int grid = std::min(P.num_units, p->num_sms);
    timing_begin(p, s);
    adj_tc_kernel<<<grid, kAdjThreads, adj_smem_bytes(p), s>>>(p->tm_badj_hi, p->tm_badj_lo, P);
    timing_end(p, s);
    p->launches += 1;
    return cudaGetLastError();
}

}  // namespace mri
