// Tensor-core forms of the two DFT products (tcgen05 + TMA, sm_103a): BF16x3
// and TF32.
//
// Complex products are real-embedded so that one real GEMM carries them:
// a complex row a of the left operand becomes two real rows (Re a, -Im a) and
// (Im a, Re a) interleaved along K, the right operand stores (Re b, Im b)
// interleaved along K, and output rows 2r, 2r+1 are Re and Im of row r.
// Every FP32 operand v is split into hi = bf16(v) and lo = bf16(v - hi); the
// product is accumulated in FP32 (TMEM) as hi*hi + hi*lo + lo*hi (the paper's
// "decomposition and accumulation" on bf16 multipliers, Section II-A).  The
// TF32 form instead rounds every operand to TF32 and issues one kind::tf32
// product; its operands take the same bytes (a K block of 64 elements is two
// 128-byte rows, where BF16x3 has a hi row and a lo row), so both forms share
// the tiles, rings and stage sizes and differ only in the operand words and
// the UMMA issue (kTf32 template parameter).
//
// Forward  (Eq. 1):  Z = A_x (S_c . X) for all coils at once
//     A  = embedded A_x          [2 nk][kx]        static, TMA
//     B  = (S_c . X)^T per coil  [nc * ny_pad][kx] written by fwd_operand_kernel, TMA
//   tile: 128 rows (64 samples) x block_n columns (whole coils, or 256-column
//   sub-tiles of one coil wider than that).  The
//   epilogue forms y_c[k] = sum_j Z[k][j] A_y[k][j] from TMEM, with the
//   matching 64-sample x 32-column tiles of A_y staged in shared memory by a
//   TMA warp.
// Adjoint: W_c = U_c conj(A_y) with U_c[i][k] = conj(A_x[k][i]) y_c[k]
//     A  = U_c                   built by producer warps from A_x^H and y tiles
//                                that a TMA warp stages, written to tensor
//                                memory (the UMMAs read A from TMEM)
//     B  = conj(A_y)^T           [badj_rows][kk]   static, TMA
//   Two tile forms.  Row pairs: 128 rows = 64 pixels of one coil, U embedded
//   as above, B one row (Re, Im) per image column, UMMA N = ny_pad (at most
//   256; a wider image takes one launch per 256-column part).  Pixel rows
//   (ny <= 128, nx_pad a multiple of 128): 128 rows = 128 pixels, row i of A
//   is (Re U, Im U) along K and B carries the complex structure instead,
//   rows 2j: (Re G, -Im G) and 2j+1: (Im G, Re G) for G = conj(A_y)[.][j],
//   so output columns 2j, 2j+1 are Re and Im of image column j and the UMMA
//   is 2 ny_pad wide: twice the columns per U element formed, on the wider
//   UMMA shape.  Either way the tile is split over contiguous k-space
//   ranges; the epilogue writes partial images that launch_adj_reduce sums
//   in a fixed order (the paper's cross-core sum).
//
// Both kernels are persistent (one CTA per SM), warp-specialised, with
// mbarrier rings between the loaders/producers and the single UMMA-issuing
// thread and a double-buffered TMEM accumulator between the UMMA thread and
// the epilogue warps.  Every wait is bounded: on give-up the block raises a
// shared abort flag, drains its own copies and UMMAs, frees TMEM, records
// kStatusTimeout and returns.
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
constexpr int kAyChunkBytes = 32 * 64 * 8;        // 32 columns x 64 samples, complex FP32
// one raw stage of the adjoint, 32 samples, complex FP32 in 128-byte-swizzled
// halves of sixteen samples: row pairs, the 64 pixel rows of A_x^T (16 KB);
// pixel rows, the 8 axP rows and 16 axQ rows whose products are the tile's
// 128 pixel rows of A_x^T (6 KB: P half 0, P half 1, Q half 0, Q half 1)
constexpr int raw_bytes_for(int px) { return px == 128 ? 2 * (8 + 16) * 128 : 2 * px * 128; }
constexpr int kRawQ0 = 2 * 8 * 128;  // offset of the axQ halves in a pixel-row raw stage
constexpr int kRawYBytes = 32 * 8;                // 32 samples of y_c
constexpr int kFwdThreads = 224;                  // w0 TMA, w1 UMMA, w2 A_y TMA, w3-6 epilogue
#ifndef MRI_ADJ_PRODUCER_WARPS
#define MRI_ADJ_PRODUCER_WARPS 8
#endif
// adjoint: producer warps (8 or 16), then the UMMA warp, 4 epilogue warps, the TMA warp
constexpr int kAdjProducerWarps = MRI_ADJ_PRODUCER_WARPS;
static_assert(kAdjProducerWarps == 8 || kAdjProducerWarps == 16, "8 or 16 producer warps");
constexpr int kAdjProducers = 32 * kAdjProducerWarps;
constexpr int kAdjMmaWarp = kAdjProducerWarps;
constexpr int kAdjLoaderWarp = kAdjProducerWarps + 5;
constexpr int kAdjThreads = 32 * (kAdjProducerWarps + 6);
constexpr int kMaxSmem = 227 * 1024;
constexpr int kSmemSlack = 1024 + 256;            // alignment + barriers
constexpr int kMaxCoilsPerTile = 4;
#ifndef MRI_ADJ_MAX_KB_PER_SPLIT
#define MRI_ADJ_MAX_KB_PER_SPLIT 32
#endif
constexpr int kMaxKbPerSplit = MRI_ADJ_MAX_KB_PER_SPLIT;  // adjoint: K blocks (32 samples each) per k-space split

// Work split of both kernels: the persistent CTAs take the tiles (units) in
// turn, CTA b units b, b + gridDim.x, ...; every CTA loads its own operands.
struct FwdParams {
    float2 *y;  // [nc][y_ld]
    int y_ld, nk, ny_pad, nc, cpt, block_n, n_tiles, num_kb, stages, ay_stages;
    // columns of one coil wider than one UMMA (ny_pad > 256): each tile is
    // n_parts sub-tiles of pw = 256 columns, one accumulator each, whose row
    // sums the epilogue adds before it writes y; otherwise n_parts = 1 and
    // pw = ny_pad (the whole coil, cpt coils per tile)
    int n_parts, pw;
    int num_units;  // m_tiles * n_tiles
    uint32_t tmem_cols;
    const DevScalars *sc;
    int skip;
    int *status;
};

struct AdjParams {
    // partial images, part[c][j][ig][p][64] (pixel i = 64 ig + (i % 64) fastest,
    // then the k-space split p, the 64-pixel group ig, the column j, the coil)
    float2 *part;
    int ksplit, n_ig;
    // ny_pad here is the tile width (the UMMA N, at most 256).  An image wider
    // than that is covered by one launch per 256-column part: part points at
    // the part's first column, b_row0 is its first conj(A_y) row and ny_lim
    // the number of its columns that lie inside the image.
    int nx, ny, ny_pad, nx_pad, nc, tiles_per_coil, m_tiles, kb_per_split, num_kb, ny_lim, b_row0;
    int stages, raw_stages;
    int n_acc, a_col0;  // accumulator buffers in TMEM; first TMEM column of the A slots
    int num_units;      // m_tiles * ksplit
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

// For U = (ur, ui): the Re-row word (ur, -ui) and the Im-row word (ui, ur) of
// the real embedding, hi and lo.  Negation and swapping are exact in bf16, so
// the four words come from one split of (ur, ui).
__device__ __forceinline__ void split_embed(float2 u, uint32_t &hre, uint32_t &lre, uint32_t &him, uint32_t &lim) {
    uint32_t h, l;
    split2(u.x, u.y, h, l);
    hre = h ^ 0x80000000u;
    lre = l ^ 0x80000000u;
    him = __byte_perm(h, 0, 0x1032);
    lim = __byte_perm(l, 0, 0x1032);
}

// Ring position: stage index and phase bit advance together.
struct Ring {
    int stage = 0;
    uint32_t phase = 0;
    __device__ __forceinline__ void next(int n) {
        if (++stage == n) {
            stage = 0;
            phase ^= 1u;
        }
    }
};

// ---------------------------------------------------------------------------
// Forward operand: B[(c*ny_pad + j)][2i + {0,1}] = (Re, Im) of S_c[i][j] x[i][j],
// split into hi/lo (BF16x3) or rounded to TF32 (t32); block (32, 8) over a
// 32 x 32 (i, j) tile of coil blockIdx.z, transposed through shared memory.
template <bool kTf32>
__global__ void fwd_operand_kernel(const float2 *__restrict__ x, const float2 *__restrict__ maps,
                                   uint32_t *__restrict__ hi, uint32_t *__restrict__ lo, uint2 *__restrict__ t32,
                                   int nx, int ny, int ny_pad, int kx, const DevScalars *sc, int skip) {
    if (should_skip(sc, skip)) return;
    __shared__ float2 ts[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32, c = blockIdx.z;
    const size_t npix = (size_t)nx * ny;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = i0 + ty + 8 * q, j = j0 + tx;
        ts[ty + 8 * q][tx] = (i < nx && j < ny)
                                 ? cmul(maps[c * npix + (size_t)i * ny + j], x[(size_t)i * ny + j])
                                 : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = j0 + ty + 8 * q, i = i0 + tx;
        if (i < nx && j < ny) {
            const float2 v = ts[tx][ty + 8 * q];
            const size_t off = ((size_t)c * ny_pad + j) * (kx / 2) + i;
            if constexpr (kTf32) {
                t32[off] = make_uint2(tf32_bits(v.x), tf32_bits(v.y));
            } else {
                uint32_t h, l;
                split2(v.x, v.y, h, l);
                hi[off] = h;
                lo[off] = l;
            }
        }
    }
}

// ---------------------------------------------------------------------------
template <bool kTf32>
__global__ void __launch_bounds__(kFwdThreads, 1)
    fwd_tc_kernel(const __grid_constant__ CUtensorMap ta_hi, const __grid_constant__ CUtensorMap ta_lo,
                  const __grid_constant__ CUtensorMap tb_hi, const __grid_constant__ CUtensorMap tb_lo,
                  const __grid_constant__ CUtensorMap t_ay, const FwdParams P) {
    if (should_skip(P.sc, P.skip)) return;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = align1024(smem_raw);
    const uint32_t b_bytes = (uint32_t)P.block_n * 128u;
    const uint32_t stage_bytes = 2u * kTileBytesA + 2u * b_bytes;
    const int S = P.stages, R = P.ay_stages;
    uint8_t *ay_ring = smem + (size_t)S * stage_bytes;
    uint64_t *bars = (uint64_t *)(ay_ring + (size_t)R * kAyChunkBytes);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + S);
    const uint32_t yfull0 = smem_u32(bars + 2 * S), yempty0 = smem_u32(bars + 2 * S + R);
    const uint32_t tfull0 = smem_u32(bars + 2 * S + 2 * R), tempty0 = smem_u32(bars + 2 * S + 2 * R + 2);
    const uint32_t fin = smem_u32(bars + 2 * S + 2 * R + 4);
    uint32_t *tmem_slot = (uint32_t *)(bars + 2 * S + 2 * R + 5);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_jc = (P.pw + 31) / 32;  // A_y chunks of 32 columns per sub-tile

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);  // released by the UMMA commit
        }
        for (int r = 0; r < R; ++r) {
            mbar_init(yfull0 + 8 * r, 1);
            mbar_init(yempty0 + 8 * r, 128);
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
        prefetch_tensormap(&t_ay);
    }
    fence_before_sync();
    __syncthreads();  // barriers initialised and TMEM allocated before any role starts
    fence_after_sync();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // operand loader: the unit's A tile and B rows
        if (lane == 0) {
            Ring rg;
            uint32_t issued_phase[4] = {0, 0, 0, 0};
            int issued_mask = 0;
            for (int g = blockIdx.x; g < P.num_units && !*abort_flag; g += gridDim.x) {
                const int m_blk = g / P.n_tiles, n_blk = g % P.n_tiles;
                for (int part = 0; part < P.n_parts; ++part)
                for (int kb = 0; kb < P.num_kb; ++kb) {
                    const int b_row = n_blk * P.cpt * P.ny_pad + part * P.pw;
                    if (!mbar_wait(empty0 + 8 * rg.stage, rg.phase ^ 1, abort_flag, kWaitLimitNs)) break;
                    const uint32_t sbase = smem_u32(smem + (size_t)rg.stage * stage_bytes);
                    const uint32_t fb = full0 + 8 * rg.stage;
                    mbar_arrive_expect_tx(fb, stage_bytes);
                    // BF16x3: hi and lo rows of K block kb; TF32: its two 32-element halves
                    const int x0 = kb * kTcBlockK, x1 = x0 + (kTf32 ? kTcBlockK / 2 : 0);
                    tma_load_2d(sbase, &ta_hi, fb, x0, m_blk * kTcBlockM);
                    tma_load_2d(sbase + kTileBytesA, &ta_lo, fb, x1, m_blk * kTcBlockM);
                    const uint32_t bh = sbase + 2 * kTileBytesA;
                    tma_load_2d(bh, &tb_hi, fb, x0, b_row);
                    tma_load_2d(bh + b_bytes, &tb_lo, fb, x1, b_row);
                    issued_phase[rg.stage] = rg.phase;
                    issued_mask |= 1 << rg.stage;
                    rg.next(S);
                }
            }
            if (*abort_flag)
                for (int s = 0; s < S; ++s)
                    if (issued_mask & (1 << s)) drain_wait(full0 + 8 * s, issued_phase[s]);
        }
    } else if (warp == 1) {
        // UMMA issuer
        if (lane == 0) {
            const uint32_t idesc = kTf32 ? idesc_tf32_f32(kTcBlockM, P.block_n) : idesc_bf16_f32(kTcBlockM, P.block_n);
            Ring rg;
            int lt = 0;
            bool issued_any = false;
            // one accumulator per (unit, sub-tile), in the loader's order
            for (int t = 0;; ++t, ++lt) {
                if ((int)blockIdx.x + (t / P.n_parts) * (int)gridDim.x >= P.num_units) break;
                const int a = lt & 1;
                const uint32_t ap = (lt >> 1) & 1;
                if (!mbar_wait(tempty0 + 8 * a, ap ^ 1, abort_flag, kWaitLimitNs)) break;
                fence_after_sync();
                const uint32_t d_tmem = tmem_base + (uint32_t)(a * P.block_n);
                bool ok = true;
                for (int kb = 0; kb < P.num_kb; ++kb) {
                    if (!mbar_wait(full0 + 8 * rg.stage, rg.phase, abort_flag, kWaitLimitNs)) {
                        ok = false;
                        break;
                    }
                    fence_after_sync();
                    const uint32_t sa_hi = smem_u32(smem + (size_t)rg.stage * stage_bytes);
                    const uint32_t sa_lo = sa_hi + kTileBytesA;
                    const uint32_t sb_hi = sa_hi + 2 * kTileBytesA;
                    const uint32_t sb_lo = sb_hi + b_bytes;
                    if constexpr (kTf32) {
                        // eight K steps of 8 TF32 elements: four in each 128-byte half
#pragma unroll
                        for (int kk = 0; kk < 8; ++kk) {
                            const uint32_t off = (kk & 3) * 32;
                            const uint64_t da = sdesc_kmajor_sw128((kk < 4 ? sa_hi : sa_lo) + off);
                            const uint64_t db = sdesc_kmajor_sw128((kk < 4 ? sb_hi : sb_lo) + off);
                            umma_tf32(d_tmem, da, db, idesc, (kb | kk) != 0);
                        }
                    } else {
#pragma unroll
                        for (int kk = 0; kk < kTcBlockK / 16; ++kk) {
                            const uint32_t off = kk * 32;
                            const uint64_t dah = sdesc_kmajor_sw128(sa_hi + off), dal = sdesc_kmajor_sw128(sa_lo + off);
                            const uint64_t dbh = sdesc_kmajor_sw128(sb_hi + off), dbl = sdesc_kmajor_sw128(sb_lo + off);
                            umma_f16(d_tmem, dah, dbh, idesc, (kb | kk) != 0);
                            umma_f16(d_tmem, dah, dbl, idesc, 1u);
                            umma_f16(d_tmem, dal, dbh, idesc, 1u);
                        }
                    }
                    issued_any = true;
                    umma_commit(empty0 + 8 * rg.stage);  // the stage is free once these UMMAs completed
                    rg.next(S);
                }
                if (!ok) break;
                umma_commit(tfull0 + 8 * a);
            }
            // all UMMAs and their commits have landed before the block frees TMEM
            if (issued_any) {
                umma_commit(fin);
                drain_wait(fin, 0);
            }
        }
    } else if (warp == 2) {
        // A_y tile loader: for each tile, the 64-sample x 32-column chunks in column order
        if (lane == 0) {
            Ring rg;
            uint32_t issued_phase[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            int issued_mask = 0;
            for (int g = blockIdx.x; g < P.num_units && !*abort_flag; g += gridDim.x) {
                const int m_blk = g / P.n_tiles;
                for (int part = 0; part < P.n_parts; ++part)
                for (int jc = 0; jc < n_jc; ++jc) {
                    if (!mbar_wait(yempty0 + 8 * rg.stage, rg.phase ^ 1, abort_flag, kWaitLimitNs)) break;
                    const uint32_t yb = yfull0 + 8 * rg.stage;
                    mbar_arrive_expect_tx(yb, kAyChunkBytes);
                    tma_load_2d(smem_u32(ay_ring + (size_t)rg.stage * kAyChunkBytes), &t_ay, yb,
                                m_blk * (kTcBlockM), part * P.pw + jc * 32);
                    issued_phase[rg.stage] = rg.phase;
                    issued_mask |= 1 << rg.stage;
                    rg.next(R);
                }
            }
            if (*abort_flag)
                for (int r = 0; r < R; ++r)
                    if (issued_mask & (1 << r)) drain_wait(yfull0 + 8 * r, issued_phase[r]);
        }
    } else {
        // epilogue: warp (w % 4) reads TMEM lanes [32 (w % 4), 32 (w % 4) + 32)
        const int wq = warp & 3;
        const int row = wq * 32 + lane;
        const int o = row & 1, kk_local = row >> 1;
        const uint32_t lane_base = (uint32_t)(wq * 32) << 16;
        Ring yr;
        int lt = 0;
        float s0[kMaxCoilsPerTile], s1[kMaxCoilsPerTile];  // row sums, carried across a tile's sub-tiles
        for (int t = 0;; ++t, ++lt) {
            const int g = (int)blockIdx.x + (t / P.n_parts) * (int)gridDim.x, part = t % P.n_parts;
            if (g >= P.num_units) break;
            const int a = lt & 1;
            const uint32_t ap = (lt >> 1) & 1;
            if (!__all_sync(0xffffffffu, mbar_wait(tfull0 + 8 * a, ap, abort_flag, kWaitLimitNs))) break;
            fence_after_sync();
            const int m_blk = g / P.n_tiles, n_blk = g % P.n_tiles;
            if (part == 0) {
#pragma unroll
                for (int cs = 0; cs < kMaxCoilsPerTile; ++cs) s0[cs] = s1[cs] = 0.f;
            }
            bool ok = true;
            for (int jc = 0; jc < n_jc; ++jc) {
                if (!__all_sync(0xffffffffu, mbar_wait(yfull0 + 8 * yr.stage, yr.phase, abort_flag, kWaitLimitNs))) {
                    ok = false;
                    break;
                }
                // A_y[k][j] of this thread's sample at column j = 32 jc + q: smem [q][k_local];
                // read once per chunk, used by every coil of the tile.  The Re
                // row (o = 0) needs (Re, Im) of A_y, the Im row (-Im, Re).
                const float2 *ay = reinterpret_cast<const float2 *>(ay_ring + (size_t)yr.stage * kAyChunkBytes) +
                                   kk_local;
                float c0[32], c1[32];
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    const float2 w = ay[q * 64];
                    c0[q] = o ? -w.y : w.x;
                    c1[q] = o ? w.x : w.y;
                }
                const bool full32 = P.pw - 32 * jc >= 32;
#pragma unroll
                for (int cs = 0; cs < kMaxCoilsPerTile; ++cs) {
                    if (cs < P.cpt) {
                        const uint32_t col = (uint32_t)(a * P.block_n + cs * P.pw + 32 * jc);
                        float v[32];
                        if (full32) {
                            tmem_ld_32cols(tmem_base + lane_base + col, v);
                        } else {
                            float v16[16];
                            tmem_ld_16cols(tmem_base + lane_base + col, v16);
#pragma unroll
                            for (int q = 0; q < 32; ++q) v[q] = q < 16 ? v16[q] : 0.f;
                        }
#pragma unroll
                        for (int q = 0; q < 32; ++q) {
                            s0[cs] = fmaf(v[q], c0[q], s0[cs]);
                            s1[cs] = fmaf(v[q], c1[q], s1[cs]);
                        }
                    }
                }
                mbar_arrive(yempty0 + 8 * yr.stage);
                yr.next(R);
            }
            fence_before_sync();
            mbar_arrive(tempty0 + 8 * a);
            if (!ok) break;
            if (part != P.n_parts - 1) continue;  // the coil's row sums are complete after its last sub-tile
            const int kappa = m_blk * (kTcBlockM / 2) + kk_local;
#pragma unroll
            for (int cs = 0; cs < kMaxCoilsPerTile; ++cs) {
                if (cs < P.cpt) {
                    const float r0 = s0[cs] + __shfl_xor_sync(0xffffffffu, s0[cs], 1);
                    const float r1 = s1[cs] + __shfl_xor_sync(0xffffffffu, s1[cs], 1);
                    const int c = n_blk * P.cpt + cs;
                    if (o == 0 && kappa < P.nk && c < P.nc) P.y[(size_t)c * P.y_ld + kappa] = make_float2(r0, r1);
                }
            }
        }
    }

    fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();  // lane 0 ran the issue loop alone; dealloc is .sync.aligned
        fence_after_sync();
        tmem_dealloc(tmem_base, P.tmem_cols);
    }
    if (threadIdx.x == 0 && *abort_flag) atomicExch(P.status, kStatusTimeout);
}

// ---------------------------------------------------------------------------
// Adjoint product.  The dynamic operand U (real-embedded, hi/lo) is written by
// the producer warps straight into tensor memory with tcgen05.st; the UMMAs
// read it from there (A in TMEM) and only the static conj(A_y) operand goes
// through shared memory.  TMEM columns: n_acc accumulators of ny_pad columns,
// then `stages` A slots of 64 columns (BF16x3: 32 hi, 32 lo, two bf16 per
// column; TF32: the 64 K elements, one per column) starting at a_col0.
// kPx128 selects the pixel-row tile form (128 pixels, one TMEM lane each).
template <bool kTf32, bool kPx128>
__global__ void __launch_bounds__(kAdjThreads, 1)
    adj_tc_kernel(const __grid_constant__ CUtensorMap tb_hi, const __grid_constant__ CUtensorMap tb_lo,
                  const __grid_constant__ CUtensorMap t_axT, const __grid_constant__ CUtensorMap t_axQ,
                  const __grid_constant__ CUtensorMap t_y, const AdjParams P) {
    // t_axT: A_x^T (row pairs) or axP (pixel rows); t_axQ: axQ (pixel rows only)
    if (should_skip(P.sc, P.skip)) return;
    constexpr int kPx = kPx128 ? 128 : 64;  // pixels per M tile
    constexpr int kRawB = raw_bytes_for(kPx);
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = align1024(smem_raw);
    const uint32_t b_bytes = (uint32_t)P.ny_pad * 128u;
    const uint32_t stage_bytes = 2u * b_bytes;  // B hi, B lo
    const int S = P.stages, R = P.raw_stages, NA = P.n_acc;
    uint8_t *raw = smem + (size_t)S * stage_bytes;
    uint8_t *yraw = raw + (size_t)R * kRawB;
    uint64_t *bars = (uint64_t *)(yraw + (size_t)R * kRawYBytes);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + S);
    const uint32_t rfull0 = smem_u32(bars + 2 * S), rempty0 = smem_u32(bars + 2 * S + R);
    const uint32_t tfull0 = smem_u32(bars + 2 * S + 2 * R), tempty0 = smem_u32(bars + 2 * S + 2 * R + 2);
    const uint32_t fin = smem_u32(bars + 2 * S + 2 * R + 4);
    uint32_t *tmem_slot = (uint32_t *)(bars + 2 * S + 2 * R + 5);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // unit u: split p = u / m_tiles, tile m = u % m_tiles with the coil
    // fastest (m = ib * nc + c)

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full0 + 8 * s, kAdjProducers + 1);  // producer threads + the B loads' expect_tx arrival
            mbar_init(empty0 + 8 * s, 1);  // released by the UMMA commit
        }
        for (int r = 0; r < R; ++r) {
            mbar_init(rfull0 + 8 * r, 1);
            mbar_init(rempty0 + 8 * r, kAdjProducers);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(tfull0 + 8 * a, 1);
            mbar_init(tempty0 + 8 * a, 128);
        }
        mbar_init(fin, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == kAdjMmaWarp) {
        tmem_alloc(smem_u32(tmem_slot), P.tmem_cols);
        tmem_relinquish();
    }
    if (warp == kAdjLoaderWarp && lane == 0) {
        prefetch_tensormap(&tb_hi);
        prefetch_tensormap(&tb_lo);
        prefetch_tensormap(&t_axT);
        if (kPx128) prefetch_tensormap(&t_axQ);
        prefetch_tensormap(&t_y);
    }
    fence_before_sync();
    __syncthreads();  // barriers initialised and TMEM allocated before any role starts
    fence_after_sync();
    const uint32_t tmem_base = *tmem_slot;

    if (warp < kAdjProducerWarps) {
        // producers: warp w owns TMEM lanes [32 (w%4), 32 (w%4) + 32) and the
        // kSpw samples [kSpw kh, kSpw kh + kSpw) of each K block (kh = w/4).
        // Row pairs: lane l holds row r = 32 (w%4) + l of U's real embedding,
        // pixel ii = r/2, Re row (o = 0) or Im row (o = 1); the two threads of
        // a pixel each form half of the warp's products and swap halves.
        // Pixel rows: lane l holds pixel ii = r and forms all kSpw products.
        constexpr int kSpw = 128 / kAdjProducerWarps;  // samples per warp and K block
        constexpr int kCpt = kSpw / 4;                  // 16-byte chunks (two samples) per thread and row half
        const int q = warp & 3, kh = warp >> 2;
        const int half = (kSpw * kh) >> 4, chunk0 = ((kSpw * kh) & 15) >> 1;
        const int row = 32 * q + lane;
        const int ii = kPx128 ? row : row >> 1, o = kPx128 ? 0 : row & 1;
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        Ring rr, rs;
        uint32_t issued_phase[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int issued_mask = 0;
        // every branch below is warp-uniform: the waits' outcomes are agreed
        // on with __all_sync and the warp reconverges after the one-thread
        // TMA issue, because tcgen05.st / wait::st are .sync.aligned and a
        // warp that reached them diverged stored part of its lanes late
        for (int u = blockIdx.x; u < P.num_units; u += gridDim.x) {
            if (__any_sync(0xffffffffu, *abort_flag != 0)) break;
            const int p = u / P.m_tiles;
            const int kb0 = p * P.kb_per_split, kb1 = min(P.num_kb, kb0 + P.kb_per_split);
            bool ok = true;
            for (int kb = kb0; kb < kb1; ++kb) {
                const bool waited = mbar_wait(rfull0 + 8 * rr.stage, rr.phase, abort_flag, kWaitLimitNs) &&
                                    mbar_wait(empty0 + 8 * rs.stage, rs.phase ^ 1, abort_flag, kWaitLimitNs);
                if (!__all_sync(0xffffffffu, waited)) {
                    ok = false;
                    break;
                }
                const uint32_t fb = full0 + 8 * rs.stage;
                if (threadIdx.x == 0) {
                    // the stage's conj(A_y) rows, hi and lo
                    const uint32_t sb = smem_u32(smem + (size_t)rs.stage * stage_bytes);
                    mbar_arrive_expect_tx(fb, 2u * b_bytes);
                    const int x0 = kb * kTcBlockK, x1 = x0 + (kTf32 ? kTcBlockK / 2 : 0);
                    tma_load_2d(sb, &tb_hi, fb, x0, P.b_row0);
                    tma_load_2d(sb + b_bytes, &tb_lo, fb, x1, P.b_row0);
                    issued_phase[rs.stage] = rs.phase;
                    issued_mask |= 1 << rs.stage;
                }
                __syncwarp();
                // staged A_x^H half-row (128-byte swizzled, sixteen samples) and
                // y_c chunk: this thread's samples are chunks chunk0 + kCpt o + c
                const uint8_t *arow = raw + (size_t)rr.stage * kRawB + (kPx128 ? half * (kRawQ0 / 2) + (ii >> 4) * 128
                                                                               : half * (kRawB / 2) + ii * 128);
                const uint8_t *qrow = raw + (size_t)rr.stage * kRawB + kRawQ0 + half * (kRawB - kRawQ0) / 2 +
                                      (ii & 15) * 128;  // pixel rows only
                const float4 *yv4 =
                    reinterpret_cast<const float4 *>(yraw + (size_t)rr.stage * kRawYBytes + half * 128);
                const uint32_t acol = (uint32_t)(P.a_col0 + 64 * rs.stage + (kTf32 ? 2 * kSpw : kSpw) * kh);
                if constexpr (kPx128) {
                    // this thread's kSpw samples: (Re U, Im U) in sample order, with
                    // U = conj(P Q) y = conj(P) (conj(Q) y)
                    uint32_t hw[kSpw], lw[kSpw];  // TF32: hw[] and lw[] are the first and second kSpw words
#pragma unroll
                    for (int c = 0; c < 2 * kCpt; ++c) {
                        const int chunk = chunk0 + c;
                        const float4 pv = *reinterpret_cast<const float4 *>(arow + ((chunk ^ ((ii >> 4) & 7)) << 4));
                        const float4 qv = *reinterpret_cast<const float4 *>(qrow + ((chunk ^ (ii & 7)) << 4));
                        const float4 yv = yv4[chunk];
                        const float2 u0 = cmulc(make_float2(pv.x, pv.y),
                                                cmulc(make_float2(qv.x, qv.y), make_float2(yv.x, yv.y)));
                        const float2 u1 = cmulc(make_float2(pv.z, pv.w),
                                                cmulc(make_float2(qv.z, qv.w), make_float2(yv.z, yv.w)));
                        if constexpr (kTf32) {
                            const uint32_t w0 = tf32_bits(u0.x), w1 = tf32_bits(u0.y);
                            const uint32_t w2 = tf32_bits(u1.x), w3 = tf32_bits(u1.y);
                            if (c < kCpt) {
                                hw[4 * c] = w0;
                                hw[4 * c + 1] = w1;
                                hw[4 * c + 2] = w2;
                                hw[4 * c + 3] = w3;
                            } else {
                                lw[4 * (c - kCpt)] = w0;
                                lw[4 * (c - kCpt) + 1] = w1;
                                lw[4 * (c - kCpt) + 2] = w2;
                                lw[4 * (c - kCpt) + 3] = w3;
                            }
                        } else {
                            split2(u0.x, u0.y, hw[2 * c], lw[2 * c]);
                            split2(u1.x, u1.y, hw[2 * c + 1], lw[2 * c + 1]);
                        }
                    }
                    mbar_arrive(rempty0 + 8 * rr.stage);
                    rr.next(R);
                    // TF32: 2 kSpw consecutive columns; BF16x3: kSpw hi columns, kSpw lo columns 32 on
                    tmem_st_cols<kSpw>(tmem_base + lane_base + acol, hw);
                    tmem_st_cols<kSpw>(tmem_base + lane_base + acol + (kTf32 ? kSpw : 32), lw);
                } else if constexpr (kTf32) {
                    // this thread's 2 kCpt samples: Re-row pairs (ur, -ui) and Im-row pairs (ui, ur)
                    uint32_t rw[4 * kCpt], iw[4 * kCpt];
#pragma unroll
                    for (int c = 0; c < kCpt; ++c) {
                        const int chunk = chunk0 + kCpt * o + c;
                        const float4 av = *reinterpret_cast<const float4 *>(arow + ((chunk ^ (ii & 7)) << 4));
                        const float4 yv = yv4[chunk];
                        const float2 u0 = cmulc(make_float2(av.x, av.y), make_float2(yv.x, yv.y));
                        const float2 u1 = cmulc(make_float2(av.z, av.w), make_float2(yv.z, yv.w));
                        const uint32_t r0 = tf32_bits(u0.x), i0 = tf32_bits(u0.y);
                        const uint32_t r1 = tf32_bits(u1.x), i1 = tf32_bits(u1.y);
                        rw[4 * c] = r0;
                        rw[4 * c + 1] = i0 ^ 0x80000000u;
                        rw[4 * c + 2] = r1;
                        rw[4 * c + 3] = i1 ^ 0x80000000u;
                        iw[4 * c] = i0;
                        iw[4 * c + 1] = r0;
                        iw[4 * c + 2] = i1;
                        iw[4 * c + 3] = r1;
                    }
                    mbar_arrive(rempty0 + 8 * rr.stage);
                    rr.next(R);
                    // the Re-row thread (o = 0) keeps its Re pairs and receives the
                    // partner's; the Im-row thread likewise, in sample order
                    uint32_t w[2 * kSpw];
#pragma unroll
                    for (int e = 0; e < 4 * kCpt; ++e) {
                        const uint32_t rcv = __shfl_xor_sync(0xffffffffu, o ? rw[e] : iw[e], 1);
                        w[e] = o ? rcv : rw[e];
                        w[4 * kCpt + e] = o ? iw[e] : rcv;
                    }
                    tmem_st_cols<2 * kSpw>(tmem_base + lane_base + acol, w);
                } else {
                    uint32_t hre[2 * kCpt], lre[2 * kCpt], him[2 * kCpt], lim[2 * kCpt];
#pragma unroll
                    for (int c = 0; c < kCpt; ++c) {
                        const int chunk = chunk0 + kCpt * o + c;
                        const float4 av = *reinterpret_cast<const float4 *>(arow + ((chunk ^ (ii & 7)) << 4));
                        const float4 yv = yv4[chunk];
                        split_embed(cmulc(make_float2(av.x, av.y), make_float2(yv.x, yv.y)), hre[2 * c],
                                    lre[2 * c], him[2 * c], lim[2 * c]);
                        split_embed(cmulc(make_float2(av.z, av.w), make_float2(yv.z, yv.w)), hre[2 * c + 1],
                                    lre[2 * c + 1], him[2 * c + 1], lim[2 * c + 1]);
                    }
                    mbar_arrive(rempty0 + 8 * rr.stage);
                    rr.next(R);
                    // the Re-row thread keeps its Re words and receives the
                    // partner's; the Im-row thread likewise, in sample order
                    uint32_t hi[kSpw], lo[kSpw];
#pragma unroll
                    for (int e = 0; e < 2 * kCpt; ++e) {
                        const uint32_t rh = __shfl_xor_sync(0xffffffffu, o ? hre[e] : him[e], 1);
                        const uint32_t rl = __shfl_xor_sync(0xffffffffu, o ? lre[e] : lim[e], 1);
                        hi[e] = o ? rh : hre[e];
                        lo[e] = o ? rl : lre[e];
                        hi[2 * kCpt + e] = o ? him[e] : rh;
                        lo[2 * kCpt + e] = o ? lim[e] : rl;
                    }
                    tmem_st_cols<kSpw>(tmem_base + lane_base + acol, hi);
                    tmem_st_cols<kSpw>(tmem_base + lane_base + acol + 32, lo);
                }
                tmem_wait_st();
                fence_before_sync();
                mbar_arrive(fb);
                rs.next(S);
            }
            if (!ok) break;
        }
        if (threadIdx.x == 0 && *abort_flag)
            for (int s = 0; s < S; ++s)
                if (issued_mask & (1 << s)) drain_wait(full0 + 8 * s, issued_phase[s]);
    } else if (warp == kAdjMmaWarp) {
        // UMMA issuer
        if (lane == 0) {
            const uint32_t idesc = kTf32 ? idesc_tf32_f32(kTcBlockM, P.ny_pad) : idesc_bf16_f32(kTcBlockM, P.ny_pad);
            Ring rg;
            int lt = 0;
            bool issued_any = false;
            for (int u = blockIdx.x; u < P.num_units; u += gridDim.x, ++lt) {
                const int p = u / P.m_tiles;
                const int kb0 = p * P.kb_per_split, kb1 = min(P.num_kb, kb0 + P.kb_per_split);
                const int a = lt % NA;
                const uint32_t ap = (lt / NA) & 1;
                if (!mbar_wait(tempty0 + 8 * a, ap ^ 1, abort_flag, kWaitLimitNs)) break;
                fence_after_sync();
                const uint32_t d_tmem = tmem_base + (uint32_t)(a * P.ny_pad);
                bool ok = true;
                for (int kb = kb0; kb < kb1; ++kb) {
                    if (!mbar_wait(full0 + 8 * rg.stage, rg.phase, abort_flag, kWaitLimitNs)) {
                        ok = false;
                        break;
                    }
                    fence_after_sync();
                    const uint32_t ta_hi = tmem_base + (uint32_t)(P.a_col0 + 64 * rg.stage);
                    const uint32_t ta_lo = ta_hi + 32;
                    const uint32_t sb_hi = smem_u32(smem + (size_t)rg.stage * stage_bytes);
                    const uint32_t sb_lo = sb_hi + b_bytes;
                    if constexpr (kTf32) {
                        // K element e of the block in TMEM column e; B halves of 32 elements
#pragma unroll
                        for (int kk = 0; kk < 8; ++kk) {
                            const uint64_t db = sdesc_kmajor_sw128((kk < 4 ? sb_hi : sb_lo) + (kk & 3) * 32);
                            umma_tf32_tmem_a(d_tmem, ta_hi + 8 * kk, db, idesc, (kb != kb0 || kk != 0) ? 1u : 0u);
                        }
                    } else {
#pragma unroll
                        for (int kk = 0; kk < kTcBlockK / 16; ++kk) {
                            const uint64_t dbh = sdesc_kmajor_sw128(sb_hi + kk * 32),
                                           dbl = sdesc_kmajor_sw128(sb_lo + kk * 32);
                            umma_f16_tmem_a(d_tmem, ta_hi + 8 * kk, dbh, idesc, (kb != kb0 || kk != 0) ? 1u : 0u);
                            umma_f16_tmem_a(d_tmem, ta_hi + 8 * kk, dbl, idesc, 1u);
                            umma_f16_tmem_a(d_tmem, ta_lo + 8 * kk, dbh, idesc, 1u);
                        }
                    }
                    issued_any = true;
                    umma_commit(empty0 + 8 * rg.stage);  // the stage is free once these UMMAs completed
                    rg.next(S);
                }
                if (!ok) break;
                umma_commit(tfull0 + 8 * a);
            }
            // all UMMAs and their commits have landed before the block frees TMEM
            if (issued_any) {
                umma_commit(fin);
                drain_wait(fin, 0);
            }
        }
    } else if (warp == kAdjLoaderWarp) {
        // loader of the A_x^H tiles (two 128-byte-swizzled halves) and the y_c chunks
        if (lane == 0) {
            Ring rg;
            uint32_t issued_phase[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            int issued_mask = 0;
            for (int u = blockIdx.x; u < P.num_units && !*abort_flag; u += gridDim.x) {
                const int p = u / P.m_tiles, m = u % P.m_tiles;
                const int c = m % P.nc, ib = m / P.nc;
                const int kb0 = p * P.kb_per_split, kb1 = min(P.num_kb, kb0 + P.kb_per_split);
                for (int kb = kb0; kb < kb1; ++kb) {
                    if (!mbar_wait(rempty0 + 8 * rg.stage, rg.phase ^ 1, abort_flag, kWaitLimitNs)) break;
                    const uint32_t rb = rfull0 + 8 * rg.stage;
                    const uint32_t dst = smem_u32(raw + (size_t)rg.stage * kRawB);
                    mbar_arrive_expect_tx(rb, kRawB + kRawYBytes);
                    if constexpr (kPx128) {
                        tma_load_2d(dst, &t_axT, rb, kb * 64, ib * 8);
                        tma_load_2d(dst + kRawQ0 / 2, &t_axT, rb, kb * 64 + 32, ib * 8);
                        tma_load_2d(dst + kRawQ0, &t_axQ, rb, kb * 64, 0);
                        tma_load_2d(dst + kRawQ0 + (kRawB - kRawQ0) / 2, &t_axQ, rb, kb * 64 + 32, 0);
                    } else {
                        tma_load_2d(dst, &t_axT, rb, kb * 64, ib * kPx);
                        tma_load_2d(dst + kRawB / 2, &t_axT, rb, kb * 64 + 32, ib * kPx);
                    }
                    tma_load_2d(smem_u32(yraw + (size_t)rg.stage * kRawYBytes), &t_y, rb, kb * 64, c);
                    issued_phase[rg.stage] = rg.phase;
                    issued_mask |= 1 << rg.stage;
                    rg.next(R);
                }
            }
            if (*abort_flag)
                for (int r = 0; r < R; ++r)
                    if (issued_mask & (1 << r)) drain_wait(rfull0 + 8 * r, issued_phase[r]);
        }
    } else {
        // epilogue: the four warps after the UMMA warp; TMEM lane quadrant = warp % 4
        const int wq = warp & 3;
        const int row = wq * 32 + lane;
        const int ii = kPx128 ? row : row >> 1, o = kPx128 ? 0 : row & 1;
        const uint32_t lane_base = (uint32_t)(wq * 32) << 16;
        int lt = 0;
        for (int u = blockIdx.x; u < P.num_units; u += gridDim.x, ++lt) {
            const int a = lt % NA;
            const uint32_t ap = (lt / NA) & 1;
            if (!__all_sync(0xffffffffu, mbar_wait(tfull0 + 8 * a, ap, abort_flag, kWaitLimitNs))) break;
            fence_after_sync();
            const int p = u / P.m_tiles, m = u % P.m_tiles;
            const int c = m % P.nc, ib = m / P.nc;
            const int i = ib * kPx + ii;
            const uint32_t col0 = (uint32_t)(a * P.ny_pad);
            const size_t js = (size_t)P.n_ig * P.ksplit * 64;  // between columns j of the partials
            float2 *pix = P.part + (size_t)c * P.ny * js + (size_t)(i >> 6) * P.ksplit * 64 + (size_t)p * 64 + (i & 63);
            if constexpr (kPx128) {
                // columns 2j, 2j+1 = Re, Im of image column j (UMMA N = 2 ny_pad, a multiple of 32)
                for (int jc = 0; jc < P.ny_pad; jc += 32) {
                    float v[32];
                    tmem_ld_32cols(tmem_base + lane_base + col0 + jc, v);
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int j = jc / 2 + q;
                        if (j < P.ny_lim) pix[(size_t)j * js] = make_float2(v[2 * q], v[2 * q + 1]);
                    }
                }
                fence_before_sync();
                mbar_arrive(tempty0 + 8 * a);
                continue;
            }
            float *dst = reinterpret_cast<float *>(pix) + o;
            const size_t jstride = 2 * js;
            int jc = 0;
            for (; jc + 32 <= P.ny_pad; jc += 32) {
                float v[32];
                tmem_ld_32cols(tmem_base + lane_base + col0 + jc, v);
#pragma unroll
                for (int q = 0; q < 32; ++q)
                    if (jc + q < P.ny_lim) dst[(size_t)(jc + q) * jstride] = v[q];
            }
            if (jc < P.ny_pad) {
                float v[16];
                tmem_ld_16cols(tmem_base + lane_base + col0 + jc, v);
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    if (jc + q < P.ny_lim) dst[(size_t)(jc + q) * jstride] = v[q];
            }
            fence_before_sync();
            mbar_arrive(tempty0 + 8 * a);
        }
    }

    fence_before_sync();
    __syncthreads();
    if (warp == kAdjMmaWarp) {
        __syncwarp();  // lane 0 ran the issue loop alone; dealloc is .sync.aligned
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

// 2-D tensor [rows][cols] (cols contiguous) of `elem`-byte elements, box = box_cols x box_rows.
bool make_map(CUtensorMap *m, CUtensorMapDataType type, int elem, void *base, uint64_t cols, uint64_t rows,
              uint32_t box_cols, uint32_t box_rows, CUtensorMapSwizzle swz) {
    EncodeTiledFn fn = get_encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {cols * (uint64_t)elem};
    cuuint32_t box[2] = {box_cols, box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(m, type, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_bf16_map(CUtensorMap *m, void *base, uint64_t cols, uint64_t rows, uint32_t box_rows) {
    return make_map(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, cols, rows, kTcBlockK, box_rows,
                    CU_TENSOR_MAP_SWIZZLE_128B);
}

// TF32 operand matrix (FP32 words): boxes of 32 elements (128 bytes) x box_rows.
bool make_tf32_map(CUtensorMap *m, void *base, uint64_t cols, uint64_t rows, uint32_t box_rows) {
    return make_map(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, cols, rows, kTcBlockK / 2, box_rows,
                    CU_TENSOR_MAP_SWIZZLE_128B);
}

// hi/lo maps of one operand: two BF16 matrices, or the same TF32 map twice.
bool make_operand_maps(const mri_plan *p, CUtensorMap *hi, CUtensorMap *lo, void *bhi, void *blo, void *t32,
                       uint64_t cols, uint64_t rows, uint32_t box_rows) {
    if (p->precision == MRI_TF32) {
        if (!make_tf32_map(hi, t32, cols, rows, box_rows)) return false;
        *lo = *hi;
        return true;
    }
    return make_bf16_map(hi, bhi, cols, rows, box_rows) && make_bf16_map(lo, blo, cols, rows, box_rows);
}

uint32_t tmem_cols_for(int cols) {
    uint32_t n = 32;
    while ((int)n < cols) n <<= 1;
    return n;
}

// shared-memory plans: (operand stages, secondary ring stages, bytes)
// The operand stages of either product: p->fwd_stages / p->adj_stages when
// set (the autotuner's choice, 2..4), else as many as fit (at most 4).
void fwd_smem_plan(const mri_plan *p, int *stages, int *ay_stages, size_t *bytes) {
    const int stage = 2 * kTileBytesA + 2 * p->fwd_block_n * 128;
    int r = 2;
    int s = std::min(p->fwd_stages > 0 ? p->fwd_stages : 4, (kMaxSmem - kSmemSlack - r * kAyChunkBytes) / stage);
    if (s >= 3 && kMaxSmem - kSmemSlack - s * stage >= 3 * kAyChunkBytes) r = 3;
    *stages = s;
    *ay_stages = r;
    *bytes = (size_t)kSmemSlack + (size_t)s * stage + (size_t)r * kAyChunkBytes;
}

void adj_smem_plan(const mri_plan *p, int *stages, int *raw_stages, size_t *bytes, int *n_acc = nullptr,
                   int *a_col0 = nullptr) {
    // shared memory holds the B (conj A_y) stages and the raw A_x^H / y ring;
    // TMEM holds the accumulators and one 64-column A slot per stage
    const int bn = p->adj_block_n;  // UMMA N: conj(A_y) operand rows per tile
    const int stage = 2 * bn * 128;
    const int raw = raw_bytes_for(p->adj_tile_px) + kRawYBytes;
    int s = p->adj_stages > 0 ? p->adj_stages : 4, r = 0, na = 2, col0 = 0;
    for (; s >= 2; --s) {
        na = (round_up(2 * bn, 64) + 64 * s <= 512) ? 2 : 1;
        col0 = round_up(na * bn, 64);
        if (col0 + 64 * s > 512) continue;
        r = std::min(6, (kMaxSmem - kSmemSlack - s * stage) / raw);
        if (r >= (s > 2 ? 3 : 2)) break;
    }
    *stages = s;
    *raw_stages = r;
    *bytes = (size_t)kSmemSlack + (size_t)s * stage + (size_t)r * raw;
    if (n_acc) *n_acc = na;
    if (a_col0) *a_col0 = col0;
}

// Column parts of the adjoint, one launch each: 256-column parts of a wider
// image in the row-pair form, always one in the pixel-row form.
int adj_parts(const mri_plan *p) { return p->adj_tile_px == 128 ? 1 : p->ny_pad / p->adj_block_n; }

// The adjoint kernel instantiation for the plan's precision and tile form.
decltype(&adj_tc_kernel<false, false>) adj_kernel_for(const mri_plan *p) {
    const bool w = p->adj_tile_px == 128;
    if (p->precision == MRI_TF32) return w ? adj_tc_kernel<true, true> : adj_tc_kernel<true, false>;
    return w ? adj_tc_kernel<false, true> : adj_tc_kernel<false, false>;
}

void fwd_set_coils_per_tile(mri_plan *p, int cpt) {
    p->fwd_coils_per_tile = cpt;
    p->fwd_block_n = p->ny_pad > 256 ? 256 : cpt * p->ny_pad;
    p->fwd_n_tiles = ceil_div(p->nc, cpt);
}

}  // namespace

int tc_max_coils_per_tile(const mri_plan *p) {
    return std::min(std::min(kMaxCoilsPerTile, p->nc), std::max(1, 256 / p->ny_pad));
}

bool tc_supported(const mri_plan *p, std::string *why) {
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, p->device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, p->device);
    if (major != 10 || minor != 3) {
        *why = "needs an sm_103 GPU (found sm_" + std::to_string(major) + std::to_string(minor) + ")";
        return false;
    }
    if (p->ny > 1024) {
        *why = "ny up to 1024 is supported by the tensor-core kernels";
        return false;
    }
    if (!get_encode_fn()) {
        *why = "cuTensorMapEncodeTiled is not available from the driver";
        return false;
    }
    return true;
}

int tc_plan_tiling(mri_plan *p) {
    // forward: whole coils per N tile, or one coil in sub-tiles of 256
    // columns when it is wider than one UMMA (ny_pad is then a multiple of 256)
    const int n_tiles = ceil_div(p->nc, tc_max_coils_per_tile(p));
    fwd_set_coils_per_tile(p, ceil_div(p->nc, n_tiles));
    p->fwd_m_tiles = ceil_div(2 * p->nk, kTcBlockM);
    // adjoint: 64 pixels as 128 embedded rows, or 128 pixels as 128 rows
    // with the complex structure in B (when the image is at most 128 columns
    // wide and nx_pad is a multiple of 128), of one coil per M tile; split K
    // (k-space samples) so that the units fill the SMs evenly, with at most
    // kMaxKbPerSplit K blocks per split.  The tensor-core accumulation into
    // TMEM loses a roughly constant, same-signed fraction of an ulp of the
    // running sum per UMMA, so its relative error grows linearly with the
    // number of K blocks accumulated in one run (measured on the N=256,
    // 65536-sample adjoint: 2.5e-5 at 108 blocks, 1.4e-5 at 64, 7.3e-6 at 32,
    // 4.8e-6 at 16, against 3.9e-6 for exact accumulation of the same BF16x3
    // products); 32 blocks keep the operator within 1e-5 for any nk at a
    // cost of 6% on that adjoint (more partial images to write and sum)
    p->adj_tile_px = (p->nx_pad % 128 == 0 && p->ny_pad <= 128) ? 128 : 64;
    p->adj_m_tiles = p->nc * (p->nx_pad / p->adj_tile_px);
    p->adj_block_n = p->adj_tile_px == 128 ? 2 * p->ny_pad : std::min(p->ny_pad, 256);
    p->badj_rows = p->adj_tile_px == 128 ? 2 * p->ny_pad : p->ny_pad;
    const int n_parts = adj_parts(p);  // column parts of the image, one launch each
    const int num_kb = p->kk / kTcBlockK;
    long best_cost = -1;
    int best_split = 1;
    // the TF32 form's operand rounding (~4e-4) dwarfs the accumulation error of
    // long runs (2.5e-5 at 108 blocks), so it takes fewer, longer splits
    const int max_kb_per_split = p->precision == MRI_TF32 ? 4 * kMaxKbPerSplit : kMaxKbPerSplit;
    const int min_split = std::min(128, ceil_div(num_kb, max_kb_per_split));
    for (int split = min_split; split <= std::min(num_kb, 128); ++split) {
        const int per = ceil_div(num_kb, split);
        const int eff = ceil_div(num_kb, per);
        const long waves = n_parts * ceil_div(p->adj_m_tiles * eff, p->num_sms);  // one launch per part
        const long cost = waves * per + (long)eff / 8;  // makespan in K blocks, small penalty per split
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best_split = eff;
        }
    }
    p->ksplit_blocks = ceil_div(num_kb, best_split);
    p->ksplit = ceil_div(num_kb, p->ksplit_blocks);
    int s, r;
    size_t fb, ab;
    fwd_smem_plan(p, &s, &r, &fb);
    if (s < 2) return MRI_ERR_UNSUPPORTED;
    adj_smem_plan(p, &s, &r, &ab);
    if (s < 2 || r < 2) return MRI_ERR_UNSUPPORTED;
    return MRI_OK;
}

int tc_make_tensor_maps(mri_plan *p) {
    const uint64_t nkf = 2ull * p->nk_pad;  // floats per sample-indexed row
    bool ok = make_operand_maps(p, &p->tm_afwd_hi, &p->tm_afwd_lo, p->afwd_hi, p->afwd_lo, p->afwd_t, p->kx,
                                2ull * p->nk, kTcBlockM) &&
              (p->adj_tile_px == 128
                   ? make_map(&p->tm_axT, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, p->axP, nkf, p->nx_pad / 16, 32, 8,
                              CU_TENSOR_MAP_SWIZZLE_128B) &&
                         make_map(&p->tm_axQ, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, p->axQ, nkf, 16, 32, 16,
                                  CU_TENSOR_MAP_SWIZZLE_128B)
                   : make_map(&p->tm_axT, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, p->axT, nkf, p->nx, 32, 64,
                              CU_TENSOR_MAP_SWIZZLE_128B)) &&
              make_map(&p->tm_y, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, p->y, nkf, p->nc, 64, 1,
                       CU_TENSOR_MAP_SWIZZLE_NONE) &&
              make_map(&p->tm_ayT, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, p->ayT, nkf, p->ny, 128, 32,
                       CU_TENSOR_MAP_SWIZZLE_NONE);
    if (!ok) {
        set_error("cuTensorMapEncodeTiled failed");
        return MRI_ERR_CUDA;
    }
    cudaError_t e = cudaFuncSetAttribute(fwd_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fwd_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(adj_kernel_for(p), cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    if (e != cudaSuccess) {
        set_error(std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
        return MRI_ERR_CUDA;
    }
    return tc_set_tiles(p, 0, 0, 0);
}

namespace {

// Co-resident CTAs of a persistent kernel (one per SM with these shared-memory sizes).
template <typename Kern>
int resident_ctas(Kern kernel, int block, size_t smem, int num_sms) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem) != cudaSuccess || per_sm <= 0) {
        cudaGetLastError();
        per_sm = 1;
    }
    return std::max(1, per_sm) * num_sms;
}

}  // namespace

bool tc_tiles_valid(const mri_plan *p, int cpt, int fwd_stages, int adj_stages) {
    if (cpt < 1 || cpt > tc_max_coils_per_tile(p)) return false;
    if (fwd_stages < 2 || fwd_stages > 4 || adj_stages < 2 || adj_stages > 4) return false;
    mri_plan q = *p;  // shared-memory plans of the candidate configuration
    fwd_set_coils_per_tile(&q, cpt);
    q.fwd_stages = fwd_stages;
    q.adj_stages = adj_stages;
    int s, r;
    size_t bytes;
    fwd_smem_plan(&q, &s, &r, &bytes);
    if (s != fwd_stages) return false;
    adj_smem_plan(&q, &s, &r, &bytes);
    return s == adj_stages && r >= 2;
}

int tc_set_tiles(mri_plan *p, int cpt, int fwd_stages, int adj_stages) {
    if (cpt == 0) cpt = p->fwd_coils_per_tile;
    int s, r;
    size_t bytes;
    if (fwd_stages == 0 || adj_stages == 0) {  // keep the current (or the largest fitting) stage counts
        mri_plan q = *p;
        fwd_set_coils_per_tile(&q, cpt);
        fwd_smem_plan(&q, &s, &r, &bytes);
        if (fwd_stages == 0) fwd_stages = s;
        adj_smem_plan(&q, &s, &r, &bytes);
        if (adj_stages == 0) adj_stages = s;
    }
    if (!tc_tiles_valid(p, cpt, fwd_stages, adj_stages)) {
        set_error("tile configuration not valid for this shape");
        return MRI_ERR_INVALID;
    }
    fwd_set_coils_per_tile(p, cpt);
    p->fwd_stages = fwd_stages;
    p->adj_stages = adj_stages;
    bool ok = make_operand_maps(p, &p->tm_bfwd_hi, &p->tm_bfwd_lo, p->bfwd_hi, p->bfwd_lo, p->bfwd_t, p->kx,
                                (uint64_t)p->nc * p->ny_pad, p->fwd_block_n) &&
              make_operand_maps(p, &p->tm_badj_hi, &p->tm_badj_lo, p->badj_hi, p->badj_lo, p->badj_t, p->kk,
                                p->badj_rows, p->adj_block_n);
    if (!ok) {
        set_error("cuTensorMapEncodeTiled failed");
        return MRI_ERR_CUDA;
    }
    invalidate_graph(p);  // captured launches carry the old maps and tile shapes
    size_t fsm, asm_;
    fwd_smem_plan(p, &s, &r, &fsm);
    adj_smem_plan(p, &s, &r, &asm_);
    const bool t = p->precision == MRI_TF32;
    p->fwd_grid = t ? resident_ctas(fwd_tc_kernel<true>, kFwdThreads, fsm, p->num_sms)
                    : resident_ctas(fwd_tc_kernel<false>, kFwdThreads, fsm, p->num_sms);
    p->adj_grid = resident_ctas(adj_kernel_for(p), kAdjThreads, asm_, p->num_sms);
    return MRI_OK;
}

cudaError_t launch_fwd_tc(mri_plan *p, const float2 *image, const float2 *maps, float2 *kspace, int ld, int skip,
                          cudaStream_t s) {
    const bool t = p->precision == MRI_TF32;
    if (image) {  // else the solver has written the operand already
        dim3 og(ceil_div(p->nx, 32), ceil_div(p->ny, 32), p->nc);
        if (t)
            fwd_operand_kernel<true><<<og, dim3(32, 8), 0, s>>>(image, maps, nullptr, nullptr, (uint2 *)p->bfwd_t,
                                                                p->nx, p->ny, p->ny_pad, p->kx, p->scal, skip);
        else
            fwd_operand_kernel<false><<<og, dim3(32, 8), 0, s>>>(image, maps, (uint32_t *)p->bfwd_hi,
                                                                 (uint32_t *)p->bfwd_lo, nullptr, p->nx, p->ny,
                                                                 p->ny_pad, p->kx, p->scal, skip);
        p->launches += 1;
    }
    FwdParams P;
    P.y = kspace;
    P.y_ld = ld;
    P.nk = p->nk;
    P.ny_pad = p->ny_pad;
    P.nc = p->nc;
    P.cpt = p->fwd_coils_per_tile;
    P.block_n = p->fwd_block_n;
    P.n_tiles = p->fwd_n_tiles;
    P.n_parts = p->ny_pad > 256 ? p->ny_pad / 256 : 1;
    P.pw = p->ny_pad > 256 ? 256 : p->ny_pad;
    P.num_kb = p->kx / kTcBlockK;
    P.num_units = p->fwd_m_tiles * p->fwd_n_tiles;
    size_t smem;
    fwd_smem_plan(p, &P.stages, &P.ay_stages, &smem);
    P.tmem_cols = tmem_cols_for(2 * p->fwd_block_n);
    P.sc = p->scal;
    P.skip = skip;
    P.status = &p->scal->status;
    const int grid = std::min(P.num_units, p->fwd_grid);
    timing_begin(p, s);
    if (t)
        fwd_tc_kernel<true><<<grid, kFwdThreads, smem, s>>>(p->tm_afwd_hi, p->tm_afwd_lo, p->tm_bfwd_hi,
                                                            p->tm_bfwd_lo, p->tm_ayT, P);
    else
        fwd_tc_kernel<false><<<grid, kFwdThreads, smem, s>>>(p->tm_afwd_hi, p->tm_afwd_lo, p->tm_bfwd_hi,
                                                             p->tm_bfwd_lo, p->tm_ayT, P);
    cudaError_t e = cudaGetLastError();
    timing_end(p, s);
    p->launches += 1;
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_adj_tc(mri_plan *p, int skip, cudaStream_t s) {
    AdjParams P;
    P.part = p->part;
    P.ksplit = p->ksplit;
    P.n_ig = p->nx_pad / 64;
    P.nx = p->nx;
    P.ny = p->ny;
    P.ny_pad = p->adj_block_n;  // the tile width
    P.nx_pad = p->nx_pad;
    P.nc = p->nc;
    P.tiles_per_coil = p->nx_pad / p->adj_tile_px;
    P.m_tiles = p->adj_m_tiles;
    P.kb_per_split = p->ksplit_blocks;
    P.num_kb = p->kk / kTcBlockK;
    P.num_units = p->adj_m_tiles * p->ksplit;
    size_t smem;
    adj_smem_plan(p, &P.stages, &P.raw_stages, &smem, &P.n_acc, &P.a_col0);
    P.tmem_cols = tmem_cols_for(P.a_col0 + 64 * P.stages);
    P.sc = p->scal;
    P.skip = skip;
    P.status = &p->scal->status;
    const int grid = std::min(P.num_units, p->adj_grid);
    // one launch per 256-column part of the image (one launch when ny <= 256)
    const int n_parts = adj_parts(p);
    timing_begin(p, s);
    cudaError_t e = cudaSuccess;
    for (int part = 0; part < n_parts && e == cudaSuccess; ++part) {
        const int j0 = part * p->adj_block_n;  // n_parts > 1 only in the row-pair form
        P.part = p->part + (size_t)j0 * P.n_ig * p->ksplit * 64;  // column j0 of every coil's partials
        P.ny_lim = p->ny - j0;
        P.b_row0 = j0;
        adj_kernel_for(p)<<<grid, kAdjThreads, smem, s>>>(p->tm_badj_hi, p->tm_badj_lo, p->tm_axT,
                                                          p->adj_tile_px == 128 ? p->tm_axQ : p->tm_axT, p->tm_y, P);
        e = cudaGetLastError();
        p->launches += 1;
    }
    timing_end(p, s);
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace mri
