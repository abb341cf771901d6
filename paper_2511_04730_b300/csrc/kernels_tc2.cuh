// Tensor-core (tcgen05) basis filter and per-rate reconstruction for the
// split-precision paths, in the paper's order (Eq. 5, Eq. 6, Eq. 7-9).
//
// k_fir_tc  (a2): Y^s_l[q] = sum_m u_l[m] x[q - m] as a GEMM over 8 output
//   phases: q = 8c + t, A'[(l,t)][j] = u_l[t + N' - 1 - j] (bases expanded
//   over the 8 phases, zero outside the filter), B'[c][j] = x[8c - N' + 1 + j].
//   B' rows are 16 bytes apart in a contiguous strip of the stream, so the
//   strip itself is the operand: a no-swizzle K-major descriptor whose
//   K-adjacent core matrices are 16 B apart (LBO) and N-adjacent 128 B apart
//   (SBO).  Nothing is materialised; the strip (hi and lo halves) is one bulk
//   copy per tile, the expanded bases stream through a TMA pipeline.  The
//   epilogue writes Y (hi/lo) into the level's operand ring through a
//   shared-memory transpose (rows = time, columns = bases).
//
// k_level_tc (a3 + a4 + a5): for ladder level j (rate r_j, lowest first)
//   Acc_j[q] = C_j Y_j[q] + Up_F(Acc_{j-1})[q], Up of Eq. 8 in its centred
//   reading; Acc is kept transposed ([q][template], templates contiguous) so
//   that the epilogue's reads and writes coalesce.  The top level (f0) forms
//   |z|^2 and the per-tile argmax instead of storing Acc.
#pragma once
#include "kernels_tc.cuh"

namespace lloid {

constexpr int kFirNC = 128;       // max c-groups per FIR tile (1024 outputs)
constexpr int kEpiThreads = 128;  // epilogue warps 2..5

// ---------------------------------------------------------------------------
struct FirTcJob {
    const uint16_t* s_hi;          // stream ring (double-mapped) of this rate, detector 0
    const uint16_t* s_lo;
    long long s_det_stride;        // elements
    uint16_t* y_hi;                // level ring, first column of this slice, detector 0
    uint16_t* y_lo;
    long long y_det_stride;        // elements
    long long J_over_D;
    int s_len;                     // stream ring length (power of two); 2*s_len stored
    int y_rows;                    // level ring rows (power of two); 2*y_rows stored
    int y_ld;                      // level ring row length (Kpad of the level)
    int Mtiles;                    // M'pad / 128 (16 bases per tile)
    int Kp;                        // K'pad (multiple of 64)
    int Np;                        // N' (padded filter length)
    int NC;                        // c-groups per tile (multiple of 16, <= kFirNC)
    int ctiles;                    // c tiles per push
    int D, Lambda, q_count, map;   // map = index into the FIR tensor-map array
};

struct LevelJob {
    const float* acc_in;           // level below, transposed [2][rows][Mpad], detector 0
    float* acc_out;                // this level (non-top), transposed, detector 0
    long long acc_in_det_stride, acc_out_det_stride;   // elements
    const float* upz;              // unused (sub-kernels live in c_upz)
    int acc_in_rows, acc_out_rows; // rows per re/im plane
    int Kp;                        // Kpad of the level (0: no slice at this rate)
    int M, Mpad, tmpl0;
    int tiles_m, tiles_t;
    int D, Lambda;                 // this level
    int F, D_lo, Lambda_lo;        // factor to the level below (0: lowest level)
    int y_rows;                    // level ring rows
    int map;                       // index into the level tensor-map array
    int nwt;                       // up-window rows per 128-sample tile: 127/F + 2 N_up + 1
};

struct FirMaps { CUtensorMap a, a_lo; };

// Eq. 7 polyphase sub-kernels z_phi[t] = g[t F + phi] (t = 0..16, N_up = 8) for
// F = 2, 4, ..., 64, packed F after F (offset 17 (F - 2)); filled once per
// device.  Indexed with compile-time constants, so each tap is one FFMA with a
// constant-bank operand.
constexpr int kUpTaps = 17;
constexpr int kUpTable = kUpTaps * (2 + 4 + 8 + 16 + 32 + 64);
__constant__ float c_upz[kUpTable];
// accin: the level below's transposed Acc planes as FP32 rows of Mpad
// templates (plane rows stacked det-major: [det][re, im][rows]); box 128
// templates x nwt rows, loaded once per tile into shared memory.
struct LevelMaps { CUtensorMap cre, cim, cre_lo, cim_lo, yhi, ylo, accin; };

// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t desc_nosw(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1u << 46;
    return d;   // layout type 0: no swizzle
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory"); }

__device__ __forceinline__ int job_of(const int* __restrict__ base, int n, int t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(base + mid) <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ long long fdiv(long long a, long long b) {
    long long q = a / b;
    return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

template <typename T>
__device__ __forceinline__ uint16_t h_bits(T v) { return *reinterpret_cast<uint16_t*>(&v); }

template <bool BF16>
__device__ __forceinline__ void split_hilo(float v, uint16_t& hi, uint16_t& lo) {
    if (BF16) {
        __nv_bfloat16 h = __float2bfloat16_rn(v);
        hi = h_bits(h);
        lo = h_bits(__float2bfloat16_rn(v - __bfloat162float(h)));
    } else {
        __half h = __float2half_rn(v);
        hi = h_bits(h);
        lo = h_bits(__float2half_rn(v - __half2float(h)));
    }
}

// ---------------------------------------------------------------------------
// a2 on the tensor cores
// ---------------------------------------------------------------------------
template <bool BF16>
struct FirCfg {
    static constexpr int STAGES = 4;
    static constexpr int TILE_A = 128 * kTcK * 2;              // 16 KB
    static constexpr int STAGE_BYTES = (BF16 ? 2 : 1) * TILE_A;
    static constexpr int STAGE_AREA = STAGES * STAGE_BYTES;
    static constexpr int EPI_LD = 24;                          // staging row pitch (halves): conflict-free, 16 B aligned
    static constexpr int EPI_BYTES = 2 * 256 * EPI_LD * 2;     // staging [256 q][16 bases (+pad)] hi + lo
};

template <bool BF16>
__global__ void __launch_bounds__(192, 1)
    k_fir_tc(const FirTcJob* __restrict__ jobs, const FirMaps* __restrict__ maps, const int* __restrict__ tile_base,
             int n_jobs, int tiles_per_det, long long k_a, int det0, int n_det_push, int strip_bytes,
             int* __restrict__ err) {
    using C = FirCfg<BF16>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* stage_area = smem;
    uint8_t* strip_area = smem + C::STAGE_AREA;                // 2 buffers x (hi, lo) x strip_bytes
    uint16_t* epi = reinterpret_cast<uint16_t*>(strip_area + 4 * strip_bytes);
    uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(epi) + C::EPI_BYTES);
    uint64_t* a_full = bars;
    uint64_t* a_empty = a_full + C::STAGES;
    uint64_t* s_full = a_empty + C::STAGES;
    uint64_t* s_empty = s_full + 2;
    uint64_t* t_full = s_empty + 2;
    uint64_t* t_empty = t_full + 2;
    uint64_t* drain = t_empty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) { mbar_init(a_full + s, 1); mbar_init(a_empty + s, 1); }
        for (int b = 0; b < 2; ++b) {
            mbar_init(s_full + b, 1); mbar_init(s_empty + b, 1);
            mbar_init(t_full + b, 1); mbar_init(t_empty + b, kEpiThreads);
        }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int total = tiles_per_det * n_det_push;

    if (warp == 0) {
        if (lane == 0) {   // ------------------------------------------------ producer
            int stage = 0, sb = 0;
            uint32_t phase = 0, sphase = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < total && ok; it += gridDim.x) {
                const int det = det0 + it / tiles_per_det;
                const int t = it % tiles_per_det;
                const int jx = job_of(tile_base, n_jobs, t);
                const FirTcJob& jb = jobs[jx];
                const int local = t - tile_base[jx];
                const int mt = local % jb.Mtiles, ct = local / jb.Mtiles;
                const long long qa = fdiv(k_a - 1 + jb.Lambda, jb.D) + 1;
                const long long c0 = fdiv(qa, 8) + (long long)ct * jb.NC;
                const long long i0 = 8 * c0 - jb.Np + 1 - jb.J_over_D;       // multiple of 8
                const long long p0 = i0 & (jb.s_len - 1);
                const uint32_t bytes = (uint32_t)(2 * (8 * jb.NC + jb.Kp));
                if (!mbar_wait(s_empty + sb, sphase ^ 1, err, 21)) { ok = false; break; }
                mbar_expect_tx(s_full + sb, 2 * bytes);
                bulk_g2s(strip_area + (2 * sb) * strip_bytes, jb.s_hi + det * jb.s_det_stride + p0, bytes, s_full + sb);
                bulk_g2s(strip_area + (2 * sb + 1) * strip_bytes, jb.s_lo + det * jb.s_det_stride + p0, bytes,
                         s_full + sb);
                if (++sb == 2) { sb = 0; sphase ^= 1; }
                const FirMaps* mp = maps + jb.map;
                for (int kc = 0; kc < jb.Kp; kc += kTcK) {
                    if (!mbar_wait(a_empty + stage, phase ^ 1, err, 22)) { ok = false; break; }
                    uint8_t* st = stage_area + stage * C::STAGE_BYTES;
                    mbar_expect_tx(a_full + stage, C::STAGE_BYTES);
                    tma_load_2d(st, &mp->a, a_full + stage, kc, mt * 128);
                    if (BF16) tma_load_2d(st + C::TILE_A, &mp->a_lo, a_full + stage, kc, mt * 128);
                    if (++stage == C::STAGES) { stage = 0; phase ^= 1; }
                }
            }
            for (int s = 0; s < C::STAGES; ++s) {                 // drain the A stages
                if (!mbar_wait(a_empty + stage, phase ^ 1, err, 23)) break;
                if (++stage == C::STAGES) { stage = 0; phase ^= 1; }
            }
            for (int s = 0; s < 2; ++s) {                         // and the strips
                if (!mbar_wait(s_empty + sb, sphase ^ 1, err, 24)) break;
                if (++sb == 2) { sb = 0; sphase ^= 1; }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {   // ------------------------------------------------ MMA issuer
            int stage = 0, sb = 0, i = 0;
            uint32_t phase = 0, sphase = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < total && ok; it += gridDim.x, ++i) {
                const int t = it % tiles_per_det;
                const int jx = job_of(tile_base, n_jobs, t);
                const int Kp = jobs[jx].Kp, NC = jobs[jx].NC;
                const uint32_t idesc = idesc_f16(BF16, 128, NC);
                const int buf = i & 1;
                if (!mbar_wait(t_empty + buf, ((i >> 1) & 1) ^ 1, err, 25)) { ok = false; break; }
                if (!mbar_wait(s_full + sb, sphase, err, 26)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d = tmem + buf * 128;
                const uint32_t s_hi = smem_u32(strip_area + (2 * sb) * strip_bytes);
                const uint32_t s_lo = smem_u32(strip_area + (2 * sb + 1) * strip_bytes);
                for (int kc = 0; kc < Kp; kc += kTcK) {
                    if (!mbar_wait(a_full + stage, phase, err, 27)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t a = smem_u32(stage_area + stage * C::STAGE_BYTES);
#pragma unroll
                    for (int k = 0; k < kTcK / 16; ++k) {
                        const uint32_t boff = 2 * (kc + 16 * k);
                        const uint64_t da = desc_sw128(a + 32 * k);
                        const uint64_t bh = desc_nosw(s_hi + boff, 16, 128);
                        const uint64_t bl = desc_nosw(s_lo + boff, 16, 128);
                        umma_f16(d, da, bh, idesc, (kc > 0 || k > 0) ? 1u : 0u);
                        umma_f16(d, da, bl, idesc, 1u);
                        if (BF16) umma_f16(d, desc_sw128(a + C::TILE_A + 32 * k), bh, idesc, 1u);
                    }
                    umma_commit(a_empty + stage);
                    if (++stage == C::STAGES) { stage = 0; phase ^= 1; }
                }
                if (!ok) break;
                umma_commit(s_empty + sb);
                umma_commit(t_full + buf);
                if (++sb == 2) { sb = 0; sphase ^= 1; }
            }
            umma_commit(drain);
            mbar_wait(drain, 0, err, 28);
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        const int et = threadIdx.x - 64;                // 0..127
        const int qd = warp & 3;                        // TMEM lane quarter
        const int row = qd * 32 + lane;                 // A' row in the tile = 8 l + t
        const int l_loc = row >> 3, tph = row & 7;
        int i = 0;
        for (int it = blockIdx.x; it < total; it += gridDim.x, ++i) {
            const int det = det0 + it / tiles_per_det;
            const int t = it % tiles_per_det;
            const int jx = job_of(tile_base, n_jobs, t);
            const FirTcJob& jb = jobs[jx];
            const int local = t - tile_base[jx];
            const int mt = local % jb.Mtiles, ct = local / jb.Mtiles;
            const long long qa = fdiv(k_a - 1 + jb.Lambda, jb.D) + 1;
            const long long c0 = fdiv(qa, 8) + (long long)ct * jb.NC;
            const int buf = i & 1;
            const bool got = mbar_wait(t_full + buf, (i >> 1) & 1, err, 29);
            if (!__all_sync(0xffffffffu, got)) break;
            tc_fence_after();
            uint16_t* yh = jb.y_hi + det * jb.y_det_stride + mt * 16;
            uint16_t* yl = jb.y_lo + det * jb.y_det_stride + mt * 16;
            for (int cc = 0; cc < jb.NC; cc += 32) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(qd * 32) << 16) + buf * 128 + cc, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    uint16_t h, l;
                    split_hilo<BF16>(v[j], h, l);
                    epi[(8 * j + tph) * C::EPI_LD + l_loc] = h;
                    epi[256 * C::EPI_LD + (8 * j + tph) * C::EPI_LD + l_loc] = l;
                }
                epi_sync();
                // 256 rows x 32 B (hi) + 256 x 32 B (lo) as 16-byte stores, both ring mappings
                for (int e = et; e < 2 * 256 * 2; e += kEpiThreads) {
                    const int part = e >> 9;             // 0 hi, 1 lo
                    const int r = (e >> 1) & 255, h16 = e & 1;
                    const long long q = 8 * (c0 + cc) + r;
                    if (cc + (r >> 3) >= jb.NC || q < qa || q >= qa + jb.q_count) continue;
                    const uint4 val = *reinterpret_cast<const uint4*>(epi + part * 256 * C::EPI_LD + r * C::EPI_LD + h16 * 8);
                    uint16_t* dst = part ? yl : yh;
                    const long long rr = q & (jb.y_rows - 1);
                    *reinterpret_cast<uint4*>(dst + rr * jb.y_ld + h16 * 8) = val;
                    *reinterpret_cast<uint4*>(dst + (rr + jb.y_rows) * jb.y_ld + h16 * 8) = val;
                }
                epi_sync();
            }
            tc_fence_before();
            mbar_arrive(t_empty + buf);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
    }
}

// ---------------------------------------------------------------------------
// a3 + a4 + a5 per ladder level
// ---------------------------------------------------------------------------
template <bool BF16>
struct LevCfg {
    static constexpr int NA = BF16 ? 4 : 2;
    static constexpr int STAGES = BF16 ? 1 : 2;
    static constexpr int TILE_A = kTcTileM * kTcK * 2;
    static constexpr int TILE_B = kTcTileN * kTcK * 2;
    static constexpr int STAGE_BYTES = NA * TILE_A + 2 * TILE_B;
    static constexpr int XCHG = 2 * 128 * 16;          // tile-argmax exchange between the column halves
    static constexpr int NWT_MAX = 80;                 // up-window rows for F = 2
    static constexpr int WIN = 2 * NWT_MAX * 128 * 4;  // re + im windows of the level below
    static constexpr int SMEM = STAGES * STAGE_BYTES + WIN + XCHG + 1024 + 256;
    static constexpr int EPI_WARPS = 8;                 // two per TMEM lane quarter, 64 columns each
    static constexpr int THREADS = 64 + 32 * EPI_WARPS;
};

// One epilogue thread: template m (TMEM lane), columns 64 h .. 64 h + 63 of
// the tile.  Acc[q] = (C Y)[q] + Up_F(Acc_below)[q] with Eq. 8 in its centred
// reading, Up[q] = sum_{t=0}^{2 N_up} z_{q mod F}[t] x[floor(q/F) + N_up - t].
// The shared-memory window holds x from floor(Q_tile/F) - N_up on (row w);
// output column c of the tile reads rows floor(c/F) + 2 N_up - t.  The rows
// this half needs are copied to registers first and the window is released
// at once, so that the next tile's window streams in while this one
// finishes.  Tiles start at multiples of 128 and F divides 64, so every
// register index is a compile-time constant.
template <int F, bool TOP, bool STORE_Z>
__device__ __forceinline__ float4 epi_half(uint32_t tb, bool has_acc, const float* __restrict__ wre,
                                        const float* __restrict__ wim, int col, int half, uint64_t* wempty,
                                        float* o_re, float* o_im, long long q0, long long lo, long long hi, int Mpad,
                                        int m, float* zr, float* zi, bool zvalid) {
    float best = -1.f, bre = 0.f, bim = 0.f;
    int bk = 0x7fffffff;
    constexpr int NUP = 8;
    constexpr int FF = F ? F : 1;
    constexpr int NWH = F ? 63 / FF + 2 * NUP + 1 : 1;
    constexpr int OFF = F ? kUpTaps * (F - 2) : 0;
    if constexpr (F >= 8 && F <= 32) {
        // One F-block of outputs per iteration, rolled, with its 2 N_up + 1 window rows read
        // from shared memory (the constant taps of a block then stay constant-bank operands
        // instead of being held in registers across unrolled blocks).  The window is
        // released when the half tile is done.
#pragma unroll 1
        for (int blk = 0; blk < 64 / FF; ++blk) {
            const int c0 = 64 * half + blk * FF;          // tile column of the block's first output
            const int wrow = c0 / FF;                     // window row of x[floor(c0/F) - N_up]
            float x_r[2 * NUP + 1], x_i[2 * NUP + 1];
#pragma unroll
            for (int w = 0; w <= 2 * NUP; ++w) {
                x_r[w] = wre[(wrow + w) * 128 + col];
                x_i[w] = wim[(wrow + w) * 128 + col];
            }
#pragma unroll
            for (int sub = 0; sub < FF / 8; ++sub) {
                uint32_t rr[16];
                if (has_acc) {
                    tmem_ld8x2_async(tb + blk * FF + sub * 8, rr);
                    tmem_wait16(rr);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) rr[j] = 0u;
                }
                float re[8], im[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    re[j] = __uint_as_float(rr[j]);
                    im[j] = __uint_as_float(rr[8 + j]);
                    const int ph = sub * 8 + j;
                    if (ph == 0) {
                        re[j] += x_r[NUP];
                        im[j] += x_i[NUP];
                        continue;
                    }
                    float sr = 0.f, si = 0.f;
#pragma unroll
                    for (int t = 0; t <= 2 * NUP; ++t) {
                        if (t * F + ph > 2 * F * NUP) continue;
                        const float zc = c_upz[OFF + ph * kUpTaps + t];
                        sr = fmaf(zc, x_r[2 * NUP - t], sr);
                        si = fmaf(zc, x_i[2 * NUP - t], si);
                    }
                    re[j] += sr;
                    im[j] += si;
                }
                const int cb = blk * FF + sub * 8;        // column within the half tile
                if (TOP) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float pw = re[j] * re[j] + im[j] * im[j];
                        if (pw > best) { best = pw; bk = 64 * half + cb + j; bre = re[j]; bim = im[j]; }
                    }
                    if (STORE_Z && zvalid) {
#pragma unroll
                        for (int j = 0; j < 8; ++j) { zr[cb + j] = re[j]; zi[cb + j] = im[j]; }
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const long long q = q0 + cb + j;
                        if (q >= lo && q <= hi) {
                            o_re[(q - lo) * Mpad + m] = re[j];
                            o_im[(q - lo) * Mpad + m] = im[j];
                        }
                    }
                }
            }
        }
        mbar_arrive(wempty);
        return make_float4(best, __int_as_float(bk), bre, bim);
    }
    constexpr int NWR = (F >= 8 && F <= 32) ? 1 : NWH;
    float xr[NWR], xi[NWR];
    if (F) {
        const int r0 = (64 * half) / FF;
        const float* pr = wre + r0 * 128 + col;
        const float* pi = wim + r0 * 128 + col;
#pragma unroll
        for (int w = 0; w < NWR; ++w) { xr[w] = pr[w * 128]; xi[w] = pi[w * 128]; }
        mbar_arrive(wempty);
    }
    // 8-column chunks, the TMEM load of chunk k + 1 in flight while chunk k is computed
    uint32_t cur[16], nxt[16];
    if (has_acc) {
        tmem_ld8x2_async(tb, cur);
        tmem_wait16(cur);
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) cur[j] = 0u;
    }
#pragma unroll
    for (int cc = 0; cc < 64; cc += 8) {
        if (has_acc && cc + 8 < 64) tmem_ld8x2_async(tb + cc + 8, nxt);
        float re[8], im[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) { re[j] = __uint_as_float(cur[j]); im[j] = __uint_as_float(cur[8 + j]); }
        if (F) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int cr = cc + j;
                const int ph = cr % FF;
                const int b = cr / FF + 2 * NUP;
                if (ph == 0) {                           // z_0 = g[t F]: 1 at t = N_up, 0 elsewhere
                    re[j] += xr[b - NUP];
                    im[j] += xi[b - NUP];
                    continue;
                }
                float sr = 0.f, si = 0.f;
#pragma unroll
                for (int t = 0; t <= 2 * NUP; ++t) {
                    if (t * F + ph > 2 * F * NUP) continue;   // beyond the kernel: identically zero
                    const float zc = c_upz[OFF + ph * kUpTaps + t];
                    sr = fmaf(zc, xr[b - t], sr);
                    si = fmaf(zc, xi[b - t], si);
                }
                re[j] += sr;
                im[j] += si;
            }
        }
        if (TOP) {
            // chunk argmax as a pairwise tree (the earlier column wins ties), then into the running one
            float p[8];
            int k[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) { p[j] = re[j] * re[j] + im[j] * im[j]; k[j] = j; }
#pragma unroll
            for (int s = 1; s < 8; s *= 2) {
#pragma unroll
                for (int j = 0; j < 8; j += 2 * s) {
                    const bool later = p[j + s] > p[j];
                    p[j] = later ? p[j + s] : p[j];
                    k[j] = later ? k[j + s] : k[j];
                }
            }
            float cre = re[0], cim = im[0];
#pragma unroll
            for (int j = 1; j < 8; ++j) {
                cre = (k[0] == j) ? re[j] : cre;
                cim = (k[0] == j) ? im[j] : cim;
            }
            if (p[0] > best) { best = p[0]; bk = 64 * half + cc + k[0]; bre = cre; bim = cim; }
            if (STORE_Z && zvalid) {
#pragma unroll
                for (int j = 0; j < 8; ++j) { zr[cc + j] = re[j]; zi[cc + j] = im[j]; }
            }
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const long long q = q0 + cc + j;
                if (q >= lo && q <= hi) {
                    o_re[(q - lo) * Mpad + m] = re[j];
                    o_im[(q - lo) * Mpad + m] = im[j];
                }
            }
        }
        if (has_acc && cc + 8 < 64) {
            tmem_wait16(nxt);
#pragma unroll
            for (int j = 0; j < 16; ++j) cur[j] = nxt[j];
        }
    }
    return make_float4(best, __int_as_float(bk), bre, bim);
}

// F (the factor to the level below, 0 at the lowest level) is a template
// parameter so that each instantiation gets the register allocation its
// epilogue needs (up to 96 registers hold the window at F = 2); 10 warps, three
// of which share one SM sub-partition's 16K registers, leave 168 per thread.
template <bool BF16, bool TOP, bool STORE_Z, int F>
__global__ void __launch_bounds__(LevCfg<BF16>::THREADS, 1)
    k_level_tc(const LevelJob* __restrict__ jobs, const LevelMaps* __restrict__ maps,
               const int* __restrict__ tile_base, int n_jobs, int tiles_per_det, long long k_a, long long k_b,
               int det0, int n_det_push, long long window, Partial* __restrict__ part, long long part_tmpl_stride,
               int n_slots, float* __restrict__ zout, int* __restrict__ err) {
    using C = LevCfg<BF16>;
    constexpr int EPI = 32 * C::EPI_WARPS;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float* win_re = reinterpret_cast<float*>(smem + C::STAGES * C::STAGE_BYTES);
    float* win_im = win_re + C::NWT_MAX * 128;
    float4* xchg = reinterpret_cast<float4*>(smem + C::STAGES * C::STAGE_BYTES + C::WIN);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::STAGES * C::STAGE_BYTES + C::WIN + C::XCHG);
    uint64_t* empty = full + C::STAGES;
    uint64_t* tfull = empty + C::STAGES;
    uint64_t* tempty = tfull + 2;
    uint64_t* drain = tempty + 2;
    uint64_t* wfull = drain + 1;
    uint64_t* wempty = wfull + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(wempty + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) { mbar_init(full + s, 1); mbar_init(empty + s, 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(tfull + b, 1); mbar_init(tempty + b, EPI); }
        mbar_init(drain, 1);
        mbar_init(wfull, 1);
        mbar_init(wempty, EPI);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int total = tiles_per_det * n_det_push;

    if (warp == 0) {
        if (lane == 0) {   // ------------------------------------------------ producer
            int stage = 0;
            uint32_t phase = 0, wphase = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < total && ok; it += gridDim.x) {
                const int det = det0 + it / tiles_per_det;
                const int t = it % tiles_per_det;
                const int jx = job_of(tile_base, n_jobs, t);
                const LevelJob& jb = jobs[jx];
                const LevelMaps* mp = maps + jb.map;
                const int local = t - tile_base[jx];
                const int tm = local % jb.tiles_m, tt = local / jb.tiles_m;
                const long long Q0 = fdiv(fdiv(k_a - jb.Lambda, jb.D), 128) * 128;
                const int yrow = det * 2 * jb.y_rows + (int)((Q0 + 128LL * tt) & (jb.y_rows - 1));
                for (int kc = 0; kc < jb.Kp; kc += kTcK) {
                    if (!mbar_wait(empty + stage, phase ^ 1, err, 31)) { ok = false; break; }
                    uint8_t* sb = smem + stage * C::STAGE_BYTES;
                    mbar_expect_tx(full + stage, C::STAGE_BYTES);
                    tma_load_2d(sb, &mp->cre, full + stage, kc, tm * 128);
                    tma_load_2d(sb + C::TILE_A, &mp->cim, full + stage, kc, tm * 128);
                    if (BF16) {
                        tma_load_2d(sb + 2 * C::TILE_A, &mp->cre_lo, full + stage, kc, tm * 128);
                        tma_load_2d(sb + 3 * C::TILE_A, &mp->cim_lo, full + stage, kc, tm * 128);
                    }
                    tma_load_2d(sb + C::NA * C::TILE_A, &mp->yhi, full + stage, kc, yrow);
                    tma_load_2d(sb + C::NA * C::TILE_A + C::TILE_B, &mp->ylo, full + stage, kc, yrow);
                    if (++stage == C::STAGES) { stage = 0; phase ^= 1; }
                }
                // The level below's window for this tile (rows outside the planes read 0).  It is
                // fetched after the tile's operand stages so that the MMAs of this tile overlap
                // the epilogue of the previous one, which still holds the (single) window buffer.
                if (F != 0 && ok) {
                    if (!mbar_wait(wempty, wphase ^ 1, err, 37)) { ok = false; break; }
                    const long long lo_in = fdiv(k_a - jb.Lambda_lo, jb.D_lo);
                    const long long a_t = fdiv(Q0 + 128LL * tt, F != 0 ? F : 1) - 8 - lo_in;
                    const int base_row = det * 2 * jb.acc_in_rows;
                    mbar_expect_tx(wfull, 2u * jb.nwt * 128 * 4);
                    tma_load_2d(win_re, &mp->accin, wfull, tm * 128, (int)(base_row + a_t));
                    tma_load_2d(win_im, &mp->accin, wfull, tm * 128, (int)(base_row + jb.acc_in_rows + a_t));
                    wphase ^= 1;
                }
            }
            for (int s = 0; s < C::STAGES; ++s) {
                if (!mbar_wait(empty + stage, phase ^ 1, err, 32)) break;
                if (++stage == C::STAGES) { stage = 0; phase ^= 1; }
            }
            mbar_wait(wempty, wphase ^ 1, err, 38);    // the last window was consumed
        }
    } else if (warp == 1) {
        if (lane == 0) {   // ------------------------------------------------ MMA issuer
            constexpr uint32_t idesc = idesc_f16(BF16, kTcTileM, kTcTileN);
            int stage = 0, i = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < total && ok; it += gridDim.x, ++i) {
                const int t = it % tiles_per_det;
                const int jx = job_of(tile_base, n_jobs, t);
                const int Kp = jobs[jx].Kp;
                const int buf = i & 1;
                if (!mbar_wait(tempty + buf, ((i >> 1) & 1) ^ 1, err, 33)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d_re = tmem + buf * 256, d_im = d_re + 128;
                for (int kc = 0; kc < Kp; kc += kTcK) {
                    if (!mbar_wait(full + stage, phase, err, 34)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sb = smem_u32(smem + stage * C::STAGE_BYTES);
                    const uint32_t a_re = sb, a_im = sb + C::TILE_A;
                    const uint32_t a_re_lo = sb + 2 * C::TILE_A, a_im_lo = sb + 3 * C::TILE_A;
                    const uint32_t b_hi = sb + C::NA * C::TILE_A, b_lo = b_hi + C::TILE_B;
#pragma unroll
                    for (int k = 0; k < kTcK / 16; ++k) {
                        const uint32_t off = k * 32;
                        const uint32_t acc0 = (kc > 0 || k > 0) ? 1u : 0u;
                        umma_f16(d_re, desc_sw128(a_re + off), desc_sw128(b_hi + off), idesc, acc0);
                        umma_f16(d_re, desc_sw128(a_re + off), desc_sw128(b_lo + off), idesc, 1u);
                        umma_f16(d_im, desc_sw128(a_im + off), desc_sw128(b_hi + off), idesc, acc0);
                        umma_f16(d_im, desc_sw128(a_im + off), desc_sw128(b_lo + off), idesc, 1u);
                        if (BF16) {
                            umma_f16(d_re, desc_sw128(a_re_lo + off), desc_sw128(b_hi + off), idesc, 1u);
                            umma_f16(d_im, desc_sw128(a_im_lo + off), desc_sw128(b_hi + off), idesc, 1u);
                        }
                    }
                    umma_commit(empty + stage);
                    if (++stage == C::STAGES) { stage = 0; phase ^= 1; }
                }
                if (!ok) break;
                umma_commit(tfull + buf);     // with Kp == 0 this only signals the epilogue
            }
            umma_commit(drain);
            mbar_wait(drain, 0, err, 35);
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        // 8 warps: warp & 3 picks the TMEM lane quarter (rows), (warp - 2) / 4 the
        // 64-column half of the 128-sample tile.
        const int qd = warp & 3;
        const int half = (warp - 2) >> 2;
        const int rowm = qd * 32 + lane;
        uint32_t wph = 0;
        int i = 0;
        for (int it = blockIdx.x; it < total; it += gridDim.x, ++i) {
            const int det = det0 + it / tiles_per_det;
            const int t = it % tiles_per_det;
            const int jx = job_of(tile_base, n_jobs, t);
            const LevelJob& jb = jobs[jx];
            const int local = t - tile_base[jx];
            const int tm = local % jb.tiles_m, tt = local / jb.tiles_m;
            const int buf = i & 1;
            const bool got = mbar_wait(tfull + buf, (i >> 1) & 1, err, 36);
            if (!__all_sync(0xffffffffu, got)) break;
            tc_fence_after();
            const long long lo = fdiv(k_a - jb.Lambda, jb.D);
            const long long hi = fdiv(k_b - 1 + jb.Lambda, jb.D);
            const long long Q0 = fdiv(lo, 128) * 128;
            const int m = tm * kTcTileM + rowm;
            const uint32_t base = tmem + ((uint32_t)(qd * 32) << 16) + buf * 256;
            float best = -1.f, bre = 0.f, bim = 0.f;
            int bk = 0x7fffffff;
            if (F != 0) {
                const bool wgot = mbar_wait(wfull, wph, err, 39);
                if (!__all_sync(0xffffffffu, wgot)) break;
                wph ^= 1;
            }
            float *o_re = nullptr, *o_im = nullptr, *zr = nullptr, *zi = nullptr;
            bool zvalid = false;
            if (!TOP) {
                o_re = jb.acc_out + det * jb.acc_out_det_stride;
                o_im = o_re + (long long)jb.acc_out_rows * jb.Mpad;
            } else if (STORE_Z && m < jb.M) {
                const int n = (int)(k_b - k_a);
                zr = zout + (long long)(2 * m) * n + tt * kTcTileN + 64 * half;
                zi = zr + n;
                zvalid = true;
            }
            const long long q0 = Q0 + 128LL * tt + 64 * half;
            const uint32_t tb = base + 64 * half;
            const bool has_acc = jb.Kp > 0;
            const float4 r = epi_half<F, TOP, STORE_Z>(tb, has_acc, win_re, win_im, rowm, half, wempty, o_re, o_im,
                                                       q0, lo, hi, jb.Mpad, m, zr, zi, zvalid);
            best = r.x;
            bk = __float_as_int(r.y);
            bre = r.z;
            bim = r.w;
            tc_fence_before();
            mbar_arrive(tempty + buf);
            if (TOP && !STORE_Z) {
                // the later half hands its tile argmax to the earlier half (which wins ties)
                float4* xb = xchg + buf * 128;
                if (half == 1) xb[rowm] = make_float4(best, __int_as_float(bk), bre, bim);
                asm volatile("bar.sync 1, %0;" ::"n"(EPI) : "memory");
                if (half == 0 && m < jb.M) {
                    const float4 o = xb[rowm];
                    if (o.x > best) { best = o.x; bk = __float_as_int(o.y); bre = o.z; bim = o.w; }
                    const long long k0 = Q0 + 128LL * tt;         // Q0 == lo == k_a at the top level
                    const long long kwin0 = (k0 / window) * window;
                    const int slot = (int)((k0 / kTcTileN) & (n_slots - 1));
                    part[(long long)(jb.tmpl0 + m) * part_tmpl_stride + (long long)det * n_slots + slot] =
                        make_float4(best, __int_as_float((int)(k0 - kwin0) + bk), bre, bim);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

// ---------------------------------------------------------------------------
// stream rings for the tensor-core FIR: FP32 stream -> hi/lo halves, written
// at i mod R and i mod R + R (double-mapped so any strip <= R is contiguous)
// ---------------------------------------------------------------------------
template <bool BF16>
__global__ void k_split_stream(const float* __restrict__ src, long long src_det_stride, int src_mask,
                               uint16_t* __restrict__ hi, uint16_t* __restrict__ lo, long long dst_det_stride,
                               int dst_len, long long i0, int count, int det0) {
    const int det = det0 + blockIdx.y;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
        const long long i = i0 + e;
        const float v = src[det * src_det_stride + (i & src_mask)];
        uint16_t h, l;
        split_hilo<BF16>(v, h, l);
        const long long p = i & (dst_len - 1);
        hi[det * dst_det_stride + p] = h;
        hi[det * dst_det_stride + p + dst_len] = h;
        lo[det * dst_det_stride + p] = l;
        lo[det * dst_det_stride + p + dst_len] = l;
    }
}

}  // namespace lloid
