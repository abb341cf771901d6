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
//   reading.  Both terms are tensor-core products accumulated into the same
//   TMEM tile: Up_F restricted to one 128-sample tile is a fixed matrix U
//   (output q x window row w, entries z_{q mod F}[t] of Eq. 7), so
//   Up_F(Acc_{j-1}) = Acc_{j-1}[window] U^T, with the window and U each split
//   into 16-bit hi + lo halves (three products).  Acc is stored as hi/lo
//   planes, template-major with time contiguous, which is the K-major layout
//   the next level's MMA reads.  The top level (f0) forms |z|^2 and the
//   per-tile argmax instead of storing Acc.
#pragma once
#include "kernels_tc.cuh"

namespace lloid {

// Both kernels run a static schedule built on the host: sched[0 .. grid] are
// per-CTA offsets into the tile ids that follow; a tile id `it` is detector
// det0 + it % n_det_push and tile it / n_det_push of the launch's job table.
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
    uint16_t* acc_out;             // non-top: hi/lo planes [det][re hi, re lo, im hi, im lo][acc_cols / 8][Mpad][8]
                                   // (time-blocked; column 0 = sample floor8(lo) - 128)
    long long acc_out_det_stride;  // elements
    int acc_cols;                  // plane row length (multiple of 128)
    int Kp;                        // Kpad of the level (0: no slice at this rate)
    int M, Mpad, tmpl0;
    int tiles_m, tiles_t;
    int D, Lambda;                 // this level
    int F, D_lo, Lambda_lo;        // factor to the level below (0: lowest level)
    int y_rows;                    // level ring rows
    int map;                       // index into the level tensor-map array
    uint32_t* zring;               // top level of an Eq. 10 bank: [det][Mpad][zring_len] z as half2, else null
    long long zring_det_stride;
    int zring_len;
};

struct FirMaps { CUtensorMap a, a_lo; };

// accw: the level below's hi/lo planes, time-blocked [det x plane][x / 8][Mpad][8]
// (4-D map whose innermost dimension is 32 templates x 8 samples = 512 B, box
// 4 of those x 4 blocks, no swizzle: a box is four contiguous 2 KB runs and lands
// in shared memory as the no-swizzle K-major layout of a 128 x 32 operand);
// uhi/ulo: the Eq. 8 tile matrices U_F of this level's factor, time-blocked the
// same way, [shift][window row / 8][128 outputs][8], same box.
struct LevelMaps { CUtensorMap cre, cim, cre_lo, cim_lo, yhi, ylo, accw, uhi, ulo; };

// Window of the level below read by one 128-sample tile (N_up = 8): rows
// floor(Q/F) - N_up - r .. floor(Q/F) + 127/F + N_up, where the shift r =
// floor(Q/F) mod 8 aligns the first row to 16 bytes (r = 0 for F <= 16, r in
// {0, 4} for F = 32, {0, 2, 4, 6} for F = 64); whole 32-row stages.
constexpr int kWinK = 32;
__host__ __device__ constexpr int win_rows(int F) { return F ? 127 / F + 17 : 0; }
__host__ __device__ constexpr int win_shift_max(int F) { return F == 64 ? 6 : (F == 32 ? 4 : 0); }
__host__ __device__ constexpr int win_chunks(int F) {
    return F ? (win_rows(F) + win_shift_max(F) + kWinK - 1) / kWinK : 0;
}

// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t desc_nosw(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1u << 46;
    return d;   // layout type 0: no swizzle
}
// A window plane in shared memory: [4 blocks of 8 window rows][128 templates][8 x 16 bit], the
// no-swizzle K-major layout with 8 x 16 B core matrices, 128 B apart along M and 2 KB along K.
__device__ __forceinline__ uint64_t desc_win(uint32_t saddr) { return desc_nosw(saddr, 2048, 128); }
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory"); }

// Per-tile facts, written by the host with the job tables: x = job, y = tile index within the
// job, z = K'pad of the job, w = its N (FIR c-groups per tile) or, for a ladder level, the
// number of 16-wide K steps that hold bases (K'pad is a multiple of 64; steps past w are zero).  One load
// replaces a search of the job table, and the MMA issuers read the next tile's entry while the
// current tile's MMAs run.
using TileInfo = int4;
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

// Two values at once: hi = round(a, b) as a packed pair, lo = round((a, b) - hi).
template <bool BF16>
__device__ __forceinline__ void split_hilo2(float a, float b, uint32_t& hi, uint32_t& lo) {
    if (BF16) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    } else {
        const __half2 h = __floats2half2_rn(a, b);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    }
}

// ---------------------------------------------------------------------------
// a2 on the tensor cores
// ---------------------------------------------------------------------------
template <bool BF16>
struct FirCfg {
    static constexpr int MAX_STAGES = 8;                       // runtime count: as many as shared memory allows
    static constexpr int TILE_A = 128 * kTcK * 2;              // 16 KB
    static constexpr int STAGE_BYTES = (BF16 ? 2 : 1) * TILE_A;
    static constexpr int EPI_LD = 24;                          // staging row pitch (halves): conflict-free, 16 B aligned
    static constexpr int EPI_BYTES = 2 * 256 * EPI_LD * 2;     // staging [256 q][16 bases (+pad)] hi + lo
};

template <bool BF16>
__global__ void __launch_bounds__(192, 1)
    k_fir_tc(const FirTcJob* __restrict__ jobs, const FirMaps* __restrict__ maps, const TileInfo* __restrict__ tinfo,
             const int* __restrict__ sched, int n_jobs, int tiles_per_det, long long k_a, int det0, int n_det_push, int strip_bytes,
             int n_stages, int* __restrict__ err) {
    using C = FirCfg<BF16>;
    pdl_launch_dependents();
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);   // 1 KB aligned, still a shared pointer
    uint8_t* stage_area = smem;
    uint8_t* strip_area = smem + n_stages * C::STAGE_BYTES;                // 2 buffers x (hi, lo) x strip_bytes
    uint16_t* epi = reinterpret_cast<uint16_t*>(strip_area + 4 * strip_bytes);
    uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(epi) + C::EPI_BYTES);
    uint64_t* a_full = bars;
    uint64_t* a_empty = a_full + n_stages;
    uint64_t* s_full = a_empty + n_stages;
    uint64_t* s_empty = s_full + 2;
    uint64_t* t_full = s_empty + 2;
    uint64_t* t_empty = t_full + 2;
    uint64_t* drain = t_empty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < n_stages; ++s) { mbar_init(a_full + s, 1); mbar_init(a_empty + s, 1); }
        for (int b = 0; b < 2; ++b) {
            mbar_init(s_full + b, 1); mbar_init(s_empty + b, 1);
            mbar_init(t_full + b, 1); mbar_init(t_empty + b, kEpiThreads);
        }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        // 256 columns: two FIR CTAs can share an SM's TMEM
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    pdl_wait();   // inputs of this launch are written by the previous kernels of the stream

    if (warp == 0) {
        if (lane == 0) {   // ------------------------------------------------ producer
            int stage = 0, sb = 0;
            uint32_t phase = 0, sphase = 0;
            bool ok = true;
            for (int k = sched[blockIdx.x]; k < sched[blockIdx.x + 1] && ok; ++k) {
                const int it = sched[gridDim.x + 1 + k];
                const int det = det0 + it % n_det_push;
                const TileInfo ti = tinfo[it / n_det_push];
                const FirTcJob jb = jobs[ti.x];   // a copy: the asm "memory" clobbers would reload it
                const int local = ti.y;
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
                    if (++stage == n_stages) { stage = 0; phase ^= 1; }
                }
            }
            for (int s = 0; s < n_stages; ++s) {                 // drain the A stages
                if (!mbar_wait(a_empty + stage, phase ^ 1, err, 23)) break;
                if (++stage == n_stages) { stage = 0; phase ^= 1; }
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
            const int kb = sched[blockIdx.x], ke = sched[blockIdx.x + 1];
            TileInfo tnext = kb < ke ? tinfo[sched[gridDim.x + 1 + kb] / n_det_push] : TileInfo{};
            int snext = kb + 1 < ke ? sched[gridDim.x + 1 + kb + 1] : 0;
            for (int k = kb; k < ke && ok; ++k, ++i) {
                const TileInfo tcur = tnext;             // the next entries load while this tile runs
                if (k + 1 < ke) tnext = tinfo[snext / n_det_push];
                if (k + 2 < ke) snext = sched[gridDim.x + 1 + k + 2];
                const int Kp = tcur.z, NC = tcur.w;
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
                    if (++stage == n_stages) { stage = 0; phase ^= 1; }
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
        for (int k = sched[blockIdx.x]; k < sched[blockIdx.x + 1]; ++k, ++i) {
            const int it = sched[gridDim.x + 1 + k];
            const int det = det0 + it % n_det_push;
            const TileInfo ti = tinfo[it / n_det_push];
            const FirTcJob jb = jobs[ti.x];   // a copy: the asm "memory" clobbers would reload it
            const int local = ti.y;
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
                // 256 rows x 32 B (hi) + 256 x 32 B (lo) as 16-byte stores.  Only the first of the
                // ring's two mappings is written: the level kernel reads 128-row boxes that start
                // at multiples of 128 in a power-of-two ring, which never wrap.
                for (int e = et; e < 2 * 256 * 2; e += kEpiThreads) {
                    const int part = e >> 9;             // 0 hi, 1 lo
                    const int r = (e >> 1) & 255, h16 = e & 1;
                    const long long q = 8 * (c0 + cc) + r;
                    if (cc + (r >> 3) >= jb.NC || q < qa || q >= qa + jb.q_count) continue;
                    const uint4 val = *reinterpret_cast<const uint4*>(epi + part * 256 * C::EPI_LD + r * C::EPI_LD + h16 * 8);
                    uint16_t* dst = part ? yl : yh;
                    const long long rr = q & (jb.y_rows - 1);
                    *reinterpret_cast<uint4*>(dst + rr * jb.y_ld + h16 * 8) = val;
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
template <bool BF16, bool TOP>
struct LevCfg {
    static constexpr int NA = BF16 ? 4 : 2;
    static constexpr int STAGES = BF16 ? 2 : 3;
    static constexpr int TILE_A = kTcTileM * kTcK * 2;
    static constexpr int TILE_B = kTcTileN * kTcK * 2;
    static constexpr int STAGE_BYTES = NA * TILE_A + 2 * TILE_B;
    static constexpr int WTILE = 128 * kWinK * 2;      // one window plane or one U half: 128 rows x 64 B
    static constexpr int WSTAGE = 6 * WTILE;           // re hi, re lo, im hi, im lo, U hi, U lo
    static_assert(WSTAGE <= STAGE_BYTES, "a window stage fits a stage slot");
    static constexpr int EPI_WARPS = 8;                 // two per TMEM lane quarter, 64 columns each
    static constexpr int STG_PITCH = 80;               // 32 samples x 2 B + 16 B pad: conflict-free rows
    static constexpr int STG_BUF = 32 * STG_PITCH;     // one warp's 32 templates x 32 samples
    static constexpr int STG = EPI_WARPS * STG_BUF;    // per-warp transpose buffers (planes; the top's SNR history)
    static constexpr int XCHG = TOP ? 4 * 128 * 16 : 0;   // top: tile and tail argmax exchange between the column halves
    static constexpr int SMEM = STAGES * STAGE_BYTES + STG + XCHG + 1024 + 256;
    static constexpr int THREADS = 64 + 32 * EPI_WARPS;
};

// F: the factor to the level below (0 at the lowest level), a template
// parameter so that the window stages and their MMAs are unrolled.
template <bool BF16, bool TOP, bool STORE_Z, int F>
__global__ void __launch_bounds__(LevCfg<BF16, TOP>::THREADS, 1)
    k_level_tc(const LevelJob* __restrict__ jobs, const LevelMaps* __restrict__ maps,
               const TileInfo* __restrict__ tinfo, const int* __restrict__ sched, int n_jobs, int tiles_per_det, long long k_a, long long k_b,
               int det0, int n_det_push, long long window, Partial* __restrict__ part, long long part_tmpl_stride,
               int n_slots, TailRing tail, float* __restrict__ zout, int* __restrict__ err) {
    using C = LevCfg<BF16, TOP>;
    pdl_launch_dependents();
    constexpr int EPI = 32 * C::EPI_WARPS;
    constexpr int NWC = win_chunks(F);
    constexpr int NK16 = (win_rows(F) + win_shift_max(F) + 15) / 16;   // K steps of 16 rows that U can reach
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);   // 1 KB aligned, still a shared pointer
    uint8_t* stg = smem + C::STAGES * C::STAGE_BYTES;
    float4* xchg = reinterpret_cast<float4*>(stg + C::STG);
    uint64_t* full = reinterpret_cast<uint64_t*>(stg + C::STG + C::XCHG);
    uint64_t* empty = full + C::STAGES;
    uint64_t* tfull = empty + C::STAGES;
    uint64_t* tempty = tfull + 2;
    uint64_t* drain = tempty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) { mbar_init(full + s, 1); mbar_init(empty + s, 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(tfull + b, 1); mbar_init(tempty + b, EPI); }
        mbar_init(drain, 1);
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
    pdl_wait();   // inputs of this launch are written by the previous kernels of the stream

    if (warp == 0) {
        if (lane == 0) {   // ------------------------------------------------ producer
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int k = sched[blockIdx.x]; k < sched[blockIdx.x + 1] && ok; ++k) {
                const int it = sched[gridDim.x + 1 + k];
                const int det = det0 + it % n_det_push;
                const TileInfo ti = tinfo[it / n_det_push];
                const LevelJob jb = jobs[ti.x];   // a copy: the asm "memory" clobbers would reload it
                const LevelMaps* mp = maps + jb.map;
                const int local = ti.y;
                const int tm = local % jb.tiles_m, tt = local / jb.tiles_m;
                const long long Qt = fdiv(fdiv(k_a - jb.Lambda, jb.D), 128) * 128 + 128LL * tt;
                const int yrow = det * 2 * jb.y_rows + (int)(Qt & (jb.y_rows - 1));
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
                if (F != 0) {
                    // window of the level below: its planes start at sample X0 = floor8(lo_below) - 128;
                    // the first row read is floor(Qt/F) - N_up - r (a multiple of 8 past X0)
                    const long long X0 = fdiv(fdiv(k_a - jb.Lambda_lo, jb.D_lo), 8) * 8 - 128;
                    const long long qf = fdiv(Qt, F != 0 ? F : 1);
                    const int r = (int)(qf & 7);
                    const int a = (int)(qf - 8 - r - X0);
#pragma unroll 1
                    for (int ch = 0; ch < NWC && ok; ++ch) {
                        if (!mbar_wait(empty + stage, phase ^ 1, err, 32)) { ok = false; break; }
                        uint8_t* sb = smem + stage * C::STAGE_BYTES;
                        mbar_expect_tx(full + stage, C::WSTAGE);
#pragma unroll
                        for (int pl = 0; pl < 4; ++pl)
                            tma_load_4d(sb + pl * C::WTILE, &mp->accw, full + stage, 0, tm * 4, (a + kWinK * ch) >> 3,
                                        det * 4 + pl);
                        tma_load_4d(sb + 4 * C::WTILE, &mp->uhi, full + stage, 0, 0, (kWinK * ch) >> 3, r);
                        tma_load_4d(sb + 5 * C::WTILE, &mp->ulo, full + stage, 0, 0, (kWinK * ch) >> 3, r);
                        if (++stage == C::STAGES) { stage = 0; phase ^= 1; }
                    }
                }
            }
            for (int s = 0; s < C::STAGES; ++s) {
                if (!mbar_wait(empty + stage, phase ^ 1, err, 38)) break;
                if (++stage == C::STAGES) { stage = 0; phase ^= 1; }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {   // ------------------------------------------------ MMA issuer
            constexpr uint32_t idesc = idesc_f16(BF16, kTcTileM, kTcTileN);
            int stage = 0, i = 0;
            uint32_t phase = 0;
            bool ok = true;
            const int kb = sched[blockIdx.x], ke = sched[blockIdx.x + 1];
            TileInfo tnext = kb < ke ? tinfo[sched[gridDim.x + 1 + kb] / n_det_push] : TileInfo{};
            int snext = kb + 1 < ke ? sched[gridDim.x + 1 + kb + 1] : 0;
            for (int k = kb; k < ke && ok; ++k, ++i) {
                const TileInfo tcur = tnext;             // the next entries load while this tile runs
                if (k + 1 < ke) tnext = tinfo[snext / n_det_push];
                if (k + 2 < ke) snext = sched[gridDim.x + 1 + k + 2];
                const int Kp = tcur.z;
                const int nk16 = tcur.w;                 // K steps of 16 that hold bases (the rest of Kp is zero)
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
                        if (kc / 16 + k >= nk16) break;
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
#pragma unroll 1
                for (int ch = 0; ch < NWC && ok; ++ch) {
                    if (!mbar_wait(full + stage, phase, err, 30)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sb = smem_u32(smem + stage * C::STAGE_BYTES);
                    const uint32_t w_rh = sb, w_rl = sb + C::WTILE, w_ih = sb + 2 * C::WTILE, w_il = sb + 3 * C::WTILE;
                    const uint32_t u_h = sb + 4 * C::WTILE, u_l = sb + 5 * C::WTILE;
#pragma unroll
                    for (int k = 0; k < kWinK / 16; ++k) {
                        if (ch * (kWinK / 16) + k >= NK16) break;   // rows past the window: U is zero there
                        const uint32_t woff = k * 4096;         // two 8-row blocks of 128 x 16 B (window and U)
                        const uint32_t acc0 = (Kp > 0 || ch > 0 || k > 0) ? 1u : 0u;
                        umma_f16(d_re, desc_win(w_rh + woff), desc_win(u_h + woff), idesc, acc0);
                        umma_f16(d_re, desc_win(w_rl + woff), desc_win(u_h + woff), idesc, 1u);
                        umma_f16(d_re, desc_win(w_rh + woff), desc_win(u_l + woff), idesc, 1u);
                        umma_f16(d_im, desc_win(w_ih + woff), desc_win(u_h + woff), idesc, acc0);
                        umma_f16(d_im, desc_win(w_il + woff), desc_win(u_h + woff), idesc, 1u);
                        umma_f16(d_im, desc_win(w_ih + woff), desc_win(u_l + woff), idesc, 1u);
                    }
                    umma_commit(empty + stage);
                    if (++stage == C::STAGES) { stage = 0; phase ^= 1; }
                }
                if (!ok) break;
                umma_commit(tfull + buf);
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
        int i = 0;
        for (int k = sched[blockIdx.x]; k < sched[blockIdx.x + 1]; ++k, ++i) {
            const int it = sched[gridDim.x + 1 + k];
            const int det = det0 + it % n_det_push;
            const TileInfo ti = tinfo[it / n_det_push];
            const LevelJob jb = jobs[ti.x];   // a copy: the asm "memory" clobbers would reload it
            const int local = ti.y;
            const int tm = local % jb.tiles_m, tt = local / jb.tiles_m;
            const int buf = i & 1;
            const bool got = mbar_wait(tfull + buf, (i >> 1) & 1, err, 36);
            if (!__all_sync(0xffffffffu, got)) break;
            tc_fence_after();
            const long long lo = fdiv(k_a - jb.Lambda, jb.D);
            const long long Q0 = fdiv(lo, 128) * 128;
            const int m = tm * kTcTileM + rowm;
            const uint32_t base = tmem + ((uint32_t)(qd * 32) << 16) + buf * 256;
            const bool has_acc = jb.Kp > 0 || F != 0;
            float best = -1.f, bre = 0.f, bim = 0.f;
            int bk = 0x7fffffff;
            // window overlap: the last ov samples of a tile that ends where a window starts
            const long long ktile = Q0 + 128LL * tt;
            const bool pre = tail.ov > 0 && (ktile + 128) % window == 0;
            const int tail_from = pre ? 128 - tail.ov : 128;
            float tbest = -1.f, tre = 0.f, tim = 0.f;
            int tk = 0x7fffffff;
            if (TOP) {
#pragma unroll 1
                for (int c = half * 64; c < half * 64 + 64; c += 16) {
                    float re[16], im[16];
                    if (has_acc) {
                        tmem_ld16(base + c, re);
                        tmem_ld16(base + 128 + c, im);
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j) { re[j] = 0.f; im[j] = 0.f; }
                    }
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float p = re[j] * re[j] + im[j] * im[j];
                        if (p > best) { best = p; bk = c + j; bre = re[j]; bim = im[j]; }
                        if (c + j >= tail_from && p > tbest) { tbest = p; tk = c + j; tre = re[j]; tim = im[j]; }
                    }
                    if (STORE_Z && m < jb.M) {
                        const int n = (int)(k_b - k_a);
                        float* zr = zout + (long long)(2 * m) * n + tt * kTcTileN + c;
                        float* zi = zr + n;
#pragma unroll
                        for (int j = 0; j < 16; ++j) { zr[j] = re[j]; zi[j] = im[j]; }
                    }
                    if (jb.zring != nullptr) {
                        // Eq. 10 history: z as half2, transposed through the warp's buffer so that
                        // each store instruction writes 8 template rows x 64 contiguous bytes
                        uint8_t* wbuf = stg + (warp - 2) * C::STG_BUF;
                        uint32_t h[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const __half2 v = __floats2half2_rn(re[j], im[j]);
                            h[j] = *reinterpret_cast<const uint32_t*>(&v);
                        }
#pragma unroll
                        for (int g = 0; g < 4; ++g)
                            *reinterpret_cast<uint4*>(wbuf + lane * C::STG_PITCH + g * 16) =
                                make_uint4(h[4 * g], h[4 * g + 1], h[4 * g + 2], h[4 * g + 3]);
                        __syncwarp();
                        const int rr = lane >> 2, cq = lane & 3;
                        const long long pos = (Q0 + 128LL * tt + c + 4 * cq) & (jb.zring_len - 1);
                        uint32_t* zbase = jb.zring + det * jb.zring_det_stride +
                                          (long long)(tm * kTcTileM + qd * 32) * jb.zring_len + pos;
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int r = 8 * i + rr;
                            *reinterpret_cast<uint4*>(zbase + (long long)r * jb.zring_len) =
                                *reinterpret_cast<const uint4*>(wbuf + r * C::STG_PITCH + cq * 16);
                        }
                        __syncwarp();
                    }
                }
            } else {
                // Acc of this warp's 32 templates x 64 samples as four hi/lo planes in the time-blocked
                // layout [plane][x / 8][Mpad][8]: for each block of 8 samples the warp's 32 rows are
                // 512 contiguous bytes, one 16-byte store per lane.  Plane columns start at
                // X0 = floor8(lo) - 128 (a tile never writes left of column 0).
                const long long X0 = fdiv(lo, 8) * 8 - 128;
                const long long x0 = Q0 + 128LL * tt + 64 * half - X0;   // a multiple of 8
                const long long pstride = (long long)jb.Mpad * jb.acc_cols;
                uint16_t* pbase = jb.acc_out + det * jb.acc_out_det_stride + (long long)(tm * 128 + qd * 32 + lane) * 8;
#pragma unroll 1
                for (int part = 0; part < 2; ++part) {          // re, im
#pragma unroll 1
                    for (int g = 0; g < 2; ++g) {               // samples 32 g .. 32 g + 31 of the half
                        float v[32];
                        if (has_acc) {
                            tmem_ld32(base + part * 128 + 64 * half + 32 * g, v);
                        } else {
#pragma unroll
                            for (int j = 0; j < 32; ++j) v[j] = 0.f;
                        }
                        uint32_t hp[16], lp[16];
#pragma unroll
                        for (int k = 0; k < 16; ++k) split_hilo2<BF16>(v[2 * k], v[2 * k + 1], hp[k], lp[k]);
                        const long long blk0 = (x0 + 32 * g) >> 3;
#pragma unroll
                        for (int bq = 0; bq < 4; ++bq) {
                            const long long o = (blk0 + bq) * jb.Mpad * 8;
                            *reinterpret_cast<uint4*>(pbase + (2 * part) * pstride + o) =
                                make_uint4(hp[4 * bq], hp[4 * bq + 1], hp[4 * bq + 2], hp[4 * bq + 3]);
                            *reinterpret_cast<uint4*>(pbase + (2 * part + 1) * pstride + o) =
                                make_uint4(lp[4 * bq], lp[4 * bq + 1], lp[4 * bq + 2], lp[4 * bq + 3]);
                        }
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(tempty + buf);
            if (TOP && !STORE_Z) {
                // the later half hands its tile argmax to the earlier half (which wins ties)
                float4* xb = xchg + buf * 128;
                float4* xt = xchg + (2 + buf) * 128;
                if (half == 1) {
                    xb[rowm] = make_float4(best, __int_as_float(bk), bre, bim);
                    xt[rowm] = make_float4(tbest, __int_as_float(tk), tre, tim);
                }
                asm volatile("bar.sync 1, %0;" ::"n"(EPI) : "memory");
                if (half == 0 && m < jb.M) {
                    const float4 o = xb[rowm];
                    if (o.x > best) { best = o.x; bk = __float_as_int(o.y); bre = o.z; bim = o.w; }
                    const long long k0 = Q0 + 128LL * tt;         // Q0 == lo == k_a at the top level
                    const long long kwin0 = (k0 / window) * window;
                    const int slot = (int)((k0 / kTcTileN) & (n_slots - 1));
                    part[(long long)(jb.tmpl0 + m) * part_tmpl_stride + (long long)det * n_slots + slot] =
                        make_float4(best, __int_as_float((int)(k0 - kwin0) + bk), bre, bim);
                    if (pre) {
                        const float4 ot = xt[rowm];
                        if (ot.x > tbest) { tbest = ot.x; tk = __float_as_int(ot.y); tre = ot.z; tim = ot.w; }
                        const long long w1 = (k0 + 128) / window;
                        tail.p[(long long)(jb.tmpl0 + m) * tail.tmpl_stride + (long long)det * tail.n + (w1 & (tail.n - 1))] =
                            make_float4(tbest, __int_as_float((int)(k0 - w1 * window) + tk), tre, tim);
                    }
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
// A slice of a bank in the f0 form (kernels_f0.cuh): where its FIR output is
// and the composed Eq. 7-8 upsampler that brings it to f0.
// ---------------------------------------------------------------------------
struct YupSlice {
    const uint16_t* y_hi;          // level ring of the slice's rate, first column of the slice, detector 0
    const uint16_t* y_lo;
    long long y_det_stride;        // elements
    const float* R;                // composed upsampler [rlen]
    int y_rows, y_ld;              // level ring rows (power of two) and row length
    int e_min, rlen, D, L;         // response support [e_min, e_min + rlen); L bases
    int tcol;                      // first column of the slice in the packed f0 ring
    int nq;                        // rows of Y a 128-sample tile reaches (the same for every tile)
    int qoff;                      // first of them: tile start / D + qoff
    int roff;                      // offset of R in the bank's staged upsamplers
};

}  // namespace lloid
