// Tensor-core (tcgen05) reconstruction for the split-precision paths.
//
// z = C Yhat (Eq. 6 with the upsampled slice outputs, so the ladder sum of
// Eq. 9 is the K-sum of one GEMM) for 128 templates x 128 samples per tile:
//   FP16 split: z = C Yhi + C Ylo                     (2 MMAs per re/im)
//   BF16 split: z = Chi Yhi + Chi Ylo + Clo Yhi       (3 MMAs per re/im)
// Operands are staged in shared memory by TMA (128-byte swizzle, K-major),
// the MMA is issued by one thread with accumulators in TMEM (two buffers of
// re + im, 4 x 128 columns), and four epilogue warps read the accumulators
// back with tcgen05.ld, form |z|^2 and keep the per-template argmax of the
// tile (the trigger stage of Section II.D.1).  Warp roles:
//   warp 0: TMA producer, warp 1: MMA issuer + TMEM owner, warps 2-5: epilogue.
// Every wait is bounded (about one second): on expiry the kernel records an
// error code, drains what it issued, frees TMEM and returns.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <vector>

#include "lloid_common.cuh"

namespace lloid {

constexpr int kTcTileN = 128;       // time samples per tile (MMA N)
constexpr int kTcTileM = 128;       // templates per tile (MMA M)
constexpr int kTcK = 64;            // K per stage: 64 x 2 B = one 128-byte swizzle row
constexpr unsigned long long kWaitNs = 1000000000ull;

struct TcMaps {
    CUtensorMap cre, cim, cre_lo, cim_lo, yhi, ylo;
};

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false (and *err set) after kWaitNs, or at once if another CTA failed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err, int code) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    for (;;) {
        for (int i = 0; i < 32; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (*reinterpret_cast<volatile int*>(err) != 0) return false;
        if (gtimer() - t0 > kWaitNs) {
            atomicCAS(err, 0, code);
            return false;
        }
    }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;                 // LBO (unused for swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;       // SBO
    d |= (uint64_t)1u << 46;                 // version
    d |= (uint64_t)2u << 61;                 // SWIZZLE_128B
    return d;
}
// Instruction descriptor, kind::f16: D = F32, A = B = F16 or BF16, K-major both.
__host__ __device__ constexpr uint32_t idesc_f16(bool bf16, int M, int N) {
    return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <bool BF16>
struct TcCfg {
    static constexpr int NA = BF16 ? 4 : 2;                 // A tiles per stage
    static constexpr int STAGES = BF16 ? 2 : 3;
    static constexpr int TILE_A = kTcTileM * kTcK * 2;      // 16 KB
    static constexpr int TILE_B = kTcTileN * kTcK * 2;      // 16 KB
    static constexpr int STAGE_BYTES = NA * TILE_A + 2 * TILE_B;
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 256;
};

// ---------------------------------------------------------------------------
// The kernel.  Work item = (detector, flat tile); a bank job's tiles run with
// the template tile fastest so that concurrent CTAs share Yhat tiles in L2.
// ---------------------------------------------------------------------------
template <bool BF16, bool STORE_Z>
__global__ void __launch_bounds__(192, 1)
    k_recon_tc(const ReconJob* __restrict__ jobs, const TcMaps* __restrict__ maps, const int* __restrict__ tile_base,
               int n_jobs, int tiles_per_det, long long k_a, int n, int det0, int n_det_push, long long window,
               Partial* __restrict__ part, long long part_tmpl_stride, int n_slots, float* __restrict__ zout,
               int* __restrict__ err) {
    using C = TcCfg<BF16>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::STAGES * C::STAGE_BYTES);
    uint64_t* empty = full + C::STAGES;
    uint64_t* tfull = empty + C::STAGES;
    uint64_t* tempty = tfull + 2;
    uint64_t* drain = tempty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) { mbar_init(full + s, 1); mbar_init(empty + s, 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(tfull + b, 1); mbar_init(tempty + b, 128); }
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
    const int total = tiles_per_det * n_det_push;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int issued = 0;            // stages issued but not yet seen consumed
            bool ok = true;
            for (int it = blockIdx.x; it < total && ok; it += gridDim.x) {
                const int det = det0 + it / tiles_per_det;
                const int t = it % tiles_per_det;
                int jlo = 0, jhi = n_jobs - 1;
                while (jlo < jhi) { int mid = (jlo + jhi + 1) >> 1; if (__ldg(tile_base + mid) <= t) jlo = mid; else jhi = mid - 1; }
                const ReconJob& jb = jobs[jlo];
                const TcMaps* mp = maps + jlo;
                const int local = t - tile_base[jlo];
                const int tm = local % jb.tiles_m, tt = local / jb.tiles_m;
                const int m0 = tm * kTcTileM;
                const int yrow = det * jb.ldy + tt * kTcTileN;
                for (int kc = 0; kc < jb.Kpad; kc += kTcK) {
                    if (!mbar_wait(empty + stage, phase ^ 1, err, 11)) { ok = false; break; }
                    uint8_t* sb = smem + stage * C::STAGE_BYTES;
                    mbar_expect_tx(full + stage, C::STAGE_BYTES);
                    tma_load_2d(sb + 0 * C::TILE_A, &mp->cre, full + stage, kc, m0);
                    tma_load_2d(sb + 1 * C::TILE_A, &mp->cim, full + stage, kc, m0);
                    if (BF16) {
                        tma_load_2d(sb + 2 * C::TILE_A, &mp->cre_lo, full + stage, kc, m0);
                        tma_load_2d(sb + 3 * C::TILE_A, &mp->cim_lo, full + stage, kc, m0);
                    }
                    tma_load_2d(sb + C::NA * C::TILE_A, &mp->yhi, full + stage, kc, yrow);
                    tma_load_2d(sb + C::NA * C::TILE_A + C::TILE_B, &mp->ylo, full + stage, kc, yrow);
                    if (++stage == C::STAGES) { stage = 0; phase ^= 1; }
                }
            }
            (void)issued;
            // Drain: every issued stage completes its transaction before exit.
            for (int s = 0; s < C::STAGES; ++s) {
                if (!mbar_wait(empty + stage, phase ^ 1, err, 12)) break;
                if (++stage == C::STAGES) { stage = 0; phase ^= 1; }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_f16(BF16, kTcTileM, kTcTileN);
            int stage = 0;
            uint32_t phase = 0;
            int i = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < total && ok; it += gridDim.x, ++i) {
                const int t = it % tiles_per_det;
                int jlo = 0, jhi = n_jobs - 1;
                while (jlo < jhi) { int mid = (jlo + jhi + 1) >> 1; if (__ldg(tile_base + mid) <= t) jlo = mid; else jhi = mid - 1; }
                const int Kpad = jobs[jlo].Kpad;
                const int buf = i & 1;
                if (!mbar_wait(tempty + buf, ((i >> 1) & 1) ^ 1, err, 13)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d_re = tmem + buf * 256;
                const uint32_t d_im = d_re + 128;
                for (int kc = 0; kc < Kpad; kc += kTcK) {
                    if (!mbar_wait(full + stage, phase, err, 14)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sb = smem_u32(smem + stage * C::STAGE_BYTES);
                    const uint32_t a_re = sb, a_im = sb + C::TILE_A;
                    const uint32_t a_re_lo = sb + 2 * C::TILE_A, a_im_lo = sb + 3 * C::TILE_A;
                    const uint32_t b_hi = sb + C::NA * C::TILE_A, b_lo = b_hi + C::TILE_B;
#pragma unroll
                    for (int k = 0; k < kTcK / 16; ++k) {
                        const uint32_t off = k * 32;      // 16 elements x 2 B along the swizzled row
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
                umma_commit(tfull + buf);
            }
            // Drain: all issued MMAs complete before TMEM is released.
            umma_commit(drain);
            mbar_wait(drain, 0, err, 15);
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int q = warp & 3;                  // TMEM lane quarter of this warp
        const int row = q * 32 + lane;           // template row within the tile
        int i = 0;
        for (int it = blockIdx.x; it < total; it += gridDim.x, ++i) {
            const int det = det0 + it / tiles_per_det;
            const int t = it % tiles_per_det;
            int jlo = 0, jhi = n_jobs - 1;
            while (jlo < jhi) { int mid = (jlo + jhi + 1) >> 1; if (__ldg(tile_base + mid) <= t) jlo = mid; else jhi = mid - 1; }
            const ReconJob& jb = jobs[jlo];
            const int local = t - tile_base[jlo];
            const int tm = local % jb.tiles_m, tt = local / jb.tiles_m;
            const int buf = i & 1;
            const bool got = mbar_wait(tfull + buf, (i >> 1) & 1, err, 16);
            if (!__all_sync(0xffffffffu, got)) break;     // warp-uniform: tcgen05.ld is .sync.aligned
            tc_fence_after();
            const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + buf * 256;
            const long long k0 = k_a + (long long)tt * kTcTileN;
            const long long kwin0 = (k0 / window) * window;
            float best = -1.f, bre = 0.f, bim = 0.f;
            int bk = 0x7fffffff;
            const int m = tm * kTcTileM + row;
#pragma unroll 1
            for (int c = 0; c < kTcTileN; c += 32) {
                float re[32], im[32];
                tmem_ld32(base + c, re);
                tmem_ld32(base + 128 + c, im);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float p = re[j] * re[j] + im[j] * im[j];
                    if (p > best) { best = p; bk = c + j; bre = re[j]; bim = im[j]; }
                }
                if (STORE_Z && m < jb.M) {
                    float* zr = zout + (long long)(2 * m) * n + tt * kTcTileN + c;
                    float* zi = zr + n;
#pragma unroll
                    for (int j = 0; j < 32; ++j) { zr[j] = re[j]; zi[j] = im[j]; }
                }
            }
            tc_fence_before();
            mbar_arrive(tempty + buf);
            if (!STORE_Z && m < jb.M) {
                const long long tile_abs = k0 / kTcTileN;
                const int slot = (int)(tile_abs & (n_slots - 1));
                part[(long long)(jb.tmpl0 + m) * part_tmpl_stride + (long long)det * n_slots + slot] =
                    make_float4(best, __int_as_float((int)(k0 - kwin0) + bk), bre, bim);
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
// a4 store for the split paths: Yhat^T[det][t][row] hi and lo halves, written
// through a shared-memory transpose so that global stores are row-contiguous.
// Tile = 64 basis rows x 64 samples, 256 threads, 16 outputs per thread.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T to_half_t(float v);
template <>
__device__ __forceinline__ __half to_half_t<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 to_half_t<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <typename T>
__device__ __forceinline__ float from_half_t(T v);
template <>
__device__ __forceinline__ float from_half_t<__half>(__half v) { return __half2float(v); }
template <>
__device__ __forceinline__ float from_half_t<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T>
__global__ void __launch_bounds__(256) k_upsample_t(const UpJob* __restrict__ jobs, const int* __restrict__ tile_base,
                                                    int n_jobs, long long k_a, int n, int det0) {
    extern __shared__ float Rs[];
    __shared__ T th[64][66];
    __shared__ T tl[64][66];
    const int t = blockIdx.x;
    int jlo = 0, jhi = n_jobs - 1;
    while (jlo < jhi) { int mid = (jlo + jhi + 1) >> 1; if (__ldg(tile_base + mid) <= t) jlo = mid; else jhi = mid - 1; }
    const UpJob& jb = jobs[jlo];
    const int local = t - tile_base[jlo];
    const int lt = local / jb.tiles_k, kt = local % jb.tiles_k;
    const int l0 = lt * 64;
    const int nl = min(64, jb.L - l0);
    for (int e = threadIdx.x; e < jb.rlen; e += blockDim.x) Rs[e] = __ldg(jb.R + e);
    __syncthreads();
    const int det = det0 + blockIdx.y;
    const int kk = threadIdx.x & 63, lg = threadIdx.x >> 6;
    const int k_local = kt * 64 + kk;
    const long long K = k_a + k_local;
    const long long e_max = (long long)jb.e_min + jb.rlen - 1;
    long long qa = K - e_max;
    const long long q_lo = (qa >= 0) ? (qa + jb.D - 1) / jb.D : -((-qa) / jb.D);
    long long qb = K - jb.e_min;
    const long long q_hi = (qb >= 0) ? qb / jb.D : -((-qb + jb.D - 1) / jb.D);
    float acc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i] = 0.f;
    const float* y = jb.yring + det * jb.y_det_stride;
    for (long long qq = q_lo; qq <= q_hi; ++qq) {
        const float r = Rs[K - (long long)jb.D * qq - jb.e_min];
        const long long yi = qq & jb.y_mask;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int l = l0 + lg * 16 + i;
            if (l < jb.L) acc[i] = fmaf(y[(long long)l * jb.y_ld + yi], r, acc[i]);
        }
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const T h = to_half_t<T>(acc[i]);
        th[kk][lg * 16 + i] = h;
        tl[kk][lg * 16 + i] = to_half_t<T>(acc[i] - from_half_t<T>(h));
    }
    __syncthreads();
    T* yh = static_cast<T*>(jb.yhat) + det * jb.yhat_det_stride;
    T* yl = static_cast<T*>(jb.yhat_lo) + det * jb.yhat_det_stride;
    // element (time r, basis c) -> Yhat^T[(kt*64 + r)][row0 + l0 + c]; yhat already points at row0
    for (int e = threadIdx.x; e < 64 * 64; e += 256) {
        const int r = e >> 6, c = e & 63;
        if (c >= nl || kt * 64 + r >= n) continue;
        const long long off = (long long)(kt * 64 + r) * jb.ldy + l0 + c;
        yh[off] = th[r][c];
        yl[off] = tl[r][c];
    }
}

// ---------------------------------------------------------------------------
// Host helpers
// ---------------------------------------------------------------------------
// FP16: C rounded to FP16 (hi only).  BF16: C = hi + lo, both BF16.
inline void pack_coeffs_tc(bool bf16, const std::vector<double>& cre, const std::vector<double>& cim, int Mpad,
                           int Kpad, std::vector<uint16_t>* hre, std::vector<uint16_t>* him,
                           std::vector<uint16_t>* lre, std::vector<uint16_t>* lim) {
    const size_t n = (size_t)Mpad * Kpad;
    hre->resize(n); him->resize(n);
    if (bf16) { lre->resize(n); lim->resize(n); } else { lre->clear(); lim->clear(); }
    for (size_t i = 0; i < n; ++i) {
        for (int part = 0; part < 2; ++part) {
            const float v = (float)(part ? cim[i] : cre[i]);
            uint16_t h, l = 0;
            if (bf16) {
                __nv_bfloat16 bh = __float2bfloat16_rn(v);
                __nv_bfloat16 bl = __float2bfloat16_rn(v - __bfloat162float(bh));
                std::memcpy(&h, &bh, 2); std::memcpy(&l, &bl, 2);
            } else {
                __half hh = __float2half_rn(v);
                std::memcpy(&h, &hh, 2);
            }
            (part ? *him : *hre)[i] = h;
            if (bf16) (part ? *lim : *lre)[i] = l;
        }
    }
}

}  // namespace lloid
