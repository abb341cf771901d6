// tcgen05 / TMA / mbarrier building blocks shared by the tensor-core kernels
// (kernels_tc2.cuh): inline-PTX wrappers, shared-memory matrix descriptors,
// the kind::f16 instruction descriptor, bounded mbarrier waits, the pipeline
// geometry constants, and host-side packing of coefficients into FP16 or
// BF16 hi + lo halves.
//
// Every wait is bounded (about one second): on expiry a kernel records an
// error code in a device flag that the host reads, drains what it issued,
// frees its TMEM and returns.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "lloid_common.cuh"

namespace lloid {

constexpr int kTcTileN = 128;       // time samples per tile (MMA N)
constexpr int kTcTileM = 128;       // templates per tile (MMA M)
constexpr int kTcK = 64;            // K per stage: 64 x 2 B = one 128-byte swizzle row
constexpr unsigned long long kWaitNs = 1000000000ull;

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
// Bounded wait: false (and *err set to code) after limit_ns, or at once if another CTA failed.
__device__ __forceinline__ bool mbar_wait_ns(uint64_t* bar, uint32_t parity, int* err, int code,
                                             unsigned long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    for (;;) {
        for (int i = 0; i < 32; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (*reinterpret_cast<volatile int*>(err) != 0) return false;
        if (gtimer() - t0 > limit_ns) {
            atomicCAS(err, 0, code);
            return false;
        }
    }
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err, int code) {
    return mbar_wait_ns(bar, parity, err, code, kWaitNs);
}

// The bounded wait itself, on its own: one thread waits on a shared-memory barrier
// that nothing completes, with the given limit; the expiry leaves `code` in *err the
// way an expired pipeline wait does.  Nothing else is in flight, so the kernel simply
// returns.  (Used to check the expiry path and its report on the host.)
__global__ void k_wait_expiry_check(int* err, int code, unsigned long long limit_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_wait_ns(&bar, 0, err, code, limit_ns);
    }
}

// A delay of the stream by a bounded spin on the global timer (a slow device, for the
// host-side timeout paths).
__global__ void k_delay(unsigned long long ns) {
    const unsigned long long t0 = gtimer();
    while (gtimer() - t0 < ns) {
    }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
        : "memory");
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2,
                                            int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
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

// The same load without the wait, so that several loads are in flight before one
// tcgen05.wait::ld (tmem_wait_ld) makes all of their registers valid.
__device__ __forceinline__ void tmem_ld32_nw(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// 16 columns, no wait; see tmem_wait_ld16 for the wait that makes them readable.
__device__ __forceinline__ void tmem_ld16_nw(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
// tcgen05.wait::ld with the destination registers of the loads in flight as in/out operands:
// the compiler then reads them only after the wait.
__device__ __forceinline__ void tmem_wait_ld16(uint32_t (&a)[16], uint32_t (&b)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7]),
                   "+r"(a[8]), "+r"(a[9]), "+r"(a[10]), "+r"(a[11]), "+r"(a[12]), "+r"(a[13]), "+r"(a[14]),
                   "+r"(a[15]), "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3]), "+r"(b[4]), "+r"(b[5]), "+r"(b[6]),
                   "+r"(b[7]), "+r"(b[8]), "+r"(b[9]), "+r"(b[10]), "+r"(b[11]), "+r"(b[12]), "+r"(b[13]),
                   "+r"(b[14]), "+r"(b[15])
                 :
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
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
// Host helpers
// ---------------------------------------------------------------------------
// v = hi + lo with both halves FP16 (or BF16): hi = round(v), lo = round(v - hi).
inline void split_hilo_host(bool bf16, const std::vector<double>& v, std::vector<uint16_t>* hi,
                            std::vector<uint16_t>* lo) {
    hi->resize(v.size());
    lo->resize(v.size());
    for (size_t i = 0; i < v.size(); ++i) {
        const float x = (float)v[i];
        if (bf16) {
            __nv_bfloat16 bh = __float2bfloat16_rn(x);
            __nv_bfloat16 bl = __float2bfloat16_rn(x - __bfloat162float(bh));
            std::memcpy(&(*hi)[i], &bh, 2);
            std::memcpy(&(*lo)[i], &bl, 2);
        } else {
            __half hh = __float2half_rn(x);
            __half hl = __float2half_rn(x - __half2float(hh));
            std::memcpy(&(*hi)[i], &hh, 2);
            std::memcpy(&(*lo)[i], &hl, 2);
        }
    }
}

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
