// The f0 form of a bank on the tensor cores: slice upsampling (Eq. 7-8),
// reconstruction (Eq. 6) and the trigger window maxima (Section II.D.1) in
// one kernel.
//
// Eq. 6 and Eq. 7-8 are linear and the coefficients do not depend on time, so
// the bank's SNR is z = C Yhat with Yhat_l[k] = sum_q Y_l[q] R[k - D q - e_min]:
// every slice's basis outputs brought up to f0 through the slice's ladder of
// Eq. 7-8 upsamplers composed into one polyphase filter R (R = [1] at f0).
// The columns of Yhat are the bank's bases packed slice after slice, so K is
// the bank's basis count rounded up to 16.
//
// A work unit is (bank, detector, a group of tpw consecutive 128-sample tiles
// of the push, tpw = window / 128).  Per tile of the group:
//   builder warps (4): Yhat rows of the tile, computed in FP32 from the FIR's
//     hi/lo output at each slice's rate, split into hi/lo halves and stored in
//     shared memory in the no-swizzle K-major layout ([K/8][128 rows][8]);
//   producer (1 thread): the coefficient tiles of the bank's 128-template
//     groups, 32 bases per TMA stage, from time-blocked planes
//     [re hi, im hi, (re lo, im lo)][K/8][Mpad][8];
//   MMA issuer (1 thread): for every template group, C Yhat into a TMEM
//     accumulator (re and im, 128 columns each, two buffers), hi/lo products
//     (FP16: C_hi Y_hi + C_hi Y_lo; BF16: + C_lo Y_hi);
//   epilogue warps (8): |z|^2 and its argmax over the tile (earliest sample on
//     ties), kept per template across the group.
// When the push starts on a window boundary every group is one whole trigger
// window: its end writes each template's window maximum to the trigger slab
// (threshold, phase) and flags the bank's loudest template, as the window
// finalisation does for the ladder form.  Otherwise each tile's maximum goes
// to the partial ring and the window finalisation takes it from there.
#pragma once
#include "kernels_tc2.cuh"

namespace lloid {

struct F0Job {
    int M, Mpad, tmpl0, K;         // templates, padded, first global template, packed K (multiple of 16)
    int tiles_m;                   // Mpad / 128 (at most kF0MaxTm)
    int s0, ns;                    // the bank's slices in the slice table (YupSlice)
    int map;                       // index into the coefficient maps
};
struct F0Maps { CUtensorMap c; };  // [planes][K/8][Mpad][8], box 128 rows x 32 bases of one plane
struct F0Unit { int job, g; };     // group g: tiles [g tpw, min((g + 1) tpw, n / 128)) of the push

constexpr int kF0MaxTm = 8;        // template groups per bank (M <= 1024)
constexpr int kF0Builders = 4;     // builder warps 2..5
constexpr int kF0EpiWarps = 8;     // epilogue warps 6..13
constexpr int kF0Threads = 32 * (2 + kF0Builders + kF0EpiWarps);
constexpr int kF0CStages = 4;

template <bool BF16>
struct F0Cfg {
    static constexpr int NPL = BF16 ? 4 : 2;               // coefficient planes
    static constexpr int CPLANE = 128 * 32 * 2;            // one plane of a 32-basis stage (8 KB)
    static constexpr int CSTAGE = NPL * CPLANE;
};
// Shared memory of one launch class: K <= kc (64 or 128) with ybufs Yhat buffers.
__host__ __device__ constexpr int f0_smem_bytes(bool bf16, int kc, int ybufs) {
    return kF0CStages * (bf16 ? 4 : 2) * 8192 + ybufs * 2 * 128 * kc * 2 + kF0MaxTm * 128 * 16 + 2 * 128 * 16 +
           4 * 16 + 1024 + 512;
}

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

template <bool BF16, bool STORE_Z>
__global__ void __launch_bounds__(kF0Threads, 1)
    k_f0_top(const F0Job* __restrict__ jobs, const F0Maps* __restrict__ maps, const YupSlice* __restrict__ slices,
             const F0Unit* __restrict__ units, const int* __restrict__ sched, int n_units, int kc, int ybufs,
             long long k_a, int n, int det0, int n_det_push, long long window, float threshold,
             Partial* __restrict__ part, long long part_tmpl_stride, int n_slots, SlabEntry* __restrict__ slab_base,
             int ring, int n_det_total, long long slab_det_stride, float* __restrict__ zout, int* __restrict__ err) {
    using C = F0Cfg<BF16>;
    pdl_launch_dependents();
    const int tpw = (int)(window / 128);
    const int n_tiles = n / 128;
    const bool aligned = (k_a % window) == 0;              // every group is one whole window
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* cst = smem;                                   // kF0CStages x CSTAGE
    uint8_t* ybuf = cst + kF0CStages * C::CSTAGE;          // ybufs x [hi, lo][kc / 8][128][8]
    const int yplane = 128 * kc * 2;
    float4* rs = reinterpret_cast<float4*>(ybuf + ybufs * 2 * yplane);   // [kF0MaxTm][128] running window maxima
    float4* xchg = rs + kF0MaxTm * 128;                    // [2][128]
    float4* red = xchg + 2 * 128;                          // [4] bank-max partials of the half-0 warps
    uint64_t* bars = reinterpret_cast<uint64_t*>(red + 4);
    uint64_t* cfull = bars;
    uint64_t* cempty = cfull + kF0CStages;
    uint64_t* yfull = cempty + kF0CStages;
    uint64_t* yempty = yfull + 2;
    uint64_t* tfull = yempty + 2;
    uint64_t* tempty = tfull + 2;
    uint64_t* drain = tempty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kF0CStages; ++s) { mbar_init(cfull + s, 1); mbar_init(cempty + s, 1); }
        for (int b = 0; b < 2; ++b) {
            mbar_init(yfull + b, 32 * kF0Builders); mbar_init(yempty + b, 1);
            mbar_init(tfull + b, 1); mbar_init(tempty + b, 32 * kF0EpiWarps);
        }
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
    pdl_wait();   // the FIR's output is written by the previous kernel of the stream
    const int ub = sched[blockIdx.x], ue = sched[blockIdx.x + 1];

    if (warp == 0) {
        if (lane == 0) {   // ------------------------------------------------ producer
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int u = ub; u < ue && ok; ++u) {
                const int it = sched[gridDim.x + 1 + u];
                const F0Unit un = units[it / n_det_push];
                const F0Job& jb = jobs[un.job];
                const F0Maps* mp = maps + jb.map;
                const int t0 = un.g * tpw, t1 = min(t0 + tpw, n_tiles);
                for (int tt = t0; tt < t1 && ok; ++tt)
                    for (int tm = 0; tm < jb.tiles_m && ok; ++tm)
                        for (int kc0 = 0; kc0 < jb.K; kc0 += 32) {
                            if (!mbar_wait(cempty + stage, phase ^ 1, err, 61)) { ok = false; break; }
                            uint8_t* sb = cst + stage * C::CSTAGE;
                            mbar_expect_tx(cfull + stage, C::CSTAGE);
#pragma unroll
                            for (int pl = 0; pl < C::NPL; ++pl)
                                tma_load_4d(sb + pl * C::CPLANE, &mp->c, cfull + stage, 0, tm * 4, kc0 >> 3, pl);
                            if (++stage == kF0CStages) { stage = 0; phase ^= 1; }
                        }
            }
            for (int s = 0; s < kF0CStages; ++s) {
                if (!mbar_wait(cempty + stage, phase ^ 1, err, 62)) break;
                if (++stage == kF0CStages) { stage = 0; phase ^= 1; }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {   // ------------------------------------------------ MMA issuer
            constexpr uint32_t idesc = idesc_f16(BF16, 128, 128);
            int stage = 0, i = 0, yi = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int u = ub; u < ue && ok; ++u) {
                const int it = sched[gridDim.x + 1 + u];
                const F0Unit un = units[it / n_det_push];
                const F0Job& jb = jobs[un.job];
                const int t0 = un.g * tpw, t1 = min(t0 + tpw, n_tiles);
                const int k16 = jb.K / 16;
                for (int tt = t0; tt < t1 && ok; ++tt, ++yi) {
                    const int yb = ybufs == 2 ? (yi & 1) : 0;
                    const uint32_t ypar = ybufs == 2 ? ((yi >> 1) & 1) : (yi & 1);
                    if (!mbar_wait(yfull + yb, ypar, err, 63)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t y_hi = smem_u32(ybuf + yb * 2 * yplane), y_lo = y_hi + yplane;
                    for (int tm = 0; tm < jb.tiles_m && ok; ++tm, ++i) {
                        const int buf = i & 1;
                        if (!mbar_wait(tempty + buf, ((i >> 1) & 1) ^ 1, err, 64)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t d_re = tmem + buf * 256, d_im = d_re + 128;
                        for (int kc0 = 0; kc0 < jb.K; kc0 += 32) {
                            if (!mbar_wait(cfull + stage, phase, err, 65)) { ok = false; break; }
                            tc_fence_after();
                            const uint32_t sb = smem_u32(cst + stage * C::CSTAGE);
#pragma unroll
                            for (int j = 0; j < 2; ++j) {
                                const int kk = kc0 / 16 + j;
                                if (kk >= k16) break;
                                const uint32_t ao = j * 4096, bo = kk * 4096;
                                const uint32_t acc0 = kk > 0 ? 1u : 0u;
                                umma_f16(d_re, desc_win(sb + ao), desc_win(y_hi + bo), idesc, acc0);
                                umma_f16(d_re, desc_win(sb + ao), desc_win(y_lo + bo), idesc, 1u);
                                umma_f16(d_im, desc_win(sb + C::CPLANE + ao), desc_win(y_hi + bo), idesc, acc0);
                                umma_f16(d_im, desc_win(sb + C::CPLANE + ao), desc_win(y_lo + bo), idesc, 1u);
                                if (BF16) {
                                    umma_f16(d_re, desc_win(sb + 2 * C::CPLANE + ao), desc_win(y_hi + bo), idesc, 1u);
                                    umma_f16(d_im, desc_win(sb + 3 * C::CPLANE + ao), desc_win(y_hi + bo), idesc, 1u);
                                }
                            }
                            umma_commit(cempty + stage);
                            if (++stage == kF0CStages) { stage = 0; phase ^= 1; }
                        }
                        if (!ok) break;
                        umma_commit(tfull + buf);
                    }
                    if (!ok) break;
                    umma_commit(yempty + yb);
                }
            }
            umma_commit(drain);
            mbar_wait(drain, 0, err, 66);
        }
    } else if (warp < 2 + kF0Builders) {
        // ---------------------------------------------------------------- Yhat builders
        const int row = threadIdx.x - 64;                  // 0..127: time row of the tile
        int yi = 0;
        bool ok = true;
        for (int u = ub; u < ue && ok; ++u) {
            const int it = sched[gridDim.x + 1 + u];
            const int det = det0 + it % n_det_push;
            const F0Unit un = units[it / n_det_push];
            const F0Job jb = jobs[un.job];
            const int t0 = un.g * tpw, t1 = min(t0 + tpw, n_tiles);
            for (int tt = t0; tt < t1; ++tt, ++yi) {
                const int yb = ybufs == 2 ? (yi & 1) : 0;
                const uint32_t ypar = ybufs == 2 ? ((yi >> 1) & 1) : (yi & 1);
                const bool got = mbar_wait(yempty + yb, ypar ^ 1, err, 67);
                if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
                uint8_t* yh = ybuf + yb * 2 * yplane;
                uint8_t* yl = yh + yplane;
                const long long k = k_a + 128LL * tt + row;
                float v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = 0.f;
                int col = 0;
                auto emit = [&](float x) {
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (j == (col & 7)) v[j] = x;
                    if ((col & 7) == 7) {
                        uint32_t h[4], w[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) split_hilo2<BF16>(v[2 * j], v[2 * j + 1], h[j], w[j]);
                        const int o = (col >> 3) * 2048 + row * 16;
                        *reinterpret_cast<uint4*>(yh + o) = make_uint4(h[0], h[1], h[2], h[3]);
                        *reinterpret_cast<uint4*>(yl + o) = make_uint4(w[0], w[1], w[2], w[3]);
                    }
                    ++col;
                };
                for (int s = jb.s0; s < jb.s0 + jb.ns; ++s) {
                    const YupSlice sl = slices[s];
                    const long long e_max = (long long)sl.e_min + sl.rlen - 1;
                    const long long qa = fdiv(k - e_max + sl.D - 1, sl.D), qb = fdiv(k - sl.e_min, sl.D);
                    const int r_a = (int)(k - sl.D * qa - sl.e_min);          // R index of qa
                    const uint16_t* yhs = sl.y_hi + det * sl.y_det_stride;
                    const uint16_t* yls = sl.y_lo + det * sl.y_det_stride;
                    for (int l0 = 0; l0 < sl.L; l0 += 8) {
                        float acc[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) acc[j] = 0.f;
                        int r = r_a;
                        for (long long q = qa; q <= qb; ++q, r -= sl.D) {
                            const float wq = __ldg(sl.R + r);
                            const long long ro = (q & (sl.y_rows - 1)) * sl.y_ld + l0;
#pragma unroll
                            for (int j = 0; j < 8; ++j)
                                if (l0 + j < sl.L) acc[j] = fmaf(hilo_value<BF16>(yhs[ro + j], yls[ro + j]), wq, acc[j]);
                        }
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            if (l0 + j < sl.L) emit(acc[j]);
                    }
                }
                while (col < jb.K) emit(0.f);
                fence_proxy_async_smem();                   // generic-proxy stores -> tensor-core reads
                mbar_arrive(yfull + yb);
            }
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        // warp & 3: the TMEM lane quarter (rows); half: which 64 columns of the tile
        const int qd = warp & 3;
        const int half = (warp - 2 - kF0Builders) >> 2;
        const int rowm = qd * 32 + lane;
        int i = 0;
        for (int u = ub; u < ue; ++u) {
            const int it = sched[gridDim.x + 1 + u];
            const int det = det0 + it % n_det_push;
            const F0Unit un = units[it / n_det_push];
            const F0Job& jb = jobs[un.job];
            const int t0 = un.g * tpw, t1 = min(t0 + tpw, n_tiles);
            float gbest = -1.f;                             // bank maximum of this thread's rows (half 0)
            int gm = 0x7fffffff;
            bool fail = false;
            for (int tt = t0; tt < t1 && !fail; ++tt) {
                for (int tm = 0; tm < jb.tiles_m; ++tm, ++i) {
                    const int buf = i & 1;
                    const bool got = __all_sync(0xffffffffu, mbar_wait(tfull + buf, (i >> 1) & 1, err, 68));
                    tc_fence_after();
                    const uint32_t base = tmem + ((uint32_t)(qd * 32) << 16) + buf * 256;
                    const int m = tm * 128 + rowm;
                    float best = -1.f, bre = 0.f, bim = 0.f;
                    int bk = 0x7fffffff;
#pragma unroll 1
                    for (int c = half * 64; got && c < half * 64 + 64; c += 16) {
                        float re[16], im[16];
                        tmem_ld16(base + c, re);
                        tmem_ld16(base + 128 + c, im);
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const float p = re[j] * re[j] + im[j] * im[j];
                            if (p > best) { best = p; bk = c + j; bre = re[j]; bim = im[j]; }
                        }
                        if (STORE_Z && m < jb.M) {
                            float* zr = zout + (long long)(2 * m) * n + 128LL * tt + c;
                            float* zi = zr + n;
#pragma unroll
                            for (int j = 0; j < 16; ++j) { zr[j] = re[j]; zi[j] = im[j]; }
                        }
                    }
                    tc_fence_before();
                    mbar_arrive(tempty + buf);
                    float4* xb = xchg + buf * 128;
                    if (!STORE_Z && half == 1) xb[rowm] = make_float4(best, __int_as_float(bk), bre, bim);
                    // every epilogue thread goes on only if every one of them got its tile (a wait that
                    // ran out stops them all here, together); this also orders the exchange above
                    uint32_t all_got;
                    asm volatile(
                        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
                        "bar.red.and.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
                        : "=r"(all_got)
                        : "r"((uint32_t)got), "n"(32 * kF0EpiWarps)
                        : "memory");
                    if (!all_got) { fail = true; break; }
                    if (STORE_Z || half == 1) continue;
                    const float4 o = xb[rowm];
                    if (o.x > best) { best = o.x; bk = __float_as_int(o.y); bre = o.z; bim = o.w; }
                    const long long k0 = k_a + 128LL * tt;
                    const long long kwin0 = (k0 / window) * window;
                    const int koff = (int)(k0 - kwin0) + bk;
                    if (!aligned) {
                        if (m < jb.M) {
                            const int slot = (int)((k0 / 128) & (n_slots - 1));
                            part[(long long)(jb.tmpl0 + m) * part_tmpl_stride + (long long)det * n_slots + slot] =
                                make_float4(best, __int_as_float(koff), bre, bim);
                        }
                        continue;
                    }
                    float4 r = make_float4(best, __int_as_float(koff), bre, bim);
                    if (tt > t0) {                           // earlier tiles win ties
                        const float4 prev = rs[tm * 128 + rowm];
                        if (!(best > prev.x)) r = prev;
                    }
                    rs[tm * 128 + rowm] = r;
                    if (tt == t1 - 1 && t1 - t0 == tpw && m < jb.M) {   // the window is complete: its trigger slot
                        const long long w = kwin0 / window;
                        SlabEntry* out = slab_base + (size_t)(w % ring) * n_det_total * slab_det_stride +
                                         (size_t)det * slab_det_stride + jb.tmpl0 + m;
                        SlabEntry e;
                        e.snr = sqrtf(r.x);
                        e.phase = atan2f(r.w, r.z);
                        e.re = r.z;
                        e.im = r.w;
                        e.k_off = __float_as_int(r.y);
                        e.flags = (e.snr > threshold) ? 1 : 0;
                        e.xi2 = -1.f;
                        e.pad = 0;
                        *out = e;
                        if (r.x > gbest) { gbest = r.x; gm = m; }   // rows in increasing m: ties keep the lower
                    }
                }
            }
            if (fail) break;
            if (STORE_Z || !aligned || t1 - t0 != tpw) continue;
            // the bank's loudest template of the window (lowest index on ties), among the
            // 128 half-0 threads; its slot gets the bank-maximum flag if it triggered
            if (half == 0) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float ob = __shfl_xor_sync(0xffffffffu, gbest, o);
                    const int om = __shfl_xor_sync(0xffffffffu, gm, o);
                    if (ob > gbest || (ob == gbest && om < gm)) { gbest = ob; gm = om; }
                }
                if (lane == 0) red[qd] = make_float4(gbest, __int_as_float(gm), 0.f, 0.f);
                asm volatile("bar.sync 2, %0;" ::"n"(128) : "memory");
                float vb = red[0].x;
                int vm = __float_as_int(red[0].y);
#pragma unroll
                for (int q = 1; q < 4; ++q) {
                    const float x = red[q].x;
                    const int mm = __float_as_int(red[q].y);
                    if (x > vb || (x == vb && mm < vm)) { vb = x; vm = mm; }
                }
                if (vm < jb.M && (vm & 127) == rowm) {        // this thread wrote that template's slot
                    const long long w = (k_a + 128LL * t0) / window;
                    SlabEntry* out = slab_base + (size_t)(w % ring) * n_det_total * slab_det_stride +
                                     (size_t)det * slab_det_stride + jb.tmpl0 + vm;
                    if (out->flags & 1) out->flags |= 2;
                }
                asm volatile("bar.sync 2, %0;" ::"n"(128) : "memory");   // red[] is reused by the next unit
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

}  // namespace lloid
