// FP32 SIMT kernels of the LLOID hot path (the plain FP32 GPU path) and the
// stages every precision shares: ingest, downsampling, slice upsampling,
// window finalisation and trigger compaction.
#pragma once
#include "lloid_common.cuh"

namespace lloid {

__device__ __forceinline__ long long floordiv(long long a, long long b) {
    long long q = a / b;
    return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

// Job that owns flat tile t: the largest j with tile_base[j] <= t.
__device__ __forceinline__ int find_job(const int* __restrict__ tile_base, int n_jobs, int t) {
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(tile_base + mid) <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// a0: block -> full-rate ring
// ---------------------------------------------------------------------------
// Split paths (mode 1 FP16, 2 BF16) also write hi/lo halves to a double-mapped
// ring: sample k at k mod s_len and k mod s_len + s_len.
__global__ void k_ingest(const float* __restrict__ src, long long src_det_stride, float* __restrict__ ring,
                         long long ring_det_stride, int mask, long long k_a, int n, int det0,
                         uint16_t* __restrict__ s_hi, uint16_t* __restrict__ s_lo, long long s_det_stride,
                         int s_len, int mode) {
    pdl_launch_dependents();
    pdl_wait();
    const int det = blockIdx.y;
    const float* s = src + det * src_det_stride;
    float* r = ring + (det0 + det) * ring_det_stride;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float v = s[i];
        r[(k_a + i) & mask] = v;
        if (mode) {
            uint16_t h, l;
            split_hilo_rt(v, mode, h, l);
            const long long p = (k_a + i) & (s_len - 1);
            const long long o = (det0 + det) * s_det_stride;
            s_hi[o + p] = h; s_hi[o + p + s_len] = h;
            s_lo[o + p] = l; s_lo[o + p + s_len] = l;
        }
    }
}

// ---------------------------------------------------------------------------
// a1: d_D[q] = sum_k w'[k] d[D q + c - k], w' = sqrt(D) g / sum(g) (Eq. 4),
// for the n/D new samples q in [k_a/D - N_down, k_b/D - N_down) of every rate.
// A block of 256 threads takes QB = clamp(256 / D, 1, 128) consecutive outputs
// of one rate and one detector, so that every block does about the same number
// of multiply-adds at every rate and all blocks of a push fit on the GPU at
// once.  With m = 2c - k the sum reads d[D (q0 + i) - c + m]: the input span of
// the block is staged in shared memory split by phase,
// x_p[j] = d[D q0 - c + m0 + D j + p], so that the taps a warp reads together
// land in distinct banks; the tap weights come through L1.  Thread t takes
// output i = t mod QB and every G-th tap, G = 256 / QB, starting at t / QB;
// taps go through in chunks of kDownMC.  The G partial sums of an output are
// added by warp shuffles and then across warps, always in the same order.
// Staging loads are issued 16 per thread before any is stored, so a chunk
// costs one or two memory round trips; six blocks fit on an SM.
// ---------------------------------------------------------------------------
constexpr int kDownThreads = 256;
constexpr int kDownMC = 4096;    // taps per shared-memory chunk (a multiple of every D <= 256)
__host__ __device__ constexpr int down_qb(int D) { return D >= 256 ? 1 : (D <= 2 ? 128 : 256 / D); }
struct DownParams {
    const float* w[kMaxRates];
    float* dst[kMaxRates];
    long long dst_det_stride[kMaxRates];
    int dst_mask[kMaxRates];
    int D[kMaxRates];
    uint16_t* s_hi[kMaxRates];          // split paths: hi/lo double-mapped rings
    uint16_t* s_lo[kMaxRates];
    long long s_det_stride[kMaxRates];
    int s_len[kMaxRates];
    int blk0[kMaxRates + 1];            // first block of each rate along grid x
    int n_rates;
    int mode;                           // 0 FP32 only, 1 FP16, 2 BF16
};
// Shared memory of k_downsample: phase rows D x Jp with Jp <= QB + kDownMC / D + 1,
// so at most D QB + D + kDownMC words (D QB = 256), and one partial sum per thread.
__host__ __device__ constexpr int down_smem_bytes(int D_max) {
    return 4 * (256 + D_max + kDownMC + kDownThreads);
}

__global__ void __launch_bounds__(kDownThreads, 6) k_downsample(DownParams p, const float* __restrict__ ring0,
                                                             long long ring0_det_stride, int mask0, long long k_a,
                                                             int n, int n_down, int det0) {
    constexpr int NT = kDownThreads, U = 16;
    extern __shared__ float dsm[];
    int r = 0;
    while (r + 1 < p.n_rates && (int)blockIdx.x >= p.blk0[r + 1]) ++r;
    const int D = p.D[r], lgD = __ffs(D) - 1;
    const int QB = down_qb(D), G = NT / QB;
    const int nq = n / D;
    const int i0 = ((int)blockIdx.x - p.blk0[r]) * QB;
    const int det = det0 + blockIdx.y;
    const int c = D * n_down, taps = 2 * c + 1;
    const int Jp = (QB + kDownMC / D) | 1;           // odd pitch of a phase row
    float* xs = dsm;                                 // [D][Jp]
    float* part = dsm + D * Jp;                      // [NT]
    const int i = threadIdx.x & (QB - 1), g = threadIdx.x / QB;
    const long long q0 = k_a / D - n_down + i0;
    const float* src = ring0 + det * ring0_det_stride;
    const float* wr = p.w[r] + taps - 1;             // wr[-m] = w'[2c - m]
    pdl_wait();
    float acc = 0.f;
    for (int m0 = 0; m0 < taps; m0 += kDownMC) {
        const int L = min(kDownMC, taps - m0);
        const long long e0 = (long long)D * q0 - c + m0;
        const int nx = D * (QB - 1) + L;             // staged words: offsets D i + m - m0 of the chunk
        for (int eb = 0; eb < nx; eb += NT * U) {
            float v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = eb + u * NT + threadIdx.x;
                v[u] = e < nx ? src[(e0 + e) & mask0] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = eb + u * NT + threadIdx.x;
                if (e < nx) xs[(e & (D - 1)) * Jp + (e >> lgD)] = v[u];
            }
        }
        __syncthreads();
        const float* wc = wr - m0;
#pragma unroll 4
        for (int m = g; m < L; m += G) acc = fmaf(__ldg(wc - m), xs[(m & (D - 1)) * Jp + (m >> lgD) + i], acc);
        __syncthreads();
    }
    // The next launch (the FIR, one wave of resident CTAs) may be scheduled once every block is
    // past its multiply-adds: earlier, its CTAs would take the SMs that this grid still needs.
    pdl_launch_dependents();
    // Lanes o apart (o = QB, 2 QB, ... < 32) hold the same output.
    for (int o = QB; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    part[threadIdx.x] = acc;
    __syncthreads();
    const int S = QB > 32 ? QB : 32;                 // threads i, i + S, ... hold the remaining partials
    if ((int)threadIdx.x < QB && i0 + i < nq) {
        float v = part[i];
        for (int t = i + S; t < NT; t += S) v += part[t];
        const long long q = q0 + i;
        p.dst[r][det * p.dst_det_stride[r] + (q & p.dst_mask[r])] = v;
        if (p.mode) {
            uint16_t h, l;
            split_hilo_rt(v, p.mode, h, l);
            const long long ps = q & (p.s_len[r] - 1);
            const long long o = det * p.s_det_stride[r];
            p.s_hi[r][o + ps] = h; p.s_hi[r][o + ps + p.s_len[r]] = h;
            p.s_lo[r][o + ps] = l; p.s_lo[r][o + ps + p.s_len[r]] = l;
        }
    }
}

// ---------------------------------------------------------------------------
// a2 (FP32): Toeplitz GEMM, tile 64 bases x 128 outputs, 256 threads, each
// thread 4 bases x 8 consecutive outputs with a sliding register window on x.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_fir_f32(const FirJob* __restrict__ jobs, const int* __restrict__ tile_base,
                                                 int n_jobs, long long k_a, int det0) {
    const int t = blockIdx.x;
    const int j = find_job(tile_base, n_jobs, t);
    const FirJob& jb = jobs[j];
    const int local = t - tile_base[j];
    if (local >= jb.tiles_l * jb.tiles_q) return;
    const int tl = local / jb.tiles_q, tq = local % jb.tiles_q;
    const int det = det0 + blockIdx.y;
    const long long q_start = (jb.D == 1) ? k_a : floordiv(k_a - 1 + jb.c_hi, jb.D) + 1;
    const int l0 = tl * 64, qi0 = tq * 128;
    const long long q0 = q_start + qi0;

    __shared__ float us[64][33];
    __shared__ float xs[128 + 32];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[i][q] = 0.f;

    const float* src = jb.src + det * jb.src_det_stride;
    for (int m0 = 0; m0 < jb.N; m0 += 32) {
        for (int e = threadIdx.x; e < 64 * 32; e += 256) {
            int l = e >> 5, mm = e & 31;
            int gl = l0 + l, gm = m0 + mm;
            us[l][mm] = (gl < jb.L && gm < jb.N) ? __ldg(jb.bases + (long long)gl * jb.N + gm) : 0.f;
        }
        // xs[s] = x[q0 - m0 - 31 + s], x[i] = stream[i - src_off]
        for (int s = threadIdx.x; s < 159; s += 256) {
            long long i = q0 - m0 - 31 + s - jb.src_off;
            xs[s] = src[i & jb.src_mask];
        }
        __syncthreads();
        float xr[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) xr[q] = xs[tx * 8 + 31 + q];
#pragma unroll 8
        for (int mm = 0; mm < 32; ++mm) {
            float u0 = us[ty * 4 + 0][mm], u1 = us[ty * 4 + 1][mm];
            float u2 = us[ty * 4 + 2][mm], u3 = us[ty * 4 + 3][mm];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                acc[0][q] = fmaf(u0, xr[q], acc[0][q]);
                acc[1][q] = fmaf(u1, xr[q], acc[1][q]);
                acc[2][q] = fmaf(u2, xr[q], acc[2][q]);
                acc[3][q] = fmaf(u3, xr[q], acc[3][q]);
            }
#pragma unroll
            for (int q = 7; q > 0; --q) xr[q] = xr[q - 1];
            xr[0] = xs[(tx * 8 + 30 - mm) >= 0 ? (tx * 8 + 30 - mm) : 0];
        }
        __syncthreads();
    }
    float* dst = jb.dst + det * jb.dst_det_stride;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int l = l0 + ty * 4 + i;
        if (l >= jb.L) continue;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int qi = qi0 + tx * 8 + q;
            if (qi >= jb.q_count) continue;
            const long long qq = q_start + qi;
            dst[(long long)l * jb.dst_ld + (qq & jb.dst_mask)] = acc[i][q];
        }
    }
}

// ---------------------------------------------------------------------------
// a4 (slice part): composed polyphase upsampler of each D > 1 slice into the
// full-rate Yhat rows of the block.  OutT = float (FP32 path) or a split pair.
// ---------------------------------------------------------------------------
template <typename Store>
__global__ void __launch_bounds__(256) k_upsample(const UpJob* __restrict__ jobs, const int* __restrict__ tile_base,
                                                  int n_jobs, long long k_a, int n, int det0, Store store) {
    extern __shared__ float Rs[];
    const int t = blockIdx.x;
    const int j = find_job(tile_base, n_jobs, t);
    const UpJob& jb = jobs[j];
    const int local = t - tile_base[j];
    const int l = local / jb.tiles_k, kt = local % jb.tiles_k;
    if (l >= jb.L) return;
    for (int e = threadIdx.x; e < jb.rlen; e += blockDim.x) Rs[e] = __ldg(jb.R + e);
    __syncthreads();
    const int det = det0 + blockIdx.y;
    const int kk = kt * 256 + threadIdx.x;
    if (kk >= n) return;
    const long long K = k_a + kk;
    const float* y = jb.yring + det * jb.y_det_stride + (long long)l * jb.y_ld;
    // q with 0 <= K - D q - e_min < rlen
    const long long e_max = (long long)jb.e_min + jb.rlen - 1;
    long long q_lo = -floordiv(-(K - e_max), jb.D);   // ceil((K - e_max) / D)
    long long q_hi = floordiv(K - jb.e_min, jb.D);
    float acc = 0.f;
    for (long long q = q_lo; q <= q_hi; ++q)
        acc = fmaf(y[q & jb.y_mask], Rs[K - (long long)jb.D * q - jb.e_min], acc);
    store(jb, det, l, kk, acc);
}

struct StoreF32 {
    __device__ __forceinline__ void operator()(const UpJob& jb, int det, int l, int kk, float v) const {
        static_cast<float*>(jb.yhat)[det * jb.yhat_det_stride + (long long)l * jb.ldy + kk] = v;
    }
};

// ---------------------------------------------------------------------------
// a3 + a5 (FP32): z = C Yhat for 64 templates x 128 samples per CTA, fused
// |z|^2 and per-tile argmax (earliest sample on ties).  STORE_Z also writes
// the SNR rows (debug / parity).
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool better(float a, int ka, float b, int kb) {
    return a > b || (a == b && ka < kb);
}

template <bool STORE_Z>
__global__ void __launch_bounds__(256) k_recon_f32(const ReconJob* __restrict__ jobs, const int* __restrict__ tile_base,
                                                   int n_jobs, long long k_a, int n, int det0, long long window,
                                                   Partial* __restrict__ part, long long part_tmpl_stride,
                                                   int n_slots, TailRing tail, float* __restrict__ zout) {
    const int t = blockIdx.x;
    const int j = find_job(tile_base, n_jobs, t);
    const ReconJob& jb = jobs[j];
    const int local = t - tile_base[j];
    const int tm = local / jb.tiles_t, tt = local % jb.tiles_t;
    const int det = det0 + blockIdx.y;
    const int m0 = tm * 64, t0 = tt * 128;
    if (t0 >= n) return;
    const float* cre = (const float*)jb.c_re;
    const float* cim = (const float*)jb.c_im;
    const float* yh = (const float*)jb.yhat + det * jb.yhat_det_stride;

    __shared__ __align__(16) float sre[16][64];
    __shared__ __align__(16) float sim[16][64];
    __shared__ __align__(16) float sy[16][128];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float are[8][4], aim[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) { are[i][q] = 0.f; aim[i][q] = 0.f; }

    for (int k0 = 0; k0 < jb.Kpad; k0 += 16) {
        for (int e = threadIdx.x; e < 64 * 16; e += 256) {
            int m = e >> 4, kk = e & 15;
            long long off = (long long)(m0 + m) * jb.Kpad + k0 + kk;
            sre[kk][m] = __ldg(cre + off);
            sim[kk][m] = __ldg(cim + off);
        }
        for (int e = threadIdx.x; e < 16 * 32; e += 256) {
            int kk = e >> 5, c4 = e & 31;
            float4 v = __ldg(reinterpret_cast<const float4*>(yh + (long long)(k0 + kk) * jb.ldy + t0) + c4);
            reinterpret_cast<float4*>(&sy[kk][0])[c4] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < 16; ++kk) {
            float4 r0 = reinterpret_cast<const float4*>(&sre[kk][w * 8])[0];
            float4 r1 = reinterpret_cast<const float4*>(&sre[kk][w * 8])[1];
            float4 i0 = reinterpret_cast<const float4*>(&sim[kk][w * 8])[0];
            float4 i1 = reinterpret_cast<const float4*>(&sim[kk][w * 8])[1];
            float4 y4 = reinterpret_cast<const float4*>(&sy[kk][lane * 4])[0];
            float cr[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
            float ci[8] = {i0.x, i0.y, i0.z, i0.w, i1.x, i1.y, i1.z, i1.w};
            float yv[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    are[i][q] = fmaf(cr[i], yv[q], are[i][q]);
                    aim[i][q] = fmaf(ci[i], yv[q], aim[i][q]);
                }
        }
        __syncthreads();
    }

    // Epilogue: window maxima.  Tile [t0, t0+128) lies inside one window.
    const long long tile_abs = (k_a + t0) / kTileT;
    const long long kwin0 = ((k_a + t0) / window) * window;
    const int slot = (int)(tile_abs & (n_slots - 1));
    // window overlap: a tile that ends where a window starts also keeps its last ov samples
    const long long w1 = (k_a + t0 + 128) / window;
    const bool pre = tail.ov > 0 && (k_a + t0 + 128) % window == 0;
    const int tail_from = pre ? 128 - tail.ov : 128;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int m = m0 + w * 8 + i;
        float best = -1.f, bre = 0.f, bim = 0.f, tbest = -1.f, tre = 0.f, tim = 0.f;
        int bk = 0x7fffffff, tk = 0x7fffffff;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float p = are[i][q] * are[i][q] + aim[i][q] * aim[i][q];
            int k = (int)(k_a + t0 + lane * 4 + q - kwin0);
            if (better(p, k, best, bk)) { best = p; bk = k; bre = are[i][q]; bim = aim[i][q]; }
            const int kt = (int)(k_a + t0 + lane * 4 + q - w1 * window);
            if (lane * 4 + q >= tail_from && better(p, kt, tbest, tk)) { tbest = p; tk = kt; tre = are[i][q]; tim = aim[i][q]; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float ob = __shfl_xor_sync(0xffffffffu, best, o);
            int ok = __shfl_xor_sync(0xffffffffu, bk, o);
            float ore = __shfl_xor_sync(0xffffffffu, bre, o);
            float oim = __shfl_xor_sync(0xffffffffu, bim, o);
            if (better(ob, ok, best, bk)) { best = ob; bk = ok; bre = ore; bim = oim; }
            if (pre) {
                ob = __shfl_xor_sync(0xffffffffu, tbest, o);
                ok = __shfl_xor_sync(0xffffffffu, tk, o);
                ore = __shfl_xor_sync(0xffffffffu, tre, o);
                oim = __shfl_xor_sync(0xffffffffu, tim, o);
                if (better(ob, ok, tbest, tk)) { tbest = ob; tk = ok; tre = ore; tim = oim; }
            }
        }
        if (m < jb.M) {
            if (lane == 0 && part != nullptr) {
                part[(long long)(jb.tmpl0 + m) * part_tmpl_stride + (long long)det * n_slots + slot] =
                    make_float4(best, __int_as_float(bk), bre, bim);
                if (pre)
                    tail.p[(long long)(jb.tmpl0 + m) * tail.tmpl_stride + (long long)det * tail.n + (w1 & (tail.n - 1))] =
                        make_float4(tbest, __int_as_float(tk), tre, tim);
            }
            if (STORE_Z) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    zout[(long long)(2 * m) * n + t0 + lane * 4 + q] = are[i][q];
                    zout[(long long)(2 * m + 1) * n + t0 + lane * 4 + q] = aim[i][q];
                }
            }
            if (jb.zring != nullptr) {   // Eq. 10 history: 4 samples of z as half2, one 16-byte store
                uint32_t h[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const __half2 v = __floats2half2_rn(are[i][q], aim[i][q]);
                    h[q] = *reinterpret_cast<const uint32_t*>(&v);
                }
                const long long pos = (k_a + t0 + lane * 4) & (jb.zring_len - 1);
                *reinterpret_cast<uint4*>(jb.zring + det * jb.zring_det_stride + (long long)m * jb.zring_len + pos) =
                    make_uint4(h[0], h[1], h[2], h[3]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// a5: finalise window w for one (bank, detector): reduce the tile partials of
// every template, threshold, and flag the bank's loudest template.
// ---------------------------------------------------------------------------
// grid (chunk, detector, window): a chunk is kFinTB templates of one bank; a
// half-warp reduces one template's tile partials (16 lanes read them side by
// side).  Windows w0 .. w0 + gridDim.z - 1; window w's slab is
// slab_base + (w mod ring) * n_det_total * slab_det_stride.  The bank's loudest
// template (largest max |z|^2, lowest index on ties) is found across chunks by
// an atomic max on an order-preserving 64-bit key; the last chunk block to
// finish flags it and clears the key and the counter for the next push.
constexpr int kFinTB = 64;          // templates per k_finalize block
constexpr int kCoincTB = 256;       // templates per k_coinc block
struct FinChunk { int job, m0; };

// Key whose unsigned order is (x ascending, m descending): float bits mapped to
// an unsigned total order in the high word, ~m in the low word.
__device__ __forceinline__ unsigned long long max_key(float x, int m) {
    uint32_t u = __float_as_uint(x);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((unsigned long long)u << 32) | (uint32_t)(0xffffffffu - (uint32_t)m);
}
__device__ __forceinline__ int max_key_index(unsigned long long k) {
    return (int)(0xffffffffu - (uint32_t)(k & 0xffffffffu));
}

// Block-wide argmax of (v, idx) (largest v, lowest idx on ties) in thread 0.
__device__ __forceinline__ void block_argmax(float& v, int& idx) {
    __shared__ float sb[32];
    __shared__ int si[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ob > v || (ob == v && oi < idx)) { v = ob; idx = oi; }
    }
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sb[wid] = v; si[wid] = idx; }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i)
            if (sb[i] > v || (sb[i] == v && si[i] < idx)) { v = sb[i]; idx = si[i]; }
}

__global__ void __launch_bounds__(256) k_finalize(const FinJob* __restrict__ jobs, const FinChunk* __restrict__ chunks,
                                                  const Partial* __restrict__ part, long long part_tmpl_stride,
                                                  int n_slots, int tiles_per_window, long long w0, float threshold,
                                                  SlabEntry* __restrict__ slab_base, int ring, int n_det_total,
                                                  long long slab_det_stride, int det0,
                                                  unsigned long long* __restrict__ red, long long fused_from,
                                                  TailRing tail) {
    constexpr int P = kFinTB / 16;
    pdl_launch_dependents();
    pdl_wait();
    const FinChunk ch = chunks[blockIdx.x];
    const FinJob jb = jobs[ch.job];
    const int det = det0 + blockIdx.y;
    const long long w = w0 + blockIdx.z;
    if (jb.fused && w >= fused_from) return;   // the f0 kernel wrote this window (every chunk returns)
    SlabEntry* out = slab_base + (size_t)(w % ring) * n_det_total * slab_det_stride + det * slab_det_stride;
    const int s0 = (int)((w * tiles_per_window) & (n_slots - 1));
    const int hw = threadIdx.x >> 4, l16 = threadIdx.x & 15;
    const Partial none = make_float4(-1.f, __int_as_float(0x7fffffff), 0.f, 0.f);
    Partial v[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {            // every first-round load in flight at once
        const int m = ch.m0 + 16 * p + hw;
        v[p] = (m < jb.M && l16 < tiles_per_window)
                   ? part[(long long)(jb.tmpl0 + m) * part_tmpl_stride + (long long)det * n_slots +
                          ((s0 + l16) & (n_slots - 1))]
                   : none;
    }
    float tbest = -1.f;
    int tidx = 0x7fffffff;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int m = ch.m0 + 16 * p + hw;
        float best = v[p].x, bre = v[p].z, bim = v[p].w;
        int bk = __float_as_int(v[p].y);
        if (m < jb.M) {
            const Partial* pt = part + (long long)(jb.tmpl0 + m) * part_tmpl_stride + (long long)det * n_slots;
            for (int s = l16 + 16; s < tiles_per_window; s += 16) {
                const float4 u = pt[(s0 + s) & (n_slots - 1)];
                const int k = __float_as_int(u.y);
                if (better(u.x, k, best, bk)) { best = u.x; bk = k; bre = u.z; bim = u.w; }
            }
            if (l16 == 0 && tail.ov > 0 && w > 0) {   // the overlap: samples before the window's start
                const float4 u = tail.p[(long long)(jb.tmpl0 + m) * tail.tmpl_stride + (long long)det * tail.n +
                                        (w & (tail.n - 1))];
                const int k = __float_as_int(u.y);
                if (better(u.x, k, best, bk)) { best = u.x; bk = k; bre = u.z; bim = u.w; }
            }
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {   // within the half-warp
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int ok = __shfl_xor_sync(0xffffffffu, bk, o);
            const float ore = __shfl_xor_sync(0xffffffffu, bre, o), oim = __shfl_xor_sync(0xffffffffu, bim, o);
            if (better(ob, ok, best, bk)) { best = ob; bk = ok; bre = ore; bim = oim; }
        }
        if (m < jb.M) {
            if (l16 == 0) {
                SlabEntry e;
                e.snr = sqrtf(best);
                e.phase = atan2f(bim, bre);
                e.re = bre;
                e.im = bim;
                e.k_off = bk;
                e.flags = (e.snr > threshold) ? 1 : 0;
                e.xi2 = -1.f;
                e.pad = 0;
                out[jb.tmpl0 + m] = e;
            }
            if (best > tbest || (best == tbest && m < tidx)) { tbest = best; tidx = m; }
        }
    }
    __threadfence();                          // slab entries visible before this block counts itself done
    block_argmax(tbest, tidx);
    if (threadIdx.x == 0) {
        const size_t slot = ((size_t)ch.job * n_det_total + det) * ring + (size_t)(w % ring);
        unsigned long long* key = red + 2 * slot;
        unsigned long long* cnt = key + 1;
        if (tidx < jb.M) atomicMax(key, max_key(tbest, tidx));
        __threadfence();
        const unsigned long long n_chunks = (unsigned long long)((jb.M + kFinTB - 1) / kFinTB);
        if (atomicAdd(cnt, 1ull) == n_chunks - 1) {   // last chunk of this (bank, detector, window)
            __threadfence();
            const unsigned long long k = atomicExch(key, 0ull);
            atomicExch(cnt, 0ull);
            const int m = max_key_index(k);
            if (k != 0ull && m >= 0 && m < jb.M) {
                int* f = &out[jb.tmpl0 + m].flags;
                if (atomicAdd(f, 0) & 1) atomicOr(f, 2);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Trigger compaction of one window slab: entries e = det * cap + tmpl, in
// order; chunk counts, then each chunk scatters at its exclusive prefix.
// ---------------------------------------------------------------------------
struct TriggerOut {       // identical layout to lloid_trigger
    int32_t detector, bank, tmpl, is_bank_max;
    long long window, sample;
    float snr, phase, re, im;
    float xi2;
    int32_t pad;
};

// Entries e = (wl * n_det + det) * M_used + m for windows w0 .. w0 + n_win - 1.
__device__ __forceinline__ const SlabEntry& slab_at(const SlabEntry* slab, long long cap, int M_used, int n_det,
                                                    long long w0, int ring, long long e, long long* w_out,
                                                    long long* det_out, long long* m_out) {
    const long long m = e % M_used, r = e / M_used;
    const long long det = r % n_det, wl = r / n_det;
    *w_out = w0 + wl; *det_out = det; *m_out = m;
    return slab[((w0 + wl) % ring) * n_det * cap + det * cap + m];
}

__global__ void k_gather_count(const SlabEntry* __restrict__ slab, long long cap, int M_used, int n_det,
                               long long w0, int n_win, int ring, int* __restrict__ counts) {
    pdl_launch_dependents();
    pdl_wait();
    const long long total = (long long)n_win * n_det * M_used;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int v = 0;
    if (e < total) {
        long long w, det, m;
        v = slab_at(slab, cap, M_used, n_det, w0, ring, e, &w, &det, &m).flags & 1;
    }
    v = __syncthreads_count(v);
    if (threadIdx.x == 0) counts[blockIdx.x] = v;
}

__global__ void k_gather_scatter(const SlabEntry* __restrict__ slab, long long cap, int M_used, int n_det,
                                 long long w0, int n_win, int ring, const int* __restrict__ counts, int n_chunks,
                                 const int* __restrict__ bank_of, const int* __restrict__ tmpl0_of, long long W,
                                 TriggerOut* __restrict__ out, long long out_cap, long long* __restrict__ total_out) {
    pdl_launch_dependents();
    pdl_wait();
    __shared__ int red[1024 / 32];
    __shared__ int base_s;
    // exclusive prefix of the chunk counts
    int s = 0;
    for (int i = threadIdx.x; i < blockIdx.x; i += blockDim.x) s += counts[i];
    int tot = 0;
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < n_chunks; i += blockDim.x) tot += counts[i];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) { s += __shfl_xor_sync(0xffffffffu, s, o); tot += __shfl_xor_sync(0xffffffffu, tot, o); }
    __shared__ int red2[1024 / 32];
    if (lane == 0) { red[wid] = s; red2[wid] = tot; }
    __syncthreads();
    if (threadIdx.x == 0) {
        int a = 0, b = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { a += red[i]; b += red2[i]; }
        base_s = a;
        if (blockIdx.x == 0) *total_out = b;
    }
    __syncthreads();
    const long long total = (long long)n_win * n_det * M_used;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    SlabEntry en;
    int v = 0;
    long long det = 0, m = 0, window = 0;
    if (e < total) {
        en = slab_at(slab, cap, M_used, n_det, w0, ring, e, &window, &det, &m);
        v = en.flags & 1;
    }
    // block-wide exclusive scan of v
    unsigned ball = __ballot_sync(0xffffffffu, v);
    int pre = __popc(ball & ((1u << lane) - 1));
    __syncthreads();
    if (lane == 0) red[wid] = __popc(ball);
    __syncthreads();
    int wpre = 0;
    for (int i = 0; i < wid; ++i) wpre += red[i];
    if (v) {
        long long pos = (long long)base_s + wpre + pre;
        if (pos < out_cap) {
            TriggerOut o;
            o.detector = (int)det;
            o.bank = bank_of[m];
            o.tmpl = (int)(m - tmpl0_of[o.bank]);
            o.is_bank_max = (en.flags >> 1) & 1;
            o.window = window;
            o.sample = window * W + en.k_off;
            o.snr = en.snr; o.phase = en.phase; o.re = en.re; o.im = en.im;
            o.xi2 = en.xi2;
            o.pad = 0;
            out[pos] = o;
        }
    }
}

// ---------------------------------------------------------------------------
// Eq. 10 for the triggers of windows w0 .. w0 + gridDim.z - 1 of one detector:
// one warp per (template, window); the lanes stride t = -d .. d.
// xi2 = sum_t |z[k* + t] - z[k*] R(t)|^2 / sum_t (2 - 2 |R(t)|^2), with z from
// the bank's half2 ring (samples before the stream start read as 0).
// grid (tiles of 8 templates over all jobs, 1, windows), 256 threads.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_xi2(const Xi2Job* __restrict__ jobs, const int* __restrict__ tile_base,
                                             int n_jobs, long long w0, long long W, int det,
                                             SlabEntry* __restrict__ slab_base, int ring, int n_det_total,
                                             long long slab_det_stride) {
    pdl_launch_dependents();
    pdl_wait();
    const int t = blockIdx.x;
    const int jx = find_job(tile_base, n_jobs, t);
    const Xi2Job& jb = jobs[jx];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = (t - tile_base[jx]) * 8 + warp;
    if (m >= jb.M) return;
    const long long w = w0 + blockIdx.z;
    SlabEntry* e = slab_base + (size_t)(w % ring) * n_det_total * slab_det_stride + det * slab_det_stride +
                   jb.tmpl0 + m;
    if ((e->flags & 1) == 0) return;
    const long long k = w * W + e->k_off;
    const float zr0 = e->re, zi0 = e->im;
    const uint32_t* zr = jb.zring + det * jb.zdet_stride + (long long)m * jb.zlen;
    const float2* R = jb.ac + (long long)m * (2 * jb.half + 1);
    float acc = 0.f;
    for (int tt = lane; tt <= 2 * jb.half; tt += 32) {
        const long long s = k + tt - jb.half;
        float zx = 0.f, zy = 0.f;
        if (s >= 0) {
            const uint32_t u = zr[s & (jb.zlen - 1)];
            const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&u));
            zx = f.x;
            zy = f.y;
        }
        const float2 r = R[tt];
        const float ex = zx - (zr0 * r.x - zi0 * r.y);
        const float ey = zy - (zr0 * r.y + zi0 * r.x);
        acc = fmaf(ex, ex, fmaf(ey, ey, acc));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) e->xi2 = acc / jb.den[m];
}

// ---------------------------------------------------------------------------
// Coincidence and clustering (Sections II.D.3-4) for windows w0 .. w0 +
// gridDim.y - 1: grid (chunk of kCoincTB templates of one bank, window), a
// thread per template.  For a template, the loudest detector's trigger (lowest
// detector on ties) is the reference; triggers of the other detectors within
// `delta` samples join; two or more detectors make an event of network SNR
// sqrt(sum snr^2).  The bank keeps its event of largest network SNR (lowest
// template on ties): an atomic max on an order-preserving key across chunks;
// the last chunk block to finish rebuilds that template's event, stores it and
// clears the key and the counter for the next push.
// ---------------------------------------------------------------------------
struct CoincHit { float net; int n, ref, k0; uint32_t mask; };
__device__ __forceinline__ CoincHit coinc_of(const SlabEntry* __restrict__ slab, long long slab_det_stride, int t,
                                             int n_det, int delta) {
    CoincHit h{-1.f, 0, -1, 0, 0u};
    float rs = 0.f;
    for (int d = 0; d < n_det; ++d) {
        const SlabEntry& e = slab[d * slab_det_stride + t];
        if ((e.flags & 1) && (h.ref < 0 || e.snr > rs)) { h.ref = d; rs = e.snr; }
    }
    if (h.ref < 0) return h;
    h.k0 = slab[h.ref * slab_det_stride + t].k_off;
    float s2 = 0.f;
    for (int d = 0; d < n_det; ++d) {
        const SlabEntry& e = slab[d * slab_det_stride + t];
        if ((e.flags & 1) && abs(e.k_off - h.k0) <= delta) {
            s2 = fmaf(e.snr, e.snr, s2);
            ++h.n;
            h.mask |= 1u << d;
        }
    }
    if (h.n >= 2) h.net = sqrtf(s2);
    return h;
}

__global__ void __launch_bounds__(256) k_coinc(const FinJob* __restrict__ jobs, const FinChunk* __restrict__ chunks,
                                               long long w0, int n_det, int delta,
                                               const SlabEntry* __restrict__ slab_base, int ring,
                                               long long slab_det_stride, EventEntry* __restrict__ ev_base, int ev_cap,
                                               unsigned long long* __restrict__ red) {
    pdl_launch_dependents();
    pdl_wait();
    const FinChunk ch = chunks[blockIdx.x];
    const FinJob jb = jobs[ch.job];
    const long long w = w0 + blockIdx.y;
    const SlabEntry* slab = slab_base + (size_t)(w % ring) * n_det * slab_det_stride;
    float best = -1.f;
    int bm = 0x7fffffff;
    const int m = ch.m0 + (int)threadIdx.x;
    if (m < jb.M) {
        const CoincHit h = coinc_of(slab, slab_det_stride, jb.tmpl0 + m, n_det, delta);
        if (h.n >= 2) { best = h.net; bm = m; }
    }
    block_argmax(best, bm);
    if (threadIdx.x == 0) {
        const size_t slot = (size_t)ch.job * ring + (size_t)(w % ring);
        unsigned long long* key = red + 2 * slot;
        unsigned long long* cnt = key + 1;
        if (bm < jb.M) atomicMax(key, max_key(best, bm));
        __threadfence();
        const unsigned long long n_chunks = (unsigned long long)((jb.M + kCoincTB - 1) / kCoincTB);
        if (atomicAdd(cnt, 1ull) == n_chunks - 1) {
            __threadfence();
            const unsigned long long k = atomicExch(key, 0ull);
            atomicExch(cnt, 0ull);
            EventEntry ev;
            ev.net_snr = -1.f; ev.tmpl = 0x7fffffff; ev.n_ifo = 0; ev.ifo_mask = 0; ev.ref_det = 0; ev.ref_k_off = 0;
            ev.pad[0] = ev.pad[1] = 0;
            const int bt = max_key_index(k);
            if (k != 0ull && bt >= 0 && bt < jb.M) {
                const CoincHit h = coinc_of(slab, slab_det_stride, jb.tmpl0 + bt, n_det, delta);
                ev.net_snr = h.net; ev.tmpl = bt; ev.n_ifo = h.n; ev.ifo_mask = h.mask; ev.ref_det = h.ref;
                ev.ref_k_off = h.k0;
            }
            ev_base[(size_t)(w % ring) * ev_cap + jb.bank] = ev;
        }
    }
}

// ---------------------------------------------------------------------------
// Background collection (Section II.D.5) for windows w0 .. w0 + gridDim.y - 1:
// a thread per template (grid.z covers the largest bank); every trigger that
// is not a member of its template's coincidence (same rule as k_coinc) adds 1
// to bin (snr, xi2) of its bank and detector.  Bins: the number of inner
// edges <= the value (float comparisons, as the host wrote the edges).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int edge_bin(float x, const float* __restrict__ e, int n) {
    int b = 0;
    for (int i = 1; i < n; ++i) b += (e[i] <= x) ? 1 : 0;
    return b;
}

__global__ void __launch_bounds__(256) k_background(const FinJob* __restrict__ jobs, long long w0, int n_det,
                                                    int delta, const SlabEntry* __restrict__ slab_base, int ring,
                                                    long long slab_det_stride, const float* __restrict__ snr_e,
                                                    int n_snr, const float* __restrict__ xi2_e, int n_xi2) {
    pdl_launch_dependents();
    pdl_wait();
    const FinJob jb = jobs[blockIdx.x];
    const int m = blockIdx.z * blockDim.x + threadIdx.x;
    if (jb.bg == nullptr || m >= jb.M) return;
    const long long w = w0 + blockIdx.y;
    const SlabEntry* slab = slab_base + (size_t)(w % ring) * n_det * slab_det_stride + jb.tmpl0 + m;
    int ref = -1;
    float rs = 0.f;
    for (int d = 0; d < n_det; ++d) {
        const SlabEntry& e = slab[d * slab_det_stride];
        if ((e.flags & 1) && (ref < 0 || e.snr > rs)) { ref = d; rs = e.snr; }
    }
    if (ref < 0) return;
    const int k0 = slab[ref * slab_det_stride].k_off;
    uint32_t mask = 0;
    int n = 0;
    for (int d = 0; d < n_det; ++d) {
        const SlabEntry& e = slab[d * slab_det_stride];
        if ((e.flags & 1) && abs(e.k_off - k0) <= delta) { mask |= 1u << d; ++n; }
    }
    if (n < 2) mask = 0;
    for (int d = 0; d < n_det; ++d) {
        const SlabEntry& e = slab[d * slab_det_stride];
        if (!(e.flags & 1) || (mask >> d & 1u)) continue;
        const int bs = edge_bin(e.snr, snr_e, n_snr), bx = edge_bin(e.xi2, xi2_e, n_xi2);
        atomicAdd(jb.bg + ((size_t)d * n_snr + bs) * n_xi2 + bx, 1u);
    }
}

}  // namespace lloid
