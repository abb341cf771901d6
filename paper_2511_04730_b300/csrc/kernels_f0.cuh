// The f0 form of a bank: slice upsampling (Eq. 7-8), then reconstruction
// (Eq. 6) and the trigger window maxima (Section II.D.1) on the tensor cores.
//
// Eq. 6 and Eq. 7-8 are linear and the coefficients do not depend on time, so
// the bank's SNR is z = C Yhat with Yhat_l[k] = sum_q Y_l[q] R[k - D q - e_min]:
// every slice's basis outputs brought up to f0 through the slice's ladder of
// Eq. 7-8 upsamplers composed into one polyphase filter R (R = [1] at f0).
// The columns of Yhat are the bank's bases packed slice after slice, so K is
// the bank's basis count rounded up to 16.
//
// k_yhat: a CTA per (bank, detector, group of tpw consecutive 128-sample tiles
// of the push, tpw = window / 128) forms Yhat tile by tile in FP32 from the
// FIR's hi/lo output at each slice's rate (staged in shared memory with the
// slice's composed taps; a thread per time row and half of the slice pieces),
// splits it into hi/lo halves and writes them to HBM as time-blocked planes
// [det][hi, lo][K/8][rows][8]: a tile is then one TMA box per plane that lands
// in the no-swizzle K-major operand layout ([K/8][128 rows][8]).  Several of
// these CTAs share an SM, which the upsampling's dependent loads need.
//
// k_f0_top: per work unit of the same shape, per tile of the group:
//   producer (1 thread): the tile's Yhat planes (one box each) and the
//     coefficient tiles of the bank's 128-template groups, 32 bases per TMA
//     stage, from time-blocked planes [re hi, im hi, (re lo, im lo)][K/8][Mpad][8];
//   MMA issuer (1 thread): for every template group, C Yhat into a TMEM
//     accumulator (re and im, 128 columns each, two buffers), hi/lo products
//     (FP16: C_hi Y_hi + C_hi Y_lo; BF16: + C_lo Y_hi);
//   epilogue warps (2 x 4): |z|^2 and its argmax over the tile (earliest sample
//     on ties), kept per template across the group of tiles; one group of four
//     warps per TMEM buffer, the buffer being the template group's parity.
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
    int map;                       // index into the maps
    int pc0, np;                   // the bank's pieces in the piece table (F0Piece)
    int bt0, nbat;                 // and the ends of its staging batches
    uint16_t* yh;                  // Yhat planes [det][hi, lo][K/8][yrows][8] of the current push
    int yrows;                     // rows (samples) of a plane: the largest push
    int pad;
};
struct F0Maps {
    CUtensorMap c;                 // [planes][K/8][Mpad][8], box 128 rows x 32 bases of one plane
    CUtensorMap y;                 // [det * 2 + plane][K/8][yrows][8], box 128 rows x K bases of one plane
};
struct F0Unit { int job, g; };     // group g: tiles [g tpw, min((g + 1) tpw, n / 128)) of the push

constexpr int kF0MaxTm = 8;        // template groups per bank (M <= 1024)
constexpr int kF0EpiWarps = 8;     // epilogue warps 2..9
constexpr int kF0Threads = 32 * (2 + kF0EpiWarps);
constexpr int kF0MaxCStages = 4;
constexpr int kYhThreads = 128;    // k_yhat: a thread per time row
constexpr int kYhRing = 4;         // k_yhat: 8-column groups of a row held until complete (pieces <= 16 bases)
constexpr int kF0Kc = 96;          // largest K of a bank in the f0 form (two Yhat buffers of this width)
constexpr int kF0StageRows = 132;  // rows of Y one slice reaches per tile: (127 + rlen - 1) / D + 2 at most
constexpr int kF0StageFloats = 4096;   // builders' staging of Y rows for one batch of slice pieces (16 KB)
constexpr int kF0RAll = 4096;      // every slice's composed upsampler, staged once per work unit (16 KB)
constexpr int kF0MaxSlices = 16;
constexpr int kF0MaxPieces = 64;   // (slice, column chunk) pieces of a bank: at most 16 + 128 / 8

// k_yhat's tables in shared memory: the unit's slices, and the pieces of slices (up to 32
// columns each) in column order, grouped in batches that fit the staging.  A push starts on a
// multiple of 128 samples and every D divides 128, so a slice reaches the same number of Y rows
// from every tile: the pieces and batches are fixed per bank (built with the job tables).
struct F0SliceS {
    const uint16_t* y_hi;          // the slice's FIR output ring, detector applied
    const uint16_t* y_lo;
    int y_rows, y_ld, D, e_min, rlen, L, roff, nq;
    int qoff;                      // first staged row of a tile: tile start / D + qoff
    int col0;                      // first column of the slice in Yhat
};
struct F0Piece { int s, c0, nc, nv, off, pitch, items, item0; };   // nv: 4-column chunks (0: a slice at f0, read directly)

template <bool BF16>
struct F0Cfg {
    static constexpr int NPL = BF16 ? 4 : 2;               // coefficient planes
    static constexpr int CPLANE = 128 * 32 * 2;            // one plane of a 32-basis stage (8 KB)
    static constexpr int CSTAGE = NPL * CPLANE;
    static constexpr int CSTAGES = BF16 ? 3 : 4;           // coefficient stages (what shared memory allows)
};
// Shared memory of k_f0_top: K <= kc with ybufs Yhat buffers.
__host__ __device__ constexpr int f0_smem_bytes(bool bf16, int kc, int ybufs) {
    return (bf16 ? 3 : 4) * (bf16 ? 4 : 2) * 8192 + ybufs * 2 * 128 * kc * 2 + kF0MaxTm * 128 * 16 +
           kF0EpiWarps * 16 + 1024 + 512;
}
// Shared memory of k_yhat: staging, composed upsamplers (rall floats, a multiple of 4), tables
// and the rows' group rings of two tiles.
__host__ __device__ constexpr int yhat_smem_bytes(int rall) {
    return (kF0StageFloats + rall) * 4 + kF0MaxSlices * (int)sizeof(F0SliceS) + kF0MaxPieces * (int)sizeof(F0Piece) +
           (kF0MaxPieces + 4) * 4 + 4 * kYhRing * 128 * 16 + 1024;
}

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Two packed hi/lo 16-bit pairs (element 0 in the low half) back to FP32 sums.
template <bool BF16>
__device__ __forceinline__ float2 hilo_pair(uint32_t h, uint32_t l) {
    if (BF16)
        return make_float2(__uint_as_float(h << 16) + __uint_as_float(l << 16),
                           __uint_as_float(h & 0xffff0000u) + __uint_as_float(l & 0xffff0000u));
    return make_float2(__half2float(__ushort_as_half((unsigned short)(h & 0xffffu))) +
                           __half2float(__ushort_as_half((unsigned short)(l & 0xffffu))),
                       __half2float(__ushort_as_half((unsigned short)(h >> 16))) +
                           __half2float(__ushort_as_half((unsigned short)(l >> 16))));
}

// One Yhat element split into its hi and lo halves, stored at byte offset o of the two planes.
template <bool BF16>
__device__ __forceinline__ void put_hilo(uint8_t* yh, uint8_t* yl, int o, float x) {
    if (BF16) {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        *reinterpret_cast<__nv_bfloat16*>(yh + o) = h;
        *reinterpret_cast<__nv_bfloat16*>(yl + o) = __float2bfloat16_rn(x - __bfloat162float(h));
    } else {
        const __half h = __float2half_rn(x);
        *reinterpret_cast<__half*>(yh + o) = h;
        *reinterpret_cast<__half*>(yl + o) = __float2half_rn(x - __half2float(h));
    }
}

// |z|^2 of two samples with the packed FP32 pipe: re^2 rounded, then + im^2 fused.
__device__ __forceinline__ void zsq2(uint32_t re0, uint32_t re1, uint32_t im0, uint32_t im1, float& p0, float& p1) {
    asm("{\n\t.reg .b64 r, i, p;\n\t"
        "mov.b64 r, {%2, %3};\n\tmov.b64 i, {%4, %5};\n\t"
        "mul.rn.f32x2 p, r, r;\n\tfma.rn.f32x2 p, i, i, p;\n\t"
        "mov.b64 {%0, %1}, p;\n\t}"
        : "=f"(p0), "=f"(p1)
        : "r"(re0), "r"(re1), "r"(im0), "r"(im1));
}
// The same, as a volatile statement: recomputed where needed instead of kept live in registers.
__device__ __forceinline__ void zsq2_again(uint32_t re0, uint32_t re1, uint32_t im0, uint32_t im1, float& p0, float& p1) {
    asm volatile("{\n\t.reg .b64 r, i, p;\n\t"
                 "mov.b64 r, {%2, %3};\n\tmov.b64 i, {%4, %5};\n\t"
                 "mul.rn.f32x2 p, r, r;\n\tfma.rn.f32x2 p, i, i, p;\n\t"
                 "mov.b64 {%0, %1}, p;\n\t}"
                 : "=f"(p0), "=f"(p1)
                 : "r"(re0), "r"(re1), "r"(im0), "r"(im1));
}
__device__ __forceinline__ float fmax3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
// Eq. 7-8 composed into one polyphase filter, for one time row of two consecutive tiles
// and NV chunks of 4 columns of a slice piece: acc0[4c + j] = sum_q R[r0 - D q] Y[q][4c + j]
// over the staged rows q in [qa, qb] (rr = R + r0, yp = the piece's staged rows), and acc1
// the same for the row 128 samples later, whose rows are sh = 128 / D further on with the
// same taps (D divides 128).  A tap is loaded once for both rows and all chunks.
template <int NV>
__device__ __forceinline__ void f0_taps2(const float* yp, int pitch, const float* rr, int D, int qa, int qb, int sh,
                                         float (&acc0)[4 * NV], float (&acc1)[4 * NV]) {
#pragma unroll
    for (int j = 0; j < 4 * NV; ++j) { acc0[j] = 0.f; acc1[j] = 0.f; }
    const int psh = sh * pitch;
#pragma unroll 2
    for (int qi = qa; qi <= qb; ++qi) {
        const float wq = rr[-D * qi];
        const float* y = yp + qi * pitch;
#pragma unroll
        for (int c = 0; c < NV; ++c) {
            const float4 a = *reinterpret_cast<const float4*>(y + 4 * c);
            const float4 a1 = *reinterpret_cast<const float4*>(y + psh + 4 * c);
            acc0[4 * c + 0] = fmaf(a.x, wq, acc0[4 * c + 0]); acc0[4 * c + 1] = fmaf(a.y, wq, acc0[4 * c + 1]);
            acc0[4 * c + 2] = fmaf(a.z, wq, acc0[4 * c + 2]); acc0[4 * c + 3] = fmaf(a.w, wq, acc0[4 * c + 3]);
            acc1[4 * c + 0] = fmaf(a1.x, wq, acc1[4 * c + 0]); acc1[4 * c + 1] = fmaf(a1.y, wq, acc1[4 * c + 1]);
            acc1[4 * c + 2] = fmaf(a1.z, wq, acc1[4 * c + 2]); acc1[4 * c + 3] = fmaf(a1.w, wq, acc1[4 * c + 3]);
        }
    }
}

// A piece's outputs for this thread's row in both tiles: nc columns from packed column col0
// on, into the two tiles' group rings (y0: [hi, lo] of the first tile, y1 of the second).
template <bool BF16, int NV>
__device__ __forceinline__ void f0_piece2(const float* yp, int pitch, const float* rr, int D, int qa, int qb, int sh,
                                          int nc, int col0, int row, uint8_t* y0, uint8_t* y1) {
    float acc0[4 * NV], acc1[4 * NV];
    f0_taps2<NV>(yp, pitch, rr, D, qa, qb, sh, acc0, acc1);
    constexpr int plane = kYhRing * 128 * 16;
#pragma unroll
    for (int j = 0; j < 4 * NV; ++j) {
        if (j < nc) {
            const int col = col0 + j;
            const int o = ((col >> 3) & (kYhRing - 1)) * 2048 + row * 16 + (col & 7) * 2;
            put_hilo<BF16>(y0, y0 + plane, o, acc0[j]);
            put_hilo<BF16>(y1, y1 + plane, o, acc1[j]);
        }
    }
}

// Yhat of one work unit (bank, detector, group of tiles) into HBM (see the file comment).
// Per unit the slices' composed upsamplers are staged once.  Tiles go in pairs: the rows of
// Y each slice reaches from both tiles are staged in FP32 for a batch of (slice, up to
// 16-column) pieces at a time (four loads per thread in flight), then each thread forms the
// outputs of its time row in both tiles piece by piece in column order (a tap serves both),
// stores their hi/lo halves into its row of each tile's ring of 8-column groups, and sends
// every group it has completed to HBM as one 16-byte store per plane (a warp: 512
// contiguous bytes), zeroing the slot for its next use.
template <bool BF16>
__global__ void __launch_bounds__(kYhThreads)
    k_yhat(const F0Job* __restrict__ jobs, const YupSlice* __restrict__ slices, const F0Piece* __restrict__ pieces,
           const int* __restrict__ batch_end, const F0Unit* __restrict__ units, long long k_a, int n, int det0,
           long long window, int rall) {
    constexpr int NB = kYhThreads;
    const int tpw = (int)(window / 128);
    const int n_tiles = n / 128;
    const int row = threadIdx.x;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    constexpr int yplane = kYhRing * 128 * 16;
    uint8_t* ring = smem;                                  // the rows' group rings: [tile][hi, lo][kYhRing][128][8]
    float* ys = reinterpret_cast<float*>(ring + 4 * yplane);   // staged Y rows of a batch
    float* rsm = ys + kF0StageFloats;                      // the unit's composed upsamplers
    F0SliceS* stab = reinterpret_cast<F0SliceS*>(rsm + rall);
    F0Piece* ptab = reinterpret_cast<F0Piece*>(stab + kF0MaxSlices);
    int* bends = reinterpret_cast<int*>(ptab + kF0MaxPieces);   // end piece of each batch

    const F0Unit un = units[blockIdx.x];
    const F0Job jb = jobs[un.job];
    const int det = det0 + (int)blockIdx.y;
    const int t0 = un.g * tpw, t1 = min(t0 + tpw, n_tiles);
    pdl_wait();   // the FIR's output is written by an earlier kernel of the stream
    for (int q = threadIdx.x; q < jb.ns; q += NB) {
        const YupSlice sl = slices[jb.s0 + q];
        F0SliceS& t = stab[q];
        t.y_hi = sl.y_hi + det * sl.y_det_stride;
        t.y_lo = sl.y_lo + det * sl.y_det_stride;
        t.y_rows = sl.y_rows; t.y_ld = sl.y_ld; t.D = sl.D; t.e_min = sl.e_min; t.rlen = sl.rlen;
        t.L = sl.L; t.roff = sl.roff; t.nq = sl.nq; t.qoff = sl.qoff; t.col0 = sl.tcol;
    }
    for (int i = threadIdx.x; i < jb.np; i += NB) ptab[i] = pieces[jb.pc0 + i];
    for (int i = threadIdx.x; i < jb.nbat; i += NB) bends[i] = batch_end[jb.bt0 + i];
    for (int q = 0; q < jb.ns; ++q) {
        const YupSlice& sl = slices[jb.s0 + q];
        for (int e = threadIdx.x; e < sl.rlen; e += NB) rsm[sl.roff + e] = __ldg(sl.R + e);
    }
    __syncthreads();
    uint4* ghi = reinterpret_cast<uint4*>(jb.yh + (long long)det * 2 * jb.K * jb.yrows) + row;
    uint4* glo = ghi + (long long)jb.K * jb.yrows / 8;
    const uint4 z4 = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int g = 0; g < 4 * kYhRing; ++g)                   // empty slots read as zero (the padding columns)
        *reinterpret_cast<uint4*>(ring + g * 2048 + row * 16) = z4;
    // group g of this row's tiles tt (and tt + 1 when `both`) to HBM, the slots zeroed
    auto flush = [&](int g, int tt, bool both) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint4* sh = reinterpret_cast<uint4*>(ring + h * 2 * yplane + (g & (kYhRing - 1)) * 2048 + row * 16);
            uint4* sl = reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(sh) + yplane);
            if (h == 0 || both) {
                const long long o = (long long)g * jb.yrows + 128LL * (tt + h);
                ghi[o] = *sh;
                glo[o] = *sl;
            }
            *sh = z4;
            *sl = z4;
        }
    };
    for (int tt = t0; tt < t1; tt += 2) {
        const long long k0 = k_a + 128LL * tt;
        const bool both = tt + 1 < t1;                      // the second tile of the pair is in the push
        int flushed = 0;                                    // groups of these tiles already sent
        for (int bt = 0, p0 = 0; bt < jb.nbat; ++bt) {
            const int p1 = bends[bt];
            const int n_items = ptab[p1 - 1].item0 + ptab[p1 - 1].items;
            // stage: four items per thread in flight at a time
            for (int e0 = threadIdx.x; e0 < n_items; e0 += 4 * NB) {
                uint2 hv[4], lv[4];
                int dst[4];
#pragma unroll
                for (int uu = 0; uu < 4; ++uu) {
                    const int e = e0 + uu * NB;
                    dst[uu] = -1;
                    if (e < n_items) {
                        int pi = p0;
                        while (pi + 1 < p1 && ptab[pi + 1].item0 <= e) ++pi;
                        const F0Piece pc = ptab[pi];
                        const F0SliceS& t = stab[pc.s];
                        const int ie = e - pc.item0, qi = ie / pc.nv, c4 = ie - qi * pc.nv;
                        const long long q_lo = k0 / t.D + t.qoff;
                        const long long o = ((q_lo + qi) & (t.y_rows - 1)) * t.y_ld + pc.c0 + 4 * c4;
                        hv[uu] = *reinterpret_cast<const uint2*>(t.y_hi + o);
                        lv[uu] = *reinterpret_cast<const uint2*>(t.y_lo + o);
                        dst[uu] = pc.off + qi * pc.pitch + 4 * c4;
                    }
                }
#pragma unroll
                for (int uu = 0; uu < 4; ++uu) {
                    if (dst[uu] < 0) continue;
                    const float2 x0 = hilo_pair<BF16>(hv[uu].x, lv[uu].x);
                    const float2 x1 = hilo_pair<BF16>(hv[uu].y, lv[uu].y);
                    *reinterpret_cast<float4*>(ys + dst[uu]) = make_float4(x0.x, x0.y, x1.x, x1.y);
                }
            }
            __syncthreads();
            for (int pi = p0; pi < p1; ++pi) {
                const F0Piece pc = ptab[pi];
                const F0SliceS& t = stab[pc.s];
                if (pc.nv == 0) {                           // a slice at f0: Yhat = Y, this row of the ring
                    for (int c = 0; c < pc.nc; c += 8) {
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const long long o = ((k0 + 128 * h + t.qoff + row) & (t.y_rows - 1)) * t.y_ld;
                            const uint4 hv = *reinterpret_cast<const uint4*>(t.y_hi + o + c);
                            const uint4 lv = *reinterpret_cast<const uint4*>(t.y_lo + o + c);
                            const float2 x[4] = {hilo_pair<BF16>(hv.x, lv.x), hilo_pair<BF16>(hv.y, lv.y),
                                                 hilo_pair<BF16>(hv.z, lv.z), hilo_pair<BF16>(hv.w, lv.w)};
                            uint8_t* yh = ring + h * 2 * yplane;
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                const int col = t.col0 + c + j;
                                if (c + j < pc.nc)
                                    put_hilo<BF16>(yh, yh + yplane,
                                                   ((col >> 3) & (kYhRing - 1)) * 2048 + row * 16 + (col & 7) * 2,
                                                   (j & 1) ? x[j >> 1].y : x[j >> 1].x);
                            }
                        }
                        for (const int done = (t.col0 + c + min(8, pc.nc - c)) >> 3; flushed < done; ++flushed)
                            flush(flushed, tt, both);
                    }
                    continue;
                }
                const int D = t.D;
                const int r0 = row - D * t.qoff - t.e_min;       // R index of (row, the tile's first row)
                const int qa = max(0, (r0 - t.rlen + D) / D), qb = min(t.nq - 1, r0 / D);
                const float* rr = rsm + t.roff + r0;
                const float* yp = ys + pc.off;
                const int c0 = t.col0 + pc.c0;
                uint8_t* r1 = ring + 2 * yplane;
                switch (pc.nv) {
                    case 1: f0_piece2<BF16, 1>(yp, pc.pitch, rr, D, qa, qb, 128 / D, pc.nc, c0, row, ring, r1); break;
                    case 2: f0_piece2<BF16, 2>(yp, pc.pitch, rr, D, qa, qb, 128 / D, pc.nc, c0, row, ring, r1); break;
                    case 3: f0_piece2<BF16, 3>(yp, pc.pitch, rr, D, qa, qb, 128 / D, pc.nc, c0, row, ring, r1); break;
                    default: f0_piece2<BF16, 4>(yp, pc.pitch, rr, D, qa, qb, 128 / D, pc.nc, c0, row, ring, r1); break;
                }
                for (const int done = (c0 + pc.nc) >> 3; flushed < done; ++flushed) flush(flushed, tt, both);
            }
            __syncthreads();                                // the staging is free for the next batch
            p0 = p1;
        }
        for (; flushed < jb.K / 8; ++flushed) flush(flushed, tt, both);   // the last group and the padding
    }
    pdl_launch_dependents();
}

template <bool BF16, bool STORE_Z>
__global__ void __launch_bounds__(kF0Threads, 1)
    k_f0_top(const F0Job* __restrict__ jobs, const F0Maps* __restrict__ maps, const F0Unit* __restrict__ units, const int* __restrict__ sched, int n_units, int kc, int ybufs,
             long long k_a, int n, int det0, int n_det_push, long long window, float threshold,
             Partial* __restrict__ part, long long part_tmpl_stride, int n_slots, TailRing tail,
             SlabEntry* __restrict__ slab_base, int ring, int n_det_total, long long slab_det_stride,
             float* __restrict__ zout, int* __restrict__ err) {
    using C = F0Cfg<BF16>;
    pdl_launch_dependents();
    const int tpw = (int)(window / 128);
    const int n_tiles = n / 128;
    // every group is one whole window, which the kernel finalises itself (with a window
    // overlap the window also needs the tail of the tile before it: the partial ring then)
    const bool aligned = (k_a % window) == 0 && tail.ov == 0;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);   // 1 KB aligned, still a shared pointer
    uint8_t* cst = smem;                                   // CSTAGES x CSTAGE
    uint8_t* ybuf = cst + C::CSTAGES * C::CSTAGE;          // ybufs x [hi, lo][kc / 8][128][8]
    const int yplane = 128 * kc * 2;
    float4* rs = reinterpret_cast<float4*>(ybuf + ybufs * 2 * yplane);   // [kF0MaxTm][128] running window maxima
    float4* red = rs + kF0MaxTm * 128;                     // [8] bank-max partials of the epilogue warps
    uint64_t* bars = reinterpret_cast<uint64_t*>(red + kF0EpiWarps);   // 2 x 4 + 2 x 2 + 2 x 2 + 1
    uint64_t* cfull = bars;
    uint64_t* cempty = cfull + kF0MaxCStages;
    uint64_t* yfull = cempty + kF0MaxCStages;
    uint64_t* yempty = yfull + 2;
    uint64_t* tfull = yempty + 2;
    uint64_t* tempty = tfull + 2;
    uint64_t* drain = tempty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < C::CSTAGES; ++s) { mbar_init(cfull + s, 1); mbar_init(cempty + s, 1); }
        for (int b = 0; b < 2; ++b) {
            mbar_init(yfull + b, 1); mbar_init(yempty + b, 1);
            mbar_init(tfull + b, 1); mbar_init(tempty + b, 32 * kF0EpiWarps / 2);
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
            // A stage is free again once the MMAs that read it are done: the issuer commits to
            // cempty after every chunk but a template group's last, whose stage the epilogue
            // group frees when it sees the group's accumulator (a commit costs the tensor pipe
            // about as much as a few MMAs).  Either way one arrival per use of the stage.
            int stage = 0, yi = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int u = ub; u < ue && ok; ++u) {
                const int it = sched[gridDim.x + 1 + u];
                const int det = det0 + it % n_det_push;
                const F0Unit un = units[it / n_det_push];
                const F0Job jb = jobs[un.job];                 // a copy: the asm "memory" clobbers would reload it
                const F0Maps* mp = maps + jb.map;
                const int t0 = un.g * tpw, t1 = min(t0 + tpw, n_tiles);
                for (int tt = t0; tt < t1 && ok; ++tt, ++yi) {
                    // the tile's Yhat: one box per plane, once the MMAs of the buffer's last tile are done
                    const int yb = ybufs == 2 ? (yi & 1) : 0;
                    const uint32_t ypar = ybufs == 2 ? ((yi >> 1) & 1) : (yi & 1);
                    if (!mbar_wait(yempty + yb, ypar ^ 1, err, 67)) { ok = false; break; }
                    mbar_expect_tx(yfull + yb, (uint32_t)(2 * jb.K * 256));
                    uint8_t* yh = ybuf + yb * 2 * yplane;
                    tma_load_4d(yh, &mp->y, yfull + yb, 0, 4 * tt, 0, det * 2);
                    tma_load_4d(yh + yplane, &mp->y, yfull + yb, 0, 4 * tt, 0, det * 2 + 1);
                    for (int tm = 0; tm < jb.tiles_m && ok; ++tm) {
                        for (int kc0 = 0; kc0 < jb.K; kc0 += 32) {
                            if (!mbar_wait(cempty + stage, phase ^ 1, err, 61)) { ok = false; break; }
                            uint8_t* sb = cst + stage * C::CSTAGE;
                            mbar_expect_tx(cfull + stage, C::CSTAGE);
#pragma unroll
                            for (int pl = 0; pl < C::NPL; ++pl)
                                tma_load_4d(sb + pl * C::CPLANE, &mp->c, cfull + stage, 0, tm * 4, kc0 >> 3, pl);
                            if (++stage == C::CSTAGES) { stage = 0; phase ^= 1; }
                        }
                    }
                }
            }
            for (int s2 = 0; s2 < C::CSTAGES && ok; ++s2) {
                if (!mbar_wait(cempty + stage, phase ^ 1, err, 62)) break;
                if (++stage == C::CSTAGES) { stage = 0; phase ^= 1; }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {   // ------------------------------------------------ MMA issuer
            constexpr uint32_t idesc = idesc_f16(BF16, 128, 128);
            int stage = 0, i = 0, yi = 0;
            uint32_t phase = 0, nb[2] = {0u, 0u};         // uses of each TMEM buffer (buffer = tm & 1)
            bool ok = true;
            for (int u = ub; u < ue && ok; ++u) {
                const int it = sched[gridDim.x + 1 + u];
                const F0Unit un = units[it / n_det_push];
                const F0Job jb = jobs[un.job];                 // a copy: the asm "memory" clobbers would reload it
                const int t0 = un.g * tpw, t1 = min(t0 + tpw, n_tiles);
                const int k16 = jb.K / 16;
                for (int tt = t0; tt < t1 && ok; ++tt, ++yi) {
                    const int yb = ybufs == 2 ? (yi & 1) : 0;
                    const uint32_t ypar = ybufs == 2 ? ((yi >> 1) & 1) : (yi & 1);
                    if (!mbar_wait(yfull + yb, ypar, err, 63)) { ok = false; break; }
                    tc_fence_after();
                    // descriptors of the tile's Yhat planes; those of a stage and of each 16-wide K step
                    // follow by adding (byte offset >> 4) to the start-address field (addresses < 256 KB:
                    // no carry out of it).  Issuing an MMA takes the issuing thread about as long as the
                    // MMA runs, so the descriptors are formed before the chunk's MMAs, not between them.
                    const uint64_t byh = desc_win(smem_u32(ybuf + yb * 2 * yplane)), byl = byh + (uint64_t)(yplane >> 4);
                    for (int tm = 0; tm < jb.tiles_m && ok; ++tm, ++i) {
                        const int buf = tm & 1;
                        const uint32_t use = nb[buf]++;
                        if (!mbar_wait(tempty + buf, (use & 1) ^ 1, err, 64)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t d_re = tmem + buf * 256, d_im = d_re + 128;
                        for (int kc0 = 0; kc0 < jb.K; kc0 += 32) {
                            if (!mbar_wait(cfull + stage, phase, err, 65)) { ok = false; break; }
                            tc_fence_after();
                            const uint64_t ba = desc_win(smem_u32(cst + stage * C::CSTAGE));
                            const int nk = min(2, k16 - kc0 / 16);    // 16-wide K steps in this chunk
                            uint64_t a[2][4], bh[2], bl[2];
#pragma unroll
                            for (int j = 0; j < 2; ++j) {
#pragma unroll
                                for (int pl = 0; pl < 4; ++pl) a[j][pl] = ba + (uint64_t)((pl * C::CPLANE + j * 4096) >> 4);
                                bh[j] = byh + (uint64_t)((kc0 / 16 + j) * 256);
                                bl[j] = byl + (uint64_t)((kc0 / 16 + j) * 256);
                            }
                            const uint32_t acc0 = kc0 > 0 ? 1u : 0u;
#pragma unroll
                            for (int j = 0; j < 2; ++j) {
                                if (j >= nk) break;
                                const uint32_t aj = j > 0 ? 1u : acc0;
                                umma_f16(d_re, a[j][0], bh[j], idesc, aj);
                                umma_f16(d_re, a[j][0], bl[j], idesc, 1u);
                                umma_f16(d_im, a[j][1], bh[j], idesc, aj);
                                umma_f16(d_im, a[j][1], bl[j], idesc, 1u);
                                if (BF16) {
                                    umma_f16(d_re, a[j][2], bh[j], idesc, 1u);
                                    umma_f16(d_im, a[j][3], bh[j], idesc, 1u);
                                }
                            }
                            if (kc0 + 32 < jb.K) umma_commit(cempty + stage);   // the last: the epilogue frees it
                            if (++stage == C::CSTAGES) { stage = 0; phase ^= 1; }
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
    } else {
        // ---------------------------------------------------------------- epilogue
        // Two groups of four warps, one per TMEM buffer: group g takes the template groups
        // tm with tm & 1 == g, all 128 samples of each tile; warp & 3 is the TMEM lane quarter.
        // No barrier inside a unit: each group runs at its own pace.
        const int qd = warp & 3;
        const int grp = (warp - 2) >> 2;
        const int rowm = qd * 32 + lane;
        uint32_t nuse = 0;                                  // uses of this group's buffer
        long long chunks = 0;                               // coefficient chunks of the CTA's earlier units
        for (int u = ub; u < ue; ++u) {
            const int it = sched[gridDim.x + 1 + u];
            const int det = det0 + it % n_det_push;
            const F0Unit un = units[it / n_det_push];
            const F0Job jb = jobs[un.job];                 // a copy: the asm "memory" clobbers would reload it
            const int t0 = un.g * tpw, t1 = min(t0 + tpw, n_tiles);
            const int nch = (jb.K + 31) / 32;                // coefficient chunks per template group
            float gbest = -1.f;                             // bank maximum of this thread's rows
            int gm = 0x7fffffff;
            bool fail = false;
            for (int tt = t0; tt < t1 && !fail; ++tt) {
                for (int tm = grp; tm < jb.tiles_m; tm += 2) {
                    const bool got = __all_sync(0xffffffffu, mbar_wait(tfull + grp, nuse & 1, err, 68));
                    ++nuse;
                    if (!got) { fail = true; break; }
                    tc_fence_after();
                    if (qd == 0 && lane == 0) {             // the MMAs have read the group's last chunk
                        const long long last = chunks + ((long long)(tt - t0) * jb.tiles_m + tm + 1) * nch - 1;
                        mbar_arrive(cempty + (int)(last % C::CSTAGES));
                    }
                    const uint32_t base = tmem + ((uint32_t)(qd * 32) << 16) + grp * 256;
                    const int m = tm * 128 + rowm;
                    const long long k0 = k_a + 128LL * tt;
                    const bool pre = tail.ov > 0 && (k0 + 128) % window == 0;   // the next window's overlap
                    const int tail_from = pre ? 128 - tail.ov : 128;
                    const long long kwin0 = (k0 / window) * window;
                    const int kb = (int)(k0 - kwin0);          // the tile's first sample in its window
                    // best: the tile's maximum, or with whole windows the window's so far (then a
                    // chunk is searched for its sample only when it beats the window, not the tile)
                    float best = -1.f, bre = 0.f, bim = 0.f, tbest = -1.f, tre = 0.f, tim = 0.f;
                    int bk = 0x7fffffff, tk = 0x7fffffff;      // bk: offset in the window
                    if (aligned && tt > t0) {
                        const float4 prev = rs[tm * 128 + rowm];
                        best = prev.x; bk = __float_as_int(prev.y); bre = prev.z; bim = prev.w;
                    }
                    // 16-sample chunks of re and im; the next chunk's loads are in flight while
                    // this one is reduced (two register sets, one wait per chunk)
                    auto chunk = [&](const uint32_t (&ru)[16], const uint32_t (&iu)[16], int c) {
                        // |z|^2 and its maximum first; the sample (the first that reaches it) and its
                        // re, im only when the chunk beats what came before (earlier samples win ties)
                        float ma = -1.f, mb = -1.f;          // two chains of three-way maxima
#pragma unroll
                        for (int j = 0; j < 16; j += 4) {
                            float p0, p1, p2, p3;
                            zsq2(ru[j], ru[j + 1], iu[j], iu[j + 1], p0, p1);
                            zsq2(ru[j + 2], ru[j + 3], iu[j + 2], iu[j + 3], p2, p3);
                            ma = fmax3f(ma, p0, p1);
                            mb = fmax3f(mb, p2, p3);
                        }
                        const float mx = fmaxf(ma, mb);
                        if (mx > best) {                     // |z|^2 again (same bits) to find the sample
                            uint32_t eq = 0;
#pragma unroll
                            for (int j = 0; j < 16; j += 2) {
                                float p0, p1;
                                zsq2_again(ru[j], ru[j + 1], iu[j], iu[j + 1], p0, p1);
                                eq |= ((p0 == mx ? 1u : 0u) | (p1 == mx ? 2u : 0u)) << j;
                            }
                            const int jj = __ffs(eq) - 1;
                            float sr = 0.f, si = 0.f;
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                sr = j == jj ? __uint_as_float(ru[j]) : sr;
                                si = j == jj ? __uint_as_float(iu[j]) : si;
                            }
                            best = mx;
                            bk = kb + c + jj;
                            bre = sr;
                            bim = si;
                        }
                        if (pre && c + 16 > tail_from) {    // the tail of a tile before a window start
#pragma unroll
                            for (int j = 0; j < 16; j += 2) {
                                float pp[2];
                                zsq2_again(ru[j], ru[j + 1], iu[j], iu[j + 1], pp[0], pp[1]);
#pragma unroll
                                for (int h = 0; h < 2; ++h)
                                    if (c + j + h >= tail_from && pp[h] > tbest) {
                                        tbest = pp[h]; tk = c + j + h;
                                        tre = __uint_as_float(ru[j + h]); tim = __uint_as_float(iu[j + h]);
                                    }
                            }
                        }
                        if (STORE_Z && m < jb.M) {
                            float* zr = zout + (long long)(2 * m) * n + 128LL * tt + c;
                            float* zi = zr + n;
#pragma unroll
                            for (int j = 0; j < 16; ++j) { zr[j] = __uint_as_float(ru[j]); zi[j] = __uint_as_float(iu[j]); }
                        }
                    };
                    uint32_t ra[16], ia[16], rb[16], ib[16];
                    tmem_ld16_nw(base, ra);
                    tmem_ld16_nw(base + 128, ia);
                    tmem_wait_ld16(ra, ia);
#pragma unroll 1
                    for (int c = 0; c < 128; c += 32) {
                        tmem_ld16_nw(base + c + 16, rb);
                        tmem_ld16_nw(base + 128 + c + 16, ib);
                        chunk(ra, ia, c);
                        tmem_wait_ld16(rb, ib);
                        if (c + 32 < 128) {
                            tmem_ld16_nw(base + c + 32, ra);
                            tmem_ld16_nw(base + 128 + c + 32, ia);
                        }
                        chunk(rb, ib, c + 16);
                        if (c + 32 < 128) tmem_wait_ld16(ra, ia);
                    }
                    tc_fence_before();
                    mbar_arrive(tempty + grp);
                    if (STORE_Z) continue;
                    if (!aligned) {
                        if (m < jb.M) {
                            const int slot = (int)((k0 / 128) & (n_slots - 1));
                            part[(long long)(jb.tmpl0 + m) * part_tmpl_stride + (long long)det * n_slots + slot] =
                                make_float4(best, __int_as_float(bk), bre, bim);
                            if (pre) {
                                const long long w1 = (k0 + 128) / window;
                                tail.p[(long long)(jb.tmpl0 + m) * tail.tmpl_stride + (long long)det * tail.n +
                                       (w1 & (tail.n - 1))] =
                                    make_float4(tbest, __int_as_float((int)(k0 - w1 * window) + tk), tre, tim);
                            }
                        }
                        continue;
                    }
                    const float4 r = make_float4(best, __int_as_float(bk), bre, bim);   // earlier tiles won ties
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
            chunks += (long long)(t1 - t0) * jb.tiles_m * nch;
            if (STORE_Z) {
                if (fail) break;
                continue;
            }
            // both groups agree that the unit went through (a wait that ran out stops them together)
            uint32_t all_ok;
            asm volatile(
                "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
                "bar.red.and.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
                : "=r"(all_ok)
                : "r"((uint32_t)!fail), "n"(32 * kF0EpiWarps)
                : "memory");
            if (!all_ok) break;
            if (!aligned || t1 - t0 != tpw) continue;
            // the bank's loudest template of the window (lowest index on ties), over both groups;
            // its slot gets the bank-maximum flag if it triggered
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, gbest, o);
                const int om = __shfl_xor_sync(0xffffffffu, gm, o);
                if (ob > gbest || (ob == gbest && om < gm)) { gbest = ob; gm = om; }
            }
            const int ew = warp - 2;
            if (lane == 0) red[ew] = make_float4(gbest, __int_as_float(gm), 0.f, 0.f);
            asm volatile("bar.sync 2, %0;" ::"n"(32 * kF0EpiWarps) : "memory");
            float vb = red[0].x;
            int vm = __float_as_int(red[0].y);
#pragma unroll
            for (int q = 1; q < kF0EpiWarps; ++q) {
                const float x = red[q].x;
                const int mm = __float_as_int(red[q].y);
                if (x > vb || (x == vb && mm < vm)) { vb = x; vm = mm; }
            }
            if (vm < jb.M && (vm & 127) == rowm && ((vm >> 7) & 1) == grp) {   // the thread that wrote that slot
                const long long w = (k_a + 128LL * t0) / window;
                SlabEntry* out = slab_base + (size_t)(w % ring) * n_det_total * slab_det_stride +
                                 (size_t)det * slab_det_stride + jb.tmpl0 + vm;
                if (out->flags & 1) out->flags |= 2;
            }
            asm volatile("bar.sync 2, %0;" ::"n"(32 * kF0EpiWarps) : "memory");   // red[] is reused by the next unit
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
