// Device-side job descriptors shared by the LLOID kernels and the host code.
//
// Every launch covers many independent pieces of work (detectors, banks,
// slices, tiles) through a flat grid: blockIdx.x enumerates tiles of all jobs,
// a job's tiles start at tile_base[job], and blockIdx.y is the detector.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace lloid {

// Split v into a 16-bit hi part and the 16-bit rounding of the remainder:
// mode 1 = FP16, mode 2 = BF16 (the data operand of the split-precision paths).
__device__ __forceinline__ void split_hilo_rt(float v, int mode, uint16_t& hi, uint16_t& lo) {
    if (mode == 2) {
        __nv_bfloat16 h = __float2bfloat16_rn(v);
        __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
        hi = *reinterpret_cast<uint16_t*>(&h);
        lo = *reinterpret_cast<uint16_t*>(&l);
    } else {
        __half h = __float2half_rn(v);
        __half l = __float2half_rn(v - __half2float(h));
        hi = *reinterpret_cast<uint16_t*>(&h);
        lo = *reinterpret_cast<uint16_t*>(&l);
    }
}

// Programmatic dependent launch: a kernel lets the next one in the stream be
// scheduled as soon as all its CTAs have started, and waits for the previous
// one to finish (and its writes to be visible) before touching its results.
// Both are no-ops for a launch without the programmatic-serialisation attribute.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

constexpr int kTileT = 128;      // time tile of the reconstruction = window granule
constexpr int kMaxRates = 8;     // downsampled streams f0/2 ... f0/256

// a2: one (bank, slice) basis-filter job.  Y^s_l[q] = sum_m u_l[m] x[q - src_off - m]
// where x is the slice-rate stream (Eq. 5 with the pre-synchronised offset, Eq. 9).
struct FirJob {
    const float* bases;          // [L][N] FP32
    const float* src;            // stream ring of this rate, detector 0
    long long src_det_stride;
    long long src_off;           // J_s / D_s
    float* dst;                  // Y ring [L][y_len], detector 0
    long long dst_det_stride;
    int src_mask;
    int dst_mask;                // ring mask
    int dst_ld;                  // row stride of dst
    int L, N, D;
    int c_hi;                    // look-ahead of the slice's upsampler (full-rate samples)
    int q_count;                 // new outputs per push (n / D)
    int tiles_l, tiles_q;
};

// a4 (slice part): Yhat_l[K] = sum_q Y_l[q] R[K - D q - e_min], the slice's
// ladder of Eq. 7-8 upsamplers composed into one polyphase filter R (R = [1]
// for slices already at f0, which this step only converts).
struct UpJob {
    const float* yring;          // [L][y_len], detector 0
    long long y_det_stride;
    void* yhat;                  // first Yhat row of this slice, detector 0
    void* yhat_lo;               // split formats: the low halves
    long long yhat_det_stride;
    const float* R;              // [rlen]
    int y_mask;
    int y_ld;
    int ldy;                     // Yhat row stride (max_block)
    int e_min, rlen;
    int D, L;
    int tiles_k;                 // K tiles of 256 per basis row
};

// a3 + a4 (sum) + a5: z = C Yhat for one bank, |z|^2 window maxima per tile.
struct ReconJob {
    const void* c_re;            // [Mpad][Kpad] real-part coefficient rows
    const void* c_im;            // [Mpad][Kpad] imaginary-part rows
    const void* yhat;            // [Kpad][ldy] (detector 0); split formats add yhat_lo
    const void* yhat_lo;
    long long yhat_det_stride;   // elements
    int ldy;
    int Kpad, Mpad, M;
    int tmpl0;                   // first global template id of the bank
    int tiles_m, tiles_t;
    uint32_t* zring;             // Eq. 10 banks: [det][Mpad][zring_len] z as half2, else null
    long long zring_det_stride;
    int zring_len;
};

// Per (template, detector, time tile) partial maximum of |z|^2.
// x = |z|^2, y = sample offset inside its window (int bits), z = Re, w = Im.
using Partial = float4;

// Window overlap (Section II.D.1): window w also covers the `ov` samples before its
// start.  A 128-sample tile that ends where a window starts keeps the maximum over its
// last ov samples (sample offsets relative to that window's start, so negative) in
// p[tmpl * tmpl_stride + det * n + (w mod n)], w the window it precedes.  ov = 0: none.
struct TailRing {
    Partial* p;
    long long tmpl_stride;
    int n;                       // windows in the ring (power of two)
    int ov;                      // 0 .. 127
};

// Dense per-window trigger slot for one (detector, template).
struct SlabEntry {
    float snr, phase, re, im;
    int32_t k_off;               // sample - window start
    int32_t flags;               // bit 0 valid (|z| > threshold), bit 1 bank max
    float xi2;                   // Eq. 10, < 0 until computed (or without autocorrelation)
    int32_t pad;
};

// Eq. 10 for one bank: its templates' autocorrelations and the ring of its
// recent SNR samples (written by the top-level reconstruction).
struct Xi2Job {
    int tmpl0, M, half;          // first global template id, templates, d
    const float2* ac;            // [M][2 d + 1] R_i(t)
    const float* den;            // [M] sum_t (2 - 2 |R_i(t)|^2)
    const uint32_t* zring;       // [det][Mpad][zlen] z as packed half2 (re low, im high)
    long long zdet_stride;       // elements
    int zlen;                    // power of two
};

struct FinJob {
    int tmpl0, M, bank;
    uint32_t* bg;                // background counts [det][n_snr][n_xi2], or null
    int fused;                   // 1: the f0 kernel finalises the windows of pushes that start on a window
};

// One (bank, window) slot of the clustered coincident events.
struct EventEntry {
    float net_snr;               // < 0: no event
    int32_t tmpl;                // bank-local
    int32_t n_ifo;
    uint32_t ifo_mask;
    int32_t ref_det;
    int32_t ref_k_off;           // sample - window start of the reference trigger
    int32_t pad[2];
};

}  // namespace lloid
