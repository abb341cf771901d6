// Allocation-free variant of the trigger stage (window maxima + compaction).
//
// Some callers cannot allocate device memory while they run: a real-time
// strain callback with a fixed latency budget must not block in cudaMalloc
// (which can synchronise the whole device), and a host framework that owns
// the GPU's memory pool may forbid allocations made behind its back.  For
// them, lloid_triggers_from_snr_noalloc finds the triggers of an SNR block the
// caller already holds on the device, using only a scratch array compiled
// into this library.
//
// The scratch lives in one file-scope __device__ array (kScratchBytes, about
// 4.2 MB), present on every GPU that loads the library until the process
// exits.  Host code must not hand the array's name to a kernel (on the host
// it is only a stand-in symbol, not a device address): the device address is
// looked up once per device with cudaGetSymbolAddress and cached.  All calls
// share the array, so calls whose GPU work overlaps (different streams, or
// different host threads on one device) race on it and must be serialised by
// the caller.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/lloid.h"

namespace {

constexpr long long kMaxPairs = 1LL << 18;                 // template x window pairs per call
constexpr long long kChunk = 1024;                         // compaction chunk (one CTA)
constexpr long long kMaxChunks = kMaxPairs / kChunk;
constexpr size_t kPairBytes = (size_t)kMaxPairs * 16;      // per pair: |z|^2, sample, re, im
constexpr size_t kScratchBytes = kPairBytes + (size_t)kMaxChunks * 4 + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct TrigOut {   // the layout of lloid_trigger
    int32_t detector, bank, tmpl, is_bank_max;
    long long window, sample;
    float snr, phase, re, im;
    float xi2;
    int32_t pad;
};

// Pair p = wl * M + i: the maximum of |z_i|^2 over window wl (earliest sample on ties).
__global__ void k_na_window_max(const float* __restrict__ z, int M, long long n, long long W, float4* __restrict__ pairs) {
    const long long p = blockIdx.x;
    const int i = (int)(p % M);
    const long long wl = p / M;
    const float* re = z + (long long)(2 * i) * n + wl * W;
    const float* im = re + n;
    float best = -1.f, bre = 0.f, bim = 0.f;
    int bk = 0x7fffffff;
    for (long long k = threadIdx.x; k < W; k += blockDim.x) {
        const float a = re[k], b = im[k];
        const float q = a * a + b * b;
        if (q > best) { best = q; bk = (int)k; bre = a; bim = b; }
    }
    __shared__ float sb[32], sre[32], sim[32];
    __shared__ int sk[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int ok = __shfl_xor_sync(0xffffffffu, bk, o);
        const float ore = __shfl_xor_sync(0xffffffffu, bre, o), oim = __shfl_xor_sync(0xffffffffu, bim, o);
        if (ob > best || (ob == best && ok < bk)) { best = ob; bk = ok; bre = ore; bim = oim; }
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { sb[w] = best; sk[w] = bk; sre[w] = bre; sim[w] = bim; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int j = 1; j < (int)(blockDim.x >> 5); ++j)
            if (sb[j] > best || (sb[j] == best && sk[j] < bk)) { best = sb[j]; bk = sk[j]; bre = sre[j]; bim = sim[j]; }
        pairs[p] = make_float4(best, __int_as_float(bk), bre, bim);
    }
}

__global__ void k_na_count(const float4* __restrict__ pairs, long long n_pairs, float thr, int* __restrict__ counts) {
    const long long p = blockIdx.x * kChunk + threadIdx.x;
    int v = 0;
    if (p < n_pairs) v = sqrtf(pairs[p].x) > thr;
    v = __syncthreads_count(v);
    if (threadIdx.x == 0) counts[blockIdx.x] = v;
}

// Scatter in (window, template) order; the loudest template of each window
// (lowest index on ties) carries is_bank_max if it passes the threshold.
__global__ void k_na_scatter(const float4* __restrict__ pairs, long long n_pairs, int M, const int* __restrict__ counts,
                             float thr, int det, int bank, long long w0, long long W, TrigOut* __restrict__ out,
                             long long cap, long long* __restrict__ n_out) {
    __shared__ int red[kChunk / 32];
    __shared__ int base_s;
    int s = 0, tot = 0;
    for (int i = threadIdx.x; i < (int)blockIdx.x; i += blockDim.x) s += counts[i];
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) tot += counts[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) { s += __shfl_xor_sync(0xffffffffu, s, o); tot += __shfl_xor_sync(0xffffffffu, tot, o); }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __shared__ int red2[kChunk / 32];
    if (lane == 0) { red[wid] = s; red2[wid] = tot; }
    __syncthreads();
    if (threadIdx.x == 0) {
        int a = 0, b = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { a += red[i]; b += red2[i]; }
        base_s = a;
        if (blockIdx.x == 0) *n_out = b;
    }
    __syncthreads();
    const long long p = blockIdx.x * kChunk + threadIdx.x;
    float4 e = make_float4(-1.f, 0.f, 0.f, 0.f);
    int v = 0;
    if (p < n_pairs) { e = pairs[p]; v = sqrtf(e.x) > thr; }
    const unsigned ball = __ballot_sync(0xffffffffu, v);
    const int pre = __popc(ball & ((1u << lane) - 1));
    __syncthreads();
    if (lane == 0) red[wid] = __popc(ball);
    __syncthreads();
    int wpre = 0;
    for (int i = 0; i < wid; ++i) wpre += red[i];
    if (!v) return;
    const long long pos = (long long)base_s + wpre + pre;
    if (pos >= cap) return;
    const int i = (int)(p % M);
    const long long wl = p / M;
    // bank maximum of this window: scan the window's templates (M is small per bank)
    const float4* row = pairs + wl * M;
    int top = 0;
    for (int j = 1; j < M; ++j)
        if (row[j].x > row[top].x) top = j;
    TrigOut o;
    o.detector = det; o.bank = bank; o.tmpl = i; o.is_bank_max = (top == i);
    o.window = w0 + wl;
    o.sample = (w0 + wl) * W + __float_as_int(e.y);
    o.snr = sqrtf(e.x); o.phase = atan2f(e.w, e.z); o.re = e.z; o.im = e.w;
    o.xi2 = -1.f;      // no autocorrelation on this path
    o.pad = 0;
    out[pos] = o;
}

std::mutex g_mu;
void* g_ptr[64] = {};

}  // namespace

extern "C" LLOID_API lloid_status lloid_triggers_from_snr_noalloc(const float* z, int32_t n_templates, int64_t n,
                                                                  int64_t t0, int64_t window, float threshold,
                                                                  int32_t detector, int32_t bank, lloid_trigger* out,
                                                                  int64_t cap, int64_t* n_out, void* stream) {
    if (!z || !out || !n_out || n_templates < 1 || n <= 0 || window <= 0 || t0 < 0 || cap < 0 ||
        n % window || t0 % window || !(threshold >= 0.f))
        return LLOID_EINVAL;
    const long long n_win = n / window;
    const long long n_pairs = n_win * (long long)n_templates;
    if (n_pairs > kMaxPairs) return LLOID_ERANGE;   // beyond the compiled-in scratch: split the block
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return LLOID_ECUDA;
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return LLOID_ECUDA;
            g_ptr[dev] = p;
        }
        base = g_ptr[dev];
    }
    float4* pairs = static_cast<float4*>(base);
    int* counts = reinterpret_cast<int*>(static_cast<unsigned char*>(base) + kPairBytes);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int chunks = (int)((n_pairs + kChunk - 1) / kChunk);
    k_na_window_max<<<(unsigned)n_pairs, 256, 0, s>>>(z, n_templates, n, window, pairs);
    k_na_count<<<chunks, (int)kChunk, 0, s>>>(pairs, n_pairs, threshold, counts);
    k_na_scatter<<<chunks, (int)kChunk, 0, s>>>(pairs, n_pairs, n_templates, counts, threshold, detector, bank,
                                                t0 / window, window, reinterpret_cast<TrigOut*>(out), cap,
                                                reinterpret_cast<long long*>(n_out));
    static_assert(sizeof(TrigOut) == sizeof(lloid_trigger), "trigger layout");
    return cudaGetLastError() == cudaSuccess ? LLOID_OK : LLOID_ECUDA;
}
