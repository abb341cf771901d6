// PSD estimation and whitening (Section II.B.2) on the GPU.
//
// Per push of a detector: the new input samples go into a ring; every block
// whose segment is complete is processed, all blocks of the push at once:
//   k_wh_blocks   Hann-windowed segment between Z zeros (N samples), gap flag
//   k_wh_fwd      bins 0 .. N_out / 2 of the length-N real DFT of each segment
//   k_wh_psd      per bin, block after block: instantaneous PSD |X|^2 / sum w^2,
//                 median of the newest odd number (<= n_med) of them divided by
//                 kappa_k (a geometric-mean estimate), running log mean over up
//                 to n_avg blocks, PSD = G e^gamma, Y = X / sqrt(PSD) scaled
//   k_wh_inv      inverse real DFT of length N_out = N rate_out / rate_in (the
//                 bins below the output Nyquist are the downsampled spectrum)
//   k_wh_ola      Tukey taper and overlap-add; the first hop_out samples of
//                 each block are final
//
// The transforms are this file's own: a radix-2 decimation-in-time FFT of
// length N_out in shared memory (two stages per barrier, one CTA per transform,
// input in bit-reversed order, twiddles from a table computed on the host in
// double precision).
// The forward transform needs only the N_out / 2 + 1 lowest of the N / 2 + 1
// bins, so it splits the segment into its R = N / N_out polyphase components
// c_r[m] = b[R m + r]: X[k] = sum_r W_N^{k r} C_r[k], C_r the length-N_out DFT
// of c_r (decimation in time, kept only for k <= N_out / 2).  Two real
// sequences make one complex transform (x + i y); the inverse transforms two
// blocks at a time the same way.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lloid.h"

namespace {

constexpr int kMaxMed = 15;
constexpr int kMaxFftOut = 16384;     // N_out: one transform of float2 in shared memory (128 KB)
constexpr int kFftThreads = 1024;
constexpr double kEulerGamma = 0.57721566490153286060651209;

struct WhDet {
    float* ring = nullptr;           // input ring [r_in]
    long long wr = 0, rd = 0;        // samples written; start of the next segment (absolute)
    float* hist = nullptr;           // [n_med][K1] instantaneous PSDs
    float* logG = nullptr;           // [K1]
    float* acc = nullptr;            // overlap-add ring [r_acc]
    long long o = 0;                 // output samples produced so far
    int* state = nullptr;            // [2][3] head, count, n_est (double-buffered by parity)
    int parity = 0;
};

}  // namespace

struct lloid_whitener {
    lloid_whitener_config cfg{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    int N = 0, Z = 0, L = 0, hop = 0, N_out = 0, Z_out = 0, hop_out = 0, K1 = 0, nb_max = 0;
    long long r_in = 0, r_acc = 0;
    double W2 = 0.0;
    float* win = nullptr;            // Hann [L]
    float* tuk = nullptr;            // Tukey [N_out]
    float* kappa = nullptr;          // [kMaxMed + 1], odd entries used
    int bits = 0, n_pairs = 0;       // log2 N_out; polyphase pairs per segment, ceil(R / 2)
    float2* tw = nullptr;            // [N_out / 2] exp(-2 pi i j / N_out)
    float* b = nullptr;              // [nb_max][N]
    float2* X = nullptr;             // [nb_max][n_pairs][K1] per-pair parts of the low bins
    float2* Y = nullptr;             // [nb_max][K1]
    float* y = nullptr;              // [nb_max][N_out]
    int* gap = nullptr;              // [nb_max]
    float* stage_in = nullptr;       // [max_push]
    float* stage_out = nullptr;      // [nb_max * hop_out]
    std::vector<WhDet> det;
};

namespace {

lloid_status wfail(lloid_whitener* w, lloid_status st, const char* fmt, ...) {
    if (w) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        w->err = buf;
    }
    return st;
}

#define WCK(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return wfail(w, e_ == cudaErrorMemoryAllocation ? LLOID_ENOMEM : LLOID_ECUDA,  \
                         "%s (%s:%d)", cudaGetErrorString(e_), __FILE__, __LINE__);        \
    } while (0)

bool pow2(long long x) { return x > 0 && (x & (x - 1)) == 0; }
long long next_pow2(long long x) {
    long long p = 1;
    while (p < x) p <<= 1;
    return p;
}

// kappa_k = exp(E[log M] + gamma), M the median of k (odd) unit exponentials:
// M has density c (1 - e^-x)^m e^-(m+1)x with m = (k - 1)/2, c = k!/(m!)^2;
// expanding the binomial and integrating log(x) e^-ax (= -(gamma + log a)/a)
// term by term gives E[log M] = -c sum_j C(m, j) (-1)^j (gamma + log(m + 1 + j)) / (m + 1 + j).
double kappa_of(int k) {
    const int m = (k - 1) / 2;
    long double c = 1.0L;
    for (int i = m + 1; i <= k; ++i) c *= i;     // k! / m!
    for (int i = 2; i <= m; ++i) c /= i;         // / m!
    long double e = 0.0L, binom = 1.0L;
    for (int j = 0; j <= m; ++j) {
        const long double a = m + 1 + j;
        const long double term = c * binom * ((j & 1) ? -1.0L : 1.0L) * (kEulerGamma + std::log(a)) / a;
        e -= term;
        binom = binom * (m - j) / (j + 1);
    }
    return std::exp((double)e + kEulerGamma);
}

__global__ void k_wh_ingest(const float* __restrict__ in, long long n, float* __restrict__ ring, long long mask,
                            long long wr) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        ring[(wr + i) & mask] = in[i];
}

// b[blk][n]: the Hann-windowed segment of block blk between Z zeros; gap[blk] |= 1
// for a non-finite input sample.
__global__ void k_wh_blocks(const float* __restrict__ ring, long long mask, long long rd0, int hop, int L, int Z, int N,
                            const float* __restrict__ win, float* __restrict__ b, int* __restrict__ gap) {
    const int blk = blockIdx.y;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
        float v = 0.f;
        if (n >= Z && n < Z + L) {
            const float x = ring[(rd0 + (long long)blk * hop + n - Z) & mask];
            if (!isfinite(x)) atomicOr(gap + blk, 1);
            v = win[n - Z] * x;
        }
        b[(size_t)blk * N + n] = v;
    }
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// In-place radix-2 decimation-in-time DFT, sum_m s[m] e^{-2 pi i k m / n}, of the n
// (a power of two) values in shared memory, stored in bit-reversed order; the result
// is in natural order.  tw[j] = e^{-2 pi i j / n}, j < n / 2.  Two radix-2 stages (half
// and 2 half) are taken per barrier: a thread owns the four points i, i + half,
// i + 2 half, i + 3 half of both; a last single stage when log2 n is odd.  All threads
// of the CTA call it after the stores of s have been made visible (__syncthreads) and
// leave it after a barrier.
__device__ void wh_fft_smem(float2* s, int n, const float2* __restrict__ tw) {
    int half = 1;
    for (; 4 * half <= n; half <<= 2) {
        const int ta = n / (2 * half), tb = n / (4 * half);
        for (int j = threadIdx.x; j < n / 4; j += blockDim.x) {
            const int pos = j & (half - 1);
            const int i0 = ((j - pos) << 2) + pos;
            float2 e0 = s[i0], e1 = s[i0 + half], e2 = s[i0 + 2 * half], e3 = s[i0 + 3 * half];
            const float2 wa = tw[pos * ta];
            float2 t = cmul(wa, e1);
            e1 = make_float2(e0.x - t.x, e0.y - t.y);
            e0 = make_float2(e0.x + t.x, e0.y + t.y);
            t = cmul(wa, e3);
            e3 = make_float2(e2.x - t.x, e2.y - t.y);
            e2 = make_float2(e2.x + t.x, e2.y + t.y);
            t = cmul(tw[pos * tb], e2);
            s[i0 + 2 * half] = make_float2(e0.x - t.x, e0.y - t.y);
            s[i0] = make_float2(e0.x + t.x, e0.y + t.y);
            t = cmul(tw[(pos + half) * tb], e3);
            s[i0 + 3 * half] = make_float2(e1.x - t.x, e1.y - t.y);
            s[i0 + half] = make_float2(e1.x + t.x, e1.y + t.y);
        }
        __syncthreads();
    }
    if (half < n) {
        const int ta = n / (2 * half);
        for (int j = threadIdx.x; j < n / 2; j += blockDim.x) {
            const int pos = j & (half - 1);
            const int i0 = ((j - pos) << 1) + pos, i1 = i0 + half;
            const float2 u = s[i0];
            const float2 t = cmul(tw[pos * ta], s[i1]);
            s[i0] = make_float2(u.x + t.x, u.y + t.y);
            s[i1] = make_float2(u.x - t.x, u.y - t.y);
        }
        __syncthreads();
    }
}

// X[blk][p][k], k <= n_out / 2: polyphase pair p's part of bin k of the length-N real
// DFT of segment blk: W_N^{k r0} C_r0[k] + W_N^{k r1} C_r1[k] with r0 = 2p, r1 = 2p + 1
// (absent when r1 = R), C_r the length-n_out DFT of c_r[m] = b[R m + r].  The pair is
// one complex transform Z of z = c_r0 + i c_r1: C_r0[k] = (Z[k] + conj Z[-k]) / 2 and
// C_r1[k] = (Z[k] - conj Z[-k]) / 2i.  Grid (segments, pairs), kFftThreads threads,
// n_out float2 of dynamic shared memory.
__global__ void __launch_bounds__(kFftThreads) k_wh_fwd(const float* __restrict__ b, int N, int R, int n_out, int bits,
                                                        const float2* __restrict__ tw, float2* __restrict__ X) {
    extern __shared__ float2 s_fft[];
    const int blk = blockIdx.x, p = blockIdx.y, n_pairs = gridDim.y;
    const int K1 = n_out / 2 + 1;
    const int r0 = 2 * p, r1 = 2 * p + 1;
    const float* bb = b + (size_t)blk * N;
    for (int m = threadIdx.x; m < n_out; m += blockDim.x) {
        const float re = bb[(size_t)R * m + r0];
        const float im = r1 < R ? bb[(size_t)R * m + r1] : 0.f;
        s_fft[__brev((unsigned)m) >> (32 - bits)] = make_float2(re, im);
    }
    __syncthreads();
    wh_fft_smem(s_fft, n_out, tw);
    float2* Xp = X + ((size_t)blk * n_pairs + p) * K1;
    const float ang = -2.0f / (float)N;   // exact: N is a power of two
    for (int k = threadIdx.x; k < K1; k += blockDim.x) {
        const float2 a = s_fft[k], q = s_fft[(n_out - k) & (n_out - 1)];
        const float2 c0 = make_float2(0.5f * (a.x + q.x), 0.5f * (a.y - q.y));
        const float2 c1 = make_float2(0.5f * (a.y + q.y), -0.5f * (a.x - q.x));
        float sn, cs;
        sincospif(ang * (float)(((long long)k * r0) & (N - 1)), &sn, &cs);
        float2 acc = make_float2(cs * c0.x - sn * c0.y, cs * c0.y + sn * c0.x);
        if (r1 < R) {
            sincospif(ang * (float)(((long long)k * r1) & (N - 1)), &sn, &cs);
            acc.x += cs * c1.x - sn * c1.y;
            acc.y += cs * c1.y + sn * c1.x;
        }
        Xp[k] = acc;
    }
}

// y[blk][n] = sum_k V[k] e^{+2 pi i k n / n_out} (unnormalised), V the Hermitian
// extension of Y[blk][0 .. n_out / 2] with the imaginary parts of bins 0 and n_out / 2
// dropped: the inverse real DFT.  Segments 2g and 2g + 1 are one complex transform of
// W = V_2g + i V_2g+1, whose inverse has real part y_2g and imaginary part y_2g+1; it is
// computed as conj(DFT(conj W)).  Grid ceil(nb / 2), kFftThreads threads, n_out float2
// of dynamic shared memory.
__global__ void __launch_bounds__(kFftThreads) k_wh_inv(const float2* __restrict__ Y, int nb, int n_out, int bits,
                                                        const float2* __restrict__ tw, float* __restrict__ y) {
    extern __shared__ float2 s_fft[];
    const int b1 = 2 * blockIdx.x, b2 = b1 + 1;
    const bool two = b2 < nb;
    const int K1 = n_out / 2 + 1, h = n_out / 2;
    const float2* Y1 = Y + (size_t)b1 * K1;
    const float2* Y2 = Y + (size_t)b2 * K1;
    for (int k = threadIdx.x; k < n_out; k += blockDim.x) {
        const int kk = k <= h ? k : n_out - k;
        float2 v1 = Y1[kk];
        float2 v2 = two ? Y2[kk] : make_float2(0.f, 0.f);
        if (kk == 0 || kk == h) { v1.y = 0.f; v2.y = 0.f; }
        if (k > h) { v1.y = -v1.y; v2.y = -v2.y; }          // V[k] = conj Y[n_out - k]
        s_fft[__brev((unsigned)k) >> (32 - bits)] = make_float2(v1.x - v2.y, -(v1.y + v2.x));
    }
    __syncthreads();
    wh_fft_smem(s_fft, n_out, tw);
    for (int n = threadIdx.x; n < n_out; n += blockDim.x) {
        const float2 r = s_fft[n];
        y[(size_t)b1 * n_out + n] = r.x;
        if (two) y[(size_t)b2 * n_out + n] = -r.y;
    }
}

// One thread per output bin k, the blocks in order (every thread replays the same
// history bookkeeping, so the shared counters stay consistent).  The bin's history
// and running log mean are read once, carried through the blocks in registers and
// local memory, and written back at the end.  kPsdThreads per CTA, so that the K1
// bins spread over many SMs.
constexpr int kPsdThreads = 64;
__global__ void __launch_bounds__(kPsdThreads) k_wh_psd(const float2* __restrict__ X, int nb, int n_pairs, int K1,
                         const int* __restrict__ gap, float* __restrict__ hist, int n_med, float* __restrict__ logG,
                         int n_avg, const int* __restrict__ st_in, int* __restrict__ st_out, float inv_w2, float scale,
                         const float* __restrict__ kappa, float2* __restrict__ Y) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    int head = st_in[0], cnt = st_in[1], nest = st_in[2];
    const bool own = k < K1;
    float hv[kMaxMed];                 // hist[s][k], s < n_med
    float g = 0.f;                     // logG[k]
    if (own) {
        for (int i = 0; i < n_med; ++i) hv[i] = hist[(size_t)i * K1 + k];
        g = logG[k];
    }
    for (int blk = 0; blk < nb; ++blk) {
        if (gap[blk]) {
            if (own) Y[(size_t)blk * K1 + k] = make_float2(0.f, 0.f);
            continue;
        }
        cnt = min(cnt + 1, n_med);
        ++nest;
        const int slot = head;
        head = (head + 1) % n_med;
        if (!own) continue;
        float2 x = make_float2(0.f, 0.f);   // the pairs' parts of bin k
        for (int p = 0; p < n_pairs; ++p) {
            const float2 xp = X[((size_t)blk * n_pairs + p) * K1 + k];
            x.x += xp.x;
            x.y += xp.y;
        }
        hv[slot] = (x.x * x.x + x.y * x.y) * inv_w2;
        const int kk = (cnt & 1) ? cnt : cnt - 1;
        float v[kMaxMed];
        for (int i = 0; i < kk; ++i) {
            const int s = ((slot - i) % n_med + n_med) % n_med;      // the newest kk estimates
            const float e = hv[s];
            int j = i;
            while (j > 0 && v[j - 1] > e) { v[j] = v[j - 1]; --j; }
            v[j] = e;
        }
        const float lg = logf(v[kk / 2] / kappa[kk]);
        g = (nest == 1) ? lg : g + (lg - g) / (float)min(nest, n_avg);
        const float s = scale * rsqrtf(expf(g + (float)kEulerGamma));
        Y[(size_t)blk * K1 + k] = make_float2(x.x * s, x.y * s);
    }
    if (own) {
        for (int i = 0; i < n_med; ++i) hist[(size_t)i * K1 + k] = hv[i];
        logG[k] = g;
    }
    if (k == 0) { st_out[0] = head; st_out[1] = cnt; st_out[2] = nest; }
}

// Overlap-add of nb Tukey-tapered blocks starting at output position o0 (block blk
// at o0 + blk hop_out); positions below o0 + nb hop_out are final.
__global__ void k_wh_ola(const float* __restrict__ y, int nb, int N_out, int hop_out, const float* __restrict__ tuk,
                         float* __restrict__ acc, long long mask, long long o0, float* __restrict__ out) {
    const int span = (nb - 1) * hop_out + N_out;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < span; p += gridDim.x * blockDim.x) {
        const long long P = (o0 + p) & mask;
        float v = acc[P];
        const int b_lo = p >= N_out ? (p - N_out) / hop_out + 1 : 0;
        const int b_hi = min(nb - 1, p / hop_out);
        for (int blk = b_lo; blk <= b_hi; ++blk) {
            const int m = p - blk * hop_out;
            if (m >= 0 && m < N_out) v = fmaf(tuk[m], y[(size_t)blk * N_out + m], v);
        }
        if (p < nb * hop_out) {
            out[p] = v;
            acc[P] = 0.f;
        } else {
            acc[P] = v;
        }
    }
}

}  // namespace

extern "C" {

void lloid_whitener_config_default(lloid_whitener_config* c) {
    if (!c) return;
    std::memset(c, 0, sizeof *c);
    c->rate_in = 16384;
    c->rate_out = 2048;
    c->n_fft = 4 * 16384;
    c->z_pad = 16384;
    c->n_med = 7;
    c->n_avg = 64;
    c->n_detectors = 1;
    c->device = 0;
    c->max_push = 16LL * 16384;
    c->cuda_stream = nullptr;
}

lloid_status lloid_whitener_create(const lloid_whitener_config* cfg, lloid_whitener** out) {
    if (!cfg || !out) return LLOID_EINVAL;
    *out = nullptr;
    const lloid_whitener_config& c = *cfg;
    if (!pow2(c.rate_in) || !pow2(c.rate_out) || c.rate_out > c.rate_in || !pow2(c.n_fft) || c.z_pad < 0 ||
        2LL * c.z_pad >= c.n_fft || c.n_med < 1 || c.n_med > kMaxMed || !(c.n_med & 1) || c.n_avg < 1 ||
        c.n_detectors < 1 || c.n_detectors > 64 || c.max_push <= 0)
        return LLOID_EINVAL;
    const int ratio = c.rate_in / c.rate_out;
    const int hop = c.n_fft / 2 - c.z_pad;
    if (c.n_fft % ratio || c.z_pad % ratio || hop % ratio || c.max_push % hop || c.n_fft / ratio < 4 ||
        c.n_fft / ratio > kMaxFftOut || c.n_fft > (1 << 24) || ratio > 4096)
        return LLOID_EINVAL;
    lloid_whitener* w = new lloid_whitener();
    w->cfg = c;
    w->N = c.n_fft; w->Z = c.z_pad; w->L = c.n_fft - 2 * c.z_pad; w->hop = hop;
    w->N_out = c.n_fft / ratio; w->Z_out = c.z_pad / ratio; w->hop_out = hop / ratio; w->K1 = w->N_out / 2 + 1;
    w->nb_max = (int)(c.max_push / hop);
    while ((1 << w->bits) < w->N_out) ++w->bits;
    w->n_pairs = (ratio + 1) / 2;
    w->r_in = next_pow2(w->L + c.max_push + hop);
    w->r_acc = next_pow2((long long)(w->nb_max - 1) * w->hop_out + w->N_out + w->hop_out);
    auto bail = [&](lloid_status st) { lloid_whitener_destroy(w); return st; };
    if (cudaSetDevice(c.device) != cudaSuccess) return bail(LLOID_ECUDA);
    if (c.cuda_stream) w->stream = (cudaStream_t)c.cuda_stream;
    else if (cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(LLOID_ECUDA);
    else w->own_stream = true;
    // windows and constants (host, double), then uploaded as FP32
    std::vector<float> hw(w->L), tk(w->N_out, 1.f), kp(kMaxMed + 1, 1.f);
    double w2 = 0.0;
    for (int n = 0; n < w->L; ++n) {
        const double s = std::sin(M_PI * n / w->L);
        hw[n] = (float)(s * s);
        w2 += (s * s) * (s * s);
    }
    w->W2 = w2;
    for (int t = 0; t < w->Z_out; ++t) {
        const double r = 0.5 * (1.0 - std::cos(M_PI * (t + 0.5) / w->Z_out));
        tk[t] = (float)r;
        tk[w->N_out - 1 - t] = (float)r;
    }
    for (int k = 1; k <= kMaxMed; k += 2) kp[k] = (float)kappa_of(k);
    std::vector<float2> twh(w->N_out / 2);
    for (int j = 0; j < w->N_out / 2; ++j) {
        const double a = 2.0 * M_PI * j / w->N_out;
        twh[j] = make_float2((float)std::cos(a), (float)-std::sin(a));
    }
    const int nd = c.n_detectors, nb = w->nb_max;
    bool ok = cudaMalloc(&w->win, w->L * 4) == cudaSuccess && cudaMalloc(&w->tuk, w->N_out * 4) == cudaSuccess &&
              cudaMalloc(&w->kappa, (kMaxMed + 1) * 4) == cudaSuccess &&
              cudaMalloc(&w->b, (size_t)nb * w->N * 4) == cudaSuccess &&
              cudaMalloc(&w->tw, (size_t)(w->N_out / 2) * sizeof(float2)) == cudaSuccess &&
              cudaMalloc(&w->X, (size_t)nb * w->n_pairs * w->K1 * sizeof(float2)) == cudaSuccess &&
              cudaMalloc(&w->Y, (size_t)nb * w->K1 * sizeof(float2)) == cudaSuccess &&
              cudaMalloc(&w->y, (size_t)nb * w->N_out * 4) == cudaSuccess &&
              cudaMalloc(&w->gap, nb * 4) == cudaSuccess &&
              cudaMalloc(&w->stage_in, c.max_push * 4) == cudaSuccess &&
              cudaMalloc(&w->stage_out, (size_t)nb * w->hop_out * 4) == cudaSuccess;
    if (!ok) return bail(LLOID_ENOMEM);
    cudaMemcpy(w->win, hw.data(), w->L * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(w->tuk, tk.data(), w->N_out * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(w->kappa, kp.data(), (kMaxMed + 1) * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(w->tw, twh.data(), twh.size() * sizeof(float2), cudaMemcpyHostToDevice);
    const int fft_smem = w->N_out * (int)sizeof(float2);
    if (cudaFuncSetAttribute(k_wh_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, fft_smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_wh_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, fft_smem) != cudaSuccess)
        return bail(LLOID_ECUDA);
    w->det.resize(nd);
    for (auto& d : w->det) {
        ok = cudaMalloc(&d.ring, w->r_in * 4) == cudaSuccess &&
             cudaMalloc(&d.hist, (size_t)c.n_med * w->K1 * 4) == cudaSuccess &&
             cudaMalloc(&d.logG, w->K1 * 4) == cudaSuccess && cudaMalloc(&d.acc, w->r_acc * 4) == cudaSuccess &&
             cudaMalloc(&d.state, 6 * sizeof(int)) == cudaSuccess;
        if (!ok) return bail(LLOID_ENOMEM);
        cudaMemset(d.ring, 0, w->r_in * 4);
        cudaMemset(d.hist, 0, (size_t)c.n_med * w->K1 * 4);
        cudaMemset(d.logG, 0, w->K1 * 4);
        cudaMemset(d.acc, 0, w->r_acc * 4);
        cudaMemset(d.state, 0, 6 * sizeof(int));
    }
    if (cudaDeviceSynchronize() != cudaSuccess) return bail(LLOID_ECUDA);
    *out = w;
    return LLOID_OK;
}

void lloid_whitener_destroy(lloid_whitener* w) {
    if (!w) return;
    cudaSetDevice(w->cfg.device);
    if (w->stream) cudaStreamSynchronize(w->stream);
    for (auto& d : w->det) { cudaFree(d.ring); cudaFree(d.hist); cudaFree(d.logG); cudaFree(d.acc); cudaFree(d.state); }
    cudaFree(w->win); cudaFree(w->tuk); cudaFree(w->kappa); cudaFree(w->tw); cudaFree(w->b); cudaFree(w->X); cudaFree(w->Y);
    cudaFree(w->y); cudaFree(w->gap); cudaFree(w->stage_in); cudaFree(w->stage_out);
    if (w->own_stream && w->stream) cudaStreamDestroy(w->stream);
    delete w;
}

lloid_status lloid_whiten(lloid_whitener* w, int32_t det, const float* in, int64_t n, int in_is_device, float* out,
                          int64_t cap, int64_t* n_out, int out_is_device) {
    if (!w) return LLOID_EINVAL;
    if (!n_out || det < 0 || det >= w->cfg.n_detectors || n < 0 || n % w->hop || n > w->cfg.max_push ||
        (n > 0 && !in))
        return wfail(w, LLOID_EINVAL, "bad arguments (n must be a multiple of %d and <= max_push)", w->hop);
    *n_out = 0;
    WCK(cudaSetDevice(w->cfg.device));
    WhDet& d = w->det[det];
    const long long mask = w->r_in - 1;
    // a0': input into the ring
    if (n > 0) {
        const float* src = in;
        if (!in_is_device) {
            WCK(cudaMemcpyAsync(w->stage_in, in, n * 4, cudaMemcpyHostToDevice, w->stream));
            src = w->stage_in;
        }
        k_wh_ingest<<<(unsigned)std::min<long long>((n + 255) / 256, 1024), 256, 0, w->stream>>>(src, n, d.ring, mask,
                                                                                                 d.wr);
        WCK(cudaGetLastError());
        d.wr += n;
    }
    int nb = 0;
    while (d.rd + (long long)(nb + 1) * w->hop - w->hop + w->L <= d.wr) ++nb;   // complete segments
    nb = std::min(nb, w->nb_max);
    if (nb == 0) return LLOID_OK;
    const long long produced = (long long)nb * w->hop_out;
    if (cap < produced || !out) return wfail(w, LLOID_ERANGE, "output needs %lld samples", produced);
    WCK(cudaMemsetAsync(w->gap, 0, nb * 4, w->stream));
    k_wh_blocks<<<dim3((w->N + 255) / 256, nb), 256, 0, w->stream>>>(d.ring, mask, d.rd, w->hop, w->L, w->Z, w->N,
                                                                      w->win, w->b, w->gap);
    WCK(cudaGetLastError());
    const size_t fft_smem = (size_t)w->N_out * sizeof(float2);
    k_wh_fwd<<<dim3(nb, w->n_pairs), kFftThreads, fft_smem, w->stream>>>(w->b, w->N, w->N / w->N_out, w->N_out,
                                                                          w->bits, w->tw, w->X);
    WCK(cudaGetLastError());
    const float scale = (float)(std::sqrt((double)w->N_out / w->N) / w->N_out);
    k_wh_psd<<<(w->K1 + kPsdThreads - 1) / kPsdThreads, kPsdThreads, 0, w->stream>>>(w->X, nb, w->n_pairs, w->K1, w->gap, d.hist,
                                                         w->cfg.n_med, d.logG, w->cfg.n_avg, d.state + 3 * d.parity,
                                                         d.state + 3 * (1 - d.parity), (float)(1.0 / w->W2), scale,
                                                         w->kappa, w->Y);
    WCK(cudaGetLastError());
    d.parity ^= 1;
    k_wh_inv<<<(nb + 1) / 2, kFftThreads, fft_smem, w->stream>>>(w->Y, nb, w->N_out, w->bits, w->tw, w->y);
    WCK(cudaGetLastError());
    float* dst = out_is_device ? out : w->stage_out;
    const int span = (nb - 1) * w->hop_out + w->N_out;
    k_wh_ola<<<(span + 255) / 256, 256, 0, w->stream>>>(w->y, nb, w->N_out, w->hop_out, w->tuk, d.acc, w->r_acc - 1,
                                                        d.o, dst);
    WCK(cudaGetLastError());
    if (!out_is_device) {
        WCK(cudaMemcpyAsync(out, w->stage_out, produced * 4, cudaMemcpyDeviceToHost, w->stream));
        WCK(cudaStreamSynchronize(w->stream));
    }
    d.rd += (long long)nb * w->hop;
    d.o += produced;
    *n_out = produced;
    return LLOID_OK;
}

lloid_status lloid_whitener_psd(lloid_whitener* w, int32_t det, float* out, int64_t cap) {
    if (!w) return LLOID_EINVAL;
    if (det < 0 || det >= w->cfg.n_detectors || !out) return wfail(w, LLOID_EINVAL, "bad arguments");
    if (cap < w->K1) return wfail(w, LLOID_ERANGE, "need %d bins", w->K1);
    std::vector<float> lg(w->K1);
    WCK(cudaMemcpyAsync(lg.data(), w->det[det].logG, w->K1 * 4, cudaMemcpyDeviceToHost, w->stream));
    WCK(cudaStreamSynchronize(w->stream));
    for (int k = 0; k < w->K1; ++k) out[k] = (float)std::exp((double)lg[k] + kEulerGamma);
    return LLOID_OK;
}

}  // extern "C"
