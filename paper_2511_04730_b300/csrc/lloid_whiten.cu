// PSD estimation and whitening (Section II.B.2) on the GPU.
//
// Per push of a detector: the new input samples go into a ring; every block
// whose segment is complete is processed, all blocks of the push at once:
//   k_wh_blocks   Hann-windowed segment between Z zeros (N samples), gap flag
//   cuFFT R2C     (N)
//   k_wh_psd      per bin, block after block: instantaneous PSD |X|^2 / sum w^2,
//                 median of the newest odd number (<= n_med) of them divided by
//                 kappa_k (a geometric-mean estimate), running log mean over up
//                 to n_avg blocks, PSD = G e^gamma, Y = X / sqrt(PSD) scaled
//   cuFFT C2R     (N_out = N rate_out / rate_in: the bins below the output
//                 Nyquist are the downsampled spectrum)
//   k_wh_ola      Tukey taper and overlap-add; the first hop_out samples of
//                 each block are final
// The transforms are plain cuFFT calls; everything else is in this file.
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/lloid.h"

namespace {

constexpr int kMaxMed = 15;
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
    float* b = nullptr;              // [nb_max][N]
    cufftComplex* X = nullptr;       // [nb_max][N/2 + 1]
    cufftComplex* Y = nullptr;       // [nb_max][K1]
    float* y = nullptr;              // [nb_max][N_out]
    int* gap = nullptr;              // [nb_max]
    float* stage_in = nullptr;       // [max_push]
    float* stage_out = nullptr;      // [nb_max * hop_out]
    std::map<int, std::pair<cufftHandle, cufftHandle>> plans;   // blocks -> (R2C, C2R)
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
#define WFFT(call)                                                                         \
    do {                                                                                   \
        cufftResult r_ = (call);                                                           \
        if (r_ != CUFFT_SUCCESS) return wfail(w, LLOID_ECUDA, "cuFFT error %d (%s:%d)", (int)r_, __FILE__, __LINE__); \
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

// One thread per output bin k, the blocks in order (every thread replays the same
// history bookkeeping, so the shared counters stay consistent).
__global__ void k_wh_psd(const cufftComplex* __restrict__ X, int nb, int xs, int K1, const int* __restrict__ gap,
                         float* __restrict__ hist, int n_med, float* __restrict__ logG, int n_avg,
                         const int* __restrict__ st_in, int* __restrict__ st_out, float inv_w2, float scale,
                         const float* __restrict__ kappa, cufftComplex* __restrict__ Y) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    int head = st_in[0], cnt = st_in[1], nest = st_in[2];
    for (int blk = 0; blk < nb; ++blk) {
        if (gap[blk]) {
            if (k < K1) Y[(size_t)blk * K1 + k] = make_cuFloatComplex(0.f, 0.f);
            continue;
        }
        cnt = min(cnt + 1, n_med);
        ++nest;
        const int slot = head;
        head = (head + 1) % n_med;
        if (k >= K1) continue;
        const cufftComplex x = X[(size_t)blk * xs + k];
        hist[(size_t)slot * K1 + k] = (x.x * x.x + x.y * x.y) * inv_w2;
        const int kk = (cnt & 1) ? cnt : cnt - 1;
        float v[kMaxMed];
        for (int i = 0; i < kk; ++i) {
            const int s = ((slot - i) % n_med + n_med) % n_med;      // the newest kk estimates
            const float e = hist[(size_t)s * K1 + k];
            int j = i;
            while (j > 0 && v[j - 1] > e) { v[j] = v[j - 1]; --j; }
            v[j] = e;
        }
        const float lg = logf(v[kk / 2] / kappa[kk]);
        const float prev = logG[k];
        const float cur = (nest == 1) ? lg : prev + (lg - prev) / (float)min(nest, n_avg);
        logG[k] = cur;
        const float s = scale * rsqrtf(expf(cur + (float)kEulerGamma));
        Y[(size_t)blk * K1 + k] = make_cuFloatComplex(x.x * s, x.y * s);
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

lloid_status get_plans(lloid_whitener* w, int nb, cufftHandle* r2c, cufftHandle* c2r) {
    auto it = w->plans.find(nb);
    if (it == w->plans.end()) {
        cufftHandle a, c;
        WFFT(cufftPlan1d(&a, w->N, CUFFT_R2C, nb));
        WFFT(cufftPlan1d(&c, w->N_out, CUFFT_C2R, nb));
        WFFT(cufftSetStream(a, w->stream));
        WFFT(cufftSetStream(c, w->stream));
        it = w->plans.emplace(nb, std::make_pair(a, c)).first;
    }
    *r2c = it->second.first;
    *c2r = it->second.second;
    return LLOID_OK;
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
    if (c.n_fft % ratio || c.z_pad % ratio || hop % ratio || c.max_push % hop || c.n_fft / ratio < 4) return LLOID_EINVAL;
    lloid_whitener* w = new lloid_whitener();
    w->cfg = c;
    w->N = c.n_fft; w->Z = c.z_pad; w->L = c.n_fft - 2 * c.z_pad; w->hop = hop;
    w->N_out = c.n_fft / ratio; w->Z_out = c.z_pad / ratio; w->hop_out = hop / ratio; w->K1 = w->N_out / 2 + 1;
    w->nb_max = (int)(c.max_push / hop);
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
    const int nd = c.n_detectors, nb = w->nb_max;
    bool ok = cudaMalloc(&w->win, w->L * 4) == cudaSuccess && cudaMalloc(&w->tuk, w->N_out * 4) == cudaSuccess &&
              cudaMalloc(&w->kappa, (kMaxMed + 1) * 4) == cudaSuccess &&
              cudaMalloc(&w->b, (size_t)nb * w->N * 4) == cudaSuccess &&
              cudaMalloc(&w->X, (size_t)nb * (w->N / 2 + 1) * sizeof(cufftComplex)) == cudaSuccess &&
              cudaMalloc(&w->Y, (size_t)nb * w->K1 * sizeof(cufftComplex)) == cudaSuccess &&
              cudaMalloc(&w->y, (size_t)nb * w->N_out * 4) == cudaSuccess &&
              cudaMalloc(&w->gap, nb * 4) == cudaSuccess &&
              cudaMalloc(&w->stage_in, c.max_push * 4) == cudaSuccess &&
              cudaMalloc(&w->stage_out, (size_t)nb * w->hop_out * 4) == cudaSuccess;
    if (!ok) return bail(LLOID_ENOMEM);
    cudaMemcpy(w->win, hw.data(), w->L * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(w->tuk, tk.data(), w->N_out * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(w->kappa, kp.data(), (kMaxMed + 1) * 4, cudaMemcpyHostToDevice);
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
    for (auto& kv : w->plans) { cufftDestroy(kv.second.first); cufftDestroy(kv.second.second); }
    for (auto& d : w->det) { cudaFree(d.ring); cudaFree(d.hist); cudaFree(d.logG); cudaFree(d.acc); cudaFree(d.state); }
    cudaFree(w->win); cudaFree(w->tuk); cudaFree(w->kappa); cudaFree(w->b); cudaFree(w->X); cudaFree(w->Y);
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
    cufftHandle r2c, c2r;
    lloid_status st;
    if ((st = get_plans(w, nb, &r2c, &c2r))) return st;
    WCK(cudaMemsetAsync(w->gap, 0, nb * 4, w->stream));
    k_wh_blocks<<<dim3((w->N + 255) / 256, nb), 256, 0, w->stream>>>(d.ring, mask, d.rd, w->hop, w->L, w->Z, w->N,
                                                                      w->win, w->b, w->gap);
    WCK(cudaGetLastError());
    WFFT(cufftExecR2C(r2c, w->b, w->X));
    const float scale = (float)(std::sqrt((double)w->N_out / w->N) / w->N_out);
    k_wh_psd<<<(w->K1 + 255) / 256, 256, 0, w->stream>>>(w->X, nb, w->N / 2 + 1, w->K1, w->gap, d.hist,
                                                         w->cfg.n_med, d.logG, w->cfg.n_avg, d.state + 3 * d.parity,
                                                         d.state + 3 * (1 - d.parity), (float)(1.0 / w->W2), scale,
                                                         w->kappa, w->Y);
    WCK(cudaGetLastError());
    d.parity ^= 1;
    WFFT(cufftExecC2R(c2r, w->Y, w->y));
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
