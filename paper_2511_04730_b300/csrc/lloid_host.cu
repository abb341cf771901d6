// Host side of the LLOID C ABI: context, bank registry, streaming state and
// the per-push launch sequence.  Every arithmetic step of the hot path runs in
// the kernels; the host validates, lays out, and enqueues.
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <queue>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "../../include/lloid.h"
#include "kernels_simt.cuh"
#include "kernels_tc.cuh"
#include "kernels_tc2.cuh"
#include "kernels_f0.cuh"

using namespace lloid;

namespace {

constexpr int kWindowRing = 16;      // retained trigger windows (slab ring)

long long next_pow2(long long x) {
    long long p = 1;
    while (p < x) p <<= 1;
    return p;
}
bool is_pow2(long long x) { return x > 0 && (x & (x - 1)) == 0; }

// Eq. 4: sinc of zero spacing f windowed by a sinc of half length c, g[c] = 1.
std::vector<double> sinc_windowed(int f, int c) {
    std::vector<double> g(2 * c + 1);
    const double pi = 3.14159265358979323846;
    for (int k = 0; k <= 2 * c; ++k) {
        int x = k - c;
        if (x == 0) { g[k] = 1.0; continue; }
        double a = pi * x / f, b = pi * x / c;
        g[k] = std::sin(a) / a * std::sin(b) / b;
    }
    return g;
}

struct SliceRT {
    int rate = 0, D = 1, N = 0, L = 0;
    long long J = 0;
    int row0 = 0;                // first Yhat row of the slice within the bank
    int e_min = 0, e_max = 0;    // support of the composed upsampler (full-rate offsets)
    float* d_bases = nullptr;
    float* d_R = nullptr;        // composed upsampler (FP32 path; split path in the f0 form)
    float* d_yring = nullptr;    // [n_det][L][y_len]
    int y_len = 0;
    int tcol = 0;                // split path, f0 form: first column of the slice in the f0 operand ring
    std::vector<double> R;       // composed upsampler (host copy)
};

// Split-precision (tensor-core) path: one ladder level per distinct rate of
// the bank plus f0, lowest first.
struct LevelRT {
    int rate = 0, D = 1, Lambda = 0;   // Lambda: look-ahead of this level (full-rate samples)
    int K = 0, Kp = 0;                 // bases at this rate (16-aligned per slice), padded to 64
    void *d_cre = nullptr, *d_cim = nullptr, *d_cre_lo = nullptr, *d_cim_lo = nullptr;  // [Mpad][Kp]
    uint16_t *d_yhi = nullptr, *d_ylo = nullptr;   // operand ring [n_det][2R][Kp]
    int R = 0;
    uint16_t* d_accp = nullptr;        // below the top: hi/lo planes [n_det][4][acc_cols / 8][Mpad][8]
    int acc_cols = 0;
};
struct FirSliceRT {
    int level = 0, col = 0, Np = 0, Kp = 0, Mtiles = 0;
    void *d_a = nullptr, *d_a_lo = nullptr;   // 8-phase expanded bases [Mtiles*128][Kp]
};

struct BankRT {
    int id = 0, M = 0, Mpad = 0, K = 0, Kpad = 0, tmpl0 = 0;
    int form = 0;                      // split path: 0 = per-rate ladder, 1 = f0 form
    std::vector<SliceRT> sl;
    std::vector<LevelRT> lev;          // split path
    LevelRT top;                       // split path, f0 form: K = the bank's bases packed, rounded up to 16
    uint16_t* d_cblk = nullptr;        // f0 form: coefficient planes [re hi, im hi, (re lo, im lo)][K/8][Mpad][8]
    uint16_t* d_yf0 = nullptr;         // f0 form: Yhat of the current push [det][hi, lo][K/8][max_block][8]
    std::vector<FirSliceRT> fs;        // split path, parallel to sl
    void* d_cre = nullptr;       // [Mpad][Kpad] (FP32 or half)
    void* d_cim = nullptr;
    void* d_cre_lo = nullptr;    // BF16 split: low parts of the coefficients
    void* d_cim_lo = nullptr;
    void* d_yhat = nullptr;      // [n_det][Kpad][max_block]
    void* d_yhat_lo = nullptr;
    long long yhat_det_stride = 0;
    // Eq. 10: autocorrelations R_i(t) [Mpad][2 d + 1], their denominators, and the
    // ring of recent z samples [det][Mpad][zlen] (half2) the reconstruction writes
    int ac_half = 0, zlen = 0;
    float2* d_ac = nullptr;
    float* d_ac_den = nullptr;
    uint32_t* d_zring = nullptr;
    uint32_t* d_bg = nullptr;          // background counts [det][n_snr][n_xi2] (own allocation)
    size_t bytes = 0;
    std::vector<void*> allocs;
};

}  // namespace

struct lloid_ctx {
    lloid_config cfg{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // Trigger lists go to the host on a stream of their own, so that the copy of one push's
    // list overlaps the next push's kernels: the compaction records `gathered` and the copy
    // stream waits for it.  Every pull slot compacts into a device list of its own, so a
    // later compaction never waits for an earlier copy.  The part of a list beyond its
    // pinned head is read from the slot's device list on rest_stream when it is collected.
    cudaStream_t copy_stream = nullptr, rest_stream = nullptr;
    cudaEvent_t gathered = nullptr;
    std::string err;
    long long launches = 0;
    size_t state_bytes = 0, bank_bytes = 0;

    // strain rings
    float* ring0 = nullptr;
    long long ring0_len = 0;
    int n_rates = 0;
    int rate_D[kMaxRates] = {};
    int down_smem = 0;                   // dynamic shared memory of k_downsample
    float* rate_ring[kMaxRates] = {};
    long long rate_len[kMaxRates] = {};
    float* w_down[kMaxRates] = {};
    std::vector<long long> pos;        // end of each detector's stream
    std::vector<long long> fin;        // last finalised window per detector

    // staging
    float* d_stage = nullptr;          // [n_det][max_block]
    float* h_stage[2] = {nullptr, nullptr};
    cudaEvent_t stage_ev[2] = {nullptr, nullptr};
    int stage_i = 0;
    long long last_n[64];              // last push length per detector (parity aid)

    // banks
    std::map<int, BankRT*> banks;
    int next_bank_id = 0;
    int M_used = 0;                    // global template ids handed out
    long long M_cap = 0;
    int* d_bank_of = nullptr;          // [M_cap]
    int* d_tmpl0_of = nullptr;         // [bank_cap]
    int bank_cap = 0;
    // coincident events (Sections II.D.3-4): [kWindowRing][bank_cap], net_snr <= 0 = none
    EventEntry* d_events = nullptr;
    EventEntry* h_events = nullptr;    // pinned staging of a pull
    long long coinc_next = 0;          // first window whose events are not formed yet
    // background bins (Section II.D.5): snr edges then xi2 edges
    float* d_bg_edges = nullptr;
    int bg_nsnr = 0, bg_nxi2 = 0;
    std::vector<int> h_bank_of, h_tmpl0_of;

    // window state
    int tiles_per_window = 0;
    int n_slots = 0;                   // partial ring slots per (template, detector)
    Partial* d_part = nullptr;         // [M_cap][n_det][n_slots]
    Partial* d_tail = nullptr;         // window overlap: [M_cap][n_det][n_tail] (TailRing)
    int n_tail = 0;
    SlabEntry* d_slab = nullptr;       // [kWindowRing][n_det][M_cap]
    int* d_counts = nullptr;
    int counts_cap = 0;
    // Pulls: slot 0 serves the blocking pulls, slots 1..kPullSlots the submitted ones.
    // A slot holds its compacted list and its count on the device until the pull is
    // collected, and, in pinned memory, the error flag, the count and the first `want`
    // triggers of the list, copied behind the pushes on copy_stream.
    struct PullSlot {
        TriggerOut* d = nullptr;           // the compacted list [d_cap]
        long long d_cap = 0;
        long long* d_total = nullptr;
        TriggerOut* h = nullptr;           // first part of the list [cap]
        long long cap = 0, want = 0;
        long long* h_total = nullptr;
        int* h_err = nullptr;
        cudaEvent_t ev = nullptr;
        long long w0 = 0, n_windows = 0;
        bool busy = false;
    };
    static constexpr int kPullSlots = 8;
    PullSlot pull[kPullSlots + 1];
    long long last_pull = 0;

    // job tables for the current push length
    bool jobs_dirty = true;
    long long jobs_n = -1;
    FirJob* d_fir = nullptr; int* d_fir_base = nullptr; int n_fir = 0, fir_tiles = 0;
    UpJob* d_up = nullptr; int* d_up_base = nullptr; int n_up = 0, up_tiles = 0, up_smem = 0;
    ReconJob* d_rec = nullptr; int* d_rec_base = nullptr; int n_rec = 0, rec_tiles = 0;
    FinJob* d_finj = nullptr; int n_fin = 0;
    // chunk tables of k_finalize (kFinTB templates) and k_coinc (kCoincTB), and their
    // cross-chunk reductions: a (key, count) pair per (job, detector, window slot) and
    // per (job, window slot), zero between launches
    FinChunk* d_fin_chunks = nullptr; int n_fin_chunks = 0;
    FinChunk* d_coinc_chunks = nullptr; int n_coinc_chunks = 0;
    unsigned long long* d_fin_red = nullptr;
    unsigned long long* d_coinc_red = nullptr;
    // split path job tables: FIR over all slices, levels per depth below the top
    FirTcJob* d_firtc = nullptr; FirMaps* d_firmaps = nullptr; TileInfo* d_firtc_base = nullptr;   // per tile
    int n_firtc = 0, firtc_tiles = 0, firtc_smem = 0, firtc_strip = 0, firtc_stages = 0, firtc_ctas = 1;
    static constexpr int kMaxDepth = 8;
    // one table per (depth, F slot): F = 0 (lowest level), 2, 4, ..., 64 -> slot 0..6
    static constexpr int kFSlots = 7;
    static constexpr int kLevTables = kMaxDepth * kFSlots;
    LevelJob* d_lev[kLevTables] = {}; LevelMaps* d_levmaps[kLevTables] = {};
    TileInfo* d_lev_base[kLevTables] = {};   // per tile of each level table
    // tile schedules ([grid + 1] offsets, then tile ids) for pushes of one detector [0]
    // and of all detectors [1]
    int* d_lev_sched[kLevTables][2] = {}; int lev_grid[kLevTables][2] = {};
    int* d_fir_sched[2] = {}; int fir_grid[2] = {};
    int n_lev[kLevTables] = {}, lev_tiles[kLevTables] = {};
    int max_depth = 0;
    std::vector<int> top_job_of_bank;  // bank id -> index in its top-level table
    std::vector<int> top_slot_of_bank; // bank id -> F slot of its top level (split path)
    // Eq. 10 table: tiles of 8 templates over the banks with autocorrelations
    Xi2Job* d_xi2 = nullptr; int* d_xi2_base = nullptr; int n_xi2 = 0, xi2_tiles = 0;
    int xi2_half_max = 0;              // largest d of the loaded banks (pull readiness)
    std::vector<long long> xi2_next;   // per detector: first window whose xi2 is not computed yet
    // f0 form: the banks' jobs, coefficient maps, work units (bank, detector, window group) and
    // their schedules, and one slice table
    static constexpr int kF0Classes = 1;
    F0Job* d_f0job[kF0Classes] = {}; F0Maps* d_f0map[kF0Classes] = {}; F0Unit* d_f0unit[kF0Classes] = {};
    int* d_f0sched[kF0Classes][2] = {}; int f0_grid[kF0Classes][2] = {}; int n_f0unit[kF0Classes] = {};
    YupSlice* d_f0slices = nullptr;
    F0Piece* d_f0pieces = nullptr;     // k_yhat's staging pieces of every bank in the f0 form
    int f0_rall = 4;                   // the largest bank's staged upsamplers (floats)
    int* d_f0bends = nullptr;          // and the ends of their batches
    std::vector<int> f0_class_of_bank, f0_job_of_bank;
    uint16_t* d_u_hi[kFSlots] = {};    // Eq. 8 tile matrices per F slot (hi, lo halves)
    uint16_t* d_u_lo[kFSlots] = {};
    // split path streams: index 0 = f0, index r + 1 = rate_D[r]; hi/lo halves, double-mapped
    uint16_t* s_hi[kMaxRates + 1] = {};
    uint16_t* s_lo[kMaxRates + 1] = {};
    long long s_len[kMaxRates + 1] = {};
    std::vector<void*> job_allocs;
    cudaEvent_t done_ev = nullptr;
    int* d_err = nullptr;              // device-side wait-expiry code (0 = none)
    int n_sm = 0;
    int smem_optin = 0;                // largest dynamic shared memory a block may opt into

    // injected faults (lloid_inject_fault) and the zero block that fills gaps
    long long fault_alloc = 0, fault_drop = 0, fault_delay_us = 0;
    float* d_zero = nullptr;

    // stage timing (LLOID_FLAG_STAGE_TIMING)
    struct Pending { int stage; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> ev_pool;
    double stage_ms[LLOID_N_STAGES] = {};
    long long stage_launches[LLOID_N_STAGES] = {};
};

namespace {

lloid_status fail(lloid_ctx* c, lloid_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return st;
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? LLOID_ENOMEM : LLOID_ECUDA, \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

#define CKL()                                                                           \
    do {                                                                                \
        ++ctx->launches;                                                                \
        cudaError_t e_ = cudaGetLastError();                                            \
        if (e_ != cudaSuccess)                                                          \
            return fail(ctx, LLOID_ECUDA, "launch: %s (%s:%d)", cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

template <typename T>
lloid_status dalloc(lloid_ctx* ctx, T** p, size_t bytes, std::vector<void*>* owner, size_t* acct) {
    void* q = nullptr;
    if (ctx->fault_alloc > 0) {
        --ctx->fault_alloc;
        return fail(ctx, LLOID_ENOMEM, "device allocation of %zu bytes failed (injected)", bytes);
    }
    CK(cudaMalloc(&q, bytes));
    CK(cudaMemsetAsync(q, 0, bytes, ctx->stream));
    *p = (T*)q;
    if (owner) owner->push_back(q);
    if (acct) *acct += bytes;
    return LLOID_OK;
}

__global__ void k_fill_partials(Partial* p, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = make_float4(-1.f, __int_as_float(0x7fffffff), 0.f, 0.f);
}

// Composed response of the ladder upsamplers (Eq. 7-8, c = F N_up at each
// stage) from `rate` up to f0, applied to a unit impulse at low-rate sample 0.
// out[e - e_min] is the full-rate response at offset e.
void compose_upsampler(const std::vector<int>& ladder_up, int n_up, std::vector<double>* out, int* e_min,
                       int* e_max) {
    // ladder_up: rates from the slice's rate (first) to f0 (last), ascending
    std::vector<double> x(1, 1.0);
    long long lo = 0;   // index of x[0] at the current rate
    for (size_t s = 0; s + 1 < ladder_up.size(); ++s) {
        int F = ladder_up[s + 1] / ladder_up[s];
        int c = F * n_up;
        std::vector<double> g = sinc_windowed(F, c);
        long long y_lo = F * lo - c;
        long long y_hi = F * (lo + (long long)x.size() - 1) + c;
        std::vector<double> y(y_hi - y_lo + 1, 0.0);
        for (size_t k = 0; k < x.size(); ++k)
            for (int i = 0; i <= 2 * c; ++i)   // y[p] += x[k] g[p - F k + c]
                y[F * (lo + (long long)k) - c + i - y_lo] += x[k] * g[i];
        x.swap(y);
        lo = y_lo;
    }
    *e_min = (int)lo;
    *e_max = (int)(lo + (long long)x.size() - 1);
    *out = x;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// 2-D K-major map: rows of `cols` 16-bit elements, box 64 x box_rows, 128-byte swizzle.
bool encode_map(CUtensorMap* m, bool bf16, const void* base, long long cols, long long rows, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                    const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// 4-D 16-bit map of time-blocked planes [planes][cols / 8][rows][8], each block of 8 samples
// seen as rows / 32 runs of 256 values (512 B) so that the TMA moves a box in 16 long rows:
// box 256 x 4 x (kWinK / 8) x 1 = 128 rows x 8 samples x 4 blocks, no swizzle.  rows % 128 == 0.
bool encode_map_blocked(CUtensorMap* m, bool bf16, const void* base, long long cols, long long rows, long long planes) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[4] = {256, (cuuint64_t)(rows / 32), (cuuint64_t)(cols / 8), (cuuint64_t)planes};
    cuuint64_t strides[3] = {512, (cuuint64_t)rows * 16, (cuuint64_t)(cols / 8) * rows * 16};
    cuuint32_t box[4] = {256, 4, (cuuint32_t)(kWinK / 8), 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4,
                    const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// The same planes with a box of 128 rows x kb blocks of 8 columns (kb <= 12): a whole Yhat tile
// of a bank (K = 8 kb bases) in one load.
bool encode_map_blocked_kb(CUtensorMap* m, bool bf16, const void* base, long long cols, long long rows,
                           long long planes, int kb) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[4] = {256, (cuuint64_t)(rows / 32), (cuuint64_t)(cols / 8), (cuuint64_t)planes};
    cuuint64_t strides[3] = {512, (cuuint64_t)rows * 16, (cuuint64_t)(cols / 8) * rows * 16};
    cuuint32_t box[4] = {256, 4, (cuuint32_t)kb, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 4,
                    const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

lloid_status ensure_template_capacity(lloid_ctx* ctx, long long need) {
    if (need <= ctx->M_cap) return LLOID_OK;
    const int nd = ctx->cfg.n_detectors;
    long long cap = std::max<long long>(need, 2 * ctx->M_cap);
    cap = std::max<long long>(cap, 1024);
    // partials: [M][det][slot] -> prefix copy
    Partial* np = nullptr;
    size_t pbytes = (size_t)cap * nd * ctx->n_slots * sizeof(Partial);
    CK(cudaMalloc(&np, pbytes));
    long long nfill = cap * nd * ctx->n_slots;
    k_fill_partials<<<(unsigned)((nfill + 255) / 256), 256, 0, ctx->stream>>>(np, nfill);
    CKL();
    if (ctx->d_part) {
        CK(cudaMemcpyAsync(np, ctx->d_part, (size_t)ctx->M_cap * nd * ctx->n_slots * sizeof(Partial),
                           cudaMemcpyDeviceToDevice, ctx->stream));
    }
    // overlap tails: [M][det][n_tail] -> prefix copy
    Partial* ntl = nullptr;
    const size_t tbytes = (size_t)cap * nd * ctx->n_tail * sizeof(Partial);
    CK(cudaMalloc(&ntl, tbytes));
    const long long tfill = cap * nd * ctx->n_tail;
    k_fill_partials<<<(unsigned)((tfill + 255) / 256), 256, 0, ctx->stream>>>(ntl, tfill);
    CKL();
    if (ctx->d_tail)
        CK(cudaMemcpyAsync(ntl, ctx->d_tail, (size_t)ctx->M_cap * nd * ctx->n_tail * sizeof(Partial),
                           cudaMemcpyDeviceToDevice, ctx->stream));
    // slab: [ring][det][M] -> pitched copy
    SlabEntry* ns = nullptr;
    size_t sbytes = (size_t)kWindowRing * nd * cap * sizeof(SlabEntry);
    CK(cudaMalloc(&ns, sbytes));
    CK(cudaMemsetAsync(ns, 0, sbytes, ctx->stream));
    if (ctx->d_slab) {
        CK(cudaMemcpy2DAsync(ns, cap * sizeof(SlabEntry), ctx->d_slab, ctx->M_cap * sizeof(SlabEntry),
                             ctx->M_cap * sizeof(SlabEntry), (size_t)kWindowRing * nd, cudaMemcpyDeviceToDevice,
                             ctx->stream));
    }
    int* nb = nullptr;
    CK(cudaMalloc(&nb, cap * sizeof(int)));
    if (ctx->d_bank_of) CK(cudaMemcpyAsync(nb, ctx->d_bank_of, ctx->M_cap * sizeof(int), cudaMemcpyDeviceToDevice, ctx->stream));
    int nchunks = (int)((nd * cap + 1023) / 1024);
    int* nc = nullptr;
    CK(cudaMalloc(&nc, nchunks * sizeof(int)));
    CK(cudaStreamSynchronize(ctx->stream));
    size_t old = ctx->M_cap ? ((size_t)ctx->M_cap * nd * ctx->n_slots * sizeof(Partial) +
                               (size_t)ctx->M_cap * nd * ctx->n_tail * sizeof(Partial) +
                               (size_t)kWindowRing * nd * ctx->M_cap * sizeof(SlabEntry) +
                               ctx->M_cap * sizeof(int))
                            : 0;
    cudaFree(ctx->d_part); cudaFree(ctx->d_slab); cudaFree(ctx->d_bank_of); cudaFree(ctx->d_counts);
    cudaFree(ctx->d_tail);
    ctx->d_part = np; ctx->d_slab = ns; ctx->d_bank_of = nb; ctx->d_counts = nc; ctx->d_tail = ntl;
    ctx->counts_cap = nchunks;
    ctx->state_bytes += pbytes + tbytes + sbytes + cap * sizeof(int) - old;
    ctx->M_cap = cap;
    ctx->h_bank_of.resize(cap, -1);
    return LLOID_OK;
}

void free_jobs(lloid_ctx* ctx) {
    for (void* p : ctx->job_allocs) cudaFree(p);
    ctx->job_allocs.clear();
    ctx->d_fir = nullptr; ctx->d_up = nullptr; ctx->d_rec = nullptr; ctx->d_finj = nullptr;
    ctx->d_fin_chunks = ctx->d_coinc_chunks = nullptr; ctx->n_fin_chunks = ctx->n_coinc_chunks = 0;
    ctx->d_fin_red = ctx->d_coinc_red = nullptr;
    ctx->d_firtc = nullptr; ctx->d_firmaps = nullptr; ctx->d_firtc_base = nullptr;
    for (int d = 0; d < lloid_ctx::kLevTables; ++d) {
        ctx->d_lev[d] = nullptr; ctx->d_levmaps[d] = nullptr; ctx->d_lev_base[d] = nullptr;
        ctx->n_lev[d] = 0; ctx->lev_tiles[d] = 0;
        ctx->d_lev_sched[d][0] = ctx->d_lev_sched[d][1] = nullptr;
    }
    ctx->d_fir_sched[0] = ctx->d_fir_sched[1] = nullptr;
    ctx->n_firtc = ctx->firtc_tiles = 0;
    ctx->d_xi2 = nullptr; ctx->d_xi2_base = nullptr; ctx->n_xi2 = ctx->xi2_tiles = 0;
    for (int k = 0; k < lloid_ctx::kF0Classes; ++k) {
        ctx->d_f0job[k] = nullptr; ctx->d_f0map[k] = nullptr; ctx->d_f0unit[k] = nullptr; ctx->n_f0unit[k] = 0;
        ctx->d_f0sched[k][0] = ctx->d_f0sched[k][1] = nullptr;
    }
    ctx->d_f0slices = nullptr; ctx->d_f0pieces = nullptr; ctx->d_f0bends = nullptr;
}

template <typename T>
lloid_status upload_vec(lloid_ctx* ctx, T** dst, const std::vector<T>& v) {
    size_t bytes = std::max<size_t>(1, v.size()) * sizeof(T);
    CK(cudaMalloc((void**)dst, bytes));
    ctx->job_allocs.push_back(*dst);
    if (!v.empty()) CK(cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
    return LLOID_OK;
}

// Launch with programmatic stream serialisation: the kernel may be scheduled
// while the previous one drains; it waits (griddepcontrol.wait) before it
// reads anything the previous kernels wrote.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), dim3 g, dim3 b, size_t smem, cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g;
    cfg.blockDim = b;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

// Static schedule of one launch over tiles t of a job table (cost[t]) for nd
// detectors: tile id it = t * nd + detector offset.  Longest tiles first, each
// to the least-loaded CTA (LPT); each CTA then runs its tiles in id order, so
// the detectors of one tile run side by side and share its operands in L2.
std::vector<int> build_sched(const std::vector<double>& cost, int nd, int n_sm, int* grid_out) {
    const long long total = (long long)cost.size() * nd;
    const int grid = (int)std::max<long long>(1, std::min<long long>(total, n_sm));
    std::vector<int> order((size_t)total);
    for (long long i = 0; i < total; ++i) order[(size_t)i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a / nd] > cost[b / nd]; });
    std::vector<std::vector<int>> per(grid);
    std::priority_queue<std::pair<double, int>, std::vector<std::pair<double, int>>, std::greater<>> load;
    for (int g = 0; g < grid; ++g) load.push({0.0, g});
    for (int it : order) {
        auto top = load.top();
        load.pop();
        per[top.second].push_back(it);
        load.push({top.first + cost[it / nd], top.second});
    }
    std::vector<int> h(grid + 1, 0);
    for (int g = 0; g < grid; ++g) {
        std::sort(per[g].begin(), per[g].end());
        h[g + 1] = h[g] + (int)per[g].size();
    }
    for (int g = 0; g < grid; ++g) h.insert(h.end(), per[g].begin(), per[g].end());
    *grid_out = grid;
    return h;
}
lloid_status upload_sched(lloid_ctx* ctx, const std::vector<double>& cost, int nd, int** d_out, int* grid_out,
                          int ctas_per_sm = 1) {
    return upload_vec(ctx, d_out, build_sched(cost, nd, ctx->n_sm * ctas_per_sm, grid_out));
}

bool split_precision(const lloid_ctx* ctx) { return ctx->cfg.precision != LLOID_FP32; }

TailRing tail_ring(const lloid_ctx* ctx) {
    return TailRing{ctx->d_tail, (long long)ctx->cfg.n_detectors * ctx->n_tail, ctx->n_tail,
                    (int)ctx->cfg.window_overlap};
}

bool timing(const lloid_ctx* ctx) { return (ctx->cfg.flags & LLOID_FLAG_STAGE_TIMING) != 0; }

lloid_status resolve_timers(lloid_ctx* ctx) {
    if (ctx->pending.empty()) return LLOID_OK;
    CK(cudaStreamSynchronize(ctx->stream));
    for (auto& p : ctx->pending) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, p.a, p.b));
        ctx->stage_ms[p.stage] += ms;
        ctx->ev_pool.push_back(p.a);
        ctx->ev_pool.push_back(p.b);
    }
    ctx->pending.clear();
    return LLOID_OK;
}

// RAII pair of events around one stage's launches on the context stream.
struct StageTimer {
    lloid_ctx* ctx;
    int stage;
    cudaEvent_t a = nullptr, b = nullptr;
    long long l0;
    StageTimer(lloid_ctx* c, int s) : ctx(c), stage(s), l0(c->launches) {
        if (!timing(ctx)) return;
        if (ctx->pending.size() > 4096) resolve_timers(ctx);
        for (cudaEvent_t* e : {&a, &b}) {
            if (!ctx->ev_pool.empty()) { *e = ctx->ev_pool.back(); ctx->ev_pool.pop_back(); }
            else cudaEventCreate(e);
        }
        cudaEventRecord(a, ctx->stream);
    }
    ~StageTimer() {
        ctx->stage_launches[stage] += ctx->launches - l0;
        if (!a) return;
        cudaEventRecord(b, ctx->stream);
        ctx->pending.push_back({stage, a, b});
    }
};


// Job tables of the split (tensor-core) path for pushes of n samples.
// Opt every k_level_tc instantiation of one precision into its shared memory.
template <bool BF16, bool TOP, bool SZ, int F>
cudaError_t level_attr1() {
    return cudaFuncSetAttribute(k_level_tc<BF16, TOP, SZ, F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                LevCfg<BF16, TOP>::SMEM);
}
template <bool BF16, bool TOP, bool SZ>
cudaError_t level_attr_f() {
    cudaError_t e = cudaSuccess;
    const cudaError_t r[] = {level_attr1<BF16, TOP, SZ, 0>(), level_attr1<BF16, TOP, SZ, 2>(),
                             level_attr1<BF16, TOP, SZ, 4>(), level_attr1<BF16, TOP, SZ, 8>(),
                             level_attr1<BF16, TOP, SZ, 16>(), level_attr1<BF16, TOP, SZ, 32>(),
                             level_attr1<BF16, TOP, SZ, 64>()};
    for (cudaError_t x : r)
        if (x != cudaSuccess) e = x;
    return e;
}
template <bool BF16>
cudaError_t level_smem_attr() {
    cudaError_t e = level_attr_f<BF16, false, false>();
    if (e == cudaSuccess) e = level_attr_f<BF16, true, false>();
    if (e == cudaSuccess) e = level_attr_f<BF16, true, true>();
    return e;
}

lloid_status build_jobs_split(lloid_ctx* ctx, long long n) {
    const lloid_config& c = ctx->cfg;
    const bool bf = c.precision == LLOID_BF16_SPLIT;
    const int nd = c.n_detectors;
    std::vector<FirTcJob> fj;
    std::vector<FirMaps> fm;
    std::vector<TileInfo> fb;
    std::vector<LevelJob> lj[lloid_ctx::kLevTables];
    std::vector<LevelMaps> lm[lloid_ctx::kLevTables];
    std::vector<TileInfo> lb[lloid_ctx::kLevTables];
    int lt[lloid_ctx::kLevTables] = {};
    int ft = 0, strip = 128, max_depth = 0;
    std::vector<YupSlice> ys;
    std::vector<F0Piece> f0pc;
    std::vector<int> f0be;
    std::vector<F0Job> f0j[lloid_ctx::kF0Classes];
    std::vector<F0Maps> f0m[lloid_ctx::kF0Classes];
    std::vector<F0Unit> f0u[lloid_ctx::kF0Classes];
    std::vector<double> f0cost[lloid_ctx::kF0Classes];
    lloid_status st0;
    ctx->f0_rall = 4;
    ctx->top_job_of_bank.assign(ctx->next_bank_id, -1);
    ctx->top_slot_of_bank.assign(ctx->next_bank_id, 0);
    ctx->f0_class_of_bank.assign(ctx->next_bank_id, -1);
    ctx->f0_job_of_bank.assign(ctx->next_bank_id, -1);
    for (auto& kv : ctx->banks) {
        BankRT* b = kv.second;
        const int nl = (int)b->lev.size();
        if (nl > lloid_ctx::kMaxDepth) return fail(ctx, LLOID_EINVAL, "bank %d has more than 8 ladder levels", b->id);
        max_depth = std::max(max_depth, b->form == 1 ? 0 : nl);
        for (size_t si = 0; si < b->sl.size(); ++si) {
            const SliceRT& sl = b->sl[si];
            const FirSliceRT& fsr = b->fs[si];
            const LevelRT& L = b->lev[fsr.level];
            int ri = 0;
            if (sl.D > 1) { ri = 1; while (ctx->rate_D[ri - 1] != sl.D) ++ri; }
            FirTcJob f{};
            f.s_hi = ctx->s_hi[ri]; f.s_lo = ctx->s_lo[ri];
            f.s_det_stride = 2 * ctx->s_len[ri]; f.s_len = (int)ctx->s_len[ri];
            f.y_hi = L.d_yhi + fsr.col; f.y_lo = L.d_ylo + fsr.col;
            f.y_det_stride = 2LL * L.R * L.Kp; f.y_rows = L.R; f.y_ld = L.Kp;
            f.J_over_D = sl.J / sl.D;
            f.Mtiles = fsr.Mtiles; f.Kp = fsr.Kp; f.Np = fsr.Np;
            const long long ncg = n / (8LL * sl.D) + 2;
            if (ncg <= kFirNC) { f.NC = (int)((ncg + 15) / 16 * 16); f.ctiles = 1; }
            else { f.NC = kFirNC; f.ctiles = (int)((ncg + kFirNC - 1) / kFirNC); }
            f.D = sl.D; f.Lambda = L.Lambda; f.q_count = (int)(n / sl.D); f.map = (int)fj.size();
            FirMaps mp;
            std::memset(&mp, 0, sizeof mp);
            bool ok = encode_map(&mp.a, bf, fsr.d_a, fsr.Kp, (long long)fsr.Mtiles * 128, 128);
            if (ok && bf) ok = encode_map(&mp.a_lo, bf, fsr.d_a_lo, fsr.Kp, (long long)fsr.Mtiles * 128, 128);
            if (!ok) return fail(ctx, LLOID_ECUDA, "cuTensorMapEncodeTiled failed (FIR bank %d)", b->id);
            strip = std::max(strip, (2 * (8 * f.NC + f.Kp) + 127) / 128 * 128);
            for (int l = 0; l < f.Mtiles * f.ctiles; ++l) fb.push_back(TileInfo{(int)fj.size(), l, f.Kp, f.NC});
            fj.push_back(f); fm.push_back(mp); ft += f.Mtiles * f.ctiles;
        }
        // Ladder form: one job per rate, lowest first (depth nl - 1 .. 0).  The f0 form's banks go
        // to the f0 kernel's tables below.
        for (int j = 0; j < nl && b->form == 0; ++j) {
            const LevelRT& L = b->lev[j];
            const int depth = nl - 1 - j;
            const bool below = j > 0;   // a ladder level below to upsample
            LevelJob q{};
            if (below) {
                const LevelRT& P = b->lev[j - 1];
                q.F = P.D / L.D; q.D_lo = P.D; q.Lambda_lo = P.Lambda;
            }
            if (j < nl - 1) {
                q.acc_out = L.d_accp; q.acc_out_det_stride = 4LL * b->Mpad * L.acc_cols; q.acc_cols = L.acc_cols;
            }
            q.Kp = L.Kp; q.M = b->M; q.Mpad = b->Mpad; q.tmpl0 = b->tmpl0;
            if (depth == 0 && b->d_zring) {
                q.zring = b->d_zring; q.zring_det_stride = (long long)b->Mpad * b->zlen; q.zring_len = b->zlen;
            }
            q.tiles_m = b->Mpad / kTcTileM;
            if (depth == 0) q.tiles_t = (int)(n / kTcTileN);
            else q.tiles_t = (int)((((n - 1 + 2LL * L.Lambda) / L.D + 2) + 127 + 127) / 128);
            q.D = L.D; q.Lambda = L.Lambda; q.y_rows = L.R;
            int fslot = 0;
            if (q.F) {
                while ((2 << fslot) < q.F) ++fslot;
                ++fslot;
                if ((1 << fslot) != q.F || fslot >= lloid_ctx::kFSlots)
                    return fail(ctx, LLOID_EINVAL, "bank %d: upsampling factor %d is not 2..64", b->id, q.F);
            }
            const int tab = depth * lloid_ctx::kFSlots + fslot;
            q.map = (int)lj[tab].size();
            LevelMaps mp;
            std::memset(&mp, 0, sizeof mp);
            if (below) {
                const LevelRT& P = b->lev[j - 1];
                const int kw = win_chunks(q.F) * kWinK;
                if (!encode_map_blocked(&mp.accw, bf, P.d_accp, P.acc_cols, b->Mpad, (long long)nd * 4) ||
                    !encode_map_blocked(&mp.uhi, bf, ctx->d_u_hi[fslot], kw, 128, 8) ||
                    !encode_map_blocked(&mp.ulo, bf, ctx->d_u_lo[fslot], kw, 128, 8))
                    return fail(ctx, LLOID_ECUDA, "cuTensorMapEncodeTiled failed (window, bank %d)", b->id);
            }
            if (L.Kp > 0) {
                bool ok = encode_map(&mp.cre, bf, L.d_cre, L.Kp, b->Mpad, kTcTileM) &&
                          encode_map(&mp.cim, bf, L.d_cim, L.Kp, b->Mpad, kTcTileM) &&
                          encode_map(&mp.yhi, bf, L.d_yhi, L.Kp, (long long)nd * 2 * L.R, kTcTileN) &&
                          encode_map(&mp.ylo, bf, L.d_ylo, L.Kp, (long long)nd * 2 * L.R, kTcTileN);
                if (ok && bf)
                    ok = encode_map(&mp.cre_lo, bf, L.d_cre_lo, L.Kp, b->Mpad, kTcTileM) &&
                         encode_map(&mp.cim_lo, bf, L.d_cim_lo, L.Kp, b->Mpad, kTcTileM);
                if (!ok) return fail(ctx, LLOID_ECUDA, "cuTensorMapEncodeTiled failed (level, bank %d)", b->id);
            }

            if (depth == 0) { ctx->top_job_of_bank[b->id] = (int)lj[tab].size(); ctx->top_slot_of_bank[b->id] = fslot; }
            for (int l = 0; l < q.tiles_m * q.tiles_t; ++l)
                lb[tab].push_back(TileInfo{(int)lj[tab].size(), l, q.Kp, L.K / 16});
            lj[tab].push_back(q); lm[tab].push_back(mp);
            lt[tab] += q.tiles_m * q.tiles_t;
        }
        if (b->form == 1) {   // f0 form: one job of the f0 kernel, its slices, its window groups
            const int cls = 0;   // one launch for every bank in the f0 form
            F0Job f{};
            f.M = b->M; f.Mpad = b->Mpad; f.tmpl0 = b->tmpl0; f.K = b->top.K; f.tiles_m = b->Mpad / 128;
            f.s0 = (int)ys.size(); f.ns = (int)b->sl.size(); f.map = (int)f0j[cls].size();
            f.yh = b->d_yf0; f.yrows = (int)c.max_block;
            // A tile starts on a multiple of 128 = a multiple of every D: slice s reaches rows
            // [k0 / D + qoff, + nq) of its Y ring, nq the same for every tile
            auto floordiv = [](long long a, long long d) { return a >= 0 ? a / d : -((-a + d - 1) / d); };
            int roff = 0;
            for (size_t si = 0; si < b->sl.size(); ++si) {
                const SliceRT& sl = b->sl[si];
                const FirSliceRT& fsr = b->fs[si];
                const LevelRT& L = b->lev[fsr.level];
                YupSlice u{};
                u.y_hi = L.d_yhi + fsr.col; u.y_lo = L.d_ylo + fsr.col; u.y_det_stride = 2LL * L.R * L.Kp;
                u.R = sl.d_R; u.y_rows = L.R; u.y_ld = L.Kp;
                u.e_min = sl.e_min; u.rlen = sl.e_max - sl.e_min + 1; u.D = sl.D; u.L = sl.L; u.tcol = sl.tcol;
                u.qoff = (int)floordiv(-(long long)sl.e_max + sl.D - 1, sl.D);
                u.nq = (int)(floordiv(127 - sl.e_min, sl.D) - u.qoff + 1);
                u.roff = roff;
                roff += u.rlen;
                ys.push_back(u);
            }
            // pieces of up to 32 columns (narrower when many rows must fit the staging), in column
            // order, in batches of at most kF0StageFloats staged values
            f.pc0 = (int)f0pc.size();
            f.bt0 = (int)f0be.size();
            int off = 0, items = 0, np = 0;
            for (int q = 0; q < f.ns; ++q) {
                const YupSlice& u = ys[f.s0 + q];
                if (u.D == 1) {   // R = [1]: Yhat is Y, read straight from the ring (no staged rows)
                    F0Piece pc{};
                    pc.s = q; pc.c0 = 0; pc.nc = u.L; pc.nv = 0; pc.off = 0; pc.pitch = 0; pc.items = 0; pc.item0 = items;
                    f0pc.push_back(pc);
                    ++np;
                    continue;
                }
                const int nq2 = u.nq + 128 / u.D;            // the rows both tiles of a pair reach
                const int cw = 4 * std::min(4, (kF0StageFloats / nq2 - 4) / 4);   // pieces <= 16 bases
                for (int c0 = 0; c0 < u.L; c0 += cw) {
                    F0Piece pc{};
                    pc.s = q; pc.c0 = c0; pc.nc = std::min(cw, u.L - c0); pc.nv = (pc.nc + 3) >> 2;
                    pc.pitch = 4 * pc.nv + 4;
                    if (off + nq2 * pc.pitch > kF0StageFloats) { f0be.push_back(np); off = 0; items = 0; }
                    pc.off = off; pc.items = nq2 * pc.nv; pc.item0 = items;
                    off += nq2 * pc.pitch;
                    items += pc.items;
                    f0pc.push_back(pc);
                    ++np;
                }
            }
            f0be.push_back(np);
            ctx->f0_rall = std::max(ctx->f0_rall, (roff + 3) / 4 * 4);
            f.np = np;
            f.nbat = (int)f0be.size() - f.bt0;
            if (np > kF0MaxPieces) return fail(ctx, LLOID_EINVAL, "bank %d: %d staging pieces", b->id, np);
            F0Maps mp;
            std::memset(&mp, 0, sizeof mp);
            if (!encode_map_blocked(&mp.c, bf, b->d_cblk, b->top.K, b->Mpad, bf ? 4 : 2) ||
                !encode_map_blocked_kb(&mp.y, bf, b->d_yf0, b->top.K, c.max_block, 2LL * nd, b->top.K / 8))
                return fail(ctx, LLOID_ECUDA, "cuTensorMapEncodeTiled failed (f0 operands, bank %d)", b->id);
            ctx->f0_class_of_bank[b->id] = cls;
            ctx->f0_job_of_bank[b->id] = (int)f0j[cls].size();
            ctx->top_job_of_bank[b->id] = -1;
            const int tpw = (int)(c.window_samples / 128), nt = (int)(n / 128);
            for (int g = 0; g * tpw < nt; ++g) {
                f0u[cls].push_back(F0Unit{(int)f0j[cls].size(), g});
                f0cost[cls].push_back((double)f.tiles_m * std::min(tpw, nt - g * tpw) * (bf ? 6 : 4) * (f.K / 16) +
                                      4.0 * std::min(tpw, nt - g * tpw));
            }
            f0j[cls].push_back(f);
            f0m[cls].push_back(mp);
        }
    }
    if ((st0 = upload_vec(ctx, &ctx->d_f0slices, ys)) || (st0 = upload_vec(ctx, &ctx->d_f0pieces, f0pc)) ||
        (st0 = upload_vec(ctx, &ctx->d_f0bends, f0be)))
        return st0;
    for (int cls = 0; cls < lloid_ctx::kF0Classes; ++cls) {
        ctx->n_f0unit[cls] = (int)f0u[cls].size();
        if (f0u[cls].empty()) continue;
        if ((st0 = upload_vec(ctx, &ctx->d_f0job[cls], f0j[cls])) || (st0 = upload_vec(ctx, &ctx->d_f0map[cls], f0m[cls])) ||
            (st0 = upload_vec(ctx, &ctx->d_f0unit[cls], f0u[cls])))
            return st0;
        for (int v = 0; v < 2; ++v)
            if ((st0 = upload_sched(ctx, f0cost[cls], v ? nd : 1, &ctx->d_f0sched[cls][v], &ctx->f0_grid[cls][v])))
                return st0;
        const int smem = f0_smem_bytes(bf, kF0Kc, 2);
        if (bf) {
            CK(cudaFuncSetAttribute(k_f0_top<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            CK(cudaFuncSetAttribute(k_f0_top<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        } else {
            CK(cudaFuncSetAttribute(k_f0_top<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            CK(cudaFuncSetAttribute(k_f0_top<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        }
        int fit = 0;   // registers (the kernel's cap) and shared memory of one CTA on one SM
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, bf ? k_f0_top<true, false> : k_f0_top<false, false>,
                                                         kF0Threads, smem));
        if (fit < 1) return fail(ctx, LLOID_ECUDA, "the f0-form kernel (%d threads, %d B shared) does not fit an SM",
                                 kF0Threads, smem);
        const int ysm = yhat_smem_bytes(kF0RAll);
        if (bf) CK(cudaFuncSetAttribute(k_yhat<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ysm));
        else CK(cudaFuncSetAttribute(k_yhat<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, ysm));
    }
    lloid_status st;
    if ((st = upload_vec(ctx, &ctx->d_firtc, fj)) || (st = upload_vec(ctx, &ctx->d_firmaps, fm)) ||
        (st = upload_vec(ctx, &ctx->d_firtc_base, fb)))
        return st;
    for (int d = 0; d < lloid_ctx::kLevTables; ++d) {
        ctx->d_lev[d] = nullptr; ctx->d_levmaps[d] = nullptr; ctx->d_lev_base[d] = nullptr;
        ctx->n_lev[d] = (int)lj[d].size(); ctx->lev_tiles[d] = lt[d];
        if (lj[d].empty()) continue;
        if ((st = upload_vec(ctx, &ctx->d_lev[d], lj[d])) || (st = upload_vec(ctx, &ctx->d_levmaps[d], lm[d])) ||
            (st = upload_vec(ctx, &ctx->d_lev_base[d], lb[d])))
            return st;
    }
    // FIR shared memory: the strips, the epilogue staging and the barriers, then A' stages.
    // Two CTAs per SM (each with 256 TMEM columns) when each still gets 2 stages; else one
    // CTA with as many stages as fit.
    const int fir_fixed = 4 * strip + FirCfg<false>::EPI_BYTES + 256 + 1024;   // EPI_BYTES is the same for both
    const int fir_sbytes = bf ? FirCfg<true>::STAGE_BYTES : FirCfg<false>::STAGE_BYTES;
    {
        const int st2 = std::min(FirCfg<false>::MAX_STAGES, (113 * 1024 - fir_fixed) / fir_sbytes);
        if (st2 >= 2 && c.fir_ctas != 1) { ctx->firtc_ctas = 2; ctx->firtc_stages = st2; }
        else { ctx->firtc_ctas = 1; ctx->firtc_stages = std::min(FirCfg<false>::MAX_STAGES, (227 * 1024 - fir_fixed) / fir_sbytes); }
    }
    {   // schedules: cost ~ MMAs of a tile plus a fixed epilogue share
        const int mk = bf ? 3 : 2;
        std::vector<double> fc;
        for (const FirTcJob& f : fj)
            for (int k = 0; k < f.Mtiles * f.ctiles; ++k) fc.push_back(mk * f.Kp / 16.0 + 16.0);
        for (int v = 0; v < 2; ++v) {
            const int ndv = v ? nd : 1;
            if ((st = upload_sched(ctx, fc, ndv, &ctx->d_fir_sched[v], &ctx->fir_grid[v], ctx->firtc_ctas))) return st;
        }
        for (int d = 0; d < lloid_ctx::kLevTables; ++d) {
            if (lj[d].empty()) continue;
            std::vector<double> lc;
            for (const LevelJob& q : lj[d])
                for (int k = 0; k < q.tiles_m * q.tiles_t; ++k)
                    lc.push_back((bf ? 6 : 4) * q.Kp / 16.0 + 12.0 * win_chunks(q.F) + 16.0);
            for (int v = 0; v < 2; ++v) {
                const int ndv = v ? nd : 1;
                if ((st = upload_sched(ctx, lc, ndv, &ctx->d_lev_sched[d][v], &ctx->lev_grid[d][v]))) return st;
            }
        }
    }
    ctx->n_firtc = (int)fj.size();
    ctx->firtc_tiles = ft;
    ctx->firtc_strip = strip;
    ctx->max_depth = max_depth;
    if (ctx->firtc_stages < 2) return fail(ctx, LLOID_EINVAL, "FIR strips of %d bytes leave no room for 2 stages", strip);
    const int fsmem = ctx->firtc_stages * fir_sbytes + fir_fixed;
    ctx->firtc_smem = fsmem;
    if (fsmem > 227 * 1024) return fail(ctx, LLOID_EINVAL, "FIR shared memory %d exceeds the limit", fsmem);
    if (bf) CK(cudaFuncSetAttribute(k_fir_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, fsmem));
    else CK(cudaFuncSetAttribute(k_fir_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, fsmem));
    if (bf) CK(level_smem_attr<true>());
    else CK(level_smem_attr<false>());
    return LLOID_OK;
}

// (Re)build the job tables for pushes of n samples.
lloid_status build_jobs(lloid_ctx* ctx, long long n) {
    if (!ctx->jobs_dirty && ctx->jobs_n == n) return LLOID_OK;
    CK(cudaStreamSynchronize(ctx->stream));
    free_jobs(ctx);
    std::vector<FinJob> fin;
    for (auto& kv : ctx->banks)
        fin.push_back(FinJob{kv.second->tmpl0, kv.second->M, kv.second->id, kv.second->d_bg,
                             split_precision(ctx) && kv.second->form == 1 ? 1 : 0});
    lloid_status st;
    if ((st = upload_vec(ctx, &ctx->d_finj, fin))) return st;
    ctx->n_fin = (int)fin.size();
    {
        std::vector<FinChunk> fc, cc;
        for (int j = 0; j < (int)fin.size(); ++j) {
            for (int m0 = 0; m0 < fin[j].M; m0 += kFinTB) fc.push_back(FinChunk{j, m0});
            for (int m0 = 0; m0 < fin[j].M; m0 += kCoincTB) cc.push_back(FinChunk{j, m0});
        }
        if ((st = upload_vec(ctx, &ctx->d_fin_chunks, fc))) return st;
        if ((st = upload_vec(ctx, &ctx->d_coinc_chunks, cc))) return st;
        ctx->n_fin_chunks = (int)fc.size();
        ctx->n_coinc_chunks = (int)cc.size();
        const std::vector<unsigned long long> zf((size_t)2 * fin.size() * ctx->cfg.n_detectors * kWindowRing, 0ull);
        const std::vector<unsigned long long> zc((size_t)2 * fin.size() * kWindowRing, 0ull);
        if ((st = upload_vec(ctx, &ctx->d_fin_red, zf))) return st;
        if ((st = upload_vec(ctx, &ctx->d_coinc_red, zc))) return st;
    }
    {   // Eq. 10: one tile per 8 templates of every bank with autocorrelations
        std::vector<Xi2Job> xj;
        std::vector<int> xb;
        int xt = 0;
        for (auto& kv : ctx->banks) {
            const BankRT* b = kv.second;
            if (b->ac_half <= 0) continue;
            Xi2Job x{};
            x.tmpl0 = b->tmpl0; x.M = b->M; x.half = b->ac_half; x.ac = b->d_ac; x.den = b->d_ac_den;
            x.zring = b->d_zring; x.zdet_stride = (long long)b->Mpad * b->zlen; x.zlen = b->zlen;
            xj.push_back(x); xb.push_back(xt); xt += (b->M + 7) / 8;
        }
        if ((st = upload_vec(ctx, &ctx->d_xi2, xj)) || (st = upload_vec(ctx, &ctx->d_xi2_base, xb))) return st;
        ctx->n_xi2 = (int)xj.size();
        ctx->xi2_tiles = xt;
    }
    if (split_precision(ctx)) {
        if ((st = build_jobs_split(ctx, n))) return st;
        CK(cudaStreamSynchronize(ctx->stream));
        ctx->jobs_dirty = false;
        ctx->jobs_n = n;
        return LLOID_OK;
    }
    std::vector<FirJob> fj;
    std::vector<int> fb;
    std::vector<UpJob> uj;
    std::vector<int> ub;
    std::vector<ReconJob> rj;
    std::vector<int> rb;
    int ft = 0, ut = 0, rt = 0, max_rlen = 1;
    ctx->top_job_of_bank.assign(ctx->next_bank_id, -1);
    for (auto& kv : ctx->banks) {
        BankRT* b = kv.second;
        for (auto& s : b->sl) {
            FirJob f{};
            f.bases = s.d_bases;
            if (s.D == 1) {
                f.src = ctx->ring0; f.src_det_stride = ctx->ring0_len; f.src_mask = (int)(ctx->ring0_len - 1);
            } else {
                int ri = 0;
                while (ctx->rate_D[ri] != s.D) ++ri;
                f.src = ctx->rate_ring[ri]; f.src_det_stride = ctx->rate_len[ri]; f.src_mask = (int)(ctx->rate_len[ri] - 1);
            }
            f.src_off = s.J / s.D;
            f.dst = s.d_yring; f.dst_det_stride = (long long)s.L * s.y_len; f.dst_mask = s.y_len - 1; f.dst_ld = s.y_len;
            f.L = s.L; f.N = s.N; f.D = s.D; f.c_hi = -s.e_min;
            f.q_count = (int)(n / s.D);
            f.tiles_l = (s.L + 63) / 64; f.tiles_q = (f.q_count + 127) / 128;
            fj.push_back(f); fb.push_back(ft); ft += f.tiles_l * f.tiles_q;

            UpJob u{};
            u.yring = s.d_yring; u.y_det_stride = (long long)s.L * s.y_len; u.y_mask = s.y_len - 1; u.y_ld = s.y_len;
            u.yhat_det_stride = b->yhat_det_stride; u.ldy = (int)ctx->cfg.max_block;
            u.R = s.d_R; u.e_min = s.e_min; u.rlen = s.e_max - s.e_min + 1; u.D = s.D; u.L = s.L;
            u.tiles_k = (int)((n + 255) / 256);
            u.yhat = (char*)b->d_yhat + (size_t)s.row0 * u.ldy * 4;
            u.yhat_lo = nullptr;
            uj.push_back(u); ub.push_back(ut); ut += u.L * u.tiles_k;
            max_rlen = std::max(max_rlen, u.rlen);
        }
        ReconJob r{};
        r.c_re = b->d_cre; r.c_im = b->d_cim; r.yhat = b->d_yhat; r.yhat_lo = nullptr;
        r.yhat_det_stride = b->yhat_det_stride; r.ldy = (int)ctx->cfg.max_block;
        r.Kpad = b->Kpad; r.Mpad = b->Mpad; r.M = b->M; r.tmpl0 = b->tmpl0;
        r.tiles_m = b->Mpad / 64;
        r.tiles_t = (int)(n / 128);
        r.zring = b->d_zring; r.zring_det_stride = (long long)b->Mpad * b->zlen; r.zring_len = b->zlen;
        ctx->top_job_of_bank[b->id] = (int)rj.size();
        rj.push_back(r); rb.push_back(rt); rt += r.tiles_m * r.tiles_t;
    }
    if ((st = upload_vec(ctx, &ctx->d_fir, fj)) || (st = upload_vec(ctx, &ctx->d_fir_base, fb)) ||
        (st = upload_vec(ctx, &ctx->d_up, uj)) || (st = upload_vec(ctx, &ctx->d_up_base, ub)) ||
        (st = upload_vec(ctx, &ctx->d_rec, rj)) || (st = upload_vec(ctx, &ctx->d_rec_base, rb)))
        return st;
    ctx->n_fir = (int)fj.size(); ctx->fir_tiles = ft;
    ctx->n_up = (int)uj.size(); ctx->up_tiles = ut; ctx->up_smem = max_rlen * 4;
    ctx->n_rec = (int)rj.size(); ctx->rec_tiles = rt;
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->jobs_dirty = false;
    ctx->jobs_n = n;
    if (ctx->up_smem > 40 * 1024)
        CK(cudaFuncSetAttribute(k_upsample<StoreF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, ctx->up_smem));
    return LLOID_OK;
}

lloid_status launch_recon_f32(lloid_ctx* ctx, long long k_a, long long n, int det0, int n_det_push, bool store_z,
                              const ReconJob* jobs, const int* base, int n_jobs, int tiles, float* zout) {
    const long long part_stride = (long long)ctx->cfg.n_detectors * ctx->n_slots;
    if (tiles == 0) return LLOID_OK;
    dim3 grid(tiles, n_det_push);
    if (store_z)
        k_recon_f32<true><<<grid, 256, 0, ctx->stream>>>(jobs, base, n_jobs, k_a, (int)n, det0, ctx->cfg.window_samples,
                                                        nullptr, part_stride, ctx->n_slots, tail_ring(ctx), zout);
    else
        k_recon_f32<false><<<grid, 256, 0, ctx->stream>>>(jobs, base, n_jobs, k_a, (int)n, det0,
                                                         ctx->cfg.window_samples, ctx->d_part, part_stride,
                                                         ctx->n_slots, tail_ring(ctx), nullptr);
    CKL();
    return LLOID_OK;
}

template <bool BF16, bool TOP, bool SZ, int F>
cudaError_t launch_lv1(dim3 g, int smem, cudaStream_t st, const LevelJob* jobs, const LevelMaps* maps, const TileInfo* base,
                const int* sched, int n_jobs, int tiles, long long k_a, long long k_b, int det0, int nd, long long W,
                Partial* part, long long part_stride, int n_slots, TailRing tail, float* zout, int* err) {
    return launch_pdl(k_level_tc<BF16, TOP, SZ, F>, g, dim3(LevCfg<BF16, TOP>::THREADS), LevCfg<BF16, TOP>::SMEM, st,
                      jobs, maps, base, sched, n_jobs, tiles, k_a, k_b, det0, nd, W, part, part_stride, n_slots, tail,
                      zout, err);
}
template <bool BF16, bool TOP, bool SZ>
cudaError_t launch_lv_f(int F, dim3 g, int smem, cudaStream_t st, const LevelJob* jobs, const LevelMaps* maps,
                 const TileInfo* base, const int* sched, int n_jobs, int tiles, long long k_a, long long k_b, int det0,
                 int nd, long long W, Partial* part, long long part_stride, int n_slots, TailRing tail, float* zout,
                 int* err) {
#define LV_F(FV) launch_lv1<BF16, TOP, SZ, FV>(g, smem, st, jobs, maps, base, sched, n_jobs, tiles, k_a, k_b, det0, nd, W, \
                                               part, part_stride, n_slots, tail, zout, err)
    switch (F) {
        case 0: return LV_F(0);
        case 2: return LV_F(2);
        case 4: return LV_F(4);
        case 8: return LV_F(8);
        case 16: return LV_F(16);
        case 32: return LV_F(32);
        default: return LV_F(64);
    }
#undef LV_F
}

// One ladder depth and upsampling factor of the split path (depth 0 = f0:
// |z|^2 and window maxima); fslot 0 = no level below, else F = 2^fslot.
lloid_status launch_level(lloid_ctx* ctx, int depth, int fslot, long long k_a, long long n, int det0, int n_det_push,
                          bool store_z, const LevelJob* jobs, const LevelMaps* maps, const TileInfo* base,
                          const int* sched, int grid, int n_jobs, int tiles, float* zout) {
    if (tiles == 0 || n_jobs == 0) return LLOID_OK;
    const bool bf = ctx->cfg.precision == LLOID_BF16_SPLIT;
    const long long part_stride = (long long)ctx->cfg.n_detectors * ctx->n_slots;
    dim3 g(grid);
    const int smem = 0;   // each instantiation launches with its own LevCfg<BF16, TOP>::SMEM
    Partial* part = store_z ? nullptr : ctx->d_part;
    const int F = fslot ? 1 << fslot : 0;
    cudaError_t le = cudaSuccess;
#define LAUNCH_LV(BFV, TOPV, SZ)                                                                                     \
    le = launch_lv_f<BFV, TOPV, SZ>(F, g, smem, ctx->stream, jobs, maps, base, sched, n_jobs, tiles, k_a, k_a + n, det0,   \
                               n_det_push, ctx->cfg.window_samples, part, part_stride, ctx->n_slots, tail_ring(ctx), zout, \
                               ctx->d_err)
    if (depth > 0) { if (bf) LAUNCH_LV(true, false, false); else LAUNCH_LV(false, false, false); }
    else if (store_z) { if (bf) LAUNCH_LV(true, true, true); else LAUNCH_LV(false, true, true); }
    else { if (bf) LAUNCH_LV(true, true, false); else LAUNCH_LV(false, true, false); }
#undef LAUNCH_LV
    CK(le);
    ++ctx->launches;
    return LLOID_OK;
}

// One launch of the f0 kernel (every bank in the f0 form; K <= kF0Kc, two Yhat buffers)
// over the work units of `units` scheduled by `sched` (STORE_Z when zout is given).
lloid_status launch_f0(lloid_ctx* ctx, int cls, const F0Job* jobs, const F0Unit* units, const int* sched, int grid,
                       long long k_a, long long n, int det0, int nd, float* zout) {
    const bool bf = ctx->cfg.precision == LLOID_BF16_SPLIT;
    const int kc = kF0Kc, yb = 2;
    const int smem = f0_smem_bytes(bf, kc, yb);
    const long long part_stride = (long long)ctx->cfg.n_detectors * ctx->n_slots;
    cudaError_t e;
#define F0_ARGS jobs, (const F0Maps*)ctx->d_f0map[cls], units, sched, 0, kc, yb, k_a, \
        (int)n, det0, nd, (long long)ctx->cfg.window_samples, ctx->cfg.snr_threshold, ctx->d_part, part_stride,        \
        ctx->n_slots, tail_ring(ctx), ctx->d_slab, (int)kWindowRing, ctx->cfg.n_detectors, (long long)ctx->M_cap, zout,   \
        ctx->d_err
    if (bf) e = zout ? launch_pdl(k_f0_top<true, true>, dim3(grid), dim3(kF0Threads), smem, ctx->stream, F0_ARGS)
                     : launch_pdl(k_f0_top<true, false>, dim3(grid), dim3(kF0Threads), smem, ctx->stream, F0_ARGS);
    else e = zout ? launch_pdl(k_f0_top<false, true>, dim3(grid), dim3(kF0Threads), smem, ctx->stream, F0_ARGS)
                  : launch_pdl(k_f0_top<false, false>, dim3(grid), dim3(kF0Threads), smem, ctx->stream, F0_ARGS);
#undef F0_ARGS
    CK(e);
    ++ctx->launches;
    return LLOID_OK;
}

// Eq. 7-8 of every bank in the f0 form: Yhat of the push into the banks' planes (k_yhat), a CTA
// per (window group of a bank, detector).
lloid_status launch_yhat(lloid_ctx* ctx, int cls, long long k_a, long long n, int det0, int nd) {
    const bool bf = ctx->cfg.precision == LLOID_BF16_SPLIT;
    const int smem = yhat_smem_bytes(ctx->f0_rall);
    const dim3 grid((unsigned)ctx->n_f0unit[cls], (unsigned)nd);
    cudaError_t e;
#define YH_ARGS (const F0Job*)ctx->d_f0job[cls], (const YupSlice*)ctx->d_f0slices, (const F0Piece*)ctx->d_f0pieces, \
        (const int*)ctx->d_f0bends, (const F0Unit*)ctx->d_f0unit[cls], k_a, (int)n, det0,                         \
        (long long)ctx->cfg.window_samples, ctx->f0_rall
    if (bf) e = launch_pdl(k_yhat<true>, grid, dim3(kYhThreads), smem, ctx->stream, YH_ARGS);
    else e = launch_pdl(k_yhat<false>, grid, dim3(kYhThreads), smem, ctx->stream, YH_ARGS);
#undef YH_ARGS
    CK(e);
    ++ctx->launches;
    return LLOID_OK;
}

// Steps a1-a5 for detectors [det0, det0+nd) whose block [k_a, k_a+n) sits in d_stage (or src).
lloid_status process(lloid_ctx* ctx, int det0, int nd, long long k_a, long long n, const float* src,
                     long long src_det_stride) {
    lloid_status st = build_jobs(ctx, n);
    if (st) return st;
    if (ctx->fault_delay_us > 0) {   // injected: a slow device
        k_delay<<<1, 1, 0, ctx->stream>>>((unsigned long long)ctx->fault_delay_us * 1000ull);
        CKL();
        ctx->fault_delay_us = 0;
    }
    const int n_i = (int)n;
    // a0 ingest
    {
        StageTimer tm(ctx, 0);
        dim3 grid((unsigned)std::min<long long>((n + 255) / 256, 1024), nd);
        CK(launch_pdl(k_ingest, grid, dim3(256), 0, ctx->stream, src, src_det_stride, ctx->ring0, ctx->ring0_len,
                      (int)(ctx->ring0_len - 1), k_a, n_i, det0, ctx->s_hi[0], ctx->s_lo[0], 2 * ctx->s_len[0],
                      (int)ctx->s_len[0], (int)ctx->cfg.precision));
        ++ctx->launches;
    }
    // a1 downsample to every rate
    {
        StageTimer tm(ctx, 1);
        DownParams p{};
        p.n_rates = ctx->n_rates;
        for (int r = 0; r < ctx->n_rates; ++r) {
            p.w[r] = ctx->w_down[r]; p.dst[r] = ctx->rate_ring[r]; p.dst_det_stride[r] = ctx->rate_len[r];
            p.dst_mask[r] = (int)(ctx->rate_len[r] - 1); p.D[r] = ctx->rate_D[r];
            p.s_hi[r] = ctx->s_hi[r + 1]; p.s_lo[r] = ctx->s_lo[r + 1];
            p.s_det_stride[r] = 2 * ctx->s_len[r + 1]; p.s_len[r] = (int)ctx->s_len[r + 1];
        }
        p.mode = ctx->cfg.precision;
        int blocks = 0;
        for (int r = 0; r < ctx->n_rates; ++r) {
            p.blk0[r] = blocks;
            const int qb = down_qb(ctx->rate_D[r]);
            blocks += (int)((n / ctx->rate_D[r] + qb - 1) / qb);
        }
        p.blk0[ctx->n_rates] = blocks;
        if (blocks > 0) {
            CK(launch_pdl(k_downsample, dim3((unsigned)blocks, nd), dim3(kDownThreads), ctx->down_smem, ctx->stream, p,
                          (const float*)ctx->ring0, ctx->ring0_len, (int)(ctx->ring0_len - 1), k_a, n_i,
                          (int)ctx->cfg.n_down, det0));
            ++ctx->launches;
        }
    }
    if (ctx->banks.empty()) return LLOID_OK;
    if (!split_precision(ctx)) {
        // a2 basis FIR (FP32)
        if (ctx->fir_tiles) {
            StageTimer tm(ctx, 2);
            dim3 grid(ctx->fir_tiles, nd);
            k_fir_f32<<<grid, 256, 0, ctx->stream>>>(ctx->d_fir, ctx->d_fir_base, ctx->n_fir, k_a, det0);
            CKL();
        }
        // a4 (slice part) composed upsampler of each slice into Yhat
        if (ctx->up_tiles) {
            StageTimer tm(ctx, 3);
            dim3 grid(ctx->up_tiles, nd);
            k_upsample<StoreF32><<<grid, 256, ctx->up_smem, ctx->stream>>>(ctx->d_up, ctx->d_up_base, ctx->n_up, k_a,
                                                                         n_i, det0, StoreF32{});
            CKL();
        }
        // a3 + a5 reconstruction with fused window maxima
        {
            StageTimer tm(ctx, 4);
            st = launch_recon_f32(ctx, k_a, n, det0, nd, false, ctx->d_rec, ctx->d_rec_base, ctx->n_rec,
                                  ctx->rec_tiles, nullptr);
        }
        if (st) return st;
    } else {
        // a2 basis FIR on the tensor cores
        if (ctx->firtc_tiles) {
            StageTimer tm(ctx, 2);
            const int v = nd == 1 ? 0 : 1;
            if (nd != 1 && nd != ctx->cfg.n_detectors) return fail(ctx, LLOID_EINVAL, "push of %d detectors", nd);
            dim3 g(ctx->fir_grid[v]);
            if (ctx->cfg.precision == LLOID_BF16_SPLIT)
                CK(launch_pdl(k_fir_tc<true>, g, dim3(192), ctx->firtc_smem, ctx->stream, (const FirTcJob*)ctx->d_firtc,
                              (const FirMaps*)ctx->d_firmaps, (const TileInfo*)ctx->d_firtc_base,
                              (const int*)ctx->d_fir_sched[v], ctx->n_firtc, ctx->firtc_tiles, k_a, det0, nd,
                              ctx->firtc_strip, ctx->firtc_stages, ctx->d_err));
            else
                CK(launch_pdl(k_fir_tc<false>, g, dim3(192), ctx->firtc_smem, ctx->stream, (const FirTcJob*)ctx->d_firtc,
                              (const FirMaps*)ctx->d_firmaps, (const TileInfo*)ctx->d_firtc_base,
                              (const int*)ctx->d_fir_sched[v], ctx->n_firtc, ctx->firtc_tiles, k_a, det0, nd,
                              ctx->firtc_strip, ctx->firtc_stages, ctx->d_err));
            CKL();
        }
        // a3 + a4: reconstruction rate by rate with the Eq. 7-8 ladder, lowest rate first
        {
            StageTimer tm(ctx, 3);
            for (int d = ctx->max_depth - 1; d >= 1; --d)
                for (int fs = 0; fs < lloid_ctx::kFSlots; ++fs) {
                    const int tb = d * lloid_ctx::kFSlots + fs;
                    const int v = nd == 1 ? 0 : 1;
                    if ((st = launch_level(ctx, d, fs, k_a, n, det0, nd, false, ctx->d_lev[tb], ctx->d_levmaps[tb],
                                           ctx->d_lev_base[tb], ctx->d_lev_sched[tb][v], ctx->lev_grid[tb][v],
                                           ctx->n_lev[tb], ctx->lev_tiles[tb], nullptr)))
                        return st;
                }
            // the f0 form's banks: every slice's basis outputs brought up to f0 (Eq. 7-8)
            for (int cls = 0; cls < lloid_ctx::kF0Classes; ++cls)
                if (ctx->n_f0unit[cls] && (st = launch_yhat(ctx, cls, k_a, n, det0, nd))) return st;
        }
        // top level (f0) + a5 window maxima; the f0 form's banks: Eq. 6 + a5 in one kernel
        {
            StageTimer tm(ctx, 4);
            const int v = nd == 1 ? 0 : 1;
            for (int fs = 0; fs < lloid_ctx::kFSlots && !st; ++fs)
                st = launch_level(ctx, 0, fs, k_a, n, det0, nd, false, ctx->d_lev[fs], ctx->d_levmaps[fs],
                                  ctx->d_lev_base[fs], ctx->d_lev_sched[fs][v], ctx->lev_grid[fs][v], ctx->n_lev[fs],
                                  ctx->lev_tiles[fs], nullptr);
            for (int cls = 0; cls < lloid_ctx::kF0Classes && !st; ++cls)
                if (ctx->n_f0unit[cls])
                    st = launch_f0(ctx, cls, ctx->d_f0job[cls], ctx->d_f0unit[cls], ctx->d_f0sched[cls][v],
                                   ctx->f0_grid[cls][v], k_a, n, det0, nd, nullptr);
        }
        if (st) return st;
    }
    // a5 finalise completed windows
    const long long W = ctx->cfg.window_samples;
    StageTimer tmf(ctx, 5);
    const long long w_first = k_a / W, w_end = (k_a + n) / W;   // windows completed by this push
    if (w_end > w_first && ctx->n_fin > 0) {
        dim3 grid(ctx->n_fin_chunks, nd, (unsigned)(w_end - w_first));
        // windows of the f0 form's banks that the f0 kernel finished (pushes that start on a window)
        const long long fused_from = (k_a % W == 0 && ctx->cfg.window_overlap == 0) ? w_first : (1LL << 62);
        CK(launch_pdl(k_finalize, grid, dim3(256), 0, ctx->stream, (const FinJob*)ctx->d_finj,
                      (const FinChunk*)ctx->d_fin_chunks, (const Partial*)ctx->d_part,
                      (long long)ctx->cfg.n_detectors * ctx->n_slots, ctx->n_slots, ctx->tiles_per_window, w_first,
                      ctx->cfg.snr_threshold, ctx->d_slab, (int)kWindowRing, ctx->cfg.n_detectors,
                      (long long)ctx->M_cap, det0, ctx->d_fin_red, fused_from, tail_ring(ctx)));
        ++ctx->launches;
    }
    // Eq. 10 for the windows whose triggers now have d samples of z past the window end
    if (ctx->n_xi2 > 0) {
        const long long w_ready = (k_a + n - ctx->xi2_half_max) / W;   // windows < w_ready are ready
        for (int d = det0; d < det0 + nd; ++d) {
            long long w_lo = std::max(ctx->xi2_next[d], w_ready - (long long)kWindowRing);
            if (w_ready <= w_lo) continue;
            CK(launch_pdl(k_xi2, dim3(ctx->xi2_tiles, 1, (unsigned)(w_ready - w_lo)), dim3(256), 0, ctx->stream,
                          (const Xi2Job*)ctx->d_xi2, (const int*)ctx->d_xi2_base, ctx->n_xi2, w_lo, W, d,
                          ctx->d_slab, (int)kWindowRing, ctx->cfg.n_detectors, (long long)ctx->M_cap));
            ++ctx->launches;
            ctx->xi2_next[d] = w_ready;
        }
    }
    // coincidence and clustering for the windows every detector has ready
    {
        long long w_all = -1;
        for (int d = 0; d < ctx->cfg.n_detectors; ++d) {
            const bool pushed = d >= det0 && d < det0 + nd;
            long long r = ctx->n_xi2 > 0 ? ctx->xi2_next[d] : (pushed ? (k_a + n) / W : ctx->fin[d] + 1);
            w_all = (w_all < 0) ? r : std::min(w_all, r);
        }
        const int ndt = ctx->cfg.n_detectors;
        long long w_lo = std::max(ctx->coinc_next, w_all - (long long)kWindowRing);
        if (ndt >= 2 && ndt <= 32 && ctx->n_fin > 0 && w_all > w_lo) {
            CK(launch_pdl(k_coinc, dim3(ctx->n_coinc_chunks, (unsigned)(w_all - w_lo)), dim3(256), 0, ctx->stream,
                          (const FinJob*)ctx->d_finj, (const FinChunk*)ctx->d_coinc_chunks, w_lo, ndt,
                          (int)ctx->cfg.coinc_window, (const SlabEntry*)ctx->d_slab, (int)kWindowRing,
                          (long long)ctx->M_cap, ctx->d_events, ctx->bank_cap, ctx->d_coinc_red));
            ++ctx->launches;
            if (ctx->bg_nsnr > 0) {
                int mmax = 1;
                for (auto& kv : ctx->banks) mmax = std::max(mmax, kv.second->M);
                CK(launch_pdl(k_background, dim3(ctx->n_fin, (unsigned)(w_all - w_lo), (unsigned)((mmax + 255) / 256)),
                              dim3(256), 0, ctx->stream, (const FinJob*)ctx->d_finj, w_lo, ndt,
                              (int)ctx->cfg.coinc_window, (const SlabEntry*)ctx->d_slab, (int)kWindowRing,
                              (long long)ctx->M_cap, (const float*)ctx->d_bg_edges, ctx->bg_nsnr,
                              (const float*)(ctx->d_bg_edges + ctx->bg_nsnr + 1), ctx->bg_nxi2));
                ++ctx->launches;
            }
        }
        if (w_all > ctx->coinc_next) ctx->coinc_next = w_all;
    }
    return LLOID_OK;
}

lloid_status push_one(lloid_ctx* ctx, int det0, int nd, long long t0, const float* block, long long n,
                      int is_device_ptr);

lloid_status push_common(lloid_ctx* ctx, int det0, int nd, long long t0, const float* block, long long n,
                         int is_device_ptr) {
    if (!block) return fail(ctx, LLOID_EINVAL, "block is NULL");
    if (n <= 0 || n % kTileT || n > ctx->cfg.max_block)
        return fail(ctx, LLOID_EINVAL, "block length %lld must be a positive multiple of %d and <= max_block %lld",
                    n, kTileT, (long long)ctx->cfg.max_block);
    if (ctx->fault_drop > 0) {   // injected: the block is lost on its way
        --ctx->fault_drop;
        return LLOID_OK;
    }
    const long long p0 = ctx->pos[det0];
    bool gap = true;
    for (int d = det0; d < det0 + nd; ++d) gap = gap && ctx->pos[d] == p0 && p0 < t0 && (t0 - p0) % kTileT == 0;
    if (gap && (ctx->cfg.flags & LLOID_FLAG_FILL_GAPS)) {   // the missing samples as zeros
        if (!ctx->d_zero) {
            lloid_status st = dalloc(ctx, &ctx->d_zero, (size_t)ctx->cfg.n_detectors * ctx->cfg.max_block * 4, nullptr,
                                     &ctx->state_bytes);
            if (st) return st;
        }
        for (long long k = p0; k < t0;) {
            const long long m = std::min<long long>(ctx->cfg.max_block, t0 - k);
            lloid_status st = push_one(ctx, det0, nd, k, ctx->d_zero, m, 1);
            if (st) return st;
            k += m;
        }
    }
    return push_one(ctx, det0, nd, t0, block, n, is_device_ptr);
}

lloid_status push_one(lloid_ctx* ctx, int det0, int nd, long long t0, const float* block, long long n,
                      int is_device_ptr) {
    for (int d = det0; d < det0 + nd; ++d)
        if (ctx->pos[d] != t0)
            return fail(ctx, LLOID_EGAP, "detector %d stream ends at %lld, push starts at %lld", d, ctx->pos[d], t0);
    const float* src = block;
    long long src_stride = n;
    if (!is_device_ptr) {
        const int i = ctx->stage_i;
        CK(cudaEventSynchronize(ctx->stage_ev[i]));
        std::memcpy(ctx->h_stage[i], block, (size_t)nd * n * sizeof(float));
        CK(cudaMemcpyAsync(ctx->d_stage, ctx->h_stage[i], (size_t)nd * n * sizeof(float), cudaMemcpyHostToDevice,
                           ctx->stream));
        CK(cudaEventRecord(ctx->stage_ev[i], ctx->stream));
        ctx->stage_i ^= 1;
        src = ctx->d_stage;
    }
    lloid_status st = process(ctx, det0, nd, t0, n, src, src_stride);
    if (st) return st;
    const long long W = ctx->cfg.window_samples;
    for (int d = det0; d < det0 + nd; ++d) {
        ctx->pos[d] = t0 + n;
        ctx->fin[d] = (t0 + n) / W - 1;
        ctx->last_n[d] = n;
    }
    CK(cudaEventRecord(ctx->done_ev, ctx->stream));
    return LLOID_OK;
}

// Wait for an event: polled without sleeping for the first 2 ms (a pull usually
// waits well under that), then every 50 us; timeout_ms < 0 waits without limit.
lloid_status wait_event(lloid_ctx* ctx, cudaEvent_t ev, int timeout_ms) {
    auto t_start = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return LLOID_OK;
        if (e != cudaErrorNotReady) return fail(ctx, LLOID_ECUDA, "device error: %s", cudaGetErrorString(e));
        auto el = std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t_start);
        if (timeout_ms >= 0 && el.count() >= 1000LL * timeout_ms)
            return fail(ctx, LLOID_ETIMEOUT, "GPU work not done after %d ms", timeout_ms);
        if (el.count() < 2000) std::this_thread::yield();
        else std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}
lloid_status wait_done(lloid_ctx* ctx, int timeout_ms) { return wait_event(ctx, ctx->done_ev, timeout_ms); }

// Form of a bank on the split path (LLOID_FLAG_FORM_*), from an estimate of the device time per
// detector-second and 128 templates in units of one 128 x 128 x 16 MMA (64 cycles): per 128-sample
// tile the MMAs of C Y (4, or 6 for BF16, per 16 bases) and of an Eq. 8 window (6 per 16 window
// rows), an epilogue share, the Acc planes that a ladder level below f0 writes and the next level
// reads (about 256 KB per tile at a 148th of the HBM bandwidth); in the f0 form the MMAs over the
// bank's bases packed (K = their count rounded up to 16) and the upsampling of the basis outputs,
// shared by the bank's template tiles.  The f0 form needs K <= 96, at most 1024 templates and no
// Eq. 10 autocorrelations (the f0 kernel keeps no SNR history).
bool f0_form_possible(const lloid_ctx* ctx, const BankRT* b, int ac_half) {
    const bool bf = ctx->cfg.precision == LLOID_BF16_SPLIT;
    if (f0_smem_bytes(bf, kF0Kc, 2) > ctx->smem_optin) return false;
    int k = 0, rall = 0;
    for (const SliceRT& s : b->sl) {
        k += s.L;
        const int rlen = s.e_max - s.e_min + 1;
        rall += rlen;
        if ((127 + rlen - 1) / s.D + 2 > kF0StageRows) return false;
    }
    return (k + 15) / 16 * 16 <= kF0Kc && b->Mpad <= 128 * kF0MaxTm && ac_half == 0 && rall <= kF0RAll &&
           (int)b->sl.size() <= kF0MaxSlices;
}

int choose_form(const lloid_ctx* ctx, const BankRT* b, const std::vector<int>& ladder, int ac_half) {
    const lloid_config& c = ctx->cfg;
    if (c.flags & LLOID_FLAG_FORM_LADDER) return 0;
    if (!f0_form_possible(ctx, b, ac_half)) return 0;
    if (c.flags & LLOID_FLAG_FORM_F0) return 1;
    const double mk = c.precision == LLOID_BF16_SPLIT ? 6.0 : 4.0, epi = 20.0, planes = 190.0;
    const int nl = (int)ladder.size();
    std::vector<int> k16(nl, 0);
    int k_all = 0;
    for (const SliceRT& s : b->sl) {
        const int j = (int)(std::find(ladder.begin(), ladder.end(), s.rate) - ladder.begin());
        k16[j] += (s.L + 15) / 16;
        k_all += s.L;
    }
    const int k16_all = (k_all + 15) / 16;
    const double up_cols = (double)k16_all * 16;
    double lad = 0.0;
    for (int j = 0; j < nl; ++j) {
        double mm = mk * k16[j] + epi;
        if (j > 0) {
            const int F = ladder[j] / ladder[j - 1];
            mm += 6.0 * ((win_rows(F) + win_shift_max(F) + 15) / 16);
        }
        if (j < nl - 1) mm += planes;
        lad += ((double)ladder[j] / 128.0 + 2.0) * mm;
    }
    // f0 form: per tile the MMAs over all bases and, shared by the bank's template groups, the
    // upsampled rows (about 24 multiply-adds per basis and row for 128 threads: ~0.2 MMA each)
    const double f0 = (double)c.f0 / 128.0 * (mk * k16_all + epi + 0.2 * up_cols / (b->Mpad / 128.0));
    const double ratio = c.form_ratio > 0.f ? c.form_ratio : 1.0;
    return f0 < ratio * lad ? 1 : 0;
}

// Split path: ladder levels, 8-phase expanded bases for the tensor-core FIR,
// per-level coefficient blocks, operand rings and Acc planes.  Uploads
// everything and accounts the bytes in b.
lloid_status prepare_split_bank(lloid_ctx* ctx, const lloid_bank_desc* bd, const std::vector<int>& ladder,
                                BankRT* b, bool dry_run, size_t* need_out) {
    const lloid_config& c = ctx->cfg;
    const bool bf = c.precision == LLOID_BF16_SPLIT;
    const int nd = c.n_detectors;
    const int nl = (int)ladder.size();
    const int M = bd->n_templates;
    const size_t es = 2;
    std::vector<LevelRT> lev(nl);
    for (int j = 0; j < nl; ++j) { lev[j].rate = ladder[j]; lev[j].D = c.f0 / ladder[j]; }
    lev[nl - 1].Lambda = 0;
    for (int j = nl - 2; j >= 0; --j) lev[j].Lambda = lev[j + 1].Lambda + c.n_up * lev[j].D;
    // Every rate keeps an operand ring of its slices' FIR output (16-aligned columns per slice).
    // The ladder form reconstructs at every rate through that rate's coefficients.  The f0 form
    // has one more level at f0, `top`: every slice's basis outputs brought up to f0, packed
    // slice after slice, and the coefficients of every slice in the same columns.
    const bool f0form = b->form == 1;
    std::vector<FirSliceRT> fs(bd->n_slices);
    int tk = 0;
    for (int s = 0; s < bd->n_slices; ++s) {
        const lloid_slice& sl = bd->slices[s];
        const int j = (int)(std::find(ladder.begin(), ladder.end(), sl.rate) - ladder.begin());
        const int D = c.f0 / sl.rate;
        fs[s].level = j;
        fs[s].col = lev[j].K;
        lev[j].K += (sl.n_basis + 15) / 16 * 16;
        b->sl[s].tcol = tk;
        tk += sl.n_basis;
        const long long JD = sl.j_start / D;
        int Np = sl.n_taps;
        while (((Np - 1 + JD) % 8 + 8) % 8) ++Np;
        fs[s].Np = Np;
        fs[s].Kp = (Np + 7 + 63) / 64 * 64;
        fs[s].Mtiles = (8 * sl.n_basis + 127) / 128;
        if (2 * (8 * kFirNC + fs[s].Kp) > 40 * 1024)
            return fail(ctx, LLOID_EINVAL, "slice %d: %d taps exceed the tensor-core FIR strip limit", s, sl.n_taps);
    }
    LevelRT top;
    const int npl = bf ? 4 : 2;
    if (f0form) {
        top.rate = c.f0;
        top.K = (tk + 15) / 16 * 16;
    }
    size_t need = 0;
    for (int j = 0; j < nl; ++j) {
        LevelRT& L = lev[j];
        L.Kp = (L.K + 63) / 64 * 64;
        const long long cnt = (c.max_block - 1 + 2LL * L.Lambda) / L.D + 2;
        L.R = (int)next_pow2(cnt + 128 + 64);
        if (j < nl - 1 && !f0form) L.acc_cols = 128 * (int)((cnt + 127 + 127) / 128 + 2);   // every column a tile writes
        if (!f0form) need += (size_t)b->Mpad * L.Kp * es * (bf ? 4 : 2);
        need += (size_t)nd * 2 * L.R * L.Kp * es * 2;
        need += (size_t)nd * 4 * b->Mpad * L.acc_cols * 2;
    }
    if (f0form) {
        need += (size_t)npl * top.K * b->Mpad * es;
        need += (size_t)nd * 2 * top.K * c.max_block * es;   // Yhat planes
        for (const SliceRT& r : b->sl) need += r.R.size() * 4;
    }
    for (auto& f : fs) need += (size_t)f.Mtiles * 128 * f.Kp * es * (bf ? 2 : 1);
    *need_out = need;
    if (dry_run) return LLOID_OK;

    lloid_status st;
    // expanded bases: A'[(8l + t)][j] = u_l[t + N' - 1 - j] inside the filter, else 0
    for (int s = 0; s < bd->n_slices; ++s) {
        const lloid_slice& sl = bd->slices[s];
        FirSliceRT& f = fs[s];
        const size_t rows = (size_t)f.Mtiles * 128;
        std::vector<double> A(rows * f.Kp, 0.0);
        for (int l = 0; l < sl.n_basis; ++l)
            for (int t = 0; t < 8; ++t)
                for (int jj = 0; jj < f.Kp; ++jj) {
                    const int m = t + f.Np - 1 - jj;
                    if (m >= 0 && m < sl.n_taps) A[(size_t)(8 * l + t) * f.Kp + jj] = sl.bases[(size_t)l * sl.n_taps + m];
                }
        std::vector<uint16_t> hi, lo, dummy_h, dummy_l;
        pack_coeffs_tc(bf, A, A, (int)rows, f.Kp, &hi, &dummy_h, &lo, &dummy_l);
        if ((st = dalloc(ctx, (uint16_t**)&f.d_a, hi.size() * 2, &b->allocs, &b->bytes))) return st;
        CK(cudaMemcpyAsync(f.d_a, hi.data(), hi.size() * 2, cudaMemcpyHostToDevice, ctx->stream));
        if (bf) {
            if ((st = dalloc(ctx, (uint16_t**)&f.d_a_lo, lo.size() * 2, &b->allocs, &b->bytes))) return st;
            CK(cudaMemcpyAsync(f.d_a_lo, lo.data(), lo.size() * 2, cudaMemcpyHostToDevice, ctx->stream));
        }
        CK(cudaStreamSynchronize(ctx->stream));
    }
    // coefficient blocks [Mpad][K'pad] (FP16, or BF16 hi + lo) and an operand ring of a level;
    // `col` gives each slice's first column (a slice whose col is < 0 has no columns there)
    auto fill_level = [&](LevelRT& L, bool with_c, const std::vector<int>& col) -> lloid_status {
        if (L.Kp == 0) return LLOID_OK;
        if (with_c) {
            std::vector<double> cre((size_t)b->Mpad * L.Kp, 0.0), cim((size_t)b->Mpad * L.Kp, 0.0);
            for (int s = 0; s < bd->n_slices; ++s) {
                if (col[s] < 0) continue;
                const lloid_slice& sl = bd->slices[s];
                for (int i = 0; i < M; ++i)
                    for (int l = 0; l < sl.n_basis; ++l) {
                        cre[(size_t)i * L.Kp + col[s] + l] = sl.coeffs[(size_t)(2 * i) * sl.n_basis + l];
                        cim[(size_t)i * L.Kp + col[s] + l] = sl.coeffs[(size_t)(2 * i + 1) * sl.n_basis + l];
                    }
            }
            std::vector<uint16_t> hre, him, lre, lim;
            pack_coeffs_tc(bf, cre, cim, b->Mpad, L.Kp, &hre, &him, &lre, &lim);
            void** dst[4] = {&L.d_cre, &L.d_cim, &L.d_cre_lo, &L.d_cim_lo};
            std::vector<uint16_t>* srcv[4] = {&hre, &him, &lre, &lim};
            for (int q = 0; q < 4; ++q) {
                if (srcv[q]->empty()) continue;
                lloid_status e;
                if ((e = dalloc(ctx, (uint16_t**)dst[q], srcv[q]->size() * 2, &b->allocs, &b->bytes))) return e;
                CK(cudaMemcpyAsync(*dst[q], srcv[q]->data(), srcv[q]->size() * 2, cudaMemcpyHostToDevice, ctx->stream));
            }
        }
        const size_t rb = (size_t)nd * 2 * L.R * L.Kp * 2;
        lloid_status e;
        if ((e = dalloc(ctx, &L.d_yhi, rb, &b->allocs, &b->bytes))) return e;
        if ((e = dalloc(ctx, &L.d_ylo, rb, &b->allocs, &b->bytes))) return e;
        CK(cudaStreamSynchronize(ctx->stream));
        return LLOID_OK;
    };
    for (int j = 0; j < nl; ++j) {
        std::vector<int> col(bd->n_slices, -1);
        for (int s = 0; s < bd->n_slices; ++s)
            if (fs[s].level == j) col[s] = fs[s].col;
        if ((st = fill_level(lev[j], !f0form, col))) return st;
        if (lev[j].acc_cols > 0) {   // zeroed: columns no tile has written read as 0
            if ((st = dalloc(ctx, &lev[j].d_accp, (size_t)nd * 4 * b->Mpad * lev[j].acc_cols * 2, &b->allocs,
                             &b->bytes)))
                return st;
        }
    }
    if (f0form) {
        // coefficients of every slice in the packed columns, as time-blocked planes
        // [re hi, im hi, (re lo, im lo)][K/8][Mpad][8] (the layout of a no-swizzle K-major operand)
        std::vector<double> cre((size_t)b->Mpad * top.K, 0.0), cim((size_t)b->Mpad * top.K, 0.0);
        for (int s = 0; s < bd->n_slices; ++s) {
            const lloid_slice& sl = bd->slices[s];
            for (int i = 0; i < M; ++i)
                for (int l = 0; l < sl.n_basis; ++l) {
                    cre[(size_t)i * top.K + b->sl[s].tcol + l] = sl.coeffs[(size_t)(2 * i) * sl.n_basis + l];
                    cim[(size_t)i * top.K + b->sl[s].tcol + l] = sl.coeffs[(size_t)(2 * i + 1) * sl.n_basis + l];
                }
        }
        std::vector<uint16_t> hre, him, lre, lim;
        pack_coeffs_tc(bf, cre, cim, b->Mpad, top.K, &hre, &him, &lre, &lim);
        std::vector<uint16_t>* pl[4] = {&hre, &him, &lre, &lim};
        std::vector<uint16_t> blk((size_t)npl * top.K * b->Mpad);
        for (int q = 0; q < npl; ++q)
            for (int i = 0; i < b->Mpad; ++i)
                for (int k = 0; k < top.K; ++k)
                    blk[(((size_t)q * (top.K / 8) + k / 8) * b->Mpad + i) * 8 + k % 8] = (*pl[q])[(size_t)i * top.K + k];
        if ((st = dalloc(ctx, &b->d_cblk, blk.size() * 2, &b->allocs, &b->bytes))) return st;
        CK(cudaMemcpyAsync(b->d_cblk, blk.data(), blk.size() * 2, cudaMemcpyHostToDevice, ctx->stream));
        if ((st = dalloc(ctx, &b->d_yf0, (size_t)nd * 2 * top.K * c.max_block * 2, &b->allocs, &b->bytes))) return st;
        CK(cudaStreamSynchronize(ctx->stream));
        for (SliceRT& r : b->sl) {   // composed upsampler of every slice (Eq. 7-8 ladder from its rate; [1] at f0)
            std::vector<float> Rf(r.R.begin(), r.R.end());
            if ((st = dalloc(ctx, &r.d_R, Rf.size() * 4, &b->allocs, &b->bytes))) return st;
            CK(cudaMemcpyAsync(r.d_R, Rf.data(), Rf.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
        }
    }
    b->lev = lev;
    b->top = top;
    b->fs = fs;
    return LLOID_OK;
}

// Checkpoint layout: header words describing the context, then every
// stateful device segment in a fixed order.
struct Segment { void* p; size_t bytes; };

void state_layout(lloid_ctx* ctx, std::vector<long long>* hdr, std::vector<Segment>* seg) {
    const lloid_config& c = ctx->cfg;
    const int nd = c.n_detectors;
    hdr->clear();
    seg->clear();
    long long h[] = {0x4C4C4F4944535431LL, 5, c.f0, nd, c.n_down, c.n_up, c.window_samples, c.precision,
                     c.max_block, c.max_history, c.min_rate, (long long)ctx->banks.size(), ctx->M_used,
                     ctx->M_cap, ctx->n_slots};
    hdr->assign(h, h + sizeof h / sizeof h[0]);
    for (int d = 0; d < nd; ++d) {
        hdr->push_back(ctx->pos[d]); hdr->push_back(ctx->fin[d]); hdr->push_back(ctx->last_n[d]);
        hdr->push_back(ctx->xi2_next[d]);
    }
    hdr->push_back(ctx->coinc_next);
    seg->push_back({ctx->ring0, (size_t)nd * ctx->ring0_len * 4});
    for (int r = 0; r < ctx->n_rates; ++r) seg->push_back({ctx->rate_ring[r], (size_t)nd * ctx->rate_len[r] * 4});
    for (int r = 0; r <= kMaxRates; ++r)
        if (ctx->s_hi[r]) {
            seg->push_back({ctx->s_hi[r], (size_t)nd * 2 * ctx->s_len[r] * 2});
            seg->push_back({ctx->s_lo[r], (size_t)nd * 2 * ctx->s_len[r] * 2});
        }
    seg->push_back({ctx->d_part, (size_t)ctx->M_cap * nd * ctx->n_slots * sizeof(Partial)});
    seg->push_back({ctx->d_tail, (size_t)ctx->M_cap * nd * ctx->n_tail * sizeof(Partial)});
    seg->push_back({ctx->d_slab, (size_t)kWindowRing * nd * ctx->M_cap * sizeof(SlabEntry)});
    if (ctx->d_events) seg->push_back({ctx->d_events, (size_t)kWindowRing * ctx->bank_cap * sizeof(EventEntry)});
    for (auto& kv : ctx->banks) {
        const BankRT* b = kv.second;
        hdr->push_back(kv.first); hdr->push_back(b->M); hdr->push_back(b->tmpl0); hdr->push_back((long long)b->sl.size());
        hdr->push_back(b->ac_half);
        if (b->d_zring) seg->push_back({b->d_zring, (size_t)nd * b->Mpad * b->zlen * 4});
        if (b->d_bg) seg->push_back({b->d_bg, (size_t)nd * ctx->bg_nsnr * ctx->bg_nxi2 * 4});
        for (const auto& sl : b->sl) {
            hdr->push_back(sl.rate); hdr->push_back(sl.J); hdr->push_back(sl.N); hdr->push_back(sl.L);
            if (sl.d_yring) seg->push_back({sl.d_yring, (size_t)nd * sl.L * sl.y_len * 4});
        }
        for (const auto& L : b->lev)
            if (L.d_yhi) {
                seg->push_back({L.d_yhi, (size_t)nd * 2 * L.R * L.Kp * 2});
                seg->push_back({L.d_ylo, (size_t)nd * 2 * L.R * L.Kp * 2});
            }
    }
    hdr->push_back((long long)seg->size());
    for (auto& x : *seg) hdr->push_back((long long)x.bytes);
}

// A kernel whose bounded wait expired leaves a code in d_err (see kernels_tc.cuh).
lloid_status check_kernel_err(lloid_ctx* ctx) {
    int e = 0;
    CK(cudaMemcpyAsync(&e, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (e) return fail(ctx, LLOID_ETIMEOUT, "a kernel wait expired (code %d); results of the last pushes are invalid", e);
    return LLOID_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void lloid_config_default(lloid_config* c) {
    if (!c) return;
    std::memset(c, 0, sizeof *c);
    c->f0 = 2048;
    c->n_detectors = 1;
    c->n_down = 32;
    c->n_up = 8;
    c->window_samples = 2048;
    c->window_overlap = 0;
    c->snr_threshold = 4.0f;
    c->precision = LLOID_FP32;
    c->max_block = 16384;
    c->max_history = 128LL * 2048;
    c->min_rate = 32;
    c->device = 0;
    c->hbm_budget_bytes = 0;
    c->cuda_stream = nullptr;
    c->flags = 0;
    c->coinc_window = 66;   // (0.0273 + 0.005) s at 2048 Hz
    c->form_ratio = 1.0f;
    c->fir_ctas = 0;
}

const char* lloid_strerror(lloid_status st) {
    switch (st) {
        case LLOID_OK: return "ok";
        case LLOID_EINVAL: return "invalid argument";
        case LLOID_ENOMEM: return "out of memory";
        case LLOID_EBUDGET: return "HBM budget exceeded";
        case LLOID_EGAP: return "discontinuous push (t0 is not the stream end)";
        case LLOID_ENOTREADY: return "window not yet covered by pushed data";
        case LLOID_ETIMEOUT: return "timed out waiting for the GPU";
        case LLOID_ECUDA: return "CUDA error";
        case LLOID_ERANGE: return "output capacity too small";
        case LLOID_EEXPIRED: return "window no longer retained";
    }
    return "unknown status";
}

const char* lloid_last_error(const lloid_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t lloid_launch_count(const lloid_ctx* ctx) { return ctx ? ctx->launches : 0; }

lloid_status lloid_inject_fault(lloid_ctx* ctx, int32_t kind, int64_t count) {
    if (!ctx) return LLOID_EINVAL;
    if (count < 0) return fail(ctx, LLOID_EINVAL, "negative fault count");
    switch (kind) {
        case LLOID_FAULT_ALLOC: ctx->fault_alloc = count; return LLOID_OK;
        case LLOID_FAULT_DROP_BLOCK: ctx->fault_drop = count; return LLOID_OK;
        case LLOID_FAULT_DELAY: ctx->fault_delay_us = std::min<int64_t>(count, 10000000); return LLOID_OK;
        case LLOID_FAULT_WAIT_EXPIRY:
            if (count == 0) return LLOID_OK;
            CK(cudaSetDevice(ctx->cfg.device));
            k_wait_expiry_check<<<1, 32, 0, ctx->stream>>>(ctx->d_err, 90,
                                                          (unsigned long long)std::min<int64_t>(count, 1000000) * 1000ull);
            CKL();
            CK(cudaEventRecord(ctx->done_ev, ctx->stream));
            return LLOID_OK;
    }
    return fail(ctx, LLOID_EINVAL, "unknown fault kind %d", kind);
}

lloid_status lloid_autotune(const lloid_config* cfg, const lloid_bank_desc* banks, int32_t n_banks, int64_t n,
                            int32_t reps, lloid_tuning* out) {
    if (!cfg || !banks || n_banks < 1 || !out || reps < 1 || n <= 0 || n > cfg->max_block || n % kTileT)
        return LLOID_EINVAL;
    std::memset(out, 0, sizeof *out);
    const int nd = cfg->n_detectors;
    float* zeros = nullptr;
    {
        cudaError_t e = cudaSetDevice(cfg->device);
        if (e == cudaSuccess) e = cudaMalloc(&zeros, (size_t)nd * n * sizeof(float));
        if (e == cudaSuccess) e = cudaMemset(zeros, 0, (size_t)nd * n * sizeof(float));
        if (e != cudaSuccess) { cudaFree(zeros); return e == cudaErrorMemoryAllocation ? LLOID_ENOMEM : LLOID_ECUDA; }
    }
    // time one candidate: a scratch context, every bank, two warm-up pushes, `reps` timed pushes
    auto trial = [&](float ratio, uint32_t form_flags, int ctas, float* ms) -> lloid_status {
        lloid_config c = *cfg;
        c.cuda_stream = nullptr;
        c.flags = (c.flags & ~(LLOID_FLAG_STAGE_TIMING | LLOID_FLAG_FORM_LADDER | LLOID_FLAG_FORM_F0)) | form_flags;
        c.form_ratio = ratio;
        c.fir_ctas = ctas;
        c.hbm_budget_bytes = 0;
        lloid_ctx* ctx = nullptr;
        lloid_status st = lloid_create(&c, &ctx);
        if (st) return st;
        int32_t id;
        for (int b = 0; b < n_banks && !st; ++b) st = lloid_load_bank(ctx, banks + b, &id);
        cudaEvent_t a = nullptr, z = nullptr;
        if (!st && (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&z) != cudaSuccess)) st = LLOID_ECUDA;
        long long t = 0;
        for (int k = 0; k < 2 && !st; ++k, t += n) st = lloid_push_strain_all(ctx, t, zeros, n, 1);
        if (!st && cudaEventRecord(a, ctx->stream) != cudaSuccess) st = LLOID_ECUDA;
        for (int k = 0; k < reps && !st; ++k, t += n) st = lloid_push_strain_all(ctx, t, zeros, n, 1);
        if (!st && (cudaEventRecord(z, ctx->stream) != cudaSuccess || cudaEventSynchronize(z) != cudaSuccess ||
                    cudaEventElapsedTime(ms, a, z) != cudaSuccess))
            st = LLOID_ECUDA;
        if (!st) st = lloid_synchronize(ctx);
        *ms /= reps;
        if (a) cudaEventDestroy(a);
        if (z) cudaEventDestroy(z);
        lloid_destroy(ctx);
        return st;
    };
    lloid_status st = LLOID_OK;
    const float ratios[5] = {1.f, 1.f, 0.5f, 2.f, 1.f};
    const uint32_t forms[5] = {LLOID_FLAG_FORM_LADDER, 0u, 0u, 0u, LLOID_FLAG_FORM_F0};
    int best = -1;
    for (int i = 0; i < 5 && !st; ++i) {
        const int k = out->n_tried++;
        out->cand_ratio[k] = ratios[i]; out->cand_flags[k] = forms[i]; out->cand_ctas[k] = cfg->fir_ctas;
        st = trial(ratios[i], forms[i], cfg->fir_ctas, &out->ms[k]);
        if (!st && (best < 0 || out->ms[k] < out->ms[best])) best = k;
    }
    for (int ctas = 1; ctas <= 2 && !st; ++ctas) {
        const int k = out->n_tried++;
        out->cand_ratio[k] = out->cand_ratio[best]; out->cand_flags[k] = out->cand_flags[best]; out->cand_ctas[k] = ctas;
        st = trial(out->cand_ratio[k], out->cand_flags[k], ctas, &out->ms[k]);
        if (!st && out->ms[k] < out->ms[best]) best = k;
    }
    cudaFree(zeros);
    if (st) return st;
    out->best = best;
    out->form_ratio = out->cand_ratio[best];
    out->flags_form = out->cand_flags[best];
    out->fir_ctas = out->cand_ctas[best];
    return LLOID_OK;
}

lloid_status lloid_clear_error(lloid_ctx* ctx) {
    if (!ctx) return LLOID_EINVAL;
    CK(cudaSetDevice(ctx->cfg.device));
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LLOID_OK;
}

int32_t lloid_bank_form(const lloid_ctx* ctx, int32_t bank) {
    if (!ctx) return -1;
    auto it = ctx->banks.find(bank);
    return it == ctx->banks.end() ? -1 : it->second->form;
}

lloid_status lloid_bytes_in_use(const lloid_ctx* ctx, size_t* state_bytes, size_t* bank_bytes) {
    if (!ctx) return LLOID_EINVAL;
    if (state_bytes) *state_bytes = ctx->state_bytes;
    if (bank_bytes) *bank_bytes = ctx->bank_bytes;
    return LLOID_OK;
}

void* lloid_stream(const lloid_ctx* ctx) { return ctx ? (void*)ctx->stream : nullptr; }

lloid_status lloid_stage_times(lloid_ctx* ctx, double* ms, int64_t* launches, int reset) {
    if (!ctx) return LLOID_EINVAL;
    lloid_status st = resolve_timers(ctx);
    if (st) return st;
    for (int i = 0; i < LLOID_N_STAGES; ++i) {
        if (ms) ms[i] = ctx->stage_ms[i];
        if (launches) launches[i] = ctx->stage_launches[i];
        if (reset) { ctx->stage_ms[i] = 0; ctx->stage_launches[i] = 0; }
    }
    return LLOID_OK;
}

lloid_status lloid_create(const lloid_config* cfg, lloid_ctx** out) {
    if (!out) return LLOID_EINVAL;
    *out = nullptr;
    if (!cfg) return LLOID_EINVAL;
    std::unique_ptr<lloid_ctx> h(new lloid_ctx());
    lloid_ctx* ctx = h.get();
    ctx->cfg = *cfg;
    const lloid_config& c = ctx->cfg;
    if (!is_pow2(c.f0) || c.n_detectors < 1 || c.n_detectors > 64 || c.n_down < 1 || c.n_up < 1 ||
        c.window_samples <= 0 || c.window_samples % kTileT || c.max_block <= 0 || c.max_block % kTileT ||
        c.max_history < 0 || !is_pow2(c.min_rate) || c.min_rate > c.f0 || c.f0 / c.min_rate > 256 ||
        c.precision < 0 || c.precision > 2 || !(c.snr_threshold >= 0.f) || c.coinc_window < 0)
        return fail(nullptr, LLOID_EINVAL, "bad configuration");
    if (c.window_overlap < 0 || c.window_overlap >= 128 || c.window_overlap >= c.window_samples)
        return fail(nullptr, LLOID_EINVAL, "window_overlap must be in [0, 128)");
    if (c.max_block / c.window_samples + 1 > kWindowRing)
        return fail(nullptr, LLOID_EINVAL, "a push may complete at most %d trigger windows", kWindowRing);
    if (c.precision != LLOID_FP32 && (c.max_block % kTcTileN || c.n_up != 8 || c.f0 / c.min_rate > 64))
        return fail(nullptr, LLOID_EINVAL, "tensor-core paths need max_block % 128 == 0 and n_up == 8");
    CK(cudaSetDevice(c.device));
    CK(cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, c.device));
    CK(cudaDeviceGetAttribute(&ctx->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c.device));
    if (c.cuda_stream) {
        ctx->stream = (cudaStream_t)c.cuda_stream;
    } else {
        CK(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
        ctx->own_stream = true;
    }
    CK(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&ctx->rest_stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&ctx->gathered, cudaEventDisableTiming));
    const int nd = c.n_detectors;
    lloid_status st;
    // full-rate ring: history for the D = 1 filters and the widest downsampler
    const long long c_max = (long long)(c.f0 / c.min_rate) * c.n_down;
    ctx->ring0_len = next_pow2(c.max_block + std::max<long long>(c.max_history, 2 * c_max) + 4 * kTileT);
    if ((st = dalloc(ctx, &ctx->ring0, (size_t)nd * ctx->ring0_len * 4, nullptr, &ctx->state_bytes))) return st;
    for (int D = 2; D <= c.f0 / c.min_rate; D *= 2) {
        int r = ctx->n_rates++;
        ctx->rate_D[r] = D;
        ctx->rate_len[r] = next_pow2((c.max_block + c.max_history) / D + 2 * c.n_down + 4 * kTileT);
        if ((st = dalloc(ctx, &ctx->rate_ring[r], (size_t)nd * ctx->rate_len[r] * 4, nullptr, &ctx->state_bytes)))
            return st;
        // w' = sqrt(D) g / sum(g), g from Eq. 4 with f = D, c = D N_down
        std::vector<double> g = sinc_windowed(D, D * c.n_down);
        double sum = 0;
        for (double v : g) sum += v;
        std::vector<float> w(g.size());
        for (size_t k = 0; k < g.size(); ++k) w[k] = (float)(std::sqrt((double)D) * g[k] / sum);
        if ((st = dalloc(ctx, &ctx->w_down[r], w.size() * 4, nullptr, &ctx->state_bytes))) return st;
        CK(cudaMemcpyAsync(ctx->w_down[r], w.data(), w.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    }
    ctx->down_smem = down_smem_bytes(ctx->n_rates ? ctx->rate_D[ctx->n_rates - 1] : 1);
    CK(cudaFuncSetAttribute(k_downsample, cudaFuncAttributeMaxDynamicSharedMemorySize, ctx->down_smem));
    if (c.precision != LLOID_FP32) {
        // hi/lo double-mapped streams for the tensor-core FIR (index 0 = f0)
        for (int r = 0; r <= ctx->n_rates; ++r) {
            const int D = r == 0 ? 1 : ctx->rate_D[r - 1];
            ctx->s_len[r] = next_pow2((c.max_block + c.max_history) / D + 2 * c.n_down + 16 * kFirNC + 1024);
            const size_t bytes = (size_t)nd * 2 * ctx->s_len[r] * sizeof(uint16_t);
            if ((st = dalloc(ctx, &ctx->s_hi[r], bytes, nullptr, &ctx->state_bytes))) return st;
            if ((st = dalloc(ctx, &ctx->s_lo[r], bytes, nullptr, &ctx->state_bytes))) return st;
        }
        // Eq. 8 tile matrices: for a 128-sample tile starting at Q (F | Q) and window row w
        // holding sample floor(Q/F) - N_up - r + w of the level below,
        //   U_F[r][q][w] = z_{q mod F}[t],  t = floor(q/F) + 2 N_up + r - w in [0, 2 N_up],
        // with the sub-kernels z_phi[t] = g[t F + phi] of Eq. 7 (g of Eq. 4, c = F N_up, the
        // sinc's zeros at multiples of F written as exact zeros).  Stored as 16-bit hi + lo,
        // time-blocked like the planes: [r][w / 8][q][w mod 8].
        for (int fs = 1; fs < lloid_ctx::kFSlots; ++fs) {
            const int F = 1 << fs;
            const int cF = F * c.n_up;
            const int kw = win_chunks(F) * kWinK;
            std::vector<double> g = sinc_windowed(F, cF);
            std::vector<double> u((size_t)8 * 128 * kw, 0.0);
            for (int r = 0; r < 8; ++r)
                for (int q = 0; q < 128; ++q)
                    for (int w = 0; w < kw; ++w) {
                        const int t = q / F + 2 * c.n_up + r - w;
                        if (t < 0 || t > 2 * c.n_up) continue;
                        const long long k = (long long)t * F + q % F;
                        if (k > 2LL * cF || ((k - cF) % F == 0 && k != cF)) continue;
                        u[(((size_t)r * (kw / 8) + w / 8) * 128 + q) * 8 + w % 8] = g[k];
                    }
            std::vector<uint16_t> uh(u.size()), ul(u.size());
            split_hilo_host(c.precision == LLOID_BF16_SPLIT, u, &uh, &ul);
            if ((st = dalloc(ctx, &ctx->d_u_hi[fs], uh.size() * 2, nullptr, &ctx->state_bytes)) ||
                (st = dalloc(ctx, &ctx->d_u_lo[fs], ul.size() * 2, nullptr, &ctx->state_bytes)))
                return st;
            CK(cudaMemcpy(ctx->d_u_hi[fs], uh.data(), uh.size() * 2, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(ctx->d_u_lo[fs], ul.data(), ul.size() * 2, cudaMemcpyHostToDevice));
        }
    }
    ctx->pos.assign(nd, 0);
    ctx->fin.assign(nd, -1);
    ctx->xi2_next.assign(nd, 0);
    for (int i = 0; i < 64; ++i) ctx->last_n[i] = 0;
    if ((st = dalloc(ctx, &ctx->d_stage, (size_t)nd * c.max_block * 4, nullptr, &ctx->state_bytes))) return st;
    for (int i = 0; i < 2; ++i) {
        CK(cudaHostAlloc((void**)&ctx->h_stage[i], (size_t)nd * c.max_block * 4, cudaHostAllocDefault));
        CK(cudaEventCreateWithFlags(&ctx->stage_ev[i], cudaEventDisableTiming));
        CK(cudaEventRecord(ctx->stage_ev[i], ctx->stream));
    }
    CK(cudaEventCreateWithFlags(&ctx->done_ev, cudaEventDisableTiming));
    CK(cudaEventRecord(ctx->done_ev, ctx->stream));
    ctx->tiles_per_window = (int)(c.window_samples / kTileT);
    ctx->n_slots = (int)next_pow2(((c.max_block + c.window_samples - 1) / c.window_samples + 2) * ctx->tiles_per_window);
    ctx->n_tail = (int)next_pow2((c.max_block + c.window_samples - 1) / c.window_samples + 3);
    for (auto& ps : ctx->pull) {
        CK(cudaHostAlloc((void**)&ps.h_total, sizeof(long long), cudaHostAllocDefault));
        CK(cudaHostAlloc((void**)&ps.h_err, sizeof(int), cudaHostAllocDefault));
        CK(cudaEventCreateWithFlags(&ps.ev, cudaEventDisableTiming));
        if ((st = dalloc(ctx, &ps.d_total, sizeof(long long), nullptr, &ctx->state_bytes))) return st;
    }
    if ((st = dalloc(ctx, &ctx->d_err, sizeof(int), nullptr, &ctx->state_bytes))) return st;
    if ((st = ensure_template_capacity(ctx, 1024))) return st;
    CK(cudaStreamSynchronize(ctx->stream));
    *out = h.release();
    return LLOID_OK;
}

void lloid_destroy(lloid_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->cfg.device);
    cudaStreamSynchronize(ctx->stream);
    for (auto& kv : ctx->banks) {
        for (void* p : kv.second->allocs) cudaFree(p);
        cudaFree(kv.second->d_bg);
        delete kv.second;
    }
    free_jobs(ctx);
    cudaFree(ctx->d_bg_edges);
    cudaFree(ctx->ring0);
    for (int r = 0; r < ctx->n_rates; ++r) { cudaFree(ctx->rate_ring[r]); cudaFree(ctx->w_down[r]); }
    cudaFree(ctx->d_stage);
    for (int i = 0; i < 2; ++i) { cudaFreeHost(ctx->h_stage[i]); if (ctx->stage_ev[i]) cudaEventDestroy(ctx->stage_ev[i]); }
    cudaFree(ctx->d_part); cudaFree(ctx->d_tail); cudaFree(ctx->d_slab); cudaFree(ctx->d_bank_of); cudaFree(ctx->d_tmpl0_of);
    cudaFree(ctx->d_counts);
    for (auto& ps : ctx->pull) {
        cudaFree(ps.d); cudaFree(ps.d_total);
        cudaFreeHost(ps.h); cudaFreeHost(ps.h_total); cudaFreeHost(ps.h_err);
        if (ps.ev) cudaEventDestroy(ps.ev);
    }
    cudaFree(ctx->d_events); cudaFreeHost(ctx->h_events);
    cudaFree(ctx->d_err);
    cudaFree(ctx->d_zero);
    for (int r = 0; r <= kMaxRates; ++r) { cudaFree(ctx->s_hi[r]); cudaFree(ctx->s_lo[r]); }
    for (int f = 0; f < lloid_ctx::kFSlots; ++f) { cudaFree(ctx->d_u_hi[f]); cudaFree(ctx->d_u_lo[f]); }

    if (ctx->done_ev) cudaEventDestroy(ctx->done_ev);
    for (auto& p : ctx->pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    if (ctx->copy_stream) { cudaStreamSynchronize(ctx->copy_stream); cudaStreamDestroy(ctx->copy_stream); }
    if (ctx->rest_stream) cudaStreamDestroy(ctx->rest_stream);
    if (ctx->gathered) cudaEventDestroy(ctx->gathered);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

lloid_status lloid_load_bank(lloid_ctx* ctx, const lloid_bank_desc* bd, int32_t* bank_id) {
    if (!ctx) return LLOID_EINVAL;
    if (!bd || !bank_id || bd->n_templates < 1 || bd->n_slices < 1 || !bd->slices)
        return fail(ctx, LLOID_EINVAL, "bank descriptor is empty or NULL");
    CK(cudaSetDevice(ctx->cfg.device));
    const lloid_config& c = ctx->cfg;
    const int M = bd->n_templates;
    // ---- validate slices
    std::vector<int> rates;
    for (int s = 0; s < bd->n_slices; ++s) {
        const lloid_slice& sl = bd->slices[s];
        if (!is_pow2(sl.rate) || sl.rate > c.f0 || sl.rate < c.min_rate)
            return fail(ctx, LLOID_EINVAL, "slice %d: rate %d is not a power of two in [min_rate, f0]", s, sl.rate);
        const int D = c.f0 / sl.rate;
        if (sl.n_taps < 1 || sl.n_basis < 1 || !sl.bases || !sl.coeffs)
            return fail(ctx, LLOID_EINVAL, "slice %d: empty bases or coefficients", s);
        if (sl.j_start < 0 || sl.j_start % D)
            return fail(ctx, LLOID_EINVAL, "slice %d: j_start %lld is not a non-negative multiple of D = %d", s,
                        (long long)sl.j_start, D);
        if (sl.j_start + (long long)sl.n_taps * D > c.max_history)
            return fail(ctx, LLOID_EINVAL, "slice %d ends at %lld samples, beyond max_history", s,
                        (long long)(sl.j_start + (long long)sl.n_taps * D));
        rates.push_back(sl.rate);
    }
    for (int a = 0; a < bd->n_slices; ++a)
        for (int b = a + 1; b < bd->n_slices; ++b) {
            const lloid_slice &x = bd->slices[a], &y = bd->slices[b];
            long long xa = x.j_start, xb = x.j_start + (long long)x.n_taps * (c.f0 / x.rate);
            long long ya = y.j_start, yb = y.j_start + (long long)y.n_taps * (c.f0 / y.rate);
            if (xa < yb && ya < xb) return fail(ctx, LLOID_EINVAL, "slices %d and %d overlap", a, b);
        }
    if (bd->ac_half < 0 || bd->ac_half > 2048 || (bd->ac_half > 0 && !bd->autocorr))
        return fail(ctx, LLOID_EINVAL, "ac_half %d must be in 0..2048 with autocorr given", bd->ac_half);
    // ---- ladder: distinct rates plus f0, ascending
    std::vector<int> ladder = rates;
    ladder.push_back(c.f0);
    std::sort(ladder.begin(), ladder.end());
    ladder.erase(std::unique(ladder.begin(), ladder.end()), ladder.end());

    std::unique_ptr<BankRT> b(new BankRT());
    b->M = M;
    int row = 0;
    for (int s = 0; s < bd->n_slices; ++s) {
        const lloid_slice& sl = bd->slices[s];
        SliceRT r;
        r.rate = sl.rate; r.D = c.f0 / sl.rate; r.N = sl.n_taps; r.L = sl.n_basis; r.J = sl.j_start;
        r.row0 = row;
        row += r.L;
        std::vector<int> up(ladder.begin() + (std::find(ladder.begin(), ladder.end(), sl.rate) - ladder.begin()),
                            ladder.end());
        std::vector<double> R;
        compose_upsampler(up, c.n_up, &R, &r.e_min, &r.e_max);
        // Pre-synchronisation without latency (Eq. 9): the newest Y sample the
        // upsampler reads must already be computable from the pushed data.
        if (r.D > 1 && r.J < -(long long)r.e_min + (long long)r.D * c.n_down)
            return fail(ctx, LLOID_EINVAL,
                        "slice %d (rate %d) starts %lld samples before merger; pre-synchronisation needs >= %lld",
                        s, r.rate, r.J, -(long long)r.e_min + (long long)r.D * c.n_down);
        b->sl.push_back(r);
        b->sl.back().R = R;
        b->sl.back().y_len = (int)next_pow2(c.max_block / r.D + (r.e_max - r.e_min) / r.D + 4);
        if (!split_precision(ctx)) {   // the FP32 path upsamples each slice with the composed filter
            std::vector<float> Rf(R.size());
            for (size_t i = 0; i < R.size(); ++i) Rf[i] = (float)R[i];
            lloid_status st;
            if ((st = dalloc(ctx, &b->sl.back().d_R, Rf.size() * 4, &b->allocs, &b->bytes))) return st;
            CK(cudaMemcpyAsync(b->sl.back().d_R, Rf.data(), Rf.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
        }
    }
    const bool split = split_precision(ctx);
    b->K = row;
    b->Kpad = (row + 63) / 64 * 64;
    b->Mpad = (M + 127) / 128 * 128;
    if (split) b->form = choose_form(ctx, b.get(), ladder, bd->ac_half);
    const int nd = c.n_detectors;
    lloid_status st;
    auto cleanup = [&]() {
        for (void* p : b->allocs) cudaFree(p);
        cudaFree(b->d_bg);
        b->d_bg = nullptr;
    };
    // ---- budget check before any large allocation
    size_t need = 0;
    if (!split) {
        for (auto& r : b->sl) need += (size_t)r.L * r.N * 4 + (size_t)nd * r.L * r.y_len * 4;
        need += (size_t)b->Mpad * b->Kpad * 4 * 2;
        need += (size_t)nd * b->Kpad * c.max_block * 4;
    } else if ((st = prepare_split_bank(ctx, bd, ladder, b.get(), true, &need))) {
        cleanup();
        return st;
    }
    b->ac_half = bd->ac_half;
    if (b->ac_half > 0) {
        b->zlen = (int)next_pow2(c.max_block + c.window_samples + 2LL * b->ac_half + 256);
        need += (size_t)b->Mpad * (2 * b->ac_half + 1) * sizeof(float2) + (size_t)b->Mpad * 4 +
                (size_t)nd * b->Mpad * b->zlen * 4;
    }
    if (c.hbm_budget_bytes && ctx->state_bytes + ctx->bank_bytes + need > c.hbm_budget_bytes) {
        cleanup();
        return fail(ctx, LLOID_EBUDGET, "bank needs %zu bytes; %zu of %zu in use", need,
                    ctx->state_bytes + ctx->bank_bytes, (size_t)c.hbm_budget_bytes);
    }
    if (split) {
        if ((st = prepare_split_bank(ctx, bd, ladder, b.get(), false, &need))) { cleanup(); return st; }
    } else {
        // ---- bases (FP32) and Y rings
        for (int s = 0; s < bd->n_slices; ++s) {
            const lloid_slice& sl = bd->slices[s];
            SliceRT& r = b->sl[s];
            std::vector<float> u((size_t)r.L * r.N);
            for (size_t i = 0; i < u.size(); ++i) u[i] = (float)sl.bases[i];
            if ((st = dalloc(ctx, &r.d_bases, u.size() * 4, &b->allocs, &b->bytes))) { cleanup(); return st; }
            CK(cudaMemcpyAsync(r.d_bases, u.data(), u.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
            if ((st = dalloc(ctx, &r.d_yring, (size_t)nd * r.L * r.y_len * 4, &b->allocs, &b->bytes))) { cleanup(); return st; }
            CK(cudaStreamSynchronize(ctx->stream));
        }
        // ---- coefficients: C[row][K] with the real rows and imaginary rows apart
        std::vector<double> cre((size_t)b->Mpad * b->Kpad, 0.0), cim((size_t)b->Mpad * b->Kpad, 0.0);
        for (int s = 0; s < bd->n_slices; ++s) {
            const lloid_slice& sl = bd->slices[s];
            const SliceRT& r = b->sl[s];
            for (int i = 0; i < M; ++i)
                for (int l = 0; l < r.L; ++l) {
                    cre[(size_t)i * b->Kpad + r.row0 + l] = sl.coeffs[(size_t)(2 * i) * r.L + l];
                    cim[(size_t)i * b->Kpad + r.row0 + l] = sl.coeffs[(size_t)(2 * i + 1) * r.L + l];
                }
        }
        const size_t n_el = (size_t)b->Mpad * b->Kpad;
        std::vector<float> a(n_el), bb(n_el);
        for (size_t i = 0; i < n_el; ++i) { a[i] = (float)cre[i]; bb[i] = (float)cim[i]; }
        if ((st = dalloc(ctx, (float**)&b->d_cre, n_el * 4, &b->allocs, &b->bytes))) { cleanup(); return st; }
        if ((st = dalloc(ctx, (float**)&b->d_cim, n_el * 4, &b->allocs, &b->bytes))) { cleanup(); return st; }
        CK(cudaMemcpyAsync(b->d_cre, a.data(), n_el * 4, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(b->d_cim, bb.data(), n_el * 4, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        // ---- Yhat block buffers (rows K..Kpad stay zero)
        b->yhat_det_stride = (long long)b->Kpad * c.max_block;
        if ((st = dalloc(ctx, (char**)&b->d_yhat, (size_t)nd * b->yhat_det_stride * 4, &b->allocs, &b->bytes))) { cleanup(); return st; }
    }
    // ---- Eq. 10 tables and the z ring (zeroed: samples before the stream start are 0)
    if (b->ac_half > 0) {
        const int na = 2 * b->ac_half + 1;
        std::vector<float2> ac((size_t)b->Mpad * na, make_float2(0.f, 0.f));
        std::vector<float> den(b->Mpad, 1.f);
        for (int i = 0; i < M; ++i) {
            double sden = 0.0;
            for (int t = 0; t < na; ++t) {
                const double re = bd->autocorr[((size_t)i * na + t) * 2], im = bd->autocorr[((size_t)i * na + t) * 2 + 1];
                ac[(size_t)i * na + t] = make_float2((float)re, (float)im);
                sden += 2.0 - 2.0 * (re * re + im * im);
            }
            if (!(sden > 0.0)) {
                cleanup();
                return fail(ctx, LLOID_EINVAL, "template %d: sum of 2 - 2|R|^2 is not positive", i);
            }
            den[i] = (float)sden;
        }
        if ((st = dalloc(ctx, &b->d_ac, ac.size() * sizeof(float2), &b->allocs, &b->bytes)) ||
            (st = dalloc(ctx, &b->d_ac_den, den.size() * 4, &b->allocs, &b->bytes)) ||
            (st = dalloc(ctx, &b->d_zring, (size_t)nd * b->Mpad * b->zlen * 4, &b->allocs, &b->bytes))) {
            cleanup();
            return st;
        }
        CK(cudaMemcpyAsync(b->d_ac, ac.data(), ac.size() * sizeof(float2), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(b->d_ac_den, den.data(), den.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    if (ctx->bg_nsnr > 0) {
        const size_t bb = (size_t)nd * ctx->bg_nsnr * ctx->bg_nxi2 * 4;
        void* q = nullptr;
        if (cudaMalloc(&q, bb) != cudaSuccess) { cleanup(); return fail(ctx, LLOID_ENOMEM, "background counts"); }
        CK(cudaMemsetAsync(q, 0, bb, ctx->stream));
        b->d_bg = (uint32_t*)q;
    }
    // ---- template ids, window state
    b->tmpl0 = ctx->M_used;
    if ((st = ensure_template_capacity(ctx, (long long)ctx->M_used + M))) { cleanup(); return st; }
    b->id = ctx->next_bank_id++;
    if (b->id >= ctx->bank_cap) {
        int ncap = std::max(64, 2 * ctx->bank_cap);
        {   // event slots follow the bank capacity
            EventEntry* ne = nullptr;
            CK(cudaMalloc(&ne, (size_t)kWindowRing * ncap * sizeof(EventEntry)));
            CK(cudaMemsetAsync(ne, 0, (size_t)kWindowRing * ncap * sizeof(EventEntry), ctx->stream));
            if (ctx->d_events)
                CK(cudaMemcpy2DAsync(ne, ncap * sizeof(EventEntry), ctx->d_events, ctx->bank_cap * sizeof(EventEntry),
                                     ctx->bank_cap * sizeof(EventEntry), kWindowRing, cudaMemcpyDeviceToDevice,
                                     ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            cudaFree(ctx->d_events);
            ctx->d_events = ne;
            cudaFreeHost(ctx->h_events);
            ctx->h_events = nullptr;
            CK(cudaHostAlloc((void**)&ctx->h_events, (size_t)kWindowRing * ncap * sizeof(EventEntry),
                             cudaHostAllocDefault));
        }
        int* nt = nullptr;
        CK(cudaMalloc(&nt, ncap * sizeof(int)));
        cudaFree(ctx->d_tmpl0_of);
        ctx->d_tmpl0_of = nt;
        ctx->bank_cap = ncap;
        ctx->h_tmpl0_of.resize(ncap, 0);
    }
    ctx->h_tmpl0_of[b->id] = b->tmpl0;
    for (int i = 0; i < M; ++i) ctx->h_bank_of[b->tmpl0 + i] = b->id;
    CK(cudaMemcpyAsync(ctx->d_tmpl0_of, ctx->h_tmpl0_of.data(), ctx->bank_cap * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_bank_of + b->tmpl0, ctx->h_bank_of.data() + b->tmpl0, M * sizeof(int),
                       cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->M_used += M;
    ctx->bank_bytes += b->bytes;
    const int id = b->id;
    *bank_id = id;
    ctx->banks[id] = b.release();
    ctx->jobs_dirty = true;
    ctx->xi2_half_max = std::max(ctx->xi2_half_max, bd->ac_half);
    return LLOID_OK;
}

lloid_status lloid_unload_bank(lloid_ctx* ctx, int32_t bank_id) {
    if (!ctx) return LLOID_EINVAL;
    auto it = ctx->banks.find(bank_id);
    if (it == ctx->banks.end()) return fail(ctx, LLOID_EINVAL, "no bank %d", bank_id);
    CK(cudaStreamSynchronize(ctx->stream));
    // forget the bank's retained triggers so later pulls do not report them
    CK(cudaMemset2DAsync(ctx->d_slab + it->second->tmpl0, ctx->M_cap * sizeof(SlabEntry), 0,
                         (size_t)it->second->M * sizeof(SlabEntry), (size_t)kWindowRing * ctx->cfg.n_detectors,
                         ctx->stream));
    if (ctx->d_events)
        CK(cudaMemset2DAsync(ctx->d_events + bank_id, ctx->bank_cap * sizeof(EventEntry), 0, sizeof(EventEntry),
                             kWindowRing, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (void* p : it->second->allocs) cudaFree(p);
    cudaFree(it->second->d_bg);
    ctx->bank_bytes -= it->second->bytes;
    delete it->second;
    ctx->banks.erase(it);
    ctx->jobs_dirty = true;
    ctx->xi2_half_max = 0;
    for (auto& kv : ctx->banks) ctx->xi2_half_max = std::max(ctx->xi2_half_max, kv.second->ac_half);
    return LLOID_OK;
}

lloid_status lloid_push_strain(lloid_ctx* ctx, int32_t det, int64_t t0, const float* block, int64_t n,
                               int is_device_ptr) {
    if (!ctx) return LLOID_EINVAL;
    if (det < 0 || det >= ctx->cfg.n_detectors) return fail(ctx, LLOID_EINVAL, "detector %d out of range", det);
    return push_common(ctx, det, 1, t0, block, n, is_device_ptr);
}

lloid_status lloid_push_strain_all(lloid_ctx* ctx, int64_t t0, const float* blocks, int64_t n, int is_device_ptr) {
    if (!ctx) return LLOID_EINVAL;
    return push_common(ctx, 0, ctx->cfg.n_detectors, t0, blocks, n, is_device_ptr);
}

// Checks that windows w0 .. w0 + n_windows - 1 can be pulled now, then enqueues their
// compaction (k_gather_count / k_gather_scatter) into the slot's device list and, on
// copy_stream, the copy of the error flag, the count and the first `want` triggers into
// the slot's pinned memory, and records the slot's event.  The slot must be free (its
// earlier pull collected).
static lloid_status pull_enqueue(lloid_ctx* ctx, long long w0, long long n_windows, lloid_ctx::PullSlot* ps) {
    if (w0 < 0 || n_windows < 1 || n_windows > kWindowRing) return fail(ctx, LLOID_EINVAL, "bad window range");
    const long long W = ctx->cfg.window_samples;
    const long long w1 = w0 + n_windows - 1;
    long long fin_min = ctx->fin[0], fin_max = ctx->fin[0];
    for (long long f : ctx->fin) { fin_min = std::min(fin_min, f); fin_max = std::max(fin_max, f); }
    if (w1 > fin_min) return fail(ctx, LLOID_ENOTREADY, "window %lld needs data through sample %lld", w1, (w1 + 1) * W);
    if (ctx->xi2_half_max > 0) {   // Eq. 10 needs d samples of z past the window's end
        for (int d = 0; d < ctx->cfg.n_detectors; ++d)
            if (w1 >= ctx->xi2_next[d])
                return fail(ctx, LLOID_ENOTREADY, "window %lld needs data through sample %lld for xi2", w1,
                            (w1 + 1) * W + ctx->xi2_half_max);
    }
    if (w0 + kWindowRing <= fin_max) return fail(ctx, LLOID_EEXPIRED, "window %lld is no longer retained", (long long)w0);
    const int nd = ctx->cfg.n_detectors;
    const int M_used = ctx->M_used;
    ps->w0 = w0;
    ps->n_windows = n_windows;
    ps->want = 0;
    if (M_used == 0) {   // nothing to compact: the error flag alone
        *ps->h_total = 0;
        CK(cudaMemcpyAsync(ps->h_err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaEventRecord(ps->ev, ctx->stream));
        return LLOID_OK;
    }
    const long long total = n_windows * nd * M_used;
    const int chunks = (int)((total + 1023) / 1024);
    if (chunks > ctx->counts_cap) {
        CK(cudaStreamSynchronize(ctx->stream));
        cudaFree(ctx->d_counts);
        ctx->d_counts = nullptr;
        ctx->counts_cap = 0;
        CK(cudaMalloc(&ctx->d_counts, chunks * sizeof(int)));
        ctx->counts_cap = chunks;
    }
    if (total > ps->d_cap) {   // the slot's list: every (window, detector, template) at most once
        CK(cudaStreamSynchronize(ctx->stream));
        cudaFree(ps->d);
        ps->d = nullptr;
        ctx->state_bytes -= (size_t)ps->d_cap * sizeof(TriggerOut);
        ps->d_cap = 0;
        CK(cudaMalloc(&ps->d, total * sizeof(TriggerOut)));
        ps->d_cap = total;
        ctx->state_bytes += (size_t)total * sizeof(TriggerOut);
    }
    CK(cudaStreamWaitEvent(ctx->stream, ps->ev, 0));   // the slot's last copy has left its list
    // the head copied now: sized from the last pull, at most what the pinned part holds
    // (the rest is read from the device list when the pull is collected)
    const long long want =
        std::min<long long>({total, ps->cap, std::max<long long>(256, ctx->last_pull + ctx->last_pull / 2 + 1024)});
    {
        StageTimer tmg(ctx, 6);
        CK(launch_pdl(k_gather_count, dim3(chunks), dim3(1024), 0, ctx->stream, (const SlabEntry*)ctx->d_slab,
                      (long long)ctx->M_cap, M_used, nd, (long long)w0, (int)n_windows, (int)kWindowRing,
                      ctx->d_counts));
        CK(launch_pdl(k_gather_scatter, dim3(chunks), dim3(1024), 0, ctx->stream, (const SlabEntry*)ctx->d_slab,
                      (long long)ctx->M_cap, M_used, nd, (long long)w0, (int)n_windows, (int)kWindowRing,
                      (const int*)ctx->d_counts, chunks, (const int*)ctx->d_bank_of, (const int*)ctx->d_tmpl0_of,
                      W, ps->d, ps->d_cap, ps->d_total));
        ctx->launches += 2;
    }
    ps->want = want;
    CK(cudaEventRecord(ctx->gathered, ctx->stream));
    CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->gathered, 0));
    CK(cudaMemcpyAsync(ps->h_err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->copy_stream));
    CK(cudaMemcpyAsync(ps->h_total, ps->d_total, sizeof(long long), cudaMemcpyDeviceToHost, ctx->copy_stream));
    if (want > 0)
        CK(cudaMemcpyAsync(ps->h, ps->d, want * sizeof(TriggerOut), cudaMemcpyDeviceToHost, ctx->copy_stream));
    CK(cudaEventRecord(ps->ev, ctx->copy_stream));
    return LLOID_OK;
}

// Waits for slot ps, then copies its list into out[cap]: the head from pinned memory,
// the rest (a list longer than the head) from the slot's device list.  A list longer
// than the pinned part grows it, for the slot's next pulls, once the list is out.
static lloid_status pull_finish(lloid_ctx* ctx, lloid_ctx::PullSlot* ps, lloid_trigger* out, int64_t cap,
                                int64_t* n_out, int32_t timeout_ms) {
    lloid_status st;
    if ((st = wait_event(ctx, ps->ev, timeout_ms))) return st;
    if (*ps->h_err)
        return fail(ctx, LLOID_ETIMEOUT, "a kernel wait expired (code %d); results of the last pushes are invalid",
                    *ps->h_err);
    const long long cnt = *ps->h_total;
    *n_out = cnt;
    ctx->last_pull = cnt;
    if (cnt > cap) return fail(ctx, LLOID_ERANGE, "%lld triggers, capacity %lld", cnt, (long long)cap);
    static_assert(sizeof(TriggerOut) == sizeof(lloid_trigger), "trigger layout");
    const long long head = std::min(cnt, ps->want);
    if (head > 0) std::memcpy(out, ps->h, head * sizeof(lloid_trigger));
    if (cnt > head) {
        CK(cudaMemcpyAsync(out + head, ps->d + head, (cnt - head) * sizeof(lloid_trigger), cudaMemcpyDeviceToHost,
                           ctx->rest_stream));
        CK(cudaStreamSynchronize(ctx->rest_stream));
    }
    if (cnt > ps->cap) {   // to twice this list, and at least a quarter of the device list
        cudaFreeHost(ps->h);
        ps->h = nullptr;
        ps->cap = 0;
        const long long cap2 = std::min<long long>(ps->d_cap, std::max<long long>({2 * cnt, 4096, ps->d_cap / 4}));
        // best effort: the list is already out, and without a pinned head a later pull
        // reads all of its list from the device
        if (cudaHostAlloc((void**)&ps->h, cap2 * sizeof(TriggerOut), cudaHostAllocDefault) == cudaSuccess) {
            ps->cap = cap2;
        } else {
            ps->h = nullptr;
            (void)cudaGetLastError();
        }
    }
    return LLOID_OK;
}

lloid_status lloid_pull_triggers_range(lloid_ctx* ctx, int64_t w0, int64_t n_windows, lloid_trigger* out,
                                       int64_t cap, int64_t* n_out, int32_t timeout_ms) {
    if (!ctx) return LLOID_EINVAL;
    if (!n_out || (cap > 0 && !out) || w0 < 0 || n_windows < 1 || n_windows > kWindowRing)
        return fail(ctx, LLOID_EINVAL, "bad output arguments");
    *n_out = 0;
    lloid_status st;
    if (ctx->M_used == 0) {
        if ((st = wait_done(ctx, timeout_ms))) return st;
        return check_kernel_err(ctx);
    }
    lloid_ctx::PullSlot* ps = &ctx->pull[0];
    if ((st = pull_enqueue(ctx, w0, n_windows, ps))) return st;
    return pull_finish(ctx, ps, out, cap, n_out, timeout_ms);
}

lloid_status lloid_pull_submit(lloid_ctx* ctx, int64_t w0, int64_t n_windows, int32_t* ticket) {
    if (!ctx) return LLOID_EINVAL;
    if (!ticket) return fail(ctx, LLOID_EINVAL, "null ticket");
    *ticket = -1;
    int k = 1;
    while (k <= lloid_ctx::kPullSlots && ctx->pull[k].busy) ++k;
    if (k > lloid_ctx::kPullSlots) return fail(ctx, LLOID_EINVAL, "%d pulls already submitted", lloid_ctx::kPullSlots);
    lloid_status st;
    if ((st = pull_enqueue(ctx, w0, n_windows, &ctx->pull[k]))) return st;
    ctx->pull[k].busy = true;
    *ticket = k - 1;
    return LLOID_OK;
}

lloid_status lloid_pull_collect(lloid_ctx* ctx, int32_t ticket, lloid_trigger* out, int64_t cap, int64_t* n_out,
                                int32_t timeout_ms) {
    if (!ctx) return LLOID_EINVAL;
    if (!n_out || (cap > 0 && !out)) return fail(ctx, LLOID_EINVAL, "bad output arguments");
    *n_out = 0;
    if (ticket < 0 || ticket >= lloid_ctx::kPullSlots || !ctx->pull[ticket + 1].busy)
        return fail(ctx, LLOID_EINVAL, "no submitted pull with ticket %d", ticket);
    lloid_ctx::PullSlot* ps = &ctx->pull[ticket + 1];
    const lloid_status st = pull_finish(ctx, ps, out, cap, n_out, timeout_ms);
    // a list too long for out, or a wait that ran out before the copy landed: kept for a retry
    if (st != LLOID_ERANGE && cudaEventQuery(ps->ev) != cudaErrorNotReady) ps->busy = false;
    return st;
}

lloid_status lloid_set_background_bins(lloid_ctx* ctx, const float* snr_edges, int32_t n_snr, const float* xi2_edges,
                                       int32_t n_xi2) {
    if (!ctx) return LLOID_EINVAL;
    if (!snr_edges || !xi2_edges || n_snr < 1 || n_xi2 < 1 || n_snr > 4096 || n_xi2 > 4096)
        return fail(ctx, LLOID_EINVAL, "background bins need 1..4096 bins and their edges");
    for (int i = 0; i < n_snr; ++i)
        if (!(snr_edges[i] < snr_edges[i + 1])) return fail(ctx, LLOID_EINVAL, "snr edges are not ascending");
    for (int i = 0; i < n_xi2; ++i)
        if (!(xi2_edges[i] < xi2_edges[i + 1])) return fail(ctx, LLOID_EINVAL, "xi2 edges are not ascending");
    CK(cudaStreamSynchronize(ctx->stream));
    std::vector<float> e(snr_edges, snr_edges + n_snr + 1);
    e.insert(e.end(), xi2_edges, xi2_edges + n_xi2 + 1);
    cudaFree(ctx->d_bg_edges);
    ctx->d_bg_edges = nullptr;
    CK(cudaMalloc(&ctx->d_bg_edges, e.size() * 4));
    CK(cudaMemcpy(ctx->d_bg_edges, e.data(), e.size() * 4, cudaMemcpyHostToDevice));
    ctx->bg_nsnr = n_snr;
    ctx->bg_nxi2 = n_xi2;
    const size_t bb = (size_t)ctx->cfg.n_detectors * n_snr * n_xi2 * 4;
    for (auto& kv : ctx->banks) {
        cudaFree(kv.second->d_bg);
        kv.second->d_bg = nullptr;
        CK(cudaMalloc(&kv.second->d_bg, bb));
        CK(cudaMemset(kv.second->d_bg, 0, bb));
    }
    ctx->jobs_dirty = true;
    return LLOID_OK;
}

lloid_status lloid_get_background(lloid_ctx* ctx, int32_t bank, uint32_t* out, int64_t cap) {
    if (!ctx) return LLOID_EINVAL;
    auto it = ctx->banks.find(bank);
    if (it == ctx->banks.end()) return fail(ctx, LLOID_EINVAL, "no bank %d", bank);
    if (ctx->bg_nsnr == 0) return fail(ctx, LLOID_EINVAL, "no background bins set");
    const long long n = (long long)ctx->cfg.n_detectors * ctx->bg_nsnr * ctx->bg_nxi2;
    if (!out || cap < n) return fail(ctx, LLOID_ERANGE, "need %lld counts", n);
    CK(cudaMemcpyAsync(out, it->second->d_bg, n * 4, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LLOID_OK;
}

lloid_status lloid_pull_events(lloid_ctx* ctx, int64_t w0, int64_t n_windows, lloid_event* out, int64_t cap,
                               int64_t* n_out, int32_t timeout_ms) {
    if (!ctx) return LLOID_EINVAL;
    if (!n_out || (cap > 0 && !out) || w0 < 0 || n_windows < 1 || n_windows > kWindowRing)
        return fail(ctx, LLOID_EINVAL, "bad output arguments");
    *n_out = 0;
    const long long w1 = w0 + n_windows - 1;
    const long long W = ctx->cfg.window_samples;
    if (w1 >= ctx->coinc_next)
        return fail(ctx, LLOID_ENOTREADY, "events of window %lld are not formed yet", (long long)w1);
    long long fin_max = ctx->fin[0];
    for (long long f : ctx->fin) fin_max = std::max(fin_max, f);
    if (w0 + kWindowRing <= fin_max) return fail(ctx, LLOID_EEXPIRED, "window %lld is no longer retained", (long long)w0);
    if (!ctx->d_events) return LLOID_OK;
    const size_t row = (size_t)ctx->bank_cap * sizeof(EventEntry);
    for (long long w = w0; w <= w1; ++w)
        CK(cudaMemcpyAsync(ctx->h_events + (w - w0) * ctx->bank_cap, ctx->d_events + (w % kWindowRing) * ctx->bank_cap,
                           row, cudaMemcpyDeviceToHost, ctx->stream));
    lloid_ctx::PullSlot& s0 = ctx->pull[0];
    CK(cudaMemcpyAsync(s0.h_err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaEventRecord(s0.ev, ctx->stream));
    lloid_status st;
    if ((st = wait_event(ctx, s0.ev, timeout_ms))) return st;
    if (*s0.h_err)
        return fail(ctx, LLOID_ETIMEOUT, "a kernel wait expired (code %d); results of the last pushes are invalid",
                    *s0.h_err);
    long long cnt = 0;
    for (long long w = w0; w <= w1; ++w)
        for (int bk = 0; bk < ctx->bank_cap; ++bk) {
            const EventEntry& e = ctx->h_events[(w - w0) * ctx->bank_cap + bk];
            if (!(e.net_snr > 0.f) || ctx->banks.find(bk) == ctx->banks.end()) continue;
            if (cnt < cap) {
                lloid_event& o = out[cnt];
                o.window = w; o.bank = bk; o.tmpl = e.tmpl; o.n_ifo = e.n_ifo; o.ifo_mask = e.ifo_mask;
                o.net_snr = e.net_snr; o.ref_detector = e.ref_det; o.ref_sample = w * W + e.ref_k_off;
            }
            ++cnt;
        }
    *n_out = cnt;
    if (cnt > cap) return fail(ctx, LLOID_ERANGE, "%lld events, capacity %lld", cnt, (long long)cap);
    return LLOID_OK;
}

lloid_status lloid_pull_triggers(lloid_ctx* ctx, int64_t window, lloid_trigger* out, int64_t cap, int64_t* n_out,
                                 int32_t timeout_ms) {
    return lloid_pull_triggers_range(ctx, window, 1, out, cap, n_out, timeout_ms);
}

lloid_status lloid_snr_block(lloid_ctx* ctx, int32_t det, int32_t bank, float* out, int64_t cap, int64_t* t0,
                             int64_t* n_samples) {
    if (!ctx) return LLOID_EINVAL;
    if (det < 0 || det >= ctx->cfg.n_detectors) return fail(ctx, LLOID_EINVAL, "detector %d out of range", det);
    auto it = ctx->banks.find(bank);
    if (it == ctx->banks.end()) return fail(ctx, LLOID_EINVAL, "no bank %d", bank);
    const long long n = ctx->last_n[det];
    if (n <= 0) return fail(ctx, LLOID_ENOTREADY, "detector %d has not pushed data", det);
    BankRT* b = it->second;
    if (cap < 2LL * b->M * n) { if (n_samples) *n_samples = n; return fail(ctx, LLOID_ERANGE, "need %lld floats", 2LL * b->M * n); }
    lloid_status st0 = build_jobs(ctx, n);
    if (st0) return st0;
    const int idx = ctx->top_job_of_bank[bank];
    int* db = nullptr;
    int* dsched = nullptr;
    TileInfo* dti = nullptr;
    CK(cudaMalloc(&db, sizeof(int)));
    CK(cudaMemsetAsync(db, 0, sizeof(int), ctx->stream));
    const long long k_a = ctx->pos[det] - n;
    lloid_status st;
    if (!split_precision(ctx)) {
        const int tiles = (b->Mpad / 64) * (int)(n / 128);
        st = launch_recon_f32(ctx, k_a, n, det, 1, true, ctx->d_rec + idx, db, 1, tiles, out);
    } else if (b->form == 1) {   // the f0 kernel over this bank's window groups, storing z
        const int cls = ctx->f0_class_of_bank[bank];
        const int tpw = (int)(ctx->cfg.window_samples / 128);
        std::vector<F0Unit> hu;
        for (int g = 0; g * tpw < (int)(n / 128); ++g) hu.push_back(F0Unit{ctx->f0_job_of_bank[bank], g});
        int grid = 0;
        const std::vector<int> hs = build_sched(std::vector<double>(hu.size(), 1.0), 1, ctx->n_sm, &grid);
        F0Unit* du = nullptr;
        CK(cudaMalloc(&dsched, hs.size() * sizeof(int)));
        CK(cudaMalloc(&du, hu.size() * sizeof(F0Unit)));
        dti = reinterpret_cast<TileInfo*>(du);   // freed below with the others
        CK(cudaMemcpyAsync(dsched, hs.data(), hs.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(du, hu.data(), hu.size() * sizeof(F0Unit), cudaMemcpyHostToDevice, ctx->stream));
        st = launch_f0(ctx, cls, ctx->d_f0job[cls], du, dsched, grid, k_a, n, det, 1, out);
    } else {
        const int tiles = (b->Mpad / kTcTileM) * (int)(n / kTcTileN);
        const int fs = ctx->top_slot_of_bank[bank];
        int grid = 0;
        const std::vector<int> hs = build_sched(std::vector<double>(tiles, 1.0), 1, ctx->n_sm, &grid);
        std::vector<TileInfo> hti(tiles);
        const LevelRT& T = b->form == 1 ? b->top : b->lev.back();
        for (int l = 0; l < tiles; ++l) hti[l] = TileInfo{0, l, T.Kp, T.K / 16};
        CK(cudaMalloc(&dsched, hs.size() * sizeof(int)));
        CK(cudaMalloc(&dti, hti.size() * sizeof(TileInfo)));
        CK(cudaMemcpyAsync(dsched, hs.data(), hs.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(dti, hti.data(), hti.size() * sizeof(TileInfo), cudaMemcpyHostToDevice, ctx->stream));
        st = launch_level(ctx, 0, fs, k_a, n, det, 1, true, ctx->d_lev[fs] + idx, ctx->d_levmaps[fs], dti, dsched, grid,
                          1, tiles, out);
    }
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    cudaFree(db);
    cudaFree(dsched);
    cudaFree(dti);
    if (st) return st;
    if (e != cudaSuccess) return fail(ctx, LLOID_ECUDA, "snr_block: %s", cudaGetErrorString(e));
    if ((st = check_kernel_err(ctx))) return st;
    if (t0) *t0 = k_a;
    if (n_samples) *n_samples = n;
    return LLOID_OK;
}

lloid_status lloid_save_state(lloid_ctx* ctx, void* buf, size_t* len) {
    if (!ctx || !len) return LLOID_EINVAL;
    std::vector<long long> hdr;
    std::vector<Segment> seg;
    state_layout(ctx, &hdr, &seg);
    size_t need = sizeof(long long) * (1 + hdr.size());
    for (auto& x : seg) need += x.bytes;
    if (!buf || *len < need) {
        *len = need;
        return buf ? fail(ctx, LLOID_ERANGE, "checkpoint needs %zu bytes", need) : LLOID_OK;
    }
    CK(cudaStreamSynchronize(ctx->stream));
    char* o = static_cast<char*>(buf);
    long long nh = (long long)hdr.size();
    std::memcpy(o, &nh, sizeof nh);
    o += sizeof nh;
    std::memcpy(o, hdr.data(), hdr.size() * sizeof(long long));
    o += hdr.size() * sizeof(long long);
    for (auto& x : seg) {
        CK(cudaMemcpy(o, x.p, x.bytes, cudaMemcpyDeviceToHost));
        o += x.bytes;
    }
    *len = need;
    return LLOID_OK;
}

lloid_status lloid_restore_state(lloid_ctx* ctx, const void* buf, size_t len) {
    if (!ctx || !buf) return LLOID_EINVAL;
    std::vector<long long> hdr;
    std::vector<Segment> seg;
    CK(cudaStreamSynchronize(ctx->stream));
    // positions are part of the header: compare everything else
    state_layout(ctx, &hdr, &seg);
    const char* in = static_cast<const char*>(buf);
    long long nh = 0;
    if (len < sizeof nh) return fail(ctx, LLOID_EINVAL, "checkpoint too short");
    std::memcpy(&nh, in, sizeof nh);
    if (nh != (long long)hdr.size() || len < sizeof(long long) * (1 + (size_t)nh))
        return fail(ctx, LLOID_EINVAL, "checkpoint does not match this context (layout)");
    std::vector<long long> saved((size_t)nh);
    std::memcpy(saved.data(), in + sizeof nh, (size_t)nh * sizeof(long long));
    const int nd = ctx->cfg.n_detectors;
    const size_t pos_at = 15, pos_end = 15 + 4 * (size_t)nd + 1;
    for (size_t i = 0; i < hdr.size(); ++i) {
        if (i >= pos_at && i < pos_end) continue;
        if (saved[i] != hdr[i]) return fail(ctx, LLOID_EINVAL, "checkpoint does not match this context (word %zu)", i);
    }
    size_t need = sizeof(long long) * (1 + hdr.size());
    for (auto& x : seg) need += x.bytes;
    if (len < need) return fail(ctx, LLOID_EINVAL, "checkpoint truncated");
    const char* o = in + sizeof(long long) * (1 + hdr.size());
    for (auto& x : seg) {
        CK(cudaMemcpy(x.p, o, x.bytes, cudaMemcpyHostToDevice));
        o += x.bytes;
    }
    for (int d = 0; d < nd; ++d) {
        ctx->pos[d] = saved[pos_at + 4 * d];
        ctx->fin[d] = saved[pos_at + 4 * d + 1];
        ctx->last_n[d] = saved[pos_at + 4 * d + 2];
        ctx->xi2_next[d] = saved[pos_at + 4 * d + 3];
    }
    ctx->coinc_next = saved[pos_at + 4 * (size_t)nd];
    CK(cudaEventRecord(ctx->done_ev, ctx->stream));
    return LLOID_OK;
}

lloid_status lloid_synchronize(lloid_ctx* ctx) {
    if (!ctx) return LLOID_EINVAL;
    CK(cudaStreamSynchronize(ctx->stream));
    return check_kernel_err(ctx);
}

}  // extern "C"
