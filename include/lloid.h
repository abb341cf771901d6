/*
 * lloid.h -- C ABI of the B300 LLOID hot path.
 *
 * LLOID (the time-domain matched filter of SGNL, Section II.C of the paper)
 * correlates whitened detector strain with a template bank that has been cut
 * into time slices, each sampled at its own rate and compressed by an SVD
 * (Eq. 3).  For every block of strain this library runs, on one GPU:
 *
 *   a0  ingest      block -> device ring (host or device source)
 *   a1  downsample  to every power-of-two rate, sinc-windowed sinc kernel of
 *                   Eq. 4 with c = D N_down, unit DC gain, scaled by sqrt(D)
 *   a2  basis FIR   Y^s_l[q] = sum_m u^s_l[m] d_s[q - J_s/D_s - m]  (Eq. 5,
 *                   read at the pre-synchronised offset of Eq. 9)
 *   a3  recon       z_row = sum_s sum_l (sigma v)^s[row][l] Y^s_l  (Eq. 6)
 *   a4  up + sum    polyphase upsampling ladder of Eq. 7-8 and the recursive
 *                   sum of Eq. 9, to the full rate f0
 *   a5  triggers    per window and template, max |z| above the threshold,
 *                   its sample and phase; per bank the loudest template
 *                   (Section II.D.1)
 *
 * Conventions shared by every call
 * --------------------------------
 * * Time is the full-rate sample index since the stream started (sample 0);
 *   the data before sample 0 are zero.  A template row is indexed by samples
 *   before merger, so z[k] is the SNR of a merger at sample k.
 * * Template i has two real rows: 2i (cosine / real part) and 2i+1 (sine /
 *   imaginary part); z_i = z[2i] + i z[2i+1] (Section II.C, Eq. 1).
 * * The downsampled stream at rate f0/D has unit variance for unit-variance
 *   input: d_D[q] = sqrt(D) sum_k w[k] d[D q + c - k], w = g / sum(g) (g of
 *   Eq. 4, zero phase).  A bank's bases are therefore built from
 *   sqrt(D) h[J + D m] (the sqrt(D) pair restores the full-rate inner product).
 * * Every call returns an lloid_status; no C++ exception crosses the ABI.
 *   lloid_last_error() gives a one-line reason for the last failure.
 * * The library copies everything it is given; the caller keeps ownership of
 *   its buffers.  One context is used by one host thread at a time.
 * * All GPU work of a context is ordered on one CUDA stream (the caller's, or
 *   one the library creates).  Calls return once the work is enqueued, except
 *   pull_triggers, snr_block and synchronize, which wait for it.
 */
#ifndef LLOID_H
#define LLOID_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LLOID_API __attribute__((visibility("default")))
#else
#define LLOID_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lloid_ctx lloid_ctx;

typedef enum {
    LLOID_OK = 0,
    LLOID_EINVAL = -1,     /* bad argument, shape or bank (message says which) */
    LLOID_ENOMEM = -2,     /* a device or host allocation failed */
    LLOID_EBUDGET = -3,    /* loading the bank would exceed hbm_budget_bytes */
    LLOID_EGAP = -4,       /* push t0 is not where the detector's stream ends */
    LLOID_ENOTREADY = -5,  /* window not yet covered by pushed data */
    LLOID_ETIMEOUT = -6,   /* GPU work not finished within timeout_ms */
    LLOID_ECUDA = -7,      /* a CUDA call failed (message has the CUDA error) */
    LLOID_ERANGE = -8,     /* output capacity too small (n_out has the need) */
    LLOID_EEXPIRED = -9    /* the window's triggers were overwritten (pull sooner) */
} lloid_status;

typedef enum {
    LLOID_FP32 = 0,        /* FP32 operands, FP32 accumulate (SIMT FMA) */
    LLOID_FP16_SPLIT = 1,  /* tensor cores: FP16 operands with the data split
                              into hi + lo halves, FP32 accumulate */
    LLOID_BF16_SPLIT = 2   /* tensor cores: BF16 hi + lo on both operands
                              (three products), FP32 accumulate */
} lloid_precision;

/* Context configuration.  lloid_config_default() fills the paper's values:
 * f0 = 2048 Hz, N_down = 32 (Section II.C.2), N_up = 8 (Section II.C.2),
 * 1 s windows with no overlap, threshold |z| > 4 (Section II.D.1). */
typedef struct {
    int32_t f0;                /* full sample rate (Hz); power of two */
    int32_t n_detectors;       /* independent strain streams (>= 1) */
    int32_t n_down;            /* downsampling half length at the target rate */
    int32_t n_up;              /* upsampling half length at the lower rate */
    int64_t window_samples;    /* trigger window W (multiple of 128) */
    int64_t window_overlap;    /* window w covers [max(0, wW - overlap), (w+1)W), so that
                                  a signal near a window's start is seen in both windows
                                  (Section II.D.1: light travel time plus a buffer, about
                                  66 samples at 2048 Hz); 0 <= overlap < 128 (EINVAL
                                  otherwise).  A window's trigger can then lie before its
                                  start (sample < wW). */
    float snr_threshold;       /* a trigger needs |z| > snr_threshold */
    int32_t precision;         /* lloid_precision */
    int64_t max_block;         /* largest push, full-rate samples (multiple of 128) */
    int64_t max_history;       /* longest template J_s + N_s D_s any bank may use */
    int32_t min_rate;          /* lowest slice rate (power of two, f0/64 at least) */
    int32_t device;            /* CUDA device ordinal */
    size_t hbm_budget_bytes;   /* 0 = no budget; else cap on bank + state bytes */
    void* cuda_stream;         /* cudaStream_t to order work on, or NULL */
    uint32_t flags;            /* LLOID_FLAG_* bits */
    int32_t coinc_window;      /* coincidence window in samples (Section II.D.3): maximum light
                                  travel time plus buffer, default 66 = (0.0273 + 0.005) s x 2048 */
    float form_ratio;          /* split path: a bank runs in the f0 form when its estimated time
                                  in that form is below form_ratio x its estimate in the ladder
                                  form (<= 0: 1); see LLOID_FLAG_FORM_* and lloid_autotune */
    int32_t fir_ctas;          /* basis-filter CTAs per SM: 1, 2, or 0 = two when each still gets
                                  two operand stages, else one */
} lloid_config;

/* One time slice of a bank (Eq. 3): the leading L bases and their
 * reconstruction coefficients.  Rate = f0 / D with D a power of two; the
 * slice covers before-merger full-rate samples [j_start, j_start + n_taps D);
 * j_start must be a multiple of D and satisfy pre-synchronisation without
 * latency (Eq. 9): j_start >= D N_down + sum over the bank's ladder rates
 * f (rate <= f < f0) of N_up f0 / f, for D > 1. */
typedef struct {
    int32_t rate;
    int32_t n_taps;            /* N_s, samples at this rate */
    int64_t j_start;           /* J_s, full-rate samples before merger */
    int32_t n_basis;           /* L_s >= 1 */
    int32_t pad0;
    const double* bases;       /* host, [n_basis][n_taps], u_l[m], m = samples
                                  before merger at this rate (row-major) */
    const double* coeffs;      /* host, [2M][n_basis], v_il sigma_l; row 2i is
                                  the real part of template i, 2i+1 imaginary */
} lloid_slice;

typedef struct {
    int32_t n_templates;       /* M (>= 1) */
    int32_t n_slices;          /* S (>= 1) */
    const lloid_slice* slices; /* host, [n_slices], any order, non-overlapping */
    /* Signal-consistency test (Eq. 10, Section II.D.2), optional: with
     * ac_half = d > 0 every trigger of the bank gets
     *   xi2 = sum_{t=-d}^{d} |z(k*+t) - z(k*) R(t)|^2 / sum_{t=-d}^{d} (2 - 2|R(t)|^2)
     * around its peak k*, where R is the template's complex autocorrelation
     * normalised to R(0) = 1 (the paper uses 2 d + 1 = 351 or 701 samples).
     * Windows of such a bank can be pulled once every detector's stream has
     * passed the window's end by d samples.  ac_half = 0: no xi2 (autocorr
     * unused). */
    int32_t ac_half;           /* d, 0 .. 2048 */
    int32_t pad1;
    const double* autocorr;    /* host, [M][2 d + 1][2]: Re, Im of R_i(t), t = -d .. d */
} lloid_bank_desc;

/* A trigger (Section II.D.1): template `tmpl` of bank `bank` in detector
 * `detector` reached its window maximum |z| = snr > threshold at `sample`,
 * with phase = atan2(im, re).  is_bank_max = 1 marks the bank's loudest
 * template in that window (lowest template index on ties). */
typedef struct {
    int32_t detector;
    int32_t bank;
    int32_t tmpl;
    int32_t is_bank_max;
    int64_t window;
    int64_t sample;
    float snr;
    float phase;
    float re;
    float im;
    float xi2;                 /* Eq. 10 statistic; < 0 when the bank has no autocorrelation */
    int32_t pad;
} lloid_trigger;

/* A coincident event after clustering (Sections II.D.3-4): in window
 * `window` of bank `bank`, template `tmpl` triggered in the n_ifo >= 2
 * detectors of ifo_mask within coinc_window samples of its loudest trigger
 * (detector ref_detector, sample ref_sample); net_snr = sqrt(sum of their
 * snr^2) is the largest of the bank's events in that window (lowest template
 * on ties), so there is at most one event per (bank, window). */
typedef struct {
    int64_t window;
    int32_t bank;
    int32_t tmpl;
    int32_t n_ifo;
    uint32_t ifo_mask;
    float net_snr;
    int32_t ref_detector;
    int64_t ref_sample;
} lloid_event;

/* Fill *cfg with the defaults above (n_detectors = 1, max_block = 16384,
 * max_history = 128 s, min_rate = 32, precision FP32). */
LLOID_API void lloid_config_default(lloid_config* cfg);

/* Create a context on cfg->device.  Allocates the per-detector strain rings
 * and window buffers.  EINVAL on a bad configuration (checked before any
 * device call), among them a max_block with which one push could complete
 * more than 16 trigger windows (max_block / window_samples + 1 > 16: the
 * retained-window ring holds 16); ECUDA/ENOMEM on device failure.  *out is
 * NULL on failure. */
LLOID_API lloid_status lloid_create(const lloid_config* cfg, lloid_ctx** out);

/* Free every device and host resource of the context (NULL is a no-op). */
LLOID_API void lloid_destroy(lloid_ctx* ctx);

/* Static text for a status code. */
LLOID_API const char* lloid_strerror(lloid_status st);

/* One-line reason for the last failing call on ctx (never NULL). */
LLOID_API const char* lloid_last_error(const lloid_ctx* ctx);

/* Load an SVD bank (Eq. 3, grouped as in Section II.C.1): validates shapes,
 * rates, slice overlap and the pre-synchronisation condition of Eq. 9,
 * converts to the context's precision and copies to the device.  Banks may be
 * loaded while streaming; a bank's SNR is exact once its longest slice
 * (j_start + n_taps D) has been streamed after loading.  *bank_id receives a
 * small integer used in triggers.  EBUDGET when hbm_budget_bytes would be
 * exceeded (nothing is kept), EINVAL with a reason otherwise. */
LLOID_API lloid_status lloid_load_bank(lloid_ctx* ctx, const lloid_bank_desc* bank, int32_t* bank_id);

/* Release a bank's device memory.  Enqueued work that uses it completes first. */
LLOID_API lloid_status lloid_unload_bank(lloid_ctx* ctx, int32_t bank_id);

/* Push n samples of whitened strain of detector `det` starting at full-rate
 * sample t0 (steps a0-a5 for every loaded bank).  `block` is a host pointer
 * (is_device_ptr = 0; pinned memory avoids a staging copy) or a device
 * pointer on the context's device (is_device_ptr = 1).  t0 must equal the
 * end of the detector's previous push (0 at first): EGAP otherwise.  n must
 * be a positive multiple of 128 and <= max_block: EINVAL otherwise.  Windows
 * that the block completes are finalised on the device. */
LLOID_API lloid_status lloid_push_strain(lloid_ctx* ctx, int32_t det, int64_t t0, const float* block,
                               int64_t n, int is_device_ptr);

/* The same for every detector at once: `blocks` is [n_detectors][n],
 * row-major, and every detector's stream must end at t0. */
LLOID_API lloid_status lloid_push_strain_all(lloid_ctx* ctx, int64_t t0, const float* blocks, int64_t n,
                                   int is_device_ptr);

/* Copy the triggers of window `window` (all detectors, all banks) into the
 * host array out[cap], ordered by detector, bank, template.  ENOTREADY if a
 * detector has not pushed data through the end of the window; waits up to
 * timeout_ms (< 0: forever) for the GPU, then ETIMEOUT; ERANGE if cap is too
 * small (*n_out = the number needed, nothing copied); EEXPIRED if the window
 * is older than the retained ring (the 16 most recent windows). */
LLOID_API lloid_status lloid_pull_triggers(lloid_ctx* ctx, int64_t window, lloid_trigger* out, int64_t cap,
                                 int64_t* n_out, int32_t timeout_ms);

/* The same for the n_windows consecutive windows w0 .. w0 + n_windows - 1
 * (1 <= n_windows <= 16), ordered by window, detector, bank, template, with
 * one compaction pass and one wait for all of them. */
LLOID_API lloid_status lloid_pull_triggers_range(lloid_ctx* ctx, int64_t w0, int64_t n_windows, lloid_trigger* out,
                                                 int64_t cap, int64_t* n_out, int32_t timeout_ms);

/* A pull in two halves, so that the host can read one block's triggers while the
 * GPU filters the next.  lloid_pull_submit checks windows w0 .. w0 + n_windows - 1
 * as lloid_pull_triggers_range does (EINVAL, ENOTREADY, EEXPIRED), enqueues their
 * compaction and the copy to pinned host memory behind the pushes already
 * enqueued, and returns at once with *ticket (0..7).  At most 8 pulls are
 * submitted and not yet collected: EINVAL for a ninth.  Each holds its compacted
 * list on the device (n_windows x detectors x loaded templates entries of 40
 * bytes) until it is collected.  The list is the one the blocking pull would
 * return at the time of the submit: later pushes and pulls do not change it. */
LLOID_API lloid_status lloid_pull_submit(lloid_ctx* ctx, int64_t w0, int64_t n_windows, int32_t* ticket);

/* Waits up to timeout_ms (< 0: forever) for a submitted pull and copies its
 * triggers into the host array out[cap], ordered as lloid_pull_triggers_range
 * orders them.  ETIMEOUT if the copy has not landed (the ticket stays valid) or
 * a kernel wait expired; ERANGE if cap is too small (*n_out = the number needed,
 * nothing copied, the ticket stays valid).  Otherwise the ticket is released.  A
 * list longer than the part copied at submit time is read from the device (a
 * blocking copy of the rest); the pinned part then grows for later pulls. */
LLOID_API lloid_status lloid_pull_collect(lloid_ctx* ctx, int32_t ticket, lloid_trigger* out, int64_t cap,
                                          int64_t* n_out, int32_t timeout_ms);

/* Coincident events of windows w0 .. w0 + n_windows - 1 (1 <= n_windows <=
 * 16), ordered by window then bank: at most one per (bank, window), formed on
 * the GPU from the windows' triggers of all detectors (Sections II.D.3-4).
 * A window's events are ready once its triggers are (for banks with
 * autocorrelations, d samples past the window's end in every detector);
 * same waiting, ENOTREADY, ERANGE and EEXPIRED rules as the trigger pulls. */
LLOID_API lloid_status lloid_pull_events(lloid_ctx* ctx, int64_t w0, int64_t n_windows, lloid_event* out,
                                         int64_t cap, int64_t* n_out, int32_t timeout_ms);

/* Background collection (Section II.D.5): from now on every window adds its
 * single-detector triggers (those that are not members of their template's
 * coincidence) to a persistent histogram per bank and detector over SNR and
 * xi2 (-1 for banks without autocorrelations), only while two or more
 * detectors are configured.  Edges are ascending (n_snr + 1 and n_xi2 + 1
 * values); a value goes to the bin of the last edge <= it, values outside
 * the edges to the first or last bin.  Calling again resets every bank's
 * counts. */
LLOID_API lloid_status lloid_set_background_bins(lloid_ctx* ctx, const float* snr_edges, int32_t n_snr,
                                                 const float* xi2_edges, int32_t n_xi2);

/* Copy bank `bank`'s counts [n_detectors][n_snr][n_xi2] into out[cap] (after
 * the context's queued work); the snapshot the paper takes every four hours. */
LLOID_API lloid_status lloid_get_background(lloid_ctx* ctx, int32_t bank, uint32_t* out, int64_t cap);

/* ---------------------------------------------------------------------------
 * PSD estimation and whitening (Section II.B.2), the front end before
 * lloid_push_strain: blocks of n_fft input samples (an n_fft - 2 z_pad
 * Hann-windowed segment between z_pad zeros) advance by hop = n_fft/2 - z_pad;
 * each is Fourier transformed, downsampled by keeping the bins below the
 * output Nyquist, used to update the PSD estimate (per bin: median of the
 * last n_med instantaneous estimates, turned into a geometric-mean estimate
 * by a constant factor and averaged in log over up to n_avg blocks; times
 * e^gamma for the arithmetic mean) and whitened with it, inverse transformed
 * at rate_out, Tukey-tapered (z_pad rate_out / rate_in samples at each end)
 * and overlap-added.  Output sample j corresponds to input sample
 * j rate_in / rate_out - z_pad, so the output lags the input by n_fft / 2
 * samples.  A block whose segment holds a non-finite sample (a gap) neither
 * updates the PSD nor adds output.  Every step runs in this library's kernels,
 * the transforms included: the forward one computes only the bins below the
 * output Nyquist (n_fft rate_out / rate_in / 2 + 1 of them), the inverse one
 * is a real transform of length n_fft rate_out / rate_in.
 * ------------------------------------------------------------------------- */
typedef struct lloid_whitener lloid_whitener;

typedef struct {
    int32_t rate_in;           /* input rate (Hz), power of two */
    int32_t rate_out;          /* output rate, power of two <= rate_in, rate_in / rate_out <= 4096 */
    int32_t n_fft;             /* N: input samples per block, power of two, <= 2^24,
                                  with N rate_out / rate_in in 4 .. 16384 */
    int32_t z_pad;             /* Z: 0 <= Z < N/2, N/2 - Z a multiple of rate_in / rate_out */
    int32_t n_med;             /* odd, 1 .. 15 */
    int32_t n_avg;             /* >= 1 */
    int32_t n_detectors;       /* 1 .. 64 */
    int32_t device;
    int64_t max_push;          /* largest push (input samples, a multiple of the hop) */
    void* cuda_stream;         /* cudaStream_t or NULL */
} lloid_whitener_config;

/* 16384 Hz -> 2048 Hz, N = 4 s, Z = 1 s, n_med = 7 (Section II.B.2), n_avg = 64,
 * one detector, max_push = 16 s. */
LLOID_API void lloid_whitener_config_default(lloid_whitener_config* cfg);
LLOID_API lloid_status lloid_whitener_create(const lloid_whitener_config* cfg, lloid_whitener** out);
LLOID_API void lloid_whitener_destroy(lloid_whitener* wh);

/* Append n input samples of detector det (n a multiple of the hop, at most
 * max_push) and write the output samples that became final (n / hop x
 * hop rate_out / rate_in of them once the first segment has filled) to
 * out[cap] (device memory if out_is_device, else host); *n_out = their count.
 * Asynchronous on the whitener's stream when the output is on the device. */
LLOID_API lloid_status lloid_whiten(lloid_whitener* wh, int32_t det, const float* in, int64_t n, int in_is_device,
                                    float* out, int64_t cap, int64_t* n_out, int out_is_device);

/* The current PSD estimate of detector det: n_fft rate_out / rate_in / 2 + 1
 * bins (0 .. rate_out / 2 Hz), in units of the input's per-sample variance. */
LLOID_API lloid_status lloid_whitener_psd(lloid_whitener* wh, int32_t det, float* out, int64_t cap);

/* Debug and parity aid: recompute the full-rate SNR rows of the most recent
 * push of detector `det` for bank `bank` into the DEVICE array out
 * [2M][n_last] (row 2i = real part of template i) with the same kernels and
 * precision as the trigger path; *n_samples receives n_last and *t0 its first
 * sample.  cap is out's length in floats (ERANGE when too small).  Waits. */
LLOID_API lloid_status lloid_snr_block(lloid_ctx* ctx, int32_t det, int32_t bank, float* out, int64_t cap,
                             int64_t* t0, int64_t* n_samples);

/* Checkpoint of the streaming state (SGNL snapshots its state periodically,
 * Section II.D.5): every per-detector stream ring, every bank's history ring,
 * the window partials and retained trigger windows, and the stream
 * positions, written to the host buffer buf[*len] after waiting for the
 * context's stream.  With buf == NULL, *len receives the size and the call
 * returns LLOID_OK; with *len too small it returns LLOID_ERANGE and the size. */
LLOID_API lloid_status lloid_save_state(lloid_ctx* ctx, void* buf, size_t* len);

/* Resume from a checkpoint: ctx must have been created with the same
 * configuration and have the same banks loaded in the same order as the
 * saved context (LLOID_EINVAL otherwise).  Streaming then continues exactly
 * as the saved context would have. */
LLOID_API lloid_status lloid_restore_state(lloid_ctx* ctx, const void* buf, size_t len);

/* Wait for all enqueued work of the context (ECUDA on a device error). */
LLOID_API lloid_status lloid_synchronize(lloid_ctx* ctx);

/* Device bytes held by the context: *state_bytes for streams, rings and
 * window state, *bank_bytes for the loaded banks (either may be NULL).  These
 * are the quantities hbm_budget_bytes is checked against. */
LLOID_API lloid_status lloid_bytes_in_use(const lloid_ctx* ctx, size_t* state_bytes, size_t* bank_bytes);

/* Number of kernel launches the context has issued so far. */
LLOID_API int64_t lloid_launch_count(const lloid_ctx* ctx);

/* The cudaStream_t every kernel of the context runs on (as void*), so that a
 * caller can order its own work (e.g. the producer of a device block) with it. */
LLOID_API void* lloid_stream(const lloid_ctx* ctx);

/* Per-stage device time, measured with CUDA events recorded on the context's
 * stream around every stage of every push and pull when cfg.flags has
 * LLOID_FLAG_STAGE_TIMING.  Fills ms[i] (milliseconds) and launches[i] for the
 * LLOID_N_STAGES stages (ingest, downsample, fir, upsample, recon, finalize,
 * gather) accumulated since the last reset; reset != 0 clears them.  Waits
 * for the context's stream.  Either output may be NULL. */
#define LLOID_FLAG_STAGE_TIMING 1u
#define LLOID_N_STAGES 7

/* Form of the split-precision path per bank (lloid_config.flags).  Both give
 * the same SNR up to rounding, because Eq. 6 and Eq. 7-8 are linear and the
 * coefficients do not depend on time:
 *   ladder: per rate, reconstruct (Eq. 6), then upsample and add into the
 *           next rate (Eq. 7-9), lowest rate first, in the paper's order;
 *   f0:     upsample each slice's basis outputs to f0 through the slice's
 *           composed ladder (Eq. 7-8), then reconstruct once at f0 over all
 *           of the bank's bases.
 * The ladder costs less when a bank has many bases at low rates, the f0 form
 * when it has few (it has no per-rate window products and no per-rate
 * intermediate SNR in device memory).  Without either flag each bank takes
 * the form an estimate of its tensor-core and memory time prefers, which
 * lloid_autotune can then replace by measured times.  Ignored by the FP32 path. */
#define LLOID_FLAG_FORM_LADDER 2u
#define LLOID_FLAG_FORM_F0 4u

/* The form bank `bank` runs in: 0 ladder, 1 f0 (always 0 on the FP32 path);
 * -1 if there is no such bank. */
LLOID_API int32_t lloid_bank_form(const lloid_ctx* ctx, int32_t bank);

/* The autotuner of the batched path: for pushes of n samples of every
 * detector with the banks banks[0 .. n_banks - 1] loaded, times candidate
 * settings on scratch contexts made from *cfg (its stream and stage timing
 * are not used): every bank in the ladder form, form_ratio 0.5, 1 and 2, every
 * bank that can in the f0 form, then 1 and 2 basis-filter CTAs per SM with the
 * fastest of those.  Each candidate gets two warm-up pushes of zeros and then
 * `reps` timed pushes (CUDA events).  out->form_ratio, out->flags_form (0,
 * LLOID_FLAG_FORM_LADDER or LLOID_FLAG_FORM_F0) and out->fir_ctas are the
 * fastest setting, to copy into the lloid_config of the context that
 * streams; ms[i] is candidate i's device time per push.  EINVAL for bad
 * arguments; any error of a candidate context is returned. */
typedef struct {
    float form_ratio;
    uint32_t flags_form;
    int32_t fir_ctas;
    int32_t n_tried;
    int32_t best;              /* index of the chosen candidate */
    float ms[16];
    float cand_ratio[16];
    uint32_t cand_flags[16];
    int32_t cand_ctas[16];
} lloid_tuning;
LLOID_API lloid_status lloid_autotune(const lloid_config* cfg, const lloid_bank_desc* banks, int32_t n_banks,
                                      int64_t n, int32_t reps, lloid_tuning* out);

/* Gaps in the strain (the pipeline's source turns missing data into gap
 * buffers, Section II.B): with this flag a push whose t0 lies past the end of
 * the detector's stream first fills the missing samples with zeros, exactly as
 * if zeros had been pushed, instead of returning LLOID_EGAP.  A push that
 * starts before the stream end is still LLOID_EGAP. */
#define LLOID_FLAG_FILL_GAPS 8u

/* Fault injection on the host side, for testing how a caller copes with
 * failures.  None of these faults, traps or stalls the GPU:
 *   LLOID_FAULT_ALLOC        the context's next `count` device allocations
 *                            fail (LLOID_ENOMEM; a failed load_bank keeps
 *                            nothing);
 *   LLOID_FAULT_DROP_BLOCK   the next `count` pushes are lost: they return
 *                            LLOID_OK and change nothing (the next push then
 *                            finds a gap);
 *   LLOID_FAULT_DELAY        the next push starts after a bounded spin of
 *                            `count` microseconds (at most 10 s) on the
 *                            context's stream: a slow device, so that a pull
 *                            with a short timeout returns LLOID_ETIMEOUT;
 *   LLOID_FAULT_WAIT_EXPIRY  one bounded device wait with a limit of `count`
 *                            microseconds (at most 1 s) on a barrier that
 *                            nothing completes: it expires as a stalled
 *                            pipeline wait would and leaves its code in the
 *                            context's error flag, so that pulls and
 *                            lloid_synchronize report LLOID_ETIMEOUT until
 *                            lloid_clear_error.
 * count = 0 cancels a pending fault of that kind.  EINVAL for an unknown
 * kind or a negative count. */
#define LLOID_FAULT_ALLOC 1
#define LLOID_FAULT_DROP_BLOCK 2
#define LLOID_FAULT_DELAY 3
#define LLOID_FAULT_WAIT_EXPIRY 4
LLOID_API lloid_status lloid_inject_fault(lloid_ctx* ctx, int32_t kind, int64_t count);

/* Clear the device-side error flag that an expired wait leaves (after waiting
 * for the context's stream).  The results of pushes enqueued before the
 * expiry are not to be trusted; the context itself stays usable. */
LLOID_API lloid_status lloid_clear_error(lloid_ctx* ctx);
LLOID_API lloid_status lloid_stage_times(lloid_ctx* ctx, double* ms, int64_t* launches, int reset);

/* Allocation-free trigger extraction (no counterpart in the paper; a service
 * for callers that cannot allocate device memory while they run, such as a
 * real-time strain callback that must not block in cudaMalloc, or a host
 * framework that owns the device memory pool).  Finds the triggers of an SNR
 * block the caller already holds: z is a DEVICE array [2 n_templates][n]
 * (row 2i real, 2i+1 imaginary part of template i) covering full-rate samples
 * [t0, t0 + n), with t0 and n multiples of `window`.  Per window and template
 * the maximum |z| (earliest sample on ties) becomes a trigger if it exceeds
 * `threshold`; the window's loudest template (lowest index on ties) is
 * flagged is_bank_max -- the same rules as lloid_pull_triggers.  Triggers go
 * to the DEVICE array out[cap] in (window, template) order with `detector`
 * and `bank` copied into each record; the total count (even when above cap)
 * goes to the DEVICE int64 *n_out.  Work is enqueued on `stream` (a
 * cudaStream_t, NULL = legacy default stream) and the call returns at once.
 * It calls no allocating routine: its scratch is one array compiled into the
 * library (about 4.2 MB on every GPU that loads it, held until exit), whose
 * device address the first call on each device looks up -- make that first
 * call before any stream capture.  Every call shares that array and leaves
 * its contents behind (each call rewrites all it reads), so calls whose GPU
 * work overlaps race: serialise them.  LLOID_ERANGE when n_templates x
 * (n / window) exceeds 262144 (split the block), LLOID_EINVAL on bad
 * arguments, LLOID_ECUDA if a launch fails. */
LLOID_API lloid_status lloid_triggers_from_snr_noalloc(const float* z, int32_t n_templates, int64_t n, int64_t t0,
                                                       int64_t window, float threshold, int32_t detector,
                                                       int32_t bank, lloid_trigger* out, int64_t cap,
                                                       int64_t* n_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LLOID_H */
