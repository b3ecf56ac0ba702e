/*
 * lsp.h -- C ABI of the GB300 (sm_103a) Lomb-Scargle periodogram engine.
 *
 * The engine evaluates the normalized Lomb-Scargle periodogram of an
 * unevenly sampled series (Townsend, "Fast Calculation of the Lomb-Scargle
 * Periodogram Using Graphics Processing Units", Sec. 3, Eq. 1-2, computed
 * through the single-pass sums of Eq. 5-8) on a uniform frequency grid
 * (Sec. 4.2, Eq. 9-11).  All arithmetic runs in the library's own CUDA
 * kernels; there is no CPU fallback.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers may be device pointers (cudaMalloc / torch CUDA tensors) or host
 *   pointers (pageable or pinned).  The kind is detected per pointer.  Host
 *   inputs are copied to library-owned device buffers; a host output makes
 *   the call block until the result has been copied back.  With device
 *   pointers only, a call is asynchronous on the context's stream: it returns
 *   after argument checks and kernel launches, and errors found on the device
 *   (non-finite data, zero variance) are reported by lsp_sync().
 * - The caller owns every array it passes; the library owns only the context
 *   and its workspace (grown on demand, freed by lsp_destroy).
 * - Every function returns an lsp_status; lsp_last_error() gives the text of
 *   the last failure on that context.  A failed call leaves outputs undefined.
 * - A context is not thread-safe: one host thread at a time.
 */
#ifndef LSP_H
#define LSP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LSP_ABI_VERSION 1

typedef struct lsp_ctx lsp_ctx;

typedef enum lsp_status {
    LSP_OK = 0,
    LSP_ERR_INVALID_ARG = 1,  /* size, grid or pointer argument out of range   */
    LSP_ERR_DEGENERATE = 2,   /* the data have zero variance (Sec. 3 needs >0)  */
    LSP_ERR_NONFINITE = 3,    /* NaN or Inf among t, X or the grid               */
    LSP_ERR_OOM = 4,          /* workspace allocation failed                     */
    LSP_ERR_CUDA = 5,         /* a CUDA runtime call failed (text in last_error) */
    LSP_ERR_TIMEOUT = 6,      /* lsp_sync deadline passed; work still queued     */
    LSP_ERR_NO_MODEL = 7,     /* false-alarm surrogate has no weights loaded     */
    LSP_ERR_UNSUPPORTED = 8   /* option combination not provided                 */
} lsp_status;

/* How sin/cos of the phase are produced in the O(N_t N_f) loop. */
typedef enum lsp_sincos_mode {
    LSP_SINCOS_AUTO = 0,   /* the library's choice (currently RECUR3_X2)                 */
    LSP_SINCOS_MUFU = 1,   /* hardware sin/cos (SFU) of every phase (Sec. 4.3's choice)  */
    LSP_SINCOS_RECUR = 2,  /* SFU seed per strip of adjacent frequencies, then the
                              angle-addition rotation by (cos, sin)(2 pi t_j df) on FMA */
    LSP_SINCOS_RECUR3 = 3, /* SFU seed, one rotation, then the three-term form
                              z_{k+1} = 2 cos(2 pi t_j df) z_k - z_{k-1} (half the FMA work
                              of RECUR; error grows faster with the strip length)      */
    LSP_SINCOS_RECUR3_X2 = 4 /* RECUR3 in packed FP32x2 FMA: the (cos, sin) pair of a
                              frequency in the two lanes of every FFMA2, each sum pair
                              and the three-term step one FFMA2, so the same roundings
                              (results bit-identical to RECUR3 at the same strip
                              length) in half the instructions                       */
} lsp_sincos_mode;

/* How the phase f_k t_j is formed. */
typedef enum lsp_phase_mode {
    LSP_PHASE_FIXED64 = 0,    /* exact: frac(t_j df), frac(t_j f_0) as 64-bit fixed-point
                                 turns, phase = v_j + k u_j mod 2^64                      */
    LSP_PHASE_NAIVE_FP32 = 1  /* the paper's single-precision f*t minus rintf (Sec. 4.3);
                                 a comparator that loses accuracy when f*t is large     */
} lsp_phase_mode;

typedef struct lsp_options {
    int32_t sincos_mode;      /* lsp_sincos_mode                                       */
    int32_t phase_mode;       /* lsp_phase_mode                                        */
    int32_t freqs_per_thread; /* adjacent frequencies per thread: 0 = auto, else 4|8|12|16|24,
                                 or 20|28 with the recurrences; multi-realization
                                 batches take it when their kernels have that shape
                                 (12 with 4 realizations, 16 with 2)                    */
    int32_t split;            /* N_t-splits per frequency block: 0 = auto (chunks of
                                 64 .. 16,384 samples), else 1 .. 65535                 */
    int32_t timing;           /* nonzero: record per-kernel CUDA-event times            */
    int32_t mlp_fp32;         /* surrogate network: 0 = BF16 activations, 1 = FP32      */
    int32_t batch_rhs;        /* lsp_batch and lsp_batch_gls_noise with n_real > 1:
                                 realizations sharing one pass over the samples
                                 (0 = auto, 1 = one at a time, 2|4|8)                  */
    int32_t reserved[5];      /* must be zero                                          */
} lsp_options;

/* Fill *opt with the defaults (AUTO sin/cos, FIXED64 phase, automatic launch shape). */
void lsp_default_options(lsp_options *opt);

/*
 * Create a context on CUDA device `device`.  `opt` may be NULL (defaults).
 * `cuda_stream` is a cudaStream_t to run on, or NULL for a stream the
 * context creates and owns.  *out receives the context.
 * Errors: INVALID_ARG (bad device or options), CUDA.
 */
lsp_status lsp_create(lsp_ctx **out, int device, const lsp_options *opt, void *cuda_stream);

/* Replace the context's options (same rules as lsp_create). */
lsp_status lsp_set_options(lsp_ctx *ctx, const lsp_options *opt);

/* Make later calls run on `cuda_stream` (NULL: the context's own stream). */
lsp_status lsp_set_stream(lsp_ctx *ctx, void *cuda_stream);

/*
 * Normalized Lomb-Scargle periodogram on a uniform grid (Eq. 1-2 through
 * Eq. 5-8; the grid of Eq. 9 with an explicit origin):
 *     P_out[k] = P_n(f_0 + k df),  k = 0 .. N_f-1.
 * t[N_t]: sample times (FP64, any order, any origin; a common offset does
 * not change P_n).  X[N_t]: measurements (FP64); the library shifts and
 * scales them to zero mean and unit population variance (Sec. 3).  f_0, df:
 * grid origin and spacing in cycles per time unit (any finite values; the
 * paper's grid is f_0 = df, see lsp_grid).  P_out[N_f]: FP32 output.
 * N_t >= 2, 0 <= N_f < 2^31.  N_f = 0 is a no-op.  A term of Eq. 1 whose
 * denominator falls below N_t * 2^-16 (e.g. the sine term at the Nyquist
 * frequency of an even grid) is taken as zero.  The fixed-point phase needs
 * |t_j - t_min| f_0 and |t_j - t_min| df below 2^52 turns; beyond that the
 * call's P is NaN and lsp_sync returns INVALID_ARG.
 * Errors: INVALID_ARG (also the phase range, on the device), NONFINITE
 * (f_0/df at call time; t/X on the device), DEGENERATE (zero variance, on
 * the device), OOM, CUDA.  Every entry point that takes arrays refuses, with
 * INVALID_ARG, device memory that belongs to another GPU than the context's.
 */
lsp_status lsp_periodogram(lsp_ctx *ctx, const double *t, const double *X, int64_t N_t,
                           double f_0, double df, int64_t N_f, float *P_out);

/*
 * Floating-mean ("generalized") periodogram on the same grid: the extension
 * Sec. 6.3 names (Shrager 2001; Zechmeister & Kuerster 2009), where the mean is
 * fitted together with the sinusoid rather than removed beforehand, and each
 * sample carries the weight w_j = (1/dy_j^2) / sum(1/dy^2) (equal weights when
 * dy is NULL).  With p(f) the fraction of the weighted variance of X that the
 * best fit a cos 2 pi f t + b sin 2 pi f t + c removes (0 <= p <= 1):
 *     P_out[k] = (N_t / 2) p(f_0 + k df),
 * the scale of lsp_periodogram's P_n (the two agree where sum w cos and
 * sum w sin vanish, e.g. Fourier frequencies of an even grid).  Where the
 * centred cos and sin are linearly dependent on the samples (f = 0, Nyquist
 * of an even grid) the fit uses the remaining direction; where both vanish,
 * P = 0.  Same t, X, grid and pointer rules as lsp_periodogram; dy[N_t]
 * (FP64, optional, host or device) must be finite and > 0, with 1/dy^2 a
 * finite nonzero FP32 number (about 1e-19 < dy < 1e19: the weights are formed
 * in FP32, summed in FP64).  N_t >= 3.
 * sincos_mode selects MUFU, RECUR, RECUR3 or RECUR3_X2 (AUTO: RECUR3_X2);
 * strips are 8, 12 or 16 frequencies (freqs_per_thread 8, 12 or 16; other
 * values use 16, 8 for MUFU).
 * Errors: INVALID_ARG (also a bad dy, on the device), NONFINITE, DEGENERATE,
 * UNSUPPORTED (phase_mode NAIVE_FP32), OOM, CUDA.
 */
lsp_status lsp_periodogram_gls(lsp_ctx *ctx, const double *t, const double *X, const double *dy,
                               int64_t N_t, double f_0, double df, int64_t N_f, float *P_out);

/*
 * The floating-mean periodogram of many measured curves in one persistent
 * launch (the lsp_batch layout without noise realizations): curve c has
 * samples t[t_off[c] .. t_off[c+1]) with values X and optional errors dy in the
 * same layout (NULL: equal weights), at least 3 samples, and its own grid
 * f_0[c] + k df[c], k < N_f[c].  Outputs as in lsp_batch with n_real = 1: P
 * of curve c at P_out[P_off[c] + k] (optional), per-curve max P and its bin
 * (optional; argmax -1 for an empty grid).  Pointers host or device; any host
 * output makes the call blocking.  The call shares lsp_batch's workspace, so
 * a later lsp_batch on the same context re-plans its graph.
 * Errors: as lsp_periodogram_gls, plus INVALID_ARG for bad metadata.
 */
lsp_status lsp_batch_gls(lsp_ctx *ctx, int32_t n_curves, const int64_t *t_off, const double *t,
                         const double *X, const double *dy, const double *f_0, const double *df,
                         const int64_t *N_f, float *P_out, const int64_t *P_off, float *maxP_out,
                         int32_t *argmax_out);

/*
 * Monte-Carlo noise periodograms in the floating-mean form (Sec. 6.2's
 * Monte Carlo applied to the Sec. 6.3 extension): the statistics of its
 * noise peaks depend on the errors as well as on the sampling pattern, so the
 * noise carries them.  Realization r of curve c (r < n_real) is
 * X_j = dy_j z_j with z_j the N(0,1) value that lsp_batch draws for
 * (seed, c, r, j) (see lsp_noise; X_j = z_j when dy is NULL), and its
 * periodogram is lsp_batch_gls's of that X with the same dy: weights 1/dy^2,
 * the offset fitted.  Layout and outputs as lsp_batch with n_real
 * realizations: P of realization r, curve c, bin k at
 * P_out[r * P_off[n_curves] + P_off[c] + k] (optional); maxP_out, argmax_out
 * [n_real * n_curves] at r * n_curves + c.  n_real in [1, 65535]; curves of at
 * least 3 samples.  Groups of R realizations (the batch_rhs option; auto: 8
 * from 8 realizations on, else 4; 1 = one at a time) share each pass over a
 * curve's samples: the phase, the recurrence and the sums of the sampling
 * pattern and weights are computed once for the group, only XC, XS per
 * realization (strips of 8 frequencies for R = 2, 4, of 4 for R = 8; one at a
 * time, strips of 16 or 8), one persistent launch over (curve, group,
 * frequency block) items; each (frequency, realization) is computed exactly
 * as the one-at-a-time kernel with the same strip length would.  Runs the
 * packed three-term strip (sin/cos mode AUTO or RECUR3_X2; other modes return
 * UNSUPPORTED).
 * Pointers host or device; any host output makes the call blocking.
 * Errors: INVALID_ARG, NONFINITE, UNSUPPORTED, OOM, CUDA.
 */
lsp_status lsp_batch_gls_noise(lsp_ctx *ctx, int32_t n_curves, const int64_t *t_off, const double *t,
                               const double *dy, uint64_t seed, int32_t n_real, const double *f_0,
                               const double *df, const int64_t *N_f, float *P_out, const int64_t *P_off,
                               float *maxP_out, int32_t *argmax_out);

/*
 * Fast approximate P_n by the method of Press & Rybicki (1989), which the
 * paper's introduction cites as the O(N log N) alternative to the direct
 * evaluation: the normalized data are spread ("extirpolated") onto a uniform
 * periodic grid of n_fft = 2^p >= 2 macc (f_0/df + N_f) nodes spanning 1/df
 * with macc-point Lagrange weights (and unit values at the positions of
 * 2(t - t0) for the tau sums), one FFT gives the sums of Eq. 5-8 at every
 * multiple of df, and Eq. 5-6 follow.  Same arguments as lsp_periodogram plus
 * macc (even, 2..16; 0 = 4).  f_0 must be a non-negative integer multiple of
 * df (the grid of Eq. 9 is: f_0 = df).  Accuracy: the extirpolation error,
 * about 1e-4 max P at macc = 4 and falling fast with macc; exact when every
 * sample sits on a grid node.  Workspace: 32 n_fft bytes (n_fft <= 2^28).
 * Errors: INVALID_ARG (also f_0 not on the FFT grid, bad macc, grid too
 * large), NONFINITE, DEGENERATE, OOM, CUDA.
 */
lsp_status lsp_press_rybicki(lsp_ctx *ctx, const double *t, const double *X, int64_t N_t, double f_0,
                             double df, int64_t N_f, int32_t macc, float *P_out);

/*
 * Many periodograms in one call: measured curves, or Monte-Carlo noise
 * realizations of sampling patterns (Sec. 6.2: the distribution of peak
 * heights under pure noise, e.g. the number of independent frequencies that
 * Eq. 3's exponent should be).  One persistent kernel takes work items
 * (realization, curve, block of frequencies) longest curve first; the whole
 * batch runs as one CUDA graph, cached and replayed while the arguments'
 * pointers and metadata stay the same (a new seed needs no new graph).
 *
 * n_curves in [1, 65535]; curve c has samples t[t_off[c] .. t_off[c+1]) (FP64,
 * t_off[0] = 0, at least 2 samples per curve) and its own grid
 * f_0[c] + k df[c], k < N_f[c] (0 <= N_f[c] < 2^31).
 * X: measurements in the same layout (n_real must then be 1), or NULL for
 *   noise: realization r of curve c, sample j, is N(0,1) from Philox-4x32-10
 *   with counter (j/4, c, r, 0) and key `seed` (see lsp_noise), normalized
 *   per realization like measured data (Sec. 3).  n_real in [1, 65535].
 * P_out (optional): P of realization r, curve c, bin k at
 *   P_out[r * P_off[n_curves] + P_off[c] + k]; P_off[c+1] - P_off[c] >= N_f[c].
 * maxP_out, argmax_out (optional, [n_real * n_curves], index r * n_curves + c):
 *   the largest P of each periodogram and its bin k (lowest k on ties; -1 and
 *   0 for a curve with N_f = 0).
 * With n_real > 1, groups of R realizations (the batch_rhs option; auto: 8
 * when n_real >= 8, else 4) share each pass over a curve's samples: the
 * phase, the sin/cos recurrence and CC, CS are computed once for the group
 * and only XC, XS per realization (strips of 16, 12, 8 frequencies for
 * R = 2, 4, 8), which halves the arithmetic per periodogram.  With
 * n_real >= 4 R, CC and CS (which depend on the sampling pattern only) come
 * from one extra pass per curve instead of from every group.  Under the AUTO
 * (= RECUR3_X2) sin/cos mode the groups run the packed strip.  Each
 * (frequency, realization) is computed exactly as the one-at-a-time kernel
 * with the same strip length would.
 * A work item sums over all samples of its curve in FP32 (the batch does not
 * split N_t), so curves far beyond 10^6 samples are better served by
 * lsp_periodogram, which bounds each running sum to 16,384 samples.
 * At least one output must be given.  Arrays may be host or device pointers
 * (metadata is read on the host in either case); the sin/cos mode and strip
 * length follow the context's options (the naive FP32 phase is not offered).
 * Errors: INVALID_ARG, NONFINITE (grid; t/X on the device), DEGENERATE
 * (measured X with zero variance, on the device), UNSUPPORTED, OOM, CUDA.
 */
lsp_status lsp_batch(lsp_ctx *ctx, int32_t n_curves, const int64_t *t_off, const double *t,
                     const double *X, uint64_t seed, int32_t n_real, const double *f_0,
                     const double *df, const int64_t *N_f, float *P_out, const int64_t *P_off,
                     float *maxP_out, int32_t *argmax_out);

/*
 * The raw N(0,1) noise lsp_batch draws for (seed, curve, realization), samples
 * 0..N-1, before normalization: Philox-4x32-10 (Salmon et al. 2011) block
 * j/4 with counter (j/4, curve, real, 0) and key (seed low word, seed high
 * word); each word w gives u = (2 (w >> 9) + 1) 2^-24, and Box-Muller turns
 * (u0, u1), (u2, u3) into sqrt(-2 ln u_a) (cos, sin)(2 pi u_b).  out[N] FP32,
 * host or device.  Errors: INVALID_ARG, OOM, CUDA.
 */
lsp_status lsp_noise(lsp_ctx *ctx, uint64_t seed, int32_t curve, int32_t real, int64_t N, float *out);

/*
 * Grid helper, Eq. 10-11 with Eq. 9's origin: df = 1/(F_over (t_max - t_min)),
 * N_f = floor(F_high F_over N_t / 2), f_0 = df.  Host-only arithmetic.
 * Errors: INVALID_ARG (t_max <= t_min, F_over <= 0, F_high <= 0, N_t < 1).
 */
lsp_status lsp_grid(double t_min, double t_max, int64_t N_t, double F_over, double F_high,
                    double *f_0, double *df, int64_t *N_f);

/*
 * Autotuner: time the sin/cos modes, strip lengths F (also the recurrence's
 * re-seed length) and N_t splits on a synthetic series of this size, keep
 * only candidates within 2e-5 max P of the all-hardware-sin/cos result, and
 * remember the fastest for this (log2 N_t, log2 N_f) bucket: later calls with
 * LSP_SINCOS_AUTO and automatic F/split use it.  *chosen (may be NULL)
 * receives the winning options.  Blocks; allocates temporary buffers.
 * Errors: INVALID_ARG, OOM, CUDA.
 */
lsp_status lsp_autotune(lsp_ctx *ctx, int64_t N_t, int64_t N_f, lsp_options *chosen);

/*
 * Autotuner of lsp_batch (the persistent Monte-Carlo launch of Sec. 6.2):
 * times launch shapes on the caller's own batch description (curves, grids
 * and n_real noise realizations, drawn from a fixed internal seed) and keeps
 * the fastest whose per-periodogram maxima agree with the first shape's to
 * 2e-5 (relative).  Shapes: for n_real = 1, the packed three-term recurrence
 * with strips of F = 24 or 16 frequencies, tail strips of 8, 4 or none after
 * a curve's last full block, and shared-memory tiles of 128, 256 or 512
 * samples, the scalar three-term and the angle-addition recurrences at their
 * default shapes; for n_real > 1, realization groups R = 4 (F = 12 or 8, the
 * three tiles), 2, 8 and 1, and the packed strips of the groups that read the
 * window pass.  The choice is
 * remembered for this batch's size bucket (log2 of its terms per
 * realization, log2 of its mean N_t, its realization count 1 / 2-3 / 4-7 / 8+):
 * later lsp_batch calls in that bucket use it when the options leave the
 * choice to the library (AUTO sin/cos, freqs_per_thread 0, batch_rhs 0).
 * *chosen (may be NULL) receives the winner as options.  Arrays as lsp_batch
 * (host or device).  Blocks; allocates temporary buffers.
 * Errors: INVALID_ARG, OOM, CUDA.
 */
lsp_status lsp_autotune_batch(lsp_ctx *ctx, int32_t n_curves, const int64_t *t_off, const double *t,
                              const double *f_0, const double *df, const int64_t *N_f, int32_t n_real,
                              lsp_options *chosen);

/*
 * The context's tuning table (lsp_autotune and lsp_autotune_batch entries)
 * to and from a JSON file keyed by the GPU's name: {"lsp_tune": 1,
 * "device": "<name>", "entries": [one object per line]}.  Loading merges the
 * file's entries into the table (an entry replaces one of the same bucket)
 * when the file was written on a GPU of the same name, and skips shapes this
 * build does not have; *n_loaded (may be NULL) receives the count.
 * Errors: INVALID_ARG (unreadable or not a tuning file).
 */
lsp_status lsp_tune_save(lsp_ctx *ctx, const char *path);
lsp_status lsp_tune_load(lsp_ctx *ctx, const char *path, int32_t *n_loaded);

/*
 * Pipe-rate probe: the per-SM, per-clock rates of the operations the
 * periodogram kernels are built from, measured on the context's GPU (Sec. 5.3
 * puts the GPU's lead down to its sin/cos throughput; these are the
 * denominators of the kernels' rooflines).  Each rate comes from one launch
 * of independent dependency chains on 4 CTAs of 256 threads per SM, timed
 * with clock64 (slowest CTA) after one untimed launch.
 */
typedef struct lsp_pipe_rates {
    int32_t sms;                   /* streaming multiprocessors                        */
    double sm_mhz;                 /* SM clock during the FMA probe: its cycles over its
                                      CUDA-event time (a little low: the event also
                                      spans the launch)                               */
    double sincos_per_clk_sm;      /* __sincosf pairs (2 SFU ops each) per clock per SM */
    double ffma_per_clk_sm;        /* FP32 FMA per clock per SM                        */
    double ffma2_lanes_per_clk_sm; /* lanes of packed FP32x2 FMA per clock per SM      */
} lsp_pipe_rates;

/*
 * Runs the probe on the context's stream and blocks until it is done;
 * allocates and frees its own small buffers (so it synchronizes the device).
 * out: host struct, filled on success.  Errors: INVALID_ARG, OOM, CUDA.
 */
lsp_status lsp_probe_pipes(lsp_ctx *ctx, lsp_pipe_rates *out);

/*
 * Wait for the context's queued work, at most `timeout_s` seconds (< 0: no
 * limit), polling a CUDA event.  Returns TIMEOUT if the deadline passes (the
 * work stays queued), else the first device-detected data error of the calls
 * since the previous lsp_sync (DEGENERATE / NONFINITE), else OK.
 */
lsp_status lsp_sync(lsp_ctx *ctx, double timeout_s);

/*
 * CUDA-event durations (milliseconds) of the kernels of the last call, when
 * the context's `timing` option is set: prep (normalization + phase
 * records), main (the O(N_t N_f) evaluation) and finalize (split reduction
 * and Eq. 5).  Blocks until those events complete.  Any pointer may be NULL.
 * Errors: INVALID_ARG (timing off or no call yet), CUDA.
 */
lsp_status lsp_last_timing(lsp_ctx *ctx, float *ms_prep, float *ms_main, float *ms_finalize);

/* Kernel launches made by the last call (0 before the first). */
int32_t lsp_last_launch_count(const lsp_ctx *ctx);

/* Text of the last error on this context ("" if none).  Owned by the context. */
const char *lsp_last_error(const lsp_ctx *ctx);

/* ---------------------------------------------------------------------------
 * Learned false-alarm surrogate.  Eq. 3 turns a peak height into a false-alarm
 * probability by treating the N_f grid frequencies as independent; Sec. 6.2
 * notes that the exponent should be an empirical number of independent
 * frequencies that depends on the sampling, estimated by Monte-Carlo noise
 * periodograms.  The surrogate learns, from 32 features of the sampling
 * pattern, the quantiles of the largest noise peak at the levels
 * p = 0.05, 0.10, 0.25, 0.50, 0.75, 0.90, 0.95, 0.98, 0.99 (the peak height
 * whose false-alarm probability is 1 - p).  Network: 32 -> H -> H -> H -> 9,
 * GELU (exact erf form), FP32 master weights, activations in BF16 (or FP32
 * with the mlp_fp32 option), and a head on Eq. 3's quantiles: with
 * e_l = log q_l^Eq3(N_t, N_f) and d_l = e_l - e_{l-1}, log q_1 = e_1 + z_1 and
 * log q_l = log q_{l-1} + d_l softplus(z_l) / log 2 (monotone in l; z = 0 is
 * Eq. 3 exactly, and the output layer starts at zero).  Trained with the mean
 * pinball loss and Adam (beta 0.9/0.999, eps 1e-8).  All of it runs in the
 * library's kernels.
 * ------------------------------------------------------------------------- */

#define LSP_FAP_FEATURES 32
#define LSP_FAP_LEVELS 9

/*
 * Features of n sampling patterns (CSR t_off/t, sorted times, 2 .. 2^31 - 1
 * samples each; grid f_0 >= 0, df > 0, N_f >= 1 as for lsp_batch) into
 * features[n][32] (FP32).  With T = t_last - t_first, dt the M = N - 1 gaps,
 * q(p) = sorted(dt)[floor(p (M - 1))], med = q(1/2), f_max = f_0 + (N_f-1) df:
 *   0 log N, 1 log T, 2 log N_f, 3 log(1/(df T)), 4 log(f_max T / N), 5 log(1 + f_0/df),
 *   6..10 log(max(q(p), 1e-12 T) / (T/M)), p = 0.05, 0.25, 0.5, 0.75, 0.95,
 *   11..13 sum of gaps with dt/med > c (1 + 1e-6), over T, c = 2, 10, 100,
 *   14 max dt / T, 15 fraction of gaps with dt/med > 2 (1 + 1e-6),
 *   16..23 the 8 highest local maxima of the spectral window
 *          W(f) = |sum_j exp(2 pi i f t_j)|^2 / N^2 on f_m = m df, m = 1..floor(f_max/df),
 *          outside the main lobe (f_m T >= 1), ties to lower m, 0 if missing,
 *   24..31 their f_m / f_max.
 * Unsorted times give NaN features and NONFINITE from lsp_sync.
 * Errors: INVALID_ARG, OOM, CUDA.
 */
lsp_status lsp_fap_features(lsp_ctx *ctx, int32_t n, const int64_t *t_off, const double *t,
                            const double *f_0, const double *df, const int64_t *N_f, float *features);

/*
 * Initialize the network with H hidden units (0: 256) from `seed` (He-normal
 * hidden weights, zero output layer and biases, Adam moments zero) and set the input standardization
 * to the column mean / standard deviation of features[n_rows][32].
 */
lsp_status lsp_fap_init(lsp_ctx *ctx, int32_t hidden, uint64_t seed, int32_t n_rows, const float *features);

/*
 * One Adam step on a minibatch of B rows.  Row r = rows[i] (device int32)
 * takes features[r % n_pat][32], counts[r % n_pat][2] = (N_t, N_f) and the
 * target targets[r] (a noise-peak maximum); all four tables are device arrays.
 * loss_out (host or device, may be NULL) receives the minibatch's mean
 * pinball loss before the step.
 */
lsp_status lsp_fap_train_step(lsp_ctx *ctx, int32_t B, const int32_t *rows, int32_t n_pat,
                              const float *features, const float *counts, const float *targets,
                              float lr, float *loss_out);

/* Report of lsp_fap_train (host struct, filled on success). */
typedef struct lsp_train_report {
    int32_t best_step;        /* steps taken before the kept weights (0: the network as it
                                 was before the call)                                    */
    int32_t evaluations;      /* validation passes run, the one before training included  */
    float val_loss_initial;   /* validation pinball loss before the first step (right after
                                 lsp_fap_init: exactly Eq. 3's quantiles)                 */
    float val_loss_best;      /* validation pinball loss of the kept weights              */
    float train_loss_last;    /* mean minibatch pinball loss of the steps after the
                                 second-to-last validation pass                           */
    float gpu_ms;             /* CUDA-event time of the whole loop on the context's stream */
} lsp_train_report;

/*
 * Training set, validation set and schedule of lsp_fap_train.  Every table is
 * a device array of the context's GPU (FP32, row-major).
 */
typedef struct lsp_train_opts {
    int32_t n_pat;              /* training patterns (>= 1)                                   */
    int32_t n_rows;             /* training rows (>= 1): row r pairs pattern r % n_pat with
                                   target r (several noise realizations per pattern)         */
    const float *features;      /* [n_pat][32]: lsp_fap_features of the patterns            */
    const float *counts;        /* [n_pat][2]: (N_t, N_f) of the patterns                   */
    const float *targets;       /* [n_rows]: the largest P of row r's noise periodogram      */
    int32_t n_val_pat;          /* validation patterns (1 .. 65535)                          */
    int32_t n_val_real;         /* noise realizations per validation pattern (>= 1)          */
    const float *val_features;  /* [n_val_pat][32]                                           */
    const float *val_counts;    /* [n_val_pat][2]                                            */
    const float *val_targets;   /* [n_val_real][n_val_pat]: largest P of realization r of
                                   validation pattern i at [r][i]                            */
    int32_t steps;              /* Adam steps (>= 1)                                          */
    int32_t batch;              /* rows per minibatch (1 .. 65536), drawn with replacement   */
    int32_t warmup_steps;       /* linear warm-up of the learning rate (0 .. steps)          */
    int32_t eval_every;         /* validation pass every so many steps, and after the last
                                   (0: only before the first and after the last step)       */
    float lr;                   /* peak learning rate (> 0)                                  */
    float lr_final;             /* cosine decay ends at lr * lr_final (0 .. 1)               */
    float weight_decay;         /* decoupled weight decay per unit of lr (>= 0; 0 = Adam)   */
    int32_t reserved0;          /* must be zero                                              */
    uint64_t seed;              /* minibatch draws: Philox-4x32-10 block (i/4, step,
                                   0x54524e52, 0) under key (seed low, seed high), word i%4
                                   w gives row floor(w n_rows / 2^32)                       */
    float *val_history;         /* optional [evaluations]: validation loss of each pass,
                                   host or device (size: 2 + (steps - 1) / eval_every with
                                   eval_every > 0, else 2)                                   */
    float *train_history;       /* optional, same size: mean minibatch loss of the steps
                                   before each pass (NaN for the pass before training)      */
    lsp_train_report *report;   /* optional host struct                                      */
} lsp_train_opts;

/*
 * Train the surrogate's network (lsp_fap_init or lsp_fap_load first) for
 * opt->steps Adam steps entirely on the GPU: each step draws its minibatch
 * rows from the Philox stream above, runs the forward and backward pass and
 * the Adam update (beta 0.9/0.999, eps 1e-8, decoupled weight decay) at the
 * step's learning rate (linear warm-up, then cosine decay from lr to
 * lr * lr_final); every eval_every steps the mean pinball loss of the
 * validation set is reduced on the device, and the weights with the lowest
 * validation loss so far (the initial weights included) are kept; they are
 * the context's network when the call returns.  This is the Monte-Carlo
 * estimate Sec. 6.2 asks for, learned: the targets are noise-periodogram
 * maxima from lsp_batch, and the head starts from Eq. 3's quantiles.
 * Blocks until the loop is done.  Deterministic for a given seed.
 * Errors: INVALID_ARG (sizes, schedule, non-device tables), NO_MODEL, OOM, CUDA.
 */
lsp_status lsp_fap_train(lsp_ctx *ctx, const lsp_train_opts *opt);

/* Gradient of the mean pinball loss of B rows w.r.t. the flat parameter
 * vector (layout W1[32][H] b1 W2[H][H] b2 W3[H][H] b3 W4[H][9] b4) into
 * grad_out, without updating anything; loss_out as above. */
lsp_status lsp_fap_gradients(lsp_ctx *ctx, int32_t B, const float *features, const float *counts,
                             const float *targets, float *grad_out, float *loss_out);

/* Quantiles q_out[B][9] of B feature rows with counts (N_t, N_f). */
lsp_status lsp_fap_eval(lsp_ctx *ctx, int32_t B, const float *features, const float *counts, float *q_out);

/* Features + quantiles of n sampling patterns (N_t >= 4): quantiles_out[n][9]. */
lsp_status lsp_fap_predict(lsp_ctx *ctx, int32_t n, const int64_t *t_off, const double *t,
                           const double *f_0, const double *df, const int64_t *N_f,
                           float *quantiles_out);

/* Flat parameters followed by the 32 feature means and 32 scales; with
 * out = NULL only *n_out is set.  set_params replaces them (Adam state reset). */
lsp_status lsp_fap_get_params(lsp_ctx *ctx, float *out, int64_t capacity, int64_t *n_out);
lsp_status lsp_fap_set_params(lsp_ctx *ctx, int32_t hidden, const float *in, int64_t n);

/* Checkpoint (weights, standardization, Adam moments and step, checksum) to
 * and from a file; load rejects a file whose checksum does not match. */
lsp_status lsp_fap_save(lsp_ctx *ctx, const char *path);
lsp_status lsp_fap_load(lsp_ctx *ctx, const char *path);

/* Release the context, its stream (if owned) and its workspace.  NULL is a no-op. */
void lsp_destroy(lsp_ctx *ctx);

/*
 * Allocation-free variant of lsp_periodogram.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * while they run -- e.g. an application whose memory pool already owns the
 * whole GPU, or a latency-critical loop that cannot afford cudaMalloc's
 * device-wide synchronization.  It computes the same P_out[k] = P_n(f_0 + k df)
 * (packed three-term recurrence sin/cos, fixed-point phase) without a context and without any
 * cudaMalloc/cudaFree or allocating library call.
 *
 * Scratch: one file-scope device array of 64 MiB + 8 KiB that every GPU which
 * loads the library holds until the process exits.  Limit: 2 <= N_t <= 524,288
 * (larger N_t returns LSP_ERR_INVALID_ARG); N_f < 2^31 as for lsp_periodogram.
 * Accuracy is that of lsp_periodogram: every FP32 running sum covers at most
 * 16,384 samples.  When the partial sums of that many chunks do not fit the
 * array at once (N_t > 16,384 with a long grid: at N_t = 524,288, beyond
 * 98,304 frequencies), the grid is evaluated in frequency tiles, one
 * main-kernel launch each, with the phase origin of each tile moved exactly.
 * t, X and P_out must be device (or managed) memory of the current device:
 * host memory and device memory of another GPU return INVALID_ARG.  The work
 * is queued on `cuda_stream` (NULL: the legacy default stream) and the call
 * returns without waiting.  The first call on a device,
 * with that device current, looks up the array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any
 * stream capture.  Every call shares the one array and it keeps the last
 * call's contents, so calls that overlap on the GPU (other streams, other
 * host threads) race and must be serialized by the caller.  Data errors
 * found on the device (non-finite input, zero variance, a phase beyond the
 * 2^52-turn range of the fixed-point phase) are not reported by status: they
 * show as NaN in P_out.
 * Errors: INVALID_ARG, NONFINITE (f_0/df), CUDA.
 */
lsp_status lsp_periodogram_noalloc(const double *t, const double *X, int64_t N_t, double f_0,
                                   double df, int64_t N_f, float *P_out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* LSP_H */
