// lsp_kernels.cuh -- internal declarations shared by the library's .cu files.
// Nothing here is part of the public ABI (include/lsp.h is).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lsp {

// Device status bits, OR-ed into a context-owned word by the kernels.
enum : int {
    kStatusNonFinite = 1,
    kStatusDegenerate = 2,
    kStatusBadWeight = 4,   // a per-sample error that is not finite and > 0
    kStatusPhaseRange = 8,  // |t - t_min| f_0 or |t - t_min| df reaches 2^52 turns
};

// Per-curve statistics written by prep_stats (Sec. 3 normalization, FP64).
struct CurveStats {
    double mean;     // mean of X (weighted with 1/dy^2 when errors are given)
    double inv_sd;   // 1/sqrt(population variance); NaN when degenerate
    double t_ref;    // earliest sample time (phase origin)
    double pad;      // the variance; with errors, the weight sum sum 1/dy^2
};

// Phase records of one sample, 32 bytes, consumed by the main kernels.
//   A = {u_lo, u_hi, v_lo, v_hi}: u = frac(t' df), v = frac(t' f0) + offsets,
//       both as 64-bit fixed-point turns (t' = t - t_ref).
//   B = {x_hat, cos 2 pi u, sin 2 pi u, 2 cos 2 pi u}; the last one is the factor
//       of the three-term recurrence, stored so the strips need not form it.
// The offsets folded into v: 2^63 (half a turn, so that the bit-trick angle
// below lands on the true phase), 2^31 (round the top word) and 2^40 (round
// the 23-bit mantissa taken from the top word).
constexpr uint64_t kPhaseOffset = (1ull << 63) + (1ull << 40) + (1ull << 31);

// Per-slice partial statistics when several CTAs share one curve.
struct StatPart {
    double n, mean, m2, tmin;
    int bad, pad;
};

// At most this many CTAs compute the statistics of one curve.
constexpr int kMaxStatSlices = 128;

// CTAs per curve that launch_prep_stats will use (parts needs n_curves * that
// entries; counters needs n_curves zero-initialized words, left zero after use).
int prep_stats_slices(int n_curves, int64_t n0);

// Kernel launchers (all asynchronous on `st`).
// Curves are given in CSR form: samples of curve c are [off[c], off[c+1]).
// When off == nullptr there is one curve of n0 samples.
// dy (optional, floating-mean periodogram): per-sample errors, weights 1/dy^2.
cudaError_t launch_prep_stats(const double* t, const double* X, const int64_t* off, int64_t n0,
                              int n_curves, CurveStats* stats, int* status, StatPart* parts,
                              unsigned* counters, cudaStream_t st, const double* dy = nullptr);

// X may be null (noise batches): then only t_ref is computed and x_hat = 0.
// xout, if given, receives x_hat as a plain FP32 array (batch layout).
// qout (floating-mean periodogram, stats from launch_prep_stats with the same
// dy, or none for equal weights) receives q_j = sqrt(w_j), sum w = 1, and x_hat
// becomes q_j (X_j - mean_w) / sd_w.
// The fixed-point phases need |t_j - t_ref| f_0 and |t_j - t_ref| df below
// 2^52 turns; a sample beyond that gets x_hat = NaN (so the classic
// periodogram of its curve is NaN) and sets kStatusPhaseRange in *status
// when status is given.
cudaError_t launch_prep_records(const double* t, const double* X, const int64_t* off, int64_t n0,
                                int n_curves, int64_t max_n, const double* f0, const double* df,
                                double f0_single, double df_single, const CurveStats* stats,
                                uint4* recA, float4* recB, float2* recN, float* xout, cudaStream_t st,
                                const double* dy = nullptr, float* qout = nullptr, int* status = nullptr);

// Kernel modes (how sin/cos and the phase are formed in the O(N_t N_f) loop).
// kModeRecur3x2 is RECUR3 with the (cos, sin) pair carried through packed
// FP32x2 FMA (FFMA2); its results are bit-identical to kModeRecur3.
enum : int { kModeMufu = 1, kModeRecur = 2, kModeNaive = 3, kModeRecur3 = 4, kModeRecur3x2 = 5 };

struct MainShape {
    int mode;      // kMode*
    int F;         // adjacent frequencies per thread
    int split;     // N_t chunks per frequency block
    int64_t chunk; // samples per chunk
    int nfb;       // frequency blocks
    int64_t nf_pad;// padded row length of the partial-sum workspace
};

// CTA shape of the classic strip kernels (single curve, batch, multi-
// realization, spectral window): one warp per CTA, tiles of 128 samples.  With
// several warps per CTA the warps of one CTA run on different SM
// sub-partitions, drift apart between tile barriers and wait for each other;
// one-warp CTAs (16 resident per SM at 121 registers a thread) measured 1.3%
// faster on the 100k x 200k periodogram and 3% on the 4096-curve batch.
constexpr int kMainThreads = 32;
constexpr int kTile = 128;
// The floating-mean (six-sum) kernels keep four-warp CTAs and 256-sample
// tiles, which measured 4.5% faster for them than one-warp CTAs.
constexpr int kGlsThreads = 128;
constexpr int kGlsTile = 256;
// CTA shape of the persistent floating-mean batch kernel.
constexpr int kGlsBatchThreads = 32;
constexpr int kGlsBatchTile = 128;
// Fewest samples per N_t chunk that the launch-shape heuristic makes.  A
// problem too small to fill one wave of CTAs is latency-bound: each thread's
// serial loop over its chunk is the critical path, so such problems are split
// down to chunks of this many samples.
constexpr int kMinChunk = 64;
// Most samples per N_t chunk that the launch-shape heuristic makes.  Each
// thread's FP32 running sums cover one chunk (the paper's chunked summation,
// Sec. 4.2, at a coarser grain) and the chunks are merged with compensated
// sums, so the rounding error of a sum stays near that of 16,384 terms
// however large N_t grows (on the 382,003 x 1,528,064 paper shape, chunks of
// 16k instead of 64k samples took the largest |dP| from 9e-6 to 1e-6 of max P,
// at no cost in time).
constexpr int64_t kMaxChunk = int64_t(1) << 14;

// Frequencies covered by one CTA of the main kernel (of a floating-mean kernel).
inline int freqs_per_block(int F) { return kMainThreads * F; }
inline int gls_freqs_per_block(int F) { return kGlsThreads * F; }
inline int gls_batch_freqs_per_block(int F) { return kGlsBatchThreads * F; }

// Resident CTAs per SM of the main kernel for (mode, F).
int main_occupancy(int mode, int F);

cudaError_t launch_main(const MainShape& s, const uint4* recA, const float4* recB, const float2* recN,
                        int64_t N, int64_t N_f, double f0, double df, float* part, float* P_out,
                        cudaStream_t st);

cudaError_t launch_finalize(const MainShape& s, const float* part, int64_t N, int64_t N_f,
                            float* P_out, cudaStream_t st);

// ---- floating-mean periodogram (gls.cu) ----

// Six partial-sum rows per chunk (XC, XS, C, S, CC', CS'); q holds sqrt(w_j).
// Strip lengths 8, 12 and 16; modes MUFU, RECUR, RECUR3 and RECUR3 x2 (packed).
constexpr int kGlsRows = 6;
int gls_occupancy(int mode, int F);
cudaError_t launch_gls(const MainShape& s, const uint4* recA, const float4* recB, const float* q, int64_t N,
                       int64_t N_f, float* part, float* P_out, cudaStream_t st);
cudaError_t launch_gls_finalize(const MainShape& s, const float* part, int64_t N, int64_t N_f, float* P_out,
                                cudaStream_t st);
struct BatchItem;
// Many curves (CSR samples, per-curve grids) in one persistent launch; F in {8, 16}.
// packed: the form held to 16 CTAs per SM (built for F = 16, RECUR3 x2), for
// batches whose work is many times their longest curve's.
// xr (noise realizations, RECUR3 x2 only): item (curve c, realization r) takes
// x from xr[r total + j] instead of the records, and writes P at
// P_out[r P_total + P_off[c] + k] and its maximum at maxkey[r n_curves + c];
// without xr every item is realization 0.
int gls_batch_occupancy(int mode, int F, bool packed = false, bool xrow = false);
cudaError_t launch_gls_batch(int mode, int F, bool packed, int grid, const BatchItem* items, int n_items,
                             unsigned* head, const int64_t* off, const int64_t* nf, const uint4* recA,
                             const float4* recB, const float* q, float* P_out, const int64_t* P_off,
                             unsigned long long* maxkey, cudaStream_t st, const float* xr = nullptr,
                             int64_t total = 0, int64_t P_total = 0, int n_curves = 0);
// Realization groups of the floating-mean Monte Carlo (RECUR3 x2): items are
// (curve, up to R realizations from w.real, frequency block) with w.pad the
// group's size; the group shares the phase, the recurrence and the pattern
// sums.  (F, R) in {(8, 4), (4, 8), (8, 2)}.  Outputs as launch_gls_batch with xr.
int gls_mrhs_occupancy(int F, int R);
cudaError_t launch_gls_mrhs(int F, int R, int grid, const BatchItem* items, int n_items, unsigned* head,
                            const int64_t* off, const int64_t* nf, const uint4* recA, const float4* recB,
                            const float* q, float* P_out, const int64_t* P_off, unsigned long long* maxkey,
                            const float* xr, int64_t total, int64_t P_total, int n_curves, cudaStream_t st);
// Noise for the floating-mean Monte Carlo: realization r of curve c is
// X_j = dy_j z_j (z_j the N(0,1) value of lsp_batch's generator for (seed, c,
// r, j); X = z without dy), normalized as prep_records does for measured
// curves: x_j = q_j (X_j - mean_w) / sd_w with the weights 1/dy^2 (FP64 mean
// and population variance), q_j = sqrt(w_j) as launch_prep_records wrote it.
// Row r of xr (stride `total`) receives x.
cudaError_t launch_gls_noise_prep(const int64_t* off, int n_curves, int n_real, uint64_t seed, int64_t total,
                                  const double* dy, const float* q, float* xr, cudaStream_t st);

// ---- Press-Rybicki fast approximation (press_rybicki.cu) ----

// FFT grid size: the smallest power of two >= 2 macc (k_hi + 1).
int64_t pr_fft_size(int64_t k_hi, int macc);
// Extirpolation onto n_fft nodes (acc: FP64 grid, zeroed here), FFT (z0/z1
// ping-pong), P at bins j0 .. j0+N_f-1 into P_out.  *launches: kernels run.
cudaError_t launch_pr(const double* t, const double* X, int64_t N, const CurveStats* stats, double df, int64_t j0,
                      int64_t N_f, int macc, int64_t n_fft, double2* acc, float2* z0, float2* z1, float* P_out,
                      int* launches, cudaStream_t st);

// ---- batched evaluation (batch.cu) and noise (noise.cu) ----

// One work item of the persistent batch kernel: a block of kMainThreads*F
// frequencies of one realization of one curve.
struct BatchItem {
    int32_t curve;
    int32_t real;    // realization (first of the group for multi-RHS items)
    int32_t fblock;
    int32_t pad;     // multi-RHS items: realizations in the group; single-realization
                     // items: a negative value marks a tail item, sub-block -1 - pad of
                     // kMainThreads*tailF frequencies after fblock full blocks
};

// Default strip length of the single-realization batch kernel's tail items:
// the frequencies after a curve's last full block of kMainThreads*F run in
// blocks of kMainThreads*kBatchTailF.  batch_default_tail(F) is it for F > 8,
// else 0 (no tail items).
constexpr int kBatchTailF = 8;
int batch_default_tail(int F);

// tailF, tile: tail-strip length (0: none) and samples per shared-memory tile
// of the kernel; batch_occupancy is 0 when that shape is not built (the
// defaults, batch_default_tail(F) and kTile, are built for every mode and F).
int batch_occupancy(int mode, int F, bool x_in_records, int tailF, int tile);

// x_in_records: every item's x is the x field of recB (one realization);
// otherwise realization r reads xr[r][*].
cudaError_t launch_batch(int mode, int F, bool x_in_records, int tailF, int tile, int grid, const BatchItem* items,
                         int n_items, unsigned* head, const int64_t* off, const int64_t* nf, int64_t total,
                         int n_curves, const uint4* recA, const float4* recB, const float* xr, float* P_out,
                         const int64_t* P_off, int64_t P_total, unsigned long long* maxkey, cudaStream_t st);

// Multi-RHS batch: items carry a group of up to R realizations (real = first,
// pad = count) sharing phases, recurrence and CC/CS; shapes (F, R) in
// {(8, 4), (12, 4), (8, 2), (16, 2), (4, 8), (8, 8)} with tiles of kTile, and for the
// three-term recurrence (12, 4) and (8, 4) also with tiles of 256 and 512.
// With win non-null the kernel takes CC and CS of curve c's frequency k from
// win[woff[c] + k] (written by launch_window with the same mode and F) instead
// of accumulating them.
int mrhs_occupancy(int mode, int F, int R, int tile, bool win);
cudaError_t launch_mrhs(int mode, int F, int R, int tile, int grid, const BatchItem* items, int n_items,
                        unsigned* head, const int64_t* off, const int64_t* nf, int64_t total, int n_curves,
                        const uint4* recA, const float4* recB, const float* xr, float* P_out, const int64_t* P_off,
                        int64_t P_total, unsigned long long* maxkey, const float2* win, const int64_t* woff,
                        cudaStream_t st);

// Window pass of a multi-realization batch: items (curve, block of
// kMainThreads * F frequencies) from a zeroed ticket counter `head`; writes
// (CC, CS) of every frequency k < N_f[c] to win[woff[c] + k].  F in {4, 8, 12, 16}.
int window_occupancy(int mode, int F);
cudaError_t launch_window(int mode, int F, int grid, const BatchItem* items, int n_items, unsigned* head,
                          const int64_t* off, const int64_t* nf, const int64_t* woff, const uint4* recA,
                          const float4* recB, float2* win, cudaStream_t st);

cudaError_t launch_unpack_max(const unsigned long long* maxkey, int64_t n, float* maxP, int32_t* argmax,
                              cudaStream_t st);

// Raw N(0,1) values of (seed, curve, realization), samples 0..n-1.
cudaError_t launch_noise_raw(uint64_t seed, uint32_t curve, uint32_t real, int64_t n, float* out, cudaStream_t st);

// Normalized noise for every (curve, realization) into xr[real][total] and,
// with a single realization, also into the x field of the sample records
// recB; the seed is read from device memory so a captured graph can be
// replayed with a new seed.
cudaError_t launch_noise_prep(const int64_t* off, int n_curves, int n_real, const uint64_t* seed_dev,
                              int64_t total, float* xr, float4* recB, cudaStream_t st);

// ---- false-alarm surrogate (features.cu, mlp.cu) ----

// Spectral window of each pattern on its own window grid (persistent items).
cudaError_t launch_window(int F, int grid, const BatchItem* items, int n_items, unsigned* head, const int64_t* off,
                          const int64_t* nw, const uint4* recA, const float4* recB, float* W, const int64_t* W_off,
                          cudaStream_t st);
int window_occupancy(int F);
// Dynamic shared memory of the features kernel for patterns of up to max_n samples.
size_t features_smem_bytes(int64_t max_n);
cudaError_t launch_features(int n_patterns, int64_t max_n, const double* t, const int64_t* off, const double* f0,
                            const double* df, const int64_t* nf, const float* W, const int64_t* W_off,
                            const int64_t* nw, float* feat, int* status, cudaStream_t st);

int64_t mlp_param_count(int H);
cudaError_t mlp_init(int H, uint64_t seed, float* params, cudaStream_t st);
cudaError_t mlp_feature_stats(int n, const float* feat, float* mu, float* sig, cudaStream_t st);
cudaError_t mlp_gather(int Bn, const int32_t* rows, int n_pat, const float* feat, const float* counts, const float* y,
                       const float* mu, const float* sig, float* X, float* cnt, float* yy, cudaStream_t st);
size_t mlp_workspace_floats(int H, int Bn);
size_t mlp_act_bytes(int H, int Bn, bool fp32);
cudaError_t mlp_forward_backward(int H, int Bn, bool fp32, const float* params, const float* X, const float* cnt,
                                 const float* y, float* q, float* grad, float* loss, float* ws, void* act,
                                 cudaStream_t st);
// Adam (Kingma & Ba 2015) with bias corrections c1, c2 and decoupled weight
// decay wd (p -= lr wd p; 0 = plain Adam).
cudaError_t mlp_adam(int64_t n, float* p, const float* g, float* m, float* v, float lr, float b1, float b2, float c1,
                     float c2, float eps, float wd, cudaStream_t st);

// ---- the training loop's device helpers (train.cu) ----
// Minibatch rows of `step`, uniform over [0, n_rows), from a Philox stream.
cudaError_t train_draw_rows(uint64_t seed, uint32_t step, int B, uint32_t n_rows, int32_t* rows, cudaStream_t st);
// *out = mean pinball loss of q[n_pat][9] against y[n_real][n_pat] (fixed order).
cudaError_t train_pinball(const float* q, const float* y, int n_pat, int n_real, float* out, cudaStream_t st);
// acc = {sum, count} of the minibatch losses since the last validation pass.
cudaError_t train_accum_loss(const float* loss, float* acc, cudaStream_t st);
// Validation pass e after `step` steps: histories, and best = params when
// *val beats state[0] = best loss (state[1] = its step).
cudaError_t train_keep_best(const float* val, float* state, int step, int* flag, float* acc, float* val_hist,
                            float* train_hist, int e, const float* params, float* best, int64_t n, cudaStream_t st);

}  // namespace lsp
