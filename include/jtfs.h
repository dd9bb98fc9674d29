/*
 * jtfs.h -- C ABI of libjtfs: joint time-frequency scattering (JTFS) forward and backward
 * on one NVIDIA GB300 (sm_103a).
 *
 * The operation is the transform of "Differentiable time-frequency scattering on GPU"
 * (Muradeli et al., DAFx 2022):
 *   Sec. 2     first-order scalogram X(t, lambda) = |x * psi_lambda|(t), analytic Morlet filters;
 *              S0 = x * phi_T and S1 = X * phi_T, subsampled every T samples (no frequential
 *              averaging on S1, Sec. 4.2).
 *   Eq. 1      psi_alpha(t) = 2^alpha psi(2^alpha t); psi_{beta,theta}(lambda) = 2^beta psi(theta 2^beta lambda).
 *   Eq. 2      joint wavelet Psi_{alpha,beta,theta}(t, lambda) = psi_alpha(t) psi_{beta,theta}(lambda).
 *   Eq. 3      S2 = (|X *_{t,lambda} Psi| *_{t,lambda} Phi_{T,F}), sampled every (T, 2^floor(log2 F)).
 *   Eq. 4      the same with time-only averaging (average_fr = 0).
 *   Sec. 5     the gradient with respect to x by reverse-ordered adjoints.
 * The discretisation (filterbank rule, critical-subsampling schedule) is documented in the
 * repository's design notes; the library and its FP64 test oracle implement the same rules
 * independently.
 *
 * Conventions for every call:
 *   - Device pointers point to memory of the plan's device; "host" pointers to host memory.
 *   - Buffers are owned by the caller; the plan owns only its filter tables.
 *   - Calls are asynchronous on the given stream (a cudaStream_t passed as void*; NULL is
 *     the legacy default stream).  They validate their arguments on the host and return
 *     a status; nothing throws across the ABI.  Kernel faults surface as JTFS_ERR_CUDA from
 *     the call that observes them (or from jtfs_sync_status).
 *   - jtfs_last_error() returns a per-thread message describing the last non-OK status.
 *   - All float buffers are contiguous, C order, float32.
 */
#ifndef JTFS_H
#define JTFS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  JTFS_OK = 0,
  JTFS_ERR_INVALID_ARG = 1,   /* null pointer, bad size, bad configuration value */
  JTFS_ERR_UNSUPPORTED = 2,   /* valid configuration outside what the kernels handle */
  JTFS_ERR_WORKSPACE = 3,     /* workspace missing or smaller than jtfs_workspace_bytes */
  JTFS_ERR_CUDA = 4,          /* a CUDA runtime call or kernel failed */
  JTFS_ERR_TIMEOUT = 5,       /* a bounded device wait gave up */
  JTFS_ERR_NUMERIC = 6        /* non-finite values where finite ones are required */
} jtfs_status;

/* Arithmetic of the log-frequency contraction (the dense lambda-contraction of Eq. 2-3).
 * Every other step (FFTs, filter products, modulus, pooling) is FP32 on CUDA cores. */
typedef enum {
  JTFS_PREC_FP32 = 0,       /* tensor cores, bf16 hi/lo split in three passes, FP32 accumulate */
  JTFS_PREC_TF32 = 1,       /* tensor cores, one TF32 pass, FP32 accumulate */
  JTFS_PREC_BF16 = 2,       /* tensor cores, one BF16 pass, FP32 accumulate */
  JTFS_PREC_FP32_SIMT = 3   /* CUDA cores, plain FP32 (the comparison form) */
} jtfs_precision;

/* Second-order joint wavelets (Eq. 2-3 with the time wavelet psi_t or the log-frequency
 * wavelet psi_f replaced by its lowpass phi_T or phi_F).  The psi_t paths (PSI_PSI, PSI_PHI)
 * are always computed; PHI_PSI and PHI_PHI add the phi_t paths. */
typedef enum {
  JTFS_BRANCH_PSI_PSI = 1,   /* psi_alpha(t) psi_{beta,theta}(lambda), both spins */
  JTFS_BRANCH_PSI_PHI = 2,   /* psi_alpha(t) phi_F(lambda) */
  JTFS_BRANCH_PHI_PSI = 4,   /* phi_T(t) psi_{beta,+1}(lambda): one spin, the input X * phi_T
                                being real makes the other spin's modulus the same */
  JTFS_BRANCH_PHI_PHI = 8    /* phi_T(t) phi_F(lambda) */
} jtfs_branch;

/* Sec. 4.2 parameters.  T and F must be >= 1; T a power of two <= N.  Q2 is the number of
 * second-order time wavelets per octave (1 in the paper).  oversampling o >= 0 divides every
 * subsampling stride by 2^o. */
typedef struct {
  int32_t J, Q, Q2, J_fr, Q_fr;
  int64_t T, F;
  int32_t average_fr;    /* 1: Eq. 3 (phi_F pooling, lambda stride 2^floor(log2 F)); 0: Eq. 4 */
  int32_t oversampling;
  int32_t precision;     /* jtfs_precision */
  int32_t out_3d;        /* 1: S0, S1 and S2 in their own buffers (S1 2-D, S2 3-D per path);
                            0: one 2-D buffer per signal, [paths][n_t] with S0, S1 and S2
                            concatenated along the path axis (Sec. 4.2's two output modes) */
  int32_t branches;      /* bit mask of jtfs_branch; 0 means PSI_PSI | PSI_PHI.  The phi_t
                            paths need oversampling 0 (their input is then S1 itself) */
  int32_t reserved[3];   /* must be 0 */
} jtfs_config;

/* Output sizes.  S0 [B, n_t]; S1 [B, n1, n_t]; S2 [B, s2_paths, n_lam_out, n_t].  The S2 paths
 * are first the psi_t paths, [n2][C] with channel c < n_fr = (beta = c, theta = +1),
 * n_fr <= c < 2 n_fr = (beta = c - n_fr, theta = -1), c = 2 n_fr = the psi_t x phi_F branch;
 * then the n_phi phi_t paths: phi_T x psi_{beta,+1} for beta < n_fr (PHI_PSI) and phi_T x
 * phi_F (PHI_PHI).  lambda increases with frequency (theta = -1 is an upward slope, Sec. 2).
 * With out_3d = 0 the single output holds, per signal, out_rows = 1 + n1 + s2_paths * n_lam_out
 * rows of n_t frames: S0, the n1 rows of S1, then S2 path by path.  u1_len is the checkpointed
 * scalogram's length per signal (rows packed at their own strides). */
typedef struct {
  int64_t N, n1, n2, n_fr, C, n_t, n_lam_out, N_fr, s_F;
  int64_t s0_len, s1_len, s2_len, u1_len;
  int64_t n_phi, s2_paths, out_rows;
} jtfs_shapes;

typedef struct jtfs_plan jtfs_plan;

/* Builds the filterbanks (FP64 on the current CUDA device, Sec. 2 / Eq. 1 with the
 * Littlewood-Paley normalisation) and the subsampling schedule for signals of length N
 * (a power of two).  Synchronous.  On success *out owns device memory until
 * jtfs_plan_destroy.  Errors: INVALID_ARG (bad values), UNSUPPORTED (e.g. a row longer
 * than the shared-memory FFT), CUDA. */
jtfs_status jtfs_plan_create(const jtfs_config* cfg, int64_t N, jtfs_plan** out);
void jtfs_plan_destroy(jtfs_plan* plan);

jtfs_status jtfs_plan_shapes(const jtfs_plan* plan, jtfs_shapes* out);

/* The schedule, for inspection: s1[n1] first-order strides, s2[n2] second-order strides
 * (0 for a skipped rate), lam_min[n2] first row used by each rate.  Host arrays. */
jtfs_status jtfs_plan_schedule(const jtfs_plan* plan, int32_t* s1, int32_t* s2,
                               int32_t* lam_min);

/* Device workspace bytes for a batch of B signals; with_grad != 0 also covers
 * jtfs_backward. */
jtfs_status jtfs_workspace_bytes(const jtfs_plan* plan, int64_t B, int32_t with_grad,
                                 size_t* out);

/* Forward transform (Sec. 2; Eq. 3, or Eq. 4 with average_fr = 0): S0 = x * phi_T and
 * S1 = |x * psi_lambda| * phi_T sampled every T, and S2 of Eq. 3 for every second-order path.
 * x [B, N] (device).  Writes s0, s1, s2 (device, sizes from
 * jtfs_plan_shapes).  With out_3d = 0, s0 receives the single [B, out_rows, n_t] output and
 * s1, s2 must be NULL.  u1_ckpt (device, [B, u1_len]) receives the first-order scalogram
 * checkpoint when not NULL; jtfs_backward needs it.  B = 0 is a no-op. */
jtfs_status jtfs_forward(const jtfs_plan* plan, const float* x, int64_t B, float* s0, float* s1,
                         float* s2, float* u1_ckpt, void* ws, size_t ws_bytes, void* stream);

/* Backward (Sec. 5: the reverse-ordered adjoints of the forward's operators):
 * g_x [B, N] = d<g, S(x)>/dx for cotangents g_s0, g_s1, g_s2 (device, same shapes
 * as the outputs; any may be NULL for zero; with out_3d = 0, g_s0 holds the single output's
 * cotangent and g_s1, g_s2 must be NULL).  Needs the forward's u1_ckpt for the same x.
 * The modulus Jacobian d|z| = Re(conj(z) dz) / |z| is taken as 0 at z = 0. */
jtfs_status jtfs_backward(const jtfs_plan* plan, const float* x, const float* u1_ckpt,
                          int64_t B, const float* g_s0, const float* g_s1, const float* g_s2,
                          float* g_x, void* ws, size_t ws_bytes, void* stream);

/* Forward and backward in one call (Sec. 2 and Sec. 5): s0, s1, s2 as jtfs_forward and
 * g_x as jtfs_backward, for x and the cotangents on the device.  Between the two halves the
 * workspace keeps x-hat, the first-order spectra and the BF16 second-order planes, which the
 * separate calls recompute from the checkpoint; the results match jtfs_forward followed by
 * jtfs_backward up to rounding order.  u1_ckpt (device, may be NULL) receives the checkpoint.
 * ws as for with_grad = 1.  Errors as jtfs_forward / jtfs_backward. */
jtfs_status jtfs_forward_backward(const jtfs_plan* plan, const float* x, int64_t B,
                                  const float* g_s0, const float* g_s1, const float* g_s2,
                                  float* s0, float* s1, float* s2, float* u1_ckpt, float* g_x,
                                  void* ws, size_t ws_bytes, void* stream);

/* Time scattering (Scattering1D), the baseline of Sec. 4.4, on the plan's filterbanks and
 * schedule: the first-order scalogram with no log-frequency stage after it.  s0 and s1 as
 * jtfs_forward; s2t [B, n2, n1, n_t] (device) with
 *   s2t[alpha][lambda'][t] = (|U1[lambda'] * psi_alpha| * phi_T)(t T)
 * on the paths (alpha, lambda') of a kept rate with lambda' >= lam_min[alpha]
 * (jtfs_plan_schedule) and 0 elsewhere.  Runs on CUDA cores in FP32 for every precision;
 * out_3d and branches do not apply.  u1_ckpt (device, may be NULL) receives the checkpoint.
 * ws as jtfs_workspace_bytes(with_grad = 0).  Errors as jtfs_forward. */
jtfs_status jtfs_scattering1d_forward(const jtfs_plan* plan, const float* x, int64_t B,
                                      float* s0, float* s1, float* s2t, float* u1_ckpt,
                                      void* ws, size_t ws_bytes, void* stream);

/* Its gradient (Sec. 5 adjoints): g_x [B, N] for cotangents g_s0, g_s1, g_s2t (device, any may
 * be NULL for zero), given x and the forward's u1_ckpt.  ws as jtfs_workspace_bytes(with_grad
 * = 1). */
jtfs_status jtfs_scattering1d_backward(const jtfs_plan* plan, const float* x,
                                       const float* u1_ckpt, int64_t B, const float* g_s0,
                                       const float* g_s1, const float* g_s2t, float* g_x,
                                       void* ws, size_t ws_bytes, void* stream);

/* End-to-end forward + backward from HOST buffers: copies x (host, [B, N]) and the
 * cotangents (host; NULL = zero) to the device, runs jtfs_forward_backward, and
 * copies s0, s1, s2 (host, may be NULL) and g_x (host) back.  dev_buf must hold
 * jtfs_host_step_bytes(plan, B) bytes of device memory; ws as for with_grad = 1.
 * Synchronous on return. */
jtfs_status jtfs_host_step_bytes(const jtfs_plan* plan, int64_t B, size_t* out);
jtfs_status jtfs_forward_backward_host(const jtfs_plan* plan, const float* x_host, int64_t B,
                                       const float* g_s0_host, const float* g_s1_host,
                                       const float* g_s2_host, float* s0_host, float* s1_host,
                                       float* s2_host, float* g_x_host, void* dev_buf,
                                       size_t dev_buf_bytes, void* ws, size_t ws_bytes,
                                       void* stream);

/* Autotuner of the launch shape of the largest FFT stage (the second-order time wavelets):
 * times every candidate (256 or 512 threads per CTA; 4096, 8192 or 16384 samples per CTA) on
 * the plan's work for B signals on `stream` and keeps the fastest in the plan; the results of
 * later calls do not change (the same arithmetic per row).  ws as for jtfs_forward.  choice
 * (host, 3 entries, may be NULL) receives threads, samples per CTA and the winner's time per
 * launch in microseconds.  Synchronous.  Not thread-safe against concurrent calls on the plan.
 * The paper has no counterpart. */
jtfs_status jtfs_plan_autotune(jtfs_plan* plan, int64_t B, void* ws, size_t ws_bytes, void* stream,
                               int32_t* choice);

/* Tracing: when enabled, forward/backward record a CUDA event pair around each stage on
 * the launching stream.  jtfs_profile_read waits for the recorded events, writes the
 * milliseconds accumulated per stage into ms[0..n_ms) (stage i is named by
 * jtfs_profile_stage_name(i), NULL past the last stage), writes the number of kernels
 * launched since the previous read (counted whether or not tracing is on), and resets both. */
jtfs_status jtfs_profile_enable(const jtfs_plan* plan, int32_t on);
jtfs_status jtfs_profile_read(const jtfs_plan* plan, double* ms, int32_t n_ms, int64_t* launches);
const char* jtfs_profile_stage_name(int32_t i);

/* First-order coefficients only (S0 [B, n_t] and S1 [B, n1, n_t], device buffers, same values
 * as jtfs_forward) computed without allocating any device memory.  The paper has no
 * counterpart; this entry point serves callers that cannot allocate while they run, such as
 * a real-time audio callback (an allocation may block for milliseconds and miss the audio
 * deadline) or a plug-in inside a host application that owns all device memory.  Its scratch
 * is a fixed 16 MiB array compiled into the library, which every GPU that loads the library
 * keeps until the process exits; a batch whose scratch would exceed it is rejected with
 * JTFS_ERR_WORKSPACE (about 2.6 MB per signal at N = 2^16, J = 12, Q = 16).  The first call on
 * a device looks up the array's device address; make that first call before any stream
 * capture.  All calls share the array: calls that overlap on the GPU race on it. */
jtfs_status jtfs_first_order_static(const jtfs_plan* plan, const float* x, int64_t B, float* s0,
                                    float* s1, void* stream);

/* ---------------------------------------------------------------------------------------
 * mu-log compression (Sec. 4.3, Eq. 6-7) of scattering paths, on any device array S
 * [B, P, M] of B examples, P paths (lambda_2) and M coefficients per path (for the transform's
 * S2: P = s2_paths, M = n_lam_out n_t; for time scattering's S2t: P = n2 n1, M = n_t).
 * Asynchronous on `stream`; INVALID_ARG for NULL pointers or non-positive sizes. */

/* Eq. 6: mu [P] (device) = (1 / B) sum over the B examples of each path's sum over its M
 * coefficients (the integral over lambda and t on the grid).  FP64 sums in a fixed order. */
jtfs_status jtfs_mulog_mean(const float* s, int64_t B, int64_t P, int64_t M, float* mu,
                            void* stream);

/* Eq. 7: out = log(1 + S / (eps mu[p])), eps > 0 (0.1 in the paper).  out may alias s. */
jtfs_status jtfs_mulog(const float* s, int64_t B, int64_t P, int64_t M, const float* mu,
                       float eps, float* out, void* stream);

/* Its gradient with mu held fixed: g_s = g_out / (eps mu[p] + S). */
jtfs_status jtfs_mulog_backward(const float* s, int64_t B, int64_t P, int64_t M,
                                const float* mu, float eps, const float* g_out, float* g_s,
                                void* stream);

/* ---------------------------------------------------------------------------------------
 * Uneven-length batches.  The paper transforms one signal length at a time; these calls take
 * B signals of lengths len[i] packed back to back (x_packed[x_off[i] .. x_off[i] + len[i])).
 * Signal i is zero-padded to N_i = jtfs_varlen_padded_length(cfg, len[i]) =
 * max(2^ceil(log2 len[i]), 2^(J+3)) and transformed with the plan of length N_i (built by
 * jtfs_varlen_create, periodic in time on N_i like every fixed-length transform); its outputs
 * keep the first frames_i = ceil(len[i] / T) frames:
 *   S0 packed [s0_off[i] ..) as [frames_i], S1 as [n1(N_i), frames_i],
 *   S2 as [n2(N_i), C, n_lam_out, frames_i]  (n1, n2, C, n_lam_out of the plan of N_i).
 * Cotangents use the same packed layouts; g_x the layout of x (first len[i] samples). */
typedef struct jtfs_varlen jtfs_varlen;

/* N_i for one length (0 for an invalid argument).  Host only. */
int64_t jtfs_varlen_padded_length(const jtfs_config* cfg, int64_t len);

/* Groups the signals by N_i, builds one plan per distinct N_i (synchronous, current device)
 * and splits each group into sub-batches of at most `chunk` signals (0: 64).  len is a host
 * array of B lengths in [1, 2^24].  Errors as jtfs_plan_create, INVALID_ARG. */
jtfs_status jtfs_varlen_create(const jtfs_config* cfg, const int64_t* len, int64_t B,
                               int32_t chunk, jtfs_varlen** out);
void jtfs_varlen_destroy(jtfs_varlen* v);

/* Packed offsets (host arrays of B + 1 entries; any may be NULL): x / g_x, S0, S1, S2.  The
 * last entry of each is the total length in floats. */
jtfs_status jtfs_varlen_layout(const jtfs_varlen* v, int64_t* x_off, int64_t* s0_off,
                               int64_t* s1_off, int64_t* s2_off);

/* Device workspace for jtfs_varlen_forward_backward / jtfs_varlen_capture (the largest
 * sub-batch's padded buffers plus its plan workspace; sub-batches run one after another). */
jtfs_status jtfs_varlen_workspace_bytes(const jtfs_varlen* v, size_t* out);

/* Forward and backward of every signal (device buffers, packed layouts above; cotangents may
 * be NULL for zero).  Per signal the results equal jtfs_forward / jtfs_backward of its
 * zero-padded copy, restricted to the kept frames and to its first len[i] samples. */
jtfs_status jtfs_varlen_forward_backward(const jtfs_varlen* v, const float* x_packed,
                                         const float* g_s0, const float* g_s1, const float* g_s2,
                                         float* s0, float* s1, float* s2, float* g_x, void* ws,
                                         size_t ws_bytes, void* stream);

/* Runs jtfs_varlen_forward_backward once on `stream` (a non-default stream), then captures it
 * into a CUDA graph owned by v (replacing an earlier one).  The graph keeps these buffer
 * addresses: jtfs_varlen_replay recomputes the step from whatever the buffers then hold. */
jtfs_status jtfs_varlen_capture(jtfs_varlen* v, const float* x_packed, const float* g_s0,
                                const float* g_s1, const float* g_s2, float* s0, float* s1,
                                float* s2, float* g_x, void* ws, size_t ws_bytes, void* stream);
jtfs_status jtfs_varlen_replay(const jtfs_varlen* v, void* stream);

/* jtfs_plan_autotune for every plan of v at its largest sub-batch (ws: the varlen
 * workspace).  Call before jtfs_varlen_capture: a captured graph keeps the launch shapes it
 * was recorded with. */
jtfs_status jtfs_varlen_autotune(jtfs_varlen* v, void* ws, size_t ws_bytes, void* stream);

/* Schedule autotuner of the uneven-length step (the paper has no counterpart): times the whole
 * step (jtfs_varlen_forward_backward on these buffers, which it overwrites) with sub-batches of
 * 16, 32, 64, ... signals up to the `chunk` given at creation (and that size), keeps the
 * fastest split and writes its size to chosen[0] (host, may be NULL).  The results do not
 * depend on the split.  Drops a captured graph (capture again afterwards).  ws as
 * jtfs_varlen_workspace_bytes (sized for the creation's chunk, so every candidate fits).
 * Synchronous. */
jtfs_status jtfs_varlen_tune_schedule(jtfs_varlen* v, const float* x_packed, const float* g_s0,
                                      const float* g_s1, const float* g_s2, float* s0, float* s1,
                                      float* s2, float* g_x, void* ws, size_t ws_bytes,
                                      void* stream, int32_t* chosen);

/* ---------------------------------------------------------------------------------------
 * Failure detection.  The paper has no counterpart; these calls report faults instead of
 * hanging or returning silently wrong numbers.
 *
 * Every wait of the tensor-core contraction kernels on a shared-memory barrier is bounded:
 * after the plan's wait budget of wall time (%globaltimer) the block records a code in the
 * plan's device status word, stops issuing work and returns, so the CUDA context stays usable.
 * With check_finite on, forward / backward / forward_backward scan their outputs for NaN or
 * Inf after the transform and record that in the same word.  The word is read and cleared by
 * jtfs_sync_status. */

/* Waits for the stream, then reports a pending CUDA error (JTFS_ERR_CUDA), a bounded wait that
 * gave up (JTFS_ERR_TIMEOUT) or a non-finite output (JTFS_ERR_NUMERIC) of any earlier call on
 * the plan, and clears the status word.  Synchronous. */
jtfs_status jtfs_sync_status(const jtfs_plan* plan, void* stream);

/* Sets the budget of every bounded device wait of later calls, in nanoseconds, within
 * [1 us, 60 s] (default 2 s; INVALID_ARG outside).  Not thread-safe against calls in flight
 * on other host threads. */
jtfs_status jtfs_plan_set_wait_budget(jtfs_plan* plan, uint64_t wait_ns);

/* on != 0: later forward / backward calls launch one scan per output (B * its length floats)
 * and record JTFS_ERR_NUMERIC for the next jtfs_sync_status if any value is NaN or Inf.
 * Default off. */
jtfs_status jtfs_plan_set_check_finite(jtfs_plan* plan, int32_t on);

/* Exercises the timeout path on the device: launches one block on `stream` that waits, with
 * the contraction kernels' bounded wait and a budget of wait_ns in [1 us, 1 s], on a barrier
 * that nothing ever completes; the wait gives up, the block records its code in the plan's
 * status word and returns.  The next jtfs_sync_status then returns JTFS_ERR_TIMEOUT.
 * Asynchronous; INVALID_ARG for a budget outside the range. */
jtfs_status jtfs_diagnose_wait_timeout(const jtfs_plan* plan, uint64_t wait_ns, void* stream);

const char* jtfs_status_string(jtfs_status s);
const char* jtfs_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* JTFS_H */
