/*
 * dc.h -- C ABI of the GB300 Doppler + ionospheric correction library
 * (libdc.so).  Method: arXiv 2508.04951, "Real-Time Doppler and Ionospheric
 * Distortion Correction Techniques for Arbitrary Waveforms Utilizing GPU
 * Compute".
 *
 * A pulse x[0..N) of complex baseband samples (interleaved float32 re/im, the
 * layout of torch.complex64) taken at rate fs is corrected for a target range
 * rate v_r and a total electron content TEC:
 *
 *   1. Doppler resampling, y[n] = x(alpha n Ts), alpha = (1 + v_r/c)/(1 - v_r/c)
 *      (Eq. 1, Eq. 2; v_r > 0 approaching), by windowed Whittaker-Shannon
 *      interpolation with a Kaiser-windowed sinc (Eq. 17 truncated, Sec. III-B,
 *      Table I) or by the exact finite sum of Eq. 17.
 *   2. Ionospheric correction (Eq. 16): y is zero-padded to L = 2^ceil(log2 n_out),
 *      transformed, multiplied by exp(-i 4 pi K2 / (c f_k)) with K2 = kappa E
 *      (Eq. 3), f_k = fc + fs kt/L (kt in numpy fftfreq order; fc = 0 means
 *      the samples are RF, a bin at f_k = 0 is left unchanged), inverse
 *      transformed with 1/L and truncated to n_out samples.
 *
 * Conventions for every entry point:
 *  - Pointers named *_dev are device pointers on the context's device,
 *    owned by the caller, 8-byte aligned (one complex sample).  Outputs must
 *    not overlap inputs unless an entry point says so.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  All work is
 *    enqueued asynchronously on it; results are ready when the stream is.
 *    Host arrays passed in (item lists, v_r/TEC lists) are read before the
 *    call returns and may be reused afterwards.
 *  - A context serialises its own scratch memory: do not run calls on one
 *    context from several host threads or streams at the same time.
 *  - Arguments are validated before anything is launched; a bad argument
 *    returns DC_EINVAL with a message in dc_last_error() and launches
 *    nothing.  Launch failures return DC_ECUDA.  Faults inside kernels
 *    (bounded waits that ran out) are reported by dc_check(), which
 *    synchronises the stream.
 *  - Limits: 1 <= n, n_out <= 2^20 samples; |v_r| < c; fs > 0; fc == 0 or
 *    fc > fs/2 (every bin frequency positive in baseband); even taps in
 *    [2, 64]; Kaiser beta in [0, 20].
 */
#ifndef DC_H
#define DC_H

#include <stddef.h>

#if defined(__GNUC__)
#define DC_API __attribute__((visibility("default")))
#else
#define DC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* One complex sample: interleaved float32, identical to torch.complex64. */
typedef struct { float re, im; } dc_c64;

typedef enum {
  DC_OK = 0,
  DC_EINVAL = 1,      /* argument rejected before any launch               */
  DC_ENOMEM = 2,      /* device or host allocation failed                   */
  DC_EBUSY = 3,       /* HBM budget or serve slots exhausted (try again)    */
  DC_ECUDA = 4,       /* CUDA runtime error (launch or copy)                */
  DC_ETIMEOUT = 5,    /* a kernel's bounded wait ran out / wait timed out   */
  DC_ECANCELLED = 6   /* request cancelled                                  */
} dc_status;

/* Resampling method (Table I rows "Whittaker-Shannon", "Windowed" and
 * "Frequency Conversion"). */
typedef enum {
  DC_WINDOWED = 0,        /* Kaiser-windowed sinc, `taps` taps, FP32        */
  DC_EXACT_FP32 = 1,      /* exact finite sum of Eq. 17, FP32 CUDA cores    */
  DC_EXACT_BF16X3 = 2,    /* exact sum as a tensor-core GEMM, bf16 hi/lo    */
  DC_EXACT_FP16X3 = 3,    /* exact sum as a tensor-core GEMM, fp16 hi/lo    */
  DC_FREQCONV = 4         /* frequency conversion (Sec. I method list): the
                             dilation approximated by the tone multiply
                             y[n] = x[n] exp(2 pi i f (alpha - 1) n Ts),
                             f = freq_ref (+ fc with carrier_shift), x = 0
                             past n; exact for a tone at f, error growing as
                             B^2 for an LFM of bandwidth B (Table I)         */
} dc_mode;

typedef struct {
  int taps;             /* windowed kernel length, even, default 32          */
  double kaiser_beta;   /* Kaiser shape, default 8                           */
  int mode;             /* dc_mode, default DC_WINDOWED                      */
  long long n_out;      /* output samples, 0 = same as input                 */
  /* 1: the samples are complex baseband about fc and the dilation is that of
   * the passband signal, so the resampled pulse also takes the carrier term
   * exp(2 pi i fc (alpha - 1) n Ts) (Eq. 2 applied to x(t) exp(2 pi i fc t),
   * mixed back down by fc).  0 (default): y[n] = x(alpha n Ts) only.  Not
   * used by resample_exact_batch.                                           */
  int carrier_shift;
  double freq_ref;      /* DC_FREQCONV: frequency (Hz, in the samples' own
                           frame) at which the tone multiply is exact,
                           default 0                                         */
} dc_opts;

typedef struct dc_ctx dc_ctx;

/* Defaults: taps 32, beta 8, DC_WINDOWED, n_out 0, carrier_shift 0, freq_ref 0. */
DC_API void dc_opts_default(dc_opts* opts);

/* Text of a status code (static storage). */
DC_API const char* dc_status_str(int status);

/* Create a context on CUDA device `device`.  It owns the twiddle tables and
 * the scratch memory of later calls; `hbm_budget_bytes` caps that scratch
 * (0 = no cap).  Writes the handle to *ctx.  DC_EINVAL for a bad device,
 * DC_ENOMEM / DC_ECUDA on allocation failure. */
DC_API dc_status dc_create(dc_ctx** ctx, int device, size_t hbm_budget_bytes);

/* Free everything the context owns.  Synchronises the device first. */
DC_API dc_status dc_destroy(dc_ctx* ctx);

/* Message of the last failed call on this context ("" if none). */
DC_API const char* dc_last_error(const dc_ctx* ctx);

/* Synchronise `stream`, then report and clear the context's device-side
 * error flag: DC_ETIMEOUT if a bounded wait inside a kernel ran out,
 * DC_EINVAL if a kernel met parameters outside its range, DC_ECUDA on an
 * asynchronous CUDA error or, in the checked build (libdc compiled with
 * DC_CHECKED: bounds checks in the kernels, a failed one skips its access),
 * on a failed bounds check. */
DC_API dc_status dc_check(dc_ctx* ctx, void* stream);

/* Failure-detection self-test: queues on `stream` one kernel that waits, with
 * the library's bounded poll, on an mbarrier nothing ever completes.  The
 * wait runs out (about 2^16 polls), the context's error flag is raised, and
 * the next dc_check on that stream returns DC_ETIMEOUT; the context stays
 * usable afterwards.  No GPU fault or hang is involved. */
DC_API dc_status dc_selftest_wait_timeout(dc_ctx* ctx, void* stream);

/* Kernels launched by this context since creation (-1 for a null context). */
DC_API long long dc_launch_count(const dc_ctx* ctx);

/* Per-phase kernel timing.  With profiling on, every kernel launch of later
 * calls is bracketed by CUDA events recorded on the call's stream (so the
 * times are device times of exactly that launch).  dc_profile_enable resets
 * the totals (waiting for events still pending).  dc_profile_read waits for
 * pending events, folds them into the totals and writes up to `max` phases
 * (name, launches, samples covered, total ms) to `out`; returns the number
 * of phases with at least one launch, or -1 for a null context. */
typedef struct {
  char name[24];
  long long launches;
  long long samples;
  double ms;
} dc_phase_time;
DC_API dc_status dc_profile_enable(dc_ctx* ctx, int on);
DC_API int dc_profile_read(dc_ctx* ctx, dc_phase_time* out, int max);

/* Doppler resampling alone (Eq. 2 via Eq. 17; Sec. III).
 * x_dev: [n] input samples.  y_dev: [n_out] output, n_out = opts->n_out or n.
 * Windowed: y[j] = sum_i x[i] h(alpha j - i), h the Kaiser-windowed sinc of
 * half width taps/2, x = 0 outside [0, n).  Exact: y[j] = sum_{i<n} x[i]
 * sinc(alpha j - i).  DC_FREQCONV: the tone multiply of dc_mode.  With
 * opts->carrier_shift the interpolating modes also multiply y[j] by
 * exp(2 pi i fc (alpha - 1) j / fs).  fs and fc enter only through the
 * carrier term and frequency conversion (positions are in units of samples).
 * Modes DC_WINDOWED, DC_EXACT_FP32, DC_FREQCONV.  opts may be NULL
 * (defaults). */
DC_API dc_status doppler_resample(dc_ctx* ctx, const dc_c64* x_dev, long long n, dc_c64* y_dev,
                           double fs, double fc, double v_r, const dc_opts* opts,
                           void* stream);

/* Ionospheric correction alone (Eq. 16, Sec. II-B).  x_dev: [n] input,
 * y_dev: [n] output; x_dev == y_dev (in place) is allowed.  tec_tecu is the
 * TEC in units of 1e16 el/m^2; a negative TEC applies the distortion of
 * Eq. 15 instead (the phase is linear in E). */
DC_API dc_status iono_correct(dc_ctx* ctx, const dc_c64* x_dev, long long n, dc_c64* y_dev,
                       double fs, double fc, double tec_tecu, void* stream);

/* Ionospheric correction with no device allocation at run time.
 *
 * The paper has no counterpart to this entry point; it exists for callers
 * that are not allowed to allocate device memory while they run: for example
 * a real-time receive loop with a fixed memory plan, where cudaMalloc could
 * stall the pipeline (it may synchronise the device), or a host application
 * whose device memory is all owned by its own pool allocator.  Such callers
 * cannot create a dc_ctx (which allocates tables and scratch), so this call
 * needs no context at all.
 *
 * Same computation and arguments as iono_correct (x_dev, y_dev: [n], in place
 * allowed), limited to 1 <= n <= 262144 (2^18) samples; a larger n, or any
 * argument iono_correct would reject, returns DC_EINVAL without launching.
 * The four-step scratch (2 MiB), the twiddle tables and the launch
 * descriptors are fixed-size __device__ arrays inside libdc.so: every GPU that
 * loads the library keeps them until the process exits, and this call never
 * calls cudaMalloc or cudaFree.  Runs on the current CUDA device.
 *
 * The first call on a device sets up that device: it resolves the arrays'
 * device addresses (cudaGetSymbolAddress, with the device current) and writes
 * the twiddle tables with a synchronous copy.  Make that first call before
 * any stream capture.  Each call hands its launch descriptors to the GPU as
 * kernel parameters (a one-thread kernel stores them into the descriptor
 * slots), so no host memory is read after the call returns.  All calls share
 * the one scratch array and descriptor slots, which keep the last call's
 * contents (the scratch is fully rewritten before it is read, so nothing
 * needs clearing); calls whose work overlaps on the GPU -- on different
 * streams, say -- race with each other, so issue them on one stream or
 * serialise them.  DC_ECUDA on a CUDA runtime error. */
DC_API dc_status iono_correct_noalloc(const dc_c64* x_dev, long long n, dc_c64* y_dev,
                                      double fs, double fc, double tec_tecu, void* stream);

/* One pulse of a batch.  Offsets and lengths count complex samples. */
typedef struct {
  long long in_off;     /* first input sample in in_dev                      */
  long long n;          /* input samples                                     */
  long long out_off;    /* first output sample in out_dev                    */
  long long n_out;      /* output samples (0 = n)                            */
  double fs, fc, v_r, tec_tecu;
} dc_item;

/* Full correction of a ragged batch: for each item, resample by alpha(v_r)
 * (opts->mode: DC_WINDOWED, DC_EXACT_FP32 or DC_FREQCONV; taps, beta,
 * carrier_shift, freq_ref; opts->n_out is ignored, items carry n_out), then
 * apply Eq. 16 with its TEC.  in_dev and out_dev hold all items at the given
 * offsets; output ranges must not overlap each other or the inputs.  Each
 * item's result does not depend on the other items of the batch. */
DC_API dc_status correct_batch(dc_ctx* ctx, const dc_c64* in_dev, dc_c64* out_dev,
                        const dc_item* items, int n_items, const dc_opts* opts,
                        void* stream);

/* Doppler bank: one pulse corrected for every (v_r, TEC) pair.  With
 * DC_WINDOWED, 32 taps and no carrier term the resampling of all range rates
 * runs as a tensor-core contraction (Sec. III-B's windowed sum over the
 * shared input; see dc_tuning.resample_tc) wherever the range rates, ordered
 * in groups of 32, stay within 30 samples of each other in delay over the
 * pulse (a group spanning the whole of -8 .. +8 km/s qualifies up to about
 * 2.6e5 samples); else on CUDA cores.
 * x_dev: [n]; v_r: host [n_v]; tec_tecu: host [n_tec];
 * out_dev: [n_v][n_tec][n_out] (n_out = opts->n_out or n).  Modes DC_WINDOWED
 *          and DC_FREQCONV.
 *          out_dev is written once and never read, so it may also be
 *          page-locked host memory (cudaHostAlloc / cudaHostRegister): the
 *          inverse-transform kernel then stores the results straight into
 *          it over the host link, overlapping the transfer with the work.
 * Resampling and the forward transform run once per v_r, the phase multiply
 * and inverse transform once per pair. */
DC_API dc_status correct_bank(dc_ctx* ctx, const dc_c64* x_dev, long long n, const double* v_r,
                       int n_v, const double* tec_tecu, int n_tec, dc_c64* out_dev,
                       double fs, double fc, const dc_opts* opts, void* stream);

/* Pulse compression bundled with the correction (Sec. II-B, the paragraph
 * after Eq. 16 and the pulse-compression figure): the frequency-domain pass
 * of Eq. 16 also applies the matched filter of a replica, so that
 *
 *   r = F^-1[ F(y) exp(-i 4 pi K2 / (c f_k)) conj(F(h)) ],  first n_out lags,
 *
 * with y the pulse resampled by alpha(v_r) (as correct_batch: opts->mode
 * DC_WINDOWED, DC_EXACT_FP32 or DC_FREQCONV, carrier_shift, freq_ref;
 * n_out = opts->n_out or n) zero-padded to L = 2^ceil(log2 n_out), and h the
 * replica zero-padded to L.  Lag m is sum_j z[(m + j) mod L] conj(h[j]), z the
 * whole corrected L-buffer: the matched filter's output at delay m, linear
 * for m <= L - n_rep, circular beyond.
 * x_dev: [n]; replica_dev: [n_rep], 1 <= n_rep <= L; y_dev: [n_out] lags.
 * The replica's spectrum is computed on the device in the same call. */
DC_API dc_status correct_compress(dc_ctx* ctx, const dc_c64* x_dev, long long n,
                                  const dc_c64* replica_dev, long long n_rep, dc_c64* y_dev,
                                  double fs, double fc, double v_r, double tec_tecu,
                                  const dc_opts* opts, void* stream);

/* The Doppler bank (correct_bank) compressed against one replica: out_dev
 * [n_v][n_tec][n_out] holds, per (v_r, TEC) pair, the lags of
 * correct_compress.  The replica's spectrum is computed once and its
 * conjugate folded into each TEC's factor table, so the per-pair
 * phase-and-inverse pass costs what it costs without compression.  Modes
 * DC_WINDOWED and DC_FREQCONV; out_dev may be page-locked host memory as for
 * correct_bank. */
DC_API dc_status correct_compress_bank(dc_ctx* ctx, const dc_c64* x_dev, long long n,
                                       const dc_c64* replica_dev, long long n_rep,
                                       const double* v_r, int n_v, const double* tec_tecu,
                                       int n_tec, dc_c64* out_dev, double fs, double fc,
                                       const dc_opts* opts, void* stream);

/* Predistorted LFM transmit waveforms: the comparison methods of the paper's
 * FFT correction (Sec. II-A, Sec. II-C, Appendix B), generated on the GPU.
 * y_dev[m] = exp(i (phi(t_m) - 2 pi f_mix t_m)), t_m = m / fs, m < n, for an
 * LFM from f0 over `bandwidth` in T seconds predistorted for the two-way
 * ionosphere of TEC tec_tecu (K2 = kappa E, Eq. 3):
 *   DC_LFM_PLAIN          the undistorted LFM, phi = 2 pi (f0 t + B t^2/(2T))
 *   DC_LFM_CUBIC          f(t) the real root of Eq. 4 (Eqs. 11-14), phi by the
 *                         trapezoidal rule over the samples
 *   DC_LFM_POLY           the pseudo-Chebyshev expansion (Eqs. 5-10), phi in
 *                         closed form
 *   DC_LFM_POLY_ORIGINAL  the same with the factor-4 coefficients of
 *                         Appendix B (the paper's negative control)
 * Phases are carried in FP64 cycles and reduced before the FP32 sincos.
 * f_mix = 0 gives RF samples; f_mix = f0 gives the baseband sweep 0 .. B.
 * 1 <= n <= 2^22; fs, f0, bandwidth, T > 0; tec_tecu >= 0 and finite. */
typedef enum {
  DC_LFM_PLAIN = 0,
  DC_LFM_CUBIC = 1,
  DC_LFM_POLY = 2,
  DC_LFM_POLY_ORIGINAL = 3
} dc_lfm_kind;
DC_API dc_status predistort_lfm(dc_ctx* ctx, dc_c64* y_dev, long long n, double fs, double f0,
                                double bandwidth, double T, double tec_tecu, double f_mix,
                                int kind, void* stream);

/* Exact-sinc resampling of many pulses per range rate (Eq. 17 as a dense
 * contraction Y_a = X_a S_a^T, S_a[j][i] = sinc(alpha_a j - i)).
 * x_dev: pulses [n_alpha][n_pulses][n] with x_alpha_stride samples between
 *        consecutive alpha groups (0 = every alpha uses the same pulses);
 * v_r:   host [n_alpha], 1 <= n_alpha <= 65535;
 * y_dev: [n_alpha][n_pulses][n_out].
 * mode:  DC_EXACT_FP32 (CUDA cores), DC_EXACT_BF16X3 or DC_EXACT_FP16X3
 *        (tcgen05 tensor cores with hi/lo split operands, FP32 accumulation). */
DC_API dc_status resample_exact_batch(dc_ctx* ctx, const dc_c64* x_dev, long long n, int n_pulses,
                               long long x_alpha_stride, const double* v_r, int n_alpha,
                               dc_c64* y_dev, long long n_out, int mode, void* stream);

/* Plans: a correct_batch or correct_bank call recorded once into a CUDA
 * graph and replayed.  Creating a plan runs the call once on a private stream
 * (the outputs are written), then records it with plan-owned scratch and item
 * lists (uploaded once) and instantiates the graph.  The buffers and host
 * lists the call was given must stay valid while the plan is used; every
 * execution recomputes the outputs from the current contents of the input
 * buffers.  dc_plan_execute enqueues one graph launch on `stream`; executions
 * of one plan must not overlap on the GPU (they share its scratch).  This is
 * how a batch runs as a single submission (Sec. II-B's bundling of FFT work). */
typedef struct dc_plan dc_plan;
DC_API dc_status dc_plan_batch(dc_ctx* ctx, const dc_c64* in_dev, dc_c64* out_dev,
                               const dc_item* items, int n_items, const dc_opts* opts,
                               dc_plan** plan);
DC_API dc_status dc_plan_bank(dc_ctx* ctx, const dc_c64* x_dev, long long n, const double* v_r,
                              int n_v, const double* tec_tecu, int n_tec, dc_c64* out_dev,
                              double fs, double fc, const dc_opts* opts, dc_plan** plan);
DC_API dc_status dc_plan_execute(dc_plan* plan, void* stream);
/* Kernel launches one execution replays (-1 for a null plan). */
DC_API long long dc_plan_launches(const dc_plan* plan);
DC_API dc_status dc_plan_destroy(dc_plan* plan);

/* Serving loop with continuous batching (Sec. II-B's real-time use; the
 * paper itself processes one pulse per launch).
 *
 * dc_serve_start creates a server on `device` whose scheduler thread keeps up
 * to `slots` batches in flight, each on its own stream and context with its
 * own pinned host staging.  `hbm_budget_bytes` (0 = 8 GiB) bounds the
 * server's device memory: 1 MiB per slot is set aside for the slot's context
 * (tables, item lists) and the rest becomes one pool, allocated at start, from
 * which every batch in flight takes one block for its inputs, its outputs and
 * its correction scratch (about 40 bytes per sample), returned when the batch
 * completes.  The pool must hold a 2^20-sample request alone (32 MiB), else
 * DC_EINVAL.  Admission: requests join the next free slot's batch in arrival
 * order while they fit its staging (up to 32 Mi samples) and the pool can
 * hold the whole batch; a request the pool cannot hold yet waits until
 * batches in flight return memory (admission by the HBM budget), one that
 * finds every slot busy waits for a slot.  A slot's batch runs H2D ->
 * correct_batch -> D2H on its stream while the next slot fills with requests
 * that arrived meanwhile.  Where the device reads and writes pageable host
 * memory through the host's page tables (GB300 with its Grace host), H2D and
 * D2H are copy kernels between the callers' buffers and the pool, with no
 * host copies; elsewhere, or with the environment variable DC_SERVE_STAGED=1
 * at dc_serve_start, host threads copy through the slot's pinned staging.
 * Results do not depend on the batch a request rode in.
 *
 * dc_serve_submit queues one pulse (x_host: [n] samples, read after the request
 * is admitted; y_host: [n] corrected samples, written before dc_serve_wait
 * returns DC_OK; both must stay valid and untouched by the caller until
 * then).  n <= 2^20.  Writes the
 * request id.  dc_serve_wait blocks up to timeout_ms (< 0: forever) for a
 * request (DC_ETIMEOUT if still running; the request stays valid), writes its
 * latency from submission to completion, and forgets it.  dc_serve_cancel
 * drops a request still queued (DC_EBUSY once admitted).  dc_serve_stats
 * reports p50 / p99 latency, completed Msamples/s since the first submission,
 * and the number of completed requests; dc_serve_counters the admission
 * counters below.  dc_serve_stop drains in-flight work and frees the server
 * (requests not yet waited for are dropped). */
typedef struct dc_server dc_server;
DC_API dc_status dc_serve_start(int device, size_t hbm_budget_bytes, int slots, const dc_opts* opts,
                                dc_server** server);
DC_API dc_status dc_serve_submit(dc_server* server, const dc_c64* x_host, long long n, double fs,
                                 double fc, double v_r, double tec_tecu, dc_c64* y_host,
                                 long long* req_id);
DC_API dc_status dc_serve_wait(dc_server* server, long long req_id, int timeout_ms, double* latency_s);
DC_API dc_status dc_serve_cancel(dc_server* server, long long req_id);
DC_API dc_status dc_serve_stats(dc_server* server, double* p50_s, double* p99_s,
                                double* msamples_per_s, long long* completed);
DC_API dc_status dc_serve_stop(dc_server* server);

typedef struct {
  long long batches;          /* batches launched                                  */
  long long completed;        /* requests completed                                */
  long long waited_memory;    /* requests that, first in line with a slot free,
                                 waited for the pool (the HBM budget)              */
  long long waited_slot;      /* requests that, first in line, found every slot busy */
  size_t pool_bytes;          /* device pool carved from the budget                */
  size_t peak_bytes_in_flight;/* most pool bytes held by batches at once           */
  long long batch_capacity;   /* samples a batch may carry (staging)               */
} dc_serve_info;
DC_API dc_status dc_serve_counters(dc_server* server, dc_serve_info* out);

/* ----------------------------------------------------------- autotuning
 * Schedule choices of correct_batch / correct_bank (plans record whatever
 * the context holds when they are created):
 *   resample_q  outputs per lane of the tiled windowed resampler, 8 or 4
 *               (8 only applies where its quadratic tap weights hold);
 *   fft[m]      for L = 2^m, 4096 <= L <= 65536: 1 = cluster-fused kernels,
 *               2 = one row pass (L = 4096) or three passes;
 *   chunk[m]    bytes of three-pass intermediate per chunk of transforms of
 *               L = 2^m (-1 = a whole length class at once);
 *   resample_tc the bank's windowed resampling: 1 = tensor cores (a GEMM of
 *               the pulse's Hankel tiles with per-range-rate tap weights and
 *               their derivatives, fp16 hi/lo operands; used where the range
 *               rates allow it), 2 = the CUDA-core kernel;
 *   apply_kind  the bank's spectrum apply (factors + inverse transform) for
 *               8192 <= L <= 65536: 1 = cluster-fused, one 4096-point row per
 *               CTA (clusters of L / 4096 CTAs); 2 = cluster-fused, two rows
 *               per CTA (L >= 32768); 3 = rows and columns as tasks of one
 *               persistent grid meeting in an L2-resident scratch (no
 *               clusters).
 * 0 in any field means the library's built-in rule (tensor cores where
 * eligible for resample_tc; for apply_kind two passes at L = 65536, one row
 * per CTA below). */
typedef struct {
  int resample_q;
  int fft[21];
  long long chunk[21];
  double ms_default;    /* the tuned call under the schedule held before tuning */
  double ms_best;       /* the same call under the chosen schedule              */
  int candidates;       /* schedules timed                                      */
  int resample_tc;
  int apply_kind;
} dc_tuning;

/* Measure the schedule choices the call meets on its own data (each
 * candidate run and timed with CUDA events on `stream`, one choice at a time
 * with the others held), keep the fastest in the context, and leave the
 * call's outputs as written by the chosen schedule.  Synchronous; arguments
 * as for correct_batch / correct_bank; not allowed while a plan is being
 * recorded.  `report` (may be NULL) receives the resulting schedule. */
DC_API dc_status dc_autotune_batch(dc_ctx* ctx, const dc_c64* in_dev, dc_c64* out_dev,
                                   const dc_item* items, int n_items, const dc_opts* opts,
                                   void* stream, dc_tuning* report);
DC_API dc_status dc_autotune_bank(dc_ctx* ctx, const dc_c64* x_dev, long long n, const double* v_r,
                                  int n_v, const double* tec_tecu, int n_tec, dc_c64* out_dev,
                                  double fs, double fc, const dc_opts* opts, void* stream,
                                  dc_tuning* report);

/* Read the context's schedule, or replace it (NULL: back to the built-in
 * rules).  dc_tuning_set validates every field (DC_EINVAL). */
DC_API dc_status dc_tuning_get(const dc_ctx* ctx, dc_tuning* out);
DC_API dc_status dc_tuning_set(dc_ctx* ctx, const dc_tuning* t);

/* Schedule cache: dc_tuning_save writes the context's schedule to `path` as
 * a small JSON object ({"format": "dc_tuning/1", "resample_q": .., "resample_tc":
 * .., "apply_kind": .., "fft": {"<m>": ..}, "chunk": {"<m>": ..}}); dc_tuning_load reads such a
 * file and applies it as dc_tuning_set would (DC_EINVAL for a missing or
 * malformed file or an invalid schedule).  With the environment variable
 * DC_TUNING_CACHE naming a file, dc_create loads it when it exists and every
 * dc_autotune_* call writes its result there. */
DC_API dc_status dc_tuning_save(const dc_ctx* ctx, const char* path);
DC_API dc_status dc_tuning_load(dc_ctx* ctx, const char* path);

#ifdef __cplusplus
}
#endif

#endif /* DC_H */
