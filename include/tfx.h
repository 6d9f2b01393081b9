/*
 * tfx.h -- C ABI of libtfx: multichannel FIR / IIR filter chains on one GB300.
 *
 * The operation is the one TorchFX (arXiv 2504.08624) applies through its
 * filter classes and pipe operator (Sec. 3): every channel of a
 * [channels x samples] signal goes through an ordered chain of linear filters,
 * each FIR filter a causal direct convolution and each IIR filter a
 * difference equation with user-supplied coefficients (lfilter semantics),
 * here given as a cascade of second-order sections.  Sec. 4 (Tables 2-4)
 * benchmarks exactly these three shapes: FIR, IIR, and a chain.
 *
 * Definitions (zero initial state, output length N, per channel c):
 *   SOS section, row (b0 b1 b2 a0 a1 a2):
 *       a0*y[n] = b0*x[n] + b1*x[n-1] + b2*x[n-2] - a1*y[n-1] - a2*y[n-2]
 *   FIR, taps h[0..L-1]:   y[n] = sum_{k=0}^{min(n,L-1)} h[k] * x[n-k]
 *   chain: stages applied in list order, output of stage i feeds stage i+1.
 *
 * Data layout: x and y are FP32 device buffers, channel-major; sample n of
 * channel c is at p[c*ld + n], ld >= N.  x == y (in place) is allowed; any
 * other overlap of the two ranges is rejected.  No alignment is required
 * (16-byte aligned rows take a vector fast path).
 *
 * Coefficients are FP64 host arrays, read during the call and not retained.
 * The library converts them to the device representation (FP32 coefficients,
 * FP64-computed matrix powers and Toeplitz tiles) when it builds a plan.
 *
 * Streams: every launch goes on the caller's stream `s` (NULL = legacy
 * default stream).  Calls return once the work is enqueued; they never
 * synchronise the device, print, or abort.
 *
 * Errors: every entry point returns a tfx_status.  Argument errors are
 * detected before any launch (nothing is enqueued).  Errors the GPU detects
 * (a bounded wait that ran out) are recorded in the plan's status word and
 * returned by tfx_plan_get_error().
 */
#ifndef TFX_H
#define TFX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; declared here so the header needs no CUDA headers. */
typedef struct CUstream_st *tfx_stream;

typedef enum {
    TFX_OK = 0,
    TFX_ERR_INVALID = -1,     /* bad pointer, size, stride, coefficient (a0 == 0) */
    TFX_ERR_UNSTABLE = -2,    /* an SOS section has a pole with |p| >= 1 */
    TFX_ERR_WORKSPACE = -3,   /* workspace missing or smaller than required */
    TFX_ERR_CUDA = -4,        /* a CUDA runtime call failed */
    TFX_ERR_TIMEOUT = -5,     /* a device-side bounded wait gave up (see tfx_plan_get_error) */
    TFX_ERR_UNSUPPORTED = -6, /* valid request outside what this build implements */
    TFX_ERR_NOMEM = -7,       /* host or device allocation failed */
    TFX_ERR_DECAY = -8        /* after a coefficient update, a spectral training plan's chain
                                 response no longer decays within its transform's overlap */
} tfx_status;

typedef enum { TFX_STAGE_FIR = 0, TFX_STAGE_SOS = 1 } tfx_stage_kind;

/* One stage of a chain.  FIR: n taps at coef[0..n-1], n >= 1.
 * SOS: n sections, row-major [n x 6] = b0 b1 b2 a0 a1 a2, n >= 0, a0 != 0,
 * every pole strictly inside the unit circle.  Consecutive SOS stages form
 * one cascade.  coef is a host pointer, read during the call only. */
typedef struct {
    int32_t kind;
    int32_t n;
    const double *coef;
} tfx_stage;

/* Plan flags (bitwise OR). */
#define TFX_PLAN_DEFAULT 0u
#define TFX_PLAN_FIR_CUDA_CORES 1u /* FIR stages on CUDA cores only (no tensor-core Toeplitz GEMM) */
#define TFX_PLAN_UNFUSED 2u        /* one kernel per stage group; intermediates go through the workspace */
#define TFX_PLAN_FIR_BF16_PLAIN 4u /* tensor-core FIR, BF16 operands, no hi/lo correction (reported-only accuracy mode) */
#define TFX_PLAN_FIR_BF16_SPLIT 8u /* tensor-core FIR with BF16 hi/lo operands instead of the default scaled FP16 hi/lo */
#define TFX_PLAN_SCAN_WARP_TILES 16u /* cascade-only units: one warp per 1024-sample tile, warp-parallel look-back */
/* The plan supports tfx_plan_forward_train / tfx_plan_backward (gradients of
 * the chain for the filters used as network layers, Sec. 3).  Every FIR runs
 * as a unit of its own and cascades as warp-tile scans of at most 8 sections
 * (longer cascades are split); tfx_plan_execute still works on such a plan. */
#define TFX_PLAN_TRAINABLE 32u
/* FIRs of 64 taps or more by FFT overlap-save instead of the tensor-core
 * Toeplitz GEMM.  This is also the default route (measured faster on GB300
 * at every length from 65 taps) for signals of at least 2L samples (the
 * transforms round relative to each block's energy, and a shorter signal is
 * all leading transient); the flag forces it for any length, and keeps it when TFX_PLAN_FIR_TC,
 * _FIR_BF16_PLAIN or _FIR_BF16_SPLIT is set too, and FIR stages on CUDA cores
 * (TFX_PLAN_FIR_CUDA_CORES) never take it.  Hand-written register-resident
 * radix-16 FFTs of M = 1024..16384 points (16 points per thread; 32 with
 * radix-32 passes at 16384; FP32, the error is ~log2(M) eps of each block's
 * energy rather than per product).  Single-block (up to 12289 taps): blocks
 * of B = M - (L - 1) outputs, two blocks per complex transform.
 * Partitioned (any length, where the model finds it cheaper):
 * overlap-save with h cut into P = ceil(L / (M/2)) partitions, every
 * input segment transformed once (two channels per complex transform) into a
 * workspace of ceil(C/2) x ceil(N / (M/2)) x M complex values, and each output
 * block the inverse transform of the sum of the P partition products (two
 * launches).  The scheme and transform size are chosen per FIR from a cost
 * model fitted to GB300 timings unless TFX_PLAN_FIR_FFT_LOG(m) fixes
 * M = 2^m (m = 10..14; the scheme is still chosen by the model). */
#define TFX_PLAN_FIR_FFT 64u
/* Every FIR of TC_MIN_TAPS (64) taps or more on the tensor-core Toeplitz
 * GEMM, none by FFT. */
#define TFX_PLAN_FIR_TC 128u
#define TFX_PLAN_FIR_FFT_LOG(m) ((uint32_t)(m) << 16)
#define TFX_PLAN_FIR_FFT_LOG_MASK (15u << 16)
/* Cascade-only units of at most 8 sections (poles of radius <= 0.999) run
 * on the tensor cores by default: blocks of 112 samples, the zero-state
 * response and the block end state by one GEMM (lower-triangular Toeplitz
 * of the cascade's impulse response, FP16 hi/lo operands, FP32 accumulation),
 * a 16-dimensional scan of the block start states, their free responses by
 * a second GEMM.  Channels are cut into segments walked by one persistent
 * CTA per SM; each segment but a channel's first starts D samples early
 * from zero state (its warm-up outputs are discarded), D chosen at plan time
 * so that the free response of the true state is below 1e-9 of its initial
 * size after D samples (the unit keeps the look-back scan when no such D
 * fits within 65536 samples).  One launch.  With this flag such units run
 * the CUDA-core block-tile scan with decoupled look-back instead. */
#define TFX_PLAN_SCAN_LOOKBACK 512u
/* A whole chain of SOS cascades and FIRs (or of cascades alone) is one
 * linear time-invariant filter (Sec. 3: the pipe composes the stages in
 * order), and when its
 * cascades' impulse response g decays it is run by default as ONE kernel:
 * the composite impulse response h_c = g * f (f: every FIR's taps
 * convolved) is formed in FP64 at plan time, g truncated at the first D
 * samples beyond which sum|g| x sum|f| is below 1e-7 of the chain's RMS gain
 * ||h_c||_2 (g must have decayed within 65536 samples: the last 4096 of them
 * below 1e-14 of sum|g|; otherwise the chain keeps its separate units), and
 * the signal is filtered by FFT overlap-save with h_c (single-block,
 * M = 1024..16384 points), so it crosses HBM once.  The truncation changes
 * no output by more than 1e-7 ||h_c||_2 max|x|; the FP32 transforms round
 * relative to each block's energy.  Chosen when the signal holds at least
 * 2 (D + L - 1) samples and a cost model fitted to GB300 timings predicts it
 * faster than the separate units; plans with a tensor-core, CUDA-core,
 * transform-size or scan flag, or a pole of radius > 0.999 never take it.
 * tfx_plan_update_sos switches such a plan back to its separate units.
 * A TFX_PLAN_TRAINABLE plan composes by its closed-form spectrum instead
 * (at most 16 sections, at most one FIR; see tfx_plan_backward): the
 * transfer function is evaluated at the transform's bins, so the response
 * is not truncated, the overlap J covers 1.5 D + L - 1 samples (at least
 * M/4; M = 4096 or 8192), and coefficient updates rebuild the spectrum on
 * the device and check that the response still decays within J
 * (TFX_ERR_DECAY otherwise).  This flag disables the composition. */
#define TFX_PLAN_NO_COMPOSE 1024u
/* Test hook for failure detection: the first tile of channel 0 never publishes
 * its carries, so its successor's bounded wait runs out; the execution
 * completes (with wrong output) and tfx_plan_get_error() returns
 * TFX_ERR_TIMEOUT.  Never set in production. */
#define TFX_PLAN_TEST_DROP_PUBLISH 256u

typedef struct tfx_plan tfx_plan;

/*
 * tfx_plan_create -- validate a chain and precompute its device constants.
 * p      : out, receives the plan (owned by the caller; free with tfx_plan_destroy)
 * C, N   : channels and samples per channel (C >= 0, N >= 0)
 * ld     : row stride of x and y in elements, ld >= max(N, 1)
 * st,nst : the stages (Sec. 3 chaining), nst >= 0; nst == 0 is the identity
 * flags  : TFX_PLAN_* bits
 * Allocates device memory for the plan's constants (host-synchronous).
 * Errors: TFX_ERR_INVALID, TFX_ERR_UNSTABLE, TFX_ERR_NOMEM, TFX_ERR_CUDA.
 */
int tfx_plan_create(tfx_plan **p, int64_t C, int64_t N, int64_t ld,
                    const tfx_stage *st, int32_t nst, uint32_t flags);

/* Bytes of device workspace tfx_plan_execute needs (0 if none). */
size_t tfx_plan_workspace_size(const tfx_plan *p);

/* Number of kernels one tfx_plan_execute launches (flag resets done with
 * cudaMemsetAsync excluded, and so is the input copy an in-place call makes
 * when its single unit reads other tiles' or segments' input: a tensor-core
 * or single-block FFT FIR, or a segmented tensor-core cascade); -1 for a
 * NULL plan. */
int tfx_plan_launch_count(const tfx_plan *p);

/* One line describing the plan's units in execution order, separated by
 * ';', each "kind:key=value,...":
 *   cascade:S=..,scan=block|warp,carry=fp32|fp64     (SOS sections only)
 *   cascade:S=..,scan=seg,carry=fp32,segments=..,D=..  (by channel segments)
 *   fused:S=..,L=..                                  (cascade + FIR, CUDA cores)
 *   fir:L=..                                         (FIR on CUDA cores)
 *   fir_tc:L=..,kernel=k_fir_tc|k_fir_tc_ws|k_fir_tc_long
 *   fir_fft:L=..,M=..,B=..,P=..                      (P = 0: single-block)
 *   chain_fft:S=..,L=..,D=..,Lc=..,M=..,B=..   (the whole chain as one FIR of
 *                                               Lc = D + L - 1 taps; L: the FIRs'
 *                                               combined length)
 * Writes at most len bytes including the terminating NUL into buf (buf may be
 * NULL when len is 0) and returns the length of the full description (as
 * snprintf does), or -1 for a NULL plan. */
int tfx_plan_describe(const tfx_plan *p, char *buf, size_t len);

/*
 * tfx_plan_execute -- run the chain: y = chain(x).  Asynchronous on s.
 * x, y : device FP32 buffers laid out as the plan's (C, N, ld); x == y allowed
 * ws   : device workspace of at least tfx_plan_workspace_size(p) bytes,
 *        256-byte aligned, owned by the caller, not touched after the work
 *        completes.  May be NULL only when the size is 0.
 * Makes no allocation and no host synchronisation, so it can be captured in
 * a CUDA graph.  Concurrent executions must use distinct workspaces.
 * Errors: TFX_ERR_INVALID, TFX_ERR_WORKSPACE, TFX_ERR_CUDA.
 */
int tfx_plan_execute(tfx_plan *p, const float *x, float *y, void *ws,
                     size_t ws_bytes, tfx_stream s);

/*
 * tfx_plan_execute_plain -- the same chain on the plain sequential path: one
 * thread per channel walks each IIR stage over time, one thread per output
 * sample sums each FIR stage, one kernel per stage.  It is the comparison
 * baseline for the scan/fused kernels.  Same arguments and workspace.
 */
int tfx_plan_execute_plain(tfx_plan *p, const float *x, float *y, void *ws,
                           size_t ws_bytes, tfx_stream s);

/*
 * tfx_plan_get_error -- status recorded by the GPU during this plan's
 * executions (TFX_OK or TFX_ERR_TIMEOUT), then cleared.  Synchronises the
 * device first, so it must not be called during stream capture.
 */
int tfx_plan_get_error(tfx_plan *p);

/* Free the plan (synchronises the device).  NULL is a no-op. */
void tfx_plan_destroy(tfx_plan *p);

/*
 * Gradients (TFX_PLAN_TRAINABLE plans).  Sec. 3 builds every filter as an
 * nn.Module so that chains sit inside neural networks; these calls give the
 * reverse-mode derivatives such a network needs.  For L = sum(g * y), y the
 * chain's output and g = dL/dy:
 *   dx    = dL/dx, [C x N] with the plan's row stride
 *   dcoef = dL/d(every coefficient), FP64, stages in chain order: an FIR stage
 *           contributes its n taps, an SOS stage its n rows of 6 raw values
 *           (b0 b1 b2 a0 a1 a2, before the a0 normalisation); summed over
 *           channels (the coefficients are shared by all channels).
 *
 * tfx_plan_saved_size     : bytes of device memory a training forward keeps
 *                           for the backward: the input of every unit after
 *                           the first (an intermediate of the chain), and
 *                           each cascade's state at every 32-sample chunk
 *                           start (8 bytes per section per chunk); 0 for a
 *                           plan without TFX_PLAN_TRAINABLE and for a plan
 *                           on the spectral route (it saves nothing).
 * tfx_plan_describe names the route: "chain_spectral:..." for the spectral
 * route, the units otherwise.
 * tfx_plan_backward_workspace_size : bytes of backward workspace (0 likewise).
 * tfx_plan_coef_count     : doubles in dcoef (-1 for a NULL plan).
 */
size_t tfx_plan_saved_size(const tfx_plan *p);
size_t tfx_plan_backward_workspace_size(const tfx_plan *p);
int64_t tfx_plan_coef_count(const tfx_plan *p);

/*
 * tfx_plan_forward_train -- y = chain(x) as tfx_plan_execute, and fill
 * `saved` (device, >= tfx_plan_saved_size bytes, 256-byte aligned, owned by
 * the caller) with what tfx_plan_backward needs.  x == y is rejected (the
 * backward reads x again); ws as for tfx_plan_execute.  Asynchronous, no
 * allocation, capturable.
 * Errors: TFX_ERR_INVALID (not trainable, x == y, overlapping buffers),
 * TFX_ERR_WORKSPACE, TFX_ERR_CUDA.
 */
int tfx_plan_forward_train(tfx_plan *p, const float *x, float *y, void *saved,
                           size_t saved_bytes, void *ws, size_t ws_bytes,
                           tfx_stream s);

/*
 * tfx_plan_forward_train_mse -- tfx_plan_forward_train followed by tfx_mse
 * against `target` (device, [C x N], the plan's row stride): y, the saved
 * state, g = dL/dy = 2 (y - target) / (C N) and *loss = mean((y - target)^2)
 * (device FP64 scalar, reset on s first).  On the spectral route the loss
 * is computed in the filter kernel's store (one launch: y is not read back);
 * otherwise the units, then the loss kernel.  g may be target (it replaces
 * it); no other buffers may overlap.  Asynchronous, no allocation,
 * capturable.  The loss is summed in FP32 per thread and FP64 across
 * threads, CTAs added by atomics (its last bits may vary between calls; y
 * and g do not).
 * tfx_plan_forward_train_mse_launch_count: kernels it launches (-1 if not
 * trainable).
 * Errors: as tfx_plan_forward_train; TFX_ERR_INVALID for a NULL loss, target
 * or g, or overlapping buffers.
 */
int tfx_plan_forward_train_mse(tfx_plan *p, const float *x, float *y,
                               const float *target, float *g, double *loss,
                               void *saved, size_t saved_bytes, void *ws,
                               size_t ws_bytes, tfx_stream s);
int tfx_plan_forward_train_mse_launch_count(const tfx_plan *p);

/*
 * tfx_plan_backward -- given the x and `saved` of a training forward (not
 * modified since) and g = dL/dy (device, [C x N], the plan's row stride),
 * write dx (may be NULL: not computed; may equal g; must not overlap x) and
 * dcoef (device FP64, tfx_plan_coef_count values, fully overwritten; may be
 * NULL: not computed).  ws: device, >= tfx_plan_backward_workspace_size
 * bytes, 256-byte aligned.  Spectral route (a chain that composes; see
 * TFX_PLAN_NO_COMPOSE): dx is the chain over the time-reversed gradient
 * by the forward's FFT kernel, and dcoef comes from the cross-spectrum of g
 * and x (accumulated by blocks) paired with the closed-form derivative
 * spectra of every section coefficient and one inverse transform for the
 * FIR taps; every reduction has a fixed order, so repeated calls give
 * bit-identical results.  With both dx and dcoef asked, dx runs on a second,
 * plan-owned stream forked from s by an event after the correlation and
 * joined back into s before the call's work ends (a capture of s captures
 * both); a plan's backward calls must therefore be issued from one host
 * thread at a time.  Otherwise the SOS cascades run as reverse-time
 * adjoint scans that recompute their section outputs from the saved
 * chunk-start states; FIRs as the FIR over the time-reversed gradient plus a
 * tap correlation.  Asynchronous, no allocation, capturable; a device-side
 * timeout is reported by tfx_plan_get_error.
 * Errors: TFX_ERR_INVALID, TFX_ERR_WORKSPACE, TFX_ERR_CUDA.
 */
int tfx_plan_backward(tfx_plan *p, const float *x, const float *g, float *dx,
                      double *dcoef, const void *saved, size_t saved_bytes,
                      void *ws, size_t ws_bytes, tfx_stream s);

/* Kernels one tfx_plan_backward launches with (with_dx, with_dcoef) set as
 * (dx != NULL, dcoef != NULL); memsets excluded; -1 if not trainable. */
int tfx_plan_backward_launch_count(const tfx_plan *p, int with_dx, int with_dcoef);

/*
 * tfx_plan_train_step_mse -- one training step of the MSE loss: the result
 * of tfx_plan_forward_train_mse (y, g = dL/dy, *loss, saved) followed by
 * tfx_plan_backward with that g (dx and/or dcoef; both NULL: the forward
 * alone), with the same arguments and the same rules for each pointer.  On a
 * spectral plan (see TFX_PLAN_NO_COMPOSE) with dcoef requested, one fused
 * launch does the forward, the loss and the block correlation of g with x
 * (the forward's input spectra kept in shared memory, g transformed straight
 * from the registers that store it), so x and g are not read a second time;
 * the correlation is summed over other block pairings than in
 * tfx_plan_backward, so dcoef agrees with the two calls to FP32 rounding
 * (y, g and dx are the same).  ws: at least the larger of the two calls'
 * sizes (tfx_plan_workspace_size, tfx_plan_backward_workspace_size).
 * Errors: as the two calls.
 */
int tfx_plan_train_step_mse(tfx_plan *p, const float *x, float *y,
                            const float *target, float *g, double *loss,
                            float *dx, double *dcoef, void *saved,
                            size_t saved_bytes, void *ws, size_t ws_bytes,
                            tfx_stream s);
/* Kernels one tfx_plan_train_step_mse launches (memsets excluded). */
int tfx_plan_train_step_mse_launch_count(const tfx_plan *p, int with_dx, int with_dcoef);

/*
 * tfx_mse -- mean squared error between y and target ([C x N], row stride
 * ld, device): *loss = mean((y - target)^2) (device FP64 scalar, written
 * after a reset on s), and g = dL/dy = 2 (y - target) / (C N) unless g is
 * NULL.  The loss the differentiable-chain workload trains with.
 * Errors: TFX_ERR_INVALID, TFX_ERR_CUDA.
 */
int tfx_mse(const float *y, const float *target, float *g, int64_t C,
            int64_t N, int64_t ld, double *loss, tfx_stream s);

/*
 * One-shot calls.  They build (or reuse from an internal cache keyed by the
 * arguments and the stream) a plan with its own library-owned workspace, then
 * execute it on s.  The first call for a configuration allocates and is
 * host-synchronous; repeats allocate nothing.  Two overlapping calls with the
 * same configuration and stream are ordered by the stream, so they are safe.
 *
 * tfx_fir  : one FIR stage (taps >= 1)       -- Sec. 3 FIR filters, Table 2
 * tfx_sos  : one SOS cascade (sections >= 0) -- Sec. 3 IIR filters, Table 3
 * tfx_chain: a chain (Sec. 3 pipe operator, Table 4).  If ws is non-NULL it
 *            is used instead of the cached workspace (ws_bytes must be at
 *            least tfx_chain_workspace_size()).
 */
int tfx_fir(const float *x, float *y, int64_t C, int64_t N, int64_t ld,
            const double *h, int32_t taps, tfx_stream s);
int tfx_sos(const float *x, float *y, int64_t C, int64_t N, int64_t ld,
            const double *sos, int32_t sections, tfx_stream s);
int tfx_chain(const float *x, float *y, int64_t C, int64_t N, int64_t ld,
              const tfx_stage *st, int32_t nst, void *ws, size_t ws_bytes,
              tfx_stream s);
/*
 * tfx_chain_host -- the chain of tfx_chain over signals in HOST memory (the
 * call a serving process makes with audio it holds on the host).  x and y are
 * host pointers with the same [C x N] layout and row stride ld (x == y
 * allowed); page-locked (pinned) buffers let the copies run asynchronously
 * and overlap, pageable ones still work but serialise.  Channels are cut
 * into groups of about 2^23 samples; group g is copied in, filtered and
 * copied out on three library-owned streams through a ring of three device
 * slots, so copies of neighbouring groups overlap each other and the
 * filtering.  The work is ordered after prior work on s and s waits for it:
 * synchronise s before reading y.  The first call for a configuration
 * builds its plans and allocates the device slots (host-synchronous); later
 * calls allocate nothing.  With x and y page-locked the whole pipeline is
 * captured once into a CUDA graph (again when x, y or ld change) and each
 * call is one graph launch on s: the host thread's timing no longer paces
 * the copies.  Do not call it while s is being captured.
 * Errors: as tfx_chain, plus TFX_ERR_NOMEM for the device slots.
 */
int tfx_chain_host(const float *x, float *y, int64_t C, int64_t N, int64_t ld,
                   const tfx_stage *st, int32_t nst, tfx_stream s);

/* Release the cached host-buffer pipelines (synchronises the device). */
void tfx_host_cache_clear(void);

/* Introspection of the host-buffer pipelines: *pipes = the number cached,
 * *graphed = how many of them hold a captured CUDA graph (each call of
 * tfx_chain_host with page-locked x and y replays its configuration's
 * graph, capturing it first when the buffers changed; pageable buffers
 * enqueue the pipeline call by call).  Either pointer may be NULL.
 * Returns TFX_OK. */
int tfx_host_cache_info(int32_t *pipes, int32_t *graphed);

/* Workspace tfx_chain needs for these arguments (SIZE_MAX if invalid). */
size_t tfx_chain_workspace_size(int64_t C, int64_t N, int64_t ld,
                                const tfx_stage *st, int32_t nst);

/* Release every cached one-shot plan (synchronises the device). */
void tfx_cache_clear(void);

/*
 * tfx_sos_noalloc -- the SOS cascade of tfx_sos for callers that cannot
 * allocate device memory: code running in a real-time audio callback or a
 * plug-in host, where cudaMalloc's implicit device synchronisation and
 * unbounded latency are not allowed, and programs whose device memory is all
 * reserved up front by an allocator they do not control.  The paper has no
 * counterpart; it is an extra entry point of this library.
 *
 * Same arguments, layout and result as tfx_sos (x == y allowed), for
 * cascades whose poles all have radius <= 0.999: this entry point keeps FP32
 * cross-tile carries, so a section with a pole beyond that radius (where
 * tfx_sos switches to FP64 carries) returns TFX_ERR_UNSUPPORTED.  The call
 * makes no cudaMalloc / cudaFree and uses no allocating library routine: the
 * scan's scratch (tile ticket, status word, look-back carries) and the
 * section constants live in one fixed static device array of about 4.3 MB
 * that every GPU loading the library holds until the process exits.  The
 * host normalises the rows in FP64 (a few hundred bytes of stack) and passes
 * them to a set-up kernel by value, which builds the section constants in
 * the array; nothing is copied from host memory.
 * Limits: sections <= 8 and C * ceil(N / 8192) <= 32768 (for example 64
 * channels of up to 4.19 M samples); larger requests return
 * TFX_ERR_UNSUPPORTED before anything is enqueued.
 * The first call on a device looks up the array's device address (a host
 * synchronising runtime query), so make that first call before any stream
 * capture on that device.  All calls share the one array and each call
 * overwrites what the previous one left there: calls whose work overlaps on
 * the GPU (different streams, or host threads racing) corrupt each other's
 * results; calls ordered on one stream are safe.  Device-side timeouts are
 * not reported (there is no plan to hold a status).
 * Errors: TFX_ERR_INVALID, TFX_ERR_UNSTABLE, TFX_ERR_UNSUPPORTED, TFX_ERR_CUDA.
 */
int tfx_sos_noalloc(const float *x, float *y, int64_t C, int64_t N, int64_t ld,
                    const double *sos, int32_t sections, tfx_stream s);

/*
 * Batched launch over many clips (Sec. 4: many channels and files at once).
 * Each clip has its own channel count C, length N and chain; the clips are
 * PACKED into one device input and one device output buffer: clip i occupies
 * floats [off_i, off_i + C_i N_i) (row stride N_i), off_i =
 * tfx_batch_clip_offset(b, i), and tfx_batch_total_samples(b) floats in all.
 *
 * tfx_batch_create -- validate and plan every clip (host FP64 precompute, as
 * tfx_plan_create).  A clip whose chain composes into one FIR (its cascades'
 * impulse response decays: the composite-response reading of
 * TFX_PLAN_NO_COMPOSE) runs by FFT overlap-save, and all such clips of one
 * transform size run as ONE launch (each CTA reads its clip from a per-CTA
 * table built with the batch and uses the clip's own spectrum).  The units of the other clips
 * are grouped by position in their chain and by kernel (fused cascade +
 * short FIR / cascade / FIR of 64+ taps by single-block FFT per transform
 * size / tensor-core FIR with NB output blocks per tile, for a FIR one FFT
 * block cannot hold); each group runs as ONE launch over the tiles of all
 * its units.
 * TFX_PLAN_NO_COMPOSE in plan_flags keeps every clip on the grouped units.
 * Allocates device memory (host-synchronous).
 * params may be NULL (defaults).  Clips whose tensor-core FIR tables do not
 * fit in shared memory beside a window are TFX_ERR_UNSUPPORTED.
 * tfx_batch_execute -- y = chain_i(x) for every clip; x and y must not
 * overlap; ws >= tfx_batch_workspace_size bytes, 256-byte aligned.  No
 * allocation and no host synchronisation: capturable in a CUDA graph (the
 * whole batch as one graph launch).  tfx_batch_launch_count kernels.
 * Errors: TFX_ERR_INVALID, TFX_ERR_UNSTABLE, TFX_ERR_WORKSPACE,
 * TFX_ERR_UNSUPPORTED, TFX_ERR_NOMEM, TFX_ERR_CUDA; device-side timeouts via
 * tfx_batch_get_error (synchronising, like tfx_plan_get_error).
 */
typedef struct {
    int64_t C;             /* channels (>= 0) */
    int64_t N;             /* samples per channel (>= 0) */
    const tfx_stage *st;   /* the clip's chain */
    int32_t nst;
} tfx_clip;

typedef struct {
    uint32_t plan_flags;   /* TFX_PLAN_* for every clip (TFX_PLAN_DEFAULT, _NO_COMPOSE, _FIR_CUDA_CORES,
                              _FIR_BF16_*); FIRs of clips that do not compose run by single-block FFT
                              where one block holds the taps, else on the tensor cores (_FIR_FFT is
                              rejected) */
    int32_t fir_nb;        /* tensor-core FIR output blocks of 128 per tile: 64, 128 or 256 (0: 128) */
    int32_t tc_min_taps;   /* FIRs not on the FFT with at least this many taps use the tensor
                              cores (0: 64) */
    int32_t fft_m[16];     /* composed clips whose composite response has Lc taps with
                              floor(log2(Lc)) = k run with transforms of 2^fft_m[k] points
                              (10..14; 0, or a size that cannot hold Lc - 1 taps with M/4
                              outputs per block: the cost model's choice) -- the knob the
                              autotuner sets per length bucket */
} tfx_batch_params;

typedef struct tfx_batch tfx_batch;

int tfx_batch_create(tfx_batch **b, const tfx_clip *clips, int32_t nclips,
                     const tfx_batch_params *params);
int64_t tfx_batch_total_samples(const tfx_batch *b);
int64_t tfx_batch_clip_offset(const tfx_batch *b, int32_t i);
size_t tfx_batch_workspace_size(const tfx_batch *b);
int tfx_batch_launch_count(const tfx_batch *b);
int tfx_batch_execute(tfx_batch *b, const float *x, float *y, void *ws,
                      size_t ws_bytes, tfx_stream s);
int tfx_batch_get_error(tfx_batch *b);
void tfx_batch_destroy(tfx_batch *b);

/* The batch's launches, for profiling: group g's kind (0 fused cascade +
 * CUDA-core FIR, 1 cascade, 2 tensor-core FIR, 3 composed chains by FFT of
 * one transform size, 4 FIR units of clips that keep their units, by
 * single-block FFT of one transform size), its level in the chains, its
 * tiles, the channel-samples it filters and its algorithmic flops (10 per
 * section-sample, 2 L per FIR sample); tfx_batch_execute_group runs group g
 * alone (its inputs must hold what the earlier levels write). */
/* Clip i of a batch: whether it runs as a composed chain (1) or by grouped
 * units (0), the taps of its composite response and its transform size
 * exponent (both 0 when not composed). */
int tfx_batch_clip_info(const tfx_batch *b, int32_t i, int32_t *composed, int32_t *taps, int32_t *fft_m);
int tfx_batch_group_count(const tfx_batch *b);
int tfx_batch_group_info(const tfx_batch *b, int32_t g, int32_t *kind, int32_t *level,
                         int64_t *tiles, int64_t *samples, double *flops);
int tfx_batch_execute_group(tfx_batch *b, int32_t g, const float *x, float *y, void *ws,
                            size_t ws_bytes, tfx_stream s);

/*
 * Filter design on the GPU in FP64, and coefficient updates without a host
 * round trip.  Sec. 3 builds IIR filters from design parameters (cutoff,
 * order, ripple, gain, Q); these calls compute the sections on the device.
 *
 * tfx_design: one filter.  kind / fields used:
 *   TFX_DESIGN_BUTTER_LOW / _HIGH : order (1..16), f1 = fc (-3 dB), fs
 *   TFX_DESIGN_CHEBY1_LOW         : order, f1 = passband edge, p1 = ripple dB, fs
 *   TFX_DESIGN_PEAKING            : f1 = f0, p1 = Q, p2 = gain dB, fs (RBJ)
 *   TFX_DESIGN_LOW_SHELF / _HIGH  : f1 = f0, p1 = gain dB, p2 = shelf slope (0: 1), fs (RBJ)
 *   TFX_DESIGN_BIQUAD_POLAR       : poles r = f1 + f2 sigmoid(p1), theta = pi sigmoid(p2),
 *                                   numerator b[0..2] (the learnable cascade's parameters)
 * Butterworth / Chebyshev-I: bilinear transform of the analog prototype with
 * the cutoff prewarped to tan(pi fc / fs); sections by increasing pole
 * radius, zeros at z = -1 (low-pass) or +1 (high-pass), unit gain at DC
 * (low) or Nyquist (high); even-order Chebyshev-I has DC gain 10^(-rp/20).
 * tfx_design_sections: sections the spec produces (-1 if invalid).
 * tfx_design_device: specs, row_off (first output row of each spec) and
 *   rows (6 doubles per row, raw b0 b1 b2 a0 a1 a2) in device memory; one
 *   thread per spec; invalid specs set *status (device int) to
 *   TFX_ERR_INVALID.  Asynchronous on s, capturable.
 * tfx_plan_update_sos: recompute the plan's section constants (normalisation,
 *   recursion coefficients, chunk-transfer powers; FP64 on the GPU) from
 *   rows = device FP64 array of every SOS row of the plan's chain in order
 *   (tfx_plan_sos_rows of them).  The plan's structure (units, kernels, the
 *   FP64-carry routing chosen at creation) is kept, except that cascades
 *   running on the tensor cores (whose GEMM tables are derived from the
 *   coefficients on the host) run the look-back scan from the first update
 *   on; FIR taps are not changed.  An unstable or invalid row sets the status read by
 *   tfx_plan_get_error.  The first call uploads per-section descriptors
 *   (host-synchronous: make it before any capture); later calls are one
 *   launch, capturable.  Must not overlap an execution of the plan.
 */
#define TFX_DESIGN_BUTTER_LOW 0
#define TFX_DESIGN_BUTTER_HIGH 1
#define TFX_DESIGN_CHEBY1_LOW 2
#define TFX_DESIGN_PEAKING 3
#define TFX_DESIGN_LOW_SHELF 4
#define TFX_DESIGN_HIGH_SHELF 5
#define TFX_DESIGN_BIQUAD_POLAR 6

typedef struct {
    int32_t kind;
    int32_t order;
    double f1, f2, fs, p1, p2;
    double b[3];
} tfx_design;

int tfx_design_sections(const tfx_design *spec);
int tfx_design_device(const tfx_design *specs, int32_t n, const int64_t *row_off,
                      double *rows, int *status, tfx_stream s);
int tfx_plan_update_sos(tfx_plan *p, const double *rows, tfx_stream s);
int64_t tfx_plan_sos_rows(const tfx_plan *p);

/*
 * tfx_plan_update_coefs -- every coefficient of the plan's chain from device
 * memory, without a host round trip: the update a training step makes after
 * its optimizer step (Sec. 3: filters as trainable modules).  coef: device
 * FP64, tfx_plan_coef_count values in the layout of tfx_plan_backward's
 * dcoef (stages in chain order; an FIR stage its taps, an SOS stage its raw
 * rows b0 b1 b2 a0 a1 a2).  Recomputes on the GPU the section constants (as
 * tfx_plan_update_sos), the FIR taps' FP32 copies and, for FIRs run by FFT,
 * their spectra (FP32 transform of the taps, as the filter's own).  The
 * plan's structure stays as created (units, kernels, transform sizes, the
 * FP64-carry routing); a tensor-core cascade runs the look-back scan and a
 * composed chain its separate units from the first update on; a plan on
 * the spectral route keeps it: the FIR's spectrum and the chain's
 * closed-form spectrum are rebuilt on the GPU, and a response that no
 * longer decays within the plan's overlap sets TFX_ERR_DECAY in the status
 * read by tfx_plan_get_error (recreate the plan).  FIRs on the
 * tensor cores (tap tables scaled on the host) are TFX_ERR_UNSUPPORTED.  The
 * first call builds the update descriptors (host-synchronous: make it before
 * any capture); later calls are tfx_plan_update_coefs_launch_count launches,
 * asynchronous and capturable.  An unstable or invalid row sets the status
 * read by tfx_plan_get_error.  Must not overlap an execution of the plan.
 * Errors: TFX_ERR_INVALID, TFX_ERR_UNSUPPORTED, TFX_ERR_NOMEM, TFX_ERR_CUDA.
 */
int tfx_plan_update_coefs(tfx_plan *p, const double *coef, tfx_stream s);
int tfx_plan_update_coefs_launch_count(const tfx_plan *p);

/*
 * Measurement helper (the paper has no counterpart): the FP32 multiply-add
 * rate of this GPU, the denominator of the CUDA-core rooflines, which must
 * be measured rather than derived from clock and unit counts.
 * tfx_fma_probe enqueues `blocks` CTAs of `threads` threads (a multiple of
 * 32, at most 1024) that each run 8 independent chains of `iters` FP32 FMAs
 * (packed != 0: the two-lane packed FMA, two per instruction) and write one
 * float per thread to `out` (device, blocks * threads floats).  Time it with
 * events on s; tfx_fma_probe_flops gives the flops one launch performs.
 * Errors: TFX_ERR_INVALID, TFX_ERR_CUDA.
 */
int tfx_fma_probe(float *out, int32_t blocks, int32_t threads, int32_t iters,
                  int32_t packed, tfx_stream s);
double tfx_fma_probe_flops(int32_t blocks, int32_t threads, int32_t iters,
                           int32_t packed);

/* Human-readable name of a tfx_status. */
const char *tfx_strerror(int status);

/* Library version, e.g. 0x000100 for 0.1.0. */
int tfx_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TFX_H */
