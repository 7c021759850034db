/*
 * tacaw.h -- C ABI of the GB300 streaming TACAW time->energy library (libtacaw.so).
 *
 * The library turns exit waves psi[probe][t][ky][kx], pushed a few frames at a time
 * from multislice runs over MD snapshots, into energy-resolved diffraction
 * patterns and detector spectra:
 *
 *   mu[k]    = (1/T) sum_t psi[t,k]                   time mean (elastic part), removed if asked
 *   Psi[k,j] = sum_t w_t (psi[t,k] - mu[k]) exp(-2 pi i frac(E_j dt t / h))
 *   I[k,j]   = B(E_j) |Psi[k,j]|^2                    Eq. 1 (B: quantum-statistics factor)
 *   S[d,j]   = sum_k M_d(k) I[k,j]                    DetectorSet apertures (Sec. II.B)
 *
 * The windowed time->energy Fourier transform of a segment ("chunk" of L snapshots,
 * Sec. II.B "Welch method") is Eq. 1's phi_MD(q,E); windows follow Sec. III.A (rectangular =
 * Tukey alpha 0, Hann = Tukey alpha 1) in scipy's periodic form (App. A); energies are
 * an explicit grid inside the Nyquist range eps = h/(2 dt) (App. B) or FFT bins; the
 * k-space region of interest is a crop of the full multislice grid (Sec. II.B, "ROI
 * slicing").  Units: h = 4.135667696 meV ps, energies in meV, dt in fs.
 *
 * Conventions for every entry point:
 *   - Device pointers ("d_") are CUDA device addresses on the current device; the
 *     caller owns them.  Host pointers are read during the call only.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  All
 *     work is enqueued on it; calls return without waiting, except tacaw_finalize and
 *     tacaw_backward, which wait for their own work to read the device error flag.
 *   - Every call returns a tacaw_status; tacaw_last_error() gives a message for the
 *     last non-OK status of the calling thread.  Argument errors leave the plan
 *     unchanged; a CUDA error or a device timeout poisons the plan (only
 *     tacaw_destroy is then accepted).
 *   - Nothing here traps or aborts; device-side waits are bounded and report
 *     TACAW_ERR_TIMEOUT.
 *   - Every entry point (and every contraction launch inside it) is a named NVTX range,
 *     visible in Nsight Systems; without a profiler attached a range costs a pointer test.
 */
#ifndef TACAW_H_
#define TACAW_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TACAW_OK = 0,
    TACAW_ERR_INVALID_ARG = 1,  /* bad descriptor or argument; nothing was changed            */
    TACAW_ERR_OOM = 2,          /* device allocation failed or the HBM budget is too small    */
    TACAW_ERR_CUDA = 3,         /* a CUDA call failed; the plan is poisoned                    */
    TACAW_ERR_STATE = 4,        /* call out of order (finalize before T frames, push after it) */
    TACAW_ERR_OVERFLOW = 5,     /* push would exceed the segment length T; nothing was pushed  */
    TACAW_ERR_TIMEOUT = 6,      /* a device-side wait ran out; the plan is poisoned            */
    TACAW_ERR_UNSUPPORTED = 7   /* valid request this build does not implement                 */
} tacaw_status;

/* Time windows, Sec. III.A and App. A (scipy periodic forms, length-1 windows are [1]):
 *   RECT   w_t = 1
 *   HANN   w_t = 1/2 - 1/2 cos(2 pi t / T)
 *   GAUSS  w_t = exp(-1/2 ((t - T/2)/sigma)^2), sigma = window_param frames (<= 0: T/6)
 *   TUKEY  cosine tapers of total fractional width alpha = window_param
 *   BLACKMANHARRIS  4-term cosine sum 0.35875, 0.48829, 0.14128, 0.01168 (Harris)
 *   KAISER I0(beta sqrt(1 - (2t/T - 1)^2)) / I0(beta), beta = window_param (>= 0)
 *   CHEBWIN Dolph-Chebyshev, side lobes window_param dB (> 0) below the main lobe      */
typedef enum {
    TACAW_WIN_RECT = 0,
    TACAW_WIN_HANN = 1,
    TACAW_WIN_GAUSS = 2,
    TACAW_WIN_TUKEY = 3,
    TACAW_WIN_BLACKMANHARRIS = 4,
    TACAW_WIN_KAISER = 5,
    TACAW_WIN_CHEBWIN = 6
} tacaw_window;

/* Arithmetic of the time->energy contraction.
 *   FP32        CUDA-core FFMA, FP32 accumulate.
 *   SPLIT_BF16  tcgen05 tensor cores: each operand x = hi + lo with hi, lo bf16; the
 *               product is hi*hi + hi*lo + lo*hi with FP32 accumulation in tensor memory.
 *   SPLIT_FP16  the same with fp16 pieces (11-bit significands: hi + lo carries 22 bits
 *               against 16 for bf16).  fp16 has a narrow exponent range, so the frames'
 *               residual psi - mu_hat is multiplied by tacaw_plan_desc.fp16_scale (a power
 *               of two, undone exactly in the epilogue) before the split; the twiddles
 *               (|w e^{-i theta}| <= 1) are split unscaled.  A scaled component beyond the
 *               fp16 range (65504) is detected: finalize / tacaw_check_errors then return
 *               TACAW_ERR_OVERFLOW and the plan is poisoned.  Staged operands only
 *               (frames_in_place must be 0).
 * Twiddle phases are always reduced in FP64; the exact mean correction is FP64-derived. */
typedef enum { TACAW_PREC_FP32 = 0, TACAW_PREC_SPLIT_BF16 = 1, TACAW_PREC_SPLIT_FP16 = 2 } tacaw_precision;

/* Accumulation of Psi across flushes (used only when a segment needs more than one
 * flush): compensated FP32 (sum + Kahan compensation), FP64, or plain FP32 (half the
 * accumulator memory and traffic; each flush adds one FP32 rounding, ~6e-8 relative, so it
 * suits segments of up to tens of flushes).                                            */
typedef enum {
    TACAW_ACC_KAHAN_FP32 = 0,
    TACAW_ACC_FP64 = 1,
    TACAW_ACC_FP32 = 2,
    TACAW_ACC_AUTO = 3 /* plain FP32 when no segment needs more than 16 flushes at the K_stage
                          that fits the budget with it (half-size accumulators leave more room
                          for staging), else compensated FP32 */
} tacaw_accum;

/* Apertures (Sec. II.B DetectorSet).  Centres are offsets in pixels from the DC pixel
 * (kx/2, ky/2) of the ROI.  Pixel (ix, iy) with squared distance d2 to the centre is in
 * a CIRCULAR aperture when d2 <= r_out^2, in an ANNULAR one when r_in^2 < d2 <= r_out^2.
 * MASK: d_mask is a caller-owned device array of ky*kx float weights (row-major, kx
 * fastest), read during tacaw_plan_create only.                                        */
typedef enum { TACAW_DET_CIRCULAR = 0, TACAW_DET_ANNULAR = 1, TACAW_DET_MASK = 2 } tacaw_detector_kind;

typedef struct {
    int kind;            /* tacaw_detector_kind */
    float cx, cy;        /* centre offset from the DC pixel, pixels */
    float r_in, r_out;   /* radii, pixels */
    const float *d_mask; /* TACAW_DET_MASK only */
} tacaw_detector;

/* One stream = one supercell partition with its own probes, ROI, segment and windows.
 * Pushed frames are complex64 (interleaved re, im float32).  Element (p, t, y, x) of a
 * pushed buffer, t the frame index inside that push, is at complex64 offset
 *   p*pitch_probe + t*pitch_frame + (roi_y0 + y)*pitch_row + (roi_x0 + x)
 * so the k-space ROI is cropped out of the full multislice grid while it is read.     */
typedef struct {
    int n_probes;              /* P >= 1 */
    int kx, ky;                /* ROI width (fastest) and height, >= 1 */
    int64_t pitch_row;         /* complex64 elements between rows of a frame (>= roi_x0 + kx) */
    int64_t pitch_frame;       /* complex64 elements between frames */
    int64_t pitch_probe;       /* complex64 elements between probes */
    int roi_x0, roi_y0;        /* crop origin inside each pushed frame */
    int T;                     /* frames in the segment (needed up front for the window) */
    double dt_fs;              /* frame interval in fs (> 0) */
    int n_omega;               /* number of energy bins Nw >= 1 */
    const double *E_meV;       /* host array of Nw energies in meV (ignored when fft_bins) */
    int fft_bins;              /* != 0: E_j = j h / (T dt), j < Nw, exact integer phase */
    int window;                /* tacaw_window */
    double window_param;       /* GAUSS sigma (frames), TUKEY alpha, KAISER beta, CHEBWIN dB */
    int subtract_mean;         /* != 0: remove the segment's time mean mu[k] */
    double bose_T_K;           /* > 0: multiply I by B(E) at this temperature; 0: B = 1 */
    int n_detectors;           /* D >= 0 */
    const tacaw_detector *detectors; /* host array of D detectors */
    /* Welch averaging (Sec. II.B): welch_segments N > 1 splits the pushed frames into N
     * segments of T frames starting welch_stride frames apart (stride = L // nu for the
     * overlap nu; 0 means T), each a segment of the definition above (its own mean, window and
     * phase origin), and the outputs are the averages I = (1/N) sum_n I_n, S likewise.  The
     * stream then takes (N - 1) * stride + T frames; each frame feeds every segment covering
     * it (up to ceil(T / stride) at once, each with its own staging).  0 or 1: one segment.  */
    int welch_segments;
    int welch_stride;
    /* Frames dropped at the start of the stream before its first segment (the trajectory's
     * initial, unequilibrated part; App. configuration `trajectory_chunks_skip_init`, read as a
     * frame count).  The stream then takes skip_init + (N - 1) * stride + T frames; the skipped
     * ones are never read.  >= 0. */
    int skip_init;
} tacaw_stream_desc;

typedef struct {
    int n_streams;                     /* >= 1 */
    const tacaw_stream_desc *streams;  /* host array */
    int precision;                     /* tacaw_precision */
    int accum;                         /* tacaw_accum */
    int64_t hbm_budget_bytes;          /* device bytes the plan may hold; 0: 90% of free memory */
    int k_stage;                       /* frames staged per flush (multiple of 8); 0: from budget */
    /* Tile autotuner of the split path (staged operands).  NULL: tiles from the built-in
     * cost rule.  Non-NULL: at plan creation every stream shape times its candidate tile
     * widths (energies per tile) on scratch operands and keeps the fastest predicted one;
     * "" keeps nothing, a file path reads and appends a text cache keyed by GPU and shape, so
     * later plans of the same shapes skip the timing.  A fixed tc_omega_tile is honoured. */
    const char *tune_cache_path;
    /* Tensor-core tiling (split path); 0 selects automatically.
     *   tc_omega_tile     complex energies per tile (multiple of 8; at most 112 on staged
     *                     operands, 80 in place)
     *   tc_block_frames   frames per staged operand row: 8, 16 or 32 (32-, 64- or 128-byte rows);
     *                     k_stage must be a multiple of it                                    */
    int tc_omega_tile;
    int tc_block_frames;
    /* != 0 (split-BF16 only): pushed buffers are read in place by the contraction instead of
     * being converted into a staging area at push time.  Each pushed buffer must then stay
     * valid and unchanged until the flush that covers its frames has completed on the stream:
     * with the default K_stage (the whole segment) that is until tacaw_finalize returns.
     * Every stream must keep each 128-row tile contiguous in a frame (kx a multiple of 128, or
     * unpadded rows with roi_x0 = 0 and probes that are whole tiles or adjacent), with even
     * sizes, row offsets and pitches, 32-frame blocks, and 16-byte aligned pushed buffers;
     * other layouts are refused with TACAW_ERR_UNSUPPORTED at plan creation.              */
    int frames_in_place;
    /* Split path: the tensor core's FP32 accumulation truncates each step against the running
     * sum, so the hi*hi products are accumulated in chunks of tc_drain_frames frames (multiple of
     * 8; 0: 512) that the epilogue warps drain into FP32 registers (round to nearest) while the
     * tensor core goes on; hi*lo + lo*hi (~2^-8 of the magnitude) keep one accumulator for the
     * whole flush.                                                                         */
    int tc_drain_frames;
    /* Persistent contraction grids (staged and in-place tensor-core kernels) take at most this
     * many CTAs, one per SM (0: every SM).  SMs left free run other work beside the
     * contraction, e.g. the conversions of another plan's segment pushed on another stream. */
    int tc_max_ctas;
    /* TACAW_PREC_SPLIT_FP16 only: power of two multiplying psi - mu_hat before the fp16 split,
     * in [2^-60, 2^60]; 0 selects 2^12, which suits exit waves of unit norm (|psi| <= 1, so
     * |psi - mu_hat| <= 2 becomes <= 8192, nearly eight times inside the fp16 range, while
     * residual pieces of components down to ~1e-4 stay in fp16's normal range).  Scale data
     * with larger components down (e.g. 2^12 / max|psi|).  Ignored by the other precisions. */
    double fp16_scale;
} tacaw_plan_desc;

typedef struct tacaw_plan_s *tacaw_plan_t;

typedef struct {
    int64_t device_bytes;      /* bytes the plan holds on the device */
    int k_stage;               /* frames per flush */
    int n_streams;
    int precision;
    int64_t I_elems;           /* total floats of d_I (sum over streams of P*Nw*ky*kx) */
    int64_t S_elems;           /* total floats of d_S (sum over streams of P*D*Nw) */
    int64_t flushes;           /* flushes run since the plan was created */
    int omega_tile;            /* complex energies per tensor-core tile (split path) */
    int stages;                /* shared-memory pipeline stages (split path) */
    int64_t kernel_launches;   /* kernels launched by push/finalize/backward since creation */
    int tc_block_frames;       /* frames per staged operand row (split path) */
    int frames_in_place;       /* pushed frames are read in place by the contraction */
    int tc_drain_frames;       /* frames per drained hi*hi accumulator chunk (split path) */
    int tuned_streams;         /* streams whose tile the autotuner picked */
    int tune_candidates;       /* candidate tiles timed at creation (0: none, or all cached) */
    double tune_ms;            /* host time spent in the autotuner at creation */
    int accum;                 /* tacaw_accum in use (TACAW_ACC_AUTO resolved at creation) */
    int64_t flush_launches;    /* contraction launches since creation (one grouped launch over
                                  several streams counts once) */
    int64_t aperture_pixels;   /* first stream: ROI pixels inside any detector (the rows the
                                  adjoint recomputes Psi on) */
} tacaw_plan_info;

/* Creates a plan: validates the descriptor, sizes and allocates device memory
 * (staging of K_stage frames per stream, FP64 mean sums, window x twiddle tables,
 * Psi accumulators when a segment needs several flushes), and builds the twiddle
 * tables on the GPU (phase reduced in FP64).  Synchronous.  *out is written on success. */
tacaw_status tacaw_plan_create(const tacaw_plan_desc *desc, tacaw_plan_t *out);

/* Sec. II.B, processing of a batch: the exit waves of a trajectory chunk arrive frame by
 * frame; here they are folded into the segment's transform as they arrive (streaming form
 * of the chunk FFT of Eq. 1's phi_MD).
 * Pushes n_frames frames of stream stream_id (layout: tacaw_stream_desc).  The library
 * reads them, removes the provisional mean (the mean of the first frames, at most 32, of the
 * segment's first push),
 * splits/converts them into its staging area and, when K_stage frames are staged and the
 * segment is not complete, runs a flush (the contraction of the staged frames into Psi).
 * d_frames may be reused once the work enqueued on `stream` has completed.
 * d_frames is device (or managed) memory, or -- staged plans only -- pinned host memory
 * (cudaHostAlloc, or cudaHostRegister'ed and mapped at the same address): the push kernels
 * then read the frames straight from host memory over the host link (NVLink-C2C on Grace
 * systems), with no separate host-to-device copy.  Outside stream capture the address is
 * checked with cudaPointerGetAttributes; pageable host memory and unknown addresses are
 * refused (INVALID_ARG) before any work is enqueued.
 * Errors: OVERFLOW if the segment would exceed T frames (nothing is pushed), STATE after
 * finalize without reset, INVALID_ARG for n_frames < 1 or frames the device cannot read. */
tacaw_status tacaw_push_frames(tacaw_plan_t plan, int stream_id, const void *d_frames,
                               int n_frames, void *stream);

/* Sec. III.C / Sec. IV, supercell partitions of uneven size streamed side by side: one push
 * of each of n distinct streams, with the same result as n calls of tacaw_push_frames
 * (stream_ids[i], d_frames[i], n_frames[i]) on `stream`.  Pushes on the staged split path
 * that fit their stream's staging ring, with n_frames and the ring position multiples of 4,
 * are converted by one kernel launch over all of them (groups of up to 16); the others run
 * as single pushes.  A ring that fills defers its flush to the next push of any of these
 * streams, where the due flushes go out as one grouped launch.
 * stream_ids, d_frames, n_frames: host arrays of n entries (n >= 1).
 * Errors: every entry is checked as tacaw_push_frames checks it, and a stream_id that
 * appears twice is INVALID_ARG, all before any work is enqueued; a CUDA error poisons the
 * plan.                                                                                   */
tacaw_status tacaw_push_frames_group(tacaw_plan_t plan, int n, const int *stream_ids,
                                     const void *const *d_frames, const int *n_frames, void *stream);

/* Eq. 1 (I = B(E) |phi_MD|^2) and the DetectorSet sum over apertures (Sec. II.B).
 * Completes the segment of every stream: flushes what is staged, applies the exact
 * mean correction Psi -= (mu - mu_hat) W(E_j), W the window's transform, forms I and
 * the detector spectra.  Outputs (caller-owned device memory, streams concatenated in
 * order; see tacaw_output_offsets):
 *   d_I   float32 [s][p][j][ky][kx]   (may be NULL)
 *   d_S   float32 [s][p][d][j]        (may be NULL)
 *   d_Psi complex64 [s][p][j][ky][kx] (may be NULL)
 * Spectra are summed in a fixed order (deterministic).  d_S requires d_I.  Waits for the
 * work on `stream`.  Outputs may be device, managed or pinned host memory; outside stream
 * capture any other address is refused (INVALID_ARG) before work is enqueued.
 * Errors: STATE unless every stream has received exactly T frames.
 * The last flush of every stream on the split path goes out as one tensor-core launch over
 * all streams (supercell partitions of uneven size; groups of up to 16 streams), its tiles
 * ordered longest first.                                                                */
tacaw_status tacaw_finalize(tacaw_plan_t plan, float *d_I, float *d_S, void *d_Psi, void *stream);

/* tacaw_finalize without the wait: enqueues the same work and returns.  With
 * tacaw_reset and tacaw_push_frames (which never wait) a whole segment can then be
 * captured into a CUDA graph on `stream` and replayed; a replay reads the frame
 * addresses given at capture time.  The device error flag is read by tacaw_check_errors. */
tacaw_status tacaw_finalize_async(tacaw_plan_t plan, float *d_I, float *d_S, void *d_Psi, void *stream);

/* Waits for the work on `stream` and reads the device error flag: TACAW_ERR_TIMEOUT if a
 * bounded device wait ran out, TACAW_ERR_OVERFLOW if a split-FP16 push met a value beyond
 * the fp16 range at the plan's fp16_scale; either poisons the plan.  tacaw_finalize and
 * tacaw_backward read the same flag when they wait.                                      */
tacaw_status tacaw_check_errors(tacaw_plan_t plan, void *stream);

/* Element offsets of stream stream_id's block inside d_I / d_Psi and d_S.              */
tacaw_status tacaw_output_offsets(tacaw_plan_t plan, int stream_id, int64_t *I_offset,
                                  int64_t *S_offset);

/* Adjoint of the path above (no counterpart in the paper, whose spectra are not
 * differentiated): the chain rule through Eq. 1, the windowed transform and the detector sum.
 * Gradient of L = sum_{p,d,j} dL_dS[p][d][j] * S[p][d][j] with respect to the frames of one
 * stream's segment, in PyTorch's convention for real losses of complex inputs:
 *   grad = dL/dRe(psi) + i dL/dIm(psi) = 2 dL/dconj(psi)
 *   g[t,k] = 2 ( w_t A[t,k] - (1/T) sum_t' w_t' A[t',k] ),  A[t,k] = sum_j e^{+i theta_jt} G[k,j],
 *   G[k,j] = B(E_j) sum_d dL_dS[d,j] M_d(k) Psi[k,j]  (mean term only with subtract_mean).
 * d_frames holds the whole segment (t = 0..T-1) in the pushed layout of the stream
 * descriptor; d_grad (complex64) has the same layout: every ROI element is written (zero
 * outside the apertures), elements outside the ROI are not touched.  Psi is recomputed
 * from the frames, not stored.  Independent of the push/finalize state of the plan.
 * Streams with skip_init or Welch averaging: d_frames / d_grad hold the whole push sequence
 * (skip_init + (N - 1) * stride + T frames); S is the segments' average, so the gradient is
 * (1/N) sum_n g_n with segment n's g_n placed at its frames (added where segments overlap)
 * and zero on the skipped frames.
 * d_dL_dS: float32 [p][d][j] on the device.  d_frames, d_grad and d_dL_dS may be device,
 * managed or pinned host memory; outside stream capture any other address is refused
 * (INVALID_ARG) before work is enqueued.  Waits for the work on `stream`.
 * Both contractions of the adjoint (Psi on the aperture pixels, then the projection back onto
 * the frames) run on the tensor cores in split BF16 by default (tacaw_set_adjoint_precision).
 * The first call that needs it allocates the plan's adjoint scratch, kept until tacaw_destroy
 * (TACAW_ERR_OOM if that fails), for R = P x (aperture pixels) rows: tensor cores
 * R x (8 T' + 8 N' + 8 n_omega + 8 T + max(T', N') / 4 + 16) bytes (T', N': T and n_omega
 * rounded up to 32), plus, per stream, its tables once (about 16 T' N' bytes); FP32 CUDA
 * cores R x (n_omega + 2) x 8 bytes.  The tensor-core adjoint runs its zero fill and its
 * contractions on two streams of the plan, forked from and joined back to `stream`.       */
tacaw_status tacaw_backward(tacaw_plan_t plan, int stream_id, const float *d_dL_dS,
                            const void *d_frames, void *d_grad, void *stream);

/* Arithmetic of tacaw_backward's two contractions (no counterpart in the paper):
 * TACAW_PREC_SPLIT_BF16 (the default, for every plan precision): tcgen05 tensor cores,
 * operands split into bf16 hi + lo pieces, three products, FP32 accumulation;
 * TACAW_PREC_FP32: FP32 CUDA cores.  Anything else is INVALID_ARG.  Applies to later calls. */
tacaw_status tacaw_set_adjoint_precision(tacaw_plan_t plan, int precision);

/* Pipelined segments (no counterpart in the paper; Sec. II.B processes batch after batch).
 * With enable != 0, a finalized segment's contraction is not launched by tacaw_finalize_async:
 * it is deferred, and the next segment's tacaw_finalize_async launches it together with the
 * conversion of that next segment's pushes, which two extra warps of the same launch do while
 * its tensor cores run (the pushes of a segment that follows a deferred one only record their
 * frame addresses; the frames must stay valid until that launch has run).  Each segment stages
 * into one of two staging areas in turn: enabling allocates the second (TACAW_ERR_OOM if it
 * does not fit).  tacaw_drain launches a deferred contraction on its own; tacaw_finalize (the
 * waiting form) does so before it waits.  Results of a segment are complete once its deferred
 * contraction has run.  All calls of the plan go to one CUDA stream.
 * Requirements (else TACAW_ERR_UNSUPPORTED): one stream without Welch averaging, the split-BF16
 * staged path (not in place) with 32-frame blocks, T a multiple of 32 and K_stage >= T.
 * Enable between segments (STATE otherwise); disabling while a contraction is deferred is STATE. */
tacaw_status tacaw_set_pipelined_segments(tacaw_plan_t plan, int enable);

/* Launches a deferred contraction (pipelined segments), on `stream`; no-op without one.
 * STATE while the current segment's pushes wait for it (finalize that segment first).       */
tacaw_status tacaw_drain(tacaw_plan_t plan, void *stream);

/* Starts a new segment on every stream (e.g. the next probe batch or trajectory chunk):
 * clears frame counters and mean sums.  Enqueued on `stream`.                           */
tacaw_status tacaw_reset(tacaw_plan_t plan, void *stream);

/* Checkpoint and resume of a segment in progress (no counterpart in the paper, whose runs
 * resume by recomputing every batch not marked finished: Sec. II.B, batch dispatching).  The
 * accumulation is a sum over the pushed frames, so between two pushes a plan's progress is a
 * few buffers, and a plan created from the same descriptor that loads them continues where the
 * saving plan stopped: the same later pushes give bit-identical results.
 * tacaw_state_size: bytes of a checkpoint of the plan as it is now (after the pushes enqueued
 *   so far): a 48-byte header, 48 bytes per internal stream (Welch lanes count one each) and 8
 *   per stream, then the device sections.  Per internal stream: the provisional mean (8 bytes a
 *   ROI row) and FP64 residual sums (16 a row); the staged frames not yet contracted (whole
 *   blocks of the staging layout: 8 bytes a row and frame); once a flush has written them, the
 *   Psi accumulators of the Nw energies (8 bytes a row and energy for FP32 accumulators, 16 for
 *   compensated FP32 or FP64).  Per Welch-averaged stream its running average of I (4 bytes an
 *   element).
 * tacaw_save_state: writes the checkpoint to h_state (host memory, pageable or pinned, of at
 *   least tacaw_state_size bytes; INVALID_ARG if smaller or device memory).  The copies run on
 *   `stream` after the plan's earlier work there; the call returns when they are done and
 *   reads the device error flag like tacaw_check_errors.
 * tacaw_restore_state: loads a checkpoint into a plan created from the same descriptor
 *   (precision, accumulators, K_stage, block frames, ROI, energies, window, time step, mean
 *   subtraction and Welch segmentation must give the same layout; energy tiles and other
 *   tuning may differ).  It replaces the plan's segment in progress, finalized or not; the
 *   copies run on `stream` and the call returns when they are done.  INVALID_ARG, with the plan
 *   unchanged, for bytes that are not a checkpoint, are truncated or corrupted, or were saved
 *   by another configuration.
 * STATE for tacaw_state_size and tacaw_save_state: a finalized segment (nothing to resume), a
 *   deferred contraction (pipelined segments: tacaw_drain first, also before a restore), or,
 *   with frames_in_place, pushed frames not yet contracted (the plan holds only their
 *   addresses: checkpoint where the pushes so far fill whole K_stage rings).
 * None of the three can be captured into a CUDA graph (they wait on the host).            */
tacaw_status tacaw_state_size(tacaw_plan_t plan, int64_t *bytes);
tacaw_status tacaw_save_state(tacaw_plan_t plan, void *h_state, int64_t bytes, void *stream);
tacaw_status tacaw_restore_state(tacaw_plan_t plan, const void *h_state, int64_t bytes, void *stream);

/* Fills *info.                                                                          */
tacaw_status tacaw_plan_get_info(tacaw_plan_t plan, tacaw_plan_info *info);

/* Bounded device waits.  Every wait of the tensor-core contraction kernels on a pipeline event
 * (operands landed, a stage or an accumulator freed) gives up after limit_ns nanoseconds of
 * the GPU's global timer; the launch then stops early (its copies in flight are waited for and
 * its tensor memory freed, under the default limit), the error word is set, and the next
 * waiting call (tacaw_finalize, tacaw_check_errors, tacaw_backward) returns TACAW_ERR_TIMEOUT
 * and poisons the plan.  0 restores the default of 4 s; other values are raised to at least
 * 1000 ns.  A limit shorter than a tile's work (tens of microseconds) makes a wait run out on
 * purpose, which is how the timeout path is tested without a fault.  Applies to later launches. */
tacaw_status tacaw_set_wait_limit_ns(tacaw_plan_t plan, uint64_t limit_ns);

/* Kernel timing: when enable != 0, CUDA events are recorded around every contraction
 * (flush) launch on the launching stream; tacaw_kernel_time_ms returns the summed
 * milliseconds and the launch count since the last call with reset != 0.  Reading the
 * times waits for the recorded events.  enable >= 2 also records, for every CTA of each
 * tensor-core flush, eight 64-bit words: globaltimer stamps (ns) at entry, set-up done,
 * first operands landed, last MMA issued, accumulators complete, epilogue done, exit, and
 * the SM id; tacaw_flush_trace copies the last flush's words (n_ctas x 8, CTA-major) to
 * host_out (at most max_ctas CTAs) and reports the CTA count.  The drained (persistent)
 * form writes one row per launched CTA (rows of tiles it did not launch stay zero): entry,
 * set-up done, first operands landed, last MMA issued, tiles processed, accumulator chunks
 * started, exit, SM id.                                                                   */
tacaw_status tacaw_set_timing(tacaw_plan_t plan, int enable);
tacaw_status tacaw_kernel_time_ms(tacaw_plan_t plan, double *flush_ms, int64_t *flush_launches,
                                  int reset);
tacaw_status tacaw_flush_trace(tacaw_plan_t plan, unsigned long long *host_out, int64_t max_ctas,
                               int64_t *n_ctas);

/* Detector spectra S[p][d][j] = sum_k M_d(k) I[p][j][k] from a caller-owned intensity array
 * d_I (float32 [p][j][ky][kx], the layout tacaw_finalize writes) without a plan and without
 * allocating device memory.  The paper has no counterpart of this entry point.  It is for
 * callers that may not allocate device memory: code inside a framework that owns the whole
 * device budget, real-time loops where cudaMalloc/cudaFree would synchronise the device,
 * hosts that only hand over raw device pointers.
 * Apertures follow tacaw_detector (MASK weights are read back from the device during the
 * call, after the caller's earlier work on `stream`).  Their (pixel, weight) lists go into one
 * fixed device array that the library holds on every device that loads it, until the process
 * exits: at most 2^20 pixel entries summed over all detectors and at most 1024 detectors; a
 * larger request returns TACAW_ERR_INVALID_ARG before any device work.  The first call on a
 * device (and the first after its context was made again, e.g. after cudaDeviceReset) looks up
 * that array's address.  Every call reuses the same array: calls whose work overlaps on the GPU
 * (other streams or threads) race, so serialise them.  The lists are copied from host memory on
 * `stream`, so the call is refused (INVALID_ARG) while `stream` is capturing a graph.  d_I, d_S
 * and mask weights must be device, managed or mapped pinned host memory (INVALID_ARG otherwise,
 * before any work is enqueued); kx * ky must stay below 2^31.
 * d_S: float32 [p][d][j].  Enqueued on `stream`; returns without waiting for the kernel.  */
tacaw_status tacaw_detector_spectra_noalloc(const float *d_I, int n_probes, int n_omega, int kx, int ky,
                                            const tacaw_detector *detectors, int n_detectors, float *d_S,
                                            void *stream);

/* Frees every device allocation of the plan.  Accepts NULL.                             */
tacaw_status tacaw_destroy(tacaw_plan_t plan);

/* Message for the calling thread's last non-OK status ("" if none).                     */
const char *tacaw_last_error(void);

/* Log sink.  The library reports every error it returns (the message tacaw_last_error
 * gives, level TACAW_LOG_ERROR) and, at TACAW_LOG_INFO, the configuration each successful
 * tacaw_plan_create chose (precision, K_stage, accumulators, tiling, device bytes).  The
 * callback runs on the thread that made the call, synchronously, and must not block for
 * long; it may call tacaw_set_log_callback.  One sink per process; NULL removes it.  The
 * message is valid during the callback only.                                            */
typedef enum { TACAW_LOG_ERROR = 0, TACAW_LOG_INFO = 1 } tacaw_log_level;
typedef void (*tacaw_log_fn)(int level, const char *message, void *user);
tacaw_status tacaw_set_log_callback(tacaw_log_fn fn, void *user);

/* Library version string.                                                               */
const char *tacaw_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TACAW_H_ */
