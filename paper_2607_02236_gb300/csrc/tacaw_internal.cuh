// Internal declarations shared by the translation units of libtacaw.so.
//
// Data layout in HBM (per stream; M = P*ky*kx rows, one row per (probe, ROI pixel),
// M_pad = M rounded up to 128; Nw_pad = n_wt * wt energies):
//   staging, split path   A_hi, A_lo  bf16 [kb][M_pad][2*bf] kb = staged frame / bf (bf = 8, 16
//                         or 32 frames per block: 32-, 64- or 128-byte rows);
//                         element 2*(f%bf)+0 = Re(psi - mu_hat), +1 = Im(...); the split-FP16
//                         path stores fp16 pieces of 2^e (psi - mu_hat) in the same layout
//   staging, FP32 path    A32        float2 [K_stage][M_pad]
//   twiddles, split path  B_hi, B_lo  bf16 [kbT][2*Nw_pad][2*bf] kbT = t / bf; rows 2j, 2j+1
//                         hold the real embedding of w_t exp(-i theta_jt) so that
//                         [Re psi, Im psi] . rows gives [Re Psi_j, Im Psi_j]
//   twiddles, FP32 path   B32        float2 [T_pad][Nw_pad]
//   accumulators          [Nw_pad][M_pad] (float2 sum + float2 compensation, or double2)
//   outputs               I float [p][j][ky][kx], Psi float2 [p][j][ky][kx], S float [p][d][j]
#pragma once
#include <vector>

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace tacaw {

constexpr double kPlanck_meV_ps = 4.135667696;
constexpr int kMTile = 128;          // rows per tensor-core tile (TMEM lanes)

enum FlushMode : int { FLUSH_STORE = 0, FLUSH_ADD = 1, FLUSH_FINAL = 2 };

// Per-CTA trace of the tensor-core contraction (globaltimer, ns):
//   0 entry  1 set-up done  2 first operands landed  3 last MMA issued
//   4 accumulators complete (epilogue start)  5 epilogue done  6 exit  7 SM id
constexpr int kTraceWords = 8;

// device error bits (OR-ed into the plan's error word)
enum : uint32_t {
    DEVERR_TIMEOUT_FULL = 1u,
    DEVERR_TIMEOUT_EMPTY = 2u,
    DEVERR_TIMEOUT_TMEM = 4u,
    DEVERR_TIMEOUT_DRAIN = 8u,
    DEVERR_FP16_RANGE = 16u,   // split-FP16 conversion: a scaled value beyond the fp16 range
};

struct FrameGeom {
    const float2 *base;        // pushed buffer
    int64_t pitch_row, pitch_frame, pitch_probe;
    int roi_x0, roi_y0;
    int kx, ky;
    int64_t npix;              // kx*ky
    int64_t M;                 // P*npix
};

// One push of one stream in a grouped split conversion (launch_convert_split_group).
struct ConvEntry {
    FrameGeom g;
    int n, s0;                 // frames pushed, first ring slot
    int64_t M_pad;
    const float2 *mu_hat;
    double2 *sum_res;
    __nv_bfloat16 *A_hi, *A_lo;
    int64_t cta_begin;         // set by the launcher
};
constexpr int kConvGroupMax = 16;
struct ConvGroup {
    ConvEntry e[kConvGroupMax];
    int n;
};

// Per-element epilogue inputs (shared by the tensor-core and the FP32 contraction).
struct EpiArgs {
    int64_t M, M_pad, npix;
    int Nw;
    int mode;                  // FlushMode
    int has_prev;              // FINAL: accumulators hold earlier flushes
    int accum;                 // 0 compensated FP32, 1 FP64
    float2 *acc_s;             // compensated FP32: sums      [Nw_pad][M_pad]
    float2 *acc_c;             // compensated FP32: compensation
    double2 *acc_d;            // FP64 accumulators
    float *I_out;              // may be null
    float2 *Psi_out;           // may be null
    const float2 *dmu;         // [M] mean residual mu - mu_hat (null: none)
    const float2 *Wc;          // [Nw] window transform W(E_j) (FP64-derived)
    const float *bose;         // [Nw]
    float out_scale;           // FINAL: I = out_scale * B(E) |Psi|^2 (Welch: 1/N per segment)
    int out_add;               // FINAL: add into I_out instead of storing (Welch segments)
    float psi_scale;           // FINAL: Psi_out = psi_scale * Psi (split FP16: the accumulators hold
                               // 2^e Psi, dmu is 2^e (mu - mu_hat), out_scale carries 2^-2e)
};

struct RowCtx {
    int64_t m;
    int64_t out_base;          // p*Nw*npix + pix
    float2 dmu;
    bool valid;
};

__device__ __forceinline__ RowCtx make_row(const EpiArgs &a, int64_t m) {
    RowCtx r;
    r.m = m;
    r.valid = m < a.M;
    int64_t p = r.valid ? m / a.npix : 0;
    int64_t pix = m - p * a.npix;
    r.out_base = p * (int64_t)a.Nw * a.npix + pix;
    r.dmu = (r.valid && a.dmu) ? a.dmu[m] : make_float2(0.f, 0.f);
    return r;
}

// Applies one flush result (re, im) for row r, energy j < Nw, given W(E_j) and B(E_j).
__device__ __forceinline__ void epi_element_wb(const EpiArgs &a, const RowCtx &r, int j, float re, float im,
                                               float2 W, float bj) {
    const size_t ai = (size_t)j * (size_t)a.M_pad + (size_t)r.m;
    if (a.mode == FLUSH_STORE) {
        if (a.accum) {
            a.acc_d[ai] = make_double2(re, im);
        } else {
            a.acc_s[ai] = make_float2(re, im);
            if (a.acc_c) a.acc_c[ai] = make_float2(0.f, 0.f);
        }
        return;
    }
    if (a.mode == FLUSH_ADD) {
        if (a.accum) {
            double2 s = a.acc_d[ai];
            s.x += re;
            s.y += im;
            a.acc_d[ai] = s;
        } else if (a.acc_c) {
            // Kahan (compensated) summation per component
            float2 s = a.acc_s[ai], c = a.acc_c[ai];
            float yr = re - c.x, yi = im - c.y;
            float tr = s.x + yr, ti = s.y + yi;
            c.x = (tr - s.x) - yr;
            c.y = (ti - s.y) - yi;
            a.acc_s[ai] = make_float2(tr, ti);
            a.acc_c[ai] = c;
        } else {
            // plain FP32 sums (one rounding per flush)
            const float2 s = a.acc_s[ai];
            a.acc_s[ai] = make_float2(s.x + re, s.y + im);
        }
        return;
    }
    // FLUSH_FINAL
    float pr, pi;
    if (a.has_prev) {
        if (a.accum) {
            double2 s = a.acc_d[ai];
            pr = (float)(s.x + (double)re);
            pi = (float)(s.y + (double)im);
        } else {
            const float2 s = a.acc_s[ai], c = a.acc_c ? a.acc_c[ai] : make_float2(0.f, 0.f);
            pr = s.x + (re - c.x);
            pi = s.y + (im - c.y);
        }
    } else {
        pr = re;
        pi = im;
    }
    // exact mean correction: Psi -= (mu - mu_hat) * W(E_j)
    pr -= r.dmu.x * W.x - r.dmu.y * W.y;
    pi -= r.dmu.x * W.y + r.dmu.y * W.x;
    const int64_t o = r.out_base + (int64_t)j * a.npix;
    if (a.I_out) {
        const float v = (pr * pr + pi * pi) * bj * a.out_scale;
        a.I_out[o] = a.out_add ? a.I_out[o] + v : v;
    }
    if (a.Psi_out) a.Psi_out[o] = make_float2(pr * a.psi_scale, pi * a.psi_scale);
}

__device__ __forceinline__ void epi_element(const EpiArgs &a, const RowCtx &r, int j, float re, float im) {
    epi_element_wb(a, r, j, re, im, __ldg(a.Wc + j), __ldg(a.bose + j));
}

// The same update with the flush mode fixed at compile time, so that an unrolled loop over
// many energies carries only one path (keeps the loop body small).
enum EpiKind : int {
    EPI_FINAL = 0,          // last flush, no earlier flushes
    EPI_FINAL_KAHAN = 1,    // last flush on top of compensated FP32 accumulators
    EPI_FINAL_FP64 = 2,     // last flush on top of FP64 accumulators
    EPI_STORE_KAHAN = 3,
    EPI_STORE_FP64 = 4,
    EPI_ADD_KAHAN = 5,
    EPI_ADD_FP64 = 6,
};

__host__ __device__ inline int epi_kind(const EpiArgs &a) {
    if (a.mode == FLUSH_STORE) return a.accum ? EPI_STORE_FP64 : EPI_STORE_KAHAN;
    if (a.mode == FLUSH_ADD) return a.accum ? EPI_ADD_FP64 : EPI_ADD_KAHAN;
    if (!a.has_prev) return EPI_FINAL;
    return a.accum ? EPI_FINAL_FP64 : EPI_FINAL_KAHAN;
}

// Read of an accumulator element that this thread alone reads once and then writes in the
// launch: written as an asm statement without a memory clobber, so the compiler may issue it
// ahead of the stores to the other elements (the store that follows it depends on its value).
__device__ __forceinline__ float2 ld_own(const float2 *p) {
    float2 v;
    asm("ld.global.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ double2 ld_own(const double2 *p) {
    double2 v;
    asm("ld.global.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
    return v;
}

template <int K>
__device__ __forceinline__ void epi_apply(const EpiArgs &a, const RowCtx &r, int j, float re, float im, float2 W,
                                          float bj) {
    const size_t ai = (size_t)j * (size_t)a.M_pad + (size_t)r.m;
    if (K == EPI_STORE_KAHAN) {
        a.acc_s[ai] = make_float2(re, im);
        if (a.acc_c) a.acc_c[ai] = make_float2(0.f, 0.f);
    } else if (K == EPI_STORE_FP64) {
        a.acc_d[ai] = make_double2(re, im);
    } else if (K == EPI_ADD_KAHAN) {
        if (a.acc_c) {
            float2 s = ld_own(a.acc_s + ai), c = ld_own(a.acc_c + ai);
            float yr = re - c.x, yi = im - c.y;
            float tr = s.x + yr, ti = s.y + yi;
            c.x = (tr - s.x) - yr;
            c.y = (ti - s.y) - yi;
            a.acc_s[ai] = make_float2(tr, ti);
            a.acc_c[ai] = c;
        } else {
            const float2 s = ld_own(a.acc_s + ai);   // plain FP32 accumulators
            a.acc_s[ai] = make_float2(s.x + re, s.y + im);
        }
    } else if (K == EPI_ADD_FP64) {
        double2 s = ld_own(a.acc_d + ai);
        s.x += re;
        s.y += im;
        a.acc_d[ai] = s;
    } else {
        // a launch that finalizes a stream writes none of its accumulators, so they are read
        // through the read-only path: those loads may be moved ahead of this loop's stores
        float pr = re, pi = im;
        if (K == EPI_FINAL_KAHAN) {
            const float2 s = __ldg(a.acc_s + ai), c = a.acc_c ? __ldg(a.acc_c + ai) : make_float2(0.f, 0.f);
            pr = s.x + (re - c.x);
            pi = s.y + (im - c.y);
        } else if (K == EPI_FINAL_FP64) {
            const double2 s = __ldg(a.acc_d + ai);
            pr = (float)(s.x + (double)re);
            pi = (float)(s.y + (double)im);
        }
        pr -= r.dmu.x * W.x - r.dmu.y * W.y;
        pi -= r.dmu.x * W.y + r.dmu.y * W.x;
        const int64_t o = r.out_base + (int64_t)j * a.npix;
        if (a.I_out) {
            const float v = (pr * pr + pi * pi) * bj * a.out_scale;
            a.I_out[o] = a.out_add ? a.I_out[o] + v : v;
        }
        if (a.Psi_out) a.Psi_out[o] = make_float2(pr * a.psi_scale, pi * a.psi_scale);
    }
}

// ---------------------------------------------------------------------------------------
// Launchers (each defined in its own translation unit); all enqueue on `st`.
// ---------------------------------------------------------------------------------------
struct TableArgs {
    int T, T_pad, Nw, Nw_pad;
    int window;
    double window_param;
    int fft_bins;
    const double *cj;          // device, cycles per frame per energy (explicit grid)
    int block_frames;          // split-path staging block (8, 16 or 32 frames)
    int swz;                   // split path: rows stored pre-swizzled (see convert_split_kernel)
    const double *win_table;   // table-driven windows (Dolph-Chebyshev): w_t, t < T
};

// f16 != 0: fp16 hi/lo pieces (the split-FP16 path) instead of bf16, same layout
cudaError_t launch_twiddles_split(const TableArgs &t, __nv_bfloat16 *B_hi, __nv_bfloat16 *B_lo, int f16,
                                  cudaStream_t st);
cudaError_t launch_twiddles_fp32(const TableArgs &t, float2 *B32, cudaStream_t st);
cudaError_t launch_window_transform(const TableArgs &t, float2 *Wc, cudaStream_t st);
cudaError_t launch_window_values(const TableArgs &t, float *w, cudaStream_t st);

cudaError_t launch_mean(const FrameGeom &g, int n, float2 *mu_hat, cudaStream_t st);
// f16 != 0: fp16 hi/lo pieces of f16_scale * (psi - mu_hat); a scaled component beyond the
// fp16 range sets DEVERR_FP16_RANGE in *err
cudaError_t launch_convert_split(const FrameGeom &g, int n, int s0, int bf, int64_t M_pad, const float2 *mu_hat,
                                 double2 *sum_res, __nv_bfloat16 *A_hi, __nv_bfloat16 *A_lo, int swz, int f16,
                                 float f16_scale, uint32_t *err, cudaStream_t st);
// the tiled split conversion takes the push (s0, n multiples of 4 frames, blocks of 16 or 32)
bool convert_split_groupable(int bf, int s0, int n);
// one launch over cg.n <= kConvGroupMax pushes of different streams (each groupable; the
// launcher sets cta_begin); plan-wide block size, swizzle and fp16 settings
cudaError_t launch_convert_split_group(ConvGroup &cg, int bf, int swz, int f16, float f16_scale, uint32_t *err,
                                       cudaStream_t st);
cudaError_t launch_convert_fp32(const FrameGeom &g, int n, int s0, int64_t M_pad, const float2 *mu_hat,
                                double2 *sum_res, float2 *A32, cudaStream_t st);
cudaError_t launch_frame_table(const float2 **table, const float2 *base, int64_t pitch_frame, int n, cudaStream_t st);
cudaError_t launch_zero_tail_split(int64_t M_pad, int staged, int bf, __nv_bfloat16 *A_hi, __nv_bfloat16 *A_lo,
                                   int swz, cudaStream_t st);
// dmu = scale * (mu - mu_hat) (scale: the split-FP16 operand scale, else 1)
cudaError_t launch_mean_residual(int64_t M, int T, int subtract_mean, const double2 *sum_res, float2 *dmu,
                                 float scale, cudaStream_t st);

struct SimtArgs {
    EpiArgs e;
    const float2 *A32;         // [K_stage][M_pad]
    const float2 *B32;         // [T_pad][Nw_pad]
    int Nw_pad;
    int n_frames;              // frames in this flush
    int t0;                    // global index of the first frame (row of B32)
};
cudaError_t launch_flush_simt(const SimtArgs &a, cudaStream_t st);

struct TcPlanArgs {
    EpiArgs e;
    int wt, n_wt, N;           // complex energies per tile, tiles, real columns per tile (2*wt)
    int n_kb;                  // staging blocks in this flush
    int kbB0;                  // first global twiddle block
    int bf;                    // frames per staging block (8, 16, 32): rows of 4*bf bytes
    int stages;
    int drain_kb;              // H (the hi*hi accumulator) is drained into FP32 registers every
                               // drain_kb staging blocks (wt <= kDrainMaxOmegaTile); the staged
                               // operands are pre-swizzled and copied as contiguous blocks:
    const void *A_hi, *A_lo, *B_hi, *B_lo;   //   staging and twiddle tables
    int64_t a_rows;            //   rows per staging block of A (M_pad)
    int b_rows;                //   rows per twiddle block of B (2 * Nw_pad)
    int max_ctas;              // persistent grids: at most this many CTAs (0: one per SM)
    int N_last;                // staged form: columns of the last energy tile (<= N, multiple of 16)
    int f16;                   // operands are fp16 pieces (split-FP16 path) instead of bf16
    unsigned long long *trace; // null, or kTraceWords globaltimer stamps per CTA (phase boundaries)
    uint32_t *err;
    uint64_t wait_ns;          // pipeline waits give up after this many ns (0: the default 4 s)
    int *tile_counter;         // staged kernel: device int the launch hands out its tiles from (the
                               // first entry's of a grouped launch is used; zeroed before the launch)
};
// In-place operand A: the contraction reads the pushed frames of this flush directly.
struct TcDirectArgs {
    const float2 *const *frame_ptr;   // [n_frames] device pointers to each staged frame (pushed layout)
    int n_frames;                     // frames in this flush
    int64_t M, npix;
    int kx;
    int64_t pitch_row, pitch_probe;
    int roi_x0, roi_y0;
    const float2 *mu_hat;             // [M] provisional mean
    double2 *sum_res;                 // [M] residual sums of earlier flushes
    int accumulate_sums;              // add this flush's sums to sum_res (non-final flushes)
    int prev_sums;                    // final flush: sum_res holds earlier flushes
    int subtract_mean;
    int T;
};
cudaError_t launch_flush_tc(const TcPlanArgs &a, cudaStream_t st);
// Conversion of the next segment's pushes, done by two extra warps of a staged contraction
// launch while its tensor cores run (pipelined segments): frames t < T of the segment through a
// table of frame pointers, rows m < M_pad (rows >= M staged as zeros), split BF16, 32-frame
// blocks, pre-swizzled; sum_res[m] = sum over the segment of (psi - mu_hat) (written, FP64).
struct TcConvJob {
    const float2 *const *frame_ptr;   // [T] device pointers to each frame (pushed layout)
    int T;                            // frames (a multiple of 32)
    int64_t M, M_pad, npix;
    int kx;
    int64_t pitch_row, pitch_probe;
    int roi_x0, roi_y0;
    const float2 *mu_hat;             // [M] provisional mean
    double2 *sum_res;                 // [M] written
    __nv_bfloat16 *A_hi, *A_lo;       // staging [T/32][M_pad][64]
    int *counter;                     // row tiles handed out (zero at launch)
};
// launch_flush_tc_group with a conversion job for its two extra warps (384 threads a CTA)
cudaError_t launch_flush_tc_group_conv(const TcPlanArgs *args, int n, const TcConvJob &conv, cudaStream_t st);
int64_t tc_grid_ctas(const TcPlanArgs &a);
constexpr int kMaxGroupStreams = 16;
constexpr int kDrainMaxOmegaTile = 112;   // staged form: complex energies per tile at most
constexpr int kInplaceMaxOmegaTile = 80;  // in-place form (worker registers at 168 a thread)
// one persistent launch over the flushes of up to kMaxGroupStreams streams (same block frames)
cudaError_t launch_flush_tc_group(const TcPlanArgs *args, int n, cudaStream_t st);
// persistent in-place drained form (A in tensor memory): tile rows contiguous and 16-byte
// aligned in every frame (host-checked), 32-frame blocks, tiles of at most
// kInplaceMaxOmegaTile energies.  tc_inplace_stages: its A/B stages for an N-column tile (0 if
// it does not fit), the raw frame stages and TMEM columns through the optional pointers.
// frame_map (optional, tc_make_frame_map): the flush's frames evenly spaced from the first
cudaError_t launch_flush_tc_inplace(const TcPlanArgs &a, const TcDirectArgs &d, const void *frame_map,
                                    cudaStream_t st);
bool tc_make_frame_map(void *map_out, const void *first_frame, int64_t pitch_frame, int n_frames, char *errbuf,
                       size_t errlen);
size_t tc_frame_map_size();
int tc_inplace_stages(int N, int bf, int *raw = nullptr, uint32_t *acc_s = nullptr, uint32_t *a_col = nullptr);
int tc_stages_for(int N, int bf);
size_t tc_smem_bytes(int N, int bf, int stages);
int tc_resident_ctas(int N, int bf, int stages);

// Tile autotuner (k_tc_tune.cu): picks the energies per tile for one stream shape.
struct TuneShape {
    int64_t M;                 // rows (probes x ROI pixels)
    int Nw, T, ring;           // energies, frames per segment, frames per flush
    int bf, wt_max;            // block frames, widest tile allowed
    int fixed_wt;              // 0: tuned
    bool multi;                // several streams share the final launch
    int drain_kb;              // staging blocks per drained H chunk
};
struct TuneCand {
    int wt;
    double ms;                 // predicted contraction time of the stream's segment
};
// Fills `table` with one prediction per candidate tile (from the cache when it holds the
// shape; *timed = candidates actually timed).  False with a message on a CUDA error.
bool tc_autotune(const TuneShape &sh, const char *cache_path, uint32_t *d_err, cudaStream_t st,
                 std::vector<TuneCand> *table, int *timed, char *err, size_t errlen);

struct ApertureArgs {
    const float *I;            // [P][Nw][npix]
    float *S;                  // [P][D][Nw]
    int P, D, Nw;
    int64_t npix;
    const int *idx;            // concatenated pixel lists
    const float *wts;          // weights
    const int *off;            // [D+1]
};
cudaError_t launch_aperture(const ApertureArgs &a, cudaStream_t st);

// records the calling thread's message for tacaw_last_error()
void set_last_error(const char *msg);
// TACAW_OK if kernels may read and write ptr (device, managed, or pinned host memory mapped at
// the same address); else TACAW_ERR_INVALID_ARG with a message naming `what`.  Not checked while
// st is capturing a graph.
int check_device_readable(const void *ptr, const char *what, cudaStream_t st);

struct AdjointArgs {
    const float2 *frames;      // pushed layout, whole segment
    int64_t pitch_row, pitch_frame, pitch_probe;
    int roi_x0, roi_y0, kx, ky;
    int P, T, Nw, D;
    int subtract_mean;
    const float *w;            // [T] window
    const float2 *B32;         // [T_pad][Nw_pad] forward twiddles w_t e^{-i theta}
    int Nw_pad;
    const float2 *Wc;          // [Nw]
    const float *bose;         // [Nw]
    const float *dLdS;         // [P][D][Nw]
    const int *mpix;           // pixels inside any aperture (sorted)
    const float *mwts;         // [n_mpix][D] mask weights of those pixels
    int n_mpix;
    float2 *grad;              // same layout as frames (pitches above)
    float2 *scratch;           // [P][n_mpix][Nw] complex (G), plus [P][n_mpix] means
    float scale;               // the gradient is scale * 2 (C - K) ...
    int accumulate;            // ... added to grad (1) or stored (0)
};
cudaError_t launch_adjoint(const AdjointArgs &a, cudaStream_t st);
cudaError_t launch_zero_roi(const AdjointArgs &a, cudaStream_t st);

// Tensor-core adjoint (k_adjoint_tc.cu): both contractions on the staged drained kernel, split
// BF16, over the aperture rows (M = P * n_mpix rows, padded to M_pad).  Tables per stream,
// scratch per plan; every staged row is written in full by each call.
struct AdjTcArgs {
    AdjointArgs a;                          // geometry, loss weights, gradient (scratch unused)
    const __nv_bfloat16 *Bf_hi, *Bf_lo;     // forward twiddles, 32-frame blocks [T_pad/32][2 wt1 n_wt1][64]
    int wt1, n_wt1;                         // energy tiles of the Psi recompute
    const __nv_bfloat16 *Bc_hi, *Bc_lo;     // conj twiddles, 32-energy blocks [E_pad/32][2 wt2 n_wt2][64]
    int wt2, n_wt2;                         // frame tiles of the back-projection
    const float2 *ones;                     // [wt2 n_wt2] (1, 0): the back-projection's "window transform"
    const float *ones_f;                    // [wt2 n_wt2] 1
    const int64_t *pix_off;                 // [n_mpix] element offset of each aperture pixel in a frame
    int64_t M_pad;
    int T_pad, E_pad;                       // frames and energies rounded up to 32
    __nv_bfloat16 *A_hi, *A_lo;             // staged frames of the aperture rows [T_pad/32][M_pad][64]
    __nv_bfloat16 *G_hi, *G_lo;             // staged G [E_pad/32][M_pad][64]
    float2 *part;                           // per-block row sums [max(T_pad, E_pad)/32][M]
    float2 *dmu, *kmean;                    // [M]: mu - psi_0, and K
    float2 *psi;                            // [P][Nw][n_mpix]
    float2 *cg;                             // [P][T][n_mpix]: C - K
    int *counters;                          // two tile counters
    uint32_t *err;
    uint64_t wait_ns;
    cudaEvent_t before_scatter;             // if set: the scatter waits for it (the gradient's zero fill)
};
cudaError_t launch_adjoint_tc(const AdjTcArgs &q, cudaStream_t st);
// kernels one launch_adjoint_tc enqueues (its two contractions included)
int adjtc_launches();
// conj(B[t][j]) = w_t exp(+i theta_jt) split into bf16 hi/lo: rows 2t, 2t+1 (t < t_rows) of
// 32-energy blocks (energies padded to e_pad), pre-swizzled like the forward tables
cudaError_t launch_twiddles_adjoint_split(const TableArgs &t, int t_rows, int e_pad, __nv_bfloat16 *B_hi,
                                          __nv_bfloat16 *B_lo, cudaStream_t st);

}  // namespace tacaw
