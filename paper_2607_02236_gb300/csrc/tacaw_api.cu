// Host implementation of the C ABI declared in include/tacaw.h: plans, pushes, flushes,
// finalize and the plan queries (tacaw_backward.cu holds the adjoint, tacaw_state.cu the
// checkpoints; tacaw_plan.cuh the plan's host-side state they share).
//
// A plan owns, per stream: the staging ring of K_stage frames (converted on push), the
// FP64 sums of the mean residual, the twiddle tables (window x exp(-i theta), built on the
// GPU in FP64), the window transform W(E_j), the Bose factors, compact detector pixel
// lists and, only when the segment needs more than one flush, the Psi accumulators.
// A flush contracts the staged frames with the twiddles of their global frame indices
// (tensor cores or FP32 CUDA cores) and folds the result into the accumulators, or, for
// the segment's last flush, directly into I / Psi with the exact mean correction.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/tacaw.h"
#include "tacaw_internal.cuh"
#include "tacaw_plan.cuh"

using namespace tacaw;

namespace {

thread_local std::string g_last_error;

// process-wide log sink (tacaw_set_log_callback); called outside the lock
std::mutex g_log_mu;
tacaw_log_fn g_log_fn = nullptr;
void *g_log_user = nullptr;

void emit_log(int level, const char *msg) {
    tacaw_log_fn fn;
    void *user;
    {
        std::lock_guard<std::mutex> lk(g_log_mu);
        fn = g_log_fn;
        user = g_log_user;
    }
    if (fn) fn(level, msg, user);
}

}  // namespace

namespace tacaw {
tacaw_status fail(tacaw_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    emit_log(TACAW_LOG_ERROR, buf);
    return st;
}

void set_last_error(const char *msg) {
    g_last_error = msg ? msg : "";
    emit_log(TACAW_LOG_ERROR, g_last_error.c_str());
}
}  // namespace tacaw



namespace {


void free_all(tacaw_plan_s *p) {
    if (p->hp_stream) cudaStreamDestroy(p->hp_stream);
    if (p->hp_in) cudaEventDestroy(p->hp_in);
    if (p->hp_out) cudaEventDestroy(p->hp_out);
    p->hp_stream = nullptr;
    p->hp_in = p->hp_out = nullptr;
    if (p->aux_stream) cudaStreamDestroy(p->aux_stream);
    if (p->adj_stream) cudaStreamDestroy(p->adj_stream);
    if (p->aux_in) cudaEventDestroy(p->aux_in);
    if (p->aux_out) cudaEventDestroy(p->aux_out);
    if (p->adj_out) cudaEventDestroy(p->adj_out);
    p->aux_stream = p->adj_stream = nullptr;
    p->aux_in = p->aux_out = p->adj_out = nullptr;
    if (p->d_trace) cudaFree(p->d_trace);
    p->d_trace = nullptr;
    for (auto &e : p->ev) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    p->ev.clear();
    for (void *q : p->allocs) cudaFree(q);
    p->allocs.clear();
    if (p->adj_scratch) cudaFree(p->adj_scratch);
    p->adj_scratch = nullptr;
    p->adj_scratch_elems = 0;
    if (p->adj_tc) cudaFree(p->adj_tc);
    p->adj_tc = nullptr;
    p->adj_tc_bytes = 0;
}

}  // namespace

namespace tacaw {
tacaw_status cuda_fail(tacaw_plan_s *p, cudaError_t e, const char *what) {
    if (p) p->poisoned = true;
    return fail(TACAW_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}
}  // namespace tacaw

namespace {


tacaw_status validate_stream(const tacaw_stream_desc &d, int i) {
    if (d.n_probes < 1 || d.kx < 1 || d.ky < 1) return fail(TACAW_ERR_INVALID_ARG, "stream %d: P, kx, ky must be >= 1", i);
    if (d.T < 1) return fail(TACAW_ERR_INVALID_ARG, "stream %d: T must be >= 1", i);
    if (!(d.dt_fs > 0.0)) return fail(TACAW_ERR_INVALID_ARG, "stream %d: dt_fs must be > 0", i);
    if (d.n_omega < 1) return fail(TACAW_ERR_INVALID_ARG, "stream %d: n_omega must be >= 1", i);
    if (!d.fft_bins && !d.E_meV) return fail(TACAW_ERR_INVALID_ARG, "stream %d: E_meV is NULL", i);
    if (d.fft_bins && d.n_omega > d.T) return fail(TACAW_ERR_INVALID_ARG, "stream %d: fft_bins needs n_omega <= T", i);
    if (d.window < TACAW_WIN_RECT || d.window > TACAW_WIN_CHEBWIN) return fail(TACAW_ERR_INVALID_ARG, "stream %d: bad window", i);
    if (d.window == TACAW_WIN_KAISER && !(d.window_param >= 0.0 && d.window_param <= 60.0))
        return fail(TACAW_ERR_INVALID_ARG, "stream %d: Kaiser beta must be in [0, 60]", i);
    if (d.window == TACAW_WIN_CHEBWIN && !(d.window_param > 0.0 && d.window_param <= 300.0))
        return fail(TACAW_ERR_INVALID_ARG, "stream %d: Chebyshev attenuation must be in (0, 300] dB", i);
    if (d.roi_x0 < 0 || d.roi_y0 < 0) return fail(TACAW_ERR_INVALID_ARG, "stream %d: negative ROI origin", i);
    if (d.pitch_row < (int64_t)d.roi_x0 + d.kx) return fail(TACAW_ERR_INVALID_ARG, "stream %d: pitch_row < roi_x0 + kx", i);
    if (d.pitch_frame < d.pitch_row * (int64_t)(d.roi_y0 + d.ky) && d.T > 1)
        return fail(TACAW_ERR_INVALID_ARG, "stream %d: pitch_frame smaller than the ROI extent", i);
    if (d.n_probes > 1 && d.pitch_probe < 1) return fail(TACAW_ERR_INVALID_ARG, "stream %d: pitch_probe must be >= 1", i);
    if (d.n_detectors < 0 || (d.n_detectors > 0 && !d.detectors))
        return fail(TACAW_ERR_INVALID_ARG, "stream %d: bad detector array", i);
    if (d.bose_T_K < 0) return fail(TACAW_ERR_INVALID_ARG, "stream %d: bose_T_K must be >= 0", i);
    if (d.welch_segments < 0 || d.welch_stride < 0)
        return fail(TACAW_ERR_INVALID_ARG, "stream %d: welch_segments and welch_stride must be >= 0", i);
    if (d.skip_init < 0) return fail(TACAW_ERR_INVALID_ARG, "stream %d: skip_init must be >= 0", i);
    if ((int64_t)d.skip_init +
            (d.welch_segments > 1 ? (int64_t)(d.welch_segments - 1) * (d.welch_stride ? d.welch_stride : d.T) : 0) +
            d.T >
        (int64_t)INT32_MAX)
        return fail(TACAW_ERR_INVALID_ARG, "stream %d: push sequence longer than 2^31 frames", i);
    for (int k = 0; k < d.n_detectors; ++k) {
        const tacaw_detector &t = d.detectors[k];
        if (t.kind < TACAW_DET_CIRCULAR || t.kind > TACAW_DET_MASK)
            return fail(TACAW_ERR_INVALID_ARG, "stream %d detector %d: bad kind", i, k);
        if (t.kind == TACAW_DET_MASK && !t.d_mask)
            return fail(TACAW_ERR_INVALID_ARG, "stream %d detector %d: mask pointer is NULL", i, k);
    }
    if ((int64_t)d.n_probes * d.kx * d.ky > (int64_t)1 << 31)
        return fail(TACAW_ERR_UNSUPPORTED, "stream %d: more than 2^31 rows", i);
    return TACAW_OK;
}

double bose_factor(double E, double TK) {
    if (TK <= 0.0 || E == 0.0) return 1.0;
    const double kB = 0.08617333262;  // meV/K
    double x = E / (kB * TK);
    return x / (-std::expm1(-x));
}

// Complex energies per tile: at most `cap` (the register sums of the tensor-core kernels; the
// FP32 path pads to 64-wide tiles on its own).  Among multiples of 8 the width with the least
// padded work plus a fixed per-tile cost (operand A is re-read once per energy tile) wins; a
// requested width is clamped.
int least_cost_tile(int n_cols, int wt_max) {
    int best = 8;
    int64_t best_cost = INT64_MAX;
    for (int wt = 8; wt <= wt_max; wt += 8) {
        const int64_t n = (n_cols + wt - 1) / wt;
        const int64_t cost = n * (wt + 24);
        if (cost < best_cost || (cost == best_cost && wt > best)) {
            best_cost = cost;
            best = wt;
        }
    }
    return best;
}

void choose_omega_tile(Stream &s, int requested, int cap) {
    const int wt_max = std::max(8, cap / 8 * 8);
    const int best = requested > 0 ? std::min(requested, wt_max) : least_cost_tile(s.Nw, wt_max);
    s.wt = best;
    s.n_wt = (s.Nw + best - 1) / best;
    s.Nw_pad = s.wt * s.n_wt;
}

// Tile counters a plan keeps for its staged-kernel launches (see tacaw_plan_s::d_counters).
constexpr int kCounterRing = 256;

// Automatic accumulators choose plain FP32 up to this many flushes per segment.
constexpr int kAutoFp32Flushes = 16;

// Staging + accumulator bytes of one stream for a given ring length.
int64_t stream_stage_bytes(const Stream &s, int ring) { return s.M_pad * 8 * (int64_t)ring; }
int64_t stream_acc_bytes(const Stream &s, int accum) {
    return (int64_t)s.Nw_pad * s.M_pad * (accum == TACAW_ACC_FP32 ? 8 : 16);
}

EpiArgs epi_args(tacaw_plan_s *p, const Stream &s, int mode, float *I_out, float2 *Psi_out) {
    EpiArgs e{};
    e.M = s.M;
    e.M_pad = s.M_pad;
    e.npix = s.npix;
    e.Nw = s.Nw;
    e.mode = mode;
    e.has_prev = s.flushes > 0 ? 1 : 0;
    e.accum = p->accum == TACAW_ACC_FP64 ? 1 : 0;   // FP64 accumulators; else FP32 (acc_c: compensation)
    e.acc_s = s.acc_s;
    e.acc_c = s.acc_c;
    e.acc_d = s.acc_d;
    e.dmu = s.dmu;
    e.Wc = s.Wc;
    e.bose = s.bose;
    e.I_out = I_out;
    e.Psi_out = Psi_out;
    // split FP16: the accumulators hold f16_scale * Psi (powers of two: exact rescaling)
    const float inv = 1.f / p->f16_scale;
    e.out_scale = p->f16 ? s.out_scale * inv * inv : s.out_scale;
    e.psi_scale = p->f16 ? inv : 1.f;
    e.out_add = s.out_add;
    return e;
}

// Tensor-core arguments of one flush of the s.staged frames of stream s.
TcPlanArgs tc_args(tacaw_plan_s *p, const Stream &s, const EpiArgs &e) {
    const int n = s.staged;
    TcPlanArgs a{};
    a.e = e;
    a.wt = s.wt;
    a.n_wt = s.n_wt;
    a.N = 2 * s.wt;
    // staged form: the last energy tile computes only the columns that hold energies
    a.N_last = a.N;
    if (!p->in_place) {
        const int last = s.Nw - (s.n_wt - 1) * s.wt;
        a.N_last = std::min(a.N, (2 * last + 15) / 16 * 16);
    }
    a.n_kb = (n + p->bf - 1) / p->bf;
    a.kbB0 = s.stage_start / p->bf;
    a.bf = p->bf;
    a.stages = s.stages;
    a.drain_kb = p->drain_kb;
    a.A_hi = s.A_hi;
    a.A_lo = s.A_lo;
    a.B_hi = s.B_hi;
    a.B_lo = s.B_lo;
    a.a_rows = s.M_pad;
    a.b_rows = 2 * s.Nw_pad;
    a.max_ctas = p->tc_max_ctas;
    a.wait_ns = p->wait_ns;
    a.f16 = p->f16;
    a.err = p->d_err;
    a.trace = nullptr;
    return a;
}

// Per-CTA phase trace of the next flush launch (nc CTAs).
tacaw_status trace_buffer(tacaw_plan_s *p, int64_t nc, unsigned long long **out) {
    *out = nullptr;
    if (!p->trace) return TACAW_OK;
    if (nc > p->trace_cap) {
        if (p->d_trace) cudaFree(p->d_trace);
        p->d_trace = nullptr;
        p->trace_cap = 0;
        CU_CHECK(p, cudaMalloc(&p->d_trace, sizeof(unsigned long long) * kTraceWords * nc), "trace buffer");
        p->trace_cap = nc;
    }
    p->trace_ctas = nc;
    // a persistent launch writes fewer CTAs than tiles: the rest stays zero
    CU_CHECK(p, cudaMemsetAsync(p->d_trace, 0, sizeof(unsigned long long) * kTraceWords * nc, nullptr), "trace reset");
    *out = p->d_trace;
    return TACAW_OK;
}

tacaw_status timing_begin(tacaw_plan_s *p, cudaEvent_t *e0, cudaEvent_t *e1, cudaStream_t st) {
    *e0 = *e1 = nullptr;
    if (!p->timing) return TACAW_OK;
    CU_CHECK(p, cudaEventCreate(e0), "cudaEventCreate");
    CU_CHECK(p, cudaEventCreate(e1), "cudaEventCreate");
    CU_CHECK(p, cudaEventRecord(*e0, st), "cudaEventRecord");
    return TACAW_OK;
}

tacaw_status timing_end(tacaw_plan_s *p, cudaEvent_t e0, cudaEvent_t e1, cudaStream_t st) {
    if (!p->timing) return TACAW_OK;
    CU_CHECK(p, cudaEventRecord(e1, st), "cudaEventRecord");
    p->ev.emplace_back(e0, e1);
    return TACAW_OK;
}

void flush_done(tacaw_plan_s *p, Stream &s) {
    s.flushes++;
    p->flushes_total++;
    s.stage_start += s.staged;
    s.staged = 0;
}

// Address of frame `a` when frames [a, a + n) of the segment are evenly spaced (pitch_frame
// apart) across the pushes that hold them, else null.
const float2 *inplace_first_frame(const Stream &s, int a, int n) {
    const float2 *first = nullptr;
    for (size_t i = 0; i < s.h_pushes.size(); ++i) {
        const int b0 = s.h_pushes[i].first;
        const int b1 = i + 1 < s.h_pushes.size() ? s.h_pushes[i + 1].first : s.pushed;
        if (b1 <= a || b0 >= a + n) continue;
        const float2 *base = s.h_pushes[i].second;
        if (!first) {
            if (b0 > a) return nullptr;
            first = base + (int64_t)(a - b0) * s.d.pitch_frame;
        } else if (base != first + (int64_t)(b0 - a) * s.d.pitch_frame) {
            return nullptr;
        }
    }
    return first;
}

tacaw_status run_flush(tacaw_plan_s *p, Stream &s, int mode, float *I_out, float2 *Psi_out, cudaStream_t st) {
    const int n = s.staged;
    if (n <= 0) return TACAW_OK;
    TraceRange trace_range(p->prec != TACAW_PREC_SPLIT_BF16 ? "contraction (FP32)"
                                                            : (p->in_place ? "contraction (tensor cores, in place)"
                                                                           : "contraction (tensor cores)"));
    if (mode != FLUSH_FINAL && !s.needs_acc) return fail(TACAW_ERR_STATE, "internal: accumulator missing");
    const EpiArgs e = epi_args(p, s, mode, I_out, Psi_out);
    cudaEvent_t e0, e1;
    tacaw_status r = timing_begin(p, &e0, &e1, st);
    if (r != TACAW_OK) return r;
    if (p->prec == TACAW_PREC_SPLIT_BF16 && p->in_place) {
        TcPlanArgs a = tc_args(p, s, e);
        r = trace_buffer(p, (s.M_pad / kMTile) * s.n_wt, &a.trace);
        if (r != TACAW_OK) return r;
        TcDirectArgs d{};
        d.frame_ptr = s.d_frame_ptr + s.stage_start;
        d.n_frames = n;
        d.M = s.M;
        d.npix = s.npix;
        d.kx = s.d.kx;
        d.pitch_row = s.d.pitch_row;
        d.pitch_probe = s.d.pitch_probe;
        d.roi_x0 = s.d.roi_x0;
        d.roi_y0 = s.d.roi_y0;
        d.mu_hat = s.mu_hat;
        d.sum_res = s.sum_res;
        d.accumulate_sums = mode != FLUSH_FINAL ? 1 : 0;
        d.prev_sums = s.flushes > 0 ? 1 : 0;
        d.subtract_mean = s.d.subtract_mean;
        d.T = s.T;
        // evenly spaced frames (one buffer, or pushes that continue each other): tensor map
        alignas(64) unsigned char fmap[128];
        const void *fm = nullptr;
        const float2 *first = inplace_first_frame(s, s.stage_start, n);
        char eb[256];
        if (first && (size_t)tc_frame_map_size() <= sizeof(fmap) && s.d.pitch_frame < (int64_t)1 << 31 &&
            tc_make_frame_map(fmap, first, s.d.pitch_frame, n, eb, sizeof(eb)))
            fm = fmap;
        CU_CHECK(p, launch_flush_tc_inplace(a, d, fm, st), "flush (tensor cores, in place)");
        p->launches++;
        p->flush_launches++;
    } else if (p->prec == TACAW_PREC_SPLIT_BF16) {
        if (n % p->bf) {
            CU_CHECK(p, launch_zero_tail_split(s.M_pad, n, p->bf, s.A_hi, s.A_lo, 1, st), "zero_tail");
            p->launches++;
        }
        TcPlanArgs a = tc_args(p, s, e);
        a.tile_counter = p->d_counters + (p->counter_slot++ % kCounterRing);
        r = trace_buffer(p, tc_grid_ctas(a), &a.trace);
        if (r != TACAW_OK) return r;
        CU_CHECK(p, launch_flush_tc(a, st), "flush (tensor cores)");
        p->launches++;
        p->flush_launches++;
    } else {
        SimtArgs a{};
        a.e = e;
        a.A32 = s.A32;
        a.B32 = s.B32;
        a.Nw_pad = s.Nw_pad;
        a.n_frames = n;
        a.t0 = s.stage_start;
        CU_CHECK(p, launch_flush_simt(a, st), "flush (fp32)");
        p->launches++;
        p->flush_launches++;
    }
    r = timing_end(p, e0, e1, st);
    if (r != TACAW_OK) return r;
    flush_done(p, s);
    return TACAW_OK;
}

// One flush of a staged tensor-core stream inside a grouped launch.
struct FlushReq {
    int s;                     // internal stream
    int mode;                  // FLUSH_STORE / FLUSH_ADD / FLUSH_FINAL
    float *I;                  // FINAL: the stream's block of I (or the Welch average), else null
    float2 *Psi;
};

// Flushes of several staged tensor-core streams as few launches as possible: up to
// kMaxGroupStreams streams share one persistent launch, their tiles ordered by decreasing
// per-tile work so that the longest tiles start first.
tacaw_status flush_grouped(tacaw_plan_s *p, std::vector<FlushReq> req, cudaStream_t st) {
    auto work = [&](const FlushReq &q) {
        const Stream &s = p->s[q.s];
        return (int64_t)((s.staged + p->bf - 1) / p->bf) * (2 * s.wt + 48);
    };
    std::stable_sort(req.begin(), req.end(), [&](const FlushReq &a, const FlushReq &b) { return work(a) > work(b); });
    for (size_t g0 = 0; g0 < req.size(); g0 += kMaxGroupStreams) {
        TraceRange trace_range("contraction (tensor cores, grouped)");
        const size_t g1 = std::min(req.size(), g0 + (size_t)kMaxGroupStreams);
        std::vector<TcPlanArgs> args;
        int64_t nc = 0;
        for (size_t k = g0; k < g1; ++k) {
            Stream &s = p->s[req[k].s];
            if (s.staged % p->bf) {
                CU_CHECK(p, launch_zero_tail_split(s.M_pad, s.staged, p->bf, s.A_hi, s.A_lo, 1, st), "zero_tail");
                p->launches++;
            }
            args.push_back(tc_args(p, s, epi_args(p, s, req[k].mode, req[k].I, req[k].Psi)));
            nc += tc_grid_ctas(args.back());
        }
        unsigned long long *tr = nullptr;
        tacaw_status r = trace_buffer(p, nc, &tr);
        if (r != TACAW_OK) return r;
        for (auto &a : args) a.trace = tr;
        args[0].tile_counter = p->d_counters + (p->counter_slot++ % kCounterRing);
        cudaEvent_t e0, e1;
        r = timing_begin(p, &e0, &e1, st);
        if (r != TACAW_OK) return r;
        CU_CHECK(p, launch_flush_tc_group(args.data(), (int)args.size(), st), "flush (tensor cores, grouped)");
        p->launches++;
        p->flush_launches++;
        r = timing_end(p, e0, e1, st);
        if (r != TACAW_OK) return r;
        for (size_t k = g0; k < g1; ++k) flush_done(p, p->s[req[k].s]);
    }
    return TACAW_OK;
}

// Final flushes of all staged tensor-core single-segment streams (Welch lanes finish their
// segments during the pushes).
tacaw_status final_flush_grouped(tacaw_plan_s *p, float *d_I, float2 *d_Psi, cudaStream_t st) {
    std::vector<FlushReq> req;
    for (int i = 0; i < (int)p->s.size(); ++i) {
        const Stream &s = p->s[i];
        if (s.staged <= 0) continue;
        req.push_back(FlushReq{i, FLUSH_FINAL, d_I ? d_I + s.I_off : nullptr, d_Psi ? d_Psi + s.I_off : nullptr});
    }
    return flush_grouped(p, req, st);
}

// Flushes of staged tensor-core streams are deferred while the caller pushes other streams, so
// that streams whose rings fill in the same round of pushes share one launch (a Welch lane, an
// in-place or an FP32 stream flushes at once).
bool deferrable(const tacaw_plan_s *p, const Stream &s) {
    return p->prec == TACAW_PREC_SPLIT_BF16 && !p->in_place && p->us[s.user].N <= 1;
}

// Runs every deferred flush: those pushed on `st` in one grouped launch there, any other on the
// stream its frames were pushed on.
tacaw_status flush_due(tacaw_plan_s *p, cudaStream_t st) {
    std::vector<FlushReq> req;
    for (int i = 0; i < (int)p->s.size(); ++i) {
        Stream &s = p->s[i];
        if (!s.due) continue;
        s.due = false;
        const int mode = s.flushes == 0 ? FLUSH_STORE : FLUSH_ADD;
        if (s.due_stream == st) {
            req.push_back(FlushReq{i, mode, nullptr, nullptr});
        } else {
            tacaw_status r = flush_grouped(p, {FlushReq{i, mode, nullptr, nullptr}}, s.due_stream);
            if (r != TACAW_OK) return r;
        }
    }
    return req.empty() ? TACAW_OK : flush_grouped(p, req, st);
}

// Periodic Dolph-Chebyshev window of length T: the symmetric window of M = T + 1 taps without
// its last tap.  The symmetric taps are the inverse DFT of M samples of the response
// T_{M-1}(x0 cos(pi k / M)), T_{M-1}(x0) = 10^(at/20), taken about the window's centre and
// scaled to a maximum of 1.  The phase pi k (2n - M + 1) / M is reduced exactly on a table of
// 2M cosines.
double chebyshev_t(int order, double x) {
    if (std::fabs(x) <= 1.0) return std::cos(order * std::acos(x));
    if (x > 1.0) return std::cosh(order * std::acosh(x));
    return ((order & 1) ? -1.0 : 1.0) * std::cosh(order * std::acosh(-x));
}

std::vector<double> chebwin_periodic(int T, double at_db) {
    const int M = T + 1;
    std::vector<double> w(T, 1.0);
    if (T <= 1) return w;
    const double x0 = std::cosh(std::acosh(std::pow(10.0, at_db / 20.0)) / (M - 1));
    std::vector<double> W(M), cs(2 * (size_t)M);
    for (int k = 0; k < M; ++k) W[k] = chebyshev_t(M - 1, x0 * std::cos(M_PI * k / M));
    for (int j = 0; j < 2 * M; ++j) cs[j] = std::cos(M_PI * j / M);
    double mx = 0.0;
    std::vector<double> full(M);
    for (int n = 0; n < M; ++n) {
        const int64_t step = (((int64_t)2 * n - M + 1) % (2 * M) + 2 * M) % (2 * M);
        int64_t idx = 0;
        double acc = 0.0;
        for (int k = 0; k < M; ++k) {
            acc += W[k] * cs[idx];
            idx += step;
            if (idx >= 2 * M) idx -= 2 * M;
        }
        full[n] = acc / M;
        mx = std::max(mx, full[n]);
    }
    for (int n = 0; n < T; ++n) w[n] = full[n] / mx;
    return w;
}

// Table arguments of stream s after build_stream (device phase and window inputs in place).
}  // namespace

namespace tacaw {
TableArgs stream_table_args(const Stream &s, int block_frames) {
    TableArgs ta{};
    ta.T = s.T;
    ta.T_pad = s.T_pad;
    ta.Nw = s.Nw;
    ta.Nw_pad = s.Nw_pad;
    ta.window = s.d.window;
    ta.window_param = s.d.window_param;
    ta.fft_bins = s.d.fft_bins;
    ta.block_frames = block_frames;
    ta.win_table = s.win_table;
    ta.swz = 1;
    ta.cj = s.cj;
    return ta;
}
}  // namespace tacaw

namespace {

tacaw_status build_stream(tacaw_plan_s *p, Stream &s, cudaStream_t st) {
    const tacaw_stream_desc &d = s.d;
    TableArgs ta{};
    ta.T = s.T;
    ta.T_pad = s.T_pad;
    ta.Nw = s.Nw;
    ta.Nw_pad = s.Nw_pad;
    ta.window = d.window;
    ta.window_param = d.window_param;
    ta.fft_bins = d.fft_bins;
    ta.block_frames = p->bf;
    if (d.window == TACAW_WIN_CHEBWIN) {
        // Dolph-Chebyshev taps (a transform over the whole window): computed here in FP64
        const std::vector<double> w = chebwin_periodic(s.T, d.window_param);
        if (!dev_alloc(p, &s.win_table, (size_t)s.T)) return fail(TACAW_ERR_OOM, "cudaMalloc(window table)");
        CU_CHECK(p, cudaMemcpy(s.win_table, w.data(), sizeof(double) * s.T, cudaMemcpyHostToDevice), "copy window");
        ta.win_table = s.win_table;
    }
    ta.swz = 1;   // the staged kernel copies pre-swizzled blocks
    // cycles per frame c_j = E_j dt / h (FP64)
    std::vector<double> cj(s.Nw), E(s.Nw);
    for (int j = 0; j < s.Nw; ++j) {
        E[j] = d.fft_bins ? (double)j * kPlanck_meV_ps / ((double)s.T * d.dt_fs * 1e-3) : d.E_meV[j];
        cj[j] = E[j] * (d.dt_fs * 1e-3) / kPlanck_meV_ps;
    }
    s.E = E;
    if (!dev_alloc(p, &s.cj, s.Nw)) return fail(TACAW_ERR_OOM, "cudaMalloc(cj)");
    CU_CHECK(p, cudaMemcpy(s.cj, cj.data(), sizeof(double) * s.Nw, cudaMemcpyHostToDevice), "copy cj");
    ta.cj = s.cj;

    std::vector<float> bose(s.Nw);
    for (int j = 0; j < s.Nw; ++j) bose[j] = (float)bose_factor(E[j], d.bose_T_K);
    if (!dev_alloc(p, &s.bose, s.Nw)) return fail(TACAW_ERR_OOM, "cudaMalloc(bose)");
    CU_CHECK(p, cudaMemcpy(s.bose, bose.data(), sizeof(float) * s.Nw, cudaMemcpyHostToDevice), "copy bose");

    if (!dev_alloc(p, &s.mu_hat, s.M) || !dev_alloc(p, &s.dmu, s.M) || !dev_alloc(p, &s.sum_res, s.M) ||
        !dev_alloc(p, &s.Wc, s.Nw) || !dev_alloc(p, &s.win, s.T))
        return fail(TACAW_ERR_OOM, "cudaMalloc(per-row buffers)");
    CU_CHECK(p, launch_window_transform(ta, s.Wc, st), "window transform");
    CU_CHECK(p, launch_window_values(ta, s.win, st), "window values");
    // adjoint needs the FP32 forward twiddles for both precisions
    if (!dev_alloc(p, &s.B32, (size_t)s.T_pad * s.Nw_pad)) return fail(TACAW_ERR_OOM, "cudaMalloc(B32)");
    CU_CHECK(p, launch_twiddles_fp32(ta, s.B32, st), "twiddles fp32");
    if (p->prec == TACAW_PREC_SPLIT_BF16) {
        const size_t nb = (size_t)s.n_kb_T * 2 * s.Nw_pad * 2 * p->bf;
        if (!dev_alloc(p, &s.B_hi, nb) || !dev_alloc(p, &s.B_lo, nb)) return fail(TACAW_ERR_OOM, "cudaMalloc(B split)");
        CU_CHECK(p, launch_twiddles_split(ta, s.B_hi, s.B_lo, p->f16, st), "twiddles split");
        if (p->in_place) {
            if (!dev_alloc(p, &s.d_frame_ptr, s.T)) return fail(TACAW_ERR_OOM, "cudaMalloc(frame table)");
        } else {
            const size_t na = (size_t)(s.ring / p->bf) * s.M_pad * 2 * p->bf;
            if (!dev_alloc(p, &s.A_hi, na) || !dev_alloc(p, &s.A_lo, na))
                return fail(TACAW_ERR_OOM, "cudaMalloc(staging)");
            // rows >= M and never-written slots must read as zeros
            CU_CHECK(p, cudaMemsetAsync(s.A_hi, 0, na * sizeof(__nv_bfloat16), st), "memset staging");
            CU_CHECK(p, cudaMemsetAsync(s.A_lo, 0, na * sizeof(__nv_bfloat16), st), "memset staging");
        }
    } else {
        const size_t na = (size_t)s.ring * s.M_pad;
        if (!dev_alloc(p, &s.A32, na)) return fail(TACAW_ERR_OOM, "cudaMalloc(staging)");
        CU_CHECK(p, cudaMemsetAsync(s.A32, 0, na * sizeof(float2), st), "memset staging");
    }
    if (s.needs_acc) {
        const size_t n = (size_t)s.Nw_pad * s.M_pad;
        if (p->accum == TACAW_ACC_FP64) {
            if (!dev_alloc(p, &s.acc_d, n)) return fail(TACAW_ERR_OOM, "cudaMalloc(accumulators)");
        } else {
            if (!dev_alloc(p, &s.acc_s, n) || (p->accum == TACAW_ACC_KAHAN_FP32 && !dev_alloc(p, &s.acc_c, n)))
                return fail(TACAW_ERR_OOM, "cudaMalloc(accumulators)");
        }
    }
    // detectors -> compact (pixel, weight) lists
    s.D = d.n_detectors;
    std::vector<int> idx;
    std::vector<float> wts;
    std::vector<float> full((size_t)std::max(1, s.D) * s.npix, 0.f);
    s.h_det_off.assign(s.D + 1, 0);
    std::vector<float> hmask;
    for (int k = 0; k < s.D; ++k) {
        const tacaw_detector &t = s.dets[k];
        if (t.kind == TACAW_DET_MASK) {
            hmask.resize(s.npix);
            CU_CHECK(p, cudaMemcpy(hmask.data(), t.d_mask, sizeof(float) * s.npix, cudaMemcpyDeviceToHost), "copy mask");
        }
        const double cx = (double)(d.kx / 2) + t.cx, cy = (double)(d.ky / 2) + t.cy;
        for (int y = 0; y < d.ky; ++y)
            for (int x = 0; x < d.kx; ++x) {
                const int64_t pix = (int64_t)y * d.kx + x;
                float w = 0.f;
                if (t.kind == TACAW_DET_MASK) {
                    w = hmask[pix];
                } else {
                    const double dx = x - cx, dy = y - cy, r2 = dx * dx + dy * dy;
                    bool in = r2 <= (double)t.r_out * (double)t.r_out;
                    if (t.kind == TACAW_DET_ANNULAR && t.r_in >= 0) in = in && r2 > (double)t.r_in * (double)t.r_in;
                    w = in ? 1.f : 0.f;
                }
                if (w != 0.f) {
                    idx.push_back((int)pix);
                    wts.push_back(w);
                    full[(size_t)k * s.npix + pix] = w;
                }
            }
        s.h_det_off[k + 1] = (int)idx.size();
    }
    s.n_det_entries = (int)idx.size();
    if (!dev_alloc(p, &s.det_idx, idx.size()) || !dev_alloc(p, &s.det_w, wts.size()) ||
        !dev_alloc(p, &s.det_off, s.h_det_off.size()))
        return fail(TACAW_ERR_OOM, "cudaMalloc(detectors)");
    if (!idx.empty()) {
        CU_CHECK(p, cudaMemcpy(s.det_idx, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice), "copy det");
        CU_CHECK(p, cudaMemcpy(s.det_w, wts.data(), sizeof(float) * wts.size(), cudaMemcpyHostToDevice), "copy det");
    }
    CU_CHECK(p, cudaMemcpy(s.det_off, s.h_det_off.data(), sizeof(int) * s.h_det_off.size(), cudaMemcpyHostToDevice),
             "copy det");
    // pixels inside any aperture, with their D weights (adjoint)
    std::vector<int> apix;
    std::vector<float> aw;
    for (int64_t pix = 0; pix < s.npix; ++pix) {
        bool any = false;
        for (int k = 0; k < s.D; ++k) any = any || full[(size_t)k * s.npix + pix] != 0.f;
        if (!any) continue;
        apix.push_back((int)pix);
        for (int k = 0; k < s.D; ++k) aw.push_back(full[(size_t)k * s.npix + pix]);
    }
    s.n_adj = (int)apix.size();
    s.h_adj_pix = apix;
    if (!dev_alloc(p, &s.adj_pix, apix.size()) || !dev_alloc(p, &s.adj_w, aw.size()))
        return fail(TACAW_ERR_OOM, "cudaMalloc(adjoint lists)");
    if (!apix.empty()) {
        CU_CHECK(p, cudaMemcpy(s.adj_pix, apix.data(), sizeof(int) * apix.size(), cudaMemcpyHostToDevice), "copy");
        CU_CHECK(p, cudaMemcpy(s.adj_w, aw.data(), sizeof(float) * aw.size(), cudaMemcpyHostToDevice), "copy");
    }
    CU_CHECK(p, cudaMemsetAsync(s.sum_res, 0, sizeof(double2) * s.M, st), "memset sums");
    CU_CHECK(p, cudaMemsetAsync(s.mu_hat, 0, sizeof(float2) * s.M, st), "memset mu");
    return TACAW_OK;
}

}  // namespace

namespace tacaw {
tacaw_status check_plan(tacaw_plan_s *p) {
    if (!p) return fail(TACAW_ERR_INVALID_ARG, "plan is NULL");
    if (p->poisoned) return fail(TACAW_ERR_STATE, "plan is poisoned by an earlier CUDA error or device timeout");
    return TACAW_OK;
}
}  // namespace tacaw

namespace {

// Buffers that kernels read or write: device or managed memory, or pinned host memory that the
// device reaches at the same address (for pushes a zero-copy ingest over the host link, on
// staged plans only: the in-place contraction copies frames with tensor copies, so
// allow_host is false there).  Anything else (pageable host memory, an address CUDA does not
// know) is refused before any work is enqueued.  Skipped while `st` is capturing a graph (the
// attribute query is not a stream operation; pointers of a captured segment are the caller's to
// keep valid).
}  // namespace

namespace tacaw {
tacaw_status check_kernel_memory(const void *ptr, const char *what, bool allow_host, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return TACAW_OK;
    }
    if (cs != cudaStreamCaptureStatusNone) return TACAW_OK;
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, ptr) != cudaSuccess) {
        cudaGetLastError();
        return fail(TACAW_ERR_INVALID_ARG, "%s is not an address CUDA knows", what);
    }
    if (pa.type == cudaMemoryTypeUnregistered)
        return fail(TACAW_ERR_INVALID_ARG, "%s is neither device memory nor pinned host memory", what);
    if (pa.type == cudaMemoryTypeHost) {
        if (pa.devicePointer != ptr)
            return fail(TACAW_ERR_INVALID_ARG, "pinned host %s is mapped at another device address; "
                        "pass the address from cudaHostGetDevicePointer", what);
        if (!allow_host)
            return fail(TACAW_ERR_INVALID_ARG, "frames_in_place plans read device memory only; push pinned "
                        "host frames into a staged plan");
    }
    return TACAW_OK;
}

int check_device_readable(const void *ptr, const char *what, cudaStream_t st) {
    return check_kernel_memory(ptr, what, true, st);
}

tacaw_status read_device_error(tacaw_plan_s *p, cudaStream_t st) {
    CU_CHECK(p, cudaStreamSynchronize(st), "cudaStreamSynchronize");
    uint32_t h = 0;
    CU_CHECK(p, cudaMemcpy(&h, p->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost), "read error word");
    if (h) {
        p->poisoned = true;
        if (h == DEVERR_FP16_RANGE)
            return fail(TACAW_ERR_OVERFLOW, "split FP16: a frame value times the operand scale %g exceeds the fp16 "
                        "range (65504); create the plan with a smaller fp16_scale", (double)p->f16_scale);
        return fail(TACAW_ERR_TIMEOUT, "device wait timed out (error bits 0x%x)", h);
    }
    return TACAW_OK;
}
}  // namespace tacaw

namespace {

// Detector spectra of stream s from its block of I.
tacaw_status launch_spectra(tacaw_plan_s *p, const Stream &s, const float *I, float *S, cudaStream_t st) {
    if (s.D <= 0 || !I || !S) return TACAW_OK;
    ApertureArgs a{};
    a.I = I;
    a.S = S;
    a.P = s.d.n_probes;
    a.D = s.D;
    a.Nw = s.Nw;
    a.npix = s.npix;
    a.idx = s.det_idx;
    a.wts = s.det_w;
    a.off = s.det_off;
    CU_CHECK(p, launch_aperture(a, st), "aperture");
    p->launches++;
    return TACAW_OK;
}

// Pipelined segments: launches the deferred segment's final contraction (its exact mean
// correction, I, Psi, then its spectra); with conv, the same launch's extra warps convert the
// recorded pushes of stream `conv` (the next segment) into its staging area.
tacaw_status launch_pending(tacaw_plan_s *p, const Stream *conv, cudaStream_t st) {
    TraceRange trace_range(conv ? "contraction (tensor cores) with the next conversion" : "contraction (tensor cores)");
    tacaw_plan_s::Pending &q = p->pend;
    Stream &ps = q.snap;
    CU_CHECK(p, launch_mean_residual(ps.M, ps.T, ps.d.subtract_mean, ps.sum_res, ps.dmu, p->f16_scale, st),
             "mean residual");
    p->launches++;
    TcPlanArgs a = tc_args(p, ps, epi_args(p, ps, FLUSH_FINAL, q.I, q.Psi));
    a.tile_counter = p->d_counters + (p->counter_slot++ % kCounterRing);
    tacaw_status r = trace_buffer(p, tc_grid_ctas(a), &a.trace);
    if (r != TACAW_OK) return r;
    cudaEvent_t e0, e1;
    r = timing_begin(p, &e0, &e1, st);
    if (r != TACAW_OK) return r;
    if (conv) {
        TcConvJob j{};
        j.frame_ptr = conv->d_frame_ptr;
        j.T = conv->T;
        j.M = conv->M;
        j.M_pad = conv->M_pad;
        j.npix = conv->npix;
        j.kx = conv->d.kx;
        j.pitch_row = conv->d.pitch_row;
        j.pitch_probe = conv->d.pitch_probe;
        j.roi_x0 = conv->d.roi_x0;
        j.roi_y0 = conv->d.roi_y0;
        j.mu_hat = conv->mu_hat;
        j.sum_res = conv->sum_res;
        j.A_hi = conv->A_hi;
        j.A_lo = conv->A_lo;
        j.counter = p->d_counters + (p->counter_slot++ % kCounterRing);
        CU_CHECK(p, launch_flush_tc_group_conv(&a, 1, j, st), "flush (tensor cores) with the next conversion");
    } else {
        CU_CHECK(p, launch_flush_tc(a, st), "flush (tensor cores)");
    }
    p->launches++;
    p->flush_launches++;
    p->flushes_total++;
    r = timing_end(p, e0, e1, st);
    if (r != TACAW_OK) return r;
    q.active = false;
    return launch_spectra(p, ps, q.I, q.S, st);
}

// Pipelined finalize: the pending segment's contraction goes out now, converting this segment's
// recorded pushes; this segment's own contraction is deferred to the next finalize (or
// tacaw_drain), and the next segment stages into the other area.
tacaw_status finalize_pipelined(tacaw_plan_s *p, float *d_I, float *d_S, float2 *d_Psi, cudaStream_t st) {
    Stream &s = p->s[0];
    if (p->pend.active) {
        tacaw_status r = launch_pending(p, p->deferred_pushes ? &s : nullptr, st);
        if (r != TACAW_OK) return r;
    }
    p->pend.snap = s;
    p->pend.I = d_I ? d_I + s.I_off : nullptr;
    p->pend.S = d_S ? d_S + s.S_off : nullptr;
    p->pend.Psi = d_Psi ? d_Psi + s.I_off : nullptr;
    p->pend.active = true;
    std::swap(s.A_hi, s.A_hi2);
    std::swap(s.A_lo, s.A_lo2);
    std::swap(s.mu_hat, s.mu_hat2);
    std::swap(s.sum_res, s.sum_res2);
    std::swap(s.dmu, s.dmu2);
    p->deferred_pushes = false;
    p->finalized = true;
    return TACAW_OK;
}

tacaw_status finalize_impl(tacaw_plan_t p, float *d_I, float *d_S, void *d_Psi, cudaStream_t st) {
    tacaw_status c = check_plan(p);
    if (c != TACAW_OK) return c;
    const void *outs[3] = {d_I, d_S, d_Psi};
    const char *names[3] = {"d_I", "d_S", "d_Psi"};
    for (int i = 0; i < 3; ++i) {
        if (!outs[i]) continue;
        c = check_kernel_memory(outs[i], names[i], true, st);
        if (c != TACAW_OK) return c;
    }
    if (p->finalized) return fail(TACAW_ERR_STATE, "segment already finalized");
    for (size_t i = 0; i < p->us.size(); ++i)
        if (p->us[i].pushed != p->us[i].total)
            return fail(TACAW_ERR_STATE, "stream %zu has %lld of %lld frames", i, (long long)p->us[i].pushed,
                        (long long)p->us[i].total);
    if (d_S && !d_I) return fail(TACAW_ERR_INVALID_ARG, "d_S requires d_I");
    for (auto &u : p->us)
        if (d_Psi && u.N > 1) return fail(TACAW_ERR_INVALID_ARG, "d_Psi is not available for Welch-averaged streams");
    if (p->pipe) return finalize_pipelined(p, d_I, d_S, static_cast<float2 *>(d_Psi), st);
    {
        tacaw_status r = flush_due(p, st);   // none expected: a due stream still awaits frames
        if (r != TACAW_OK) return r;
    }
    // single-segment streams: their last flush (Welch lanes finished theirs during the pushes)
    if (!p->in_place)
        for (auto &s : p->s) {
            if (p->us[s.user].N > 1) continue;
            CU_CHECK(p, launch_mean_residual(s.M, s.T, s.d.subtract_mean, s.sum_res, s.dmu, p->f16_scale, st),
                     "mean residual");
            p->launches++;
        }
    float2 *Psi_all = static_cast<float2 *>(d_Psi);
    if (p->prec == TACAW_PREC_SPLIT_BF16 && !p->in_place) {
        cudaStream_t fs = st;
        if (p->tc_max_ctas > 0) {
            if (!p->hp_stream) {
                int lo = 0, hi = 0;
                CU_CHECK(p, cudaDeviceGetStreamPriorityRange(&lo, &hi), "stream priorities");
                CU_CHECK(p, cudaStreamCreateWithPriority(&p->hp_stream, cudaStreamNonBlocking, hi), "flush stream");
                CU_CHECK(p, cudaEventCreateWithFlags(&p->hp_in, cudaEventDisableTiming), "cudaEventCreate");
                CU_CHECK(p, cudaEventCreateWithFlags(&p->hp_out, cudaEventDisableTiming), "cudaEventCreate");
            }
            CU_CHECK(p, cudaEventRecord(p->hp_in, st), "cudaEventRecord");
            CU_CHECK(p, cudaStreamWaitEvent(p->hp_stream, p->hp_in, 0), "cudaStreamWaitEvent");
            fs = p->hp_stream;
        }
        tacaw_status r = final_flush_grouped(p, d_I, Psi_all, fs);
        if (r != TACAW_OK) return r;
        if (fs != st) {
            CU_CHECK(p, cudaEventRecord(p->hp_out, fs), "cudaEventRecord");
            CU_CHECK(p, cudaStreamWaitEvent(st, p->hp_out, 0), "cudaStreamWaitEvent");
        }
    } else {
        for (auto &s : p->s) {
            if (p->us[s.user].N > 1) continue;
            tacaw_status r = run_flush(p, s, FLUSH_FINAL, d_I ? d_I + s.I_off : nullptr,
                                       Psi_all ? Psi_all + s.I_off : nullptr, st);
            if (r != TACAW_OK) return r;
        }
    }
    for (auto &u : p->us)
        if (u.N > 1 && d_I)
            CU_CHECK(p, cudaMemcpyAsync(d_I + u.I_off, u.I_acc, sizeof(float) * u.I_elems, cudaMemcpyDeviceToDevice, st),
                     "Welch average");
    if (d_S)
        for (auto &u : p->us) {
            const Stream &s = p->s[u.first];
            if (s.D <= 0) continue;
            ApertureArgs a{};
            a.I = d_I + u.I_off;
            a.S = d_S + u.S_off;
            a.P = s.d.n_probes;
            a.D = s.D;
            a.Nw = s.Nw;
            a.npix = s.npix;
            a.idx = s.det_idx;
            a.wts = s.det_w;
            a.off = s.det_off;
            CU_CHECK(p, launch_aperture(a, st), "aperture");
            p->launches++;
        }
    p->finalized = true;
    return TACAW_OK;
}

// Pushes n frames (device pointer, the stream's layout) into internal stream s.
tacaw_status push_internal(tacaw_plan_s *p, Stream &s, const float2 *frames, int n_frames, cudaStream_t st) {
    FrameGeom g{};
    g.pitch_row = s.d.pitch_row;
    g.pitch_frame = s.d.pitch_frame;
    g.pitch_probe = s.d.pitch_probe;
    g.roi_x0 = s.d.roi_x0;
    g.roi_y0 = s.d.roi_y0;
    g.kx = s.d.kx;
    g.ky = s.d.ky;
    g.npix = s.npix;
    g.M = s.M;
    g.base = frames;
    if (s.due) {
        // this stream's ring is full: its deferred flush (with any others) goes first
        tacaw_status r = flush_due(p, st);
        if (r != TACAW_OK) return r;
    }
    if (s.pushed == 0 && s.d.subtract_mean) {
        CU_CHECK(p, launch_mean(g, n_frames, s.mu_hat, st), "provisional mean");
        p->launches++;
    }
    if (p->pipe && p->pend.active) {
        // pipelined segments: the pending contraction's launch converts this segment's frames;
        // here only their addresses are recorded (by a kernel on the stream)
        CU_CHECK(p, launch_frame_table(s.d_frame_ptr + s.pushed, frames, g.pitch_frame, n_frames, st), "frame table");
        p->launches++;
        s.staged += n_frames;
        s.pushed += n_frames;
        p->deferred_pushes = true;
        return TACAW_OK;
    }
    int done = 0;
    while (done < n_frames) {
        const int chunk = std::min(n_frames - done, s.ring - s.staged);
        FrameGeom gc = g;
        gc.base = g.base + (int64_t)done * g.pitch_frame;
        if (p->in_place) {
            if (s.pushed == 0) s.h_pushes.clear();
            s.h_pushes.emplace_back((int)s.pushed, gc.base);
            // the frames' addresses go to the device table by a kernel on the stream: ordered
            // with the flushes that read them, and fixed inside a captured graph
            CU_CHECK(p, launch_frame_table(s.d_frame_ptr + s.pushed, gc.base, g.pitch_frame, chunk, st), "frame table");
            p->launches++;
        } else {
            if (p->prec == TACAW_PREC_SPLIT_BF16)
                CU_CHECK(p, launch_convert_split(gc, chunk, s.staged, p->bf, s.M_pad, s.mu_hat, s.sum_res, s.A_hi,
                                                 s.A_lo, 1, p->f16, p->f16_scale, p->d_err, st),
                         "convert");
            else
                CU_CHECK(p, launch_convert_fp32(gc, chunk, s.staged, s.M_pad, s.mu_hat, s.sum_res, s.A32, st),
                         "convert");
            p->launches++;
        }
        s.staged += chunk;
        s.pushed += chunk;
        done += chunk;
        if (s.staged == s.ring && s.pushed < s.T) {
            if (deferrable(p, s)) {
                s.due = true;
                s.due_stream = st;
                // more frames of this push follow: the ring must be emptied now
                tacaw_status r = done < n_frames ? flush_due(p, st) : TACAW_OK;
                if (r != TACAW_OK) return r;
            } else {
                tacaw_status r = run_flush(p, s, s.flushes == 0 ? FLUSH_STORE : FLUSH_ADD, nullptr, nullptr, st);
                if (r != TACAW_OK) return r;
            }
        }
    }
    return TACAW_OK;
}

// A Welch lane has all T frames of its segment: finish the segment into the user's average
// and make the lane ready for its next segment.
tacaw_status finish_segment(tacaw_plan_s *p, UserStream &u, Stream &s, cudaStream_t st) {
    if (!p->in_place) {
        CU_CHECK(p, launch_mean_residual(s.M, s.T, s.d.subtract_mean, s.sum_res, s.dmu, p->f16_scale, st),
                 "mean residual");
        p->launches++;
    }
    tacaw_status r = run_flush(p, s, FLUSH_FINAL, u.I_acc, nullptr, st);
    if (r != TACAW_OK) return r;
    CU_CHECK(p, cudaMemsetAsync(s.sum_res, 0, sizeof(double2) * s.M, st), "reset sums");
    s.pushed = s.staged = s.stage_start = s.flushes = 0;
    s.seg += u.lanes;
    return TACAW_OK;
}

}  // namespace

extern "C" {

const char *tacaw_last_error(void) { return g_last_error.c_str(); }

tacaw_status tacaw_set_log_callback(tacaw_log_fn fn, void *user) {
    std::lock_guard<std::mutex> lk(g_log_mu);
    g_log_fn = fn;
    g_log_user = fn ? user : nullptr;
    return TACAW_OK;
}

const char *tacaw_version(void) { return "tacaw-gb300 0.1 (sm_103a)"; }

tacaw_status tacaw_plan_create(const tacaw_plan_desc *desc, tacaw_plan_t *out) {
    TraceRange trace_range("tacaw_plan_create");
    g_last_error.clear();
    if (!desc || !out) return fail(TACAW_ERR_INVALID_ARG, "desc and out must not be NULL");
    *out = nullptr;
    if (desc->n_streams < 1 || !desc->streams) return fail(TACAW_ERR_INVALID_ARG, "n_streams must be >= 1");
    if (desc->precision != TACAW_PREC_FP32 && desc->precision != TACAW_PREC_SPLIT_BF16 &&
        desc->precision != TACAW_PREC_SPLIT_FP16)
        return fail(TACAW_ERR_INVALID_ARG, "bad precision");
    // both split paths share the staged tensor-core machinery; they differ in the 16-bit type
    // of the pieces (and the operand scale the fp16 range needs)
    const bool f16 = desc->precision == TACAW_PREC_SPLIT_FP16;
    const int prec = f16 ? (int)TACAW_PREC_SPLIT_BF16 : desc->precision;
    double f16_scale = 1.0;
    if (f16) {
        f16_scale = desc->fp16_scale == 0.0 ? 4096.0 : desc->fp16_scale;
        int ex = 0;
        if (!(f16_scale > 0.0) || std::frexp(f16_scale, &ex) != 0.5 || ex - 1 < -60 || ex - 1 > 60)
            return fail(TACAW_ERR_INVALID_ARG, "fp16_scale must be 0 or a power of two in [2^-60, 2^60]");
        if (desc->frames_in_place)
            return fail(TACAW_ERR_UNSUPPORTED, "frames_in_place converts frames to bf16 inside the contraction; "
                        "the split-FP16 path stages its operands (frames_in_place 0)");
    }
    if (desc->accum < TACAW_ACC_KAHAN_FP32 || desc->accum > TACAW_ACC_AUTO)
        return fail(TACAW_ERR_INVALID_ARG, "bad accum");
    if (desc->k_stage < 0 || (desc->k_stage % 8) != 0) return fail(TACAW_ERR_INVALID_ARG, "k_stage must be a multiple of 8");
    for (int i = 0; i < desc->n_streams; ++i) {
        tacaw_status v = validate_stream(desc->streams[i], i);
        if (v != TACAW_OK) return v;
    }
    if (desc->tc_drain_frames < 0 || desc->tc_drain_frames % 8)
        return fail(TACAW_ERR_INVALID_ARG, "tc_drain_frames must be a non-negative multiple of 8");
    if (desc->tc_omega_tile < 0 || desc->tc_omega_tile % 8)
        return fail(TACAW_ERR_INVALID_ARG, "tc_omega_tile must be a multiple of 8");
    if (desc->tc_block_frames != 0 && desc->tc_block_frames != 8 && desc->tc_block_frames != 16 &&
        desc->tc_block_frames != 32)
        return fail(TACAW_ERR_INVALID_ARG, "tc_block_frames must be 0 (auto), 8, 16 or 32");
    if (prec == TACAW_PREC_SPLIT_BF16 && desc->tc_block_frames && desc->k_stage % desc->tc_block_frames)
        return fail(TACAW_ERR_INVALID_ARG, "k_stage must be a multiple of tc_block_frames");
    if (desc->frames_in_place) {
        // the in-place kernel reads each tile's 128 rows of every frame with one contiguous copy:
        // per stream, the rows of a tile contiguous in the frame, even element offsets (16-byte
        // aligned copies), 32-frame blocks
        if (prec != TACAW_PREC_SPLIT_BF16)
            return fail(TACAW_ERR_UNSUPPORTED, "frames_in_place needs the split-BF16 path");
        if ((desc->tc_block_frames != 0 && desc->tc_block_frames != 32) || desc->k_stage % 32)
            return fail(TACAW_ERR_UNSUPPORTED, "frames_in_place reads 32-frame blocks: tc_block_frames 0 or 32, "
                        "k_stage a multiple of 32");
        for (int i = 0; i < desc->n_streams; ++i) {
            const tacaw_stream_desc &d = desc->streams[i];
            const int64_t npix = (int64_t)d.kx * d.ky, M = npix * d.n_probes;
            const bool even = M % 2 == 0 && d.kx % 2 == 0 && d.pitch_row % 2 == 0 && d.roi_x0 % 2 == 0 &&
                              d.pitch_frame % 2 == 0 && (d.n_probes == 1 || d.pitch_probe % 2 == 0);
            const bool rows_contiguous =
                d.kx % kMTile == 0 ||
                (d.pitch_row == d.kx && d.roi_x0 == 0 &&
                 (npix % kMTile == 0 || d.n_probes == 1 || d.pitch_probe == npix));
            if (!even || !rows_contiguous)
                return fail(TACAW_ERR_UNSUPPORTED,
                            "stream %d: frames_in_place needs every 128-row tile contiguous in a frame (kx a "
                            "multiple of 128, or unpadded rows from roi_x0 = 0 with probes that are whole tiles or "
                            "adjacent) and even sizes, offsets and pitches; stage the frames instead", i);
        }
    }
    tacaw_plan_s *p = new (std::nothrow) tacaw_plan_s();
    if (!p) return fail(TACAW_ERR_OOM, "host allocation failed");
    // split path: hi*hi drained from tensor memory into FP32 registers every 512 frames (default)
    const int drain_frames = desc->tc_drain_frames ? desc->tc_drain_frames : 512;
    // widest tile: the staged form's register sums; in place, also the raw frame ring
    const int tile_cap = desc->frames_in_place ? kInplaceMaxOmegaTile : kDrainMaxOmegaTile;
    p->in_place = desc->frames_in_place != 0;
    if (prec == TACAW_PREC_SPLIT_BF16) {
        // widest rows first: fewer, larger TMA requests per MMA K-step
        if (desc->tc_block_frames) {
            p->bf = desc->tc_block_frames;
        } else {
            p->bf = 32;
            while (p->bf > 8 && desc->k_stage % p->bf) p->bf /= 2;
        }
    }
    p->prec = prec;
    p->prec_user = desc->precision;
    p->f16 = f16 ? 1 : 0;
    p->f16_scale = (float)f16_scale;
    p->accum = desc->accum == TACAW_ACC_AUTO ? TACAW_ACC_KAHAN_FP32 : desc->accum;   // resolved with K_stage
    if (!dev_alloc(p, &p->d_err, 1) || cudaMemset(p->d_err, 0, sizeof(uint32_t)) != cudaSuccess ||
        !dev_alloc(p, &p->d_counters, kCounterRing)) {
        cudaGetLastError();
        free_all(p);
        delete p;
        return fail(TACAW_ERR_OOM, "cudaMalloc(error word)");
    }
    auto bail = [&](tacaw_status st) {
        free_all(p);
        delete p;
        return st;
    };
    int T_pad_max = 0;
    for (int i = 0; i < desc->n_streams; ++i) {
        Stream s;
        s.d = desc->streams[i];
        s.dets.assign(s.d.detectors, s.d.detectors + s.d.n_detectors);
        s.d.detectors = nullptr;
        s.d.E_meV = nullptr;
        s.npix = (int64_t)s.d.kx * s.d.ky;
        s.M = (int64_t)s.d.n_probes * s.npix;
        s.M_pad = round_up(s.M, kMTile);
        s.T = s.d.T;
        s.T_pad = (int)round_up(s.T, p->prec == TACAW_PREC_SPLIT_BF16 ? p->bf : 8);
        s.n_kb_T = s.T_pad / (p->prec == TACAW_PREC_SPLIT_BF16 ? p->bf : 8);
        s.Nw = s.d.n_omega;
        choose_omega_tile(s, desc->tc_omega_tile, tile_cap);
        if (p->prec == TACAW_PREC_FP32) s.Nw_pad = (int)round_up(s.Nw, 64);
        T_pad_max = std::max(T_pad_max, s.T_pad);
        // Welch: ceil(T / stride) lanes (segments that overlap in time), each an internal stream
        UserStream u;
        u.N = std::max(1, s.d.welch_segments);
        u.L = s.T;
        u.stride = s.d.welch_stride ? s.d.welch_stride : s.T;
        u.lanes = u.N > 1 ? (int)std::min<int64_t>(u.N, (s.T + u.stride - 1) / u.stride) : 1;
        u.skip = desc->streams[i].skip_init;
        u.total = u.skip + (int64_t)(u.N - 1) * u.stride + u.L;
        u.first = (int)p->s.size();
        s.user = i;
        if (u.N > 1) {
            s.out_scale = (float)(1.0 / (double)u.N);
            s.out_add = 1;
        }
        for (int l = 0; l < u.lanes; ++l) {
            s.lane = l;
            s.seg = l;
            p->s.push_back(s);
        }
        p->us.push_back(u);
    }
    // keep the energies (host) for the tables
    std::vector<std::vector<double>> Es(desc->n_streams);
    for (int i = 0; i < desc->n_streams; ++i)
        if (!desc->streams[i].fft_bins) Es[i].assign(desc->streams[i].E_meV, desc->streams[i].E_meV + desc->streams[i].n_omega);

    auto max_cols = [&]() {
        int n = 0;
        for (auto &s : p->s) n = std::max(n, 2 * s.wt);
        return n;
    };
    if (p->prec == TACAW_PREC_SPLIT_BF16) {
        // widest rows that still leave two stages (wider rows beat deeper rings in measurements)
        if (!desc->tc_block_frames)
            while (p->bf > 8 && tc_stages_for(max_cols(), p->bf) < 2) p->bf /= 2;
        for (auto &s : p->s) s.n_kb_T = s.T_pad / p->bf;
        p->tc_max_ctas = desc->tc_max_ctas > 0 ? desc->tc_max_ctas : 0;
        p->drain_kb = std::max(1, drain_frames / p->bf);
        // autotuner: time the candidate tiles of every stream shape (staged operands only)
        if (desc->tune_cache_path && !p->in_place) {
            const auto t0 = std::chrono::steady_clock::now();
            std::vector<std::vector<TuneCand>> tabs(p->s.size());
            for (size_t i = 0; i < p->s.size(); ++i) {
                Stream &s = p->s[i];
                TuneShape sh{};
                sh.M = s.M;
                sh.Nw = s.Nw;
                sh.T = s.T;
                sh.ring = desc->k_stage ? std::min(desc->k_stage, s.T_pad) : s.T_pad;
                sh.bf = p->bf;
                sh.wt_max = kDrainMaxOmegaTile;
                sh.drain_kb = p->drain_kb;
                sh.fixed_wt = desc->tc_omega_tile ? s.wt : 0;
                sh.multi = desc->n_streams > 1;
                int timed = 0;
                char eb[256];
                if (!tc_autotune(sh, desc->tune_cache_path, p->d_err, nullptr, &tabs[i], &timed, eb, sizeof(eb)))
                    return bail(fail(TACAW_ERR_CUDA, "%s", eb));
                p->tune_timed += timed;
            }
            // each stream's fastest energy tile
            for (size_t i = 0; i < p->s.size(); ++i) {
                Stream &s = p->s[i];
                double b = 1e300;
                for (const TuneCand &c : tabs[i])
                    if (c.ms < b) {
                        b = c.ms;
                        s.wt = c.wt;
                    }
                if (b == 1e300) return bail(fail(TACAW_ERR_UNSUPPORTED, "autotune: no tile fits stream %zu", i));
                s.n_wt = (s.Nw + s.wt - 1) / s.wt;
                s.Nw_pad = s.wt * s.n_wt;
                s.tuned = true;
                p->tuned_streams++;
            }
            p->tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        }
    }

    // budget and K_stage
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaError_t e = cudaGetLastError();
        return bail(fail(TACAW_ERR_CUDA, "cudaMemGetInfo: %s", cudaGetErrorString(e)));
    }
    const int64_t budget = desc->hbm_budget_bytes > 0 ? desc->hbm_budget_bytes : (int64_t)(0.9 * (double)free_b);
    int64_t fixed = 0;
    for (auto &u : p->us)   // Welch averages
        if (u.N > 1) fixed += 4 * (int64_t)p->s[u.first].d.n_probes * p->s[u.first].Nw * p->s[u.first].npix;
    for (auto &s : p->s) {
        fixed += s.M * (8 + 8 + 16) + (int64_t)s.T_pad * s.Nw_pad * 8 + (int64_t)s.n_kb_T * 2 * s.Nw_pad * 16 * 4 +
                 (int64_t)s.npix * 16 + (1 << 20);
    }
    int accum = desc->accum == TACAW_ACC_AUTO ? TACAW_ACC_FP32 : desc->accum;
    auto need = [&](int K) {
        int64_t b = fixed;
        for (auto &s : p->s) {
            const int ring = std::min(K, s.T_pad);
            b += p->in_place ? (int64_t)ring * 8 : stream_stage_bytes(s, ring);
            if (s.T > ring) b += stream_acc_bytes(s, accum);
        }
        return b;
    };
    // automatic accumulators: plain FP32 while no segment takes more than kAutoFp32Flushes
    // flushes at the K_stage they allow, else compensated FP32
    auto max_flushes = [&](int K) {
        int f = 1;
        for (auto &s : p->s) f = std::max(f, (s.T + std::min(K, s.T_pad) - 1) / std::min(K, s.T_pad));
        return f;
    };
    auto pick_k = [&]() {
        if (need(T_pad_max) <= budget) return T_pad_max;
        for (int k = (T_pad_max / 64) * 64; k >= 64; k -= 64)  // multiples of 64: any block size divides
            if (need(k) <= budget) return k;
        return 0;
    };
    int K = desc->k_stage;
    if (desc->accum == TACAW_ACC_AUTO) {
        const int k32 = K ? K : pick_k();
        if (k32 == 0 || max_flushes(k32) > kAutoFp32Flushes) accum = TACAW_ACC_KAHAN_FP32;
    }
    p->accum = accum;
    if (K == 0) {
        if (need(T_pad_max) <= budget) {
            K = T_pad_max;
        } else {
            K = 0;
            for (int k = (T_pad_max / 64) * 64; k >= 64; k -= 64)  // multiples of 64: any block size divides
                if (need(k) <= budget) {
                    K = k;
                    break;
                }
            if (K == 0)
                return bail(fail(TACAW_ERR_OOM, "HBM budget of %lld bytes is too small (needs %lld at K_stage=64)",
                                 (long long)budget, (long long)need(64)));
        }
    } else if (need(K) > budget) {
        return bail(fail(TACAW_ERR_OOM, "k_stage=%d needs %lld bytes, budget %lld", K, (long long)need(K),
                         (long long)budget));
    }
    p->k_stage = K;
    // each segment in equal flush rounds of at most K frames (the same number of rounds as K
    // gives, none of them a short remainder): a flush's tiles then all carry about as many
    // frames as the others, enough to cover their epilogue
    const int ring_unit = p->in_place ? 32 : (p->prec == TACAW_PREC_SPLIT_BF16 ? p->bf : 8);
    for (auto &s : p->s) {
        const int rounds = (s.T_pad + K - 1) / K;
        const int even = (s.T_pad + rounds - 1) / rounds;
        s.ring = std::min({K, s.T_pad, (even + ring_unit - 1) / ring_unit * ring_unit});
        s.needs_acc = s.T > s.ring;
    }
    if (p->prec == TACAW_PREC_SPLIT_BF16) {
        for (auto &s : p->s) {
            const int N = 2 * s.wt;
            s.stages = p->in_place ? tc_inplace_stages(N, p->bf) : tc_stages_for(N, p->bf);
            if (s.stages < 2)
                return bail(fail(TACAW_ERR_UNSUPPORTED, "tensor-core tile of %d columns does not fit shared memory", N));
        }
        p->stages = p->s[0].stages;
    }
    cudaStream_t st = nullptr;
    tacaw_status rc = TACAW_OK;
    int64_t I_off = 0, S_off = 0;
    for (size_t i = 0; i < p->s.size() && rc == TACAW_OK; ++i) {
        Stream &s = p->s[i];
        s.d.E_meV = Es[s.user].empty() ? nullptr : Es[s.user].data();
        rc = build_stream(p, s, st);
        s.d.E_meV = nullptr;
    }
    for (auto &u : p->us) {
        if (rc != TACAW_OK) break;
        Stream &s0 = p->s[u.first];
        u.I_elems = (int64_t)s0.d.n_probes * s0.Nw * s0.npix;
        u.I_off = I_off;
        u.S_off = S_off;
        for (int l = 0; l < u.lanes; ++l) {
            p->s[u.first + l].I_off = I_off;
            p->s[u.first + l].S_off = S_off;
        }
        I_off += u.I_elems;
        S_off += (int64_t)s0.d.n_probes * s0.D * s0.Nw;
        if (u.N > 1) {
            if (!dev_alloc(p, &u.I_acc, (size_t)u.I_elems)) {
                rc = fail(TACAW_ERR_OOM, "cudaMalloc(Welch average)");
                break;
            }
            if (cudaMemsetAsync(u.I_acc, 0, sizeof(float) * u.I_elems, st) != cudaSuccess)
                rc = fail(TACAW_ERR_CUDA, "memset");
        }
    }
    p->I_elems = I_off;
    p->S_elems = S_off;
    if (rc == TACAW_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) rc = fail(TACAW_ERR_CUDA, "plan tables: %s", cudaGetErrorString(e));
    }
    if (rc != TACAW_OK) {
        free_all(p);
        delete p;
        return rc;
    }
    *out = p;
    {
        char buf[512];
        const Stream &s0 = p->s[0];
        snprintf(buf, sizeof(buf),
                 "plan: %d stream(s) (%zu internal), precision %s, K_stage %d frames, accumulators %s, "
                 "first stream: %d energies in tiles of %d, block frames %d, drained chunks %d frames, "
                 "in place %d, autotuned streams %d, %.2f GB on the device",
                 (int)p->us.size(), p->s.size(),
                 p->prec_user == TACAW_PREC_FP32 ? "fp32" : (p->f16 ? "split_fp16" : "split_bf16"), p->k_stage,
                 p->accum == TACAW_ACC_FP64 ? "fp64" : (p->accum == TACAW_ACC_FP32 ? "fp32" : "kahan"), s0.Nw,
                 s0.wt, p->bf, p->drain_kb * p->bf, p->in_place ? 1 : 0, p->tuned_streams, p->bytes / 1e9);
        emit_log(TACAW_LOG_INFO, buf);
    }
    return TACAW_OK;
}

}  // extern "C"

namespace {

// The checks of one push, before any device work.
tacaw_status validate_push(tacaw_plan_s *p, int sid, const void *d_frames, int n_frames, cudaStream_t st) {
    if (sid < 0 || sid >= (int)p->us.size()) return fail(TACAW_ERR_INVALID_ARG, "stream_id %d out of range", sid);
    if (!d_frames) return fail(TACAW_ERR_INVALID_ARG, "d_frames is NULL");
    if (n_frames < 1) return fail(TACAW_ERR_INVALID_ARG, "n_frames must be >= 1");
    if (p->finalized) return fail(TACAW_ERR_STATE, "segment finalized; call tacaw_reset first");
    if ((reinterpret_cast<uintptr_t>(d_frames) & 7) != 0) return fail(TACAW_ERR_INVALID_ARG, "d_frames must be 8-byte aligned");
    if (p->in_place && (reinterpret_cast<uintptr_t>(d_frames) & 15) != 0)
        return fail(TACAW_ERR_INVALID_ARG, "in-place frames must be 16-byte aligned (contiguous row copies)");
    tacaw_status pk = check_kernel_memory(d_frames, "d_frames", !p->in_place, st);
    if (pk != TACAW_OK) return pk;
    const UserStream &u = p->us[sid];
    if (u.pushed + n_frames > u.total)
        return fail(TACAW_ERR_OVERFLOW, "push of %d frames exceeds %lld (already %lld)", n_frames, (long long)u.total,
                    (long long)u.pushed);
    return TACAW_OK;
}

// One validated push of a user stream.
tacaw_status push_user(tacaw_plan_s *p, int sid, const float2 *base, int n_frames, cudaStream_t st) {
    UserStream &u = p->us[sid];
    // leading frames of the stream that precede its first segment are dropped unread
    if (u.pushed + n_frames <= u.skip) {
        u.pushed += n_frames;
        return TACAW_OK;
    }
    if (u.pushed < u.skip) {
        const int64_t drop = u.skip - u.pushed;
        base += drop * p->s[u.first].d.pitch_frame;
        n_frames -= (int)drop;
        u.pushed = u.skip;
    }
    if (u.N <= 1) {
        tacaw_status r = push_internal(p, p->s[u.first], base, n_frames, st);
        if (r == TACAW_OK) u.pushed += n_frames;
        return r;
    }
    // Welch: every lane takes the part of this push inside its current segment, finishing
    // segments (and starting the next ones of the lane) as their last frames arrive; frame
    // positions count from the first frame after the skipped ones
    const int64_t a = u.pushed - u.skip, b = a + n_frames;
    for (int l = 0; l < u.lanes; ++l) {
        Stream &s = p->s[u.first + l];
        while (s.seg < u.N) {
            const int64_t s0 = s.seg * (int64_t)u.stride;
            const int64_t lo = std::max(a, s0 + s.pushed), hi = std::min(b, s0 + u.L);
            if (lo >= hi) break;
            tacaw_status r = push_internal(p, s, base + (lo - a) * s.d.pitch_frame, (int)(hi - lo), st);
            if (r != TACAW_OK) return r;
            if (s.pushed < s.T) break;
            r = finish_segment(p, u, s, st);
            if (r != TACAW_OK) return r;
        }
    }
    u.pushed = u.skip + b;
    return TACAW_OK;
}

}  // namespace

extern "C" {

tacaw_status tacaw_push_frames(tacaw_plan_t p, int sid, const void *d_frames, int n_frames, void *stream) {
    TraceRange trace_range("tacaw_push_frames");
    tacaw_status c = check_plan(p);
    if (c != TACAW_OK) return c;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    c = validate_push(p, sid, d_frames, n_frames, st);
    if (c != TACAW_OK) return c;
    return push_user(p, sid, static_cast<const float2 *>(d_frames), n_frames, st);
}

tacaw_status tacaw_push_frames_group(tacaw_plan_t p, int n, const int *stream_ids, const void *const *d_frames,
                                     const int *n_frames, void *stream) {
    TraceRange trace_range("tacaw_push_frames_group");
    tacaw_status c = check_plan(p);
    if (c != TACAW_OK) return c;
    if (n < 1 || !stream_ids || !d_frames || !n_frames)
        return fail(TACAW_ERR_INVALID_ARG, "push group: n >= 1 and non-NULL arrays required");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<char> seen(p->us.size(), 0);
    for (int i = 0; i < n; ++i) {
        c = validate_push(p, stream_ids[i], d_frames[i], n_frames[i], st);
        if (c != TACAW_OK) return c;
        if (seen[stream_ids[i]]) return fail(TACAW_ERR_INVALID_ARG, "push group: stream_id %d appears twice", stream_ids[i]);
        seen[stream_ids[i]] = 1;
    }
    // deferred flushes of these streams go first (flush_due runs every due flush, grouped)
    const bool split = p->prec == TACAW_PREC_SPLIT_BF16 && !p->in_place;
    for (int i = 0; i < n; ++i) {
        const UserStream &u = p->us[stream_ids[i]];
        if (u.N <= 1 && p->s[u.first].due) {
            c = flush_due(p, st);
            if (c != TACAW_OK) return c;
            break;
        }
    }
    // pushes that fit their stream's ring as one tiled conversion go out together, the others
    // one by one as tacaw_push_frames does them
    std::vector<int> grouped;
    for (int i = 0; i < n; ++i) {
        const UserStream &u = p->us[stream_ids[i]];
        const Stream &s = p->s[u.first];
        const bool ok = split && u.N <= 1 && u.pushed >= u.skip && !s.due && s.staged + n_frames[i] <= s.ring &&
                        convert_split_groupable(p->bf, s.staged, n_frames[i]);
        if (ok) {
            grouped.push_back(i);
        } else {
            c = push_user(p, stream_ids[i], static_cast<const float2 *>(d_frames[i]), n_frames[i], st);
            if (c != TACAW_OK) return c;
        }
    }
    for (size_t g0 = 0; g0 < grouped.size(); g0 += kConvGroupMax) {
        ConvGroup cg{};
        cg.n = (int)std::min(grouped.size() - g0, (size_t)kConvGroupMax);
        for (int k = 0; k < cg.n; ++k) {
            const int i = grouped[g0 + k];
            Stream &s = p->s[p->us[stream_ids[i]].first];
            ConvEntry &e = cg.e[k];
            e.g.base = static_cast<const float2 *>(d_frames[i]);
            e.g.pitch_row = s.d.pitch_row;
            e.g.pitch_frame = s.d.pitch_frame;
            e.g.pitch_probe = s.d.pitch_probe;
            e.g.roi_x0 = s.d.roi_x0;
            e.g.roi_y0 = s.d.roi_y0;
            e.g.kx = s.d.kx;
            e.g.ky = s.d.ky;
            e.g.npix = s.npix;
            e.g.M = s.M;
            e.n = n_frames[i];
            e.s0 = s.staged;
            e.M_pad = s.M_pad;
            e.mu_hat = s.mu_hat;
            e.sum_res = s.sum_res;
            e.A_hi = s.A_hi;
            e.A_lo = s.A_lo;
            if (s.pushed == 0 && s.d.subtract_mean) {
                CU_CHECK(p, launch_mean(e.g, e.n, s.mu_hat, st), "provisional mean");
                p->launches++;
            }
        }
        CU_CHECK(p, launch_convert_split_group(cg, p->bf, 1, p->f16, p->f16_scale, p->d_err, st), "convert (group)");
        p->launches++;
        for (int k = 0; k < cg.n; ++k) {
            const int i = grouped[g0 + k];
            UserStream &u = p->us[stream_ids[i]];
            Stream &s = p->s[u.first];
            s.staged += n_frames[i];
            s.pushed += n_frames[i];
            u.pushed += n_frames[i];
            if (s.staged == s.ring && s.pushed < s.T) {
                s.due = true;     // deferrable: split, staged, one segment
                s.due_stream = st;
            }
        }
    }
    return TACAW_OK;
}

tacaw_status tacaw_finalize(tacaw_plan_t p, float *d_I, float *d_S, void *d_Psi, void *stream) {
    TraceRange trace_range("tacaw_finalize");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    tacaw_status r = finalize_impl(p, d_I, d_S, d_Psi, st);
    if (r != TACAW_OK) return r;
    if (p->pend.active) {
        r = launch_pending(p, nullptr, st);
        if (r != TACAW_OK) return r;
    }
    return read_device_error(p, st);
}

tacaw_status tacaw_drain(tacaw_plan_t p, void *stream) {
    TraceRange trace_range("tacaw_drain");
    tacaw_status c = check_plan(p);
    if (c != TACAW_OK) return c;
    if (p->deferred_pushes)
        return fail(TACAW_ERR_STATE, "the segment's pushes wait for the pending contraction: finalize the segment first");
    if (!p->pend.active) return TACAW_OK;
    return launch_pending(p, nullptr, static_cast<cudaStream_t>(stream));
}

tacaw_status tacaw_set_pipelined_segments(tacaw_plan_t p, int enable) {
    tacaw_status c = check_plan(p);
    if (c != TACAW_OK) return c;
    if (!enable) {
        if (p->pend.active || p->deferred_pushes)
            return fail(TACAW_ERR_STATE, "a segment's contraction is deferred: call tacaw_drain first");
        p->pipe = false;
        return TACAW_OK;
    }
    if (p->pipe) return TACAW_OK;
    if (p->us.size() != 1 || p->s.size() != 1)
        return fail(TACAW_ERR_UNSUPPORTED, "pipelined segments: one stream without Welch averaging");
    Stream &s = p->s[0];
    if (p->prec != TACAW_PREC_SPLIT_BF16 || p->f16 || p->in_place || p->bf != 32)
        return fail(TACAW_ERR_UNSUPPORTED, "pipelined segments: staged split-BF16 plans with 32-frame blocks");
    if (s.T % 32 || s.ring < s.T)
        return fail(TACAW_ERR_UNSUPPORTED, "pipelined segments: T a multiple of 32 and K_stage >= T (one flush a segment)");
    if (s.pushed != 0) return fail(TACAW_ERR_STATE, "pipelined segments: enable between segments");
    if (!s.A_hi2) {
        const size_t na = (size_t)(s.ring / p->bf) * s.M_pad * 2 * p->bf;
        if (!dev_alloc(p, &s.A_hi2, na) || !dev_alloc(p, &s.A_lo2, na) || !dev_alloc(p, &s.mu_hat2, s.M) ||
            !dev_alloc(p, &s.dmu2, s.M) || !dev_alloc(p, &s.sum_res2, s.M))
            return fail(TACAW_ERR_OOM, "cudaMalloc(second staging area of %.1f GB)", 2.0 * na * 2 / 1e9);
        CU_CHECK(p, cudaMemset(s.A_hi2, 0, na * sizeof(__nv_bfloat16)), "memset staging");
        CU_CHECK(p, cudaMemset(s.A_lo2, 0, na * sizeof(__nv_bfloat16)), "memset staging");
        CU_CHECK(p, cudaMemset(s.sum_res2, 0, sizeof(double2) * s.M), "memset sums");
        CU_CHECK(p, cudaMemset(s.mu_hat2, 0, sizeof(float2) * s.M), "memset mean");
    }
    if (!s.d_frame_ptr && !dev_alloc(p, &s.d_frame_ptr, (size_t)s.T))
        return fail(TACAW_ERR_OOM, "cudaMalloc(frame table)");
    p->pipe = true;
    return TACAW_OK;
}

tacaw_status tacaw_finalize_async(tacaw_plan_t p, float *d_I, float *d_S, void *d_Psi, void *stream) {
    TraceRange trace_range("tacaw_finalize_async");
    return finalize_impl(p, d_I, d_S, d_Psi, static_cast<cudaStream_t>(stream));
}

tacaw_status tacaw_check_errors(tacaw_plan_t p, void *stream) {
    TraceRange trace_range("tacaw_check_errors");
    tacaw_status c = check_plan(p);
    if (c != TACAW_OK) return c;
    return read_device_error(p, static_cast<cudaStream_t>(stream));
}

tacaw_status tacaw_output_offsets(tacaw_plan_t p, int sid, int64_t *I_offset, int64_t *S_offset) {
    if (!p) return fail(TACAW_ERR_INVALID_ARG, "plan is NULL");
    if (sid < 0 || sid >= (int)p->us.size()) return fail(TACAW_ERR_INVALID_ARG, "stream_id out of range");
    if (I_offset) *I_offset = p->us[sid].I_off;
    if (S_offset) *S_offset = p->us[sid].S_off;
    return TACAW_OK;
}

tacaw_status tacaw_reset(tacaw_plan_t p, void *stream) {
    TraceRange trace_range("tacaw_reset");
    tacaw_status c = check_plan(p);
    if (c != TACAW_OK) return c;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (auto &s : p->s) {
        CU_CHECK(p, cudaMemsetAsync(s.sum_res, 0, sizeof(double2) * s.M, st), "reset sums");
        CU_CHECK(p, cudaMemsetAsync(s.mu_hat, 0, sizeof(float2) * s.M, st), "reset mean");
        s.pushed = s.staged = s.stage_start = s.flushes = 0;
        s.seg = s.lane;
        s.due = false;
    }
    for (auto &u : p->us) {
        u.pushed = 0;
        if (u.I_acc) CU_CHECK(p, cudaMemsetAsync(u.I_acc, 0, sizeof(float) * u.I_elems, st), "reset Welch average");
    }
    p->deferred_pushes = false;
    p->finalized = false;
    return TACAW_OK;
}

tacaw_status tacaw_plan_get_info(tacaw_plan_t p, tacaw_plan_info *info) {
    if (!p || !info) return fail(TACAW_ERR_INVALID_ARG, "NULL argument");
    info->device_bytes = p->bytes;
    info->k_stage = p->k_stage;
    info->n_streams = (int)p->us.size();
    info->precision = p->prec_user;
    info->I_elems = p->I_elems;
    info->S_elems = p->S_elems;
    info->flushes = p->flushes_total;
    info->omega_tile = p->s.empty() ? 0 : p->s[0].wt;
    info->stages = p->stages;
    info->kernel_launches = p->launches;
    info->tc_block_frames = p->prec == TACAW_PREC_SPLIT_BF16 ? p->bf : 0;
    info->tuned_streams = p->tuned_streams;
    info->tune_candidates = p->tune_timed;
    info->tune_ms = p->tune_ms;
    info->frames_in_place = p->in_place ? 1 : 0;
    info->tc_drain_frames = p->prec == TACAW_PREC_SPLIT_BF16 ? p->drain_kb * p->bf : 0;
    info->accum = p->accum;
    info->flush_launches = p->flush_launches;
    info->aperture_pixels = p->s.empty() ? 0 : p->s[0].n_adj;
    return TACAW_OK;
}

tacaw_status tacaw_set_wait_limit_ns(tacaw_plan_t p, uint64_t limit_ns) {
    tacaw_status c = check_plan(p);
    if (c != TACAW_OK) return c;
    p->wait_ns = limit_ns == 0 ? 0 : std::max<uint64_t>(limit_ns, 1000);
    return TACAW_OK;
}

tacaw_status tacaw_set_timing(tacaw_plan_t p, int enable) {
    if (!p) return fail(TACAW_ERR_INVALID_ARG, "plan is NULL");
    p->timing = enable != 0;
    p->trace = enable >= 2;
    return TACAW_OK;
}

tacaw_status tacaw_flush_trace(tacaw_plan_t p, unsigned long long *host_out, int64_t max_ctas, int64_t *n_ctas) {
    if (!p) return fail(TACAW_ERR_INVALID_ARG, "plan is NULL");
    if (n_ctas) *n_ctas = p->trace_ctas;
    if (!host_out || !p->d_trace || p->trace_ctas == 0) return TACAW_OK;
    const int64_t n = std::min(max_ctas, p->trace_ctas);
    if (n <= 0) return TACAW_OK;
    cudaError_t e = cudaMemcpy(host_out, p->d_trace, sizeof(unsigned long long) * kTraceWords * n,
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(p, e, "copy trace");
    return TACAW_OK;
}

tacaw_status tacaw_kernel_time_ms(tacaw_plan_t p, double *flush_ms, int64_t *flush_launches, int reset) {
    if (!p) return fail(TACAW_ERR_INVALID_ARG, "plan is NULL");
    for (auto &e : p->ev) {
        cudaError_t r = cudaEventSynchronize(e.second);
        if (r != cudaSuccess) return cuda_fail(p, r, "cudaEventSynchronize");
        float ms = 0.f;
        r = cudaEventElapsedTime(&ms, e.first, e.second);
        if (r != cudaSuccess) return cuda_fail(p, r, "cudaEventElapsedTime");
        p->timed_ms += ms;
        p->timed_launches++;
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    p->ev.clear();
    if (flush_ms) *flush_ms = p->timed_ms;
    if (flush_launches) *flush_launches = p->timed_launches;
    if (reset) {
        p->timed_ms = 0.0;
        p->timed_launches = 0;
    }
    return TACAW_OK;
}

tacaw_status tacaw_destroy(tacaw_plan_t p) {
    TraceRange trace_range("tacaw_destroy");
    if (!p) return TACAW_OK;
    free_all(p);
    delete p;
    return TACAW_OK;
}

}  // extern "C"
