// tacaw_backward and tacaw_set_adjoint_precision: the adjoint of the forward path (the chain
// rule through Eq. 1, the windowed transform and the detector sum) on one stream's segment,
// on the tensor cores (split BF16: Psi recomputed on the aperture rows, G, back-projection with
// the conjugate twiddles) or on FP32 CUDA cores.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/tacaw.h"
#include "tacaw_internal.cuh"
#include "tacaw_plan.cuh"

using namespace tacaw;

extern "C" {

namespace {

// Output-column tile of an adjoint contraction over row_tiles row tiles: the multiple of 8 (at
// most wt_max) with the least cost in rounds of the persistent grid (one tile per SM a round)
// times columns plus a fixed per-tile cost, as in least_cost_tile.
int adjoint_tile(int n_cols, int64_t row_tiles, int sms, int wt_max) {
    int best = 8;
    int64_t best_cost = INT64_MAX;
    for (int wt = 8; wt <= wt_max; wt += 8) {
        const int64_t tiles = row_tiles * ((n_cols + wt - 1) / wt);
        const int64_t cost = (tiles + sms - 1) / sms * (wt + 24);
        if (cost < best_cost || (cost == best_cost && wt > best)) {
            best_cost = cost;
            best = wt;
        }
    }
    return best;
}

// Tables of the tensor-core adjoint for stream s, built on its first backward: the forward
// twiddles in 32-frame blocks with least-padding energy tiles, and the conj twiddles with the
// frames as output columns in least-padding frame tiles.
tacaw_status adjoint_tc_tables(tacaw_plan_s *p, Stream &s, cudaStream_t st) {
    if (s.adjF_hi) return TACAW_OK;
    const int wt_max = kDrainMaxOmegaTile;
    int dev = 0, sms = 0;
    CU_CHECK(p, cudaGetDevice(&dev), "cudaGetDevice");
    CU_CHECK(p, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    const int64_t row_tiles = round_up((int64_t)s.d.n_probes * s.n_adj, kMTile) / kMTile;
    s.adj_wt1 = adjoint_tile(s.Nw, row_tiles, std::max(1, sms), wt_max);
    s.adj_nwt1 = (s.Nw + s.adj_wt1 - 1) / s.adj_wt1;
    s.adj_wt2 = adjoint_tile(s.T, row_tiles, std::max(1, sms), wt_max);
    s.adj_nwt2 = (s.T + s.adj_wt2 - 1) / s.adj_wt2;
    const int T_pad = (int)round_up(s.T, 32), E_pad = (int)round_up(s.Nw, 32);
    const int Nw_rows = s.adj_wt1 * s.adj_nwt1, T_rows = s.adj_wt2 * s.adj_nwt2;
    const size_t nf = (size_t)(T_pad / 32) * 2 * Nw_rows * 64, nc = (size_t)(E_pad / 32) * 2 * T_rows * 64;
    __nv_bfloat16 *fh, *fl, *ch, *cl;
    float2 *ones;
    float *ones_f;
    int64_t *off;
    if (!dev_alloc(p, &fh, nf) || !dev_alloc(p, &fl, nf) || !dev_alloc(p, &ch, nc) || !dev_alloc(p, &cl, nc) ||
        !dev_alloc(p, &ones, (size_t)T_rows) || !dev_alloc(p, &ones_f, (size_t)T_rows) ||
        !dev_alloc(p, &off, (size_t)s.n_adj))
        return fail(TACAW_ERR_OOM, "cudaMalloc(adjoint tables)");
    {
        const std::vector<int> &pix = s.h_adj_pix;
        std::vector<int64_t> o((size_t)s.n_adj);
        for (int i = 0; i < s.n_adj; ++i)
            o[i] = (int64_t)(s.d.roi_y0 + pix[i] / s.d.kx) * s.d.pitch_row + (s.d.roi_x0 + pix[i] % s.d.kx);
        CU_CHECK(p, cudaMemcpy(off, o.data(), sizeof(int64_t) * s.n_adj, cudaMemcpyHostToDevice), "copy offsets");
    }
    TableArgs ta = stream_table_args(s, 32);
    ta.T_pad = T_pad;
    ta.Nw_pad = Nw_rows;
    CU_CHECK(p, launch_twiddles_split(ta, fh, fl, 0, st), "adjoint twiddles");
    CU_CHECK(p, launch_twiddles_adjoint_split(ta, T_rows, E_pad, ch, cl, st), "adjoint conj twiddles");
    std::vector<float2> h1((size_t)T_rows, make_float2(1.f, 0.f));
    std::vector<float> h2((size_t)T_rows, 1.f);
    CU_CHECK(p, cudaMemcpy(ones, h1.data(), sizeof(float2) * T_rows, cudaMemcpyHostToDevice), "copy ones");
    CU_CHECK(p, cudaMemcpy(ones_f, h2.data(), sizeof(float) * T_rows, cudaMemcpyHostToDevice), "copy ones");
    s.adjF_hi = fh;
    s.adjF_lo = fl;
    s.adjC_hi = ch;
    s.adjC_lo = cl;
    s.adj_ones = ones;
    s.adj_ones_f = ones_f;
    s.adj_off = off;
    return TACAW_OK;
}

// Carves the tensor-core adjoint's buffers for stream s out of the plan's scratch (grown, never
// shrunk, kept until tacaw_destroy).  q.a must be filled.
tacaw_status adjoint_tc_scratch(tacaw_plan_s *p, const Stream &s, AdjTcArgs &q) {
    const int64_t M = (int64_t)s.d.n_probes * s.n_adj;
    q.M_pad = round_up(M, kMTile);
    q.T_pad = (int)round_up(s.T, 32);
    q.E_pad = (int)round_up(s.Nw, 32);
    const size_t a_piece = (size_t)q.T_pad * q.M_pad * 4, g_piece = (size_t)q.E_pad * q.M_pad * 4;
    const size_t sizes[10] = {a_piece, a_piece, g_piece, g_piece,
                              (size_t)(std::max(q.T_pad, q.E_pad) / 32) * M * sizeof(float2),
                              (size_t)M * sizeof(float2), (size_t)M * sizeof(float2),
                              (size_t)M * s.Nw * sizeof(float2), (size_t)M * s.T * sizeof(float2), 2 * sizeof(int)};
    size_t off[10], total = 0;
    for (int i = 0; i < 10; ++i) {
        off[i] = total;
        total += (sizes[i] + 255) & ~(size_t)255;
    }
    if (total > p->adj_tc_bytes) {
        // the previous backward ended with a synchronize, so the old buffer is idle
        if (p->adj_tc) {
            cudaFree(p->adj_tc);
            p->bytes -= (int64_t)p->adj_tc_bytes;
        }
        p->adj_tc = nullptr;
        p->adj_tc_bytes = 0;
        void *b = nullptr;
        if (cudaMalloc(&b, total) != cudaSuccess) {
            cudaGetLastError();
            return fail(TACAW_ERR_OOM, "tensor-core adjoint scratch of %zu bytes", total);
        }
        p->adj_tc = b;
        p->adj_tc_bytes = total;
        p->bytes += (int64_t)total;
    }
    uint8_t *b = static_cast<uint8_t *>(p->adj_tc);
    q.A_hi = reinterpret_cast<__nv_bfloat16 *>(b + off[0]);
    q.A_lo = reinterpret_cast<__nv_bfloat16 *>(b + off[1]);
    q.G_hi = reinterpret_cast<__nv_bfloat16 *>(b + off[2]);
    q.G_lo = reinterpret_cast<__nv_bfloat16 *>(b + off[3]);
    q.part = reinterpret_cast<float2 *>(b + off[4]);
    q.dmu = reinterpret_cast<float2 *>(b + off[5]);
    q.kmean = reinterpret_cast<float2 *>(b + off[6]);
    q.psi = reinterpret_cast<float2 *>(b + off[7]);
    q.cg = reinterpret_cast<float2 *>(b + off[8]);
    q.counters = reinterpret_cast<int *>(b + off[9]);
    q.Bf_hi = s.adjF_hi;
    q.Bf_lo = s.adjF_lo;
    q.wt1 = s.adj_wt1;
    q.n_wt1 = s.adj_nwt1;
    q.Bc_hi = s.adjC_hi;
    q.Bc_lo = s.adjC_lo;
    q.wt2 = s.adj_wt2;
    q.n_wt2 = s.adj_nwt2;
    q.ones = s.adj_ones;
    q.ones_f = s.adj_ones_f;
    q.pix_off = s.adj_off;
    q.err = p->d_err;
    q.wait_ns = p->wait_ns;
    return TACAW_OK;
}

}  // namespace

tacaw_status tacaw_set_adjoint_precision(tacaw_plan_t p, int precision) {
    tacaw_status c = check_plan(p);
    if (c != TACAW_OK) return c;
    if (precision == TACAW_PREC_SPLIT_BF16)
        p->adj_fp32 = false;
    else if (precision == TACAW_PREC_FP32)
        p->adj_fp32 = true;
    else
        return fail(TACAW_ERR_INVALID_ARG, "adjoint precision %d: TACAW_PREC_SPLIT_BF16 or TACAW_PREC_FP32", precision);
    return TACAW_OK;
}

tacaw_status tacaw_backward(tacaw_plan_t p, int sid, const float *d_dL_dS, const void *d_frames, void *d_grad,
                            void *stream) {
    TraceRange trace_range("tacaw_backward");
    tacaw_status c = check_plan(p);
    if (c != TACAW_OK) return c;
    if (sid < 0 || sid >= (int)p->us.size()) return fail(TACAW_ERR_INVALID_ARG, "stream_id %d out of range", sid);
    if (!d_dL_dS || !d_frames || !d_grad) return fail(TACAW_ERR_INVALID_ARG, "NULL device pointer");
    {
        cudaStream_t cs = static_cast<cudaStream_t>(stream);
        tacaw_status k = check_kernel_memory(d_frames, "d_frames", true, cs);
        if (k == TACAW_OK) k = check_kernel_memory(d_grad, "d_grad", true, cs);
        if (k == TACAW_OK) k = check_kernel_memory(d_dL_dS, "d_dL_dS", true, cs);
        if (k != TACAW_OK) return k;
    }
    const UserStream &u = p->us[sid];
    Stream &s = p->s[u.first];
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    AdjointArgs a{};
    a.frames = static_cast<const float2 *>(d_frames);
    a.pitch_row = s.d.pitch_row;
    a.pitch_frame = s.d.pitch_frame;
    a.pitch_probe = s.d.pitch_probe;
    a.roi_x0 = s.d.roi_x0;
    a.roi_y0 = s.d.roi_y0;
    a.kx = s.d.kx;
    a.ky = s.d.ky;
    a.P = s.d.n_probes;
    a.T = s.T;
    a.Nw = s.Nw;
    a.D = s.D;
    a.subtract_mean = s.d.subtract_mean;
    a.w = s.win;
    a.B32 = s.B32;
    a.Nw_pad = s.Nw_pad;
    a.Wc = s.Wc;
    a.bose = s.bose;
    a.dLdS = d_dL_dS;
    a.mpix = s.adj_pix;
    a.mwts = s.adj_w;
    a.n_mpix = s.n_adj;
    a.grad = static_cast<float2 *>(d_grad);
    a.scale = 1.f;
    a.accumulate = 0;
    // the whole push sequence's gradient: skipped frames and frames of no segment get zero
    AdjointArgs z = a;
    z.T = (int)u.total;
    const bool tc = s.n_adj > 0 && s.D > 0 && !p->adj_fp32;
    if (!tc) {
        CU_CHECK(p, launch_zero_roi(z, st), "zero gradient");
        p->launches++;
    }
    if (tc) {
        // tensor cores, split BF16: one segment, or each Welch segment at its start frame with
        // weight 1/N, its gradient added where segments overlap
        tacaw_status r = adjoint_tc_tables(p, s, st);
        if (r != TACAW_OK) return r;
        AdjTcArgs q{};
        q.a = a;
        r = adjoint_tc_scratch(p, s, q);
        if (r != TACAW_OK) return r;
        // the zero fill runs on a side stream beside the contractions (it needs the SMs' memory
        // pipes, they the tensor cores), the contractions on a stream of the greatest priority;
        // the first scatter into the gradient waits for the fill, the caller's stream for both
        if (!p->aux_stream) {
            int lo = 0, hi = 0;
            CU_CHECK(p, cudaDeviceGetStreamPriorityRange(&lo, &hi), "stream priorities");
            CU_CHECK(p, cudaStreamCreateWithPriority(&p->aux_stream, cudaStreamNonBlocking, lo), "adjoint fill stream");
            CU_CHECK(p, cudaStreamCreateWithPriority(&p->adj_stream, cudaStreamNonBlocking, hi), "adjoint stream");
            CU_CHECK(p, cudaEventCreateWithFlags(&p->aux_in, cudaEventDisableTiming), "cudaEventCreate");
            CU_CHECK(p, cudaEventCreateWithFlags(&p->aux_out, cudaEventDisableTiming), "cudaEventCreate");
            CU_CHECK(p, cudaEventCreateWithFlags(&p->adj_out, cudaEventDisableTiming), "cudaEventCreate");
        }
        CU_CHECK(p, cudaEventRecord(p->aux_in, st), "cudaEventRecord");
        CU_CHECK(p, cudaStreamWaitEvent(p->aux_stream, p->aux_in, 0), "cudaStreamWaitEvent");
        CU_CHECK(p, cudaStreamWaitEvent(p->adj_stream, p->aux_in, 0), "cudaStreamWaitEvent");
        CU_CHECK(p, launch_zero_roi(z, p->aux_stream), "zero gradient");
        CU_CHECK(p, cudaEventRecord(p->aux_out, p->aux_stream), "cudaEventRecord");
        p->launches++;
        q.before_scatter = p->aux_out;
        cudaStream_t cst = p->adj_stream;
        const int nseg = u.N > 1 ? u.N : 1;
        cudaError_t e = cudaSuccess;
        for (int n = 0; n < nseg && e == cudaSuccess; ++n) {
            const int64_t f0 = u.skip + (int64_t)n * u.stride;
            AdjTcArgs qn = q;
            qn.a.frames = a.frames + f0 * s.d.pitch_frame;
            qn.a.grad = a.grad + f0 * s.d.pitch_frame;
            qn.a.scale = 1.f / (float)nseg;
            qn.a.accumulate = nseg > 1 ? 1 : 0;
            e = launch_adjoint_tc(qn, cst);
            p->launches += adjtc_launches();
        }
        if (e != cudaSuccess) return cuda_fail(p, e, "tensor-core adjoint");
        CU_CHECK(p, cudaEventRecord(p->adj_out, cst), "cudaEventRecord");
        CU_CHECK(p, cudaStreamWaitEvent(st, p->adj_out, 0), "cudaStreamWaitEvent");
    } else if (s.n_adj > 0 && s.D > 0) {
        const size_t n_scr = (size_t)s.d.n_probes * s.n_adj * (s.Nw + 2);
        if (n_scr > p->adj_scratch_elems) {
            // the previous call ended with a synchronize, so the old buffer is idle
            if (p->adj_scratch) {
                cudaFree(p->adj_scratch);
                p->bytes -= (int64_t)(p->adj_scratch_elems * sizeof(float2));
            }
            p->adj_scratch = nullptr;
            p->adj_scratch_elems = 0;
            void *q = nullptr;
            if (cudaMalloc(&q, n_scr * sizeof(float2)) != cudaSuccess) {
                cudaGetLastError();
                return fail(TACAW_ERR_OOM, "adjoint scratch of %zu bytes", n_scr * sizeof(float2));
            }
            p->adj_scratch = static_cast<float2 *>(q);
            p->adj_scratch_elems = n_scr;
            p->bytes += (int64_t)(n_scr * sizeof(float2));
        }
        a.scratch = p->adj_scratch;
        // one segment, or each Welch segment at its start frame with weight 1/N, its gradient
        // added where segments overlap (one segment stores over the zeros, no read-back)
        const int nseg = u.N > 1 ? u.N : 1;
        cudaError_t e = cudaSuccess;
        for (int n = 0; n < nseg && e == cudaSuccess; ++n) {
            const int64_t f0 = u.skip + (int64_t)n * u.stride;
            AdjointArgs an = a;
            an.frames = a.frames + f0 * s.d.pitch_frame;
            an.grad = a.grad + f0 * s.d.pitch_frame;
            an.scale = 1.f / (float)nseg;
            an.accumulate = nseg > 1 ? 1 : 0;
            e = launch_adjoint(an, st);
            p->launches += 2;
        }
        if (e != cudaSuccess) return cuda_fail(p, e, "adjoint");
    }
    return read_device_error(p, st);
}

}  // extern "C"
