// Host-side state of a plan (tacaw_api.cu, tacaw_backward.cu, tacaw_state.cu): the internal
// streams with their device buffers and segment counters, the streams as the caller sees them
// (Welch lanes), the plan, and the helpers the three files share.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/tacaw.h"
#include "tacaw_internal.cuh"

namespace tacaw {

struct Stream {
    tacaw_stream_desc d{};
    std::vector<double> E;
    std::vector<tacaw_detector> dets;
    int64_t npix = 0, M = 0, M_pad = 0;
    int T = 0, T_pad = 0, n_kb_T = 0;
    int Nw = 0, wt = 0, n_wt = 0, Nw_pad = 0;
    int ring = 0;                    // frames the staging ring holds: min(K_stage, T_pad)
    bool needs_acc = false;
    // device buffers
    float2 *mu_hat = nullptr, *dmu = nullptr, *Wc = nullptr;
    double2 *sum_res = nullptr;
    double *cj = nullptr;
    float *bose = nullptr, *win = nullptr;
    __nv_bfloat16 *A_hi = nullptr, *A_lo = nullptr, *B_hi = nullptr, *B_lo = nullptr;
    float2 *A32 = nullptr, *B32 = nullptr;
    float2 *acc_s = nullptr, *acc_c = nullptr;
    double2 *acc_d = nullptr;
    int *det_idx = nullptr, *det_off = nullptr;
    float *det_w = nullptr;
    int D = 0, n_det_entries = 0;
    std::vector<int> h_det_off;
    // adjoint support: pixels inside any aperture and their per-detector weights
    int *adj_pix = nullptr;
    float *adj_w = nullptr;
    int n_adj = 0;
    // tensor-core adjoint tables, built by the stream's first tacaw_backward: forward twiddles in
    // 32-frame blocks (energy tiles wt1), conj twiddles with frames as columns (frame tiles wt2)
    __nv_bfloat16 *adjF_hi = nullptr, *adjF_lo = nullptr, *adjC_hi = nullptr, *adjC_lo = nullptr;
    float2 *adj_ones = nullptr;
    float *adj_ones_f = nullptr;
    int64_t *adj_off = nullptr;      // element offset of each aperture pixel within a frame
    std::vector<int> h_adj_pix;      // host copy of adj_pix
    // pipelined segments (tacaw_set_pipelined_segments): the second staging area and per-row
    // buffers, swapped with the first at each deferred finalize
    __nv_bfloat16 *A_hi2 = nullptr, *A_lo2 = nullptr;
    float2 *mu_hat2 = nullptr, *dmu2 = nullptr;
    double2 *sum_res2 = nullptr;
    int adj_wt1 = 0, adj_nwt1 = 0, adj_wt2 = 0, adj_nwt2 = 0;
    int stages = 0;            // shared-memory pipeline stages of this stream's tiles
    double *win_table = nullptr;   // table-driven windows (Dolph-Chebyshev)
    // Welch lanes: internal stream `lane` of user stream `user` runs segments lane, lane +
    // lanes, ... one after another; its last flush adds out_scale * I into the user's average
    int user = 0, lane = 0;
    int64_t seg = 0;           // current segment of this lane
    float out_scale = 1.f;
    int out_add = 0;
    bool tuned = false;        // tile picked by the autotuner
    // in-place frames: per staged frame, a pointer into the pushed buffer
    // host record of the segment's pushes (first frame, address): a flush whose frames are
    // evenly spaced reads them through one 2-D tensor map
    std::vector<std::pair<int, const float2 *>> h_pushes;
    const float2 **d_frame_ptr = nullptr;       // one slot per frame of the segment, written on
                                                // the stream at push time (no host copy)
    // segment state
    int pushed = 0, staged = 0, stage_start = 0, flushes = 0;
    // a full staging ring whose flush waits for the next push of this stream (or of finalize),
    // so that the flushes of several streams that fill up together share one launch
    bool due = false;
    cudaStream_t due_stream = nullptr;
    int64_t I_off = 0, S_off = 0;
};

}  // namespace tacaw

// A stream as the caller sees it: one internal stream, or the lanes of a Welch average.
struct UserStream {
    int first = 0, lanes = 1;  // internal streams [first, first + lanes)
    int N = 1, stride = 0, L = 0;
    int64_t total = 0;         // frames of the whole push sequence: skip + (N - 1) * stride + L
    int64_t skip = 0;          // leading frames dropped before the first segment
    int64_t pushed = 0;
    float *I_acc = nullptr;    // Welch: plan-owned running average of the segments' I
    int64_t I_elems = 0;
    int64_t I_off = 0, S_off = 0;
};

struct tacaw_plan_s {
    std::vector<tacaw::Stream> s;     // internal streams (Welch lanes expanded)
    std::vector<UserStream> us;
    int prec = 0, accum = 0, k_stage = 0;   // prec: TACAW_PREC_SPLIT_BF16 for both split paths
    int prec_user = 0;         // the precision asked for (tacaw_plan_info)
    int f16 = 0;               // split path with fp16 pieces of the scaled operands
    float f16_scale = 1.f;     // split FP16: operand A is f16_scale * (psi - mu_hat), a power of two
    int stages = 0;
    int drain_kb = 0;          // split path: staging blocks per drained H chunk
    int bf = 8;                // frames per staged operand row (split path)
    bool in_place = false;     // the contraction reads pushed frames directly (in-place kernel)
    int tc_max_ctas = 0;       // persistent contraction grids: at most this many CTAs (0: all SMs)
    uint64_t wait_ns = 0;      // tensor-core pipeline waits give up after this (0: the kernels' default)
    // with a capped grid the last flush runs on a highest-priority stream of the plan, forked
    // from and joined back to the caller's stream, so that its CTAs take SMs ahead of other
    // streams' queued work
    cudaStream_t hp_stream = nullptr;
    cudaEvent_t hp_in = nullptr, hp_out = nullptr;
    // tacaw_backward's streams: the gradient's zero fill (HBM-bound) runs on aux_stream beside the
    // tensor-core adjoint's contractions, which run on adj_stream at the greatest priority (freed
    // SMs go to their CTAs ahead of the fill's blocks)
    cudaStream_t aux_stream = nullptr, adj_stream = nullptr;
    cudaEvent_t aux_in = nullptr, aux_out = nullptr, adj_out = nullptr;
    int64_t bytes = 0;
    int64_t I_elems = 0, S_elems = 0;
    int64_t flushes_total = 0;
    int64_t launches = 0;
    int64_t flush_launches = 0;    // contraction launches (a grouped launch counts once)
    bool poisoned = false;
    bool finalized = false;
    uint32_t *d_err = nullptr;
    // tile counters of the staged kernel's launches: one per launch in a ring, so that launches of
    // this plan on different CUDA streams (up to kCounterRing of them in flight) never share one
    int *d_counters = nullptr;
    int64_t counter_slot = 0;
    // the adjoint's G matrix and row means: allocated by the first tacaw_backward that needs it
    // (grown when a later stream needs more), kept until tacaw_destroy
    float2 *adj_scratch = nullptr;
    size_t adj_scratch_elems = 0;
    // the tensor-core adjoint's staged operands and intermediates (same lifetime as adj_scratch)
    void *adj_tc = nullptr;
    size_t adj_tc_bytes = 0;
    bool adj_fp32 = false;     // tacaw_set_adjoint_precision(TACAW_PREC_FP32): CUDA-core adjoint
    // pipelined segments: a finalized segment's contraction is deferred and launched with the
    // conversion of the next segment's pushes (done by extra warps of the same launch)
    bool pipe = false;
    bool deferred_pushes = false;  // this segment's pushes were recorded, not converted
    struct Pending {
        bool active = false;
        tacaw::Stream snap;                   // the deferred segment (its staging slot, sums, lists)
        float *I = nullptr, *S = nullptr;
        float2 *Psi = nullptr;
    } pend;
    std::vector<void *> allocs;
    bool timing = false;
    bool trace = false;                      // record per-CTA phase stamps of tensor-core flushes
    unsigned long long *d_trace = nullptr;   // stamps of the last traced flush
    int64_t trace_ctas = 0, trace_cap = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    double timed_ms = 0.0;
    int64_t timed_launches = 0;
    int tuned_streams = 0, tune_timed = 0;
    double tune_ms = 0.0;
};

namespace tacaw {

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Sets the calling thread's last error (and the log sink) and returns st.
tacaw_status fail(tacaw_status st, const char *fmt, ...);
// A failed CUDA call: poisons the plan and returns TACAW_ERR_CUDA.
tacaw_status cuda_fail(tacaw_plan_s *p, cudaError_t e, const char *what);
tacaw_status check_plan(tacaw_plan_s *p);
// Buffers a kernel reads or writes: device, managed or mapped pinned host memory (see the definition).
tacaw_status check_kernel_memory(const void *ptr, const char *what, bool allow_host, cudaStream_t st);
// Waits for `st` and turns the device error word into a status (poisoning the plan).
tacaw_status read_device_error(tacaw_plan_s *p, cudaStream_t st);
// Table arguments of stream s after its tables were built.
TableArgs stream_table_args(const Stream &s, int block_frames);

// A named range on the profiler timeline (NVTX: costs a test of a null function pointer unless
// a tool such as Nsight Systems is attached), from construction to the end of the scope.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

// Device allocation of `count` elements owned by the plan (freed by tacaw_destroy).
template <typename T>
bool dev_alloc(tacaw_plan_s *p, T **ptr, size_t count) {
    *ptr = nullptr;
    if (count == 0) count = 1;
    void *q = nullptr;
    if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    p->allocs.push_back(q);
    p->bytes += (int64_t)(count * sizeof(T));
    *ptr = static_cast<T *>(q);
    return true;
}

}  // namespace tacaw

#define CU_CHECK(plan, call, what)                                      \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return cuda_fail((plan), e_, (what));    \
    } while (0)
