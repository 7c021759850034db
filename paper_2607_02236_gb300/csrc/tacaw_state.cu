// tacaw_state_size, tacaw_save_state, tacaw_restore_state: checkpoints of a segment in progress.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/tacaw.h"
#include "tacaw_internal.cuh"
#include "tacaw_plan.cuh"

using namespace tacaw;

namespace {

// Checkpoints (tacaw_save_state).  The accumulation of a segment is a sum over its pushed
// frames, so between two pushes a plan's progress is a handful of buffers: the provisional
// means and FP64 residual sums, the staged frames not yet contracted, the running Psi
// accumulators once a flush has written them, and the Welch averages.  A checkpoint is a fixed
// header, the host counters of every stream, then those device sections in a fixed order;
// everything else a plan holds (tables, detector lists) follows from its descriptor, which the
// fingerprint ties to the checkpoint.
constexpr uint64_t kStateMagic = 0x314B435741434154ULL;   // the bytes "TACAWCK1"
constexpr uint32_t kStateVersion = 1;

struct StateHeader {
    uint64_t magic;
    uint32_t version;
    uint32_t n_streams;       // internal streams (Welch lanes counted one each)
    uint32_t n_user;
    uint32_t reserved;
    uint64_t fingerprint;     // plan_fingerprint of the saving plan
    int64_t total_bytes;      // the whole checkpoint
    uint64_t counters_hash;   // FNV-1a of the counter records that follow the header
};
struct StreamCounters {
    int64_t pushed, staged, stage_start, flushes, seg;
    int32_t due, reserved;
};
struct UserCounters {
    int64_t pushed;
};
static_assert(sizeof(StateHeader) == 48 && sizeof(StreamCounters) == 48 && sizeof(UserCounters) == 8,
              "checkpoint records are packed");

// 64-bit FNV-1a (Fowler, Noll and Vo): offset basis 0xcbf29ce484222325, prime 0x100000001b3.
struct Fnv {
    uint64_t h = 0xcbf29ce484222325ULL;
    void add(const void *ptr, size_t n) {
        const unsigned char *b = static_cast<const unsigned char *>(ptr);
        for (size_t i = 0; i < n; ++i) {
            h ^= b[i];
            h *= 0x100000001b3ULL;
        }
    }
    template <class V>
    void val(const V &v) { add(&v, sizeof v); }
};

// What the saved buffers' contents and layout depend on: precision, accumulators, staging
// geometry, the frames' ROI and the arithmetic of the tables (energies, window, time step,
// mean subtraction), and the Welch segmentation.  Tuning that does not change a saved layout
// (energy tiles, pipeline depth, CTA caps) is left out.
uint64_t plan_fingerprint(const tacaw_plan_s *p) {
    Fnv f;
    f.val(p->prec);
    f.val(p->prec_user);
    f.val(p->f16);
    f.val(p->f16_scale);
    f.val(p->accum);
    f.val(p->k_stage);
    f.val(p->bf);
    f.val((int)p->in_place);
    f.val((int)p->s.size());
    f.val((int)p->us.size());
    for (const Stream &s : p->s) {
        f.val(s.npix);
        f.val(s.M);
        f.val(s.M_pad);
        f.val(s.T);
        f.val(s.T_pad);
        f.val(s.Nw);
        f.val(s.ring);
        f.val((int)s.needs_acc);
        f.val(s.user);
        f.val(s.lane);
        f.val(s.d.n_probes);
        f.val(s.d.kx);
        f.val(s.d.ky);
        f.val(s.d.roi_x0);
        f.val(s.d.roi_y0);
        f.val(s.d.dt_fs);
        f.val(s.d.fft_bins);
        f.val(s.d.window);
        f.val(s.d.window_param);
        f.val(s.d.subtract_mean);
        f.val(s.d.bose_T_K);
        f.add(s.E.data(), sizeof(double) * s.E.size());
    }
    for (const UserStream &u : p->us) {
        f.val(u.first);
        f.val(u.lanes);
        f.val(u.N);
        f.val(u.stride);
        f.val(u.L);
        f.val(u.total);
        f.val(u.skip);
    }
    return f.h;
}

struct StateSection {
    void *dev;
    size_t bytes;
};

// Device sections of a checkpoint whose streams have the counters c, in checkpoint order.
std::vector<StateSection> state_sections(const tacaw_plan_s *p, const std::vector<StreamCounters> &c) {
    std::vector<StateSection> v;
    for (size_t i = 0; i < p->s.size(); ++i) {
        const Stream &s = p->s[i];
        v.push_back({s.mu_hat, sizeof(float2) * (size_t)s.M});
        v.push_back({s.sum_res, sizeof(double2) * (size_t)s.M});
        if (c[i].staged > 0) {
            // staged frames fill ring slots [0, staged): whole blocks of bf frames (split) or
            // frame-major rows of M_pad (FP32)
            if (p->prec == TACAW_PREC_SPLIT_BF16) {
                const size_t n = (size_t)((c[i].staged + p->bf - 1) / p->bf) * (size_t)s.M_pad * 2 * p->bf *
                                 sizeof(__nv_bfloat16);
                v.push_back({s.A_hi, n});
                v.push_back({s.A_lo, n});
            } else {
                v.push_back({s.A32, sizeof(float2) * (size_t)c[i].staged * (size_t)s.M_pad});
            }
        }
        if (s.needs_acc && c[i].flushes > 0) {
            const size_t n = (size_t)s.Nw * (size_t)s.M_pad;   // energies j < Nw, rows of M_pad
            if (s.acc_d) v.push_back({s.acc_d, sizeof(double2) * n});
            if (s.acc_s) v.push_back({s.acc_s, sizeof(float2) * n});
            if (s.acc_c) v.push_back({s.acc_c, sizeof(float2) * n});
        }
    }
    for (const UserStream &u : p->us)
        if (u.I_acc) v.push_back({u.I_acc, sizeof(float) * (size_t)u.I_elems});
    return v;
}

std::vector<StreamCounters> plan_counters(const tacaw_plan_s *p) {
    std::vector<StreamCounters> c(p->s.size());
    for (size_t i = 0; i < p->s.size(); ++i) {
        const Stream &s = p->s[i];
        c[i] = StreamCounters{s.pushed, s.staged, s.stage_start, s.flushes, s.seg, s.due ? 1 : 0, 0};
    }
    return c;
}

int64_t state_total(const tacaw_plan_s *p, const std::vector<StreamCounters> &c) {
    int64_t b = (int64_t)sizeof(StateHeader) + (int64_t)(sizeof(StreamCounters) * p->s.size()) +
                (int64_t)(sizeof(UserCounters) * p->us.size());
    for (const StateSection &x : state_sections(p, c)) b += (int64_t)x.bytes;
    return b;
}

tacaw_status check_saveable(const tacaw_plan_s *p) {
    if (p->finalized)
        return fail(TACAW_ERR_STATE, "segment finalized: nothing to resume (tacaw_reset starts the next)");
    if (p->pend.active || p->deferred_pushes)
        return fail(TACAW_ERR_STATE, "a segment's contraction is deferred: call tacaw_drain first");
    if (p->in_place)
        for (size_t i = 0; i < p->s.size(); ++i)
            if (p->s[i].staged > 0)
                return fail(TACAW_ERR_STATE,
                            "in-place stream %zu holds %d pushed frames not yet contracted (their addresses only): "
                            "checkpoint when the pushes fill whole K_stage rings",
                            i, p->s[i].staged);
    return TACAW_OK;
}

tacaw_status check_host_buffer(const void *buf, const char *what) {
    if (!buf) return fail(TACAW_ERR_INVALID_ARG, "%s is NULL", what);
    cudaPointerAttributes at{};
    const cudaError_t e = cudaPointerGetAttributes(&at, buf);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return TACAW_OK;   // unknown to CUDA: pageable host memory
    }
    if (at.type == cudaMemoryTypeDevice) return fail(TACAW_ERR_INVALID_ARG, "%s must be host memory", what);
    return TACAW_OK;
}

// Counters read from a checkpoint that this plan's pushes could have produced.
tacaw_status check_counters(const tacaw_plan_s *p, const std::vector<StreamCounters> &c,
                            const std::vector<UserCounters> &uc) {
    for (size_t i = 0; i < p->s.size(); ++i) {
        const Stream &s = p->s[i];
        const StreamCounters &k = c[i];
        const UserStream &u = p->us[s.user];
        const bool ok = k.pushed >= 0 && k.pushed <= s.T && k.staged >= 0 && k.staged <= s.ring &&
                        k.stage_start >= 0 && k.stage_start + k.staged == k.pushed && k.flushes >= 0 &&
                        k.flushes <= k.stage_start && (s.needs_acc || k.flushes == 0) &&
                        (!p->in_place || k.staged == 0) && (k.due == 0 || (k.due == 1 && k.staged == s.ring)) &&
                        k.seg >= s.lane && (k.seg - s.lane) % u.lanes == 0 &&
                        k.seg < s.lane + (int64_t)u.lanes * (u.N + 1);
        if (!ok) return fail(TACAW_ERR_INVALID_ARG, "checkpoint: counters of stream %zu are inconsistent", i);
    }
    for (size_t i = 0; i < p->us.size(); ++i)
        if (uc[i].pushed < 0 || uc[i].pushed > p->us[i].total)
            return fail(TACAW_ERR_INVALID_ARG, "checkpoint: frame count of stream %zu is out of range", i);
    return TACAW_OK;
}

}  // namespace

extern "C" {

tacaw_status tacaw_state_size(tacaw_plan_t p, int64_t *bytes) {
    tacaw_status c = check_plan(p);
    if (c != TACAW_OK) return c;
    if (!bytes) return fail(TACAW_ERR_INVALID_ARG, "bytes is NULL");
    c = check_saveable(p);
    if (c != TACAW_OK) return c;
    *bytes = state_total(p, plan_counters(p));
    return TACAW_OK;
}

tacaw_status tacaw_save_state(tacaw_plan_t p, void *h_state, int64_t bytes, void *stream) {
    TraceRange trace_range("tacaw_save_state");
    tacaw_status c = check_plan(p);
    if (c != TACAW_OK) return c;
    c = check_host_buffer(h_state, "h_state");
    if (c != TACAW_OK) return c;
    c = check_saveable(p);
    if (c != TACAW_OK) return c;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const std::vector<StreamCounters> cnt = plan_counters(p);
    std::vector<UserCounters> uc(p->us.size());
    for (size_t i = 0; i < p->us.size(); ++i) uc[i].pushed = p->us[i].pushed;
    const int64_t total = state_total(p, cnt);
    if (bytes < total)
        return fail(TACAW_ERR_INVALID_ARG, "h_state holds %lld bytes, the checkpoint needs %lld", (long long)bytes,
                    (long long)total);
    unsigned char *o = static_cast<unsigned char *>(h_state);
    StateHeader h{};
    h.magic = kStateMagic;
    h.version = kStateVersion;
    h.n_streams = (uint32_t)p->s.size();
    h.n_user = (uint32_t)p->us.size();
    h.fingerprint = plan_fingerprint(p);
    h.total_bytes = total;
    Fnv f;
    f.add(cnt.data(), sizeof(StreamCounters) * cnt.size());
    f.add(uc.data(), sizeof(UserCounters) * uc.size());
    h.counters_hash = f.h;
    size_t off = 0;
    std::memcpy(o, &h, sizeof h);
    off += sizeof h;
    std::memcpy(o + off, cnt.data(), sizeof(StreamCounters) * cnt.size());
    off += sizeof(StreamCounters) * cnt.size();
    std::memcpy(o + off, uc.data(), sizeof(UserCounters) * uc.size());
    off += sizeof(UserCounters) * uc.size();
    for (const StateSection &x : state_sections(p, cnt)) {
        CU_CHECK(p, cudaMemcpyAsync(o + off, x.dev, x.bytes, cudaMemcpyDeviceToHost, st), "checkpoint copy");
        off += x.bytes;
    }
    CU_CHECK(p, cudaStreamSynchronize(st), "checkpoint copies");
    return read_device_error(p, st);
}

tacaw_status tacaw_restore_state(tacaw_plan_t p, const void *h_state, int64_t bytes, void *stream) {
    TraceRange trace_range("tacaw_restore_state");
    tacaw_status c = check_plan(p);
    if (c != TACAW_OK) return c;
    c = check_host_buffer(h_state, "h_state");
    if (c != TACAW_OK) return c;
    if (p->pend.active || p->deferred_pushes)
        return fail(TACAW_ERR_STATE, "a segment's contraction is deferred: call tacaw_drain first");
    const unsigned char *in = static_cast<const unsigned char *>(h_state);
    StateHeader h{};
    if (bytes < (int64_t)sizeof h)
        return fail(TACAW_ERR_INVALID_ARG, "checkpoint: %lld bytes is too short", (long long)bytes);
    std::memcpy(&h, in, sizeof h);
    if (h.magic != kStateMagic) return fail(TACAW_ERR_INVALID_ARG, "checkpoint: not a plan checkpoint");
    if (h.version != kStateVersion)
        return fail(TACAW_ERR_INVALID_ARG, "checkpoint: version %u, this library reads %u", h.version, kStateVersion);
    if (h.n_streams != p->s.size() || h.n_user != p->us.size() || h.fingerprint != plan_fingerprint(p))
        return fail(TACAW_ERR_INVALID_ARG, "checkpoint: saved by a plan of another configuration");
    if (h.total_bytes > bytes)
        return fail(TACAW_ERR_INVALID_ARG, "checkpoint: truncated (%lld of %lld bytes)", (long long)bytes,
                    (long long)h.total_bytes);
    const size_t hdr = sizeof h + sizeof(StreamCounters) * p->s.size() + sizeof(UserCounters) * p->us.size();
    if ((int64_t)hdr > h.total_bytes) return fail(TACAW_ERR_INVALID_ARG, "checkpoint: truncated counters");
    std::vector<StreamCounters> cnt(p->s.size());
    std::vector<UserCounters> uc(p->us.size());
    size_t off = sizeof h;
    std::memcpy(cnt.data(), in + off, sizeof(StreamCounters) * cnt.size());
    off += sizeof(StreamCounters) * cnt.size();
    std::memcpy(uc.data(), in + off, sizeof(UserCounters) * uc.size());
    off += sizeof(UserCounters) * uc.size();
    Fnv f;
    f.add(cnt.data(), sizeof(StreamCounters) * cnt.size());
    f.add(uc.data(), sizeof(UserCounters) * uc.size());
    if (f.h != h.counters_hash) return fail(TACAW_ERR_INVALID_ARG, "checkpoint: counter records corrupted");
    c = check_counters(p, cnt, uc);
    if (c != TACAW_OK) return c;
    if (state_total(p, cnt) != h.total_bytes)
        return fail(TACAW_ERR_INVALID_ARG, "checkpoint: section sizes do not match its counters");
    // the checkpoint is this plan's: load the device sections, then the counters
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (const StateSection &x : state_sections(p, cnt)) {
        CU_CHECK(p, cudaMemcpyAsync(x.dev, in + off, x.bytes, cudaMemcpyHostToDevice, st), "checkpoint copy");
        off += x.bytes;
    }
    CU_CHECK(p, cudaStreamSynchronize(st), "checkpoint copies");
    for (size_t i = 0; i < p->s.size(); ++i) {
        Stream &s = p->s[i];
        s.pushed = (int)cnt[i].pushed;
        s.staged = (int)cnt[i].staged;
        s.stage_start = (int)cnt[i].stage_start;
        s.flushes = (int)cnt[i].flushes;
        s.seg = cnt[i].seg;
        s.due = cnt[i].due != 0;
        s.due_stream = st;
        s.h_pushes.clear();
    }
    for (size_t i = 0; i < p->us.size(); ++i) p->us[i].pushed = uc[i].pushed;
    p->finalized = false;
    return TACAW_OK;
}

}  // extern "C"
