// Tile autotuner of the tensor-core contraction (host code).
//
// For one stream shape (rows M, energies Nw, segment length T, frames per flush) it times the
// staged contraction kernel itself for each candidate tile width -- energies per tile wt -- on
// scratch operands, and keeps the fastest predicted one.  Candidates: for n_wt energy tiles
// from the fewest that fit the widest tile up to three more, the narrowest multiple of 8
// covering Nw in n_wt tiles.  Each candidate runs one wave of tiles (one per co-resident CTA)
// at two flush lengths; the per-tile time is linear in the staged blocks (fill + main loop +
// epilogue), so the two points give the time of any flush length.  The prediction is
//   one stream per plan:  ceil(tiles / resident) waves x wave time
//   several streams:      tiles x wave time / resident   (their tiles share one launch)
// summed over the segment's flushes.  Operand values do not change the instruction stream,
// so the scratch operands hold one constant bit pattern.
//
// Tables are kept in a text cache (one line per shape: "<key> | <wt>:<ms> ...") so a later
// plan of the same shape on the same kind of GPU skips the timing.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "tacaw_internal.cuh"

namespace tacaw {

namespace {

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    bool alloc(size_t bytes) {
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return false;
        }
        return true;
    }
};

struct Cand {
    int wt, n_wt, stages, resident;
    int64_t n_mt_sub;
};

std::string shape_key(const TuneShape &s) {
    int dev = 0, maj = 0, mnr = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&mnr, cudaDevAttrComputeCapabilityMinor, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    char b[320];
    snprintf(b, sizeof(b), "tacaw-tune-v2 sm%d%dx%d drain=%d bf=%d M=%lld Nw=%d T=%d ring=%d multi=%d wt=%d", maj,
             mnr, sms, s.drain_kb, s.bf, (long long)s.M, s.Nw, s.T, s.ring, s.multi ? 1 : 0, s.fixed_wt);
    return b;
}

bool cache_lookup(const char *path, const std::string &key, std::vector<TuneCand> *tab) {
    if (!path || !*path) return false;
    FILE *f = fopen(path, "r");
    if (!f) return false;
    std::vector<char> line(1 << 16);
    bool found = false;
    while (fgets(line.data(), (int)line.size(), f)) {
        const char *bar = strstr(line.data(), " | ");
        if (!bar || (size_t)(bar - line.data()) != key.size() || strncmp(line.data(), key.c_str(), key.size()) != 0)
            continue;
        std::vector<TuneCand> t;
        const char *q = bar + 3;
        int w, used;
        double ms;
        while (sscanf(q, "%d:%lf%n", &w, &ms, &used) == 2) {
            if (w > 0 && ms >= 0.0) t.push_back(TuneCand{w, ms});
            q += used;
        }
        if (!t.empty()) {
            *tab = t;           // the last matching line wins
            found = true;
        }
    }
    fclose(f);
    return found;
}

void cache_store(const char *path, const std::string &key, const std::vector<TuneCand> &tab) {
    if (!path || !*path) return;
    std::string line = key + " |";
    char b[64];
    for (const TuneCand &c : tab) {
        snprintf(b, sizeof(b), " %d:%.6f", c.wt, c.ms);
        line += b;
    }
    line += "\n";
    FILE *f = fopen(path, "a");
    if (!f) return;
    fputs(line.c_str(), f);     // one write per line: concurrent plans append whole lines
    fclose(f);
}

}  // namespace

bool tc_autotune(const TuneShape &sh, const char *cache_path, uint32_t *d_err, cudaStream_t st,
                 std::vector<TuneCand> *table, int *timed, char *err, size_t errlen) {
    table->clear();
    *timed = 0;
    const std::string key = shape_key(sh);
    std::vector<TuneCand> cached;
    if (cache_lookup(cache_path, key, &cached)) {
        for (const TuneCand &c : cached)
            if (c.wt % 8 == 0 && c.wt <= sh.wt_max && tc_stages_for(2 * c.wt, sh.bf) >= 2) table->push_back(c);
        if (!table->empty()) return true;
    }
    const int64_t n_mt = (sh.M + kMTile - 1) / kMTile;
    // candidate tiles
    std::vector<int> wts;
    if (sh.fixed_wt) {
        wts.push_back(sh.fixed_wt);
    } else {
        const int n0 = (sh.Nw + sh.wt_max - 1) / sh.wt_max;
        for (int n = n0; n <= n0 + 3; ++n) {
            const int w = ((sh.Nw + n - 1) / n + 7) / 8 * 8;
            if (w <= sh.wt_max && (wts.empty() || wts.back() != w)) wts.push_back(w);
        }
    }
    std::vector<Cand> cands;
    for (int w : wts) {
        const int N = 2 * w;
        const int stages = tc_stages_for(N, sh.bf);
        if (stages < 2) continue;
        const int n_wt = (sh.Nw + w - 1) / w;
        const int R = tc_resident_ctas(N, sh.bf, stages);
        if (R <= 0) continue;
        Cand c{w, n_wt, stages, R, 0};
        // one wave: at most R tiles, no more row tiles than the stream has
        int64_t m = (int64_t)(R / n_wt);
        if (m < 1) m = 1;
        c.n_mt_sub = m < n_mt ? m : n_mt;
        cands.push_back(c);
    }
    if (cands.empty()) {
        snprintf(err, errlen, "autotune: no tensor-core tile fits (Nw=%d, bf=%d)", sh.Nw, sh.bf);
        return false;
    }
    // flush lengths timed (staging blocks), and the flushes of one segment
    const int kb_ring = sh.ring / sh.bf;
    const int kb2 = kb_ring < 512 / sh.bf ? kb_ring : 512 / sh.bf;
    const int kb1 = kb2 >= 8 ? kb2 / 4 : kb2;
    std::vector<int> flush_kb;
    for (int t = 0; t < sh.T; t += sh.ring) {
        const int n = sh.T - t < sh.ring ? sh.T - t : sh.ring;
        flush_kb.push_back((n + sh.bf - 1) / sh.bf);
    }
    // scratch operands sized for the largest candidate
    int64_t rows = 0;
    int nw_pad_max = 0;
    for (const Cand &c : cands) {
        rows = std::max(rows, c.n_mt_sub * kMTile);
        nw_pad_max = std::max(nw_pad_max, c.wt * c.n_wt);
    }
    const size_t a_elems = (size_t)kb2 * rows * 2 * sh.bf;
    const size_t b_elems = (size_t)kb2 * 2 * nw_pad_max * 2 * sh.bf;
    DevBuf a_hi, a_lo, b_hi, b_lo, wc, bose, iout, counter;
    if (!a_hi.alloc(a_elems * 2) || !a_lo.alloc(a_elems * 2) || !b_hi.alloc(b_elems * 2) || !b_lo.alloc(b_elems * 2) ||
        !wc.alloc(sizeof(float2) * sh.Nw) || !bose.alloc(sizeof(float) * sh.Nw) ||
        !iout.alloc(sizeof(float) * (size_t)sh.Nw * rows) || !counter.alloc(sizeof(int))) {
        snprintf(err, errlen, "autotune: scratch allocation failed");
        return false;
    }
    // 0x3F3F: bf16 0.746 (finite, non-zero); W(E) = 0
    if (cudaMemsetAsync(a_hi.p, 0x3F, a_elems * 2, st) != cudaSuccess ||
        cudaMemsetAsync(a_lo.p, 0x3F, a_elems * 2, st) != cudaSuccess ||
        cudaMemsetAsync(b_hi.p, 0x3F, b_elems * 2, st) != cudaSuccess ||
        cudaMemsetAsync(b_lo.p, 0x3F, b_elems * 2, st) != cudaSuccess ||
        cudaMemsetAsync(wc.p, 0, sizeof(float2) * sh.Nw, st) != cudaSuccess ||
        cudaMemsetAsync(bose.p, 0x3F, sizeof(float) * sh.Nw, st) != cudaSuccess) {
        snprintf(err, errlen, "autotune: memset failed");
        return false;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        snprintf(err, errlen, "autotune: cudaEventCreate failed");
        return false;
    }
    bool ok = true;
    for (const Cand &c : cands) {
        const int N = 2 * c.wt;
        const int64_t m_sub = c.n_mt_sub * kMTile;
        TcPlanArgs a{};
        a.e.M = m_sub;
        a.e.M_pad = m_sub;
        a.e.npix = m_sub;
        a.e.Nw = sh.Nw;
        a.e.mode = FLUSH_FINAL;
        a.e.out_scale = 1.f;
        a.e.psi_scale = 1.f;
        a.e.I_out = static_cast<float *>(iout.p);
        a.e.Wc = static_cast<const float2 *>(wc.p);
        a.e.bose = static_cast<const float *>(bose.p);
        a.wt = c.wt;
        a.n_wt = c.n_wt;
        a.N = N;
        a.kbB0 = 0;
        a.bf = sh.bf;
        a.stages = c.stages;
        a.drain_kb = sh.drain_kb;
        a.N_last = N;
        a.A_hi = a_hi.p;
        a.A_lo = a_lo.p;
        a.B_hi = b_hi.p;
        a.B_lo = b_lo.p;
        a.a_rows = rows;
        a.b_rows = 2 * c.wt * c.n_wt;
        a.err = d_err;
        a.tile_counter = static_cast<int *>(counter.p);
        double t[2] = {0.0, 0.0};
        const int kbs[2] = {kb1, kb2};
        for (int q = 0; q < 2 && ok; ++q) {
            a.n_kb = kbs[q];
            const int reps = 3;
            cudaError_t e = launch_flush_tc(a, st);       // warm-up
            e = e == cudaSuccess ? cudaEventRecord(e0, st) : e;
            for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_flush_tc(a, st);
            e = e == cudaSuccess ? cudaEventRecord(e1, st) : e;
            e = e == cudaSuccess ? cudaEventSynchronize(e1) : e;
            float ms = 0.f;
            e = e == cudaSuccess ? cudaEventElapsedTime(&ms, e0, e1) : e;
            if (e != cudaSuccess) {
                snprintf(err, errlen, "autotune: %s", cudaGetErrorString(e));
                ok = false;
                break;
            }
            t[q] = ms / reps;
            if (kb1 == kb2) {
                t[1] = t[0];
                break;
            }
        }
        if (!ok) break;
        const double slope = kb2 > kb1 ? (t[1] - t[0]) / (double)(kb2 - kb1) : 0.0;
        const int64_t ctas = n_mt * c.n_wt;
        const int64_t per_launch = c.n_mt_sub * c.n_wt;
        double pred = 0.0;
        for (int kb : flush_kb) {
            double tw = t[1] + slope * (double)(kb - kb2);
            if (tw < 0.0) tw = 0.0;
            if (sh.multi)
                pred += tw * (double)ctas / (double)c.resident;
            else
                pred += tw * (double)((ctas + per_launch - 1) / per_launch);
        }
        table->push_back(TuneCand{c.wt, pred});
        ++*timed;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok) return false;
    uint32_t h = 0;
    if (cudaMemcpy(&h, d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess || h != 0) {
        cudaGetLastError();
        snprintf(err, errlen, "autotune: device wait timed out (error bits 0x%x)", h);
        return false;
    }
    cache_store(cache_path, key, *table);
    return true;
}

}  // namespace tacaw
