// Detector spectra without any device allocation.
//
// tacaw_detector_spectra_noalloc() serves callers that hold an energy-resolved dataset
// I[p][E][ky][kx] in device memory but are not allowed to allocate device memory
// themselves or through the libraries they call: code that runs inside a framework that
// owns the whole device budget, real-time loops where cudaMalloc/cudaFree would
// synchronise the device, or hosts that only receive raw device pointers.  It creates no
// plan.  The compact (pixel, weight) lists of the apertures, which a plan keeps in memory
// it allocated, live here in one file-scope device array of fixed size instead.
//
// The array is shared by every call in the process (one instance per device that loads
// the library, held until exit) and keeps the last call's lists: calls whose work
// overlaps on the GPU (different streams, or threads) race on it and must be serialised
// by the caller.  Nothing in it is accumulated, so nothing needs clearing between calls.
#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/tacaw.h"
#include "tacaw_internal.cuh"

namespace {

constexpr int kMaxEntries = 1 << 20;      // (pixel, weight) pairs summed over all detectors
constexpr int kMaxDetectors = 1024;
constexpr int kMaxDevices = 64;
constexpr size_t kWords = 2 * (size_t)kMaxEntries + kMaxDetectors + 1;

// [0, kMaxEntries): pixel indices; [kMaxEntries, 2 kMaxEntries): weights (float bits);
// then kMaxDetectors + 1 list offsets.  8 MiB + 4 KiB per device.
static __device__ __align__(256) uint32_t g_noalloc_scratch[kWords];

// The array's device address, looked up once per device and context: a context torn down and
// made again (cudaDeviceReset, then new work on the device) gets a new id and a new lookup.
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Id of the calling thread's current context (0 if the driver does not report one).  Called with
// g_mu held.
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_cur = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool looked = false;
    if (!looked) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = reinterpret_cast<CtxGetCurrentFn>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(p);
        looked = true;
    }
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_cur && get_id && get_cur(&c) == CUDA_SUCCESS && c && get_id(c, &id) == CUDA_SUCCESS) return id;
    return 0;
}

// Device address of the array on the current device.  The first call on a device (and the
// first after its context was made again) looks it up with cudaGetSymbolAddress.
tacaw_status scratch_address(uint32_t **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        tacaw::set_last_error("tacaw_detector_spectra_noalloc: no usable current CUDA device");
        return TACAW_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    const unsigned long long ctx = current_context_id();
    if (!g_scratch_ptr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            char buf[256];
            snprintf(buf, sizeof(buf), "tacaw_detector_spectra_noalloc: cudaGetSymbolAddress failed: %s",
                     cudaGetErrorString(e));
            tacaw::set_last_error(buf);
            return TACAW_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
        g_scratch_ctx[dev] = ctx;
    }
    *out = static_cast<uint32_t *>(g_scratch_ptr[dev]);
    return TACAW_OK;
}

tacaw_status bad(const char *msg) {
    tacaw::set_last_error(msg);
    return TACAW_ERR_INVALID_ARG;
}

tacaw_status spectra(const float *d_I, int n_probes, int n_omega, int kx, int ky, const tacaw_detector *detectors,
                     int n_detectors, float *d_S, cudaStream_t cs) {
    if (!d_I || !d_S) return bad("tacaw_detector_spectra_noalloc: d_I and d_S must not be NULL");
    if (n_probes < 1 || n_omega < 1 || kx < 1 || ky < 1)
        return bad("tacaw_detector_spectra_noalloc: n_probes, n_omega, kx, ky must be >= 1");
    if (n_detectors < 1 || !detectors) return bad("tacaw_detector_spectra_noalloc: need at least one detector");
    if (n_detectors > kMaxDetectors) {
        char buf[160];
        snprintf(buf, sizeof(buf), "tacaw_detector_spectra_noalloc: %d detectors exceed the maximum of %d",
                 n_detectors, kMaxDetectors);
        return bad(buf);
    }
    const int64_t npix = (int64_t)kx * ky;
    if (npix > (int64_t)INT32_MAX) return bad("tacaw_detector_spectra_noalloc: kx * ky exceeds 2^31 - 1 pixels");
    if (n_probes > 65535) return bad("tacaw_detector_spectra_noalloc: more than 65535 probes");
    // the lists are copied from host memory on `stream`: a graph capturing it could not replay them
    cudaStreamCaptureStatus capt = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(cs, &capt) != cudaSuccess) {
        cudaGetLastError();
        tacaw::set_last_error("tacaw_detector_spectra_noalloc: cudaStreamIsCapturing failed on the stream");
        return TACAW_ERR_CUDA;
    }
    if (capt != cudaStreamCaptureStatusNone)
        return bad("tacaw_detector_spectra_noalloc: the stream is capturing a graph; this call copies host-side "
                   "aperture lists and is refused inside a capture");
    // d_I is read and d_S written by the kernel: device, managed or mapped pinned host memory only
    if (tacaw::check_device_readable(d_I, "d_I", cs) != TACAW_OK) return TACAW_ERR_INVALID_ARG;
    if (tacaw::check_device_readable(d_S, "d_S", cs) != TACAW_OK) return TACAW_ERR_INVALID_ARG;
    // aperture lists on the host (same conventions as tacaw_plan_create)
    std::vector<uint32_t> idx, wts;
    std::vector<uint32_t> off(n_detectors + 1, 0);
    std::vector<float> hmask;
    for (int k = 0; k < n_detectors; ++k) {
        const tacaw_detector &t = detectors[k];
        if (t.kind < TACAW_DET_CIRCULAR || t.kind > TACAW_DET_MASK)
            return bad("tacaw_detector_spectra_noalloc: bad detector kind");
        if (t.kind == TACAW_DET_MASK) {
            if (!t.d_mask) return bad("tacaw_detector_spectra_noalloc: mask pointer is NULL");
            if (tacaw::check_device_readable(t.d_mask, "d_mask", cs) != TACAW_OK) return TACAW_ERR_INVALID_ARG;
            hmask.resize(npix);
            // ordered after the caller's earlier work on `stream` that may write the mask
            cudaError_t e = cudaMemcpyAsync(hmask.data(), t.d_mask, sizeof(float) * npix, cudaMemcpyDeviceToHost, cs);
            if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
            if (e != cudaSuccess) {
                cudaGetLastError();
                tacaw::set_last_error("tacaw_detector_spectra_noalloc: reading a mask failed");
                return TACAW_ERR_CUDA;
            }
        }
        const double cx = (double)(kx / 2) + t.cx, cy = (double)(ky / 2) + t.cy;
        for (int y = 0; y < ky; ++y)
            for (int x = 0; x < kx; ++x) {
                float w;
                if (t.kind == TACAW_DET_MASK) {
                    w = hmask[(size_t)y * kx + x];
                } else {
                    const double dx = x - cx, dy = y - cy, r2 = dx * dx + dy * dy;
                    bool in = r2 <= (double)t.r_out * (double)t.r_out;
                    if (t.kind == TACAW_DET_ANNULAR && t.r_in >= 0) in = in && r2 > (double)t.r_in * (double)t.r_in;
                    w = in ? 1.f : 0.f;
                }
                if (w == 0.f) continue;
                if ((int64_t)idx.size() >= kMaxEntries) {
                    char buf[200];
                    snprintf(buf, sizeof(buf),
                             "tacaw_detector_spectra_noalloc: apertures cover more than %d pixel entries "
                             "(the size of the library's fixed device array)", kMaxEntries);
                    return bad(buf);
                }
                idx.push_back((uint32_t)((int64_t)y * kx + x));
                uint32_t bits;
                memcpy(&bits, &w, 4);
                wts.push_back(bits);
            }
        off[k + 1] = (uint32_t)idx.size();
    }
    uint32_t *scr = nullptr;
    tacaw_status st = scratch_address(&scr);
    if (st != TACAW_OK) return st;
    const size_t n = idx.size();
    cudaError_t e = cudaSuccess;
    // pageable host sources: each copy returns once the host data has been taken
    if (n) e = cudaMemcpyAsync(scr, idx.data(), n * 4, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess && n) e = cudaMemcpyAsync(scr + kMaxEntries, wts.data(), n * 4, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(scr + 2 * (size_t)kMaxEntries, off.data(), off.size() * 4, cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess) {
        cudaGetLastError();
        tacaw::set_last_error("tacaw_detector_spectra_noalloc: copying the aperture lists failed");
        return TACAW_ERR_CUDA;
    }
    tacaw::ApertureArgs a{};
    a.I = d_I;
    a.S = d_S;
    a.P = n_probes;
    a.D = n_detectors;
    a.Nw = n_omega;
    a.npix = npix;
    a.idx = reinterpret_cast<const int *>(scr);
    a.wts = reinterpret_cast<const float *>(scr + kMaxEntries);
    a.off = reinterpret_cast<const int *>(scr + 2 * (size_t)kMaxEntries);
    e = tacaw::launch_aperture(a, cs);
    if (e != cudaSuccess) {
        tacaw::set_last_error(cudaGetErrorString(e));
        return TACAW_ERR_CUDA;
    }
    return TACAW_OK;
}

}  // namespace

extern "C" tacaw_status tacaw_detector_spectra_noalloc(const float *d_I, int n_probes, int n_omega, int kx, int ky,
                                                       const tacaw_detector *detectors, int n_detectors,
                                                       float *d_S, void *stream) {
    // a named range on the profiler timeline (NVTX), as around every entry point of the library
    struct Range {
        Range() { nvtxRangePushA("tacaw_detector_spectra_noalloc"); }
        ~Range() { nvtxRangePop(); }
    } trace_range;
    try {
        return spectra(d_I, n_probes, n_omega, kx, ky, detectors, n_detectors, d_S, static_cast<cudaStream_t>(stream));
    } catch (const std::bad_alloc &) {
        tacaw::set_last_error("tacaw_detector_spectra_noalloc: host memory for the aperture lists ran out");
        return TACAW_ERR_OOM;
    }
}
