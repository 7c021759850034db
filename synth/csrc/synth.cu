// CUDA twin of synth/frames.py: seeded synthetic exit waves written straight into device
// memory (inputs for tests and the bench; none of the TACAW arithmetic lives here).
//
// psi[p,t,k] = psi0[p,k] + sum_m a[p,k,m] exp(2 pi i (f_m t + phi[p,k,m])) + noise[p,t,k]
// with Philox4x32-10 draws keyed by (seed, 0x5EED0000 ^ stream_id) and counters
// (full-grid pixel, probe, purpose | mode << 8, frame), parameters in FP64 as in the NumPy
// twin; the sum itself is evaluated in FP32 (phases advanced from an FP64 frame-t0 base).
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kMaxModes = 64;

struct SynthArgs {
    float2 *out;
    long long pitch_row, pitch_frame, pitch_probe;
    int out_x0, out_y0;
    int P, p0, kx, ky, t0, n;
    int gx, gy, rx, ry;
    double sigma_env, env_norm;
    unsigned seed, stream_id;
    int n_modes;
    double f[kMaxModes];
    int amp_law;
    double amp;
    double su[kMaxModes], sv[kMaxModes], chi[kMaxModes];
    int kdiv;
    double noise;
};

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        if (r != 9) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
    }
    return c;
}

__device__ __forceinline__ double u01(uint32_t x) { return ((double)x + 0.5) * 2.3283064365386963e-10; }

__global__ void synth_kernel(SynthArgs a) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t npix = (int64_t)a.kx * a.ky;
    if (id >= (int64_t)a.P * npix) return;
    const int pl = (int)(id / npix);
    const int pix = (int)(id - (int64_t)pl * npix);
    const int iy = pix / a.kx, ix = pix - (pix / a.kx) * a.kx;
    const int p = a.p0 + pl;
    const int X = ix + a.rx, Y = iy + a.ry;
    const uint32_t cpix = (uint32_t)Y * (uint32_t)a.gx + (uint32_t)X;
    const uint2 key = make_uint2(a.seed, 0x5EED0000u ^ a.stream_id);
    const double dx = (double)(X - a.gx / 2), dy = (double)(Y - a.gy / 2);
    const double env = exp(-(dx * dx + dy * dy) / (2.0 * a.sigma_env * a.sigma_env)) / a.env_norm;
    uint4 r = philox4x32_10(make_uint4(cpix, (uint32_t)p, 1u, 0u), key);
    double s0, c0;
    sincospi(2.0 * u01(r.x), &s0, &c0);
    const float psr = (float)(env * c0), psi_ = (float)(env * s0);
    float amp[kMaxModes], base[kMaxModes], fm[kMaxModes];
    for (int m = 0; m < a.n_modes; ++m) {
        uint4 q = philox4x32_10(make_uint4(cpix, (uint32_t)p, 3u | ((uint32_t)m << 8), 0u), key);
        const double phi = u01(q.x);
        double s;
        if (a.amp_law == 1) {
            s = 0.5 + 0.5 * cospi(2.0 * ((a.su[m] * dx + a.sv[m] * dy) / (double)a.kdiv + a.chi[m]));
        } else {
            s = u01(q.y);
        }
        amp[m] = (float)(a.amp * env * (0.5 + 0.5 * s));
        const double x = a.f[m] * (double)a.t0 + phi;
        base[m] = (float)(x - floor(x));
        fm[m] = (float)a.f[m];
    }
    const float nsc = (float)(a.noise / 1.4142135623730951);
    float2 *dst = a.out + (int64_t)pl * a.pitch_probe + (int64_t)(a.out_y0 + iy) * a.pitch_row + (a.out_x0 + ix);
    for (int tt = 0; tt < a.n; ++tt) {
        float re = psr, im = psi_;
        for (int m = 0; m < a.n_modes; ++m) {
            float cyc = fmaf(fm[m], (float)tt, base[m]);
            cyc -= floorf(cyc);
            float sn, cs;
            sincospif(2.f * cyc, &sn, &cs);
            re = fmaf(amp[m], cs, re);
            im = fmaf(amp[m], sn, im);
        }
        if (a.noise > 0.0) {
            uint4 q = philox4x32_10(make_uint4(cpix, (uint32_t)p, 5u, (uint32_t)(a.t0 + tt)), key);
            const float rho = sqrtf(-2.f * logf((float)u01(q.x)));
            float sn, cs;
            sincospif(2.f * (float)u01(q.y), &sn, &cs);
            re = fmaf(nsc * rho, cs, re);
            im = fmaf(nsc * rho, sn, im);
        }
        dst[(int64_t)tt * a.pitch_frame] = make_float2(re, im);
    }
}

}  // namespace

extern "C" {

// Writes frames t0..t0+n-1 of probes p0..p0+P-1 for the ROI pixels (ix < kx, iy < ky) into
// out + p*pitch_probe + t*pitch_frame + (out_y0+iy)*pitch_row + (out_x0+ix) (complex64
// elements).  (rx, ry) is the ROI origin in the full gx x gy grid, which keys the draws.
// Returns 0 on success, else the CUDA error code.
int synth_frames(void *out, long long pitch_row, long long pitch_frame, long long pitch_probe, int out_x0,
                 int out_y0, int P, int p0, int kx, int ky, int t0, int n, int gx, int gy, int rx, int ry,
                 double sigma_env, double env_norm, unsigned seed, unsigned stream_id, int n_modes,
                 const double *f, int amp_law, double amp, const double *su, const double *sv, const double *chi,
                 int kdiv, double noise, void *stream) {
    if (n_modes > kMaxModes || n_modes < 0 || P < 1 || n < 1 || kx < 1 || ky < 1) return (int)cudaErrorInvalidValue;
    SynthArgs a;
    a.out = static_cast<float2 *>(out);
    a.pitch_row = pitch_row;
    a.pitch_frame = pitch_frame;
    a.pitch_probe = pitch_probe;
    a.out_x0 = out_x0;
    a.out_y0 = out_y0;
    a.P = P;
    a.p0 = p0;
    a.kx = kx;
    a.ky = ky;
    a.t0 = t0;
    a.n = n;
    a.gx = gx;
    a.gy = gy;
    a.rx = rx;
    a.ry = ry;
    a.sigma_env = sigma_env;
    a.env_norm = env_norm;
    a.seed = seed;
    a.stream_id = stream_id;
    a.n_modes = n_modes;
    a.amp_law = amp_law;
    a.amp = amp;
    a.kdiv = kdiv;
    a.noise = noise;
    for (int m = 0; m < kMaxModes; ++m) {
        a.f[m] = m < n_modes ? f[m] : 0.0;
        a.su[m] = (m < n_modes && su) ? su[m] : 0.0;
        a.sv[m] = (m < n_modes && sv) ? sv[m] : 0.0;
        a.chi[m] = (m < n_modes && chi) ? chi[m] : 0.0;
    }
    const int64_t threads = (int64_t)P * kx * ky;
    synth_kernel<<<(unsigned)((threads + 127) / 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(a);
    return (int)cudaGetLastError();
}

}  // extern "C"
