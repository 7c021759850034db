// Window and twiddle tables (built once per plan, on the GPU, in FP64).
//
// Phase of energy j at frame t: theta_jt = 2 pi frac(c_j t), c_j = E_j dt / h cycles per
// frame (App. B: energies are resolved up to eps = h/(2 dt)).  The fractional part is
// taken in FP64; on an FFT grid (E_j = j h/(T dt)) it is the exact integer form
// ((j t) mod T) / T.  Trigonometry is CUDA's FP64 sincospi/cospi.
// Windows follow Sec. III.A / App. A (scipy's periodic forms; length-1 windows are [1]).
#include "tacaw_internal.cuh"

namespace tacaw {

enum { WIN_RECT = 0, WIN_HANN = 1, WIN_GAUSS = 2, WIN_TUKEY = 3, WIN_BLACKMANHARRIS = 4, WIN_KAISER = 5,
       WIN_CHEBWIN = 6 };

// Modified Bessel function I0 by its power series sum_k ((x/2)^k / k!)^2, FP64 (x <= 60)
__device__ double bessel_i0(double x) {
    const double q = 0.25 * x * x;
    double term = 1.0, total = 1.0;
    for (int k = 1; k < 200; ++k) {
        term *= q / ((double)k * (double)k);
        total += term;
        if (term <= 1e-18 * total) break;
    }
    return total;
}

__device__ double window_value(const TableArgs &a, int t) {
    const int kind = a.window, T = a.T;
    const double param = a.window_param;
    if (T == 1) return 1.0;
    switch (kind) {
        case WIN_RECT:
            return 1.0;
        case WIN_HANN:
            return 0.5 - 0.5 * cospi(2.0 * (double)t / (double)T);
        case WIN_GAUSS: {
            double s = param > 0.0 ? param : (double)T / 6.0;
            double z = ((double)t - 0.5 * (double)T) / s;
            return exp(-0.5 * z * z);
        }
        case WIN_TUKEY: {
            double alpha = param;
            if (alpha <= 0.0) return 1.0;
            if (alpha >= 1.0) return 0.5 - 0.5 * cospi(2.0 * (double)t / (double)T);
            double edge = alpha * (double)T / 2.0;
            if ((double)t < edge) return 0.5 * (1.0 - cospi((double)t / edge));
            if ((double)t > (double)T - edge) return 0.5 * (1.0 - cospi((double)(T - t) / edge));
            return 1.0;
        }
        case WIN_BLACKMANHARRIS: {
            const double x = 2.0 * (double)t / (double)T;   // in units of pi
            return 0.35875 - 0.48829 * cospi(x) + 0.14128 * cospi(2.0 * x) - 0.01168 * cospi(3.0 * x);
        }
        case WIN_KAISER: {
            const double u = 2.0 * (double)t / (double)T - 1.0;
            const double r = 1.0 - u * u;
            return bessel_i0(param * sqrt(r > 0.0 ? r : 0.0)) / bessel_i0(param);
        }
        case WIN_CHEBWIN:
            return a.win_table ? a.win_table[t] : 1.0;
    }
    return 1.0;
}

// exp(-i theta_jt) = (cos, -sin) of 2 pi f, f = frac(c_j t) in [0, 1)
__device__ void twiddle(const TableArgs &a, int j, int t, double &c, double &s) {
    double f;
    if (a.fft_bins) {
        long long r = ((long long)j * (long long)t) % (long long)a.T;
        f = (double)r / (double)a.T;
    } else {
        double x = a.cj[j] * (double)t;
        f = x - floor(x);
    }
    sincospi(2.0 * f, &s, &c);
}

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// fp16 pieces (split-FP16 path), stored in the bf16-typed table as raw 16-bit patterns;
// |B| <= 1, so no scaling: residuals below the fp16 normal range keep an absolute
// resolution of 2^-24, far below the 2^-22 relative resolution of the largest twiddles
__device__ __forceinline__ void split_f16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    const __half h = __float2half_rn(x);
    const __half l = __float2half_rn(x - __half2float(h));
    hi = __ushort_as_bfloat16(__half_as_ushort(h));
    lo = __ushort_as_bfloat16(__half_as_ushort(l));
}

// One thread per (energy j < Nw_pad, frame t < T_pad).  Rows 2j and 2j+1 of block t/bf
// (rows of 2*bf bf16) receive, at elements 2(t%bf) and 2(t%bf)+1, the real embedding of
// B = w_t exp(-i theta):
//   row 2j   : ( Re B, -Im B)  ->  Re Psi_j = Re psi Re B - Im psi Im B
//   row 2j+1 : ( Im B,  Re B)  ->  Im Psi_j = Re psi Im B + Im psi Re B
template <bool F16>
__global__ void twiddles_split_kernel(TableArgs a, __nv_bfloat16 *B_hi, __nv_bfloat16 *B_lo) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int t = blockIdx.y * blockDim.y + threadIdx.y;
    if (j >= a.Nw_pad || t >= a.T_pad) return;
    double br = 0.0, bi = 0.0;
    if (j < a.Nw && t < a.T) {
        double c, s;
        twiddle(a, j, t, c, s);
        double w = window_value(a, t);
        br = w * c;
        bi = -w * s;
    }
    const int bf = a.block_frames;
    const int kb = t / bf, tt = t % bf;
    const size_t rows = 2 * (size_t)a.Nw_pad;
    // word tt (a bf16 pair) of rows 2j and 2j+1; pre-swizzled rows keep their 16-byte chunks
    // where the tensor core's shared-memory swizzle of the row width expects them
    const int cpr = bf >> 2;
    const int sw0 = a.swz ? (int)(((2 * j * cpr) >> 3) & (cpr - 1)) : 0;
    const int sw1 = a.swz ? (int)((((2 * j + 1) * cpr) >> 3) & (cpr - 1)) : 0;
    const int w0 = (((tt >> 2) ^ sw0) << 2) | (tt & 3), w1 = (((tt >> 2) ^ sw1) << 2) | (tt & 3);
    const size_t r0 = ((size_t)kb * rows + 2 * (size_t)j) * (2 * bf) + 2 * w0;
    const size_t r1 = ((size_t)kb * rows + 2 * (size_t)j + 1) * (2 * bf) + 2 * w1;
    float v0[2] = {(float)br, (float)(-bi)};
    float v1[2] = {(float)bi, (float)br};
    for (int e = 0; e < 2; ++e) {
        __nv_bfloat16 h, l;
        if (F16) split_f16(v0[e], h, l);
        else split_bf16(v0[e], h, l);
        B_hi[r0 + e] = h;
        B_lo[r0 + e] = l;
        if (F16) split_f16(v1[e], h, l);
        else split_bf16(v1[e], h, l);
        B_hi[r1 + e] = h;
        B_lo[r1 + e] = l;
    }
}

// Table of the adjoint's back-projection C[m, t] = sum_j G[m, j] conj(B[t, j]): frames are the
// output columns and energies the contraction.  One thread per (energy j < e_pad, frame
// t < t_rows); b = conj(w_t exp(-i theta_jt)) = w_t exp(+i theta_jt) goes to elements 2(j%32),
// 2(j%32)+1 of rows 2t and 2t+1 of block j/32 (rows of 32 bf16 pairs, pre-swizzled):
//   row 2t   : ( Re b, -Im b)  ->  Re C_t = Re G Re b - Im G Im b
//   row 2t+1 : ( Im b,  Re b)  ->  Im C_t = Re G Im b + Im G Re b
__global__ void twiddles_adjoint_split_kernel(TableArgs a, int t_rows, int e_pad, __nv_bfloat16 *B_hi,
                                              __nv_bfloat16 *B_lo) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = blockIdx.y * blockDim.y + threadIdx.y;
    if (j >= e_pad || t >= t_rows) return;
    double br = 0.0, bi = 0.0;
    if (j < a.Nw && t < a.T) {
        double c, s;
        twiddle(a, j, t, c, s);
        const double w = window_value(a, t);
        br = w * c;
        bi = w * s;
    }
    const int kb = j / 32, jj = j % 32;
    const size_t rows = 2 * (size_t)t_rows;
    const int r0 = 2 * t, r1 = 2 * t + 1;
    // 128-byte rows: chunk c of row r stored at c ^ (r mod 8)
    const int w0 = (((jj >> 2) ^ (r0 & 7)) << 2) | (jj & 3), w1 = (((jj >> 2) ^ (r1 & 7)) << 2) | (jj & 3);
    const size_t o0 = ((size_t)kb * rows + (size_t)r0) * 64 + 2 * (size_t)w0;
    const size_t o1 = ((size_t)kb * rows + (size_t)r1) * 64 + 2 * (size_t)w1;
    const float v0[2] = {(float)br, (float)(-bi)};
    const float v1[2] = {(float)bi, (float)br};
    for (int e = 0; e < 2; ++e) {
        __nv_bfloat16 h, l;
        split_bf16(v0[e], h, l);
        B_hi[o0 + e] = h;
        B_lo[o0 + e] = l;
        split_bf16(v1[e], h, l);
        B_hi[o1 + e] = h;
        B_lo[o1 + e] = l;
    }
}

__global__ void twiddles_fp32_kernel(TableArgs a, float2 *B32) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int t = blockIdx.y * blockDim.y + threadIdx.y;
    if (j >= a.Nw_pad || t >= a.T_pad) return;
    float2 v = make_float2(0.f, 0.f);
    if (j < a.Nw && t < a.T) {
        double c, s;
        twiddle(a, j, t, c, s);
        double w = window_value(a, t);
        v = make_float2((float)(w * c), (float)(-w * s));
    }
    B32[(size_t)t * a.Nw_pad + j] = v;
}

// W(E_j) = sum_t w_t exp(-i theta_jt), one block per energy, fixed-order tree reduction.
__global__ void window_transform_kernel(TableArgs a, float2 *Wc) {
    const int j = blockIdx.x;
    double sr = 0.0, si = 0.0;
    for (int t = threadIdx.x; t < a.T; t += blockDim.x) {
        double c, s;
        twiddle(a, j, t, c, s);
        double w = window_value(a, t);
        sr += w * c;
        si -= w * s;
    }
    __shared__ double rr[256], ri[256];
    rr[threadIdx.x] = sr;
    ri[threadIdx.x] = si;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            rr[threadIdx.x] += rr[threadIdx.x + h];
            ri[threadIdx.x] += ri[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) Wc[j] = make_float2((float)rr[0], (float)ri[0]);
}

__global__ void window_values_kernel(TableArgs a, float *w) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < a.T) w[t] = (float)window_value(a, t);
}

cudaError_t launch_twiddles_split(const TableArgs &t, __nv_bfloat16 *B_hi, __nv_bfloat16 *B_lo, int f16,
                                  cudaStream_t st) {
    dim3 blk(32, 8);
    dim3 grd((t.Nw_pad + 31) / 32, (t.T_pad + 7) / 8);
    if (f16)
        twiddles_split_kernel<true><<<grd, blk, 0, st>>>(t, B_hi, B_lo);
    else
        twiddles_split_kernel<false><<<grd, blk, 0, st>>>(t, B_hi, B_lo);
    return cudaGetLastError();
}

cudaError_t launch_twiddles_adjoint_split(const TableArgs &t, int t_rows, int e_pad, __nv_bfloat16 *B_hi,
                                          __nv_bfloat16 *B_lo, cudaStream_t st) {
    dim3 blk(32, 8);
    dim3 grd((e_pad + 31) / 32, (t_rows + 7) / 8);
    twiddles_adjoint_split_kernel<<<grd, blk, 0, st>>>(t, t_rows, e_pad, B_hi, B_lo);
    return cudaGetLastError();
}

cudaError_t launch_twiddles_fp32(const TableArgs &t, float2 *B32, cudaStream_t st) {
    dim3 blk(32, 8);
    dim3 grd((t.Nw_pad + 31) / 32, (t.T_pad + 7) / 8);
    twiddles_fp32_kernel<<<grd, blk, 0, st>>>(t, B32);
    return cudaGetLastError();
}

cudaError_t launch_window_transform(const TableArgs &t, float2 *Wc, cudaStream_t st) {
    window_transform_kernel<<<t.Nw, 256, 0, st>>>(t, Wc);
    return cudaGetLastError();
}

cudaError_t launch_window_values(const TableArgs &t, float *w, cudaStream_t st) {
    window_values_kernel<<<(t.T + 255) / 256, 256, 0, st>>>(t, w);
    return cudaGetLastError();
}

}  // namespace tacaw
