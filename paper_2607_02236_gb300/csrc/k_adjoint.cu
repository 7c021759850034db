// Adjoint of the spectrum with respect to the frames (hand-written, FP32).
//
// For L = sum_{p,d,j} dL/dS[p,d,j] S[p,d,j] and Psi = sum_t w_t (psi_t - mu) e^{-i theta_jt}:
//   G[p,k,j] = B(E_j) (sum_d dL/dS[p,d,j] M_d(k)) Psi[p,k,j]
//   C[p,k,t] = sum_j conj(w_t e^{-i theta_jt}) G[p,k,j] = w_t sum_j e^{+i theta_jt} G[p,k,j]
//   grad[p,t,k] = 2 (C[p,k,t] - (1/T) sum_t' C[p,k,t'])            (mean term with subtract_mean)
// and (1/T) sum_t C = (1/T) sum_j conj(W_j) G_j with W_j = sum_t w_t e^{-i theta_jt}.
// A Welch-averaged stream (S = (1/N) sum_n S_n, Sec. II.B) runs this per segment with
// scale 1/N, adding into the gradient of the frames the segments share.
// Only pixels inside an aperture have G != 0, so both contractions run over that compact
// pixel list; Psi is recomputed from the frames (the window and twiddles come from the
// plan's table), never stored between forward and backward.
#include "tacaw_internal.cuh"

namespace tacaw {

constexpr int ADJ_PIX = 8;    // pixels per block
constexpr int ADJ_TCH = 64;   // frames staged per step

__device__ __forceinline__ const float2 *adj_src(const AdjointArgs &a, int p, int pix) {
    const int y = pix / a.kx, x = pix - (pix / a.kx) * a.kx;
    return a.frames + (int64_t)p * a.pitch_probe + (int64_t)(a.roi_y0 + y) * a.pitch_row + (a.roi_x0 + x);
}

// block (pixel group, probe): mean, Psi over all energies, G, and the constant K
__global__ void __launch_bounds__(256) adj_forward_kernel(AdjointArgs a) {
    const int g0 = blockIdx.x * ADJ_PIX;
    const int p = blockIdx.y;
    const int npx = min(ADJ_PIX, a.n_mpix - g0);
    __shared__ float2 xs[ADJ_TCH][ADJ_PIX];
    __shared__ float2 mu[ADJ_PIX];
    __shared__ float2 red[ADJ_PIX][8];
    const int tid = threadIdx.x;
    // exact mean of each pixel's series
    if (tid < 32 * ADJ_PIX) {
        const int i = tid >> 5, lane = tid & 31;
        float sr = 0.f, si = 0.f;
        if (i < npx && a.subtract_mean) {
            const float2 *src = adj_src(a, p, a.mpix[g0 + i]);
            for (int t = lane; t < a.T; t += 32) {
                float2 v = src[(int64_t)t * a.pitch_frame];
                sr += v.x;
                si += v.y;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sr += __shfl_xor_sync(0xffffffffu, sr, o);
            si += __shfl_xor_sync(0xffffffffu, si, o);
        }
        if (lane == 0) mu[i] = make_float2(sr / a.T, si / a.T);
    }
    __syncthreads();
    float2 *G = a.scratch;                                   // [P][n_mpix][Nw]
    float2 *Kc = a.scratch + (size_t)a.P * a.n_mpix * a.Nw;  // [P][n_mpix]
    float kr[ADJ_PIX], ki[ADJ_PIX];
#pragma unroll
    for (int i = 0; i < ADJ_PIX; ++i) kr[i] = ki[i] = 0.f;
    for (int jb = 0; jb < a.Nw; jb += 256) {
        const int j = jb + tid;
        float pr[ADJ_PIX], pi[ADJ_PIX];
#pragma unroll
        for (int i = 0; i < ADJ_PIX; ++i) pr[i] = pi[i] = 0.f;
        for (int t0 = 0; t0 < a.T; t0 += ADJ_TCH) {
            __syncthreads();
            for (int e = tid; e < ADJ_TCH * ADJ_PIX; e += 256) {
                const int tt = e / ADJ_PIX, i = e % ADJ_PIX;
                float2 v = make_float2(0.f, 0.f);
                if (i < npx && t0 + tt < a.T) {
                    v = adj_src(a, p, a.mpix[g0 + i])[(int64_t)(t0 + tt) * a.pitch_frame];
                    v.x -= mu[i].x;
                    v.y -= mu[i].y;
                }
                xs[tt][i] = v;
            }
            __syncthreads();
            if (j < a.Nw) {
                const int tn = min(ADJ_TCH, a.T - t0);
                for (int tt = 0; tt < tn; ++tt) {
                    const float2 b = a.B32[(size_t)(t0 + tt) * a.Nw_pad + j];
#pragma unroll
                    for (int i = 0; i < ADJ_PIX; ++i) {
                        const float2 x = xs[tt][i];
                        pr[i] = fmaf(x.x, b.x, fmaf(-x.y, b.y, pr[i]));
                        pi[i] = fmaf(x.x, b.y, fmaf(x.y, b.x, pi[i]));
                    }
                }
            }
        }
        if (j < a.Nw) {
            const float2 W = a.Wc[j];
            const float bj = a.bose[j];
#pragma unroll
            for (int i = 0; i < ADJ_PIX; ++i) {
                if (i >= npx) break;
                float c = 0.f;
                for (int d = 0; d < a.D; ++d)
                    c += a.dLdS[((size_t)p * a.D + d) * a.Nw + j] * a.mwts[(size_t)(g0 + i) * a.D + d];
                c *= bj;
                const float gr = c * pr[i], gi = c * pi[i];
                G[((size_t)p * a.n_mpix + g0 + i) * a.Nw + j] = make_float2(gr, gi);
                // conj(W) G
                kr[i] += W.x * gr + W.y * gi;
                ki[i] += W.x * gi - W.y * gr;
            }
        }
    }
    // block reduction of K over energies: warp shuffles, then fixed-order sum of 8 warps
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int i = 0; i < ADJ_PIX; ++i) {
        float vr = kr[i], vi = ki[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            vr += __shfl_xor_sync(0xffffffffu, vr, o);
            vi += __shfl_xor_sync(0xffffffffu, vi, o);
        }
        if (lane == 0) red[i][warp] = make_float2(vr, vi);
    }
    __syncthreads();
    if (tid < npx) {
        float sr = 0.f, si = 0.f;
        for (int w = 0; w < 8; ++w) {
            sr += red[tid][w].x;
            si += red[tid][w].y;
        }
        Kc[(size_t)p * a.n_mpix + g0 + tid] =
            a.subtract_mean ? make_float2(sr / a.T, si / a.T) : make_float2(0.f, 0.f);
    }
}

// block (pixel group, probe): C_t = sum_j G_j conj(B[t][j]) for every frame; grad = 2 (C - K)
__global__ void __launch_bounds__(256) adj_backward_kernel(AdjointArgs a) {
    const int g0 = blockIdx.x * ADJ_PIX;
    const int p = blockIdx.y;
    const int npx = min(ADJ_PIX, a.n_mpix - g0);
    constexpr int JCH = 128;
    __shared__ float2 gs[JCH][ADJ_PIX];
    const float2 *G = a.scratch;
    const float2 *Kc = a.scratch + (size_t)a.P * a.n_mpix * a.Nw;
    const int tid = threadIdx.x;
    for (int tb = 0; tb < a.T; tb += 256) {
        const int t = tb + tid;
        float cr[ADJ_PIX], ci[ADJ_PIX];
#pragma unroll
        for (int i = 0; i < ADJ_PIX; ++i) cr[i] = ci[i] = 0.f;
        for (int j0 = 0; j0 < a.Nw; j0 += JCH) {
            __syncthreads();
            for (int e = tid; e < JCH * ADJ_PIX; e += 256) {
                const int jj = e / ADJ_PIX, i = e % ADJ_PIX;
                float2 v = make_float2(0.f, 0.f);
                if (i < npx && j0 + jj < a.Nw) v = G[((size_t)p * a.n_mpix + g0 + i) * a.Nw + j0 + jj];
                gs[jj][i] = v;
            }
            __syncthreads();
            if (t < a.T) {
                const int jn = min(JCH, a.Nw - j0);
                for (int jj = 0; jj < jn; ++jj) {
                    const float2 b = a.B32[(size_t)t * a.Nw_pad + j0 + jj];   // w_t e^{-i theta}
#pragma unroll
                    for (int i = 0; i < ADJ_PIX; ++i) {
                        const float2 g = gs[jj][i];
                        // g * conj(b)
                        cr[i] = fmaf(g.x, b.x, fmaf(g.y, b.y, cr[i]));
                        ci[i] = fmaf(g.y, b.x, fmaf(-g.x, b.y, ci[i]));
                    }
                }
            }
        }
        if (t < a.T) {
            for (int i = 0; i < npx; ++i) {
                const int pix = a.mpix[g0 + i];
                const int y = pix / a.kx, x = pix - (pix / a.kx) * a.kx;
                const float2 K = Kc[(size_t)p * a.n_mpix + g0 + i];
                float2 *gp = a.grad + (int64_t)p * a.pitch_probe + (int64_t)t * a.pitch_frame +
                             (int64_t)(a.roi_y0 + y) * a.pitch_row + (a.roi_x0 + x);
                const float2 v = make_float2(2.f * a.scale * (cr[i] - K.x), 2.f * a.scale * (ci[i] - K.y));
                if (a.accumulate) {
                    const float2 o = *gp;
                    *gp = make_float2(o.x + v.x, o.y + v.y);
                } else {
                    *gp = v;
                }
            }
        }
    }
}

// zero every ROI element of the gradient (layout of the frames)
__global__ void zero_roi_kernel(AdjointArgs a) {
    const int64_t npix = (int64_t)a.kx * a.ky;
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (int64_t)a.P * a.T * npix) return;
    const int64_t pix = id % npix;
    const int64_t pt = id / npix;
    const int t = (int)(pt % a.T), p = (int)(pt / a.T);
    const int64_t y = pix / a.kx, x = pix - (pix / a.kx) * a.kx;
    a.grad[(int64_t)p * a.pitch_probe + (int64_t)t * a.pitch_frame + (a.roi_y0 + y) * a.pitch_row + (a.roi_x0 + x)] =
        make_float2(0.f, 0.f);
}

cudaError_t launch_zero_roi(const AdjointArgs &a, cudaStream_t st) {
    const int64_t n = (int64_t)a.P * a.T * a.kx * a.ky;
    zero_roi_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adjoint(const AdjointArgs &a, cudaStream_t st) {
    if (a.n_mpix == 0 || a.P == 0) return cudaSuccess;
    dim3 grd((a.n_mpix + ADJ_PIX - 1) / ADJ_PIX, a.P);
    adj_forward_kernel<<<grd, 256, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    adj_backward_kernel<<<grd, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace tacaw
