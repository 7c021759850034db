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
// pixel list: rows m = p * n_mpix + i (probe p, aperture pixel i).  Psi is recomputed from
// the frames (the window and twiddles come from the plan's table), never stored between
// forward and backward.
//
// Both contractions are complex GEMMs tiled for the CUDA cores: a block of 4 x TN threads owns a
// 64-row x TN-column tile (TN = 64, or 32 for the forward when that pads the energies less),
// each thread a 4 x 4 tile of complex accumulators (rows tx + 16a, columns ty + (TN/4) b), with
// 16-deep slices of both operands staged in shared memory by coalesced loads, double-buffered
// (the next slice's loads in flight during the FMAs).
//   forward  Psi'[m][j] = sum_t (psi[t,m] - psi[0,m]) B[t][j]      (K = T, N = Nw)
//            Psi = Psi' - (mu - psi_0) W_j  (the first frame as provisional mean keeps the
//            elastic part out of the FP32 sums; the row sums ride along in the tile loads);
//            G is written transposed, Gt[j][m], for the backward's coalesced loads
//   backward C[m][t] = sum_j Gt[j][m] conj(B[t][j])                 (K = Nw, N = T)
//            with K[m] = (1/T) sum_j conj(W_j) Gt[j][m] summed by the same tile loads
#include "tacaw_internal.cuh"

namespace tacaw {

constexpr int ADJ_TM = 64;     // rows per block tile
constexpr int ADJ_TN = 64;     // columns (energies or frames) per block tile
constexpr int ADJ_TK = 16;     // contraction depth per staged slice

// complex64 offset of row m's pixel in frame 0 of the pushed layout
__device__ __forceinline__ int64_t adj_row_offset(const AdjointArgs &a, int64_t m) {
    const int p = (int)(m / a.n_mpix);
    const int pix = a.mpix[m - (int64_t)p * a.n_mpix];
    const int y = pix / a.kx, x = pix - (pix / a.kx) * a.kx;
    return (int64_t)p * a.pitch_probe + (int64_t)(a.roi_y0 + y) * a.pitch_row + (a.roi_x0 + x);
}

__device__ __forceinline__ void cmac(float2 &acc, float2 x, float2 b) {
    acc.x = fmaf(x.x, b.x, fmaf(-x.y, b.y, acc.x));
    acc.y = fmaf(x.x, b.y, fmaf(x.y, b.x, acc.y));
}

// One 16-deep step of the 4 x 4 complex register tile: rows tx + 16 i, columns ty + (TN / 4) j.
template <int TN>
__device__ __forceinline__ void tile_step(const float2 (*As)[ADJ_TM], const float2 (*Bs)[TN + 1], int tx, int ty,
                                          float2 (&acc)[4][4]) {
#pragma unroll
    for (int kk = 0; kk < ADJ_TK; ++kk) {
        float2 x[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) x[i] = As[kk][tx + 16 * i];
#pragma unroll
        for (int i = 0; i < 4; ++i) b[i] = Bs[kk][ty + (TN / 4) * i];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) cmac(acc[i][jj], x[i], b[jj]);
    }
}

// grid (row tiles, energy tiles of TN): G^T[j][m] for all aperture rows.  16 x TN/4 threads, each a
// 4 x 4 complex register tile.  The operand slices are double-buffered: the next slice's global
// loads are in flight (in registers) while the current slice's FMAs run from shared memory, one
// barrier per slice.
template <int TN>
__global__ void __launch_bounds__(4 * TN, 128 / TN) adj_psi_kernel(AdjointArgs a) {
    constexpr int NT = 4 * TN;                 // threads
    constexpr int NA = ADJ_TM * ADJ_TK / NT;   // A elements each thread stages per slice
    constexpr int NB = TN * ADJ_TK / NT;       // B elements each thread stages per slice (4)
    __shared__ float2 As[2][ADJ_TK][ADJ_TM];
    __shared__ float2 Bs[2][ADJ_TK][TN + 1];
    __shared__ float2 rsum[NT / ADJ_TM][ADJ_TM];
    __shared__ float2 ref[ADJ_TM];
    __shared__ int64_t roff[ADJ_TM];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t M = (int64_t)a.P * a.n_mpix;
    const int64_t m0 = (int64_t)blockIdx.x * ADJ_TM;
    const int n0 = blockIdx.y * TN;
    // this thread's load slot: row lr of every slice, frames lk, lk + NT/64, ...
    const int lr = tid & (ADJ_TM - 1), lk = tid / ADJ_TM;
    if (tid < ADJ_TM) {
        const int64_t m = m0 + tid;
        float2 v = make_float2(0.f, 0.f);
        int64_t o = 0;
        if (m < M) {
            o = adj_row_offset(a, m);
            if (a.subtract_mean) v = a.frames[o];      // provisional mean: the first frame
        }
        roff[tid] = o;
        ref[tid] = v;
    }
    __syncthreads();
    const bool row_ok = m0 + lr < M;
    const int64_t my_off = roff[lr];
    const float2 my_ref = ref[lr];
    float sr = 0.f, si = 0.f;
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) acc[i][jj] = make_float2(0.f, 0.f);
    float2 ra[NA], rb[NB];
    // slice t0 of both operands into registers (frames minus the provisional mean; twiddles)
    auto load = [&](int t0) {
#pragma unroll
        for (int q = 0; q < NA; ++q) {
            const int t = t0 + lk + (NT / ADJ_TM) * q;
            float2 v = make_float2(0.f, 0.f);
            if (row_ok && t < a.T) {
                v = a.frames[my_off + (int64_t)t * a.pitch_frame];
                v.x -= my_ref.x;
                v.y -= my_ref.y;
            }
            ra[q] = v;
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int e = tid + NT * q, kk = e / TN, nn = e % TN, tb = t0 + kk, j = n0 + nn;
            rb[q] = (tb < a.T && j < a.Nw) ? a.B32[(size_t)tb * a.Nw_pad + j] : make_float2(0.f, 0.f);
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int q = 0; q < NA; ++q) {
            sr += ra[q].x;
            si += ra[q].y;
            As[buf][lk + (NT / ADJ_TM) * q][lr] = ra[q];
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int e = tid + NT * q;
            Bs[buf][e / TN][e % TN] = rb[q];
        }
    };
    load(0);
    store(0);
    __syncthreads();
    int buf = 0;
    for (int t0 = 0; t0 < a.T; t0 += ADJ_TK) {
        const bool more = t0 + ADJ_TK < a.T;
        if (more) load(t0 + ADJ_TK);
        tile_step<TN>(As[buf], Bs[buf], tx, ty, acc);
        if (more) store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
    rsum[lk][lr] = make_float2(sr, si);
    __syncthreads();
    float2 *Gt = a.scratch;                                   // [Nw][M]
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = tx + 16 * i;
        const int64_t m = m0 + r;
        if (m >= M) continue;
        // Psi = Psi' - (mu - psi_0) W  (subtract_mean), else Psi' itself (psi_0 = 0)
        float2 dmu = make_float2(0.f, 0.f);
        if (a.subtract_mean) {
            float xr = 0.f, xi = 0.f;
#pragma unroll
            for (int h = 0; h < NT / ADJ_TM; ++h) {
                xr += rsum[h][r].x;
                xi += rsum[h][r].y;
            }
            dmu = make_float2(xr / a.T, xi / a.T);
        }
        const int p = (int)(m / a.n_mpix);
        const int64_t ip = m - (int64_t)p * a.n_mpix;
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int j = n0 + ty + (TN / 4) * jj;
            if (j >= a.Nw) continue;
            const float2 W = a.Wc[j];
            float c = 0.f;
            for (int d = 0; d < a.D; ++d) c += a.dLdS[((size_t)p * a.D + d) * a.Nw + j] * a.mwts[ip * a.D + d];
            c *= a.bose[j];
            const float pr = acc[i][jj].x - (dmu.x * W.x - dmu.y * W.y);
            const float pi = acc[i][jj].y - (dmu.x * W.y + dmu.y * W.x);
            Gt[(size_t)j * M + m] = make_float2(c * pr, c * pi);
        }
    }
}

// grid (row tiles, frame tiles): C[m][t] = sum_j Gt[j][m] conj(B[t][j]); grad = 2 scale (C - K).
// Double-buffered operand slices as in adj_psi_kernel.
__global__ void __launch_bounds__(256, 2) adj_grad_kernel(AdjointArgs a) {
    __shared__ float2 As[2][ADJ_TK][ADJ_TM];
    __shared__ float2 Bs[2][ADJ_TK][ADJ_TN + 1];
    __shared__ float2 ksum[4][ADJ_TM];
    __shared__ int64_t roff[ADJ_TM];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t M = (int64_t)a.P * a.n_mpix;
    const int64_t m0 = (int64_t)blockIdx.x * ADJ_TM;
    const int tb0 = blockIdx.y * ADJ_TN;
    const int lr = tid & (ADJ_TM - 1), lk = tid >> 6;
    if (tid < ADJ_TM) roff[tid] = (m0 + tid < M) ? adj_row_offset(a, m0 + tid) : 0;
    const float2 *Gt = a.scratch;
    const bool row_ok = m0 + lr < M;
    float kr = 0.f, ki = 0.f;
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) acc[i][jj] = make_float2(0.f, 0.f);
    float2 ra[4], rb[4];
    // slice j0: G rows (energies j0 + lk + 4q of row lr) and conj(B[t][j]) for 64 frames x 16
    // energies, 16 consecutive energies of a frame per 16 threads (128-byte rows of the table)
    auto load = [&](int j0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = j0 + lk + 4 * q;
            ra[q] = (row_ok && j < a.Nw) ? Gt[(size_t)j * M + m0 + lr] : make_float2(0.f, 0.f);
            const int e = tid + 256 * q, kk = e & 15, nn = e >> 4, t = tb0 + nn, jb = j0 + kk;
            float2 bv = make_float2(0.f, 0.f);
            if (t < a.T && jb < a.Nw) {
                bv = a.B32[(size_t)t * a.Nw_pad + jb];
                bv.y = -bv.y;
            }
            rb[q] = bv;
        }
    };
    auto store = [&](int buf, int j0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = j0 + lk + 4 * q;
            if (j < a.Nw) {
                const float2 W = a.Wc[j];
                kr += W.x * ra[q].x + W.y * ra[q].y;       // conj(W) G
                ki += W.x * ra[q].y - W.y * ra[q].x;
            }
            As[buf][lk + 4 * q][lr] = ra[q];
            const int e = tid + 256 * q;
            Bs[buf][e & 15][e >> 4] = rb[q];
        }
    };
    load(0);
    store(0, 0);
    __syncthreads();
    int buf = 0;
    for (int j0 = 0; j0 < a.Nw; j0 += ADJ_TK) {
        const bool more = j0 + ADJ_TK < a.Nw;
        if (more) load(j0 + ADJ_TK);
        tile_step<ADJ_TN>(As[buf], Bs[buf], tx, ty, acc);
        if (more) store(buf ^ 1, j0 + ADJ_TK);
        __syncthreads();
        buf ^= 1;
    }
    ksum[lk][lr] = make_float2(kr, ki);
    __syncthreads();
    const float s2 = 2.f * a.scale;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = tx + 16 * i;
        if (m0 + r >= M) continue;
        float2 K = make_float2(0.f, 0.f);
        if (a.subtract_mean) {
            K.x = (((ksum[0][r].x + ksum[1][r].x) + ksum[2][r].x) + ksum[3][r].x) / a.T;
            K.y = (((ksum[0][r].y + ksum[1][r].y) + ksum[2][r].y) + ksum[3][r].y) / a.T;
        }
        const int64_t o = roff[r];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int t = tb0 + ty + 16 * jj;
            if (t >= a.T) continue;
            float2 *gp = a.grad + o + (int64_t)t * a.pitch_frame;
            const float2 v = make_float2(s2 * (acc[i][jj].x - K.x), s2 * (acc[i][jj].y - K.y));
            if (a.accumulate) {
                const float2 old = *gp;
                *gp = make_float2(old.x + v.x, old.y + v.y);
            } else {
                *gp = v;
            }
        }
    }
}

// zero every ROI element of the gradient (layout of the frames): one warp per frame row
// (p, t, y) of the ROI, consecutive lanes on consecutive pixels
__global__ void __launch_bounds__(256) zero_roi_kernel(AdjointArgs a, int64_t rows) {
    const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (r >= rows) return;
    const int y = (int)(r % a.ky);
    const int64_t pt = r / a.ky;
    const int t = (int)(pt % a.T), p = (int)(pt / a.T);
    float2 *row = a.grad + (int64_t)p * a.pitch_probe + (int64_t)t * a.pitch_frame +
                  (int64_t)(a.roi_y0 + y) * a.pitch_row + a.roi_x0;
    for (int x = threadIdx.x & 31; x < a.kx; x += 32) row[x] = make_float2(0.f, 0.f);
}

cudaError_t launch_zero_roi(const AdjointArgs &a, cudaStream_t st) {
    const int64_t rows = (int64_t)a.P * a.T * a.ky;
    if (rows == 0) return cudaSuccess;
    zero_roi_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(a, rows);
    return cudaGetLastError();
}

cudaError_t launch_adjoint(const AdjointArgs &a, cudaStream_t st) {
    const int64_t M = (int64_t)a.P * a.n_mpix;
    if (M == 0 || a.T == 0) return cudaSuccess;
    const unsigned mt = (unsigned)((M + ADJ_TM - 1) / ADJ_TM);
    if ((a.T + ADJ_TN - 1) / ADJ_TN > 65535 || (a.Nw + 31) / 32 > 65535) return cudaErrorInvalidValue;
    // energy tiles of 64 or 32: the narrower one when it pads the energies less (200 energies:
    // 224 columns issued against 256)
    const int64_t pad64 = (a.Nw + 63) / 64 * 64, pad32 = (a.Nw + 31) / 32 * 32;
    if (pad32 < pad64)
        adj_psi_kernel<32><<<dim3(mt, (a.Nw + 31) / 32), 128, 0, st>>>(a);
    else
        adj_psi_kernel<64><<<dim3(mt, (a.Nw + 63) / 64), 256, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    adj_grad_kernel<<<dim3(mt, (a.T + ADJ_TN - 1) / ADJ_TN), 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace tacaw
