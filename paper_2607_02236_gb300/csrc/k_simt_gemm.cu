// FP32 CUDA-core contraction of staged frames with the twiddle table:
//   Psi[m, j] (+)= sum_{f < n_frames} A32[f][m] * B32[t0 + f][j]     (complex, FP32 FFMA)
// the windowed time->energy transform of Eq. 1 for the frames of one flush.  This is the
// plain-precision path (and the baseline the tensor-core path is measured against).
//
// Tile: 128 rows x 64 complex energies per 256-thread block, 8 frames per step staged in
// shared memory; each thread owns 8 rows x 4 energies (rows tx + 16 i, energies ty + 16 jj).
#include "tacaw_internal.cuh"

namespace tacaw {

constexpr int SB_M = 128, SB_N = 64, SB_K = 8;

__global__ void __launch_bounds__(256) flush_simt_kernel(SimtArgs a, int n_jt) {
    __shared__ float2 As[SB_K][SB_M];
    __shared__ float2 Bs[SB_K][SB_N];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int jt = blockIdx.x % n_jt;
    const int64_t mt = blockIdx.x / n_jt;
    const int64_t m0 = mt * SB_M;
    const int j0 = jt * SB_N;
    const int64_t M_pad = a.e.M_pad;

    float ar[8][4], ai[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) ar[i][q] = ai[i][q] = 0.f;

    for (int k0 = 0; k0 < a.n_frames; k0 += SB_K) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int idx = tid + 256 * q;
            int kk = idx >> 7, r = idx & 127;
            float2 v = make_float2(0.f, 0.f);
            if (k0 + kk < a.n_frames) v = a.A32[(size_t)(k0 + kk) * M_pad + m0 + r];
            As[kk][r] = v;
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            int idx = tid + 256 * q;
            int kk = idx >> 6, c = idx & 63;
            float2 v = make_float2(0.f, 0.f);
            if (k0 + kk < a.n_frames && j0 + c < a.e.Nw)
                v = a.B32[(size_t)(a.t0 + k0 + kk) * a.Nw_pad + j0 + c];
            Bs[kk][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < SB_K; ++kk) {
            float2 x[8], b[4];
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int q = 0; q < 4; ++q) b[q] = Bs[kk][ty + 16 * q];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    ar[i][q] = fmaf(x[i].x, b[q].x, ar[i][q]);
                    ar[i][q] = fmaf(-x[i].y, b[q].y, ar[i][q]);
                    ai[i][q] = fmaf(x[i].x, b[q].y, ai[i][q]);
                    ai[i][q] = fmaf(x[i].y, b[q].x, ai[i][q]);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t m = m0 + tx + 16 * i;
        RowCtx row = make_row(a.e, m);
        if (!row.valid) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = j0 + ty + 16 * q;
            if (j < a.e.Nw) epi_element(a.e, row, j, ar[i][q], ai[i][q]);
        }
    }
}

cudaError_t launch_flush_simt(const SimtArgs &a, cudaStream_t st) {
    const int n_jt = (a.e.Nw + SB_N - 1) / SB_N;
    const int64_t n_mt = a.e.M_pad / SB_M;
    const int64_t blocks = n_mt * n_jt;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    flush_simt_kernel<<<(unsigned)blocks, 256, 0, st>>>(a, n_jt);
    return cudaGetLastError();
}

}  // namespace tacaw
