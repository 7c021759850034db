// Adjoint of the spectrum on the tensor cores (split BF16): the two contractions of the adjoint
// (see k_adjoint.cu for the algebra) run on the staged drained tcgen05 kernel of k_tc_gemm.cu,
// over the compact list of aperture rows m = p * n_mpix + i (probe p, aperture pixel i):
//
//   1. Psi on the aperture rows
//        Psi[m, j] = sum_t (psi[t, m] - psi[0, m]) B[t, j] - (mu - psi_0)[m] W_j
//      operand A: each row's frames minus its first frame (the provisional mean keeps the
//      elastic part out of the bf16 pieces), staged as bf16 hi/lo rows of 32 frames; operand B:
//      the forward twiddles w_t exp(-i theta_jt) in 32-frame blocks.  The flush epilogue applies
//      the exact mean correction and writes Psi[p][j][i].
//   2. G[m, j] = 2 s B(E_j) (sum_d dL/dS[p, d, j] M_d(k)) Psi[m, j]  (s: the segment's weight),
//      staged the same way with 32 energies per block, and K[m] = (1/T) sum_j conj(W_j) G[m, j]
//   3. C[m, t] = sum_j G[m, j] conj(B[t, j]) - K[m]
//      the same kernel with frames as its output columns: operand B is the table of
//      conj(B[t, j]) = w_t exp(+i theta_jt) whose rows 2t, 2t+1 hold its real embedding, the
//      per-row correction is K (a "window transform" of ones), output C[p][t][i]
//   4. grad[p, t, k] = C[m, t] (or +=, for Welch segments that overlap) at the element of the
//      frame layout that row m's pixel occupies
// Every staged row is written in full (zeros past the frames, energies or rows that exist), so
// the scratch needs no clearing between calls.
#include <algorithm>

#include "tacaw_internal.cuh"

namespace tacaw {

constexpr int kAdjBlock = 32;   // frames (or energies) per staged block: 128-byte rows of bf16 pairs

// complex64 offset of row m's pixel in frame 0 of the pushed layout
__device__ __forceinline__ int64_t adjtc_row_offset(const AdjointArgs &a, int64_t m) {
    const int p = (int)(m / a.n_mpix);
    const int pix = a.mpix[m - (int64_t)p * a.n_mpix];
    const int y = pix / a.kx, x = pix - y * a.kx;
    return (int64_t)p * a.pitch_probe + (int64_t)(a.roi_y0 + y) * a.pitch_row + (a.roi_x0 + x);
}

// (re, im) -> bf16 pairs hi = RN(re, im) and lo = RN(residuals), re in the low half
__device__ __forceinline__ void adjtc_split(float re, float im, uint32_t &hi, uint32_t &lo) {
    const __nv_bfloat16 hr = __float2bfloat16_rn(re), hm = __float2bfloat16_rn(im);
    const __nv_bfloat16 lr = __float2bfloat16_rn(re - __bfloat162float(hr));
    const __nv_bfloat16 lm = __float2bfloat16_rn(im - __bfloat162float(hm));
    hi = (uint32_t)__bfloat16_as_ushort(hr) | ((uint32_t)__bfloat16_as_ushort(hm) << 16);
    lo = (uint32_t)__bfloat16_as_ushort(lr) | ((uint32_t)__bfloat16_as_ushort(lm) << 16);
}

// Shared-memory tile of one block of 128 staged rows: 32 bf16 pairs a row (hi and lo), rows
// padded to 36 words so that a thread's 16-byte chunk stores and the store phase's row reads
// are free of bank conflicts.
constexpr int kAdjRowWords = 36;
struct AdjTile {
    uint32_t hi[128 * kAdjRowWords];
    uint32_t lo[128 * kAdjRowWords];
};

__device__ __forceinline__ void adjtc_put(AdjTile &sm, int r, int w4, uint32_t h0, uint32_t h1, uint32_t h2,
                                          uint32_t h3, uint32_t l0, uint32_t l1, uint32_t l2, uint32_t l3) {
    *reinterpret_cast<uint4 *>(&sm.hi[r * kAdjRowWords + 4 * w4]) = make_uint4(h0, h1, h2, h3);
    *reinterpret_cast<uint4 *>(&sm.lo[r * kAdjRowWords + 4 * w4]) = make_uint4(l0, l1, l2, l3);
}

// Writes the block's 128 rows (rows m0 .. m0 + 127 of block kb, 128 bytes each, M_pad rows a
// block) from shared memory, the 16-byte chunks in the order of the tensor core's 128-byte
// shared-memory swizzle (chunk c of row m at c ^ (m mod 8)), so that a contiguous copy of the
// rows gives the swizzled operand tile.  A warp writes four whole rows (512 contiguous bytes).
__device__ __forceinline__ void adjtc_store_tile(const AdjTile &sm, __nv_bfloat16 *dst_hi, __nv_bfloat16 *dst_lo,
                                                 int64_t M_pad, int kb, int64_t m0) {
    uint4 *H = reinterpret_cast<uint4 *>(dst_hi) + ((size_t)kb * (size_t)M_pad + (size_t)m0) * 8;
    uint4 *L = reinterpret_cast<uint4 *>(dst_lo) + ((size_t)kb * (size_t)M_pad + (size_t)m0) * 8;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int q = (int)threadIdx.x + 128 * k;     // chunk q of the 1024 in the tile
        const int r = q >> 3, c = q & 7;
        const int pos = r * 8 + (c ^ (int)((m0 + r) & 7));
        H[pos] = *reinterpret_cast<const uint4 *>(&sm.hi[r * kAdjRowWords + 4 * c]);
        L[pos] = *reinterpret_cast<const uint4 *>(&sm.lo[r * kAdjRowWords + 4 * c]);
    }
}

// grid (M_pad / 128, T_pad / 32): thread = (row m, block kb of 32 frames).  Stages
// psi[t, m] - ref[m] (ref = the first frame with subtract_mean, else 0) as bf16 hi/lo and
// writes the block's FP32 sum of those residuals to part[kb][m].
__global__ void __launch_bounds__(128) adjtc_stage_frames_kernel(AdjTcArgs q) {
    __shared__ __align__(16) AdjTile sm;
    const AdjointArgs &a = q.a;
    const int64_t M = (int64_t)a.P * a.n_mpix;
    const int64_t m0 = (int64_t)blockIdx.x * 128, m = m0 + threadIdx.x;
    const int kb = blockIdx.y;
    if (m < M) {
        const float2 *src = a.frames + adjtc_row_offset(a, m);
        const float2 ref = a.subtract_mean ? src[0] : make_float2(0.f, 0.f);
        float2 v[kAdjBlock];
#pragma unroll
        for (int i = 0; i < kAdjBlock; ++i) {
            const int t = kb * kAdjBlock + i;
            v[i] = t < a.T ? __ldg(src + (int64_t)t * a.pitch_frame) : ref;
        }
        float sr = 0.f, si = 0.f;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            uint32_t h[4], l[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float re = v[4 * c + u].x - ref.x, im = v[4 * c + u].y - ref.y;
                sr += re;
                si += im;
                adjtc_split(re, im, h[u], l[u]);
            }
            adjtc_put(sm, threadIdx.x, c, h[0], h[1], h[2], h[3], l[0], l[1], l[2], l[3]);
        }
        q.part[(size_t)kb * (size_t)M + (size_t)m] = make_float2(sr, si);
    } else {
#pragma unroll
        for (int c = 0; c < 8; ++c) adjtc_put(sm, threadIdx.x, c, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u);
    }
    __syncthreads();
    adjtc_store_tile(sm, q.A_hi, q.A_lo, q.M_pad, kb, m0);
}

// out[m] = inv * sum_k part[k][m] (FP64, fixed order), or 0 when inv == 0
__global__ void __launch_bounds__(256) adjtc_rowsum_kernel(const float2 *part, int n_parts, int64_t M, double inv,
                                                           float2 *out) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double sr = 0.0, si = 0.0;
    if (inv != 0.0)
        for (int k = 0; k < n_parts; ++k) {
            const float2 v = part[(size_t)k * (size_t)M + (size_t)m];
            sr += v.x;
            si += v.y;
        }
    out[m] = make_float2((float)(sr * inv), (float)(si * inv));
}

// grid (M_pad / 128, E_pad / 32): thread = (row m, block e of 32 energies).  Stages
// G[m, j] = 2 s B(E_j) c_j(p, i) Psi[p][j][i], c_j = sum_d dL/dS[p, d, j] M_d(pixel i), as bf16
// hi/lo and writes the block's part of sum_j conj(W_j) G[m, j] to part[e][m].  Energies go in
// groups of 8 (their loads issued together).
__global__ void __launch_bounds__(128) adjtc_stage_g_kernel(AdjTcArgs q) {
    __shared__ __align__(16) AdjTile sm;
    const AdjointArgs &a = q.a;
    const int64_t M = (int64_t)a.P * a.n_mpix;
    const int64_t m0 = (int64_t)blockIdx.x * 128, m = m0 + threadIdx.x;
    const int e = blockIdx.y;
    if (m < M) {
        const int p = (int)(m / a.n_mpix);
        const int64_t i = m - (int64_t)p * a.n_mpix;
        const float s2 = 2.f * a.scale;
        const float2 *ps = q.psi + (size_t)p * a.Nw * (size_t)a.n_mpix + (size_t)i;
        const float *dl = a.dLdS + (size_t)p * a.D * a.Nw;
        const float *mw = a.mwts + i * a.D;
        float kr = 0.f, ki = 0.f;
#pragma unroll 1
        for (int g8 = 0; g8 < kAdjBlock / 8; ++g8) {
            const int j0 = e * kAdjBlock + 8 * g8;
            float2 v[8];
            float c[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const bool ok = j0 + u < a.Nw;
                v[u] = ok ? ps[(size_t)(j0 + u) * a.n_mpix] : make_float2(0.f, 0.f);
                c[u] = 0.f;
            }
            for (int d = 0; d < a.D; ++d) {
                const float w = mw[d];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (j0 + u < a.Nw) c[u] += dl[(size_t)d * a.Nw + j0 + u] * w;
            }
            uint32_t h[8], l[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                float gr = 0.f, gi = 0.f;
                if (j0 + u < a.Nw) {
                    const float cc = c[u] * s2 * a.bose[j0 + u];
                    gr = cc * v[u].x;
                    gi = cc * v[u].y;
                    const float2 W = a.Wc[j0 + u];
                    kr += W.x * gr + W.y * gi;      // conj(W) G
                    ki += W.x * gi - W.y * gr;
                }
                adjtc_split(gr, gi, h[u], l[u]);
            }
            adjtc_put(sm, threadIdx.x, 2 * g8, h[0], h[1], h[2], h[3], l[0], l[1], l[2], l[3]);
            adjtc_put(sm, threadIdx.x, 2 * g8 + 1, h[4], h[5], h[6], h[7], l[4], l[5], l[6], l[7]);
        }
        q.part[(size_t)e * (size_t)M + (size_t)m] = make_float2(kr, ki);
    } else {
#pragma unroll
        for (int c = 0; c < 8; ++c) adjtc_put(sm, threadIdx.x, c, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u);
    }
    __syncthreads();
    adjtc_store_tile(sm, q.G_hi, q.G_lo, q.M_pad, e, m0);
}

// grad[p, t, pixel of i] = C[p][t][i] (stored, or added with accumulate): one block per (p, t)
// (blockIdx.x = p * T + t), threads over the aperture pixels, whose offsets within a frame are
// tabulated (pix_off)
__global__ void __launch_bounds__(256) adjtc_scatter_kernel(AdjTcArgs q) {
    const AdjointArgs &a = q.a;
    const int64_t r = blockIdx.x;
    const int t = (int)(r % a.T), p = (int)(r / a.T);
    float2 *g = a.grad + (int64_t)p * a.pitch_probe + (int64_t)t * a.pitch_frame;
    const float2 *c = q.cg + r * a.n_mpix;
    for (int i = threadIdx.x; i < a.n_mpix; i += blockDim.x) {
        const float2 v = c[i];
        float2 *d = g + q.pix_off[i];
        if (a.accumulate) {
            const float2 o = *d;
            *d = make_float2(o.x + v.x, o.y + v.y);
        } else {
            *d = v;
        }
    }
}

// Tensor-core arguments of one adjoint contraction: rows = the aperture rows, output columns
// n_out (energies, or frames) in tiles of wt, contraction over n_kb blocks of 32.
static TcPlanArgs adjtc_flush_args(const AdjTcArgs &q, int n_out, int wt, int n_wt, int n_kb,
                                   const __nv_bfloat16 *A_hi, const __nv_bfloat16 *A_lo, const __nv_bfloat16 *B_hi,
                                   const __nv_bfloat16 *B_lo, float2 *out, const float2 *dmu, const float2 *W,
                                   const float *bose, int *counter) {
    TcPlanArgs t{};
    EpiArgs &e = t.e;
    e.M = (int64_t)q.a.P * q.a.n_mpix;
    e.M_pad = q.M_pad;
    e.npix = q.a.n_mpix;
    e.Nw = n_out;
    e.mode = FLUSH_FINAL;
    e.Psi_out = out;
    e.dmu = dmu;
    e.Wc = W;
    e.bose = bose;
    e.out_scale = 1.f;
    e.psi_scale = 1.f;
    t.wt = wt;
    t.n_wt = n_wt;
    t.N = 2 * wt;
    const int last = n_out - (n_wt - 1) * wt;
    t.N_last = std::min(t.N, (2 * last + 15) / 16 * 16);
    t.n_kb = n_kb;
    t.kbB0 = 0;
    t.bf = kAdjBlock;
    t.drain_kb = 512 / kAdjBlock;   // H drained every 512 frames, as in the forward flushes
    t.A_hi = A_hi;
    t.A_lo = A_lo;
    t.B_hi = B_hi;
    t.B_lo = B_lo;
    t.a_rows = q.M_pad;
    t.b_rows = 2 * wt * n_wt;
    t.err = q.err;
    t.wait_ns = q.wait_ns;
    t.tile_counter = counter;
    return t;
}

int adjtc_launches() { return 7; }

cudaError_t launch_adjoint_tc(const AdjTcArgs &q, cudaStream_t st) {
    const AdjointArgs &a = q.a;
    const int64_t M = (int64_t)a.P * a.n_mpix;
    if (M == 0 || a.T == 0 || a.Nw == 0) return cudaSuccess;
    if (q.M_pad % kMTile || q.M_pad < M || q.T_pad % kAdjBlock || q.E_pad % kAdjBlock || q.T_pad < a.T ||
        q.E_pad < a.Nw || q.wt1 * q.n_wt1 < a.Nw || q.wt2 * q.n_wt2 < a.T || q.M_pad / kMTile > 0x7fffffffLL)
        return cudaErrorInvalidValue;
    const unsigned rows = (unsigned)(q.M_pad / 128);
    const int n_kbT = q.T_pad / kAdjBlock, n_kbE = q.E_pad / kAdjBlock;
    if (n_kbT > 65535 || n_kbE > 65535) return cudaErrorInvalidValue;
    // 1. frames of the aperture rows -> staged bf16 pieces; mean residual mu - psi_0
    adjtc_stage_frames_kernel<<<dim3(rows, n_kbT), 128, 0, st>>>(q);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned rb = (unsigned)((M + 255) / 256);
    adjtc_rowsum_kernel<<<rb, 256, 0, st>>>(q.part, n_kbT, M, a.subtract_mean ? 1.0 / a.T : 0.0, q.dmu);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    //    Psi on the aperture rows (exact mean correction in the epilogue)
    TcPlanArgs f1 = adjtc_flush_args(q, a.Nw, q.wt1, q.n_wt1, n_kbT, q.A_hi, q.A_lo, q.Bf_hi, q.Bf_lo, q.psi,
                                     q.dmu, a.Wc, a.bose, q.counters);
    if ((e = launch_flush_tc(f1, st)) != cudaSuccess) return e;
    // 2. G and K
    adjtc_stage_g_kernel<<<dim3(rows, n_kbE), 128, 0, st>>>(q);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    adjtc_rowsum_kernel<<<rb, 256, 0, st>>>(q.part, n_kbE, M, a.subtract_mean ? 1.0 / a.T : 0.0, q.kmean);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // 3. C - K over the frames
    TcPlanArgs f2 = adjtc_flush_args(q, a.T, q.wt2, q.n_wt2, n_kbE, q.G_hi, q.G_lo, q.Bc_hi, q.Bc_lo, q.cg, q.kmean,
                                     q.ones, q.ones_f, q.counters + 1);
    if ((e = launch_flush_tc(f2, st)) != cudaSuccess) return e;
    // 4. into the frame layout (after the zero fill of the whole gradient, if it runs elsewhere)
    if (q.before_scatter && (e = cudaStreamWaitEvent(st, q.before_scatter, 0)) != cudaSuccess) return e;
    const int64_t blocks = (int64_t)a.P * a.T;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    adjtc_scatter_kernel<<<(unsigned)blocks, 256, 0, st>>>(q);
    return cudaGetLastError();
}

}  // namespace tacaw
