// FP32 CUDA-core contraction of staged frames with the twiddle table:
//   Psi[m, j] (+)= sum_{f < n_frames} A32[f][m] * B32[t0 + f][j]     (complex, FP32 FFMA)
// the windowed time->energy transform of Eq. 1 for the frames of one flush.  This is the
// plain-precision path (and the baseline the tensor-core path is measured against).
//
// Tile: 128 rows x SN = Q*TY complex energies per block of 16 x TY threads; each thread owns
// 8 rows x Q energies (rows tx + 16 i, energies ty + TY q).  Shapes: TY = 16, Q = 4 (64
// energies, 8 warps); TY = 8, Q = 4 (32 energies) or Q = 5 (40 energies, 4 warps): whichever
// pads the energy count least (200 or 400 energies: 40, no padding).  Slices of 8 frames of
// both operands are copied global -> shared with cp.async (16-byte pieces, no registers) into
// a 4-deep ring, so three slices are in flight while one is multiplied; one barrier per slice.
#include "tacaw_internal.cuh"

namespace tacaw {

constexpr int SB_M = 128, SB_K = 8, SB_STAGES = 4;

template <int TY, int Q>
constexpr size_t simt_smem_bytes() { return (size_t)SB_STAGES * SB_K * (SB_M + Q * TY) * sizeof(float2); }

__device__ __forceinline__ void cp_async16_zfill(uint32_t dst, const void *src, bool valid) {
    // src-size 0 writes 16 zero bytes and reads nothing
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int TY, int Q>
__global__ void __launch_bounds__(16 * TY) flush_simt_kernel(SimtArgs a, int n_jt) {
    constexpr int NT = 16 * TY, SN = Q * TY;
    constexpr int A_CHUNKS = SB_K * SB_M / 2;    // 16-byte pieces of one A slice
    constexpr int B_CHUNKS = SB_K * SN / 2;      // ... of one B slice
    static_assert(SN % 2 == 0, "whole 16-byte pieces of B");
    extern __shared__ __align__(16) unsigned char simt_smem[];
    float2 (*As)[SB_K][SB_M] = reinterpret_cast<float2 (*)[SB_K][SB_M]>(simt_smem);
    float2 (*Bs)[SB_K][SN] =
        reinterpret_cast<float2 (*)[SB_K][SN]>(simt_smem + (size_t)SB_STAGES * SB_K * SB_M * sizeof(float2));
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int jt = blockIdx.x % n_jt;
    const int64_t mt = blockIdx.x / n_jt;
    const int64_t m0 = mt * SB_M;
    const int j0 = jt * SN;
    const int64_t M_pad = a.e.M_pad;
    const int n_slices = (a.n_frames + SB_K - 1) / SB_K;

    // slice s into ring slot s % SB_STAGES; frames past n_frames and energies past the twiddle
    // table's padded width are zero-filled (their addresses are not read)
    auto issue = [&](int s) {
        const int slot = s % SB_STAGES, k0 = s * SB_K;
        for (int c = tid; c < A_CHUNKS; c += NT) {
            const int kk = c / (SB_M / 2), ch = c % (SB_M / 2);
            const bool ok = k0 + kk < a.n_frames;
            const float2 *src = ok ? a.A32 + (size_t)(k0 + kk) * M_pad + m0 + 2 * ch : a.A32;
            cp_async16_zfill((uint32_t)__cvta_generic_to_shared(&As[slot][kk][2 * ch]), src, ok);
        }
        for (int c = tid; c < B_CHUNKS; c += NT) {
            const int kk = c / (SN / 2), ch = c % (SN / 2), col = j0 + 2 * ch;
            const bool ok = k0 + kk < a.n_frames && col < a.Nw_pad;
            const float2 *src = ok ? a.B32 + (size_t)(a.t0 + k0 + kk) * a.Nw_pad + col : a.B32;
            cp_async16_zfill((uint32_t)__cvta_generic_to_shared(&Bs[slot][kk][2 * ch]), src, ok);
        }
    };

    float ar[8][Q], ai[8][Q];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int q = 0; q < Q; ++q) ar[i][q] = ai[i][q] = 0.f;

#pragma unroll
    for (int s = 0; s < SB_STAGES - 1; ++s) {
        if (s < n_slices) issue(s);
        cp_async_commit();
    }
    for (int s = 0; s < n_slices; ++s) {
        cp_async_wait<SB_STAGES - 2>();     // slice s has landed (for this thread's pieces) ...
        __syncthreads();                    // ... and for every thread's; slot (s-1) is free
        if (s + SB_STAGES - 1 < n_slices) issue(s + SB_STAGES - 1);
        cp_async_commit();
        const int slot = s % SB_STAGES;
#pragma unroll
        for (int kk = 0; kk < SB_K; ++kk) {
            float2 x[8], b[Q];
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = As[slot][kk][tx + 16 * i];
#pragma unroll
            for (int q = 0; q < Q; ++q) b[q] = Bs[slot][kk][ty + TY * q];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    ar[i][q] = fmaf(x[i].x, b[q].x, ar[i][q]);
                    ar[i][q] = fmaf(-x[i].y, b[q].y, ar[i][q]);
                    ai[i][q] = fmaf(x[i].x, b[q].y, ai[i][q]);
                    ai[i][q] = fmaf(x[i].y, b[q].x, ai[i][q]);
                }
        }
    }
    cp_async_wait<0>();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t m = m0 + tx + 16 * i;
        RowCtx row = make_row(a.e, m);
        if (!row.valid) continue;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int j = j0 + ty + TY * q;
            if (j < a.e.Nw) epi_element(a.e, row, j, ar[i][q], ai[i][q]);
        }
    }
}

// energies per block tile: 64 (8 warps), 32 or 40 (4 warps), whichever pads the energy count
// least (ties: 64, then 32).  Blocks of 4 or 8 warps keep the SM's four schedulers evenly
// loaded (a 5-warp 40-wide tile measured slower than either on 200 and 400 energies).
static int simt_tile_cols(int Nw) {
    const int64_t c64 = (int64_t)(Nw + 63) / 64 * 64, c32 = (int64_t)(Nw + 31) / 32 * 32,
                  c40 = (int64_t)(Nw + 39) / 40 * 40;
    if (c64 <= c32 && c64 <= c40) return 64;
    return c32 <= c40 ? 32 : 40;
}

template <int TY, int Q>
cudaError_t launch_simt_shape(const SimtArgs &a, cudaStream_t st) {
    static const cudaError_t attr = cudaFuncSetAttribute(
        flush_simt_kernel<TY, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)simt_smem_bytes<TY, Q>());
    if (attr != cudaSuccess) return attr;
    const int n_jt = (a.e.Nw + Q * TY - 1) / (Q * TY);
    const int64_t n_mt = a.e.M_pad / SB_M;
    const int64_t blocks = n_mt * n_jt;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    flush_simt_kernel<TY, Q><<<(unsigned)blocks, 16 * TY, simt_smem_bytes<TY, Q>(), st>>>(a, n_jt);
    return cudaGetLastError();
}

cudaError_t launch_flush_simt(const SimtArgs &a, cudaStream_t st) {
    if (a.e.M_pad % SB_M != 0 || a.Nw_pad % 2 != 0) return cudaErrorInvalidValue;
    switch (simt_tile_cols(a.e.Nw)) {
        case 64: return launch_simt_shape<16, 4>(a, st);
        case 40: return launch_simt_shape<8, 5>(a, st);
        default: return launch_simt_shape<8, 4>(a, st);
    }
}

}  // namespace tacaw
