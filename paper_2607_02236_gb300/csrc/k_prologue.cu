// Frame ingest (push) kernels: ROI crop, provisional-mean removal, operand conversion.
//
// The elastic (time-mean) part of each pixel is ~100x the inelastic signal, so it is
// removed before the reduced-precision contraction.  The exact mean of the segment is
// not known until its last frame, so pushes subtract a provisional mean mu_hat (the mean
// of the segment's first push) and accumulate sum_t (psi_t - mu_hat) in FP64; finalize
// then applies the exact linear correction -(mu - mu_hat) W(E_j) to Psi.
//
// One thread per (probe, ROI pixel) row; consecutive threads read consecutive pixels of
// a frame row (coalesced 8-byte loads).
#include "tacaw_internal.cuh"

namespace tacaw {

__device__ __forceinline__ const float2 *row_src(const FrameGeom &g, int64_t m) {
    int64_t p = m / g.npix;
    int64_t pix = m - p * g.npix;
    int64_t y = pix / g.kx;
    int64_t x = pix - y * g.kx;
    return g.base + p * g.pitch_probe + (g.roi_y0 + y) * g.pitch_row + (g.roi_x0 + x);
}

// Provisional mean of each row over the first n frames of the first push (launch_mean caps n).  Block = 32 rows x 8
// frame lanes: lane f sums frames f, f + 8, ... of its row (a warp reads 32 consecutive
// pixels of one frame), the eight partial sums are added in a fixed order.  Any rounding of
// mu_hat is harmless: the exact mean correction uses the FP64 residual sums of the pushes.
__global__ void __launch_bounds__(256) mean_kernel(FrameGeom g, int n, float2 *mu_hat) {
    __shared__ float2 part[8][32];
    const int r = threadIdx.x & 31, f = threadIdx.x >> 5;
    const int64_t m = (int64_t)blockIdx.x * 32 + r;
    double sr = 0.0, si = 0.0;
    if (m < g.M) {
        const float2 *src = row_src(g, m);
        for (int t0 = f; t0 < n; t0 += 64) {
            float br = 0.f, bi = 0.f;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int t = t0 + 8 * i;
                if (t < n) {
                    const float2 v = __ldcs(src + (int64_t)t * g.pitch_frame);
                    br += v.x;
                    bi += v.y;
                }
            }
            sr += br;
            si += bi;
        }
    }
    part[f][r] = make_float2((float)sr, (float)si);
    __syncthreads();
    if (f == 0 && m < g.M) {
        float ar = 0.f, ai = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            ar += part[k][r].x;
            ai += part[k][r].y;
        }
        mu_hat[m] = make_float2(ar / n, ai / n);
    }
}

__device__ __forceinline__ uint32_t pack_bf16x2(__nv_bfloat16 a, __nv_bfloat16 b) {
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

__device__ __forceinline__ uint32_t pack_f16x2(__half a, __half b) {
    return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
}

// (re, im) -> hi = RN(re, im), lo = RN(residuals), packed pairs with re in the low half:
// bf16 pieces, or on the split-FP16 path fp16 pieces of the scaled value sc * r (sc = 2^e;
// amax tracks the largest scaled component for the range check).
template <bool F16>
__device__ __forceinline__ void split2(float2 r, float sc, float &amax, uint32_t &hi, uint32_t &lo) {
    if (F16) {
        const float qr = r.x * sc, qi = r.y * sc;
        amax = fmaxf(amax, fmaxf(fabsf(qr), fabsf(qi)));
        __half hr = __float2half_rn(qr), hi_ = __float2half_rn(qi);
        __half lr = __float2half_rn(qr - __half2float(hr));
        __half li = __float2half_rn(qi - __half2float(hi_));
        hi = pack_f16x2(hr, hi_);
        lo = pack_f16x2(lr, li);
    } else {
        __nv_bfloat16 hr = __float2bfloat16_rn(r.x), hi_ = __float2bfloat16_rn(r.y);
        __nv_bfloat16 lr = __float2bfloat16_rn(r.x - __bfloat162float(hr));
        __nv_bfloat16 li = __float2bfloat16_rn(r.y - __bfloat162float(hi_));
        hi = pack_bf16x2(hr, hi_);
        lo = pack_bf16x2(lr, li);
    }
}

// largest finite fp16 value: a scaled component above it does not survive the split
constexpr float kF16Max = 65504.f;

// Pre-swizzled staging (swz != 0): the 16-byte chunks of row m are stored in the order the
// tensor core's shared-memory swizzle of the row width expects (chunk c at c ^ sw(m), sw(m) =
// (m * chunks_per_row / 8) mod chunks_per_row: 128-, 64- and 32-byte swizzle), so that a plain
// contiguous copy of a block of rows into 1024-byte-aligned shared memory gives the swizzled
// operand layout.  Word w (bf16 pair) of the row -> its stored position:
__host__ __device__ __forceinline__ int swz_word(int w, int64_t m, int bf, int swz) {
    if (!swz) return w;
    const int cpr = bf >> 2;
    const int sw = (int)(((m * cpr) >> 3) & (cpr - 1));
    return ((((w >> 2) ^ sw)) << 2) | (w & 3);
}

// Staged frame slot s (s0 + t) goes to block s/bf, elements 2(s%bf), 2(s%bf)+1 of row m
// (rows of 2*bf bf16 = 4*bf bytes; bf is 8, 16 or 32).
template <bool F16>
__global__ void convert_split_kernel(FrameGeom g, int n, int s0, int bf, int64_t M_pad, const float2 *mu_hat,
                                     double2 *sum_res, __nv_bfloat16 *A_hi, __nv_bfloat16 *A_lo, int swz,
                                     float sc, uint32_t *err) {
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= g.M) return;
    const float2 *src = row_src(g, m);
    const float2 mu = mu_hat[m];
    uint32_t *Hi = reinterpret_cast<uint32_t *>(A_hi);
    uint32_t *Lo = reinterpret_cast<uint32_t *>(A_lo);
    double sr = 0.0, si = 0.0;
    float amax = 0.f;
    int t = 0;
    // leading frames up to the next block boundary
    while (t < n && ((s0 + t) & 7)) {
        const int s = s0 + t;
        float2 v = __ldcs(src + (int64_t)t * g.pitch_frame);
        float2 r = make_float2(v.x - mu.x, v.y - mu.y);
        sr += r.x;
        si += r.y;
        uint32_t h, l;
        split2<F16>(r, sc, amax, h, l);
        size_t o = ((size_t)(s / bf) * M_pad + m) * bf + swz_word(s % bf, m, bf, swz);   // in bf16x2 units
        Hi[o] = h;
        Lo[o] = l;
        ++t;
    }
    // groups of 8 frames -> 32 bytes of the row of hi and of lo
    for (; t + 8 <= n; t += 8) {
        float2 v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = __ldcs(src + (int64_t)(t + i) * g.pitch_frame);
        uint32_t h[8], l[8];
        float br = 0.f, bi = 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float2 r = make_float2(v[i].x - mu.x, v[i].y - mu.y);
            br += r.x;
            bi += r.y;
            split2<F16>(r, sc, amax, h[i], l[i]);
        }
        sr += br;
        si += bi;
        const int s = s0 + t;
        const size_t row = ((size_t)(s / bf) * M_pad + m) * bf;
        const size_t o0 = row + swz_word(s % bf, m, bf, swz), o1 = row + swz_word(s % bf + 4, m, bf, swz);
        *reinterpret_cast<uint4 *>(Hi + o0) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4 *>(Hi + o1) = make_uint4(h[4], h[5], h[6], h[7]);
        *reinterpret_cast<uint4 *>(Lo + o0) = make_uint4(l[0], l[1], l[2], l[3]);
        *reinterpret_cast<uint4 *>(Lo + o1) = make_uint4(l[4], l[5], l[6], l[7]);
    }
    // trailing frames
    for (; t < n; ++t) {
        const int s = s0 + t;
        float2 v = __ldcs(src + (int64_t)t * g.pitch_frame);
        float2 r = make_float2(v.x - mu.x, v.y - mu.y);
        sr += r.x;
        si += r.y;
        uint32_t h, l;
        split2<F16>(r, sc, amax, h, l);
        size_t o = ((size_t)(s / bf) * M_pad + m) * bf + swz_word(s % bf, m, bf, swz);
        Hi[o] = h;
        Lo[o] = l;
    }
    double2 a = sum_res[m];
    a.x += sr;
    a.y += si;
    sum_res[m] = a;
    if (F16 && amax > kF16Max) atomicOr(err, DEVERR_FP16_RANGE);
}

// Staging blocks of BF frames, 128 rows per CTA, for pushes whose start s0 and length n are
// multiples of 4 frames (one 16-byte chunk of a row): the push is walked in pieces that each
// lie inside one block (a whole block, or part of one when a push is shorter than a block or
// starts inside one).  Each thread converts its row's frames of the piece into a shared tile
// (16-byte chunks XOR-swizzled by row to spread the banks); the CTA then writes the piece's
// chunks of the 128 rows with consecutive threads on consecutive chunks.  The stored swizzle
// only exchanges chunks inside 32-byte sectors, so a piece always writes whole sectors.
// The rows of block `blk` (rows 128 blk ..) of one push; run by 128 threads.  PF: the longest
// piece the caller passes (BF, or 16 for pushes of at most 16 frames: half the registers and
// shared memory, twice the CTAs an SM holds; the pieces, and so the sums, are the same).
template <int BF, int PF, bool F16>
__device__ __forceinline__ void convert_tiled_rows(const FrameGeom &g, int n, int s0, int64_t M_pad,
                                                   const float2 *mu_hat, double2 *sum_res, __nv_bfloat16 *A_hi,
                                                   __nv_bfloat16 *A_lo, int swz, float sc, uint32_t *err, int64_t blk) {
    constexpr int bf = BF;
    constexpr int cpr = BF / 4;             // 16-byte chunks per staged row
    constexpr int lcpr = PF / 4;            // 16-byte chunks of a piece
    __shared__ uint4 tile_h[128 * lcpr], tile_l[128 * lcpr];
    const int r = threadIdx.x;
    const int64_t m0 = blk * 128;
    const int64_t m = m0 + r;
    const bool valid = m < g.M;
    const float2 *src = valid ? row_src(g, m) : nullptr;
    const float2 mu = valid ? mu_hat[m] : make_float2(0.f, 0.f);
    uint4 *Hi = reinterpret_cast<uint4 *>(A_hi);
    uint4 *Lo = reinterpret_cast<uint4 *>(A_lo);
    double sr = 0.0, si = 0.0;
    float amax = 0.f;
    for (int t0 = 0; t0 < n;) {
        const int f0 = (s0 + t0) % bf;                 // first frame of the piece inside its block
        const int len = min(bf - f0, n - t0);          // a multiple of 4
        const int c0 = f0 / 4, nc = len / 4;
        float2 v[PF];
#pragma unroll
        for (int i = 0; i < PF; ++i)
            v[i] = (valid && i < len) ? __ldcs(src + (int64_t)(t0 + i) * g.pitch_frame) : make_float2(0.f, 0.f);
        float br = 0.f, bi = 0.f;
#pragma unroll
        for (int k = 0; k < lcpr; ++k) {
            if (k >= nc) break;
            uint32_t h[4], l[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float2 q = valid ? make_float2(v[4 * k + i].x - mu.x, v[4 * k + i].y - mu.y) : make_float2(0.f, 0.f);
                br += q.x;
                bi += q.y;
                split2<F16>(q, sc, amax, h[i], l[i]);
            }
            const int slot = r * lcpr + (k ^ (r & (lcpr - 1)));
            tile_h[slot] = make_uint4(h[0], h[1], h[2], h[3]);
            tile_l[slot] = make_uint4(l[0], l[1], l[2], l[3]);
        }
        sr += br;
        si += bi;
        __syncthreads();
        const size_t base = ((size_t)((s0 + t0) / bf) * M_pad + m0) * cpr;   // in 16-byte units
        for (int q = r; q < 128 * nc; q += 128) {
            const int rr = q / nc, k = q - (q / nc) * nc, c = c0 + k;
            const int slot = rr * lcpr + (k ^ (rr & (lcpr - 1)));
            // stored chunk position of chunk c (m0 is a multiple of 128: row rr's pattern)
            const int cs = swz ? (c ^ (((rr * cpr) >> 3) & (cpr - 1))) : c;
            Hi[base + rr * cpr + cs] = tile_h[slot];
            Lo[base + rr * cpr + cs] = tile_l[slot];
        }
        __syncthreads();
        t0 += len;
    }
    if (valid) {
        double2 a = sum_res[m];
        a.x += sr;
        a.y += si;
        sum_res[m] = a;
    }
    if (F16 && amax > kF16Max) atomicOr(err, DEVERR_FP16_RANGE);
}

template <int BF, int PF, bool F16>
__global__ void __launch_bounds__(128) convert_split_tiled_kernel(FrameGeom g, int n, int s0, int64_t M_pad,
                                                                  const float2 *mu_hat, double2 *sum_res,
                                                                  __nv_bfloat16 *A_hi, __nv_bfloat16 *A_lo, int swz,
                                                                  float sc, uint32_t *err) {
    convert_tiled_rows<BF, PF, F16>(g, n, s0, M_pad, mu_hat, sum_res, A_hi, A_lo, swz, sc, err, blockIdx.x);
}

// One push of each of several streams in one launch: CTA b converts block b - e.cta_begin of
// the entry whose range holds b (entries in order of cta_begin).
template <int BF, int PF, bool F16>
__global__ void __launch_bounds__(128) convert_split_group_kernel(const __grid_constant__ ConvGroup cg, int swz,
                                                                  float sc, uint32_t *err) {
    int k = 0;
    while (k + 1 < cg.n && (int64_t)blockIdx.x >= cg.e[k + 1].cta_begin) ++k;
    const ConvEntry &e = cg.e[k];
    convert_tiled_rows<BF, PF, F16>(e.g, e.n, e.s0, e.M_pad, e.mu_hat, e.sum_res, e.A_hi, e.A_lo, swz, sc, err,
                                    (int64_t)blockIdx.x - e.cta_begin);
}

__global__ void convert_fp32_kernel(FrameGeom g, int n, int s0, int64_t M_pad, const float2 *mu_hat,
                                    double2 *sum_res, float2 *A32) {
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= g.M) return;
    const float2 *src = row_src(g, m);
    const float2 mu = mu_hat[m];
    double sr = 0.0, si = 0.0;
    int t = 0;
    for (; t + 8 <= n; t += 8) {
        float2 v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = __ldcs(src + (int64_t)(t + i) * g.pitch_frame);
        float br = 0.f, bi = 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float2 r = make_float2(v[i].x - mu.x, v[i].y - mu.y);
            br += r.x;
            bi += r.y;
            A32[(size_t)(s0 + t + i) * M_pad + m] = r;
        }
        sr += br;
        si += bi;
    }
    for (; t < n; ++t) {
        float2 v = __ldcs(src + (int64_t)t * g.pitch_frame);
        float2 r = make_float2(v.x - mu.x, v.y - mu.y);
        sr += r.x;
        si += r.y;
        A32[(size_t)(s0 + t) * M_pad + m] = r;
    }
    double2 a = sum_res[m];
    a.x += sr;
    a.y += si;
    sum_res[m] = a;
}

// Zeroes staged slots [staged, next multiple of bf) of the last block, all M_pad rows.
__global__ void zero_tail_split_kernel(int64_t M_pad, int staged, int bf, uint32_t *Hi, uint32_t *Lo, int swz) {
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M_pad) return;
    const int blk = staged / bf;
    for (int tt = staged % bf; tt < bf; ++tt) {
        size_t o = ((size_t)blk * M_pad + m) * bf + swz_word(tt, m, bf, swz);
        Hi[o] = 0u;
        Lo[o] = 0u;
    }
}

__global__ void mean_residual_kernel(int64_t M, int T, int sub, const double2 *sum_res, float2 *dmu, double sc) {
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double2 s = sum_res[m];
    dmu[m] = sub ? make_float2((float)(sc * s.x / T), (float)(sc * s.y / T)) : make_float2(0.f, 0.f);
}

static inline unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// In-place frames: slot t of the table <- base + t * pitch_frame (t < n)
__global__ void frame_table_kernel(const float2 **table, const float2 *base, int64_t pitch_frame, int n) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) table[t] = base + (int64_t)t * pitch_frame;
}

cudaError_t launch_frame_table(const float2 **table, const float2 *base, int64_t pitch_frame, int n, cudaStream_t st) {
    frame_table_kernel<<<blocks_for(n, 128), 128, 0, st>>>(table, base, pitch_frame, n);
    return cudaGetLastError();
}

// The provisional mean of a segment is taken over the first (at most kMeanFrames) frames of its
// first push: any value is exact after the finalize correction Psi -= (mu - mu_hat) W(E), and a
// few frames already put mu_hat on the elastic part, which is what keeps the residuals small.
constexpr int kMeanFrames = 32;
cudaError_t launch_mean(const FrameGeom &g, int n, float2 *mu_hat, cudaStream_t st) {
    mean_kernel<<<blocks_for(g.M, 32), 256, 0, st>>>(g, n < kMeanFrames ? n : kMeanFrames, mu_hat);
    return cudaGetLastError();
}

template <bool F16>
static cudaError_t convert_split(const FrameGeom &g, int n, int s0, int bf, int64_t M_pad, const float2 *mu_hat,
                                 double2 *sum_res, __nv_bfloat16 *A_hi, __nv_bfloat16 *A_lo, int swz, float sc,
                                 uint32_t *err, cudaStream_t st) {
    if (convert_split_groupable(bf, s0, n)) {
        const unsigned grid = (unsigned)(M_pad / 128);
        if (bf == 32 && n > 16)
            convert_split_tiled_kernel<32, 32, F16><<<grid, 128, 0, st>>>(g, n, s0, M_pad, mu_hat, sum_res, A_hi,
                                                                          A_lo, swz, sc, err);
        else if (bf == 32)
            convert_split_tiled_kernel<32, 16, F16><<<grid, 128, 0, st>>>(g, n, s0, M_pad, mu_hat, sum_res, A_hi,
                                                                          A_lo, swz, sc, err);
        else
            convert_split_tiled_kernel<16, 16, F16><<<grid, 128, 0, st>>>(g, n, s0, M_pad, mu_hat, sum_res, A_hi,
                                                                          A_lo, swz, sc, err);
        return cudaGetLastError();
    }
    convert_split_kernel<F16><<<blocks_for(g.M, 256), 256, 0, st>>>(g, n, s0, bf, M_pad, mu_hat, sum_res, A_hi,
                                                                    A_lo, swz, sc, err);
    return cudaGetLastError();
}

cudaError_t launch_convert_split(const FrameGeom &g, int n, int s0, int bf, int64_t M_pad, const float2 *mu_hat,
                                 double2 *sum_res, __nv_bfloat16 *A_hi, __nv_bfloat16 *A_lo, int swz, int f16,
                                 float f16_scale, uint32_t *err, cudaStream_t st) {
    if (f16) return convert_split<true>(g, n, s0, bf, M_pad, mu_hat, sum_res, A_hi, A_lo, swz, f16_scale, err, st);
    return convert_split<false>(g, n, s0, bf, M_pad, mu_hat, sum_res, A_hi, A_lo, swz, 1.f, err, st);
}

bool convert_split_groupable(int bf, int s0, int n) { return bf >= 16 && s0 % 4 == 0 && n % 4 == 0; }

cudaError_t launch_convert_split_group(ConvGroup &cg, int bf, int swz, int f16, float f16_scale, uint32_t *err,
                                       cudaStream_t st) {
    if (cg.n < 1 || cg.n > kConvGroupMax || (bf != 16 && bf != 32)) return cudaErrorInvalidValue;
    int64_t ctas = 0;
    for (int i = 0; i < cg.n; ++i) {
        if (!convert_split_groupable(bf, cg.e[i].s0, cg.e[i].n) || cg.e[i].M_pad % 128) return cudaErrorInvalidValue;
        cg.e[i].cta_begin = ctas;
        ctas += cg.e[i].M_pad / 128;
    }
    if (ctas == 0) return cudaSuccess;
    if (ctas > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const unsigned grid = (unsigned)ctas;
    const float sc = f16 ? f16_scale : 1.f;
    // pushes of at most 16 frames everywhere: the half-size variant (more CTAs an SM)
    bool short_pushes = true;
    for (int i = 0; i < cg.n; ++i) short_pushes = short_pushes && cg.e[i].n <= 16;
    if (bf == 32 && !short_pushes) {
        if (f16) convert_split_group_kernel<32, 32, true><<<grid, 128, 0, st>>>(cg, swz, sc, err);
        else convert_split_group_kernel<32, 32, false><<<grid, 128, 0, st>>>(cg, swz, sc, err);
    } else if (bf == 32) {
        if (f16) convert_split_group_kernel<32, 16, true><<<grid, 128, 0, st>>>(cg, swz, sc, err);
        else convert_split_group_kernel<32, 16, false><<<grid, 128, 0, st>>>(cg, swz, sc, err);
    } else {
        if (f16) convert_split_group_kernel<16, 16, true><<<grid, 128, 0, st>>>(cg, swz, sc, err);
        else convert_split_group_kernel<16, 16, false><<<grid, 128, 0, st>>>(cg, swz, sc, err);
    }
    return cudaGetLastError();
}

cudaError_t launch_convert_fp32(const FrameGeom &g, int n, int s0, int64_t M_pad, const float2 *mu_hat,
                                double2 *sum_res, float2 *A32, cudaStream_t st) {
    convert_fp32_kernel<<<blocks_for(g.M, 256), 256, 0, st>>>(g, n, s0, M_pad, mu_hat, sum_res, A32);
    return cudaGetLastError();
}

cudaError_t launch_zero_tail_split(int64_t M_pad, int staged, int bf, __nv_bfloat16 *A_hi, __nv_bfloat16 *A_lo,
                                   int swz, cudaStream_t st) {
    zero_tail_split_kernel<<<blocks_for(M_pad, 256), 256, 0, st>>>(
        M_pad, staged, bf, reinterpret_cast<uint32_t *>(A_hi), reinterpret_cast<uint32_t *>(A_lo), swz);
    return cudaGetLastError();
}

cudaError_t launch_mean_residual(int64_t M, int T, int subtract_mean, const double2 *sum_res, float2 *dmu,
                                 float scale, cudaStream_t st) {
    mean_residual_kernel<<<blocks_for(M, 256), 256, 0, st>>>(M, T, subtract_mean, sum_res, dmu, (double)scale);
    return cudaGetLastError();
}

}  // namespace tacaw
