// Tensor-core (tcgen05) contraction of the frames of one flush with the twiddle table, split
// BF16 (or split FP16):
//
//   Psi[m, j] (+)= sum_f y[m, f] B[t0 + f, j]        y = psi - mu_hat, B = w_t exp(-i theta_jt)
//
// the windowed time->energy transform of Eq. 1 over the frames of one flush, as a real
// GEMM on the embedding  [Re y, Im y] x [[Re B, Im B], [-Im B, Re B]].  Every operand is
// split x = hi + lo (16-bit pieces each); the product is accumulated as hi*hi + hi*lo + lo*hi
// in FP32 in tensor memory (the dropped lo*lo term is ~2^-16 relative).  A tile is 128 rows
// (one TMEM lane each) x N = 2*wt real columns (wt complex energies).
//
// Kernels of this file (both persistent: one CTA per SM walks the tiles; every mbarrier wait is
// bounded by the globaltimer, and on a timeout the kernel records an error bit, lets its
// in-flight copies land, frees its TMEM and returns):
//   flush_tc_drain2_kernel   staged operands (converted at push time into pre-swizzled bf16 or
//                            fp16 rows): the path every staged split plan takes; one launch may
//                            cover the tiles of several streams (supercell partitions)
//   flush_tc_inplace_kernel  the pushed complex64 frames read in place, operand A converted into
//                            tensor memory inside the kernel (no staging pass)
#include <cuda.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>

#include "tacaw_internal.cuh"

namespace tacaw {

// One launch over the tiles of several streams (supercell partitions): entry i owns tiles
// [cta_begin, cta_begin + ctas) of the concatenated tile list.
struct TcGroupEntry {
    TcPlanArgs args;
    int cta_begin;
    int ctas;
};
struct TcGroup {
    TcGroupEntry e[kMaxGroupStreams];
    int n;
    int stages, n_max;         // ring stages and ring/TMEM width (widest tile of the group)
    int64_t tiles;             // tiles of all entries
    int *counter;              // tile queue: the next tile index to hand out (zero at launch)
    int conv_on;               // warps 10 and 11 convert the next segment's pushes (conv)
    TcConvJob conv;
};

constexpr uint64_t kWaitLimitNs = 4000000000ull;  // 4 s per wait
constexpr int kMaxStages = 12;
constexpr int kSmemLimit = 232448;                 // 227 KB opt-in per block
constexpr int kTileQueue = 4;                      // tiles handed out ahead (staged kernel)

struct TcShared {
    uint64_t full[kMaxStages];
    uint64_t empty[kMaxStages];
    uint64_t tmem_full;
    uint32_t tmem_addr;
    int abort_flag;
    uint64_t chunk_full[2];   // [0] a chunk of H is complete, [1] the tile's last H and S are
    uint64_t chunk_free[2];   // the epilogue warps have drained them
    uint64_t tq_full[kTileQueue];    // tile queue: the producer wrote tile_q[i]
    uint64_t tq_empty[kTileQueue];   //   the MMA thread and the eight epilogue warps read it
    int tile_q[kTileQueue];          //   tile index, or -1 when the launch's tiles are all handed out
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t smid() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait.  Gives up after limit_ns, or early when *abort_flag is set (if given).  Waits
// for work that always completes (copies in flight, issued MMAs) keep the default limit.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag, uint64_t limit_ns = kWaitLimitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (abort_flag && *abort_flag) return false;
        if (globaltimer() - t0 > limit_ns) return false;
    }
}
// Warp-uniform bounded wait: lane 0 waits, every lane gets its verdict (so no lane of the warp
// can leave a loop that the others stay in), and the warp synchronises for memory ordering.
__device__ __forceinline__ bool mbar_wait_warp(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                               uint64_t limit_ns = kWaitLimitNs) {
    int ok = 1;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, abort_flag, limit_ns) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    return ok != 0;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}
// 16-byte asynchronous copy global -> shared through L2 (LSU path), and the arrive on an
// mbarrier once all of this thread's earlier such copies have landed (counted as one of the
// barrier's expected arrivals)
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(reinterpret_cast<uint64_t>(src))
                 : "memory");
}
__device__ __forceinline__ void cp_async_arrive(uint32_t bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// Running FP32 sum with a compensation term (Kahan)
__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}
// Contiguous copy global -> shared (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
                 : "memory");
}
// The same with an L2 eviction policy (createpolicy) for the lines it brings in.
__device__ __forceinline__ void bulk_load_hint(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar,
                                               uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar), "l"(policy)
        : "memory");
}
// Policy that keeps lines in L2 ahead of ordinary ones: the twiddle rows, which every pass of a
// persistent grid reads again, against the staged rows, which are streamed once per row tile.
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mma_bf16_ss(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tmem_ld_x16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major operand whose rows are one swizzle atom wide
// (32, 64 or 128 bytes): 8-row core groups 8*row_bytes apart (stride byte offset),
// descriptor version 1 (bit 46), layout type (bits 61-63) 6 = SWIZZLE_32B, 4 = 64B,
// 2 = 128B.  The leading byte offset is unused when the K extent stays inside one atom.
__device__ __forceinline__ uint64_t sdesc_k(uint32_t saddr, uint32_t row_bytes) {
    const uint64_t layout = row_bytes == 128 ? 2 : (row_bytes == 64 ? 4 : 6);
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)((8u * row_bytes) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= layout << 61;
    return d;
}
// Instruction descriptor, kind::f16: D = F32 (bit 4), A = B = BF16 (bits 7, 10), both
// K-major, N>>3 at bit 17, M>>4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// The same with A = B = F16 (format fields 0) when f16 is set: both operands always share
// one type (the split-FP16 path stages fp16 pieces of A and of B alike).
__host__ __device__ constexpr uint32_t idesc_f32acc(int M, int N, int f16) {
    return f16 ? (idesc_bf16_f32(M, N) & ~((1u << 7) | (1u << 10))) : idesc_bf16_f32(M, N);
}

__host__ __device__ inline uint32_t tc_a_bytes(int bf) { return (uint32_t)kMTile * 4u * (uint32_t)bf; }
__host__ __device__ inline uint32_t tc_b_bytes_padded(int N, int bf) {
    return ((uint32_t)N * 4u * (uint32_t)bf + 1023u) & ~1023u;
}
__host__ __device__ inline uint32_t tc_stage_bytes(int N, int bf) {
    return 2u * tc_a_bytes(bf) + 2u * tc_b_bytes_padded(N, bf);
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// (re, im) -> packed bf16x2 hi = RN(re, im) and lo = RN(residuals), re in the low half: one
// paired conversion each (the unpacking of hi back to FP32 is two bit operations).
__device__ __forceinline__ void split2_bf16(float2 r, uint32_t &hi, uint32_t &lo) {
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(r.x, r.y);
    uint32_t hb;
    memcpy(&hb, &h2, sizeof(hb));
    const float hr = __uint_as_float(hb << 16), him = __uint_as_float(hb & 0xffff0000u);
    const __nv_bfloat162 l2 = __floats2bfloat162_rn(r.x - hr, r.y - him);
    hi = hb;
    memcpy(&lo, &l2, sizeof(lo));
}

// Drained form: per-thread FP32 running sums of up to kDrainCols accumulator columns (one TMEM
// lane, a contiguous column range: tiles of at most 112 complex energies).  Loads are
// warp-uniform; columns past `cols` (up to 15 of them, inside the allocation) are loaded and
// ignored.
constexpr int kDrainCols = 112;
template <int C>
__device__ __forceinline__ void drain_add(float (&sum)[C], uint32_t taddr, int cols) {
#pragma unroll
    for (int r = 0; r < (C + 15) / 16; ++r) {
        if (r * 16 < cols) {
            uint32_t x[16];
            tmem_ld_x16(taddr + (uint32_t)(r * 16), x);
            tmem_ld_wait();
#pragma unroll
            for (int i = 0; i < 16; ++i)
                if (r * 16 + i < C && r * 16 + i < cols) sum[r * 16 + i] += __uint_as_float(x[i]);
        }
        __syncwarp();
    }
}

__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// L2 prefetch of what this thread's flush epilogue will read for row m (earlier flushes'
// accumulators, I when Welch segments add into it).  Each of the epilogue's reads feeds a store
// that the next read may not pass (the compiler cannot tell the addresses apart), and the 112
// running sums leave no registers to batch them under the 168-register cap of a 10-warp CTA;
// so the reads are issued as prefetches while the tile's last chunk of products runs, and the
// epilogue's chain of reads then waits on L2 rather than DRAM.
__device__ __forceinline__ void tc_epilogue_prefetch(const TcPlanArgs &a, int64_t m, int col0, int cols, int jbase) {
    const EpiArgs &e = a.e;
    if (m >= e.M) return;
    const int kind = epi_kind(e);
    const bool acc32 = kind == EPI_ADD_KAHAN || kind == EPI_FINAL_KAHAN;
    const bool acc64 = kind == EPI_ADD_FP64 || kind == EPI_FINAL_FP64;
    const bool iadd = (kind == EPI_FINAL || kind == EPI_FINAL_KAHAN || kind == EPI_FINAL_FP64) && e.I_out && e.out_add;
    if (!acc32 && !acc64 && !iadd) return;
    const int64_t p = m / e.npix;
    const int64_t o0 = p * (int64_t)e.Nw * e.npix + (m - p * e.npix);
    for (int c = 0; c < cols; c += 2) {
        const int j = jbase + ((col0 + c) >> 1);
        if (j >= e.Nw) break;
        const size_t ai = (size_t)j * (size_t)e.M_pad + (size_t)m;
        if (acc32) {
            prefetch_l2(e.acc_s + ai);
            if (e.acc_c) prefetch_l2(e.acc_c + ai);
        }
        if (acc64) prefetch_l2(e.acc_d + ai);
        if (iadd) prefetch_l2(e.I_out + o0 + (int64_t)j * e.npix);
    }
}

// Flush epilogue of the split drained form: the tile's result is all in the running sums.
template <int KIND, int C>
__device__ __forceinline__ void tc_epilogue_regs(const TcPlanArgs &a, const RowCtx &row, int col0, int cols,
                                                 int jbase, const float (&sum)[C]) {
    if (!row.valid) return;
#pragma unroll
    for (int i = 0; i < C / 2; ++i) {
        const int c = 2 * i;
        const int j = jbase + ((col0 + c) >> 1);
        if (c < cols && j < a.e.Nw)
            epi_apply<KIND>(a.e, row, j, sum[c], sum[c + 1], __ldg(a.e.Wc + j), __ldg(a.e.bose + j));
    }
}

// Conversion job of a staged contraction launch (pipelined segments), run by its two extra
// warps beside the tensor-core pipeline: each warp takes row tiles of 128 rows from a counter;
// lane l converts rows 4l .. 4l + 3 of the tile over every frame of the segment: psi - mu_hat
// split into bf16 hi/lo, 16-byte chunks of 4 frames stored at their pre-swizzled place (chunk c
// of row m at c ^ (m mod 8)); per 32-frame block an FP32 sum of the residuals in frame order,
// added to an FP64 row sum (the roundings of the tiled push conversion of block-aligned pushes).
__device__ void tc_convert_job(const TcConvJob &j, int lane) {
    uint4 *Hi = reinterpret_cast<uint4 *>(j.A_hi);
    uint4 *Lo = reinterpret_cast<uint4 *>(j.A_lo);
    const int n_kb = j.T / 32;
    const int64_t n_tiles = j.M_pad / kMTile;
    for (;;) {
        int tile = 0;
        if (lane == 0) tile = atomicAdd(j.counter, 1);
        tile = __shfl_sync(0xffffffffu, tile, 0);
        if ((int64_t)tile >= n_tiles) break;
        int64_t m[4], off[4];
        float2 mu[4];
        double sr[4], si[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            m[r] = (int64_t)tile * kMTile + 4 * lane + r;
            const bool ok = m[r] < j.M;
            const int64_t p = ok ? m[r] / j.npix : 0;
            const int64_t pix = ok ? m[r] - p * j.npix : 0;
            const int64_t y = pix / j.kx, x = pix - y * j.kx;
            off[r] = ok ? p * j.pitch_probe + (j.roi_y0 + y) * j.pitch_row + (j.roi_x0 + x) : -1;
            mu[r] = ok ? j.mu_hat[m[r]] : make_float2(0.f, 0.f);
            sr[r] = si[r] = 0.0;
        }
        // rows past M read row 0's place (a valid address) and are zeroed below, so that every
        // load issues without a branch
        int64_t roff[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) roff[r] = off[r] >= 0 ? off[r] : (off[0] >= 0 ? off[0] : 0);
        const bool any = off[0] >= 0;
        for (int kb = 0; kb < n_kb; ++kb) {
            float br[4] = {0.f, 0.f, 0.f, 0.f}, bi[4] = {0.f, 0.f, 0.f, 0.f};
            // the block's 32 frame addresses, one a lane, handed to the others by shuffles
            const float2 *my_fp = j.frame_ptr[kb * 32 + lane];
#pragma unroll 2
            for (int c = 0; c < 8; ++c) {
                float2 v[4][4];
#pragma unroll
                for (int f = 0; f < 4; ++f) {
                    const float2 *fp = reinterpret_cast<const float2 *>(
                        __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(my_fp), 4 * c + f));
#pragma unroll
                    for (int r = 0; r < 4; ++r) v[r][f] = any ? __ldcs(fp + roff[r]) : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    uint32_t h[4], l[4];
#pragma unroll
                    for (int f = 0; f < 4; ++f) {
                        const float2 q = off[r] >= 0 ? make_float2(v[r][f].x - mu[r].x, v[r][f].y - mu[r].y)
                                                     : make_float2(0.f, 0.f);
                        br[r] += q.x;
                        bi[r] += q.y;
                        split2_bf16(q, h[f], l[f]);
                    }
                    const size_t o = ((size_t)kb * (size_t)j.M_pad + (size_t)m[r]) * 8 + (size_t)(c ^ (int)(m[r] & 7));
                    Hi[o] = make_uint4(h[0], h[1], h[2], h[3]);
                    Lo[o] = make_uint4(l[0], l[1], l[2], l[3]);
                }
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                sr[r] += br[r];
                si[r] += bi[r];
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (off[r] >= 0) j.sum_res[m[r]] = make_double2(sr[r], si[r]);
    }
}

// --------------------------------------------------------------------------------------
// Staged contraction (split drained form), persistent: one CTA per SM walks the tiles of all
// streams of the group (tile t of the concatenated tile lists, t = blockIdx.x, blockIdx.x +
// gridDim.x, ...); a tile is 128 rows x one energy tile over every staged frame.
//
// hi*hi goes to TMEM accumulator H (columns 0..), the small products hi*lo + lo*hi to S
// (columns 256..).  The tensor core's FP32 accumulation truncates each step against the
// running sum, so H is drained every drain_kb staging blocks into FP32 registers (round to
// nearest) by eight epilogue warps (two per TMEM lane quarter, each half of the columns)
// while the MMA thread goes on with the next stage's small products; the small terms carry
// ~2^-8 of the magnitude, so S keeps the whole tile.  At the end of a tile the last chunk of
// H and all of S are added to the registers, both accumulators are released at once, and the
// flush epilogue runs from registers while the next tile accumulates.
//
//   warp 0     bulk-copy producer over the ring (a stage counter running across tiles): the
//              staging rows and twiddle rows are stored pre-swizzled, so each operand block
//              of a stage is one contiguous cp.async.bulk copy
//   warp 1     TMEM allocation and MMA issue (one thread); commits release stages and mark
//              finished chunks
//   warps 2-9  drains and epilogues
// The shared-memory ring and TMEM are laid out for the widest tile of the group.
// 320 threads: warps are spread over the SM's four register files, three on two of them, so a
// thread may hold at most 16384 / (3 * 32) = 170 registers (168 allocatable).
__device__ __forceinline__ int group_entry(const TcGroup &g, int64_t tile) {
    int gi = 0;
    while (gi + 1 < g.n && tile >= (int64_t)g.e[gi + 1].cta_begin) ++gi;
    return gi;
}

__global__ void __maxnreg__(168) flush_tc_drain2_kernel(const __grid_constant__ TcGroup g) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int bf = g.e[0].args.bf, stages = g.stages, n_max = g.n_max;
    const uint32_t RB = 4u * (uint32_t)bf;
    const uint32_t kABytes = tc_a_bytes(bf);
    const uint32_t b_pad = tc_b_bytes_padded(n_max, bf);
    const uint32_t stage_bytes = tc_stage_bytes(n_max, bf);
    TcShared *sh = reinterpret_cast<TcShared *>(base + (size_t)stages * stage_bytes);
    const uint32_t base_s = smem_u32(base);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t ncols = 512u;
    const int64_t n_tiles = g.tiles;
    uint32_t *err = g.e[0].args.err;
    unsigned long long *trace = g.e[0].args.trace ? g.e[0].args.trace + (size_t)blockIdx.x * kTraceWords : nullptr;
    if (trace && threadIdx.x == 0) {
        trace[0] = globaltimer();
        trace[7] = smid();
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(smem_u32(&sh->full[s]), 1);
            mbar_init(smem_u32(&sh->empty[s]), 1);
        }
        mbar_init(smem_u32(&sh->tmem_full), 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&sh->chunk_full[b]), 1);
            mbar_init(smem_u32(&sh->chunk_free[b]), 8);   // one arrival per epilogue warp
        }
        for (int q = 0; q < kTileQueue; ++q) {
            mbar_init(smem_u32(&sh->tq_full[q]), 1);
            mbar_init(smem_u32(&sh->tq_empty[q]), 9);     // the MMA thread and eight epilogue warps
        }
        sh->abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(&sh->tmem_addr), ncols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tmem_addr;
    volatile int *abort_flag = &sh->abort_flag;
    // pipeline waits give up after the plan's limit (default 4 s); see mbar_wait
    const uint64_t wait_ns = g.e[0].args.wait_ns ? g.e[0].args.wait_ns : kWaitLimitNs;
    if (trace && threadIdx.x == 0) trace[1] = globaltimer();

    // Ring position: slot s and its use parity advance by one per staging block, across tiles
    // (no divisions in the issue loops: the single MMA thread's loop sits on the critical path).
    if (warp == 0) {
        if (lane == 0) {
            const uint64_t keep = l2_evict_last_policy();
            int s = 0;
            uint32_t ph = 0;                          // parity of the current use of slot s
            int issued = 0;                           // copies in flight that may still land
            int q = 0;
            uint32_t qph = 0;                         // tile queue slot and its use parity
            while (!*abort_flag) {
                // the next tile of the launch (tiles go out in order: longest streams first, the
                // energy tiles of a row tile side by side, so they share its rows in L2)
                int64_t t = atomicAdd(g.counter, 1);
                if (t >= n_tiles) t = -1;
                if (!mbar_wait(smem_u32(&sh->tq_empty[q]), qph ^ 1u, abort_flag, wait_ns)) {
                    if (!*abort_flag) atomicOr(err, DEVERR_TIMEOUT_EMPTY);
                    *abort_flag = 1;
                    break;
                }
                sh->tile_q[q] = (int)t;
                mbar_arrive(smem_u32(&sh->tq_full[q]));
                if (++q == kTileQueue) {
                    q = 0;
                    qph ^= 1u;
                }
                if (t < 0) break;
                const int gi = group_entry(g, t);
                const TcGroupEntry &en = g.e[gi];
                const int64_t lt = t - en.cta_begin;
                const int wtile = (int)(lt % en.args.n_wt);
                const int m0 = (int)(lt / en.args.n_wt) * kMTile;
                const int N = en.args.N;
                // columns of this tile (N_last: a narrower last energy tile; 0 = full width)
                const int Nt = (wtile == en.args.n_wt - 1 && en.args.N_last > 0) ? en.args.N_last : N;
                const uint32_t tx_bytes = 2u * kABytes + 2u * (uint32_t)Nt * RB;
                const uint8_t *pAhi = static_cast<const uint8_t *>(en.args.A_hi) + (size_t)m0 * RB;
                const uint8_t *pAlo = static_cast<const uint8_t *>(en.args.A_lo) + (size_t)m0 * RB;
                const size_t b0 = ((size_t)en.args.kbB0 * (size_t)en.args.b_rows + (size_t)wtile * N) * RB;
                const uint8_t *pBhi = static_cast<const uint8_t *>(en.args.B_hi) + b0;
                const uint8_t *pBlo = static_cast<const uint8_t *>(en.args.B_lo) + b0;
                const size_t a_step = (size_t)en.args.a_rows * RB, b_step = (size_t)en.args.b_rows * RB;
                for (int kb = 0; kb < en.args.n_kb; ++kb) {
                    if (!mbar_wait(smem_u32(&sh->empty[s]), ph ^ 1u, abort_flag, wait_ns)) {
                        if (!*abort_flag) atomicOr(err, DEVERR_TIMEOUT_EMPTY);
                        *abort_flag = 1;
                        break;
                    }
                    const uint32_t full = smem_u32(&sh->full[s]);
                    const uint32_t st = base_s + (uint32_t)s * stage_bytes;
                    mbar_arrive_expect_tx(full, tx_bytes);
                    // the tables are pre-swizzled: each operand block is one contiguous copy
                    bulk_load(st, pAhi, kABytes, full);
                    bulk_load(st + kABytes, pAlo, kABytes, full);
                    bulk_load_hint(st + 2 * kABytes, pBhi, (uint32_t)Nt * RB, full, keep);
                    bulk_load_hint(st + 2 * kABytes + b_pad, pBlo, (uint32_t)Nt * RB, full, keep);
                    pAhi += a_step;
                    pAlo += a_step;
                    pBhi += b_step;
                    pBlo += b_step;
                    issued = issued < stages ? issued + 1 : stages;
                    if (++s == stages) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
            if (*abort_flag) {
                // let every copy into this CTA's ring land before it can exit: the last `issued`
                // slots before the current position
                int ks = s;
                uint32_t kp = ph;
                for (int i = 0; i < issued; ++i) {
                    if (--ks < 0) {
                        ks = stages - 1;
                        kp ^= 1u;
                    }
                    if (!mbar_wait(smem_u32(&sh->full[ks]), kp, nullptr)) atomicOr(err, DEVERR_TIMEOUT_DRAIN);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const int ksteps = bf / 8;
            int s = 0;
            uint32_t ph = 0;
            uint32_t hph = 0, tph = 0;                // parities of the H drain and tile release
            int64_t tiles = 0, chunks = 0;
            bool stop = false;
            const uint32_t accH = tmem, accS = tmem + 256u;
            int q = 0;
            uint32_t qph = 0;
            for (;; ++tiles) {
                if (!mbar_wait(smem_u32(&sh->tq_full[q]), qph, abort_flag, wait_ns)) {
                    if (!*abort_flag) atomicOr(err, DEVERR_TIMEOUT_FULL);
                    *abort_flag = 1;
                    break;
                }
                const int64_t t = sh->tile_q[q];
                mbar_arrive(smem_u32(&sh->tq_empty[q]));
                if (++q == kTileQueue) {
                    q = 0;
                    qph ^= 1u;
                }
                if (t < 0) break;
                const TcGroupEntry &en = g.e[group_entry(g, t)];
                const bool last_w = en.args.N_last > 0 && (t - en.cta_begin) % en.args.n_wt == en.args.n_wt - 1;
                const int N = last_w ? en.args.N_last : en.args.N, n_kb = en.args.n_kb, cb = en.args.drain_kb;
                const uint32_t id = idesc_f32acc(kMTile, N, en.args.f16);
                if (tiles > 0) {
                    // the previous tile's H and S must be in registers before they are reused
                    if (!mbar_wait(smem_u32(&sh->chunk_free[1]), tph, abort_flag, wait_ns)) {
                        if (!*abort_flag) atomicOr(err, DEVERR_TIMEOUT_TMEM);
                        *abort_flag = 1;
                        break;
                    }
                    tph ^= 1u;
                    tc_fence_after();
                }
                int kc = 0;                           // staging block inside the chunk
                for (int kb = 0; kb < n_kb; ++kb) {
                    if (!mbar_wait(smem_u32(&sh->full[s]), ph, abort_flag, wait_ns)) {
                        if (!*abort_flag) atomicOr(err, DEVERR_TIMEOUT_FULL);
                        *abort_flag = 1;
                        stop = true;
                        break;
                    }
                    tc_fence_after();
                    if (trace && tiles == 0 && kb == 0) trace[2] = globaltimer();
                    const uint32_t st = base_s + (uint32_t)s * stage_bytes;
                    const uint64_t dAhi0 = sdesc_k(st, RB);
                    const uint64_t dAlo0 = sdesc_k(st + kABytes, RB);
                    const uint64_t dBhi0 = sdesc_k(st + 2 * kABytes, RB);
                    const uint64_t dBlo0 = sdesc_k(st + 2 * kABytes + b_pad, RB);
                    // small products of the whole stage first (S never waits inside a tile)
                    for (int ks = 0; ks < ksteps; ++ks) {
                        const uint64_t adv = (uint64_t)(2 * ks);
                        mma_bf16_ss(accS, dAhi0 + adv, dBlo0 + adv, id, (kb == 0 && ks == 0) ? 0u : 1u);
                        mma_bf16_ss(accS, dAlo0 + adv, dBhi0 + adv, id, 1u);
                    }
                    if (kc == 0 && kb > 0) {
                        // the previous chunk of H must be drained before this chunk overwrites it
                        if (!mbar_wait(smem_u32(&sh->chunk_free[0]), hph, abort_flag, wait_ns)) {
                            if (!*abort_flag) atomicOr(err, DEVERR_TIMEOUT_TMEM);
                            *abort_flag = 1;
                            stop = true;
                            break;
                        }
                        hph ^= 1u;
                        tc_fence_after();
                    }
                    for (int ks = 0; ks < ksteps; ++ks) {
                        const uint64_t adv = (uint64_t)(2 * ks);
                        mma_bf16_ss(accH, dAhi0 + adv, dBhi0 + adv, id, (kc == 0 && ks == 0) ? 0u : 1u);
                    }
                    mma_commit(smem_u32(&sh->empty[s]));
                    if (++s == stages) {
                        s = 0;
                        ph ^= 1u;
                    }
                    if (++kc == cb && kb != n_kb - 1) {
                        mma_commit(smem_u32(&sh->chunk_full[0]));   // a finished chunk of H
                        kc = 0;
                        ++chunks;
                    }
                }
                if (stop) break;
                mma_commit(smem_u32(&sh->chunk_full[1]));           // the tile's last H and S
            }
            mma_commit(smem_u32(&sh->tmem_full));   // always: nothing writes TMEM after this
            if (trace) {
                trace[3] = globaltimer();
                trace[4] = (unsigned long long)tiles;
                trace[5] = (unsigned long long)chunks;
            }
        }
    } else if (warp < 10) {
        // epilogue warps 2..9: TMEM lane quarter q4 = warp % 4, column half h
        const int q4 = warp & 3, h = (warp - 2) >> 2;
        float sum[kDrainCols];
        int64_t hc = 0, tiles = 0;                    // H drains done, tiles done
        bool ok = true;
        int q = 0;
        uint32_t qph = 0;
        for (;; ++tiles) {
            if (!mbar_wait_warp(smem_u32(&sh->tq_full[q]), qph, abort_flag, wait_ns)) {
                if (lane == 0 && !*abort_flag) atomicOr(err, DEVERR_TIMEOUT_TMEM);
                *abort_flag = 1;
                break;
            }
            const int64_t t = sh->tile_q[q];
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&sh->tq_empty[q]));
            if (++q == kTileQueue) {
                q = 0;
                qph ^= 1u;
            }
            if (t < 0) break;
            const TcGroupEntry &en = g.e[group_entry(g, t)];
            const TcPlanArgs &a = en.args;
            const int64_t lt = t - en.cta_begin;
            const int wtile = (int)(lt % a.n_wt);
            const int m0 = (int)(lt / a.n_wt) * kMTile;
            // N / 2 columns per thread (the last energy tile may be narrower)
            const int cols = ((wtile == a.n_wt - 1 && a.N_last > 0) ? a.N_last : a.N) / 2;
            const int col0 = h * cols;
            const uint32_t lane_base = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)col0;
            const int n_chunks = (a.n_kb + a.drain_kb - 1) / a.drain_kb;
            // plain FP32 accumulators of earlier flushes start this tile's running sums: read while
            // the tile's first products run, so that the tile's epilogue only stores (the reads
            // then wait on nothing); compensated and FP64 accumulators are added at the end
            const int kind0 = epi_kind(a.e);
            const bool preload = (kind0 == EPI_ADD_KAHAN || kind0 == EPI_FINAL_KAHAN) && a.e.acc_c == nullptr;
            {
                // this thread's energies j0 .. j0 + nv - 1 of row mrow (accumulators [Nw_pad][M_pad])
                const int64_t mrow = (int64_t)m0 + q4 * 32 + lane;
                const int j0 = wtile * a.wt + (col0 >> 1);
                const int nv = (preload && mrow < a.e.M) ? max(0, min(cols >> 1, a.e.Nw - j0)) : 0;
                const float2 *ap = preload ? a.e.acc_s + (size_t)j0 * (size_t)a.e.M_pad + (size_t)mrow : nullptr;
                const size_t stride = (size_t)a.e.M_pad;
#pragma unroll
                for (int i = 0; i < kDrainCols / 2; ++i) {
                    const float2 v = i < nv ? ap[(size_t)i * stride] : make_float2(0.f, 0.f);
                    sum[2 * i] = v.x;
                    sum[2 * i + 1] = v.y;
                }
            }
            for (int lc = 0; lc + 1 < n_chunks; ++lc, ++hc) {
                if (!mbar_wait(smem_u32(&sh->chunk_full[0]), (uint32_t)(hc & 1), abort_flag, wait_ns)) {
                    if (!*abort_flag) atomicOr(err, DEVERR_TIMEOUT_TMEM);
                    *abort_flag = 1;
                    ok = false;
                    break;
                }
                tc_fence_after();
                drain_add(sum, lane_base, cols);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&sh->chunk_free[0]));
            }
            if (!ok) break;
            if (!preload) tc_epilogue_prefetch(a, (int64_t)m0 + q4 * 32 + lane, col0, cols, wtile * a.wt);
            if (!mbar_wait(smem_u32(&sh->chunk_full[1]), (uint32_t)(tiles & 1), abort_flag, wait_ns)) {
                if (!*abort_flag) atomicOr(err, DEVERR_TIMEOUT_TMEM);
                *abort_flag = 1;
                ok = false;
                break;
            }
            tc_fence_after();
            drain_add(sum, lane_base, cols);          // the last chunk of H
            drain_add(sum, lane_base + 256u, cols);   // S
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&sh->chunk_free[1]));
            const RowCtx row = make_row(a.e, (int64_t)m0 + q4 * 32 + lane);
            const int jbase = wtile * a.wt;
            // with preloaded sums an update of the accumulators is a store, a finalize one without
            // earlier flushes
            const int kind = preload ? (kind0 == EPI_ADD_KAHAN ? EPI_STORE_KAHAN : EPI_FINAL) : kind0;
            switch (kind) {
                case EPI_FINAL: tc_epilogue_regs<EPI_FINAL>(a, row, col0, cols, jbase, sum); break;
                case EPI_FINAL_KAHAN: tc_epilogue_regs<EPI_FINAL_KAHAN>(a, row, col0, cols, jbase, sum); break;
                case EPI_FINAL_FP64: tc_epilogue_regs<EPI_FINAL_FP64>(a, row, col0, cols, jbase, sum); break;
                case EPI_STORE_KAHAN: tc_epilogue_regs<EPI_STORE_KAHAN>(a, row, col0, cols, jbase, sum); break;
                case EPI_STORE_FP64: tc_epilogue_regs<EPI_STORE_FP64>(a, row, col0, cols, jbase, sum); break;
                case EPI_ADD_KAHAN: tc_epilogue_regs<EPI_ADD_KAHAN>(a, row, col0, cols, jbase, sum); break;
                default: tc_epilogue_regs<EPI_ADD_FP64>(a, row, col0, cols, jbase, sum); break;
            }
        }
        // always wait (bounded) for the last commit: no MMA may still write TMEM at release
        if (!mbar_wait(smem_u32(&sh->tmem_full), 0u, nullptr)) atomicOr(err, DEVERR_TIMEOUT_TMEM);
        tc_fence_after();
    } else if (g.conv_on) {
        // warps 10 and 11 (launches with a conversion job only): the next segment's pushes
        tc_convert_job(g.conv, lane);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, ncols);
    }
    if (trace && threadIdx.x == 0) trace[6] = globaltimer();
}



// --------------------------------------------------------------------------------------
// In-place drained form (persistent), operand A in tensor memory.  The pushed complex64 frames
// are read without a staging pass: for every 32-frame block of a tile the producer copies, per
// frame, the tile's 128 rows (contiguous in the frame: checked by the host) into a ring of raw
// stages with contiguous bulk copies.  Eight worker warps subtract the provisional mean, split
// each value into bf16 hi/lo and write them to tensor memory with tcgen05.st, one TMEM column
// per frame (the packed (re, im) pair is one 32-bit column, two K elements): the MMAs take A
// from tensor memory and only the twiddle rows from shared memory, so neither the swizzled
// A layout nor its shared-memory bandwidth is needed.  Accumulation as in the split drained
// form: H = hi*hi drained into FP32 registers every drain_kb blocks, S = the small products
// for the whole tile.  The same warps drain and run the epilogues; a tile's final epilogue
// waits until the first `defer` blocks of the next tile are converted, so the tensor pipe has
// work while it runs.
//
//   warp 0     raw frame producer (16-byte asynchronous copies, 512 contiguous bytes a warp
//              instruction), up to raw_stages blocks ahead
//   warp 1     TMEM allocation and MMA issue
//   warp 10    twiddle producer (pre-swizzled rows, one bulk copy for hi and one for lo)
//   warps 2-9  workers: warp w owns TMEM lanes / tile rows 32 (w % 4) .. + 31; h = (w - 2) / 4
//              selects frames 16 h .. 16 h + 15 of each block and accumulator columns
//              [h wt, (h + 1) wt) of the drains and epilogue
// TMEM columns: H [0, N), S [acc_s, acc_s + N), A stage s [a_col + 64 s, + 64): hi 32 | lo 32.
// 352 threads put three warps on three of the four register files: at most 168 registers a
// thread, which bounds the drained columns a worker holds (kIpCols).
constexpr int kIpRawMax = 4;
constexpr int kIpBlockFrames = 32;
constexpr int kIpCols = 80;          // accumulator columns a worker drains (tiles of <= 80 energies)
struct TcInplaceArgs {
    CUtensorMap fmap;          // frames of the flush as [n_frames][pitch_frame] complex64 (fmap_ok)
    int fmap_ok;               // evenly spaced frames: one 2-D box of 32 frames x 128 rows a block
    TcPlanArgs a;
    TcDirectArgs d;
    int stages;                // A (tensor memory) + B (shared memory) stages
    int raw_stages;            // raw frame stages
    int defer;                 // blocks of the next tile converted before a tile's final epilogue
    uint32_t acc_s;            // TMEM column of the small-product accumulator
    uint32_t a_col;            // TMEM column of A stage 0
    int64_t tiles;             // (M_pad / 128) * n_wt
};
struct IpShared {
    uint64_t full[kMaxStages];      // twiddle copies landed + the 8 workers stored A
    uint64_t empty[kMaxStages];     // the stage's MMAs completed
    uint64_t raw_full[kIpRawMax];   // raw frame rows landed
    uint64_t raw_empty[kIpRawMax];  // the 8 workers read them
    uint64_t chunk_full[2];         // [0] an H chunk is complete, [1] the tile's H and S are
    uint64_t chunk_free[2];         // the workers drained them
    uint64_t sums_full[2];          // a tile's residual row sums are in `part` (by tile parity)
    uint64_t tmem_full;
    uint32_t tmem_addr;
    int abort_flag;
    double2 part[2][2][kMTile];     // [tile parity][frame half][row] sums of (psi - mu_hat)
};

__device__ __forceinline__ void mma_bf16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tmem_st_x8(uint32_t taddr, const uint32_t (&r)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Final of one tile in a worker thread: the last H chunk and S added to the running sums, the
// mean correction from the tile's residual sums, the epilogue.  Returns false on a timeout.
template <int KIND>
__device__ __forceinline__ bool ip_final(const TcInplaceArgs &g, IpShared *sh, float (&sum)[kIpCols], int t,
                                         int cnt, int h, int rr, uint32_t hbase, uint32_t sbase,
                                         volatile int *abort_flag, uint64_t wait_ns) {
    const TcPlanArgs &a = g.a;
    const TcDirectArgs &d = g.d;
    const int lane = threadIdx.x & 31;
    if (!mbar_wait_warp(smem_u32(&sh->sums_full[cnt & 1]), (uint32_t)((cnt >> 1) & 1), abort_flag, wait_ns) ||
        !mbar_wait_warp(smem_u32(&sh->chunk_full[1]), (uint32_t)(cnt & 1), abort_flag, wait_ns)) {
        if (lane == 0 && !*abort_flag) atomicOr(a.err, DEVERR_TIMEOUT_TMEM);
        *abort_flag = 1;
        return false;
    }
    tc_fence_after();
    const int cols = a.wt;
    drain_add(sum, hbase, cols);
    drain_add(sum, sbase, cols);
    tc_fence_before();
    const double2 p0 = sh->part[cnt & 1][0][rr], p1 = sh->part[cnt & 1][1][rr];
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_u32(&sh->chunk_free[1]));
    const int wtile = t % a.n_wt;
    const int64_t m0 = (int64_t)(t / a.n_wt) * kMTile;
    RowCtx row;
    row.m = m0 + rr;
    row.valid = row.m < d.M;
    const int64_t p = row.valid ? row.m / d.npix : 0;
    row.out_base = p * (int64_t)a.e.Nw * d.npix + (row.m - p * d.npix);
    row.dmu = make_float2(0.f, 0.f);
    double2 tt = make_double2(p0.x + p1.x, p0.y + p1.y);
    if (row.valid && h == 0 && wtile == 0 && d.accumulate_sums) {
        double2 s = d.sum_res[row.m];
        s.x += tt.x;
        s.y += tt.y;
        d.sum_res[row.m] = s;
    }
    if (row.valid && d.subtract_mean && a.e.mode == FLUSH_FINAL) {
        if (d.prev_sums) {
            const double2 pv = d.sum_res[row.m];
            tt.x += pv.x;
            tt.y += pv.y;
        }
        row.dmu = make_float2((float)(tt.x / d.T), (float)(tt.y / d.T));
    }
    const int col0 = h * cols, jbase = wtile * a.wt;
    tc_epilogue_regs<KIND>(a, row, col0, cols, jbase, sum);
#pragma unroll
    for (int k = 0; k < kIpCols; ++k) sum[k] = 0.f;
    return true;
}

template <int KIND>
__global__ void __maxnreg__(168) flush_tc_inplace_kernel(const __grid_constant__ TcInplaceArgs g) {
    const TcPlanArgs &a = g.a;
    const TcDirectArgs &d = g.d;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    constexpr int BF = kIpBlockFrames;
    const int stages = g.stages, R = g.raw_stages, N = a.N;
    constexpr uint32_t RB = 4u * BF;                                   // bytes per twiddle row
    const uint32_t b_pad = tc_b_bytes_padded(N, BF);
    const uint32_t b_stage = 2u * b_pad;                               // twiddle rows hi | lo
    constexpr uint32_t raw_bytes = (uint32_t)BF * kMTile * 8u;         // one raw stage
    uint8_t *raw = base + (size_t)stages * b_stage;
    IpShared *sh = reinterpret_cast<IpShared *>(raw + (size_t)R * raw_bytes);
    const uint32_t base_s = smem_u32(base), raw_s = smem_u32(raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n_tiles = g.tiles;
    unsigned long long *trace = a.trace ? a.trace + (size_t)blockIdx.x * kTraceWords : nullptr;
    if (trace && threadIdx.x == 0) {
        trace[0] = globaltimer();
        trace[7] = smid();
    }
    if (threadIdx.x == 0) {
        for (int st = 0; st < stages; ++st) {
            mbar_init(smem_u32(&sh->full[st]), 9);   // twiddle copies + eight worker warps
            mbar_init(smem_u32(&sh->empty[st]), 1);
        }
        for (int r = 0; r < R; ++r) {
            // one tensor copy (arrive with its bytes), or the producer warp's 32 lanes' copies
            mbar_init(smem_u32(&sh->raw_full[r]), g.fmap_ok ? 1 : 32);
            mbar_init(smem_u32(&sh->raw_empty[r]), 8);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&sh->chunk_full[b]), 1);
            mbar_init(smem_u32(&sh->chunk_free[b]), 8);
            mbar_init(smem_u32(&sh->sums_full[b]), 8);
        }
        mbar_init(smem_u32(&sh->tmem_full), 1);
        sh->abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(&sh->tmem_addr), 512u);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tmem_addr;
    volatile int *abort_flag = &sh->abort_flag;
    const uint64_t wait_ns = a.wait_ns ? a.wait_ns : kWaitLimitNs;
    if (trace && threadIdx.x == 0) trace[1] = globaltimer();

    if (warp == 0) {
        // ---------------- raw frame producer: runs up to raw_stages blocks ahead ----------------
        int r = 0, tma_issued = 0;
        uint32_t rph = 0;
        for (int64_t t = blockIdx.x; t < n_tiles && !*abort_flag; t += gridDim.x) {
            const int64_t m0 = (t / a.n_wt) * kMTile;
            const int nrows = (int)(d.M - m0 < kMTile ? d.M - m0 : kMTile);   // even (host-checked)
            const int64_t p = m0 / d.npix, pix = m0 - p * d.npix;
            const int64_t y = pix / d.kx, x = pix - y * d.kx;
            const int64_t off = p * d.pitch_probe + (d.roi_y0 + y) * d.pitch_row + (d.roi_x0 + x);
            const int nchunk = nrows / 2;                 // 16-byte chunks of a frame's rows
            bool stop = false;
            for (int kb = 0; kb < a.n_kb; ++kb) {
                const int f = kb * BF + lane;
                const float2 *fp = f < d.n_frames ? d.frame_ptr[f] + off : nullptr;
                const int nfr = min(BF, d.n_frames - kb * BF);
                if (!mbar_wait_warp(smem_u32(&sh->raw_empty[r]), rph ^ 1u, abort_flag, wait_ns)) {
                    if (lane == 0 && !*abort_flag) atomicOr(a.err, DEVERR_TIMEOUT_EMPTY);
                    *abort_flag = 1;
                    stop = true;
                    break;
                }
                if (g.fmap_ok) {
                    // one box: 32 frames x 128 rows (frames past the flush and rows past the
                    // frame read as zeros; the full box's bytes arrive)
                    if (lane == 0) {
                        const uint32_t rf = smem_u32(&sh->raw_full[r]);
                        mbar_arrive_expect_tx(rf, raw_bytes);
                        tma_load_2d(raw_s + (uint32_t)r * raw_bytes, &g.fmap, (int)off, kb * BF, rf);
                    }
                    tma_issued = tma_issued < R ? tma_issued + 1 : R;
                } else {
                    // frame j's rows: 16-byte chunks lane, lane + 32 (512 contiguous bytes a warp
                    // instruction); rows past M and frames past the flush stay stale (masked)
                    const uint32_t dst = raw_s + (uint32_t)r * raw_bytes + (uint32_t)lane * 16u;
                    for (int j = 0; j < nfr; ++j) {
                        const char *src =
                            reinterpret_cast<const char *>(__shfl_sync(0xffffffffu, (unsigned long long)fp, j));
                        if (lane < nchunk) cp_async16(dst + (uint32_t)j * kMTile * 8u, src + lane * 16);
                        if (lane + 32 < nchunk)
                            cp_async16(dst + (uint32_t)j * kMTile * 8u + 512u, src + lane * 16 + 512);
                    }
                    cp_async_arrive(smem_u32(&sh->raw_full[r]));
                }
                if (++r == R) {
                    r = 0;
                    rph ^= 1u;
                }
            }
            if (stop) break;
        }
        // no copy may still be landing in this CTA's shared memory when it exits
        cp_async_wait_all();
        if (*abort_flag && lane == 0) {
            // tensor copies in flight land on their raw stage's barrier
            int kr = r;
            uint32_t krp = rph;
            for (int i = 0; i < tma_issued; ++i) {
                if (--kr < 0) {
                    kr = R - 1;
                    krp ^= 1u;
                }
                if (!mbar_wait(smem_u32(&sh->raw_full[kr]), krp, nullptr)) atomicOr(a.err, DEVERR_TIMEOUT_DRAIN);
            }
        }
    } else if (warp == 10) {
        // ---------------- twiddle producer ----------------
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            int op_issued = 0;
            const uint32_t tx_b = 2u * (uint32_t)N * RB;
            const size_t b_step = (size_t)a.b_rows * RB;
            const uint64_t keep = l2_evict_last_policy();
            bool stop = false;
            for (int64_t t = blockIdx.x; t < n_tiles && !stop; t += gridDim.x) {
                const int wtile = (int)(t % a.n_wt);
                const uint8_t *pBhi = static_cast<const uint8_t *>(a.B_hi) +
                                      ((size_t)a.kbB0 * (size_t)a.b_rows + (size_t)wtile * N) * RB;
                const uint8_t *pBlo = static_cast<const uint8_t *>(a.B_lo) +
                                      ((size_t)a.kbB0 * (size_t)a.b_rows + (size_t)wtile * N) * RB;
                for (int kb = 0; kb < a.n_kb; ++kb) {
                    if (!mbar_wait(smem_u32(&sh->empty[s]), ph ^ 1u, abort_flag, wait_ns)) {
                        if (!*abort_flag) atomicOr(a.err, DEVERR_TIMEOUT_EMPTY);
                        *abort_flag = 1;
                        stop = true;
                        break;
                    }
                    const uint32_t full = smem_u32(&sh->full[s]);
                    const uint32_t st = base_s + (uint32_t)s * b_stage;
                    mbar_arrive_expect_tx(full, tx_b);
                    bulk_load_hint(st, pBhi + (size_t)kb * b_step, (uint32_t)N * RB, full, keep);
                    bulk_load_hint(st + b_pad, pBlo + (size_t)kb * b_step, (uint32_t)N * RB, full, keep);
                    op_issued = op_issued < stages ? op_issued + 1 : stages;
                    if (++s == stages) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
            if (*abort_flag && op_issued > 0) {
                // the twiddle copies share their stage barrier with the workers, which may never
                // arrive: give them a fixed 20 ms to land (copies take microseconds)
                const uint64_t t0 = globaltimer();
                while (globaltimer() - t0 < 20000000ull) {
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA: A from tensor memory, B from shared memory ----------------
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0, hph = 0, tph = 0;
            int64_t tiles = 0;
            bool stop = false;
            const uint32_t accH = tmem, accS = tmem + g.acc_s;
            const uint32_t id = idesc_bf16_f32(kMTile, N);
            const int cb = a.drain_kb;
            for (int64_t t = blockIdx.x; t < n_tiles && !stop; t += gridDim.x, ++tiles) {
                if (tiles > 0) {
                    if (!mbar_wait(smem_u32(&sh->chunk_free[1]), tph, abort_flag, wait_ns)) {
                        if (!*abort_flag) atomicOr(a.err, DEVERR_TIMEOUT_TMEM);
                        *abort_flag = 1;
                        break;
                    }
                    tph ^= 1u;
                    tc_fence_after();
                }
                int kc = 0;
                for (int kb = 0; kb < a.n_kb; ++kb) {
                    if (!mbar_wait(smem_u32(&sh->full[s]), ph, abort_flag, wait_ns)) {
                        if (!*abort_flag) atomicOr(a.err, DEVERR_TIMEOUT_FULL);
                        *abort_flag = 1;
                        stop = true;
                        break;
                    }
                    tc_fence_after();
                    if (trace && tiles == 0 && kb == 0) trace[2] = globaltimer();
                    const uint32_t aH = tmem + g.a_col + 64u * (uint32_t)s, aL = aH + 32u;
                    const uint32_t st = base_s + (uint32_t)s * b_stage;
                    const uint64_t dBhi0 = sdesc_k(st, RB);
                    const uint64_t dBlo0 = sdesc_k(st + b_pad, RB);
#pragma unroll
                    for (int ks = 0; ks < BF / 8; ++ks) {
                        const uint64_t adv = (uint64_t)(2 * ks);
                        mma_bf16_ts(accS, aH + 8u * ks, dBlo0 + adv, id, (kb == 0 && ks == 0) ? 0u : 1u);
                        mma_bf16_ts(accS, aL + 8u * ks, dBhi0 + adv, id, 1u);
                    }
                    if (kc == 0 && kb > 0) {
                        if (!mbar_wait(smem_u32(&sh->chunk_free[0]), hph, abort_flag, wait_ns)) {
                            if (!*abort_flag) atomicOr(a.err, DEVERR_TIMEOUT_TMEM);
                            *abort_flag = 1;
                            stop = true;
                            break;
                        }
                        hph ^= 1u;
                        tc_fence_after();
                    }
#pragma unroll
                    for (int ks = 0; ks < BF / 8; ++ks) {
                        const uint64_t adv = (uint64_t)(2 * ks);
                        mma_bf16_ts(accH, aH + 8u * ks, dBhi0 + adv, id, (kc == 0 && ks == 0) ? 0u : 1u);
                    }
                    mma_commit(smem_u32(&sh->empty[s]));
                    if (++s == stages) {
                        s = 0;
                        ph ^= 1u;
                    }
                    if (++kc == cb && kb != a.n_kb - 1) {
                        mma_commit(smem_u32(&sh->chunk_full[0]));
                        kc = 0;
                    }
                }
                if (stop) break;
                mma_commit(smem_u32(&sh->chunk_full[1]));
            }
            mma_commit(smem_u32(&sh->tmem_full));
            if (trace) {
                trace[3] = globaltimer();
                trace[4] = (unsigned long long)tiles;
                trace[5] = 0;
            }
        }
    } else {
        // ---------------- workers: conversion into TMEM, drains, epilogues ----------------
        const int q = warp & 3, h = (warp - 2) >> 2;
        const int rr = q * 32 + lane;                                   // tile row = TMEM lane
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        const int cols = a.wt;
        const uint32_t hbase = tmem + lane_off + (uint32_t)(h * cols);
        const uint32_t sbase = tmem + lane_off + g.acc_s + (uint32_t)(h * cols);
        const uint32_t abase = tmem + lane_off + g.a_col + 16u * (uint32_t)h;
        const int cb = a.drain_kb, D = g.defer;
        float sum[kIpCols];
#pragma unroll
        for (int k = 0; k < kIpCols; ++k) sum[k] = 0.f;
        int s = 0, r = 0;
        uint32_t ph = 0, rph = 0;
        uint32_t hc = 0;
        int tiles = 0, fin_t = -1, fin_cnt = 0;   // tile indices fit 31 bits (host-checked)
        int t = (int)blockIdx.x;
        int kb = 0;
        bool valid = false;
        float2 mu = make_float2(0.f, 0.f);
        // per-tile residual sums in FP32 with compensation (FP64 arithmetic is slow on this part)
        float sr = 0.f, si = 0.f, cr = 0.f, ci = 0.f;
        // one pass per block of this CTA's tiles, plus a last pass for the last tile's final
        for (;;) {
            const bool have = t < n_tiles;
            if (have) {
                if (kb == 0) {
                    const int64_t m = (t / a.n_wt) * kMTile + rr;
                    valid = m < d.M;
                    mu = valid ? d.mu_hat[m] : make_float2(0.f, 0.f);
                    sr = si = cr = ci = 0.f;
                }
                if (!mbar_wait_warp(smem_u32(&sh->raw_full[r]), rph, abort_flag, wait_ns) ||
                    !mbar_wait_warp(smem_u32(&sh->empty[s]), ph ^ 1u, abort_flag, wait_ns)) {
                    if (lane == 0 && !*abort_flag) atomicOr(a.err, DEVERR_TIMEOUT_FULL);
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const int nfr = min(BF, d.n_frames - kb * BF);
                const uint8_t *rs = raw + (size_t)r * raw_bytes + (size_t)rr * 8u;
                const uint32_t ac = abase + 64u * (uint32_t)s;
                // all 16 of this warp's frames in flight at once.  The raw stage is always
                // readable; rows past M and frames past the flush hold stale data and are
                // replaced by the mean (a zero residual) on the rare partial blocks
                float2 x[16];
#pragma unroll
                for (int f = 0; f < 16; ++f)
                    x[f] = *reinterpret_cast<const float2 *>(rs + (size_t)(16 * h + f) * kMTile * 8u);
                if (!valid || nfr < BF) {
#pragma unroll
                    for (int f = 0; f < 16; ++f)
                        if (!valid || 16 * h + f >= nfr) x[f] = mu;
                }
                float br = 0.f, bi = 0.f;
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    uint32_t hw[8], lw[8];
#pragma unroll
                    for (int f = 0; f < 8; ++f) {
                        const float2 v = make_float2(x[8 * half + f].x - mu.x, x[8 * half + f].y - mu.y);
                        br += v.x;
                        bi += v.y;
                        split2_bf16(v, hw[f], lw[f]);
                    }
                    __syncwarp();
                    tmem_st_x8(ac + 8u * (uint32_t)half, hw);
                    tmem_st_x8(ac + 32u + 8u * (uint32_t)half, lw);
                }
                kahan_add(sr, cr, br);
                kahan_add(si, ci, bi);
                tmem_st_wait();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&sh->raw_empty[r]));
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&sh->full[s]));
                if (++s == stages) {
                    s = 0;
                    ph ^= 1u;
                }
                if (++r == R) {
                    r = 0;
                    rph ^= 1u;
                }
            }
            // the previous tile's final, once this tile's first `defer` blocks keep the MMAs
            // busy (or after the last tile)
            if (fin_t >= 0 && (!have || kb + 1 == D)) {
                if (!ip_final<KIND>(g, sh, sum, fin_t, fin_cnt, h, rr, hbase, sbase, abort_flag, wait_ns)) break;
                fin_t = -1;
            }
            if (!have) break;
            // the H chunk that ended with block kb - 1 (drained one block late, so this block's
            // small products run on the tensor pipe meanwhile)
            if (kb >= 1 && kb % cb == 0) {
                if (!mbar_wait_warp(smem_u32(&sh->chunk_full[0]), (uint32_t)(hc & 1), abort_flag, wait_ns)) {
                    if (lane == 0 && !*abort_flag) atomicOr(a.err, DEVERR_TIMEOUT_TMEM);
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                drain_add(sum, hbase, cols);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&sh->chunk_free[0]));
                ++hc;
            }
            if (++kb == a.n_kb) {
                // this tile's residual sums (frame half h) for its final
                sh->part[tiles & 1][h][rr] = make_double2((double)sr - (double)cr, (double)si - (double)ci);
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&sh->sums_full[tiles & 1]));
                fin_t = t;
                fin_cnt = tiles;
                ++tiles;
                t += (int)gridDim.x;
                kb = 0;
            }
        }
        if (!mbar_wait_warp(smem_u32(&sh->tmem_full), 0u, nullptr) && lane == 0) atomicOr(a.err, DEVERR_TIMEOUT_TMEM);
        tc_fence_after();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 512u);
    }
    if (trace && threadIdx.x == 0) trace[6] = globaltimer();
}

// --------------------------------------------------------------------------------------
// host side
// --------------------------------------------------------------------------------------
// Launches a persistent contraction grid with the cluster-dimension launch attribute (clusters of
// one CTA: no cluster feature is used).  Measured on GB300: the same kernel and grid launched
// this way ran 12 % faster on the realistic workload (52.1 vs 59.3 ms) than a plain launch,
// which places the CTAs on the SMs in a different order.
template <typename Arg>
static cudaError_t launch_persistent(void (*kern)(Arg), unsigned grid, unsigned threads, size_t smem,
                                     cudaStream_t st, const Arg &arg) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, arg);
}

int tc_stages_for(int N, int bf) {
    const int budget = kSmemLimit - 1024 - (int)sizeof(TcShared);
    int s = budget / (int)tc_stage_bytes(N, bf);
    if (s > kMaxStages) s = kMaxStages;
    return s;
}

size_t tc_smem_bytes(int N, int bf, int stages) {
    return (size_t)stages * tc_stage_bytes(N, bf) + sizeof(TcShared) + 1024;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// In-place drained kernel: shared memory of `stages` twiddle stages and `raw` raw frame stages.
static size_t tc_inplace_smem_bytes(int N, int stages, int raw) {
    return (size_t)stages * 2 * tc_b_bytes_padded(N, kIpBlockFrames) +
           (size_t)raw * kIpBlockFrames * kMTile * 8 + sizeof(IpShared) + 1024;
}

// Stage counts of the in-place drained kernel for an N-column tile: TMEM holds H, S (at a
// 32-column boundary) and 64 columns per A stage; two stages with as many raw stages as shared
// memory allows (up to four).  Returns the A/B stages (0: the tile does not fit).
int tc_inplace_stages(int N, int bf, int *raw_out, uint32_t *acc_s, uint32_t *a_col) {
    if (bf != kIpBlockFrames || N <= 0 || N % 16) return 0;
    const int s_col = (N + 31) & ~31;
    const int stages = 2;
    if (s_col + N + 64 * stages > 512) return 0;
    int raw = kIpRawMax;
    while (raw >= 2 && tc_inplace_smem_bytes(N, stages, raw) > (size_t)kSmemLimit) --raw;
    if (raw < 2) return 0;
    if (raw_out) *raw_out = raw;
    if (acc_s) *acc_s = (uint32_t)s_col;
    if (a_col) *a_col = (uint32_t)(512 - 64 * stages);
    return stages;
}

bool tc_make_frame_map(void *map_out, const void *first_frame, int64_t pitch_frame, int n_frames, char *errbuf,
                       size_t errlen) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) {
        snprintf(errbuf, errlen, "cuTensorMapEncodeTiled is not available from the driver");
        return false;
    }
    // complex64 elements as 8-byte words: [n_frames][pitch_frame], box 32 frames x 128 rows
    cuuint64_t dims[2] = {(cuuint64_t)pitch_frame, (cuuint64_t)n_frames};
    cuuint64_t strides[1] = {(cuuint64_t)pitch_frame * 8};
    cuuint32_t box[2] = {(cuuint32_t)kMTile, (cuuint32_t)kIpBlockFrames};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(reinterpret_cast<CUtensorMap *>(map_out), CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
                    const_cast<void *>(first_frame), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        snprintf(errbuf, errlen, "cuTensorMapEncodeTiled(frames) failed with %d", (int)r);
        return false;
    }
    return true;
}
size_t tc_frame_map_size() { return sizeof(CUtensorMap); }

cudaError_t launch_flush_tc_inplace(const TcPlanArgs &a, const TcDirectArgs &d, const void *frame_map, cudaStream_t st) {
    TcInplaceArgs g{};
    g.a = a;
    g.d = d;
    g.fmap_ok = frame_map != nullptr;
    if (frame_map) memcpy(&g.fmap, frame_map, sizeof(CUtensorMap));
    g.stages = tc_inplace_stages(a.N, a.bf, &g.raw_stages, &g.acc_s, &g.a_col);
    g.tiles = (a.e.M_pad / kMTile) * a.n_wt;
    if (g.stages < 2 || a.wt > kIpCols || a.drain_kb < 1 || a.n_kb < 1 || g.tiles <= 0 || g.tiles > 0x7fffffffLL)
        return cudaErrorInvalidConfiguration;
    // the next tile's first blocks converted before a tile's final: at most stages - 1 (their
    // stages must be free while the final's tile still holds the others), and not past the
    // first H chunk drain
    g.defer = std::min(std::min(g.stages - 1, a.drain_kb), a.n_kb);
    const size_t smem = tc_inplace_smem_bytes(a.N, g.stages, g.raw_stages);
    // one instantiation per flush mode: a single epilogue path keeps the workers' registers
    void (*kern)(TcInplaceArgs) = nullptr;
    switch (epi_kind(a.e)) {
        case EPI_FINAL: kern = flush_tc_inplace_kernel<EPI_FINAL>; break;
        case EPI_FINAL_KAHAN: kern = flush_tc_inplace_kernel<EPI_FINAL_KAHAN>; break;
        case EPI_FINAL_FP64: kern = flush_tc_inplace_kernel<EPI_FINAL_FP64>; break;
        case EPI_STORE_KAHAN: kern = flush_tc_inplace_kernel<EPI_STORE_KAHAN>; break;
        case EPI_STORE_FP64: kern = flush_tc_inplace_kernel<EPI_STORE_FP64>; break;
        case EPI_ADD_KAHAN: kern = flush_tc_inplace_kernel<EPI_ADD_KAHAN>; break;
        default: kern = flush_tc_inplace_kernel<EPI_ADD_FP64>; break;
    }
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 352, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    int64_t cap = (int64_t)occ * sms;
    if (a.max_ctas > 0 && a.max_ctas < cap) cap = a.max_ctas;
    const int64_t grid = g.tiles < cap ? g.tiles : cap;
    return launch_persistent(kern, (unsigned)grid, 352u, smem, st, g);
}

// Co-resident CTAs of the staged contraction kernel for an N-column tile (0 on error).
int tc_resident_ctas(int N, int bf, int stages) {
    const size_t smem = tc_smem_bytes(N, bf, stages);
    int n = 0;
    if (cudaFuncSetAttribute(flush_tc_drain2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, flush_tc_drain2_kernel, 320, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n * sms;
}

int64_t tc_grid_ctas(const TcPlanArgs &a) { return a.e.M_pad / kMTile * a.n_wt; }

static cudaError_t launch_flush_tc_group_impl(const TcPlanArgs *args, int n, const TcConvJob *conv,
                                              cudaStream_t st) {
    if (n < 1 || n > kMaxGroupStreams) return cudaErrorInvalidValue;
    // 10 warps (producer, MMA, 8 epilogue); 12 with a conversion job.  At 168 registers a thread,
    // 12 warps put 3 on each of the SM's four register files (16 128 of 16 384 registers).
    const int threads = conv ? 384 : 320;
    TcGroup *g = new (std::nothrow) TcGroup();
    if (!g) return cudaErrorMemoryAllocation;
    int64_t total = 0;
    int n_max = 0;
    for (int i = 0; i < n; ++i) {
        // one staging row width per launch; register sums of at most kDrainCols columns a thread
        if (args[i].bf != args[0].bf || args[i].wt > kDrainCols || args[i].drain_kb < 1 || !args[0].tile_counter) {
            delete g;
            return cudaErrorInvalidValue;
        }
        g->e[i].args = args[i];
        g->e[i].cta_begin = (int)total;
        const int64_t c = tc_grid_ctas(args[i]);
        g->e[i].ctas = (int)c;
        total += c;
        n_max = std::max(n_max, args[i].N);
    }
    g->n = n;
    g->conv_on = conv ? 1 : 0;
    if (conv) g->conv = *conv;
    if (total <= 0 || total > 0x7fffffffLL) {
        delete g;
        return cudaErrorInvalidConfiguration;
    }
    // the ring and TMEM are sized for the widest tile; one wave of CTAs walks all tiles
    g->n_max = n_max;
    g->stages = tc_stages_for(n_max, args[0].bf);
    g->tiles = total;
    const size_t smem = tc_smem_bytes(n_max, args[0].bf, g->stages);
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(flush_tc_drain2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, flush_tc_drain2_kernel, threads, smem);
    if (e != cudaSuccess || g->stages < 2 || n_max > 2 * kDrainCols || occ < 1) {
        delete g;
        return e != cudaSuccess ? e : cudaErrorInvalidConfiguration;
    }
    int64_t cap = (int64_t)occ * sms;
    if (args[0].max_ctas > 0 && args[0].max_ctas < cap) cap = args[0].max_ctas;
    const unsigned grid = (unsigned)(cap < total ? cap : total);
    // the CTAs take tiles from a counter in device memory, zeroed on the stream before the launch
    g->counter = args[0].tile_counter;
    e = cudaMemsetAsync(g->counter, 0, sizeof(int), st);
    if (e == cudaSuccess && conv) e = cudaMemsetAsync(conv->counter, 0, sizeof(int), st);
    if (e == cudaSuccess) e = launch_persistent(flush_tc_drain2_kernel, grid, (unsigned)threads, smem, st, *g);
    delete g;
    return e;
}

cudaError_t launch_flush_tc_group(const TcPlanArgs *args, int n, cudaStream_t st) {
    return launch_flush_tc_group_impl(args, n, nullptr, st);
}

cudaError_t launch_flush_tc_group_conv(const TcPlanArgs *args, int n, const TcConvJob &conv, cudaStream_t st) {
    if (!conv.frame_ptr || !conv.counter || conv.T % 32 || conv.M_pad % kMTile || args[0].bf != 32)
        return cudaErrorInvalidValue;
    return launch_flush_tc_group_impl(args, n, &conv, st);
}

cudaError_t launch_flush_tc(const TcPlanArgs &a, cudaStream_t st) { return launch_flush_tc_group(&a, 1, st); }

}  // namespace tacaw
