// Tensor-core (tcgen05) contraction of staged frames with the twiddle table, split BF16:
//
//   Psi[m, j] (+)= sum_f y[m, f] B[t0 + f, j]        y = psi - mu_hat, B = w_t exp(-i theta_jt)
//
// the windowed time->energy transform of Eq. 1 over the frames of one flush, as a real
// GEMM on the embedding  [Re y, Im y] x [[Re B, Im B], [-Im B, Re B]].  Every operand is
// split x = hi + lo (bf16 each); the product is accumulated as hi*hi + hi*lo + lo*hi in
// FP32 in tensor memory (the dropped lo*lo term is ~2^-16 relative).
//
// Tensor-core FP32 accumulation rounds each accumulate step relative to the running sum,
// so long K loops into one accumulator lose precision in proportion to their length.  With
// split accumulators the hi*hi products alternate between two TMEM accumulators (even and
// odd 8-frame blocks) and the small hi*lo + lo*hi terms go to a third, which keeps every
// accumulate step short relative to its own sum; the epilogue adds the three.
//
// CTA = 128 rows (one TMEM lane each) x N real columns (2*wt complex energies).
//   warp 0      TMA producer: per staging block of bf frames (8, 16 or 32), A_hi/A_lo boxes
//               [128 x 2bf] and this CTA's share of the B_hi/B_lo rows (bf16 rows of 32, 64
//               or 128 bytes with the matching 32B/64B/128B swizzle) into an s-stage ring;
//               with a cluster of C CTAs (same energy tile, C consecutive row tiles) each
//               CTA loads N/C rows of B and multicasts them to the whole cluster
//               Each stage holds bf/8 MMA K-steps of K=16: the descriptors of step k start
//               32*k bytes into the swizzled rows.
//   warp 1      TMEM allocator + single-thread MMA issuer; tcgen05.commit releases ring
//               slots in every CTA of the cluster
//   warps 2..5  epilogue: tcgen05.ld of the accumulators (warp w reads lanes 32*(w%4)..)
//               and the per-element flush update (store / compensated add / finalize)
// Every mbarrier wait is bounded (globaltimer); on timeout the kernel records an error
// bit, lets in-flight copies land, frees TMEM and returns.
//
// Kernels of this file:
//   flush_tc_kernel          the layout above (1, 2 or 3 accumulators, optional multicast)
//   flush_tc_pair_kernel     CTA pairs (cta_group::2, 256-row MMAs over two SMs)
//   flush_tc_drain_kernel    persistent, one double-buffered accumulator drained into FP32
//   flush_tc_drain2_kernel   persistent, hi*hi drained, small products apart (the default)
//   flush_tc_inplace_kernel  persistent, pushed frames read in place, operand A converted into
//                            tensor memory (no staging pass)
//   flush_tc_direct_kernel   pushed frames read in place, converted in shared memory
#include <cuda.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>

#include "tacaw_internal.cuh"

namespace tacaw {

struct TcMaps {
    CUtensorMap a_hi, a_lo, b_hi, b_lo;
    int box_b_rows;
    int nbox_b;
};

// One launch over the tiles of several streams (supercell partitions): entry i owns CTAs
// [cta_begin, cta_begin + ctas) (a multiple of the cluster size).
struct TcGroupEntry {
    TcMaps maps;
    TcPlanArgs args;
    int cta_begin;
    int ctas;
};
struct TcGroup {
    TcGroupEntry e[kMaxGroupStreams];
    int n;
    int stages, n_max;         // drained kernel: ring stages and ring/TMEM width (widest tile)
    int64_t tiles;             // drained kernel: tiles of all entries
    int rot;                   // drained kernel: rotate energy tiles across a CTA's passes (see wtile_of)
};

// Energy tile of local tile lt on a CTA's k-th pass.  Tiles go out in row-major order (the
// energy tiles of a row tile run side by side and share its operand rows in L2).  When the
// grid is a multiple of the tile count per row (one stream), every pass hands each CTA the
// same energy slot; rotating the slot by the pass number keeps each row tile's set of energy
// tiles intact while cycling every CTA through all of them (a narrower last tile then shortens
// every CTA's work alike).
__device__ __forceinline__ int wtile_of(int64_t lt, int n_wt, int rot, int64_t pass) {
    const int w = (int)(lt % n_wt);
    return rot ? (int)((w + pass) % n_wt) : w;
}

constexpr uint64_t kWaitLimitNs = 4000000000ull;  // 4 s per wait
constexpr int kMaxStages = 12;
constexpr int kSmemLimit = 232448;                 // 227 KB opt-in per block

struct TcShared {
    uint64_t full[kMaxStages];
    uint64_t empty[kMaxStages];
    uint64_t tmem_full;
    uint32_t tmem_addr;
    int abort_flag;
    float2 W[256];      // window transform W(E_j) of this CTA's energies
    float bose[256];    // Bose factors of this CTA's energies
    double2 rowsum[kMTile];   // in-place kernel: sum over this flush of (psi - mu_hat) per row
    uint64_t sums_ready;      // in-place kernel: producers -> epilogue
    uint64_t chunk_full[2];   // drained kernel: a chunk's accumulator buffer is complete
    uint64_t chunk_free[2];   // drained kernel: the epilogue warps have drained it
    uint64_t raw_full[2];     // in-place drained kernel: raw frame rows landed
    uint64_t raw_empty[2];    //   converters are done with a raw stage
    uint64_t sums_full[2];    //   a tile's row sums are in `tsum`
    uint64_t sums_free[2];    //   the epilogue has read them
    double2 tsum[2][kMTile];  //   per-tile sums of (psi - mu_hat) over this flush, double-buffered
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
// Bounded wait.  Gives up after kWaitLimitNs, or early when *abort_flag is set (if given).
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (abort_flag && *abort_flag) return false;
        if (globaltimer() - t0 > kWaitLimitNs) return false;
    }
}
// Warp-uniform bounded wait: lane 0 waits, every lane gets its verdict (so no lane of the warp
// can leave a loop that the others stay in), and the warp synchronises for memory ordering.
__device__ __forceinline__ bool mbar_wait_warp(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
    int ok = 1;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, abort_flag) ? 1 : 0;
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
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
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
// L2 prefetch of a tensor box (no shared-memory destination, no completion)
__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap *map, int c0, int c1, int c2) {
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(c0), "r"(c1), "r"(c2)
                 : "memory");
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
// CTA-pair forms (tcgen05 ... cta_group::2): one warp of EACH CTA of the pair performs the
// allocation, relinquish and deallocation collectively; MMAs and commits are issued by the
// even CTA only.
__device__ __forceinline__ void tmem_alloc2(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish2() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc2(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void mma2_bf16_ss(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                             uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma2_commit_mc(uint32_t bar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
        "h"(mask)
        : "memory");
}
// Copy into this CTA's shared memory whose completion is counted on a barrier of the pair's
// even CTA (bar: shared::cluster address).
__device__ __forceinline__ void tma_load_3d_pair(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                                 uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
        "%4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}
// shared::cluster address of the same shared-memory offset in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cluster(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait on a barrier that also receives arrivals from the peer CTA.
__device__ bool mbar_wait_cluster(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
    if (mbar_try_wait_cluster(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (;;) {
        if (mbar_try_wait_cluster(bar, parity)) return true;
        if (abort_flag && *abort_flag) return false;
        if (globaltimer() - t0 > kWaitLimitNs) return false;
    }
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
__device__ __forceinline__ void mma_commit_mc(uint32_t bar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
        "h"(mask)
        : "memory");
}
__device__ __forceinline__ void tma_load_3d_mc(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                               uint32_t bar, uint16_t mask) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster"
        " [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar), "h"(mask)
        : "memory");
}
__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
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
// B rows held by one CTA: the whole tile, or half of it in the CTA-pair form
__host__ __device__ inline int tc_b_rows(int N, int pair) { return pair ? N / 2 : N; }
__host__ __device__ inline uint32_t tc_stage_bytes(int N, int bf, int pair = 0) {
    return 2u * tc_a_bytes(bf) + 2u * tc_b_bytes_padded(tc_b_rows(N, pair), bf);
}
__host__ __device__ inline uint32_t tc_tmem_cols(int N) {
    uint32_t c = 32;
    while (c < (uint32_t)N) c <<= 1;
    return c;
}

// Epilogue of one row (one TMEM lane) of a tile: drains the accumulators 32 columns at a time
// and applies the flush update of kind KIND to every energy of the tile.
template <int KIND>
__device__ __forceinline__ void tc_epilogue(const TcPlanArgs &a, const TcShared *sh, const RowCtx &row,
                                            uint32_t lane_base, int jbase, int n_big_used) {
    const uint32_t o_big1 = (uint32_t)a.N, o_small = (uint32_t)(a.n_big * a.N);
    // 32 columns (16 energies) per round: every accumulator's loads are issued before one wait
    for (int c0 = 0; c0 < a.N; c0 += 32) {
        __syncwarp();
        const bool two = c0 + 16 < a.N;
        uint32_t r0[16], r1[16], s0[16], s1[16], t0[16], t1[16];
        tmem_ld_x16(lane_base + (uint32_t)c0, r0);
        if (two) tmem_ld_x16(lane_base + (uint32_t)(c0 + 16), r1);
        if (a.split) {
            if (n_big_used == 2) {
                tmem_ld_x16(lane_base + o_big1 + (uint32_t)c0, s0);
                if (two) tmem_ld_x16(lane_base + o_big1 + (uint32_t)(c0 + 16), s1);
            }
            tmem_ld_x16(lane_base + o_small + (uint32_t)c0, t0);
            if (two) tmem_ld_x16(lane_base + o_small + (uint32_t)(c0 + 16), t1);
        }
        tmem_ld_wait();
        if (row.valid) {
            float v[32];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                v[i] = __uint_as_float(r0[i]);
                v[16 + i] = two ? __uint_as_float(r1[i]) : 0.f;
            }
            if (a.split) {
                if (n_big_used == 2) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        v[i] += __uint_as_float(s0[i]);
                        if (two) v[16 + i] += __uint_as_float(s1[i]);
                    }
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    v[i] += __uint_as_float(t0[i]);
                    if (two) v[16 + i] += __uint_as_float(t1[i]);
                }
            }
            const int jn = two ? 16 : 8;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int jl = (c0 >> 1) + i;
                const int j = jbase + jl;
                if (i < jn && j < a.e.Nw)
                    epi_apply<KIND>(a.e, row, j, v[2 * i], v[2 * i + 1], sh->W[jl], sh->bose[jl]);
            }
        }
        __syncwarp();   // the next round's tcgen05.ld needs the whole warp converged
    }
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

// MMA issue loop of the in-place kernel (one thread): per stage, bf/8 K-steps of 3 products
// into the accumulators; tcgen05.commit releases the stage and, at the end, signals the
// epilogue.  (The staged kernel keeps its own copy of this loop inline, with the cluster
// multicast release.)
__device__ __forceinline__ void tc_mma_loop(const TcPlanArgs &a, TcShared *sh, uint32_t base_s, uint32_t stage_bytes,
                                            uint32_t kABytes, uint32_t b_pad, uint32_t RB, uint32_t tmem,
                                            volatile int *abort_flag, unsigned long long *trace, bool multicast) {
    const uint16_t cmask = (uint16_t)((1u << a.cluster) - 1u);
    const int n0 = a.N < 256 ? a.N : 256;
    const int n1 = a.N - n0;
    const uint32_t id0 = idesc_f32acc(kMTile, n0, a.f16);
    const uint32_t id1 = n1 > 0 ? idesc_f32acc(kMTile, n1, a.f16) : 0u;
    const uint64_t b_half_off = (uint64_t)((n0 * RB) >> 4);
    const uint32_t acc_small = tmem + (uint32_t)(a.n_big * a.N);
    const int ksteps = a.bf / 8;
    int s_ring = -1;       // ring slot and use of staging block kb (no divisions)
    uint32_t u_ring = 0;
    for (int kb = 0; kb < a.n_kb; ++kb) {
        if (++s_ring == a.stages) {
            s_ring = 0;
            ++u_ring;
        }
        const int s = s_ring;
        const uint32_t use = u_ring;
        if (!mbar_wait(smem_u32(&sh->full[s]), use & 1u, abort_flag)) {
            if (!*abort_flag) atomicOr(a.err, DEVERR_TIMEOUT_FULL);
            *abort_flag = 1;
            break;
        }
        tc_fence_after();
        if (trace && kb == 0) trace[2] = globaltimer();
        const uint32_t st = base_s + (uint32_t)s * stage_bytes;
        const uint64_t dAhi0 = sdesc_k(st, RB);
        const uint64_t dAlo0 = sdesc_k(st + kABytes, RB);
        const uint64_t dBhi0 = sdesc_k(st + 2 * kABytes, RB);
        const uint64_t dBlo0 = sdesc_k(st + 2 * kABytes + b_pad, RB);
        for (int ks = 0; ks < ksteps; ++ks) {
            // K-step ks starts 32*ks bytes into the swizzled rows (start address in 16 B units)
            const uint64_t adv = (uint64_t)(2 * ks);
            const uint64_t dAhi = dAhi0 + adv, dAlo = dAlo0 + adv, dBhi = dBhi0 + adv, dBlo = dBlo0 + adv;
            const int g = kb * ksteps + ks;       // global K-step index
            if (a.split) {
                // N <= 256: one MMA per product
                const int big = a.n_big == 2 ? (g & 1) : 0;
                mma_bf16_ss(tmem + (uint32_t)(big * a.N), dAhi, dBhi, id0, g >= a.n_big ? 1u : 0u);
                mma_bf16_ss(acc_small, dAhi, dBlo, id0, g > 0 ? 1u : 0u);
                mma_bf16_ss(acc_small, dAlo, dBhi, id0, 1u);
            } else {
#pragma unroll
                for (int pass = 0; pass < 3; ++pass) {
                    const uint64_t dA = pass == 2 ? dAlo : dAhi;
                    const uint64_t dB = pass == 1 ? dBlo : dBhi;
                    const uint32_t acc = (g > 0 || pass > 0) ? 1u : 0u;
                    mma_bf16_ss(tmem, dA, dB, id0, acc);
                    if (n1 > 0) mma_bf16_ss(tmem + (uint32_t)n0, dA, dB + b_half_off, id1, acc);
                }
            }
        }
        if (multicast)
            mma_commit_mc(smem_u32(&sh->empty[s]), cmask);
        else
            mma_commit(smem_u32(&sh->empty[s]));
    }
    // always signal: the epilogue (and TMEM release) wait for every issued MMA
    mma_commit(smem_u32(&sh->tmem_full));
    if (trace) trace[3] = globaltimer();
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

// Final epilogue of the drained form: the last chunk's accumulator plus the running sums, for
// the thread's columns [col0, col0 + cols) (energies col0/2 ...).
template <int KIND>
__device__ __forceinline__ void tc_epilogue_drained(const TcPlanArgs &a, const RowCtx &row, uint32_t taddr,
                                                    int col0, int cols, int jbase,
                                                    const float (&sum)[kDrainCols]) {
#pragma unroll
    for (int r = 0; r < kDrainCols / 16; ++r) {
        if (r * 16 < cols) {
            uint32_t x[16];
            tmem_ld_x16(taddr + (uint32_t)(r * 16), x);
            tmem_ld_wait();
            if (row.valid) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int c = r * 16 + 2 * i;          // column of the thread's range (even)
                    const int j = jbase + ((col0 + c) >> 1);
                    // W(E_j), B(E_j): the same address across the warp (broadcast loads)
                    if (c < cols && j < a.e.Nw)
                        epi_apply<KIND>(a.e, row, j, sum[c] + __uint_as_float(x[2 * i]),
                                        sum[c + 1] + __uint_as_float(x[2 * i + 1]), __ldg(a.e.Wc + j),
                                        __ldg(a.e.bose + j));
                }
            }
        }
        __syncwarp();
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

// Body of the staged contraction kernel.  PAIR: the CTA-pair form -- clusters of two CTAs run
// M = 256 MMAs (tcgen05 cta_group::2) issued by the even CTA: each CTA stages its own 128 rows
// of A and half of the tile's B rows, so each SM reads half the B operand per MMA; both CTAs
// receive their 128 accumulator rows in their own TMEM.  The odd CTA's warp 1 relays its
// stage-full events to the even CTA's barrier (remote arrive), so every CTA still waits only
// on barriers in its own shared memory when it drains its copies.
template <bool PAIR>
__device__ __forceinline__ void flush_tc_body(const TcGroup &g) {
    int gi = 0;
    while (gi + 1 < g.n && (int)blockIdx.x >= g.e[gi + 1].cta_begin) ++gi;
    const TcMaps &maps = g.e[gi].maps;
    const TcPlanArgs a = g.e[gi].args;
    const unsigned bid = blockIdx.x - (unsigned)g.e[gi].cta_begin;   // CTA index inside its stream
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t RB = 4u * (uint32_t)a.bf;           // bytes per operand row
    const uint32_t kABytes = tc_a_bytes(a.bf);
    const uint32_t b_pad = tc_b_bytes_padded(tc_b_rows(a.N, PAIR), a.bf);
    const uint32_t stage_bytes = tc_stage_bytes(a.N, a.bf, PAIR);
    TcShared *sh = reinterpret_cast<TcShared *>(base + (size_t)a.stages * stage_bytes);
    const uint32_t base_s = smem_u32(base);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int C = PAIR ? 2 : a.cluster;
    const uint32_t crank = C > 1 ? cluster_ctarank() : 0u;
    const unsigned cid = bid / (unsigned)C;
    const int wtile = (int)(cid % (unsigned)a.n_wt);
    const int m0 = ((int)(cid / (unsigned)a.n_wt) * C + (int)crank) * kMTile;
    const int n_acc = a.split ? a.n_big + 1 : 1;
    const uint32_t ncols = tc_tmem_cols(n_acc * a.N);
    // bytes landing in this CTA's stage: its A rows plus the B rows it holds (the whole tile
    // when the cluster multicasts B, half of it in the pair form)
    const uint32_t tx_bytes = 2u * kABytes + 2u * (uint32_t)tc_b_rows(a.N, PAIR) * RB;
    const int rows_cta = a.N / C;                 // B rows this CTA loads (for the whole cluster)
    const uint16_t cmask = (uint16_t)((1u << C) - 1u);
    const bool leader = !PAIR || crank == 0;      // issues the MMAs
    unsigned long long *trace = a.trace ? a.trace + (size_t)bid * kTraceWords : nullptr;
    if (trace && threadIdx.x == 0) {
        trace[0] = globaltimer();
        trace[7] = smid();
    }

    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) {
            // pair form, relay: the even CTA's stage is full after its own copies AND the odd
            // CTA's relay; direct: after the copies of both CTAs (one arrival, both byte counts)
            mbar_init(smem_u32(&sh->full[s]), PAIR && leader && a.pair == 1 ? 2u : 1u);
            // one release per CTA of a multicast cluster; the pair's MMAs release both CTAs at once
            mbar_init(smem_u32(&sh->empty[s]), PAIR ? 1u : (uint32_t)C);
        }
        mbar_init(smem_u32(&sh->tmem_full), 1);
        sh->abort_flag = 0;
        fence_mbar_init();
    }
    if (PAIR) cluster_sync();   // the peer's barriers exist before the collective allocation
    if (warp == 1) {
        if (PAIR) {
            tmem_alloc2(smem_u32(&sh->tmem_addr), ncols);
            tmem_relinquish2();
        } else {
            tmem_alloc(smem_u32(&sh->tmem_addr), ncols);
            tmem_relinquish();
        }
    }
    tc_fence_before();
    __syncthreads();
    if (C > 1) cluster_sync();   // every CTA's barriers exist before any multicast reaches them
    tc_fence_after();
    const uint32_t tmem = sh->tmem_addr;
    volatile int *abort_flag = &sh->abort_flag;
    if (trace && threadIdx.x == 0) trace[1] = globaltimer();

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            // operand A streams from HBM: prefetch its boxes into L2 ahead of the ring so that
            // the ring's loads hit L2 (the twiddle rows are shared by all CTAs and stay in L2)
            const int pf_dist = a.prefetch;
            for (int kb = 0; kb < pf_dist && kb < a.n_kb; ++kb) {
                tma_prefetch_3d(&maps.a_hi, 0, m0, kb);
                tma_prefetch_3d(&maps.a_lo, 0, m0, kb);
            }
            int s_ring = -1;       // ring slot and use of staging block kb (no divisions)
            uint32_t u_ring = 0;
            for (int kb = 0; kb < a.n_kb; ++kb) {
                if (++s_ring == a.stages) {
                    s_ring = 0;
                    ++u_ring;
                }
                const int s = s_ring;
                const uint32_t use = u_ring;
                if (!mbar_wait(smem_u32(&sh->empty[s]), (use & 1u) ^ 1u, abort_flag)) {
                    if (!*abort_flag) atomicOr(a.err, DEVERR_TIMEOUT_EMPTY);
                    *abort_flag = 1;
                    break;
                }
                const uint32_t full = smem_u32(&sh->full[s]);
                const uint32_t st = base_s + (uint32_t)s * stage_bytes;
                if (PAIR && a.pair == 2) {
                    // direct form: every copy of the pair completes on the even CTA's barrier
                    const uint32_t fb = mapa_shared(full, 0u);
                    if (leader) mbar_arrive_expect_tx(full, 2u * tx_bytes);
                    tma_load_3d_pair(st, &maps.a_hi, 0, m0, kb, fb);
                    tma_load_3d_pair(st + kABytes, &maps.a_lo, 0, m0, kb, fb);
                    for (int b = 0; b < maps.nbox_b; ++b) {
                        const int row = wtile * a.N + (int)crank * rows_cta + b * maps.box_b_rows;
                        const uint32_t off = (uint32_t)(b * maps.box_b_rows) * RB;
                        tma_load_3d_pair(st + 2 * kABytes + off, &maps.b_hi, 0, row, a.kbB0 + kb, fb);
                        tma_load_3d_pair(st + 2 * kABytes + b_pad + off, &maps.b_lo, 0, row, a.kbB0 + kb, fb);
                    }
                    issued = kb + 1;
                    continue;
                }
                mbar_arrive_expect_tx(full, tx_bytes);
                tma_load_3d(st, &maps.a_hi, 0, m0, kb, full);
                tma_load_3d(st + kABytes, &maps.a_lo, 0, m0, kb, full);
                for (int b = 0; b < maps.nbox_b; ++b) {
                    const int r0 = (int)crank * rows_cta + b * maps.box_b_rows;
                    const int row = wtile * a.N + r0;
                    // multicast pieces sit at their row in every CTA; a pair CTA keeps its half at 0
                    const uint32_t off = (uint32_t)(PAIR ? b * maps.box_b_rows : r0) * RB;
                    if (PAIR) {
                        tma_load_3d(st + 2 * kABytes + off, &maps.b_hi, 0, row, a.kbB0 + kb, full);
                        tma_load_3d(st + 2 * kABytes + b_pad + off, &maps.b_lo, 0, row, a.kbB0 + kb, full);
                    } else if (C > 1) {
                        tma_load_3d_mc(st + 2 * kABytes + off, &maps.b_hi, 0, row, a.kbB0 + kb, full, cmask);
                        tma_load_3d_mc(st + 2 * kABytes + b_pad + off, &maps.b_lo, 0, row, a.kbB0 + kb, full, cmask);
                    } else {
                        tma_load_3d(st + 2 * kABytes + off, &maps.b_hi, 0, row, a.kbB0 + kb, full);
                        tma_load_3d(st + 2 * kABytes + b_pad + off, &maps.b_lo, 0, row, a.kbB0 + kb, full);
                    }
                }
                issued = kb + 1;
                if (pf_dist > 0 && kb + pf_dist < a.n_kb) {
                    tma_prefetch_3d(&maps.a_hi, 0, m0, kb + pf_dist);
                    tma_prefetch_3d(&maps.a_lo, 0, m0, kb + pf_dist);
                }
            }
            if (*abort_flag && PAIR && a.pair == 2 && !leader) {
                // this CTA's copies complete on the peer's barriers: give those in flight time
                // to land before the CTA can exit
                const uint64_t t0 = globaltimer();
                while (globaltimer() - t0 < 50000ull) {
                }
            } else if (*abort_flag) {
                // let every copy into this CTA's ring land before it can exit
                const int first = issued > a.stages ? issued - a.stages : 0;
                for (int kb = first; kb < issued; ++kb) {
                    const int s = kb % a.stages;
                    if (!mbar_wait(smem_u32(&sh->full[s]), (uint32_t)(kb / a.stages) & 1u, nullptr))
                        atomicOr(a.err, DEVERR_TIMEOUT_DRAIN);
                }
            } else if (C > 1) {
                // every CTA of the cluster releases every slot of this CTA's ring by a remote
                // arrive; wait until the releases of the last use of each slot have landed, so
                // that none can reach this shared memory after the CTA has exited
                for (int s = 0; s < a.stages && s < a.n_kb; ++s) {
                    const int last = (a.n_kb - 1 - s) / a.stages;
                    if (!mbar_wait(smem_u32(&sh->empty[s]), (uint32_t)last & 1u, nullptr))
                        atomicOr(a.err, DEVERR_TIMEOUT_DRAIN);
                }
            }
        }
    } else if (warp == 1 && PAIR && !leader) {
        if (lane == 0 && a.pair == 1) {
            // relay: each stage of this CTA is complete -> one arrival on the even CTA's barrier
            int s_ring = -1;
            uint32_t u_ring = 0;
            for (int kb = 0; kb < a.n_kb; ++kb) {
                if (++s_ring == a.stages) {
                    s_ring = 0;
                    ++u_ring;
                }
                const int s = s_ring;
                if (!mbar_wait(smem_u32(&sh->full[s]), u_ring & 1u, abort_flag)) {
                    if (!*abort_flag) atomicOr(a.err, DEVERR_TIMEOUT_FULL);
                    *abort_flag = 1;
                    break;
                }
                if (trace && kb == 0) trace[2] = globaltimer();
                mbar_arrive_remote(mapa_shared(smem_u32(&sh->full[s]), 0u));
            }
            if (trace) trace[3] = globaltimer();
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const int n0 = a.N < 256 ? a.N : 256;
            const int n1 = a.N - n0;
            const int m_mma = PAIR ? 2 * kMTile : kMTile;
            const uint32_t id0 = idesc_f32acc(m_mma, n0, a.f16);
            const uint32_t id1 = n1 > 0 ? idesc_f32acc(m_mma, n1, a.f16) : 0u;
            const uint64_t b_half_off = (uint64_t)((n0 * RB) >> 4);
            const uint32_t acc_small = tmem + (uint32_t)(a.n_big * a.N);
            const int ksteps = a.bf / 8;
            int s_ring = -1;       // ring slot and use of staging block kb (no divisions)
            uint32_t u_ring = 0;
            for (int kb = 0; kb < a.n_kb; ++kb) {
                if (++s_ring == a.stages) {
                    s_ring = 0;
                    ++u_ring;
                }
                const int s = s_ring;
                const uint32_t use = u_ring;
                const bool got = PAIR ? mbar_wait_cluster(smem_u32(&sh->full[s]), use & 1u, abort_flag)
                                      : mbar_wait(smem_u32(&sh->full[s]), use & 1u, abort_flag);
                if (!got) {
                    if (!*abort_flag) atomicOr(a.err, DEVERR_TIMEOUT_FULL);
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                if (trace && kb == 0) trace[2] = globaltimer();
                const uint32_t st = base_s + (uint32_t)s * stage_bytes;
                const uint64_t dAhi0 = sdesc_k(st, RB);
                const uint64_t dAlo0 = sdesc_k(st + kABytes, RB);
                const uint64_t dBhi0 = sdesc_k(st + 2 * kABytes, RB);
                const uint64_t dBlo0 = sdesc_k(st + 2 * kABytes + b_pad, RB);
                for (int ks = 0; ks < ksteps; ++ks) {
                    // K-step ks starts 32*ks bytes into the swizzled rows (start address in 16 B units)
                    const uint64_t adv = (uint64_t)(2 * ks);
                    const uint64_t dAhi = dAhi0 + adv, dAlo = dAlo0 + adv, dBhi = dBhi0 + adv, dBlo = dBlo0 + adv;
                    const int g = kb * ksteps + ks;       // global K-step index
                    if (PAIR) {
                        // N <= 256 (host-checked); the even CTA's descriptors address both CTAs
                        if (a.split) {
                            const int big = a.n_big == 2 ? (g & 1) : 0;
                            mma2_bf16_ss(tmem + (uint32_t)(big * a.N), dAhi, dBhi, id0, g >= a.n_big ? 1u : 0u);
                            mma2_bf16_ss(acc_small, dAhi, dBlo, id0, g > 0 ? 1u : 0u);
                            mma2_bf16_ss(acc_small, dAlo, dBhi, id0, 1u);
                        } else {
                            mma2_bf16_ss(tmem, dAhi, dBhi, id0, g > 0 ? 1u : 0u);
                            mma2_bf16_ss(tmem, dAhi, dBlo, id0, 1u);
                            mma2_bf16_ss(tmem, dAlo, dBhi, id0, 1u);
                        }
                    } else if (a.split) {
                        // N <= 256: one MMA per product
                        const int big = a.n_big == 2 ? (g & 1) : 0;
                        mma_bf16_ss(tmem + (uint32_t)(big * a.N), dAhi, dBhi, id0, g >= a.n_big ? 1u : 0u);
                        mma_bf16_ss(acc_small, dAhi, dBlo, id0, g > 0 ? 1u : 0u);
                        mma_bf16_ss(acc_small, dAlo, dBhi, id0, 1u);
                    } else {
#pragma unroll
                        for (int pass = 0; pass < 3; ++pass) {
                            const uint64_t dA = pass == 2 ? dAlo : dAhi;
                            const uint64_t dB = pass == 1 ? dBlo : dBhi;
                            const uint32_t acc = (g > 0 || pass > 0) ? 1u : 0u;
                            mma_bf16_ss(tmem, dA, dB, id0, acc);
                            if (n1 > 0) mma_bf16_ss(tmem + (uint32_t)n0, dA, dB + b_half_off, id1, acc);
                        }
                    }
                }
                if (PAIR)
                    mma2_commit_mc(smem_u32(&sh->empty[s]), cmask);
                else if (C > 1)
                    mma_commit_mc(smem_u32(&sh->empty[s]), cmask);
                else
                    mma_commit(smem_u32(&sh->empty[s]));
            }
            // always signal: the epilogue (and TMEM release) wait for every issued MMA
            if (PAIR)
                mma2_commit_mc(smem_u32(&sh->tmem_full), cmask);
            else
                mma_commit(smem_u32(&sh->tmem_full));
            if (trace) trace[3] = globaltimer();
        }
    } else {
        // epilogue warps 2..5 -> TMEM lane quarter q = warp % 4
        const int q = warp & 3;
        {
            // while the main loop runs: stage this tile's per-energy constants in shared memory
            const int jb = wtile * a.wt;
            for (int i = threadIdx.x - 64; i < a.wt; i += 128) {
                const int j = jb + i;
                sh->W[i] = j < a.e.Nw ? __ldg(a.e.Wc + j) : make_float2(0.f, 0.f);
                sh->bose[i] = j < a.e.Nw ? __ldg(a.e.bose + j) : 0.f;
            }
            asm volatile("bar.sync 1, 128;" ::: "memory");   // the four epilogue warps only
        }
        const bool ok = mbar_wait(smem_u32(&sh->tmem_full), 0u, nullptr);
        if (!ok) {
            atomicOr(a.err, DEVERR_TIMEOUT_TMEM);
            *abort_flag = 1;
        }
        tc_fence_after();
        if (trace && warp == 2 && lane == 0) trace[4] = globaltimer();
        if (ok && !*abort_flag) {
            const int64_t m = (int64_t)m0 + q * 32 + lane;
            const RowCtx row = make_row(a.e, m);
            const int jbase = wtile * a.wt;
            const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
            const int total_steps = a.n_kb * (a.bf / 8);
            const int n_big_used = a.split ? (total_steps < a.n_big ? total_steps : a.n_big) : 0;
            switch (epi_kind(a.e)) {
                case EPI_FINAL: tc_epilogue<EPI_FINAL>(a, sh, row, lane_base, jbase, n_big_used); break;
                case EPI_FINAL_KAHAN: tc_epilogue<EPI_FINAL_KAHAN>(a, sh, row, lane_base, jbase, n_big_used); break;
                case EPI_FINAL_FP64: tc_epilogue<EPI_FINAL_FP64>(a, sh, row, lane_base, jbase, n_big_used); break;
                case EPI_STORE_KAHAN: tc_epilogue<EPI_STORE_KAHAN>(a, sh, row, lane_base, jbase, n_big_used); break;
                case EPI_STORE_FP64: tc_epilogue<EPI_STORE_FP64>(a, sh, row, lane_base, jbase, n_big_used); break;
                case EPI_ADD_KAHAN: tc_epilogue<EPI_ADD_KAHAN>(a, sh, row, lane_base, jbase, n_big_used); break;
                default: tc_epilogue<EPI_ADD_FP64>(a, sh, row, lane_base, jbase, n_big_used); break;
            }
        }
    }
    if (trace && warp == 2 && lane == 0) trace[5] = globaltimer();
    tc_fence_before();
    __syncthreads();
    if (C > 1) cluster_sync();   // no CTA leaves while a peer may still signal its barriers
    if (warp == 1) {
        tc_fence_after();
        if (PAIR)
            tmem_dealloc2(tmem, ncols);
        else
            tmem_dealloc(tmem, ncols);
    }
    if (trace && threadIdx.x == 0) trace[6] = globaltimer();
}

__global__ void __launch_bounds__(192, 1) flush_tc_kernel(const __grid_constant__ TcGroup g) {
    flush_tc_body<false>(g);
}
__global__ void __launch_bounds__(192, 1) flush_tc_pair_kernel(const __grid_constant__ TcGroup g) {
    flush_tc_body<true>(g);
}

// --------------------------------------------------------------------------------------
// Drained form, persistent: one CTA per SM walks the tiles of all streams of the group
// (tile t of the concatenated tile lists, t = blockIdx.x, blockIdx.x + gridDim.x, ...).
//
// All three products of a tile go to one TMEM accumulator, double-buffered: the tile's K range
// is cut into chunks of drain_kb staging blocks that alternate between the two buffers (a
// buffer parity that runs on across tiles), and eight epilogue warps (two per TMEM lane
// quarter, each half of the columns) add every finished chunk into FP32 registers (round to
// nearest) while the next chunk accumulates; the last chunk of a tile goes, with the sums,
// through the flush epilogue while the next tile's first chunk accumulates.  The tensor
// core's truncating FP32 accumulation thus spans one chunk instead of the segment, tiles keep
// the full width of one accumulator (up to 256 columns), and neither the operand fill nor the
// epilogue of a tile is exposed.
//
//   warp 0     TMA producer over the ring (a stage counter running across tiles)
//   warp 1     TMEM allocation and MMA issue (one thread); commits release stages and mark
//              finished chunks
//   warps 2-9  drains and epilogues
// The shared-memory ring and the two TMEM buffers are laid out for the widest tile of the group.
// 320 threads: warps are spread over the SM's four register files, three on two of them, so a
// thread may hold at most 16384 / (3 * 32) = 170 registers (168 allocatable).
__device__ __forceinline__ int group_entry(const TcGroup &g, int64_t tile) {
    int gi = 0;
    while (gi + 1 < g.n && tile >= (int64_t)g.e[gi + 1].cta_begin) ++gi;
    return gi;
}

// FORM 2 (split): hi*hi goes to accumulator H, the small products hi*lo + lo*hi to S (TMEM
// columns 256 on).  Only H is drained, every chunk, into the FP32 registers (the small terms
// carry ~2^-8 of the magnitude, so their truncation stays far below the bound); at the end of
// a tile the last chunk of H and all of S are added to the registers and both accumulators
// are released at once, the flush epilogue then runs from registers while the next tile
// accumulates.  The MMA thread issues a stage's small products before it waits for H to be
// drained, so the tensor core has work while the epilogue warps empty H.
template <int FORM>
__device__ __forceinline__ void flush_tc_drain_body(const TcGroup &g) {
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
    const uint32_t ncols = FORM == 2 ? 512u : tc_tmem_cols(2 * n_max);
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
    if (trace && threadIdx.x == 0) trace[1] = globaltimer();

    // Ring position: slot s and its use parity advance by one per staging block, across tiles
    // (no divisions in the issue loops: the single MMA thread's loop sits on the critical path).
    if (warp == 0) {
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;                          // parity of the current use of slot s
            int issued = 0;                           // copies in flight that may still land
            int64_t pass = 0;
            for (int64_t t = blockIdx.x; t < n_tiles && !*abort_flag; t += gridDim.x, ++pass) {
                const int gi = group_entry(g, t);
                const TcGroupEntry &en = g.e[gi];
                const int64_t lt = t - en.cta_begin;
                const int wtile = wtile_of(lt, en.args.n_wt, g.rot, pass);
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
                    if (!mbar_wait(smem_u32(&sh->empty[s]), ph ^ 1u, abort_flag)) {
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
                    bulk_load(st + 2 * kABytes, pBhi, (uint32_t)Nt * RB, full);
                    bulk_load(st + 2 * kABytes + b_pad, pBlo, (uint32_t)Nt * RB, full);
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
    } else if (warp == 1 && FORM == 2) {
        if (lane == 0) {
            const int ksteps = bf / 8;
            int s = 0;
            uint32_t ph = 0;
            uint32_t hph = 0, tph = 0;                // parities of the H drain and tile release
            int64_t tiles = 0, chunks = 0;
            bool stop = false;
            const uint32_t accH = tmem, accS = tmem + 256u;
            for (int64_t t = blockIdx.x; t < n_tiles && !stop; t += gridDim.x, ++tiles) {
                const TcGroupEntry &en = g.e[group_entry(g, t)];
                const bool last_w = en.args.N_last > 0 &&
                                    wtile_of(t - en.cta_begin, en.args.n_wt, g.rot, tiles) == en.args.n_wt - 1;
                const int N = last_w ? en.args.N_last : en.args.N, n_kb = en.args.n_kb, cb = en.args.drain_kb;
                const uint32_t id = idesc_f32acc(kMTile, N, en.args.f16);
                if (tiles > 0) {
                    // the previous tile's H and S must be in registers before they are reused
                    if (!mbar_wait(smem_u32(&sh->chunk_free[1]), tph, abort_flag)) {
                        if (!*abort_flag) atomicOr(err, DEVERR_TIMEOUT_TMEM);
                        *abort_flag = 1;
                        break;
                    }
                    tph ^= 1u;
                    tc_fence_after();
                }
                int kc = 0;                           // staging block inside the chunk
                for (int kb = 0; kb < n_kb; ++kb) {
                    if (!mbar_wait(smem_u32(&sh->full[s]), ph, abort_flag)) {
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
                        if (!mbar_wait(smem_u32(&sh->chunk_free[0]), hph, abort_flag)) {
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
    } else if (warp == 1) {
        if (lane == 0) {
            const int ksteps = bf / 8;
            int s = 0;
            uint32_t ph = 0;
            int buf = 0;                              // accumulator buffer of the current chunk
            uint32_t fph = 0u;                        // bit b: parity of buffer b's next release
            int64_t tiles = 0, chunks = 0;            // chunks started by this CTA
            bool stop = false;
            for (int64_t t = blockIdx.x; t < n_tiles && !stop; t += gridDim.x, ++tiles) {
                const TcGroupEntry &en = g.e[group_entry(g, t)];
                const int N = en.args.N, n_kb = en.args.n_kb, cb = en.args.drain_kb;   // form 1: full tiles
                const uint32_t id = idesc_f32acc(kMTile, N, en.args.f16);
                int kc = 0;
                for (int kb = 0; kb < n_kb; ++kb) {
                    if (kc == 0) {
                        if (chunks >= 2) {
                            // the buffer's previous chunk must be drained before it is overwritten
                            if (!mbar_wait(smem_u32(&sh->chunk_free[buf]), (fph >> buf) & 1u, abort_flag)) {
                                if (!*abort_flag) atomicOr(err, DEVERR_TIMEOUT_TMEM);
                                *abort_flag = 1;
                                stop = true;
                                break;
                            }
                            fph ^= 1u << buf;
                            tc_fence_after();
                        }
                        ++chunks;
                    }
                    if (!mbar_wait(smem_u32(&sh->full[s]), ph, abort_flag)) {
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
                    const uint32_t acc = tmem + (uint32_t)(buf * n_max);
                    for (int ks = 0; ks < ksteps; ++ks) {
                        const uint64_t adv = (uint64_t)(2 * ks);
                        const uint32_t first = (kc == 0 && ks == 0) ? 0u : 1u;   // a chunk starts from zero
                        mma_bf16_ss(acc, dAhi0 + adv, dBhi0 + adv, id, first);
                        mma_bf16_ss(acc, dAhi0 + adv, dBlo0 + adv, id, 1u);
                        mma_bf16_ss(acc, dAlo0 + adv, dBhi0 + adv, id, 1u);
                    }
                    mma_commit(smem_u32(&sh->empty[s]));
                    if (++s == stages) {
                        s = 0;
                        ph ^= 1u;
                    }
                    if (++kc == cb || kb == n_kb - 1) {
                        mma_commit(smem_u32(&sh->chunk_full[buf]));
                        kc = 0;
                        buf ^= 1;
                    }
                }
            }
            mma_commit(smem_u32(&sh->tmem_full));   // always: nothing writes TMEM after this
            if (trace) {
                trace[3] = globaltimer();
                trace[4] = (unsigned long long)tiles;
                trace[5] = (unsigned long long)chunks;
            }
        }
    } else if (FORM == 2) {
        // epilogue warps 2..9: TMEM lane quarter q4 = warp % 4, column half h
        const int q4 = warp & 3, h = (warp - 2) >> 2;
        float sum[kDrainCols];
        int64_t hc = 0, tiles = 0;                    // H drains done, tiles done
        bool ok = true;
        for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, ++tiles) {
            const TcGroupEntry &en = g.e[group_entry(g, t)];
            const TcPlanArgs &a = en.args;
            const int64_t lt = t - en.cta_begin;
            const int wtile = wtile_of(lt, a.n_wt, g.rot, tiles);
            const int m0 = (int)(lt / a.n_wt) * kMTile;
            // N / 2 columns per thread (the last energy tile may be narrower)
            const int cols = ((wtile == a.n_wt - 1 && a.N_last > 0) ? a.N_last : a.N) / 2;
            const int col0 = h * cols;
            const uint32_t lane_base = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)col0;
            const int n_chunks = (a.n_kb + a.drain_kb - 1) / a.drain_kb;
#pragma unroll
            for (int i = 0; i < kDrainCols; ++i) sum[i] = 0.f;
            for (int lc = 0; lc + 1 < n_chunks; ++lc, ++hc) {
                if (!mbar_wait(smem_u32(&sh->chunk_full[0]), (uint32_t)(hc & 1), abort_flag)) {
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
            if (!mbar_wait(smem_u32(&sh->chunk_full[1]), (uint32_t)(tiles & 1), abort_flag)) {
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
            switch (epi_kind(a.e)) {
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
    } else {
        // epilogue warps 2..9: TMEM lane quarter q4 = warp % 4, column half h
        const int q4 = warp & 3, h = (warp - 2) >> 2;
        float sum[kDrainCols];
        int64_t c = 0;                                // chunks consumed
        bool ok = true;
        int64_t pass = 0;
        for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, ++pass) {
            const TcGroupEntry &en = g.e[group_entry(g, t)];
            const TcPlanArgs &a = en.args;
            const int64_t lt = t - en.cta_begin;
            const int wtile = wtile_of(lt, a.n_wt, g.rot, pass);
            const int m0 = (int)(lt / a.n_wt) * kMTile;
            const int cols = a.wt;                    // N / 2 columns per thread (form 1: full tiles)
            const int col0 = h * cols;
            const uint32_t lane_base = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)col0;
            const int n_chunks = (a.n_kb + a.drain_kb - 1) / a.drain_kb;
#pragma unroll
            for (int i = 0; i < kDrainCols; ++i) sum[i] = 0.f;
            for (int lc = 0; lc < n_chunks; ++lc, ++c) {
                const int buf = (int)(c & 1);
                if (!mbar_wait(smem_u32(&sh->chunk_full[buf]), (uint32_t)(c >> 1) & 1u, abort_flag)) {
                    if (!*abort_flag) atomicOr(err, DEVERR_TIMEOUT_TMEM);
                    *abort_flag = 1;
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tl = lane_base + (uint32_t)(buf * n_max);
                if (lc + 1 < n_chunks) {
                    drain_add(sum, tl, cols);
                } else {
                    const RowCtx row = make_row(a.e, (int64_t)m0 + q4 * 32 + lane);
                    const int jbase = wtile * a.wt;
                    switch (epi_kind(a.e)) {
                        case EPI_FINAL: tc_epilogue_drained<EPI_FINAL>(a, row, tl, col0, cols, jbase, sum); break;
                        case EPI_FINAL_KAHAN: tc_epilogue_drained<EPI_FINAL_KAHAN>(a, row, tl, col0, cols, jbase, sum); break;
                        case EPI_FINAL_FP64: tc_epilogue_drained<EPI_FINAL_FP64>(a, row, tl, col0, cols, jbase, sum); break;
                        case EPI_STORE_KAHAN: tc_epilogue_drained<EPI_STORE_KAHAN>(a, row, tl, col0, cols, jbase, sum); break;
                        case EPI_STORE_FP64: tc_epilogue_drained<EPI_STORE_FP64>(a, row, tl, col0, cols, jbase, sum); break;
                        case EPI_ADD_KAHAN: tc_epilogue_drained<EPI_ADD_KAHAN>(a, row, tl, col0, cols, jbase, sum); break;
                        default: tc_epilogue_drained<EPI_ADD_FP64>(a, row, tl, col0, cols, jbase, sum); break;
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&sh->chunk_free[buf]));
            }
        }
        // always wait (bounded) for the last commit: no MMA may still write TMEM at release
        if (!mbar_wait(smem_u32(&sh->tmem_full), 0u, nullptr)) atomicOr(err, DEVERR_TIMEOUT_TMEM);
        tc_fence_after();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, ncols);
    }
    if (trace && threadIdx.x == 0) trace[6] = globaltimer();
}

__global__ void __maxnreg__(168) flush_tc_drain_kernel(const __grid_constant__ TcGroup g) {
    flush_tc_drain_body<1>(g);
}
__global__ void __maxnreg__(168) flush_tc_drain2_kernel(const __grid_constant__ TcGroup g) {
    flush_tc_drain_body<2>(g);
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
                                         volatile int *abort_flag) {
    const TcPlanArgs &a = g.a;
    const TcDirectArgs &d = g.d;
    const int lane = threadIdx.x & 31;
    if (!mbar_wait_warp(smem_u32(&sh->sums_full[cnt & 1]), (uint32_t)((cnt >> 1) & 1), abort_flag) ||
        !mbar_wait_warp(smem_u32(&sh->chunk_full[1]), (uint32_t)(cnt & 1), abort_flag)) {
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
                if (!mbar_wait_warp(smem_u32(&sh->raw_empty[r]), rph ^ 1u, abort_flag)) {
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
            bool stop = false;
            for (int64_t t = blockIdx.x; t < n_tiles && !stop; t += gridDim.x) {
                const int wtile = (int)(t % a.n_wt);
                const uint8_t *pBhi = static_cast<const uint8_t *>(a.B_hi) +
                                      ((size_t)a.kbB0 * (size_t)a.b_rows + (size_t)wtile * N) * RB;
                const uint8_t *pBlo = static_cast<const uint8_t *>(a.B_lo) +
                                      ((size_t)a.kbB0 * (size_t)a.b_rows + (size_t)wtile * N) * RB;
                for (int kb = 0; kb < a.n_kb; ++kb) {
                    if (!mbar_wait(smem_u32(&sh->empty[s]), ph ^ 1u, abort_flag)) {
                        if (!*abort_flag) atomicOr(a.err, DEVERR_TIMEOUT_EMPTY);
                        *abort_flag = 1;
                        stop = true;
                        break;
                    }
                    const uint32_t full = smem_u32(&sh->full[s]);
                    const uint32_t st = base_s + (uint32_t)s * b_stage;
                    mbar_arrive_expect_tx(full, tx_b);
                    bulk_load(st, pBhi + (size_t)kb * b_step, (uint32_t)N * RB, full);
                    bulk_load(st + b_pad, pBlo + (size_t)kb * b_step, (uint32_t)N * RB, full);
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
                    if (!mbar_wait(smem_u32(&sh->chunk_free[1]), tph, abort_flag)) {
                        if (!*abort_flag) atomicOr(a.err, DEVERR_TIMEOUT_TMEM);
                        *abort_flag = 1;
                        break;
                    }
                    tph ^= 1u;
                    tc_fence_after();
                }
                int kc = 0;
                for (int kb = 0; kb < a.n_kb; ++kb) {
                    if (!mbar_wait(smem_u32(&sh->full[s]), ph, abort_flag)) {
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
                        if (!mbar_wait(smem_u32(&sh->chunk_free[0]), hph, abort_flag)) {
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
                if (!mbar_wait_warp(smem_u32(&sh->raw_full[r]), rph, abort_flag) ||
                    !mbar_wait_warp(smem_u32(&sh->empty[s]), ph ^ 1u, abort_flag)) {
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
                if (!ip_final<KIND>(g, sh, sum, fin_t, fin_cnt, h, rr, hbase, sbase, abort_flag)) break;
                fin_t = -1;
            }
            if (!have) break;
            // the H chunk that ended with block kb - 1 (drained one block late, so this block's
            // small products run on the tensor pipe meanwhile)
            if (kb >= 1 && kb % cb == 0) {
                if (!mbar_wait_warp(smem_u32(&sh->chunk_full[0]), (uint32_t)(hc & 1), abort_flag)) {
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
// In-place variant: operand A is read from the caller's pushed complex64 frames.
//
//   warps 0-3   A producers: thread r owns tile row r; per staging block it loads the row's bf
//               frames (coalesced 8-byte loads across the warp, through a per-frame pointer
//               table), subtracts the provisional mean, splits into bf16 hi/lo and writes the
//               16-byte chunks of the swizzled K-major rows (128/64/32-byte swizzle pattern of
//               the row width); fence.proxy.async makes them visible to the tensor core before
//               the thread arrives on the stage barrier.  Each row's residual sum is kept: the
//               CTA's epilogue derives the exact mean correction from it (and earlier flushes'
//               sums), and the first energy tile adds it to the running sums for later flushes.
//   warp 4      B producer (TMA of this CTA's twiddle rows)
//   warp 5      TMEM allocator + MMA issuer
//   warps 6..9  epilogue
// --------------------------------------------------------------------------------------
__global__ void __launch_bounds__(320, 1) flush_tc_direct_kernel(const __grid_constant__ TcMaps maps,
                                                                 const TcPlanArgs a, const TcDirectArgs d) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t RB = 4u * (uint32_t)a.bf;
    const uint32_t kABytes = tc_a_bytes(a.bf);
    const uint32_t b_pad = tc_b_bytes_padded(a.N, a.bf);
    const uint32_t stage_bytes = tc_stage_bytes(a.N, a.bf);
    TcShared *sh = reinterpret_cast<TcShared *>(base + (size_t)a.stages * stage_bytes);
    const uint32_t base_s = smem_u32(base);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wtile = (int)(blockIdx.x % (unsigned)a.n_wt);
    const int m0 = (int)(blockIdx.x / (unsigned)a.n_wt) * kMTile;
    const int n_acc = a.split ? a.n_big + 1 : 1;
    const uint32_t ncols = tc_tmem_cols(n_acc * a.N);
    const uint32_t tx_bytes_b = 2u * (uint32_t)a.N * RB;
    unsigned long long *trace = a.trace ? a.trace + (size_t)blockIdx.x * kTraceWords : nullptr;
    if (trace && threadIdx.x == 0) {
        trace[0] = globaltimer();
        trace[7] = smid();
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(smem_u32(&sh->full[s]), kMTile + 1);   // 128 A rows + the B producer
            mbar_init(smem_u32(&sh->empty[s]), 1);
        }
        mbar_init(smem_u32(&sh->tmem_full), 1);
        mbar_init(smem_u32(&sh->sums_ready), kMTile);
        sh->abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 5) {
        tmem_alloc(smem_u32(&sh->tmem_addr), ncols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tmem_addr;
    volatile int *abort_flag = &sh->abort_flag;
    if (trace && threadIdx.x == 0) trace[1] = globaltimer();

    if (warp < 4) {
        // ---------------- A producers ----------------
        const int r = threadIdx.x;
        const int64_t m = (int64_t)m0 + r;
        const bool valid = m < d.M;
        int64_t off = 0;
        float2 mu = make_float2(0.f, 0.f);
        if (valid) {
            const int64_t p = m / d.npix, pix = m - (m / d.npix) * d.npix;
            const int64_t y = pix / d.kx, x = pix - (pix / d.kx) * d.kx;
            off = p * d.pitch_probe + (d.roi_y0 + y) * d.pitch_row + (d.roi_x0 + x);
            mu = d.mu_hat[m];
        }
        const int cpr = a.bf / 4;                                   // 16-byte chunks per row
        const uint32_t row_byte = (uint32_t)r * RB;
        const uint32_t sw = (row_byte >> 7) & (uint32_t)(cpr - 1);  // swizzle phase of this row
        double sr = 0.0, si = 0.0;
        bool ok = true;
        int s_ring = -1;           // ring slot and use of staging block kb (no divisions)
        uint32_t u_ring = 0;
        for (int kb = 0; kb < a.n_kb && ok; ++kb) {
            if (++s_ring == a.stages) {
                s_ring = 0;
                ++u_ring;
            }
            const int s = s_ring;
            const uint32_t use = u_ring;
            if (!mbar_wait(smem_u32(&sh->empty[s]), (use & 1u) ^ 1u, abort_flag)) {
                if (!*abort_flag) atomicOr(a.err, DEVERR_TIMEOUT_EMPTY);
                *abort_flag = 1;
                ok = false;
                break;
            }
            uint8_t *st = base + (size_t)s * stage_bytes;
            const int f0 = kb * a.bf;
            // all of the block's loads in flight at once (independent pointer + data loads)
            float2 v[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const int f = f0 + i;
                v[i] = (i < a.bf && valid && f < d.n_frames) ? __ldcs(d.frame_ptr[f] + off) : mu;
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                if (c < cpr) {
                    uint32_t h[4], l[4];
                    float br = 0.f, bi = 0.f;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float2 q = make_float2(v[4 * c + i].x - mu.x, v[4 * c + i].y - mu.y);
                        br += q.x;
                        bi += q.y;
                        split2_bf16(q, h[i], l[i]);
                    }
                    sr += br;
                    si += bi;
                    const uint32_t chunk = ((uint32_t)c ^ sw) * 16u;
                    *reinterpret_cast<uint4 *>(st + row_byte + chunk) = make_uint4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<uint4 *>(st + kABytes + row_byte + chunk) = make_uint4(l[0], l[1], l[2], l[3]);
                }
            }
            // generic-proxy writes -> visible to the tensor core (async proxy) before the arrive
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(smem_u32(&sh->full[s]));
        }
        // this flush's residual sums: to the epilogue, and (first energy tile) to the running sums
        sh->rowsum[r] = make_double2(sr, si);
        if (valid && wtile == 0 && d.accumulate_sums) {
            double2 t = d.sum_res[m];
            t.x += sr;
            t.y += si;
            d.sum_res[m] = t;
        }
        mbar_arrive(smem_u32(&sh->sums_ready));
    } else if (warp == 4) {
        // ---------------- B producer ----------------
        if (lane == 0) {
            int s_ring = -1;       // ring slot and use of staging block kb (no divisions)
            uint32_t u_ring = 0;
            for (int kb = 0; kb < a.n_kb; ++kb) {
                if (++s_ring == a.stages) {
                    s_ring = 0;
                    ++u_ring;
                }
                const int s = s_ring;
                const uint32_t use = u_ring;
                if (!mbar_wait(smem_u32(&sh->empty[s]), (use & 1u) ^ 1u, abort_flag)) {
                    if (!*abort_flag) atomicOr(a.err, DEVERR_TIMEOUT_EMPTY);
                    *abort_flag = 1;
                    break;
                }
                const uint32_t full = smem_u32(&sh->full[s]);
                const uint32_t st = base_s + (uint32_t)s * stage_bytes;
                mbar_arrive_expect_tx(full, tx_bytes_b);
                for (int b = 0; b < maps.nbox_b; ++b) {
                    const int r0 = b * maps.box_b_rows;
                    const uint32_t off = (uint32_t)r0 * RB;
                    tma_load_3d(st + 2 * kABytes + off, &maps.b_hi, 0, wtile * a.N + r0, a.kbB0 + kb, full);
                    tma_load_3d(st + 2 * kABytes + b_pad + off, &maps.b_lo, 0, wtile * a.N + r0, a.kbB0 + kb, full);
                }
            }
        }
    } else if (warp == 5) {
        if (lane == 0) tc_mma_loop(a, sh, base_s, stage_bytes, kABytes, b_pad, RB, tmem, abort_flag, trace, false);
    } else {
        // ---------------- epilogue: warps 6..9 ----------------
        const int q = warp & 3;
        {
            const int jb = wtile * a.wt;
            for (int i = threadIdx.x - 192; i < a.wt; i += 128) {
                const int j = jb + i;
                sh->W[i] = j < a.e.Nw ? __ldg(a.e.Wc + j) : make_float2(0.f, 0.f);
                sh->bose[i] = j < a.e.Nw ? __ldg(a.e.bose + j) : 0.f;
            }
            asm volatile("bar.sync 1, 128;" ::: "memory");
        }
        const bool ok = mbar_wait(smem_u32(&sh->tmem_full), 0u, nullptr);
        if (!ok) {
            atomicOr(a.err, DEVERR_TIMEOUT_TMEM);
            *abort_flag = 1;
        }
        const bool ok2 = ok && mbar_wait(smem_u32(&sh->sums_ready), 0u, abort_flag);
        tc_fence_after();
        if (trace && warp == 6 && lane == 0) trace[4] = globaltimer();
        if (ok2 && !*abort_flag) {
            const int rr = q * 32 + lane;
            const int64_t m = (int64_t)m0 + rr;
            RowCtx row;
            row.m = m;
            row.valid = m < d.M;
            const int64_t p = row.valid ? m / d.npix : 0;
            row.out_base = p * (int64_t)a.e.Nw * d.npix + (m - p * d.npix);
            row.dmu = make_float2(0.f, 0.f);
            if (row.valid && d.subtract_mean && a.e.mode == FLUSH_FINAL) {
                double2 t = sh->rowsum[rr];
                if (d.prev_sums) {
                    const double2 pv = d.sum_res[m];
                    t.x += pv.x;
                    t.y += pv.y;
                }
                row.dmu = make_float2((float)(t.x / d.T), (float)(t.y / d.T));
            }
            const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
            const int total_steps = a.n_kb * (a.bf / 8);
            const int n_big_used = a.split ? (total_steps < a.n_big ? total_steps : a.n_big) : 0;
            const int jbase = wtile * a.wt;
            switch (epi_kind(a.e)) {
                case EPI_FINAL: tc_epilogue<EPI_FINAL>(a, sh, row, lane_base, jbase, n_big_used); break;
                case EPI_FINAL_KAHAN: tc_epilogue<EPI_FINAL_KAHAN>(a, sh, row, lane_base, jbase, n_big_used); break;
                case EPI_FINAL_FP64: tc_epilogue<EPI_FINAL_FP64>(a, sh, row, lane_base, jbase, n_big_used); break;
                case EPI_STORE_KAHAN: tc_epilogue<EPI_STORE_KAHAN>(a, sh, row, lane_base, jbase, n_big_used); break;
                case EPI_STORE_FP64: tc_epilogue<EPI_STORE_FP64>(a, sh, row, lane_base, jbase, n_big_used); break;
                case EPI_ADD_KAHAN: tc_epilogue<EPI_ADD_KAHAN>(a, sh, row, lane_base, jbase, n_big_used); break;
                default: tc_epilogue<EPI_ADD_FP64>(a, sh, row, lane_base, jbase, n_big_used); break;
            }
        }
        if (trace && warp == 6 && lane == 0) trace[5] = globaltimer();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 5) {
        tc_fence_after();
        tmem_dealloc(tmem, ncols);
    }
    if (trace && threadIdx.x == 0) trace[6] = globaltimer();
}

// --------------------------------------------------------------------------------------
// host side
// --------------------------------------------------------------------------------------
int tc_stages_for(int N, int bf, int pair) {
    const int budget = kSmemLimit - 1024 - (int)sizeof(TcShared);
    int s = budget / (int)tc_stage_bytes(N, bf, pair);
    if (s > kMaxStages) s = kMaxStages;
    return s;
}

size_t tc_smem_bytes(int N, int bf, int stages, int pair) {
    return (size_t)stages * tc_stage_bytes(N, bf, pair) + sizeof(TcShared) + 1024;
}

size_t tc_maps_size() { return sizeof(TcMaps); }

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

static bool encode3d(CUtensorMap *m, const void *ptr, uint64_t d0, uint64_t d1, uint64_t d2, uint32_t b1,
                     char *errbuf, size_t errlen, const char *what) {
    // d0 bf16 elements per row: 16, 32 or 64 -> rows of 32, 64 or 128 bytes, swizzled alike
    const CUtensorMapSwizzle sw = d0 == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                                           : (d0 == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
    EncodeTiledFn fn = encode_fn();
    if (!fn) {
        snprintf(errbuf, errlen, "cuTensorMapEncodeTiled is not available from the driver");
        return false;
    }
    cuuint64_t dims[3] = {d0, d1, d2};
    cuuint64_t strides[2] = {d0 * 2, d0 * 2 * d1};
    cuuint32_t box[3] = {(cuuint32_t)d0, b1, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(ptr), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        snprintf(errbuf, errlen, "cuTensorMapEncodeTiled(%s) failed with %d", what, (int)r);
        return false;
    }
    return true;
}

// B rows loaded by one CTA: N / cluster, in boxes of at most 256 rows whose shared-memory
// offsets stay on 256-byte (8-row) swizzle-atom boundaries.
bool tc_b_boxes(int N, int cluster, int *box_rows, int *nbox) {
    if (cluster < 1 || N % cluster) return false;
    const int rows = N / cluster;
    if (rows % 8) return false;
    const int nb = (rows + 255) / 256;
    if (rows % nb || (rows / nb) % 8) return false;
    *box_rows = rows / nb;
    *nbox = nb;
    return true;
}

bool tc_make_maps(void *maps_out, const __nv_bfloat16 *A_hi, const __nv_bfloat16 *A_lo, int64_t M_pad,
                  int n_kb_stage, const __nv_bfloat16 *B_hi, const __nv_bfloat16 *B_lo, int Nw_pad, int n_kb_T,
                  int N, int cluster, int bf, char *errbuf, size_t errlen) {
    TcMaps *m = reinterpret_cast<TcMaps *>(maps_out);
    const uint64_t d0 = 2 * (uint64_t)bf;
    memset(m, 0, sizeof(TcMaps));
    if (!tc_b_boxes(N, cluster, &m->box_b_rows, &m->nbox_b)) {
        snprintf(errbuf, errlen, "tile of %d columns cannot be split over a cluster of %d", N, cluster);
        return false;
    }
    if (!encode3d(&m->a_hi, A_hi, d0, (uint64_t)M_pad, (uint64_t)n_kb_stage, kMTile, errbuf, errlen, "A_hi")) return false;
    if (!encode3d(&m->a_lo, A_lo, d0, (uint64_t)M_pad, (uint64_t)n_kb_stage, kMTile, errbuf, errlen, "A_lo")) return false;
    if (!encode3d(&m->b_hi, B_hi, d0, 2 * (uint64_t)Nw_pad, (uint64_t)n_kb_T, (uint32_t)m->box_b_rows, errbuf, errlen,
                  "B_hi"))
        return false;
    if (!encode3d(&m->b_lo, B_lo, d0, 2 * (uint64_t)Nw_pad, (uint64_t)n_kb_T, (uint32_t)m->box_b_rows, errbuf, errlen,
                  "B_lo"))
        return false;
    return true;
}

bool tc_make_maps_b(void *maps_out, const __nv_bfloat16 *B_hi, const __nv_bfloat16 *B_lo, int Nw_pad, int n_kb_T,
                    int N, int bf, char *errbuf, size_t errlen) {
    TcMaps *m = reinterpret_cast<TcMaps *>(maps_out);
    memset(m, 0, sizeof(TcMaps));
    if (!tc_b_boxes(N, 1, &m->box_b_rows, &m->nbox_b)) {
        snprintf(errbuf, errlen, "tile of %d columns has no valid twiddle box split", N);
        return false;
    }
    const uint64_t d0 = 2 * (uint64_t)bf;
    if (!encode3d(&m->b_hi, B_hi, d0, 2 * (uint64_t)Nw_pad, (uint64_t)n_kb_T, (uint32_t)m->box_b_rows, errbuf, errlen,
                  "B_hi"))
        return false;
    return encode3d(&m->b_lo, B_lo, d0, 2 * (uint64_t)Nw_pad, (uint64_t)n_kb_T, (uint32_t)m->box_b_rows, errbuf, errlen,
                    "B_lo");
}

size_t tc_smem_bytes_direct(int N, int bf, int stages) { return tc_smem_bytes(N, bf, stages); }

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
    kern<<<(unsigned)grid, 352, smem, st>>>(g);
    return cudaGetLastError();
}

cudaError_t launch_flush_tc_direct(const TcPlanArgs &a, const TcDirectArgs &d, const void *maps, cudaStream_t st) {
    const size_t smem = tc_smem_bytes(a.N, a.bf, a.stages);
    cudaError_t e = cudaFuncSetAttribute(flush_tc_direct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (a.e.M_pad / kMTile) * a.n_wt;
    if (blocks <= 0 || blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    flush_tc_direct_kernel<<<(unsigned)blocks, 320, smem, st>>>(*reinterpret_cast<const TcMaps *>(maps), a, d);
    return cudaGetLastError();
}

// Co-resident CTAs of the contraction kernel for a cluster size (0 on error).
int tc_resident_ctas(int N, int bf, int stages, int cluster, int pair, int drain) {
    const size_t smem = tc_smem_bytes(N, bf, stages, pair);
    auto kern = drain ? (drain == 2 ? flush_tc_drain2_kernel : flush_tc_drain_kernel)
                      : (pair ? flush_tc_pair_kernel : flush_tc_kernel);
    if (pair) cluster = 2;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster * 1024, 1, 1);
    cfg.blockDim = dim3(drain ? 320 : 192, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n * cluster;
}

int64_t tc_grid_ctas(const TcPlanArgs &a) {
    const int64_t n_mt = a.e.M_pad / kMTile;
    return (n_mt + a.cluster - 1) / a.cluster * a.cluster * a.n_wt;
}

cudaError_t launch_flush_tc_group(const TcPlanArgs *args, const void *const *maps, int n, cudaStream_t st) {
    if (n < 1 || n > kMaxGroupStreams) return cudaErrorInvalidValue;
    TcGroup *g = new (std::nothrow) TcGroup();
    if (!g) return cudaErrorMemoryAllocation;
    const int C = args[0].cluster;
    const int pair = args[0].pair;
    const bool drain = args[0].drain_kb > 0;
    const int form = args[0].drain_form == 2 ? 2 : 1;
    size_t smem = 0;
    int64_t total = 0;
    for (int i = 0; i < n; ++i) {
        // the pair form needs clusters of 2 and tiles of at most 256 columns (one MMA each);
        // the drained form one CTA per tile and two buffers of at most 256 columns
        if (args[i].cluster != C || args[i].bf != args[0].bf || args[i].pair != pair ||
            (args[i].drain_kb > 0) != drain || (drain && (args[i].drain_form == 2 ? 2 : 1) != form) ||
            (pair && (C != 2 || args[i].N > 256 || args[i].N % 32)) ||
            (drain && (C != 1 || pair || args[i].wt > kDrainCols))) {
            delete g;
            return cudaErrorInvalidValue;
        }
        g->e[i].maps = *reinterpret_cast<const TcMaps *>(maps[i]);
        g->e[i].args = args[i];
        g->e[i].cta_begin = (int)total;
        if (args[i].trace && !drain) g->e[i].args.trace = args[i].trace + (size_t)total * kTraceWords;
        const int64_t c = tc_grid_ctas(args[i]);
        g->e[i].ctas = (int)c;
        total += c;
        smem = std::max(smem, tc_smem_bytes(args[i].N, args[i].bf, args[i].stages, pair));
    }
    g->n = n;
    if (total <= 0 || total > 0x7fffffffLL) {
        delete g;
        return cudaErrorInvalidConfiguration;
    }
    unsigned grid = (unsigned)total;
    if (drain) {
        // persistent: the ring and the two TMEM buffers are sized for the widest tile; one wave
        // of CTAs walks all tiles
        int n_max = 0;
        for (int i = 0; i < n; ++i) n_max = std::max(n_max, args[i].N);
        g->n_max = n_max;
        g->stages = tc_stages_for(n_max, args[0].bf);
        g->tiles = total;
        smem = tc_smem_bytes(n_max, args[0].bf, g->stages);
        int dev = 0, sms = 0, occ = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        auto dk = form == 2 ? flush_tc_drain2_kernel : flush_tc_drain_kernel;
        if (e == cudaSuccess) e = cudaFuncSetAttribute(dk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dk, 320, smem);
        if (e != cudaSuccess || g->stages < 2 || n_max > 2 * kDrainCols || occ < 1) {
            delete g;
            return e != cudaSuccess ? e : cudaErrorInvalidConfiguration;
        }
        int64_t cap = (int64_t)occ * sms;
        if (args[0].max_ctas > 0 && args[0].max_ctas < cap) cap = args[0].max_ctas;
        if (cap < total) grid = (unsigned)cap;
        // one stream whose row of energy tiles divides the grid: rotate the energy slots
        g->rot = (n == 1 && args[0].n_wt > 1 && grid % (unsigned)args[0].n_wt == 0) ? 1 : 0;
    }
    auto kern = drain ? (form == 2 ? flush_tc_drain2_kernel : flush_tc_drain_kernel)
                      : (pair ? flush_tc_pair_kernel : flush_tc_kernel);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid, 1, 1);
        cfg.blockDim = dim3(drain ? 320 : 192, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, kern, *g);
    }
    delete g;
    return e;
}

cudaError_t launch_flush_tc(const TcPlanArgs &a, const void *maps, cudaStream_t st) {
    return launch_flush_tc_group(&a, &maps, 1, st);
}

}  // namespace tacaw
