// FP32-accurate GEMM on the 5th-generation tensor cores: C = A B with A [R x K] (rows of all
// domains stacked) and B [K x N] shared, as the split product A_hi B_hi + A_hi B_lo + A_lo B_hi of
// TF32 parts (3xTF32), accumulated in FP32 in tensor memory.
//
//   - A_hi/A_lo (blocked layout, see blk_index; R padded to whole 128-row tiles) and BT_hi/BT_lo
//     [N][ldk] (B transposed, K contiguous) are FP32 arrays whose values are TF32-representable;
//     ldk is a multiple of 32 and the padding columns are zero.
//   - One CTA computes a 128 x BN tile over the whole K range; the column tile is the fastest grid
//     index, so the CTAs that share a row tile of A run together and read it once from HBM.
//     Thread 0 issues the TMA loads (cp.async.bulk.tensor, 128-byte swizzle, 32-float K chunks),
//     thread 32 issues tcgen05.mma (kind::tf32, M = 128, N = BN, K = 8 per instruction), and the
//     epilogue warps drain TMEM (tcgen05.ld 32x32b).
//   - Stages are handed over with mbarriers (TMA complete_tx for "full", tcgen05.commit for
//     "empty").  Every wait is bounded by a clock budget; on expiry the kernel raises *err, stops
//     issuing, drains its own copies (bounded), frees TMEM and returns.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cstdint>
#include "common.cuh"

namespace tc {

constexpr int BM = 128;
constexpr int BK = 32;  // floats per K chunk: one 128-byte swizzle row
constexpr long long kWaitCycles = 4000000000ll;  // about 2 s at 2 GHz

__host__ __device__ constexpr int stage_bytes(int bn) { return 2 * BM * BK * 4 + 2 * bn * BK * 4; }
__host__ __device__ constexpr int tmem_cols(int cols) {
    return cols <= 32 ? 32 : (cols <= 64 ? 64 : (cols <= 128 ? 128 : (cols <= 256 ? 256 : 512)));
}

// Left operands (A parts) live in a blocked layout: 128-row x 32-column blocks of 16 KB, stored
// contiguously in (row tile, K chunk) order, so one TMA box is one contiguous 16 KB read and an
// epilogue's 32 x 32 sub-block is one contiguous 4 KB write.  nk = ldk / 32 chunks per row tile.
__host__ __device__ __forceinline__ int64_t blk_index(int64_t row, int k, int nk) {
    return (((row >> 7) * nk + (k >> 5)) << 12) + ((row & 127) << 5) + (k & 31);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// Test with a suspend-time hint (ns): the thread sleeps until the phase completes or the hint
// runs out instead of re-polling the barrier word in shared memory.
__device__ __forceinline__ bool mbar_try_sleep(uint64_t* bar, uint32_t parity, uint32_t ns) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}
// Bounded wait on an mbarrier phase, suspended between tests (a spinning test loop takes issue
// slots from the warps doing the work); false when `budget` SM clock cycles ran out.
__device__ __forceinline__ bool mbar_wait_for(uint64_t* bar, uint32_t parity, long long budget) {
    const long long t0 = clock64();
    while (!mbar_try_sleep(bar, parity, 100000u)) {
        if (clock64() - t0 > budget) return false;
    }
    return true;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) { return mbar_wait_for(bar, parity, kWaitCycles); }

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand in the 128-byte swizzle layout written by TMA
// (8-row groups of 128-byte rows, 1024 bytes apart).  Bits: start address >> 4 [0,14), leading
// offset >> 4 [16,30) (unused for this layout), stride offset >> 4 [32,46), version 1 [46,48),
// layout type 2 = 128-byte swizzle [61,64).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of kind::tf32: D = F32 [4,6), A = B = TF32 [7,10) [10,13), both K-major,
// N >> 3 [17,23), M >> 4 [24,29).
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// The same arrival on the mbarrier at this offset in every CTA of the cluster in cta_mask.
__device__ __forceinline__ void mma_commit_mc(uint64_t* bar, uint16_t cta_mask) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
                     smem_u32(bar)),
                 "h"(cta_mask)
                 : "memory");
}
// TMA load of one box into this shared-memory offset of every CTA of the cluster in cta_mask, each
// CTA's mbarrier at `bar`'s offset receiving the bytes that land in it.
__device__ __forceinline__ void tma_load_2d_mc(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, uint16_t cta_mask) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster [%0], [%1, {%3, %4}], [%2], %5;" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "h"(cta_mask)
        : "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_size() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
// Pair form (cta_group::2): one MMA of M = 256 on the two SMs of a CTA pair, each CTA holding its 128
// rows of A and half of B's columns in its own shared memory; each CTA's TMEM receives its 128 rows.
__device__ __forceinline__ void mma_tf32_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit_pair_mc(uint64_t* bar, uint16_t cta_mask) {
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
                     smem_u32(bar)),
                 "h"(cta_mask)
                 : "memory");
}
// Address of the same shared-memory offset in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t cluster_addr(const void* p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}
// TMA load into this CTA's shared memory whose completion is signalled on an mbarrier of either CTA
// of the pair (cluster address).
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* map, uint32_t bar_cluster, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar_cluster), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar_cluster) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster) : "memory");
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__host__ __device__ constexpr int pstages_for(int bn) { return bn >= 128 ? 3 : 4; }

__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float* v) {
    uint32_t r[64];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 64; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// TMA tensor store of one box from shared memory (bulk-group completion).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(reinterpret_cast<uint64_t>(map)),
                 "r"(smem_u32(src)), "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// Chain epilogue: the output columns are the coefficients on the activations of a hidden layer;
// instead of storing C the epilogue forms that layer's intercept partials over its column tile
// (sum pos(x) d, sum neg(x) d, sum x s b) and the next level's left operand x*s as TF32 parts.
// With W1 set (the last level of a chain, whose columns are layer 1's activations) the epilogue
// instead multiplies x*s by W1 [N][n0] in FP32 and writes per-tile partial rows of Lambda_x.
struct ChainEpi {
    const float* hs;   // [domains][hidden] slopes
    const float* hd;   // [domains][hidden] intercepts
    const float* bias; // [N] bias of the layer
    int hidden, hoff;  // row stride of hs/hd and the layer's offset
    int rows_per_dom;  // stacked rows per domain
    float* Ah;         // next left operand, TF32 parts (blocked layout, ldk columns)
    float* Al;
    int ldk;
    float* part;       // [column tiles * column groups][3][R] partial intercepts (rows contiguous)
    const float* W1;   // final level: W_1 [N][n0] (row-major), else null
    int n0;            // columns of W_1 (<= kFinalCols)
    float* lxpart;     // final level: [column tiles][n0][R] partial Lambda_x entries
    float* lev;        // keep mode: the level Lambda (before the slopes), blocked like the operands (blk_index,
                       // ru32(N) columns), or null
    // reverse chain level (EPI 3, see pp_row_epilogue_rev): the per-row intercept adjoints of the
    // target, the forward level read back, and the per-warp column sums
    const float* rklo;  // [domains][kld]
    const float* rkhi;
    int kld;
    const float* rlev;  // forward level, blocked (blk_index, ru32(N) columns); with rlev_shared the rows are row % rows_per_dom
    int rlev_shared;
    float* colpart;     // [R / 32][2][N]: sums over each warp's 32 rows of lev*g (slope) and of the intercept term
};

constexpr int kFinalCols = 16;  // widest input layer the fused final level handles
// Shared memory: pipeline stages, 256 B of barriers, the epilogue's per-column table, then (1 KB
// aligned) the final level's right operand W_1^T as TF32 parts in the 128-byte swizzle layout
// ([part][32-column chunk][kFinalCols rows][128 B]), plus 1 KB of base alignment slack.
__host__ __device__ constexpr int w1b_offset(int bn) { return (pstages_for(bn) * stage_bytes(bn) + 256 + 16 * bn + 1023) & ~1023; }
__host__ __device__ constexpr int psmem_bytes(int bn) { return w1b_offset(bn) + 2 * bn * kFinalCols * 4 + 1024; }
constexpr int kPartials = 3;  // TMEM partial buffers: the MMA issuer may run two chunks ahead of the epilogue

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Same contraction with promoted accumulation: every 32-wide K chunk is accumulated in a fresh
// TMEM buffer (three buffers, round robin) and the four epilogue warps add the chunk partials into
// FP32 registers, one output row per thread.  The tensor core then never accumulates more than one
// chunk (12 MMAs), and the long sum over K runs in IEEE FP32 adds, which keeps the 3xTF32 product
// as accurate as an FP32 SGEMM.  BN <= 128 (a thread holds BN partial sums).
// Warp roles: warp 0 lane 0 = TMA producer, warp 1 = TMEM owner and (lane 0) MMA issuer, warps
// 2.. = epilogue, in EG groups of four warps (EG = 2 for BN >= 64: two warps per TMEM lane
// quadrant, each with half of the tile's columns, so each thread holds BN / EG partial sums).
__host__ __device__ constexpr int epi_groups(int bn) { return bn >= 64 ? 2 : 1; }
__host__ __device__ constexpr int gemm_threads(int bn) { return 64 + 128 * epi_groups(bn); }
template <int EG>
__device__ __forceinline__ void epi_bar() {
    if constexpr (EG == 2) asm volatile("bar.sync 1, 256;" ::: "memory");
    else asm volatile("bar.sync 1, 128;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ float tf32_part_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// EPI: 0 = store C, 1 = chain level (next operand by TMA), 2 = final chain level (W_1 product).
template <int BN, int EPI>
__global__ void __launch_bounds__(gemm_threads(BN), 1) k_tc_gemm_p(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
                                                      const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
                                                      const __grid_constant__ CUtensorMap mOh, const __grid_constant__ CUtensorMap mOl,
                                                      float* __restrict__ C, int R, int K, int N, int ldc, int* __restrict__ err,
                                                      const ChainEpi epi) {
    static_assert(BN <= 128, "promoted accumulation keeps BN partial sums per thread");
    constexpr int S = pstages_for(BN);
    constexpr int SB = stage_bytes(BN);
    constexpr int PB = BN < 32 ? 32 : BN;  // TMEM columns per partial buffer (32-column loads stay inside)
    constexpr int NP = kPartials;
    constexpr int EG = epi_groups(BN);
    constexpr int BNH = BN / EG;
    constexpr int TC = tmem_cols(NP * PB);
    constexpr uint32_t IDESC = idesc_tf32(BM, BN);
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(base + S * SB);
    uint64_t* empty = full + S;
    uint64_t* pfull = empty + S;   // [NP] partial ready (MMA commit)
    uint64_t* pfree = pfull + NP;  // [NP] partial consumed (4 epilogue warps)
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(pfree + NP + 1);
    int* abort_flag = reinterpret_cast<int*>(tmem_holder + 1);
    float4* coltab = reinterpret_cast<float4*>(base + S * SB + 256);  // [BN] (s, d, bias) of the tile's columns
    unsigned char* w1b = base + w1b_offset(BN);  // final level: W_1^T TF32 parts (see psmem_bytes)
    uint64_t* fbar = pfree + NP;                 // final level: the W_1 product is in TMEM (after tmem_holder)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int nk = (K + BK - 1) / BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int p = 0; p < NP; ++p) {
            mbar_init(&pfull[p], 1);
            mbar_init(&pfree[p], 4 * EG);
        }
        mbar_init(pfree + NP, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mAh)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mBh)) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)), "r"(TC)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_holder;

    if (threadIdx.x == 0) {
        int issued = 0;
        for (int kc = 0; kc < nk; ++kc) {
            const int s = kc % S;
            if (kc >= S && !mbar_wait(&empty[s], ((kc / S) - 1) & 1)) {
                atomicExch(err, 1);
                *(volatile int*)abort_flag = 1;
                break;
            }
            if (*(volatile int*)abort_flag) break;
            unsigned char* st = base + s * SB;
            mbar_expect_tx(&full[s], SB);
            const int ay = ((int)blockIdx.y * nk + kc) * BM;  // row of the A block in the blocked view
            tma_load_2d(st, &mAh, &full[s], 0, ay);
            tma_load_2d(st + BM * BK * 4, &mAl, &full[s], 0, ay);
            tma_load_2d(st + 2 * BM * BK * 4, &mBh, &full[s], kc * BK, n0);
            tma_load_2d(st + 2 * BM * BK * 4 + BN * BK * 4, &mBl, &full[s], kc * BK, n0);
            ++issued;
        }
        for (int kc = (issued > S ? issued - S : 0); kc < issued; ++kc) {
            if (!mbar_wait(&full[kc % S], (kc / S) & 1)) {
                atomicExch(err, 1);
                break;
            }
        }
    } else if (threadIdx.x == 32) {
        for (int kc = 0; kc < nk; ++kc) {
            const int s = kc % S, p = kc % NP;
            if (!mbar_wait(&full[s], (kc / S) & 1) || (kc >= NP && !mbar_wait(&pfree[p], ((kc / NP) - 1) & 1))) {
                atomicExch(err, 1);
                *(volatile int*)abort_flag = 1;
                break;
            }
            fence_after();
            const uint32_t d = tmem + (uint32_t)(p * PB);
            const uint32_t sa = smem_u32(base + s * SB);
            const uint64_t ah = sw128_desc(sa), al = sw128_desc(sa + BM * BK * 4);
            const uint64_t bh = sw128_desc(sa + 2 * BM * BK * 4), bl = sw128_desc(sa + 2 * BM * BK * 4 + BN * BK * 4);
            // small cross terms first, the large hi*hi terms last: the tensor core's accumulation
            // rounds toward zero relative to the running magnitude, so fewer steps at full size
#pragma unroll
            for (int kk = 0; kk < BK / 8; ++kk) {
                const uint64_t o = (uint64_t)(kk * 32) >> 4;
                mma_tf32(d, ah + o, bl + o, IDESC, kk ? 1u : 0u);
                mma_tf32(d, al + o, bh + o, IDESC, 1u);
            }
#pragma unroll
            for (int kk = 0; kk < BK / 8; ++kk) {
                const uint64_t o = (uint64_t)(kk * 32) >> 4;
                mma_tf32(d, ah + o, bh + o, IDESC, 1u);
            }
            mma_commit(&empty[s]);
            mma_commit(&pfull[p]);
        }
    }
    if (warp >= 2) {
        // ---- epilogue warps: add every chunk partial into FP32 registers.  Warp w drains TMEM lane
        // quadrant w % 4 (the quadrant a warp may access), columns [cofs, cofs + BNH) of the tile.
        const int sub = warp & 3;
        const int cofs = ((warp - 2) >> 2) * BNH;
        const int grp = (warp - 2) >> 2;
        float acc[BNH];
#pragma unroll
        for (int j = 0; j < BNH; ++j) acc[j] = 0.f;
        bool ok = true;
        const uint32_t lane_base = (uint32_t)(sub * 32) << 16;
        // chain epilogue: when the tile's rows all belong to one domain, its columns' slope,
        // intercept and bias are staged once in shared memory while the first chunk is computed
        bool uniform = false;
        if constexpr (EPI != 0) {
            if constexpr (EPI == 2) {
                // W_1 rows of this tile's columns as the K-major right operand (N = kFinalCols outputs)
                constexpr int NCH = BN / 32;
                for (int idx = threadIdx.x - 64; idx < NCH * kFinalCols * 32; idx += 128 * EG) {
                    const int c = idx / (kFinalCols * 32), rem = idx - c * (kFinalCols * 32);
                    const int r = rem >> 5, k = rem & 31;
                    const int col = n0 + c * 32 + k;
                    const float x = (col < N && r < epi.n0) ? epi.W1[(int64_t)col * epi.n0 + r] : 0.f;
                    const float h = tf32_part_rna(x);
                    const int off = c * (kFinalCols * 128) + r * 128 + ((((k >> 2) ^ (r & 7))) << 4) + ((k & 3) << 2);
                    *reinterpret_cast<float*>(w1b + off) = h;
                    *reinterpret_cast<float*>(w1b + NCH * kFinalCols * 128 + off) = tf32_part_rna(x - h);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            }
            const int dom0 = m0 / epi.rows_per_dom;
            uniform = R > 0 && dom0 == (min(m0 + BM, R) - 1) / epi.rows_per_dom;
            if (uniform) {
                for (int j = threadIdx.x - 64; j < BN; j += 128 * EG) {
                    const int col = n0 + j;
                    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (col < N)
                        q = make_float4(epi.hs[(int64_t)dom0 * epi.hidden + epi.hoff + col],
                                        epi.hd[(int64_t)dom0 * epi.hidden + epi.hoff + col], epi.bias[col], 0.f);
                    coltab[j] = q;
                }
            }
            epi_bar<EG>();
        }
        for (int kc = 0; kc < nk; ++kc) {
            const int p = kc % NP;
            const bool good = !*(volatile int*)abort_flag && mbar_wait(&pfull[p], (kc / NP) & 1);
            if (!__all_sync(0xffffffffu, good)) {  // TMEM loads are warp-collective: decide per warp
                ok = false;
                break;
            }
            fence_after();
            if constexpr (BNH >= 64) {
#pragma unroll
                for (int c0 = 0; c0 < BNH; c0 += 64) {
                    float v[64];
                    tmem_ld64(tmem + lane_base + (uint32_t)(p * PB + cofs + c0), v);
#pragma unroll
                    for (int j = 0; j < 64; ++j) acc[c0 + j] += v[j];
                }
            } else {
#pragma unroll
                for (int c0 = 0; c0 < BNH; c0 += 32) {
                    float v[32];
                    tmem_ld32(tmem + lane_base + (uint32_t)(p * PB + cofs + c0), v);
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (c0 + j < BNH) acc[c0 + j] += v[j];
                }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&pfree[p]);
        }
        if (!ok) atomicExch(err, 1);
        const int row = m0 + sub * 32 + lane;
        if constexpr (EPI != 0) {
            const bool live = ok && row < R;
            const int rr = live ? row : (R > 0 ? R - 1 : 0);
            const int dom = rr / epi.rows_per_dom;
            const float* sl = epi.hs + (int64_t)dom * epi.hidden + epi.hoff;
            const float* dl = epi.hd + (int64_t)dom * epi.hidden + epi.hoff;
            float spos = 0.f, sneg = 0.f, sb = 0.f;
            if (uniform) {
                // padding columns carry (0, 0, 0): x*s = 0 and no intercept contribution
                if (epi.lev && live) {
#pragma unroll
                    for (int j = 0; j < BNH; ++j)
                        if (n0 + cofs + j < N) epi.lev[blk_index(row, n0 + cofs + j, (N + 31) >> 5)] = acc[j];
                }
#pragma unroll
                for (int j = 0; j < BNH; ++j) {
                    const float4 q = coltab[cofs + j];
                    const float x = acc[j], xs = x * q.x;
                    spos = fmaf(fmaxf(x, 0.f), q.y, spos);
                    sneg = fmaf(fminf(x, 0.f), q.y, sneg);
                    sb = fmaf(xs, q.z, sb);
                    acc[j] = xs;
                }
            } else {
#pragma unroll
                for (int j = 0; j < BNH; ++j) {
                    const int col = n0 + cofs + j;
                    float xs = 0.f;
                    if (col < N) {
                        const float x = acc[j], dj = dl[col];
                        if (epi.lev && live) epi.lev[blk_index(row, col, (N + 31) >> 5)] = x;
                        xs = x * sl[col];
                        spos = fmaf(fmaxf(x, 0.f), dj, spos);
                        sneg = fmaf(fminf(x, 0.f), dj, sneg);
                        sb = fmaf(xs, epi.bias[col], sb);
                    }
                    acc[j] = xs;
                }
            }
            if (live) {
                // partial intercepts, one set per (column tile, column group); consecutive rows are
                // consecutive in memory, so a warp's stores coalesce
                const int64_t t = (int64_t)blockIdx.x * EG + grp;
                epi.part[(t * 3 + 0) * R + row] = spos;
                epi.part[(t * 3 + 1) * R + row] = sneg;
                epi.part[(t * 3 + 2) * R + row] = sb;
            }
            const int cmax = min(BN, epi.ldk - n0);  // columns of this tile inside the operand (incl. zero padding)
            if constexpr (EPI == 2) {
                // final level: Lambda_x partial = (x*s) W_1 over this tile's columns on the tensor
                // cores.  x*s is staged as TF32 parts in the 128-byte swizzle layout (the MMA's K-major
                // A operand), one thread issues M = 128, N = kFinalCols MMAs per 32-column chunk into
                // its own TMEM accumulator, and the first column group sums the chunks in FP32.
                constexpr int NCH = BN / 32;
                const int rr = sub * 32 + lane;
                const int nch = cmax >> 5;
#pragma unroll
                for (int cl = 0; cl < BNH / 32; ++cl) {
                    const int c = cofs / 32 + cl;
                    if (c < nch) {
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int j = cl * 32 + u * 4;
                            const float h0 = tf32_part_rna(acc[j]), h1 = tf32_part_rna(acc[j + 1]);
                            const float h2 = tf32_part_rna(acc[j + 2]), h3 = tf32_part_rna(acc[j + 3]);
                            const float4 lv = make_float4(tf32_part_rna(acc[j] - h0), tf32_part_rna(acc[j + 1] - h1),
                                                          tf32_part_rna(acc[j + 2] - h2), tf32_part_rna(acc[j + 3] - h3));
                            const int off = c * 16384 + rr * 128 + ((u ^ (rr & 7)) << 4);
                            *reinterpret_cast<float4*>(base + off) = make_float4(h0, h1, h2, h3);
                            *reinterpret_cast<float4*>(base + NCH * 16384 + off) = lv;
                        }
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                epi_bar<EG>();
                const uint32_t dcol = (uint32_t)(NP * PB);  // accumulators after the partial buffers
                if (threadIdx.x == 64) {
                    fence_after();
                    if (ok) {
                        constexpr uint32_t ID16 = idesc_tf32(BM, kFinalCols);
                        const uint32_t sa = smem_u32(base), sb = smem_u32(w1b);
                        for (int c = 0; c < nch; ++c) {
                            const uint32_t d = tmem + dcol + (uint32_t)(c * kFinalCols);
                            const uint64_t ah = sw128_desc(sa + c * 16384), al = sw128_desc(sa + NCH * 16384 + c * 16384);
                            const uint64_t bh = sw128_desc(sb + c * (kFinalCols * 128));
                            const uint64_t bl = sw128_desc(sb + NCH * kFinalCols * 128 + c * (kFinalCols * 128));
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const uint64_t o = (uint64_t)(kk * 32) >> 4;
                                mma_tf32(d, ah + o, bl + o, ID16, kk ? 1u : 0u);
                                mma_tf32(d, al + o, bh + o, ID16, 1u);
                            }
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const uint64_t o = (uint64_t)(kk * 32) >> 4;
                                mma_tf32(d, ah + o, bh + o, ID16, 1u);
                            }
                        }
                        mma_commit(fbar);
                    } else {
                        mbar_expect_tx(fbar, 0);  // complete the phase so the readers do not wait out their budget
                    }
                }
                if (grp == 0) {
                    const bool have = mbar_wait(fbar, 0);
                    fence_after();
                    if (!have) atomicExch(err, 1);
                    float px[kFinalCols];
#pragma unroll
                    for (int q = 0; q < kFinalCols; ++q) px[q] = 0.f;
                    if (have && ok) {
                        for (int c = 0; c < nch; ++c) {
                            float v[kFinalCols];
                            tmem_ld16(tmem + lane_base + dcol + (uint32_t)(c * kFinalCols), v);
#pragma unroll
                            for (int q = 0; q < kFinalCols; ++q) px[q] += v[q];
                        }
                    }
                    if (live) {
                        float* o = epi.lxpart + (int64_t)blockIdx.x * epi.n0 * (int64_t)R + row;
#pragma unroll
                        for (int q = 0; q < kFinalCols; ++q)
                            if (q < epi.n0) o[(int64_t)q * R] = px[q];
                    }
                }
            } else if constexpr (BN >= 32) {
                // Both TF32 parts staged in the idle pipeline buffers as 128-row x 32-column boxes in
                // the 128-byte swizzle layout ([part][chunk][row][16-byte unit ^ (row & 7)]); one
                // thread then writes every box with a TMA tensor store (a box of the blocked operand
                // is 16 KB contiguous in global memory).
                constexpr int NCH = BN / 32;
                const int rr = sub * 32 + lane;
                const int nch = cmax >> 5;
#pragma unroll
                for (int cl = 0; cl < BNH / 32; ++cl) {
                    const int c = cofs / 32 + cl;  // chunk of the tile
                    if (c < nch) {
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int j = cl * 32 + u * 4;
                            const float h0 = tf32_part_rna(acc[j]), h1 = tf32_part_rna(acc[j + 1]);
                            const float h2 = tf32_part_rna(acc[j + 2]), h3 = tf32_part_rna(acc[j + 3]);
                            const float4 hv = make_float4(h0, h1, h2, h3);
                            const float4 lv = make_float4(tf32_part_rna(acc[j] - h0), tf32_part_rna(acc[j + 1] - h1),
                                                          tf32_part_rna(acc[j + 2] - h2), tf32_part_rna(acc[j + 3] - h3));
                            const int off = c * 16384 + rr * 128 + ((u ^ (rr & 7)) << 4);
                            *reinterpret_cast<float4*>(base + off) = hv;
                            *reinterpret_cast<float4*>(base + NCH * 16384 + off) = lv;
                        }
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                epi_bar<EG>();
                if (threadIdx.x == 64 && ok) {
                    const int enk = epi.ldk >> 5;
                    for (int c = 0; c < nch; ++c) {
                        const int y = ((int)blockIdx.y * enk + (n0 >> 5) + c) * BM;
                        tma_store_2d(&mOh, base + c * 16384, 0, y);
                        tma_store_2d(&mOl, base + NCH * 16384 + c * 16384, 0, y);
                    }
                    bulk_commit();
                    bulk_wait_read();  // the boxes are read before the CTA releases its shared memory
                }
            } else {
                // narrow tiles (BN = 16, one column group): x*s as TF32 parts staged per warp as a
                // 32 x BN tile with an odd row stride, stored row by row with lanes across columns
                constexpr int TLD = BN + 1;
                float* tile = reinterpret_cast<float*>(base) + sub * 32 * TLD;
                for (int part_i = 0; part_i < 2; ++part_i) {
#pragma unroll
                    for (int j = 0; j < BN; ++j) {
                        const float h = tf32_part_rna(acc[j]);
                        tile[lane * TLD + j] = part_i == 0 ? h : tf32_part_rna(acc[j] - h);
                    }
                    __syncwarp();
                    // blocked layout: the warp's 32 rows of one 32-column chunk are 4 KB contiguous
                    float* dst = part_i == 0 ? epi.Ah : epi.Al;
                    const int enk = epi.ldk >> 5;
                    const int nr = ok ? max(0, min(32, R - (m0 + sub * 32))) : 0;  // live rows of this warp
                    for (int c0 = 0; c0 < cmax; c0 += 32) {
                        const int j = c0 + lane;
                        if (j >= cmax) continue;
                        // rows m0 + sub*32 .. +31 stay inside one 128-row block: consecutive rows are 32 apart
                        float* col = dst + blk_index(m0 + sub * 32, n0 + j, enk);
                        float v[32];
#pragma unroll
                        for (int r = 0; r < 32; ++r) v[r] = tile[r * TLD + j];
#pragma unroll
                        for (int r = 0; r < 32; ++r)
                            if (r < nr) col[r * 32] = v[r];
                    }
                    __syncwarp();
                }
            }
        } else if (ok && row < R) {
#pragma unroll
            for (int j = 0; j < BNH; ++j) {
                const int col = n0 + cofs + j;
                if (col < N) C[(int64_t)row * ldc + col] = acc[j];
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC) : "memory");
    }
}

// TF32 part of x with round-to-nearest (ties away), as an FP32 value whose low 13 bits are zero.
__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Split rows of X [R][K] (ld ldx) into TF32 parts H/L with zero padding in K..ldk-1: row-major
// [R][ldk] (B operands) or, with `blocked`, the blocked left-operand layout.
__global__ void k_split_tf32(const float* __restrict__ X, int ldx, int R, int K, int ldk, float* __restrict__ Hh,
                             float* __restrict__ Ll, int blocked) {
    const int64_t total = (int64_t)R * ldk;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = idx / ldk;
        const int k = (int)(idx - r * ldk);
        const float x = k < K ? X[r * ldx + k] : 0.f;
        const float h = tf32_rna(x);
        const int64_t o = blocked ? blk_index(r, k, ldk >> 5) : idx;
        Hh[o] = h;
        Ll[o] = tf32_rna(x - h);
    }
}

}  // namespace tc
