// Persistent variant of the 3xTF32 chain GEMM for 128-column tiles: one CTA per SM walks a strided
// list of 128 x 128 output tiles, and two epilogue groups take the tiles in turn, so one group's
// epilogue (intercept partials and the next operand, or the final level's W_1 product) runs while
// the tensor cores already work on the next tile for the other group.
//
//   warp 0 lane 0  TMA producer over all tiles' 32-wide K chunks (three-stage ring)
//   warp 1         TMEM owner (512 columns = 2 groups x 2 partial buffers x 128)
//   warps 1, 2     lane 0 of each issues MMAs: tile j goes into group j % 2's buffers, alternating
//                  per fill (kPromote chunks); warp 1 issues the even fills, warp 2 the odd ones
//   warp 3         idle (it completes the first warpgroup for the register split)
//   warps 4..7     epilogue group 0 (tiles 0, 2, 4, ... of this CTA), warps 8..11 group 1; warp w
//                  reads TMEM lane quadrant w % 4 and holds that quadrant's rows x 128 columns
//
// Two issuers: a tcgen05.mma of 128 x 128 x 8 (TF32) keeps the tensor pipe busy for only 64 cycles,
// and the pipe holds almost no queued work behind it, so any time the issuing thread spends between
// MMAs (a barrier test, index arithmetic, losing issue slots to the epilogue warps on its
// sub-partition) is idle tensor time.  With the fills split between two threads in different
// warps, one thread's MMAs run while the other waits for its next stage; each thread owns its own
// partial buffers (fill parity), and its commits track only its own MMAs.  Each stage has one
// `full` barrier per issuer, signalled by the chunks that issuer consumes: a thread then tests only
// phases of its own chunks, in order, and no barrier can run two phases ahead of the thread waiting
// on it (one barrier shared by both would, whenever one thread lags the other).
//
// Registers: the launch gives 168 per thread (384 threads, one CTA per SM); the first warpgroup
// drops to kRegsCtl and the two epilogue warpgroups rise to kRegsEpi, which the released registers
// cover exactly (128 x (168 - 56) = 256 x (224 - 168)).  The host launches this kernel only when
// the compiled entry count is 168, so the increase never waits for registers that do not exist.
//
// The three TF32 products and their order are those of k_tc_gemm_p.  Accumulation is promoted per
// fill: the tensor core sums kPromote chunks of 32 into a partial buffer, which the epilogue then
// adds into FP32 registers.  The tensor core's accumulation rounds toward zero relative to the running
// sum, so longer fills err more.  kPromote = 2 (every 64 of K): with the intercepts summed in FP64
// across the chain levels (wide.cuh), the boxes of the 16-512x4-8 workload over 50 steps use at
// most 4 % of their outward margin against the FP64 oracle (7 % on the branch workload), against
// 1 % (0.4 %) with one chunk per fill, and a pass is 3.6 % faster; four chunks per fill made a lower
// bound of the branch workload tighter than the oracle's.  The intercept partials keep the two
// 64-column sets per tile.  The final level's (x*s) W_1 product is taken with FP32 FMAs (the TMEM is
// all partial buffers), not with 3xTF32 MMAs.  The next operand (chain levels) leaves through a
// per-warp staging tile in shared memory, so its global stores cover whole 64-byte row segments.
//
// Every wait is bounded.  On expiry the error flag is raised and each role runs through its
// remaining loop structure without waiting (group barriers stay matched), so the CTA always exits.
#pragma once
#include "tc_gemm.cuh"

namespace tc {

constexpr int kPersistThreads = 128 + 2 * 128;
constexpr int kRegsLaunch = 168, kRegsCtl = 56, kRegsEpi = 224;
static_assert(128 * (kRegsLaunch - kRegsCtl) >= 256 * (kRegsEpi - kRegsLaunch), "register split exceeds the launch's registers");
constexpr int kPS = 3;                              // ring stages
constexpr int kPromote = 2;                         // K chunks (of 32) per partial buffer fill
constexpr int kPSB = stage_bytes(128);              // 64 KB per stage
__host__ __device__ constexpr int pp_coltab_offset() { return kPS * kPSB + 256; }
__host__ __device__ constexpr int pp_w1tab_offset() { return pp_coltab_offset() + 2 * 128 * 16; }
__host__ __device__ constexpr int pp_smem_bytes() { return pp_w1tab_offset() + 2 * 128 * kFinalCols * 4 + 1024; }

__device__ __forceinline__ void group_bar(int g) {
    if (g == 0) asm volatile("bar.sync 1, 128;" ::: "memory");
    else asm volatile("bar.sync 2, 128;" ::: "memory");
}

// FP32 pairs in one 64-bit register (low word first).  Holding the W_1 product's accumulators and
// table rows as pairs keeps the final level's epilogue within its register budget.
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(unsigned long long v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

// One row's chain epilogue over the tile's 128 columns in a single pass, so every accumulator dies
// as soon as its column is done: x -> x*s (slope s of the column's neuron), the partial intercepts
// (two 64-column sets), and either the next operand's TF32 parts (EPI 1) or the (x*s) W_1 product
// (EPI 2).  U: the tile's rows share one domain, whose (s, d, bias) per column are in coltab.
//
// EPI 1 writes the next operand through a 2 KB per-warp staging tile (32 rows x 16 columns, 16-byte
// units XOR-swizzled by row so both the row-wise writes and the transposed reads are free of bank
// conflicts): a global store instruction then covers 8 rows x 64 contiguous bytes instead of 32 rows
// x 16 bytes.  ok is warp-uniform; rows at or past R are not written.
template <int EPI, bool U>
__device__ __forceinline__ void pp_row_epilogue(float* acc, const float4* coltab, const float* w1tab, float* stg,
                                                const ChainEpi& epi, int row, bool ok, int n0, int N, int R) {
    constexpr int BN = 128;
    const int lane = threadIdx.x & 31;
    const bool live = ok && row < R;
    const int rr = live ? row : (R > 0 ? R - 1 : 0);
    const int dom = rr / epi.rows_per_dom;
    const float* sl = epi.hs + (int64_t)dom * epi.hidden + epi.hoff;
    const float* dl = epi.hd + (int64_t)dom * epi.hidden + epi.hoff;
    float spos[2] = {0.f, 0.f}, sneg[2] = {0.f, 0.f}, sb[2] = {0.f, 0.f};
    unsigned long long px2[kFinalCols / 2];  // EPI 2: Lambda_x partial as pairs
#pragma unroll
    for (int c = 0; c < kFinalCols / 2; ++c) px2[c] = 0ull;
    const int enk = epi.ldk >> 5;
    const int nch = min(BN, epi.ldk - n0) >> 5;  // 32-column chunks of this tile inside the operand
    const int row0 = row - lane;                 // first row of this warp
    float* levp = live ? epi.lev : nullptr;  // keep mode: the level itself, blocked with ru32(N) columns
    const int ldl = (N + 31) & ~31;
    constexpr int CB = EPI == 1 ? 16 : 4;  // columns per block (EPI 1: one staging tile)
#pragma unroll
    for (int hc = 0; hc < BN / CB; ++hc) {
        float xv[CB];
#pragma unroll
        for (int e = 0; e < CB; ++e) {
            const int j = CB * hc + e, h = j >> 6;
            const float x = acc[j];
            float xs = 0.f;
            if constexpr (U) {
                // padding columns carry (0, 0, 0): x*s = 0 and no intercept contribution
                const float4 qv = coltab[j];
                xs = x * qv.x;
                spos[h] = fmaf(fmaxf(x, 0.f), qv.y, spos[h]);
                sneg[h] = fmaf(fminf(x, 0.f), qv.y, sneg[h]);
                sb[h] = fmaf(xs, qv.z, sb[h]);
            } else {
                const int col = n0 + j;
                if (col < N) {
                    const float dj = dl[col];
                    xs = x * sl[col];
                    spos[h] = fmaf(fmaxf(x, 0.f), dj, spos[h]);
                    sneg[h] = fmaf(fminf(x, 0.f), dj, sneg[h]);
                    sb[h] = fmaf(xs, epi.bias[col], sb[h]);
                }
            }
            xv[e] = xs;
        }
        if (levp) {
#pragma unroll
            for (int u = 0; u < CB / 4; ++u) {
                const int c0 = n0 + CB * hc + 4 * u;
                if (c0 < ldl)
                    *reinterpret_cast<float4*>(levp + blk_index(row, c0, ldl >> 5)) =
                        make_float4(acc[CB * hc + 4 * u], acc[CB * hc + 4 * u + 1], acc[CB * hc + 4 * u + 2], acc[CB * hc + 4 * u + 3]);
            }
        }
        if constexpr (EPI == 1) {
            const int c = hc >> 1;
            if (c < nch) {  // uniform across the warp
#pragma unroll
                for (int part = 0; part < 2; ++part) {
                    float v[CB];
#pragma unroll
                    for (int e = 0; e < CB; ++e) {
                        const float hi = tf32_part_rna(xv[e]);
                        v[e] = part == 0 ? hi : tf32_part_rna(xv[e] - hi);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        *reinterpret_cast<float4*>(stg + lane * 16 + ((u ^ ((lane >> 1) & 3)) << 2)) =
                            make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
                    __syncwarp();
                    float* dst = part == 0 ? epi.Ah : epi.Al;
                    const int u = lane & 3;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int r = (lane >> 2) + 8 * i;
                        const float4 w = *reinterpret_cast<const float4*>(stg + r * 16 + ((u ^ ((r >> 1) & 3)) << 2));
                        if (ok && row0 + r < R)
                            *reinterpret_cast<float4*>(dst + blk_index(row0 + r, n0 + 16 * hc + 4 * u, enk)) = w;
                    }
                    __syncwarp();
                }
            }
        } else {
#pragma unroll
            for (int e = 0; e < CB; ++e) {
                const ulonglong2* w = reinterpret_cast<const ulonglong2*>(w1tab + (CB * hc + e) * kFinalCols);
#pragma unroll
                for (int k = 0; k < kFinalCols / 4; ++k) {
                    const ulonglong2 wv = w[k];
                    float w0, w1, w2, w3, p0, p1, p2, p3;
                    unpack2(wv.x, w0, w1);
                    unpack2(wv.y, w2, w3);
                    unpack2(px2[2 * k], p0, p1);
                    unpack2(px2[2 * k + 1], p2, p3);
                    px2[2 * k] = pack2(fmaf(xv[e], w0, p0), fmaf(xv[e], w1, p1));
                    px2[2 * k + 1] = pack2(fmaf(xv[e], w2, p2), fmaf(xv[e], w3, p3));
                }
            }
        }
    }
    if (live) {
        const int nt = n0 / BN;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t t = (int64_t)nt * 2 + h;
            epi.part[(t * 3 + 0) * R + row] = spos[h];
            epi.part[(t * 3 + 1) * R + row] = sneg[h];
            epi.part[(t * 3 + 2) * R + row] = sb[h];
        }
        if constexpr (EPI == 2) {
            float px[kFinalCols];
#pragma unroll
            for (int c = 0; c < kFinalCols / 2; ++c) unpack2(px2[c], px[2 * c], px[2 * c + 1]);
            float* o = epi.lxpart + (int64_t)nt * epi.n0 * (int64_t)R + row;
#pragma unroll
            for (int c = 0; c < kFinalCols; ++c)
                if (c < epi.n0) o[(int64_t)c * R] = px[c];
        }
    }
}

// Warp reduce-scatter of 32 values per lane over segments of lanes: with G = 32, after five rounds of
// pairwise exchange (31 shuffles) v[0] of lane L is the sum over the warp of the lanes' value L.
// The same over segments of G lanes (G a power of two, at most 32; uniform across the warp): each
// round halves the live values and pairs lanes inside the segment, so that afterwards lane L holds in
// v[0 .. 32/G) the segment's sums of the values (L mod G) * 32/G + q.
template <int HALF>
__device__ __forceinline__ void bfly_masked(float* v, int lane, int mask) {
    const bool up = (lane & mask) != 0;
#pragma unroll
    for (int q = 0; q < HALF; ++q) {
        const float send = up ? v[q] : v[q + HALF];
        const float keep = up ? v[q + HALF] : v[q];
        v[q] = keep + __shfl_xor_sync(0xffffffffu, send, mask);
    }
}
__device__ __forceinline__ void seg_reduce_scatter32(float* v, int lane, int G) {
    if (G >= 2) bfly_masked<16>(v, lane, G >> 1);
    if (G >= 4) bfly_masked<8>(v, lane, G >> 2);
    if (G >= 8) bfly_masked<4>(v, lane, G >> 3);
    if (G >= 16) bfly_masked<2>(v, lane, G >> 4);
    if (G >= 32) bfly_masked<1>(v, lane, 1);
}

// Reverse chain level (EPI 3) of one row over the tile's 128 columns, the neurons j of hidden layer
// m: acc = (adjoint of the level below) W_m^T.  Per entry, g = acc + (gklo_i + gkhi_i) b_j adds the
// adjoint through the level's intercept term Lambda_s b_m; with lam = Lambda^(m)_ij of the forward
// pass, the warp sums lam g (the adjoint of the slope s_j) and gkhi_i lam^+ + gklo_i lam^- (the
// adjoint of the relaxation intercept d_j) over each row segment into colpart, and the adjoint of
// Lambda^(m), g s_j + d_j (gkhi_i [lam > 0] + gklo_i [lam < 0]), becomes the next reverse level's
// left operand (TF32 parts through the staging tile, as in EPI 1) unless epi.Ah is null (the
// target's top level).  Segments lie inside one domain: 32 rows when n_ell is a multiple of 32, else
// the domain's n_ell rows (2, 4, 8 or 16).
// The row's intercept adjoints, read by the reverse epilogue.
struct RevPre {
    float kl, kh;
};
__device__ __forceinline__ int64_t rev_level_row(const ChainEpi& epi, int row, int R) {
    const int rr = row < R ? row : (R > 0 ? R - 1 : 0);
    return epi.rlev_shared ? (int64_t)(rr % epi.rows_per_dom) : (int64_t)rr;
}
__device__ __forceinline__ void rev_level_load(const ChainEpi& epi, int64_t lrow, bool in, int c0, int N, float4* l) {
    const int nkl = (N + 31) >> 5;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        l[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (in && c0 + 4 * u < N) l[u] = *reinterpret_cast<const float4*>(epi.rlev + blk_index(lrow, c0 + 4 * u, nkl));
    }
}
__device__ __forceinline__ RevPre rev_preload(const ChainEpi& epi, int row, int R) {
    RevPre p;
    const bool in = row < R;
    const int rr = in ? row : (R > 0 ? R - 1 : 0);
    const int dom = rr / epi.rows_per_dom, i = rr - dom * epi.rows_per_dom;
    p.kl = in ? epi.rklo[(int64_t)dom * epi.kld + i] : 0.f;
    p.kh = in ? epi.rkhi[(int64_t)dom * epi.kld + i] : 0.f;
    return p;
}

template <bool U, bool SEG32>
__device__ __forceinline__ void pp_row_epilogue_rev(float* acc, const float4* coltab, float* stg, const ChainEpi& epi, int row,
                                                    bool ok, int n0, int N, int R, const RevPre& pre) {
    constexpr int BN = 128, CB = 16;
    const int lane = threadIdx.x & 31;
    const bool live = ok && row < R;
    const int rr = live ? row : (R > 0 ? R - 1 : 0);
    const int dom = rr / epi.rows_per_dom;
    const float* sl = epi.hs + (int64_t)dom * epi.hidden + epi.hoff;
    const float* dl = epi.hd + (int64_t)dom * epi.hidden + epi.hoff;
    const float kl = live ? pre.kl : 0.f;
    const float kh = live ? pre.kh : 0.f;
    const float kb = kl + kh;
    const int64_t lrow = rev_level_row(epi, row, R);  // row of the forward level read
    const int enk = epi.ldk >> 5;
    const int nch = epi.Ah ? (min(BN, epi.ldk - n0) >> 5) : 0;  // 32-column chunks of the next operand in this tile
    const int row0 = row - lane;
    const int G = SEG32 ? 32 : epi.rows_per_dom;  // row segment of the column sums
#pragma unroll
    for (int hc = 0; hc < BN / CB; ++hc) {
        float v[32], xv[CB], lv[CB];
        {
            float4 q4[4];
            rev_level_load(epi, lrow, live, n0 + CB * hc, N, q4);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                lv[4 * u] = q4[u].x;
                lv[4 * u + 1] = q4[u].y;
                lv[4 * u + 2] = q4[u].z;
                lv[4 * u + 3] = q4[u].w;
            }
        }
#pragma unroll
        for (int e = 0; e < CB; ++e) {
            const int j = CB * hc + e, col = n0 + j;
            float sj = 0.f, dj = 0.f, bj = 0.f;
            if constexpr (U) {
                const float4 qv = coltab[j];  // padding columns carry (0, 0, 0)
                sj = qv.x;
                dj = qv.y;
                bj = qv.z;
            } else if (col < N) {
                sj = sl[col];
                dj = dl[col];
                bj = epi.bias[col];
            }
            const bool in = live && col < N;
            const float lam = in ? lv[e] : 0.f;
            const float g = in ? fmaf(kb, bj, acc[j]) : 0.f;
            const float kv = lam > 0.f ? kh : kl;  // the intercept adjoint of lam's sign (lam = 0 adds nothing)
            v[e] = lam * g;
            v[CB + e] = lam * kv;
            xv[e] = fmaf(g, sj, lam != 0.f ? dj * kv : 0.f);  // the adjoint of Lambda^(m): the next operand
        }
        if constexpr (SEG32) {
            bfly_masked<16>(v, lane, 16);
            bfly_masked<8>(v, lane, 8);
            bfly_masked<4>(v, lane, 4);
            bfly_masked<2>(v, lane, 2);
            bfly_masked<1>(v, lane, 1);
        } else {
            seg_reduce_scatter32(v, lane, G);
        }
        // value index x < 16: slope sum of column CB*hc + x; x >= 16: intercept sum of column CB*hc + x - 16
        if constexpr (SEG32) {
            const int col = n0 + CB * hc + (lane & 15);
            if (ok && row0 < R && col < N) epi.colpart[((int64_t)(row0 >> 5) * 2 + (lane >> 4)) * N + col] = v[0];
        } else {
            const int cnt = 32 / G, seg = (row0 + lane) / G;
            const bool seg_live = ok && row0 + (lane & ~(G - 1)) < R;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                if (q < cnt) {
                    const int x = (lane & (G - 1)) * cnt + q;
                    const int col = n0 + CB * hc + (x & 15);
                    if (seg_live && col < N) epi.colpart[((int64_t)seg * 2 + (x >> 4)) * N + col] = v[q];
                }
            }
        }
        const int c = hc >> 1;
        if (c < nch) {  // uniform across the warp
#pragma unroll
            for (int part = 0; part < 2; ++part) {
                float w4[CB];
#pragma unroll
                for (int e = 0; e < CB; ++e) {
                    const float hi = tf32_part_rna(xv[e]);
                    w4[e] = part == 0 ? hi : tf32_part_rna(xv[e] - hi);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    *reinterpret_cast<float4*>(stg + lane * 16 + ((u ^ ((lane >> 1) & 3)) << 2)) =
                        make_float4(w4[4 * u], w4[4 * u + 1], w4[4 * u + 2], w4[4 * u + 3]);
                __syncwarp();
                float* dst = part == 0 ? epi.Ah : epi.Al;
                const int u = lane & 3;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int r = (lane >> 2) + 8 * q;
                    const float4 w = *reinterpret_cast<const float4*>(stg + r * 16 + ((u ^ ((r >> 1) & 3)) << 2));
                    if (ok && row0 + r < R) *reinterpret_cast<float4*>(dst + blk_index(row0 + r, n0 + 16 * hc + 4 * u, enk)) = w;
                }
                __syncwarp();
            }
        }
    }
}

// PAIR: the pair form (launched in clusters of two).  One thread of the leader CTA (rank 0) issues
// tcgen05.mma.cta_group::2 with M = 256: each CTA of the pair loads its own 128-row tile of A and
// half of the 128 columns of B (64 rows of B^T) into its stages (48 KB, four of them), every load
// signalling the leader's `full` barrier, and each CTA's TMEM receives its 128 rows, so the
// epilogues are those of the single-CTA form.  Per SM the tensor core then reads 6 KB of operands
// per 128 x 128 x 8 product instead of 8 KB.  The leader's commits arrive on both CTAs' `empty` and
// `pfull` barriers; the follower's epilogue warps release a partial buffer on the leader's `pfree`.
template <int EPI, bool PAIR = false>
__global__ void __launch_bounds__(kPersistThreads, 1) k_tc_gemm_pp(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
                                                                  const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
                                                                  float* __restrict__ C, int R, int K, int N, int ldc, int* __restrict__ err,
                                                                  const ChainEpi epi) {
    constexpr int BN = 128, S = PAIR ? 4 : kPS, SB = PAIR ? (2 * BM * BK * 4 + BN * BK * 4) : kPSB;
    static_assert(S * SB == kPS * kPSB, "the pair form keeps the single-CTA form's stage area");
    constexpr uint32_t IDESC = idesc_tf32(PAIR ? 2 * BM : BM, BN);
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(base + S * SB);  // [2][S] stage landed, per MMA issuer
    uint64_t* empty = full + 2 * S;
    uint64_t* pfull = empty + S;  // [4] buffer ready (MMA commit)
    uint64_t* pfree = pfull + 4;  // [4] buffer consumed (the owning group's 4 warps)
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(pfree + 4);
    int* abort_flag = reinterpret_cast<int*>(tmem_holder + 1);
    static_assert((3 * S + 8) * 8 + 8 <= pp_coltab_offset() - kPS * kPSB, "barriers fit their area");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = (K + BK - 1) / BK;
    const int npc = (nk + kPromote - 1) / kPromote;  // partial buffer fills per tile
    const int ntn = (N + BN - 1) / BN;
    // Launched in clusters of cs CTAs (cs = 1 or 2), the CTAs of a cluster take cs consecutive row
    // tiles of the same column tile at the same time: the leader loads the shared right-operand tile
    // once and multicasts it into every CTA's stage (half the right operand's traffic per SM at
    // cs = 2), each CTA loads its own left-operand rows.  A stage is free again when every CTA of the
    // cluster has consumed it: each MMA issuer's commit arrives on every CTA's `empty` barrier.
    const int cs = (int)cluster_size(), crank = (int)cluster_rank();
    const int nclu = gridDim.x / cs, cid = blockIdx.x / cs;
    const uint16_t cmask = (uint16_t)((1u << cs) - 1u);
    const int mtc = ((R + BM - 1) / BM + cs - 1) / cs;  // row-tile groups of the cluster
    const int tiles = mtc * ntn;                          // cluster tiles (row-tile group, column tile)

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&full[S + s], 1);
            mbar_init(&empty[s], PAIR ? 1 : cs);
        }
        for (int p = 0; p < 4; ++p) {
            mbar_init(&pfull[p], 1);
            mbar_init(&pfree[p], PAIR ? 8 : 4);  // pair: the release of both CTAs' four epilogue warps
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mAh)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mBh)) : "memory");
    }
    if (warp == 1) {
        if constexpr (PAIR) {
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)), "r"(512)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)), "r"(512)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
    }
    fence_before();
    if (cs > 1) cluster_sync_all();  // every CTA's barriers exist before a peer signals them
    else __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_holder;
    if (warp < 4) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegsCtl));
    else asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kRegsEpi));

    // ---- MMA issuers (in the pair's leader only in the pair form): fills of parity `own`
    auto issue_fills = [&](const int own) {
        int q = 0, lt = 0;
        uint32_t par = 0;  // bit s: parity of the next phase of full[own][s]
        bool ok = !PAIR || crank == 0;
        for (int tile = cid; tile < tiles && ok; tile += nclu, ++lt) {
            const int g = lt & 1, kg = lt >> 1;
            for (int kc = 0; kc < nk; ++kc, ++q) {
                const int s = q % S, ps = kc / kPromote, r = ps & 1, p = 2 * g + r;
                const int uses = kg * ((npc + 1 - r) >> 1) + (ps >> 1);  // earlier fills of buffer p
                const bool first = kc % kPromote == 0;                    // this chunk starts a fill
                const bool last = kc % kPromote == kPromote - 1 || kc == nk - 1;
                if (r != own) continue;  // the other issuer's chunk
                const uint32_t ph = (par >> s) & 1u;
                par ^= 1u << s;
                if (!mbar_wait(&full[own * S + s], ph) || (first && uses >= 1 && !mbar_wait(&pfree[p], (uses - 1) & 1))) {
                    atomicExch(err, 1);
                    *(volatile int*)abort_flag = 1;
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t d = tmem + (uint32_t)(p * BN);
                const uint32_t sa = smem_u32(base + s * SB);
                const uint64_t ah = sw128_desc(sa), al = sw128_desc(sa + BM * BK * 4);
                const uint64_t bh = sw128_desc(sa + 2 * BM * BK * 4), bl = sw128_desc(sa + 2 * BM * BK * 4 + BN * BK * 4);
                if constexpr (PAIR) {
                    const uint64_t bh2 = sw128_desc(sa + 2 * BM * BK * 4), bl2 = sw128_desc(sa + 2 * BM * BK * 4 + 64 * BK * 4);
#pragma unroll
                    for (int kk = 0; kk < BK / 8; ++kk) {
                        const uint64_t o = (uint64_t)(kk * 32) >> 4;
                        mma_tf32_pair(d, ah + o, bl2 + o, IDESC, (kk || !first) ? 1u : 0u);
                        mma_tf32_pair(d, al + o, bh2 + o, IDESC, 1u);
                    }
#pragma unroll
                    for (int kk = 0; kk < BK / 8; ++kk) {
                        const uint64_t o = (uint64_t)(kk * 32) >> 4;
                        mma_tf32_pair(d, ah + o, bh2 + o, IDESC, 1u);
                    }
                    mma_commit_pair_mc(&empty[s], cmask);
                    if (last) mma_commit_pair_mc(&pfull[p], cmask);
                } else {
#pragma unroll
                    for (int kk = 0; kk < BK / 8; ++kk) {
                        const uint64_t o = (uint64_t)(kk * 32) >> 4;
                        mma_tf32(d, ah + o, bl + o, IDESC, (kk || !first) ? 1u : 0u);
                        mma_tf32(d, al + o, bh + o, IDESC, 1u);
                    }
#pragma unroll
                    for (int kk = 0; kk < BK / 8; ++kk) {
                        const uint64_t o = (uint64_t)(kk * 32) >> 4;
                        mma_tf32(d, ah + o, bh + o, IDESC, 1u);
                    }
                    if (cs == 1) mma_commit(&empty[s]);
                    else mma_commit_mc(&empty[s], cmask);
                    if (last) mma_commit(&pfull[p]);
                }
            }
        }
    };

    if (threadIdx.x == 0) {
        // ---- TMA producer
        int q = 0;
        bool ok = true;
        uint32_t fpar = 0, lastr = 0;  // phases begun on full[r][s] (bit r S + s, mod 2); owner of stage s's last chunk
        for (int tile = cid; tile < tiles && ok; tile += nclu) {
            const int mg = tile / ntn, n0 = (tile - mg * ntn) * BN, mt = mg * cs + crank;
            for (int kc = 0; kc < nk; ++kc, ++q) {
                const int s = q % S, r = (kc / kPromote) & 1;
                if (q >= S && !mbar_wait(&empty[s], ((q / S) - 1) & 1)) {
                    atomicExch(err, 1);
                    *(volatile int*)abort_flag = 1;
                    ok = false;
                    break;
                }
                if (*(volatile int*)abort_flag) {
                    ok = false;
                    break;
                }
                unsigned char* st = base + s * SB;
                const int ay = (mt * nk + kc) * BM;
                uint64_t* fb0 = &full[r * S + s];  // the barrier of the issuer that consumes this chunk
                fpar ^= 1u << (r * S + s);
                lastr = (lastr & ~(1u << s)) | ((uint32_t)r << s);
                if constexpr (PAIR) {
                    // both CTAs' bytes land on the leader's barrier: A rows of this CTA, B^T rows
                    // n0 + 64 rank .. + 63 (this CTA's half of the tile's columns)
                    if (crank == 0) mbar_expect_tx(fb0, 2 * SB);
                    const uint32_t fb = cluster_addr(fb0, 0);
                    tma_load_2d_pair(st, &mAh, fb, 0, ay);
                    tma_load_2d_pair(st + BM * BK * 4, &mAl, fb, 0, ay);
                    tma_load_2d_pair(st + 2 * BM * BK * 4, &mBh, fb, kc * BK, n0 + 64 * crank);
                    tma_load_2d_pair(st + 2 * BM * BK * 4 + 64 * BK * 4, &mBl, fb, kc * BK, n0 + 64 * crank);
                } else {
                    mbar_expect_tx(fb0, SB);
                    tma_load_2d(st, &mAh, fb0, 0, ay);  // row tiles past R read zeros
                    tma_load_2d(st + BM * BK * 4, &mAl, fb0, 0, ay);
                    if (cs == 1) {
                        tma_load_2d(st + 2 * BM * BK * 4, &mBh, fb0, kc * BK, n0);
                        tma_load_2d(st + 2 * BM * BK * 4 + BN * BK * 4, &mBl, fb0, kc * BK, n0);
                    } else if (crank == 0) {
                        // the same barrier offset in every CTA of the cluster: the chunk's owner is the same there
                        tma_load_2d_mc(st + 2 * BM * BK * 4, &mBh, fb0, kc * BK, n0, cmask);
                        tma_load_2d_mc(st + 2 * BM * BK * 4 + BN * BK * 4, &mBl, fb0, kc * BK, n0, cmask);
                    }
                }
            }
        }
        if (!PAIR || crank == 0) {
            for (int s = 0; s < S && s < q; ++s) {  // the last chunk of every stage lands before exit
                const int r = (int)((lastr >> s) & 1u);
                if (!mbar_wait(&full[r * S + s], ((fpar >> (r * S + s)) & 1u) ^ 1u)) {
                    atomicExch(err, 1);
                    break;
                }
            }
        }
        if (cs > 1) {
            // every CTA's release of the last use of each stage has arrived here, so no peer signals
            // this CTA's barriers after it exits
            for (int k = (q > S ? q - S : 0); k < q; ++k) {
                if (!mbar_wait(&empty[k % S], (k / S) & 1)) {
                    atomicExch(err, 1);
                    break;
                }
            }
        }
    } else if (threadIdx.x == 32) {
        issue_fills(0);
    } else if (threadIdx.x == 64) {
        issue_fills(1);
    }
    if (warp >= 4) {
        // ---- epilogue groups
        const int g = (warp - 4) >> 2, sub = warp & 3, gt = threadIdx.x - 128 - 128 * g;
        float4* coltab = reinterpret_cast<float4*>(base + pp_coltab_offset()) + g * 128;
        float* w1tab = reinterpret_cast<float*>(base + pp_w1tab_offset()) + g * 128 * kFinalCols;
        const uint32_t lane_base = (uint32_t)(sub * 32) << 16;
        bool ok = true;
        int lt = g;
        for (int tile = cid + g * nclu; tile < tiles; tile += 2 * nclu, lt += 2) {
            const int kg = lt >> 1;
            const int mg = tile / ntn, mt = mg * cs + crank, m0 = mt * BM, n0 = (tile - mg * ntn) * BN;
            bool uniform = false;
            if constexpr (EPI != 0) {
                group_bar(g);  // the group's previous tile no longer reads the tables
                const int dom0 = m0 / epi.rows_per_dom;
                uniform = R > 0 && dom0 == (min(m0 + BM, R) - 1) / epi.rows_per_dom;
                if (uniform) {
                    const int col = n0 + gt;
                    float4 qv = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (col < N)
                        qv = make_float4(epi.hs[(int64_t)dom0 * epi.hidden + epi.hoff + col],
                                         epi.hd[(int64_t)dom0 * epi.hidden + epi.hoff + col], epi.bias[col], 0.f);
                    coltab[gt] = qv;
                }
                if constexpr (EPI == 2) {
                    // all 16 loads of a thread in flight together, then the shared-memory stores
                    constexpr int PER = BN * kFinalCols / 128;
                    float wv[PER];
#pragma unroll
                    for (int it = 0; it < PER; ++it) {
                        const int idx = gt + it * 128;
                        const int j = idx / kFinalCols, c = idx - j * kFinalCols;
                        const int col = n0 + j;
                        wv[it] = (col < N && c < epi.n0) ? __ldg(epi.W1 + (int64_t)col * epi.n0 + c) : 0.f;
                    }
#pragma unroll
                    for (int it = 0; it < PER; ++it) w1tab[gt + it * 128] = wv[it];
                }
                group_bar(g);
            }
            if constexpr (EPI == 3) {
                // the forward level this warp's rows read in the epilogue: into L2 while the tile's MMAs
                // run (one 128-byte line per column of the 32-row block; lane L takes columns L + 32 q)
                const int r0 = m0 + sub * 32;
                if (r0 < R) {
                    // blocked layout: the warp's 32 rows of one 32-column chunk are 4 KB contiguous
                    const int rl = epi.rlev_shared ? (r0 % epi.rows_per_dom) : r0;
                    const int nkl = (N + 31) >> 5;
#pragma unroll
                    for (int q = 0; q < BN / 32; ++q) {
                        const int c0 = n0 + 32 * q;
                        if (c0 < N) asm volatile("prefetch.global.L2 [%0];" ::"l"(epi.rlev + blk_index(rl, c0, nkl) + 32 * lane));
                    }
                }
            }
            float acc[BN];
#pragma unroll
            for (int j = 0; j < BN; ++j) acc[j] = 0.f;
            for (int ps = 0; ps < npc; ++ps) {
                const int r = ps & 1, p = 2 * g + r;
                const int uses = kg * ((npc + 1 - r) >> 1) + (ps >> 1);
                bool good = ok && !*(volatile int*)abort_flag && mbar_wait(&pfull[p], uses & 1);
                ok = __all_sync(0xffffffffu, good);  // TMEM loads are warp-collective: decide per warp
                if (ok) {
                    fence_after();
#pragma unroll
                    for (int c0 = 0; c0 < BN; c0 += 64) {
                        float v[64];
                        tmem_ld64(tmem + lane_base + (uint32_t)(p * BN + c0), v);
#pragma unroll
                        for (int j = 0; j < 64; ++j) acc[c0 + j] += v[j];
                    }
                    fence_before();
                }
                __syncwarp();
                if (ok && lane == 0) {
                    if (PAIR && crank != 0) mbar_arrive_cluster(cluster_addr(&pfree[p], 0));  // the leader issues the MMAs
                    else mbar_arrive(&pfree[p]);
                }
            }
            if (!ok) atomicExch(err, 1);
            const int row = m0 + sub * 32 + lane;
            const bool live = ok && row < R;
            if constexpr (EPI == 0) {
                if (live) {
#pragma unroll
                    for (int j = 0; j < BN; ++j)
                        if (n0 + j < N) C[(int64_t)row * ldc + n0 + j] = acc[j];
                }
            } else {
                // EPI 1 has no W_1 table: its per-warp staging tiles (2 KB each) take that space
                float* stg = w1tab + sub * 512;
                if constexpr (EPI == 3) {
                    const RevPre pre = rev_preload(epi, row, R);
                    if (epi.rows_per_dom % 32 != 0) pp_row_epilogue_rev<false, false>(acc, coltab, stg, epi, row, ok, n0, N, R, pre);
                    else if (uniform) pp_row_epilogue_rev<true, true>(acc, coltab, stg, epi, row, ok, n0, N, R, pre);
                    else pp_row_epilogue_rev<false, true>(acc, coltab, stg, epi, row, ok, n0, N, R, pre);
                } else {
                    if (uniform) pp_row_epilogue<EPI, true>(acc, coltab, w1tab, stg, epi, row, ok, n0, N, R);
                    else pp_row_epilogue<EPI, false>(acc, coltab, w1tab, stg, epi, row, ok, n0, N, R);
                }
            }
        }
    }
    fence_before();
    if (cs > 1) cluster_sync_all();  // no CTA leaves while a peer may still write its stages
    else __syncthreads();
    if (warp == 1) {
        __syncwarp();
        fence_after();
        if constexpr (PAIR) asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
        else asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

}  // namespace tc
