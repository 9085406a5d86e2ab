// Register-tiled shared-memory products used by the fused kernels (FP32 CUDA cores): each thread
// owns a TR x 4 tile of the output and streams K, so a multiply-add costs (TR + 4) / (4 TR) loads.
#pragma once

__host__ __device__ __forceinline__ int ru4(int x) { return (x + 3) & ~3; }

// Rows per register tile: 4 unless the 4 x 4 tiles would leave more than half of the CTA's threads
// idle; then 1 (short, wide products such as an output layer's chain level).
template <int NT>
__device__ __forceinline__ bool tile4(int M, int N) {
    return ((M + 3) >> 2) * ((N + 3) >> 2) * 2 >= NT;
}

// C [M x N] (ld ldc) = A [M x K] (ld lda) * B [K x N] (ld ldb, ldb % 4 == 0, 16-byte aligned, padding
// columns finite): TR x 4 register tiles, one float4 of B and TR A values per k.
template <int NT, int TR>
__device__ __forceinline__ void gemm_shared_a_t(const float* __restrict__ A, int lda, const float* __restrict__ B, int ldb,
                                                float* __restrict__ C, int ldc, int M, int K, int N) {
    const int tilesM = (M + TR - 1) / TR, tilesN = (N + 3) >> 2;
    for (int tt = threadIdx.x; tt < tilesM * tilesN; tt += NT) {
        const int tm = tt / tilesN, tn = tt - tm * tilesN;
        const int i0 = tm * TR, c0 = tn << 2;
        const float* ar[TR];
#pragma unroll
        for (int r = 0; r < TR; ++r) ar[r] = A + min(i0 + r, M - 1) * lda;
        const float* bp = B + c0;
        float acc[TR][4];
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[r][q] = 0.f;
#pragma unroll 4
        for (int j = 0; j < K; ++j) {
            const float4 b = *reinterpret_cast<const float4*>(bp + j * ldb);
#pragma unroll
            for (int r = 0; r < TR; ++r) {
                const float x = ar[r][j];
                acc[r][0] = fmaf(x, b.x, acc[r][0]);
                acc[r][1] = fmaf(x, b.y, acc[r][1]);
                acc[r][2] = fmaf(x, b.z, acc[r][2]);
                acc[r][3] = fmaf(x, b.w, acc[r][3]);
            }
        }
#pragma unroll
        for (int r = 0; r < TR; ++r) {
            if (i0 + r >= M) break;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (c0 + q < N) C[(i0 + r) * ldc + c0 + q] = acc[r][q];
        }
    }
}
template <int NT>
__device__ __forceinline__ void gemm_shared_a(const float* __restrict__ A, int lda, const float* __restrict__ B, int ldb,
                                              float* __restrict__ C, int ldc, int M, int K, int N) {
    if (tile4<NT>(M, N)) gemm_shared_a_t<NT, 4>(A, lda, B, ldb, C, ldc, M, K, N);
    else gemm_shared_a_t<NT, 1>(A, lda, B, ldb, C, ldc, M, K, N);
}

// Stacked rows of all domains: C[(g*rows + i)*ldc + k] = sum_j A_g[i][j] s_g[j] B[j][k] for g < gcount,
// A_g = Ab + g*a_gs + i*lda (a_gs = 0: one shared A), s_g = sb + g*s_gs, B [K][N] (ld ldb).  4 x 4 tiles.
template <int NT, int TR>
__device__ __forceinline__ void gemm_stacked_scaled_t(const float* __restrict__ Ab, int a_gs, int lda, const float* __restrict__ sb,
                                                      int s_gs, const float* __restrict__ B, int ldb, float* __restrict__ C,
                                                      int ldc, int gcount, int rows, int K, int N) {
    const int M = gcount * rows;
    const int tilesM = (M + TR - 1) / TR, tilesN = (N + 3) >> 2;
    for (int tt = threadIdx.x; tt < tilesM * tilesN; tt += NT) {
        const int tm = tt / tilesN, tn = tt - tm * tilesN;
        const int i0 = tm * TR, c0 = tn << 2;
        const float* ap[TR];
        const float* sp[TR];
#pragma unroll
        for (int r = 0; r < TR; ++r) {
            const int R = min(i0 + r, M - 1), g = R / rows, i = R - g * rows;
            ap[r] = Ab + g * a_gs + i * lda;
            sp[r] = sb + g * s_gs;
        }
        const int cc[4] = {min(c0, N - 1), min(c0 + 1, N - 1), min(c0 + 2, N - 1), min(c0 + 3, N - 1)};
        float acc[TR][4];
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[r][q] = 0.f;
#pragma unroll 2
        for (int j = 0; j < K; ++j) {
            const float* brow = B + j * ldb;
            const float b[4] = {brow[cc[0]], brow[cc[1]], brow[cc[2]], brow[cc[3]]};
#pragma unroll
            for (int r = 0; r < TR; ++r) {
                const float x = ap[r][j] * sp[r][j];
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[r][q] = fmaf(x, b[q], acc[r][q]);
            }
        }
#pragma unroll
        for (int r = 0; r < TR; ++r) {
            if (i0 + r >= M) break;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (c0 + q < N) C[(i0 + r) * ldc + c0 + q] = acc[r][q];
        }
    }
}
// One output element per thread (products too small for the CTA to fill even with 1 x 4 tiles).
template <int NT>
__device__ __forceinline__ void gemm_stacked_scaled_1(const float* __restrict__ Ab, int a_gs, int lda, const float* __restrict__ sb,
                                                      int s_gs, const float* __restrict__ B, int ldb, float* __restrict__ C,
                                                      int ldc, int gcount, int rows, int K, int N) {
    const int M = gcount * rows;
    for (int idx = threadIdx.x; idx < M * N; idx += NT) {
        const int R = idx / N, k = idx - R * N, g = R / rows, i = R - g * rows;
        const float* a = Ab + g * a_gs + i * lda;
        const float* sv = sb + g * s_gs;
        float acc = 0.f;
        for (int j = 0; j < K; ++j) acc = fmaf(a[j] * sv[j], B[j * ldb + k], acc);
        C[R * ldc + k] = acc;
    }
}
template <int NT>
__device__ __forceinline__ void gemm_stacked_scaled(const float* __restrict__ Ab, int a_gs, int lda, const float* __restrict__ sb,
                                                    int s_gs, const float* __restrict__ B, int ldb, float* __restrict__ C,
                                                    int ldc, int gcount, int rows, int K, int N) {
    const int M = gcount * rows;
    if (tile4<NT>(M, N))
        gemm_stacked_scaled_t<NT, 4>(Ab, a_gs, lda, sb, s_gs, B, ldb, C, ldc, gcount, rows, K, N);
    else if (M * ((N + 3) >> 2) * 2 >= NT)
        gemm_stacked_scaled_t<NT, 1>(Ab, a_gs, lda, sb, s_gs, B, ldb, C, ldc, gcount, rows, K, N);
    else
        gemm_stacked_scaled_1<NT>(Ab, a_gs, lda, sb, s_gs, B, ldb, C, ldc, gcount, rows, K, N);
}


// ---- slab mode (fused kernels whose working set lives in global memory, 256 threads): the wide
// products are staged through shared-memory tiles (kSlabTileFloats floats of dynamic shared memory):
// 128 x 128 outputs per pass, an 8 x 8 register tile per thread (rows 4ty..4ty+3 and 64+4ty..,
// columns likewise), K in slices of 32 held transposed ([k][row], rows padded to 132 floats), two
// slices in flight: the next slice is copied element by element with cp.async (the slab rows are
// odd-padded, so 4-byte copies) while the current one is multiplied.
constexpr int kSlabLd = 132;
constexpr int kSlabStage = 2 * 32 * kSlabLd + 32;  // A slice, B slice, 32 slopes
constexpr int kSlabTileFloats = 2 * kSlabStage;

__device__ __forceinline__ void slab_cp4(float* dst, const float* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void slab_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void slab_wait_all_but_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void slab_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ int slab_row(int base, int ty, int r) { return base + (r < 4 ? 4 * ty + r : 64 + 4 * ty + r - 4); }

// One 128 x 128 output tile, K streamed in slices of 32 through two stages.  NN: C = (A diag(s)) B with
// B [Kd][N] row-major, the scaled value a * s formed before its multiply-add; NT: C = A B^T with B
// [N][Kd].  acc is initialised by the caller; per element the multiply-adds run over k ascending.
template <bool NN>
__device__ __forceinline__ void slab_tile(const float* A, int lda, const float* sv, const float* B, int ldb, int M, int N,
                                          int Kd, int mt, int nt, float* tiles, float (&acc)[8][8]) {
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    auto stage = [&](int buf, int k0) {
        float* At = tiles + buf * kSlabStage;
        float* Bt = At + 32 * kSlabLd;
        float* St = Bt + 32 * kSlabLd;
#pragma unroll 4
        for (int u = 0; u < 16; ++u) {
            const int idx = tid + 256 * u;
            const int ii = idx >> 5, ka = idx & 31;
            float* da = At + ka * kSlabLd + ii;
            if (k0 + ka < Kd && mt + ii < M) slab_cp4(da, A + (int64_t)(mt + ii) * lda + k0 + ka);
            else *da = 0.f;
            if constexpr (NN) {
                const int kb = idx >> 7, jj = idx & 127;
                float* db = Bt + kb * kSlabLd + jj;
                if (k0 + kb < Kd && nt + jj < N) slab_cp4(db, B + (int64_t)(k0 + kb) * ldb + nt + jj);
                else *db = 0.f;
            } else {
                float* db = Bt + ka * kSlabLd + ii;
                if (k0 + ka < Kd && nt + ii < N) slab_cp4(db, B + (int64_t)(nt + ii) * ldb + k0 + ka);
                else *db = 0.f;
            }
        }
        if constexpr (NN) {
            if (tid < 32) {
                if (k0 + tid < Kd) slab_cp4(St + tid, sv + k0 + tid);
                else St[tid] = 0.f;
            }
        }
        slab_commit();
    };
    const int ns = (Kd + 31) >> 5;
    __syncthreads();  // both stages free (previous tile or caller)
    stage(0, 0);
    for (int sidx = 0; sidx < ns; ++sidx) {
        if (sidx + 1 < ns) {
            stage((sidx + 1) & 1, (sidx + 1) * 32);
            slab_wait_all_but_one();
        } else {
            slab_wait_all();
        }
        __syncthreads();  // slice sidx visible to every thread
        const float* At = tiles + (sidx & 1) * kSlabStage;
        const float* Bt = At + 32 * kSlabLd;
        const float* St = Bt + 32 * kSlabLd;
        const int kn = min(32, Kd - sidx * 32);
        for (int kk = 0; kk < kn; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(At + kk * kSlabLd + 4 * ty);
            const float4 a1 = *reinterpret_cast<const float4*>(At + kk * kSlabLd + 64 + 4 * ty);
            const float4 b0 = *reinterpret_cast<const float4*>(Bt + kk * kSlabLd + 4 * tx);
            const float4 b1 = *reinterpret_cast<const float4*>(Bt + kk * kSlabLd + 64 + 4 * tx);
            float ar[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            if constexpr (NN) {
                const float s = St[kk];
#pragma unroll
                for (int r = 0; r < 8; ++r) ar[r] = ar[r] * s;
            }
            const float br[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[r][q] = fmaf(ar[r], br[q], acc[r][q]);
        }
        __syncthreads();  // slice sidx no longer read: its stage may be refilled
    }
    slab_wait_all();  // nothing left in flight (also when Kd == 0)
}

// C[i][j] = (glo_i + ghi_i) b_j + sum_k A[i][k] B[j][k] for i < M, j < N (A [M][Kd], B [N][Kd]).  Per
// element the same operations in the same order as the register-tiled loop of the reverse sweep's
// wide levels (the intercept term first, then k ascending), so the results are identical.
__device__ __forceinline__ void gemm_nt_tiled256(const float* A, int lda, const float* B, int ldb, float* C, int ldc, int M,
                                                 int N, int Kd, const float* glo, const float* ghi, const float* bvec,
                                                 float* tiles) {
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    for (int mt = 0; mt < M; mt += 128) {
        for (int nt = 0; nt < N; nt += 128) {
            float acc[8][8];
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int i = min(slab_row(mt, ty, r), M - 1);
                const float gk = glo[i] + ghi[i];
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[r][q] = gk * bvec[min(slab_row(nt, tx, q), N - 1)];
            }
            slab_tile<false>(A, lda, nullptr, B, ldb, M, N, Kd, mt, nt, tiles, acc);
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int i = slab_row(mt, ty, r);
                if (i >= M) continue;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int j = slab_row(nt, tx, q);
                    if (j < N) C[(int64_t)i * ldc + j] = acc[r][q];
                }
            }
        }
    }
    __syncthreads();
}

// C[i][k] = sum_j (A[i][j] s_j) B[j][k] for i < M, k < N, j < Kd (B row-major [Kd][N]); per element the
// same operations and order as gemm_stacked_scaled_t (the scaled A value formed first, j ascending).
__device__ __forceinline__ void gemm_nn_scaled_tiled256(const float* A, int lda, const float* sv, const float* B, int ldb,
                                                        float* C, int ldc, int M, int Kd, int N, float* tiles) {
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    for (int mt = 0; mt < M; mt += 128) {
        for (int nt = 0; nt < N; nt += 128) {
            float acc[8][8];
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[r][q] = 0.f;
            slab_tile<true>(A, lda, sv, B, ldb, M, N, Kd, mt, nt, tiles, acc);
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int i = slab_row(mt, ty, r);
                if (i >= M) continue;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int k = slab_row(nt, tx, q);
                    if (k < N) C[(int64_t)i * ldc + k] = acc[r][q];
                }
            }
        }
    }
    __syncthreads();
}
