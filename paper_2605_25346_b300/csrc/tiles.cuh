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

