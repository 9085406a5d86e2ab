// Staged forward pass for wide controllers (widths beyond the fused kernel's shared memory).
//
// Domains are processed in chunks; per closed-loop step (Alg. 2, closed loop of Sec. IV-E) the
// phases are separate kernels over the whole chunk, with per-domain state in global scratch:
//   view     FP64 TM -> FP32 view (remainder widened to cover the cast)
//   for each target layer l = 1..L:
//     init   kappa = b_l; first chain level from the shared W_l: Lambda^+/- intercepts with the
//            relaxation of layer l-1 and A = W_l diag(s_{l-1}) per domain
//     levels Lambda <- A W_m (batched GEMM, shared W_m; tensor cores or CUDA cores), then the
//            next level's intercepts and A = Lambda diag(s_{m-1}) (row reductions)      (Thm. 2)
//     proj   G = Lambda_x P, a = Lambda_x c, R = Lambda_x (x) I, concretisation with the
//            split dual and the outward margin (Thm. 3), or the controller TM
//
// The intercepts kappa are summed across chain levels in FP64 and the concretisation adds its terms
// in FP64 (the per-level and per-row partial sums stay FP32); pre-activation bounds are rounded to
// FP32 outward and the controller TM stays FP64.  Accumulating kappa in FP32 was the largest source
// of deviation from FP64 arithmetic over long horizons.
//     relax  split clipping / dual records, shared-slope relaxation              (Sec. IV-C)
//   dyn      FP64 dynamics on the TM and EvalInt (Alg. 2)
#pragma once
#include "common.cuh"

struct WideArgs {
    NetDesc net;
    const float* W;
    const float* b;
    const double* A;
    const double* B;
    const double* e;
    const double* eoff;  // [D][H][n] per-step offsets of the dynamics or null
    const double* lo0;
    const double* hi0;
    int64_t d0;  // first domain of the chunk
    int Dc;      // domains in the chunk
    const int64_t* sp_row;
    const SplitRec* sp;
    const float* beta;
    const float* alpha;
    int mode;
    float rho;
    double box_margin;
    double* lo;
    double* hi;
    double* V;
    uint32_t* status;
    float* alpha_used;
    // chunk scratch (index = domain within the chunk)
    double *c, *P, *Ilo, *Ihi, *v, *w, *vacc;
    int* cursor;
    uint32_t* st;
    float *cf, *Pf, *Ilof, *Ihif, *vf;  // vf: [Dc][n+1] (last = wf)
    float *hl, *hu, *hs, *hd;           // [Dc][hidden]
    double *klo, *khi;                  // [Dc][maxw] intercepts, accumulated in FP64
    float *G, *sa, *sRlo, *sRhi, *sS;   // [Dc][maxw][n], [Dc][maxw]
    double *cu, *Iulo, *Iuhi;           // [Dc][m] controller TM, FP64
    int64_t lam_stride;                 // floats per domain in a Lambda buffer
    // rigorous mode (CUDA-core chain only): rounding-error bounds carried with the intercepts
    int rigorous;
    float* xmax;   // [Dc][n] bound on |x| over the Taylor model (rounded up)
    float* hq;     // [Dc][hidden] q_m = |W_m| hmax_{m-1} per neuron of hidden layer m (rounded up)
    float* xscale; // [Dc] Taylor-model scale of the step (DR_STATUS_MARGIN_BIT)
    double* kerr;  // [Dc][maxw] accumulated error bound of each target row's linear bound
    // keep mode (the staged reverse sweep reads these back; null otherwise).  The host points
    // cf/Pf/Ilof/Ihif and hl/hu/hs/hd at the step's slot of the keep store as well.
    float* vsnap;        // [Dc][L][n+1] dual vector (and w) seen by target l's concretisation
    float *hl0, *hu0;    // [Dc][hidden] pre-activation bounds before the split clipping
    float* sph;          // [nnz] value h of every split constraint recorded in this pass
    float *Gk, *LXk;     // [Dc][krows][n] G = Lambda_x P and Lambda_x of every target
    int krows, koff;     // krows = hidden + m; koff = row offset of the target being projected
    double* tape;        // [Dc][H+1][n*n + 4n + 2] FP64 TM (P, c, Ilo, Ihi, v, w, cursor) per step
};

// Rigorous mode.  For IEEE FP32 with round-to-nearest (the CUDA-core FMA chains used in this mode),
// a sum or dot product of K terms computed in any order errs by at most gamma(K) times the sum of the
// absolute values of its terms, gamma(K) = K u / (1 - K u), u = 2^-24 (the standard forward error
// bound of recursive summation).  Each bound below takes K + 2 to also cover the rounding of the
// operands' products and the final addition.
__device__ __forceinline__ double gamma_k(int K) {
    const double ku = (double)(K + 2) * 5.9604644775390625e-8;  // (K + 2) * 2^-24
    return ku / (1.0 - ku);
}
// Absolute error weight of one column j of a chain level: the level's product Lambda_s W_m (K = n_m
// terms per entry, each bounded by |Lambda_ij| s_j |W_m[j,k]| hmax_{m-1}[k], summed over k into q_j)
// and its intercept sums (terms |Lambda_ij| d_j and |Lambda_ij| s_j |b_j|).
__device__ __forceinline__ float err_weight(float s, float d, float b, float q, double gk) {
    return (float)(gk * ((double)s * ((double)q + fabs((double)b)) + (double)d)) * 1.0009765625f;  // (1 + 2^-10): rounding of this product
}

__device__ __forceinline__ float warp_sum(float x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// a1 + box_0: seed the TM of every domain in the chunk.
__global__ void k_w_seed(const WideArgs a) {
    const NetDesc& N = a.net;
    const int n = N.n, H = N.H;
    const int64_t total = (int64_t)a.Dc * n;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int d = (int)(idx / n), i = (int)(idx - (int64_t)d * n);
        const int64_t dom = a.d0 + d;
        const double lo = a.lo0[dom * n + i], hi = a.hi0[dom * n + i];
        a.c[idx] = 0.5 * (lo + hi);
        for (int k = 0; k < n; ++k) a.P[(int64_t)d * n * n + i * n + k] = (i == k) ? 0.5 * (hi - lo) : 0.0;
        a.Ilo[idx] = 0.0;
        a.Ihi[idx] = 0.0;
        a.v[idx] = 0.0;
        if (a.lo) a.lo[(dom * (H + 1)) * n + i] = lo;
        if (a.hi) a.hi[(dom * (H + 1)) * n + i] = hi;
        if (i == 0) {
            a.w[d] = 0.0;
            a.vacc[d] = 0.0;
            a.st[d] = 0u;
            a.cursor[d] = a.sp_row ? (int)a.sp_row[dom] : 0;
        }
    }
}

// FP32 view of each domain's TM; one block per domain.
__global__ void k_w_view(const WideArgs a) {
    __shared__ unsigned int xs_bits;  // max over rows of the TM scale's row sums (non-negative floats)
    const int n = a.net.n, d = blockIdx.x;
    const double* P = a.P + (int64_t)d * n * n;
    float* Pf = a.Pf + (int64_t)d * n * n;
    if (threadIdx.x == 0) xs_bits = 0u;
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) Pf[idx] = (float)P[idx];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        // row i of tm_scale (common.cuh), in its order; the rows' maximum is taken below
        float rs = fabsf((float)a.c[(int64_t)d * n + i]) +
                   fmaxf(fabsf((float)a.Ilo[(int64_t)d * n + i]), fabsf((float)a.Ihi[(int64_t)d * n + i]));
        for (int k = 0; k < n; ++k) rs += fabsf((float)P[i * n + k]);
        if (!isnan(rs)) atomicMax(&xs_bits, __float_as_uint(rs));  // as fmaxf: a NaN row is skipped
        const double ci = a.c[(int64_t)d * n + i];
        const float cf = (float)ci;
        double dev = 0.0;
        for (int k = 0; k < n; ++k) dev += fabs(P[i * n + k] - (double)(float)P[i * n + k]);
        const double dc = ci - (double)cf;
        a.cf[(int64_t)d * n + i] = cf;
        a.Ilof[(int64_t)d * n + i] = __double2float_rd(a.Ilo[(int64_t)d * n + i] + dc - dev);
        a.Ihif[(int64_t)d * n + i] = __double2float_ru(a.Ihi[(int64_t)d * n + i] + dc + dev);
        if (a.rigorous) {
            // |x| <= |c_f| + sum |P_f| + max |I_f| over the FP32 view (whose remainder covers the cast)
            double mag = fabs((double)cf) + fmax(fabs((double)a.Ilof[(int64_t)d * n + i]), fabs((double)a.Ihif[(int64_t)d * n + i]));
            for (int k = 0; k < n; ++k) mag += fabs((double)(float)P[i * n + k]);
            a.xmax[(int64_t)d * n + i] = __double2float_ru(mag * (1.0 + 1e-12));
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double dv = 0.0;
        float* vf = a.vf + (int64_t)d * (n + 1);
        for (int k = 0; k < n; ++k) {
            vf[k] = (float)a.v[(int64_t)d * n + k];
            dv += fabs(a.v[(int64_t)d * n + k] - (double)vf[k]);
        }
        vf[n] = __double2float_ru(a.w[d] + dv);
        // tm_scale of the TM with its rows spread over the threads: this GPU's FP64 pipe (which
        // also converts FP64 to FP32) takes as long for one thread's instruction as for a warp's
        a.xscale[d] = __uint_as_float(xs_bits);
        if (a.vsnap)
            for (int k = 0; k <= n; ++k) a.vsnap[(int64_t)d * a.net.L * (n + 1) + k] = vf[k];
    }
}

// Keep mode: the FP64 TM of every domain of the chunk at the start of step t (t = H: after the
// last step) into the chunk's tape, laid out as P, c, Ilo, Ihi, v, w, split cursor.
__global__ void k_w_tape(const WideArgs a, int t) {
    const int n = a.net.n, d = blockIdx.x, H = a.net.H;
    const int ts = n * n + 4 * n + 2;
    double* tp = a.tape + ((int64_t)d * (H + 1) + t) * ts;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) tp[idx] = a.P[(int64_t)d * n * n + idx];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        tp[n * n + i] = a.c[(int64_t)d * n + i];
        tp[n * n + n + i] = a.Ilo[(int64_t)d * n + i];
        tp[n * n + 2 * n + i] = a.Ihi[(int64_t)d * n + i];
        tp[n * n + 3 * n + i] = a.v[(int64_t)d * n + i];
    }
    if (threadIdx.x == 0) {
        tp[n * n + 4 * n] = a.w[d];
        tp[n * n + 4 * n + 1] = (double)a.cursor[d];
    }
}

// Target ell: kappa = b_ell and, for ell >= 2, the first chain level from the shared W_ell:
// intercepts with the relaxation of layer ell-1 and A = W_ell diag(s_{ell-1}) into Aout.
// One warp per (domain, row).
__global__ void k_w_chain_init(const WideArgs a, int ell, float* __restrict__ Aout) {
    const NetDesc& N = a.net;
    const int rows = N.w[ell];
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= (int64_t)a.Dc * rows) return;
    const int d = (int)(wid / rows), i = (int)(wid - (int64_t)d * rows);
    const float bi = a.b[N.boff[ell - 1] + i];
    if (ell == 1) {
        if (lane == 0) {
            a.klo[(int64_t)d * N.maxw + i] = (double)bi;
            a.khi[(int64_t)d * N.maxw + i] = (double)bi;
            if (a.rigorous) a.kerr[(int64_t)d * N.maxw + i] = 0.0;
        }
        return;
    }
    const int K = N.w[ell - 1];
    const float* Wrow = a.W + N.Woff[ell - 1] + (int64_t)i * K;
    const float* s = a.hs + (int64_t)d * N.hidden + N.hoff[ell - 1];
    const float* dd = a.hd + (int64_t)d * N.hidden + N.hoff[ell - 1];
    const float* bm = a.b + N.boff[ell - 2];
    const float* q = a.rigorous ? a.hq + (int64_t)d * N.hidden + N.hoff[ell - 1] : nullptr;
    const double gk = gamma_k(K);
    float* out = Aout + (int64_t)d * a.lam_stride + (int64_t)i * K;
    float spos = 0.f, sneg = 0.f, sb = 0.f, se = 0.f;
    for (int j = lane; j < K; j += 32) {
        const float x = Wrow[j];
        spos = fmaf(posf(x), dd[j], spos);
        sneg = fmaf(negf(x), dd[j], sneg);
        const float xs = x * s[j];
        sb = fmaf(xs, bm[j], sb);
        if (q) se = __fmaf_ru(fabsf(x), err_weight(s[j], dd[j], bm[j], q[j], gk), se);
        out[j] = xs;
    }
    spos = warp_sum(spos);
    sneg = warp_sum(sneg);
    sb = warp_sum(sb);
    if (q) se = warp_sum(se);
    if (lane == 0 && q) a.kerr[(int64_t)d * N.maxw + i] = (double)se * 1.0009765625;
    if (lane == 0) {
        a.khi[(int64_t)d * N.maxw + i] = (double)bi + (double)spos + (double)sb;
        a.klo[(int64_t)d * N.maxw + i] = (double)bi + (double)sneg + (double)sb;
    }
}

// After a GEMM level produced Lambda^(mm) (mm >= 1) in buf [d][i][k], k < n_mm: the intercepts of the
// relaxation of layer mm and, in place, A = Lambda diag(s_mm).  One warp per (domain, row).  With
// lev set, Lambda^(mm) itself is also kept (keep mode).
__global__ void k_w_level_epi(const WideArgs a, int ell, int mm, float* __restrict__ buf, float* __restrict__ lev) {
    const NetDesc& N = a.net;
    const int rows = N.w[ell], K = N.w[mm];
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= (int64_t)a.Dc * rows) return;
    const int d = (int)(wid / rows), i = (int)(wid - (int64_t)d * rows);
    const float* s = a.hs + (int64_t)d * N.hidden + N.hoff[mm];
    const float* dd = a.hd + (int64_t)d * N.hidden + N.hoff[mm];
    const float* bm = a.b + N.boff[mm - 1];
    const float* q = a.rigorous ? a.hq + (int64_t)d * N.hidden + N.hoff[mm] : nullptr;
    const double gk = gamma_k(K);
    float* row = buf + (int64_t)d * a.lam_stride + (int64_t)i * K;
    float spos = 0.f, sneg = 0.f, sb = 0.f, se = 0.f;
    for (int j = lane; j < K; j += 32) {
        const float x = row[j];
        spos = fmaf(posf(x), dd[j], spos);
        sneg = fmaf(negf(x), dd[j], sneg);
        const float xs = x * s[j];
        sb = fmaf(xs, bm[j], sb);
        if (q) se = __fmaf_ru(fabsf(x), err_weight(s[j], dd[j], bm[j], q[j], gk), se);
        if (lev) lev[tc::blk_index(wid, j, (K + 31) >> 5)] = x;
        row[j] = xs;
    }
    spos = warp_sum(spos);
    sneg = warp_sum(sneg);
    sb = warp_sum(sb);
    if (q) se = warp_sum(se);
    if (lane == 0 && q) a.kerr[(int64_t)d * N.maxw + i] += (double)se * 1.0009765625;
    if (lane == 0) {
        a.khi[(int64_t)d * N.maxw + i] += (double)spos + (double)sb;
        a.klo[(int64_t)d * N.maxw + i] += (double)sneg + (double)sb;
    }
}

// Batched C[d] = A[d] B with A[d] M x K (row-major, ld K), B K x N shared (row-major, ld N),
// C[d] M x N (ld N); CUDA-core FP32, 64x64 tiles, 4x4 per thread.
__global__ void __launch_bounds__(256) k_w_gemm_simt(const float* __restrict__ Ab, const float* __restrict__ B,
                                                     float* __restrict__ Cb, int M, int K, int N, int64_t stride) {
    __shared__ float As[16][64 + 4];
    __shared__ float Bs[16][64 + 4];
    const float* A = Ab + blockIdx.z * stride;
    float* C = Cb + blockIdx.z * stride;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int idx = threadIdx.x; idx < 64 * 16; idx += 256) {
            const int r = idx >> 4, q = idx & 15;
            const int gm = m0 + r, gk = k0 + q;
            As[q][r] = (gm < M && gk < K) ? A[(int64_t)gm * K + gk] : 0.f;
            const int br = idx >> 6, bc = idx & 63;
            const int gk2 = k0 + br, gn = n0 + bc;
            Bs[br][bc] = (gk2 < K && gn < N) ? B[(int64_t)gk2 * N + gn] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            float ar[4], br[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) ar[u] = As[q][ty * 4 + u];
#pragma unroll
            for (int u = 0; u < 4; ++u) br[u] = Bs[q][tx * 4 + u];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int w = 0; w < 4; ++w) acc[u][w] = fmaf(ar[u], br[w], acc[u][w]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int gm = m0 + ty * 4 + u;
        if (gm >= M) continue;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int gn = n0 + tx * 4 + w;
            if (gn < N) C[(int64_t)gm * N + gn] = acc[u][w];
        }
    }
}

// The concretisation of one row from its FP32 partial sums (centre term av, remainder rlo/rhi, |G|,
// |G -+ v|) and its FP64 intercepts: the terms are added in FP64; pre-activation bounds are rounded
// to FP32 outward (they feed the FP32 relaxation), the controller TM stays FP64.
__device__ __forceinline__ void concretise(const WideArgs& a, int ell, int d, int i, float av, float rlo, float rhi,
                                           float g1, float gm, float gp, float wf, double klo, double khi, double err = 0.0) {
    const NetDesc& N = a.net;
    const float S = fabsf(av) + g1 + (float)fabs(klo) + (float)fabs(khi) + fabsf(rlo) + fabsf(rhi) + fabsf(wf);
    if (!a.rigorous && S > DR_MARGIN_RATIO * a.xscale[d]) atomicOr(&a.st[d], DR_STATUS_MARGIN_BIT);
    // rigorous mode: the row's error bound plus the FP64 rounding of the few additions below
    const double mr = (double)a.rho * (double)S + (a.rigorous ? err + 1e-15 * (double)S : 0.0);
    if (ell < N.L) {
        a.hl[(int64_t)d * N.hidden + N.hoff[ell] + i] = __double2float_rd((double)av + klo + (double)rlo - (double)gm - (double)wf - mr);
        a.hu[(int64_t)d * N.hidden + N.hoff[ell] + i] = __double2float_ru((double)av + khi + (double)rhi + (double)gp + (double)wf + mr);
        a.sa[(int64_t)d * N.maxw + i] = av;
        a.sRlo[(int64_t)d * N.maxw + i] = rlo;
        a.sRhi[(int64_t)d * N.maxw + i] = rhi;
        a.sS[(int64_t)d * N.maxw + i] = __double2float_ru(mr);  // the outward margin applied (split records reuse it)
    } else {
        a.cu[(int64_t)d * N.m + i] = (double)av + 0.5 * (klo + khi);
        a.Iulo[(int64_t)d * N.m + i] = 0.5 * (klo - khi) + (double)rlo - mr;
        a.Iuhi[(int64_t)d * N.m + i] = 0.5 * (khi - klo) + (double)rhi + mr;
    }
}

// Concretisation of target ell over the TM input.  One warp per (domain, row); Lx is the
// domain's Lambda_x (rows x n, ld n) or, for ell == 1, the shared W_1.
__global__ void k_w_project(const WideArgs a, int ell, const float* __restrict__ Lxb, int shared_lx) {
    const NetDesc& N = a.net;
    const int n = N.n, rows = N.w[ell];
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= (int64_t)a.Dc * rows) return;
    const int d = (int)(wid / rows), i = (int)(wid - (int64_t)d * rows);
    const float* Lx = shared_lx ? (Lxb + (int64_t)i * n) : (Lxb + (int64_t)d * a.lam_stride + (int64_t)i * n);
    const float* Pf = a.Pf + (int64_t)d * n * n;
    const float* cf = a.cf + (int64_t)d * n;
    const float* Ilof = a.Ilof + (int64_t)d * n;
    const float* Ihif = a.Ihif + (int64_t)d * n;
    const float* vf = a.vf + (int64_t)d * (n + 1);
    float* G = a.G + ((int64_t)d * N.maxw + i) * n;
    float g1 = 0.f, gm = 0.f, gp = 0.f;
    float* Gk = a.Gk ? a.Gk + ((int64_t)d * a.krows + a.koff + i) * n : nullptr;
    for (int k = lane; k < n; k += 32) {
        float acc = 0.f;
        for (int j = 0; j < n; ++j) acc = fmaf(Lx[j], Pf[j * n + k], acc);
        G[k] = acc;
        if (Gk) {
            Gk[k] = acc;
            a.LXk[((int64_t)d * a.krows + a.koff + i) * n + k] = Lx[k];
        }
        g1 += fabsf(acc);
        gm += fabsf(acc - vf[k]);
        gp += fabsf(acc + vf[k]);
    }
    float av = 0.f, rlo = 0.f, rhi = 0.f;
    for (int j = lane; j < n; j += 32) {
        const float x = Lx[j];
        av = fmaf(x, cf[j], av);
        rlo = fmaf(posf(x), Ilof[j], fmaf(negf(x), Ihif[j], rlo));
        rhi = fmaf(posf(x), Ihif[j], fmaf(negf(x), Ilof[j], rhi));
    }
    g1 = warp_sum(g1);
    gm = warp_sum(gm);
    gp = warp_sum(gp);
    av = warp_sum(av);
    rlo = warp_sum(rlo);
    rhi = warp_sum(rhi);
    // rigorous mode: bound of this row's own rounding (G, the centre and remainder terms, the |G -+ v|
    // sums; n terms each, every term at most |Lambda_x j| xmax_j or |G_k| + |v_k|) plus the chain's
    float re = 0.f;
    if (a.rigorous) {
        const float* xm = a.xmax + (int64_t)d * n;
        for (int j = lane; j < n; j += 32) re = __fmaf_ru(fabsf(Lx[j]), xm[j], re);
        float vs = 0.f;
        for (int k = lane; k < n; k += 32) vs += fabsf(vf[k]);
        re = __fadd_ru(re, __fadd_ru(g1, vs));
        re = warp_sum(re);
    }
    if (lane != 0) return;
    const double klo = a.klo[(int64_t)d * N.maxw + i], khi = a.khi[(int64_t)d * N.maxw + i];
    double err = 0.0;
    if (a.rigorous)
        err = a.kerr[(int64_t)d * N.maxw + i] + 4.0 * gamma_k(n) * (double)re * 1.0009765625;
    concretise(a, ell, d, i, av, rlo, rhi, g1, gm, gp, vf[n], klo, khi, err);
}

// Rigorous mode: q_m = |W_m| hmax_{m-1} for hidden layer m (hmax_0 = xmax, else max(u_{m-1}, 0)), the
// magnitude each level's product error is measured in.  One warp per (domain, neuron of layer m); the
// FP32 sum of non-negative terms is rounded up and enlarged by 2^-10, far above its relative error.
__global__ void k_r_q(const WideArgs a, int mm) {
    const NetDesc& N = a.net;
    const int rows = N.w[mm], K = N.w[mm - 1];
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= (int64_t)a.Dc * rows) return;
    const int d = (int)(wid / rows), j = (int)(wid - (int64_t)d * rows);
    const float* Wrow = a.W + N.Woff[mm - 1] + (int64_t)j * K;
    const float* hu = mm == 1 ? a.xmax + (int64_t)d * N.n : a.hu + (int64_t)d * N.hidden + N.hoff[mm - 1];
    float acc = 0.f;
    for (int k = lane; k < K; k += 32) acc = __fmaf_ru(fabsf(Wrow[k]), mm == 1 ? hu[k] : fmaxf(hu[k], 0.f), acc);
    acc = warp_sum(acc);
    if (lane == 0) a.hq[(int64_t)d * N.hidden + N.hoff[mm] + j] = __fmul_ru(acc, 1.0009765625f);
}

// Splits of (t, ell) and the shared-slope relaxation of hidden layer ell; one block per domain.
__global__ void k_w_relax(const WideArgs a, int ell, int t) {
    const NetDesc& N = a.net;
    const int n = N.n, rows = N.w[ell], H = N.H, d = blockIdx.x;
    const int64_t dom = a.d0 + d;
    float* lh = a.hl + (int64_t)d * N.hidden + N.hoff[ell];
    float* uh = a.hu + (int64_t)d * N.hidden + N.hoff[ell];
    if (a.hl0) {
        // keep mode: the bounds before the clipping below
        for (int j = threadIdx.x; j < rows; j += blockDim.x) {
            a.hl0[(int64_t)d * N.hidden + N.hoff[ell] + j] = lh[j];
            a.hu0[(int64_t)d * N.hidden + N.hoff[ell] + j] = uh[j];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && a.sp_row) {
        const int64_t sp_end = a.sp_row[dom + 1];
        int cpos = a.cursor[d];
        bool changed = false;
        while (cpos < sp_end) {
            const SplitRec r = a.sp[cpos];
            if (r.t > t || (r.t == t && r.layer > ell)) break;
            if (r.t == t && r.layer == ell) {
                const int j = r.neuron;
                const int64_t q = (int64_t)d * N.maxw + j;
                const float bt = a.beta ? a.beta[cpos] : 0.f;
                const double hh = r.sign > 0 ? ((double)a.sa[q] + a.khi[q] + (double)a.sRhi[q] + (double)a.sS[q])
                                             : (-((double)a.sa[q] + a.klo[q] + (double)a.sRlo[q]) + (double)a.sS[q]);
                if (a.sph) a.sph[cpos] = (float)hh;
                if (r.sign > 0) {
                    if (lh[j] < 0.f) lh[j] = 0.f;
                } else {
                    if (uh[j] > 0.f) uh[j] = 0.f;
                }
                if (bt != 0.f) {
                    const float* Gj = a.G + q * n;
                    for (int k = 0; k < n; ++k) a.v[(int64_t)d * n + k] += (double)bt * (double)r.sign * (double)Gj[k];
                    a.w[d] += (double)bt * (double)hh;
                    changed = true;
                }
            }
            ++cpos;
        }
        a.cursor[d] = cpos;
        if (changed) {
            double dv = 0.0;
            float* vf = a.vf + (int64_t)d * (n + 1);
            for (int k = 0; k < n; ++k) {
                vf[k] = (float)a.v[(int64_t)d * n + k];
                dv += fabs(a.v[(int64_t)d * n + k] - (double)vf[k]);
            }
            vf[n] = __double2float_ru(a.w[d] + dv);
        }
    }
    if (threadIdx.x == 0 && a.vsnap && ell + 1 <= N.L) {
        // keep mode: the dual vector the next target's concretisation sees
        const float* vf = a.vf + (int64_t)d * (n + 1);
        float* vs = a.vsnap + ((int64_t)d * N.L + ell) * (n + 1);
        for (int k = 0; k <= n; ++k) vs[k] = vf[k];
    }
    __syncthreads();
    for (int j = threadIdx.x; j < rows; j += blockDim.x) {
        const float l = lh[j], u = uh[j];
        if (l > u) atomicOr(&a.st[d], DR_STATUS_INFEASIBLE_BIT);
        float sl = 0.f, dd = 0.f, al = 0.f;
        if (l >= 0.f) {
            sl = 1.f;
        } else if (u > 0.f) {
            if (a.mode == DR_SLOPE_CHORD_K) al = u / (u - l);
            else if (a.mode == DR_SLOPE_ADAPTIVE_K) al = (u >= -l) ? 1.f : 0.f;
            else if (a.mode == DR_SLOPE_ZERO_K) al = 0.f;
            else al = a.alpha[(dom * H + t) * (int64_t)N.hidden + N.hoff[ell] + j];
            const float b1 = a.rigorous ? __fmul_ru(-al, l) : -al * l;
            const float b2 = a.rigorous ? __fmul_ru(__fadd_ru(1.f, -al), u) : (1.f - al) * u;
            sl = al;
            dd = (b1 >= b2) ? b1 : b2;
        }
        a.hs[(int64_t)d * N.hidden + N.hoff[ell] + j] = sl;
        a.hd[(int64_t)d * N.hidden + N.hoff[ell] + j] = dd;
        if (a.alpha_used) a.alpha_used[(dom * H + t) * (int64_t)N.hidden + N.hoff[ell] + j] = al;
    }
}

// FP64 dynamics on the TM, EvalInt of box t+1 and the running objective; one block per domain.
__global__ void k_w_dyn(const WideArgs a, int t) {
    extern __shared__ __align__(16) unsigned char smraw[];
    double* sm = reinterpret_cast<double*>(smraw);
    const NetDesc& N = a.net;
    const int n = N.n, m = N.m, H = N.H, d = blockIdx.x;
    const int64_t dom = a.d0 + d;
    double* Pn = sm;           // n*n
    double* cn = Pn + n * n;   // n
    double* Ilon = cn + n;     // n
    double* Ihin = Ilon + n;   // n
    double* red = Ihin + n;    // blockDim
    const double* P = a.P + (int64_t)d * n * n;
    const double* c = a.c + (int64_t)d * n;
    const double* Ilo = a.Ilo + (int64_t)d * n;
    const double* Ihi = a.Ihi + (int64_t)d * n;
    const float* G = a.G + (int64_t)d * N.maxw * n;
    const double* cu = a.cu + (int64_t)d * m;
    const double* Iulo = a.Iulo + (int64_t)d * m;
    const double* Iuhi = a.Iuhi + (int64_t)d * m;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx / n, k = idx - i * n;
        double acc = 0.0;
        for (int j = 0; j < n; ++j) acc = fma(a.A[i * n + j], P[j * n + k], acc);
        for (int j = 0; j < m; ++j) acc = fma(a.B[i * m + j], (double)G[j * n + k], acc);
        Pn[idx] = acc;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double acc = (a.e ? a.e[i] : 0.0) + (a.eoff ? a.eoff[(dom * H + t) * n + i] : 0.0), lo_ = 0.0, hi_ = 0.0;
        for (int j = 0; j < n; ++j) {
            const double x = a.A[i * n + j];
            acc = fma(x, c[j], acc);
            lo_ += posd(x) * Ilo[j] + negd(x) * Ihi[j];
            hi_ += posd(x) * Ihi[j] + negd(x) * Ilo[j];
        }
        for (int j = 0; j < m; ++j) {
            const double x = a.B[i * m + j];
            acc = fma(x, cu[j], acc);
            lo_ += posd(x) * Iulo[j] + negd(x) * Iuhi[j];
            hi_ += posd(x) * Iuhi[j] + negd(x) * Iulo[j];
        }
        if (a.rigorous) {
            // FP64 rounding of c', P' and the interval products (<= 34 terms each): 2^-47 of their
            // magnitude (>= (34 + 2) 2^-53), folded into the remainder
            double mag = fabs(a.e ? a.e[i] : 0.0) + fabs(a.eoff ? a.eoff[(dom * H + t) * n + i] : 0.0);
            for (int j = 0; j < n; ++j) {
                double pj = 0.0;
                for (int k = 0; k < n; ++k) pj += fabs(P[j * n + k]);
                mag += fabs(a.A[i * n + j]) * (fabs(c[j]) + pj + fmax(fabs(Ilo[j]), fabs(Ihi[j])));
            }
            for (int j = 0; j < m; ++j) {
                double gj = 0.0;
                for (int k = 0; k < n; ++k) gj += fabs((double)G[j * n + k]);
                mag += fabs(a.B[i * m + j]) * (fabs(cu[j]) + gj + fmax(fabs(Iulo[j]), fabs(Iuhi[j])));
            }
            lo_ -= 7.105427357601002e-15 * mag;
            hi_ += 7.105427357601002e-15 * mag;
        }
        cn[i] = acc;
        Ilon[i] = lo_;
        Ihin[i] = hi_;
    }
    __syncthreads();
    double* Pw = a.P + (int64_t)d * n * n;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) Pw[idx] = Pn[idx];
    const double* v = a.v + (int64_t)d * n;
    const double wv = a.w[d];
    double vsum = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        a.c[(int64_t)d * n + i] = cn[i];
        a.Ilo[(int64_t)d * n + i] = Ilon[i];
        a.Ihi[(int64_t)d * n + i] = Ihin[i];
        double pm = 0.0, pp = 0.0, mag = fabs(cn[i]) + fabs(Ilon[i]) + fabs(Ihin[i]) + fabs(wv);
        for (int k = 0; k < n; ++k) {
            const double x = Pn[i * n + k];
            pm += fabs(x - v[k]);
            pp += fabs(x + v[k]);
            mag += fabs(x) + fabs(v[k]);
        }
        const double bl = cn[i] + Ilon[i] - pm - wv - a.box_margin * mag;
        const double bh = cn[i] + Ihin[i] + pp + wv + a.box_margin * mag;
        if (a.lo) a.lo[(dom * (H + 1) + t + 1) * n + i] = bl;
        if (a.hi) a.hi[(dom * (H + 1) + t + 1) * n + i] = bh;
        vsum += bh - bl;
        if (!isfinite(bl) || !isfinite(bh)) atomicOr(&a.st[d], DR_STATUS_NONFINITE_BIT);
        if (bl > bh) atomicOr(&a.st[d], DR_STATUS_INFEASIBLE_BIT);
    }
    red[threadIdx.x] = vsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < (int)blockDim.x; ++q) s += red[q];
        a.vacc[d] += s;
        if (t == H - 1) {
            if (a.V) a.V[dom] = a.vacc[d];
            if (a.status) a.status[dom] = a.st[d];
        }
    }
}

// ---- tensor-core variant of the chain (rows of all domains stacked: row = d * n_ell + i) -------

__device__ __forceinline__ float tf32_part(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// First chain level of target ell >= 2 from the shared W_ell, writing A = W_ell diag(s_{ell-1}) as
// TF32 parts Ah/Al in the blocked left-operand layout (rows Dc*n_ell, ldk zero-padded columns; see
// tc::blk_index) plus kappa.  One warp per (domain, row).
//
// kappa = b + (row sums) is formed in FP64.  The FP64 pipe of this GPU takes about as long for one
// warp instruction as for 32 active lanes' worth of work, and runs at a small fraction of the FP32
// rate, so the warps' three sums go through shared memory and one lane per row of the block does
// the FP64 additions: one set of FP64 instructions per block instead of one per row (with K = 256
// the per-row sets were what bound this kernel, not its HBM writes).
constexpr int kChainInitThreads = 256;
// One row of k_t_chain_init: the operand's TF32 parts, and the row's three FP32 sums into `sums`.
__device__ __forceinline__ void k_t_chain_init_row(const WideArgs& a, int ell, float* __restrict__ Ah, float* __restrict__ Al,
                                                   int ldk, int64_t wid, int lane, float (*sums)[kChainInitThreads / 32]) {
    const NetDesc& N = a.net;
    const int rows = N.w[ell];
    const int d = (int)(wid / rows), i = (int)(wid - (int64_t)d * rows);
    const int K = N.w[ell - 1];
    const float* Wrow = a.W + N.Woff[ell - 1] + (int64_t)i * K;
    const float* s = a.hs + (int64_t)d * N.hidden + N.hoff[ell - 1];
    const float* dd = a.hd + (int64_t)d * N.hidden + N.hoff[ell - 1];
    const float* bm = a.b + N.boff[ell - 2];
    const int nk = ldk >> 5;
    float spos = 0.f, sneg = 0.f, sb = 0.f;
    const bool vec = K == ldk && ((reinterpret_cast<uintptr_t>(Wrow) | reinterpret_cast<uintptr_t>(s) |
                                   reinterpret_cast<uintptr_t>(dd) | reinterpret_cast<uintptr_t>(bm)) & 15) == 0;
    if (vec) {
        // four consecutive columns per lane (16-byte loads and stores; K is a multiple of 32)
        for (int j = 4 * lane; j < K; j += 128) {
            const float4 x = *reinterpret_cast<const float4*>(Wrow + j);
            const float4 dv = *reinterpret_cast<const float4*>(dd + j);
            const float4 sv = *reinterpret_cast<const float4*>(s + j);
            const float4 bv = *reinterpret_cast<const float4*>(bm + j);
            const float xa[4] = {x.x, x.y, x.z, x.w}, da[4] = {dv.x, dv.y, dv.z, dv.w};
            const float sa[4] = {sv.x, sv.y, sv.z, sv.w}, ba[4] = {bv.x, bv.y, bv.z, bv.w};
            float h[4], l[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                spos = fmaf(posf(xa[q]), da[q], spos);
                sneg = fmaf(negf(xa[q]), da[q], sneg);
                const float xs = xa[q] * sa[q];
                sb = fmaf(xs, ba[q], sb);
                h[q] = tf32_part(xs);
                l[q] = tf32_part(xs - h[q]);
            }
            const int64_t o = tc::blk_index(wid, j, nk);
            *reinterpret_cast<float4*>(Ah + o) = make_float4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<float4*>(Al + o) = make_float4(l[0], l[1], l[2], l[3]);
        }
    } else {
        for (int j = lane; j < ldk; j += 32) {
            float xs = 0.f;
            if (j < K) {
                const float x = Wrow[j];
                spos = fmaf(posf(x), dd[j], spos);
                sneg = fmaf(negf(x), dd[j], sneg);
                xs = x * s[j];
                sb = fmaf(xs, bm[j], sb);
            }
            const float h = tf32_part(xs);
            const int64_t o = tc::blk_index(wid, j, nk);
            Ah[o] = h;
            Al[o] = tf32_part(xs - h);
        }
    }
    spos = warp_sum(spos);
    sneg = warp_sum(sneg);
    sb = warp_sum(sb);
    if (lane == 0) {
        const int w = (threadIdx.x >> 5);
        sums[0][w] = spos;
        sums[1][w] = sneg;
        sums[2][w] = sb;
    }
}

__global__ void __launch_bounds__(kChainInitThreads) k_t_chain_init(const WideArgs a, int ell, float* __restrict__ Ah,
                                                                   float* __restrict__ Al, int ldk) {
    __shared__ float sums[3][kChainInitThreads / 32];
    const NetDesc& N = a.net;
    const int rows = N.w[ell];
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t nrows = (int64_t)a.Dc * rows;
    if (wid < nrows) {
        k_t_chain_init_row(a, ell, Ah, Al, ldk, wid, lane, sums);
    }
    __syncthreads();
    const int nw = blockDim.x >> 5;
    const int64_t r = (blockIdx.x * (int64_t)blockDim.x >> 5) + threadIdx.x;
    if (threadIdx.x < nw && r < nrows) {
        const int d = (int)(r / rows), i = (int)(r - (int64_t)d * rows);
        const float bi = a.b[N.boff[ell - 1] + i];
        a.khi[(int64_t)d * N.maxw + i] = (double)bi + (double)sums[0][threadIdx.x] + (double)sums[2][threadIdx.x];
        a.klo[(int64_t)d * N.maxw + i] = (double)bi + (double)sums[1][threadIdx.x] + (double)sums[2][threadIdx.x];
    }
}

// The same first chain level with the domain's per-column vectors held in registers: a warp takes
// kChainRowsPerWarp consecutive rows (of one domain, mostly), loads s, d (per domain) and the bias
// b_{ell-1} once, and then reads only the W_ell row per row.  For K = 128 KV columns, K = ldk, and
// 16-byte aligned rows and vectors (the host checks).  Per row the arithmetic and its order are
// k_t_chain_init_row's, so the outputs are identical; the instruction count per row falls about
// four-fold (no per-row index divisions or vector loads), which makes the kernel bound by its
// HBM writes also for K = 256.
constexpr int kChainRowsPerWarp = 16;
template <int KV>
__global__ void __launch_bounds__(kChainInitThreads) k_t_chain_init_rc(const WideArgs a, int ell, float* __restrict__ Ah,
                                                                      float* __restrict__ Al, int ldk) {
    constexpr int kRowsPerBlock = kChainInitThreads / 32 * kChainRowsPerWarp;
    __shared__ float sums[3][kRowsPerBlock];
    const NetDesc& N = a.net;
    const int rows = N.w[ell];
    const int K = N.w[ell - 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nrows = (int64_t)a.Dc * rows;
    const int64_t rb0 = (int64_t)blockIdx.x * kRowsPerBlock;
    const int64_t r0 = rb0 + (int64_t)warp * kChainRowsPerWarp;
    const int nk = ldk >> 5;
    const float* Wl = a.W + N.Woff[ell - 1];
    const float* bm = a.b + N.boff[ell - 2];
    float4 bv[KV], sv[KV], dv[KV];
#pragma unroll
    for (int v = 0; v < KV; ++v) bv[v] = *reinterpret_cast<const float4*>(bm + 4 * lane + 128 * v);
    int d = (int)(r0 / rows), i = (int)(r0 - (int64_t)d * rows), dl = -1;
    for (int q = 0; q < kChainRowsPerWarp; ++q, ++i) {
        const int64_t r = r0 + q;
        if (r >= nrows) break;  // uniform across the warp
        if (i == rows) {
            i = 0;
            ++d;
        }
        if (d != dl) {
            const float* sd = a.hs + (int64_t)d * N.hidden + N.hoff[ell - 1];
            const float* dd = a.hd + (int64_t)d * N.hidden + N.hoff[ell - 1];
#pragma unroll
            for (int v = 0; v < KV; ++v) {
                sv[v] = *reinterpret_cast<const float4*>(sd + 4 * lane + 128 * v);
                dv[v] = *reinterpret_cast<const float4*>(dd + 4 * lane + 128 * v);
            }
            dl = d;
        }
        const float* Wrow = Wl + (int64_t)i * K;
        float spos = 0.f, sneg = 0.f, sb = 0.f;
#pragma unroll
        for (int v = 0; v < KV; ++v) {
            const int j = 4 * lane + 128 * v;
            const float4 x = *reinterpret_cast<const float4*>(Wrow + j);
            const float xa[4] = {x.x, x.y, x.z, x.w}, da[4] = {dv[v].x, dv[v].y, dv[v].z, dv[v].w};
            const float sa[4] = {sv[v].x, sv[v].y, sv[v].z, sv[v].w}, ba[4] = {bv[v].x, bv[v].y, bv[v].z, bv[v].w};
            float h[4], l[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                spos = fmaf(posf(xa[e]), da[e], spos);
                sneg = fmaf(negf(xa[e]), da[e], sneg);
                const float xs = xa[e] * sa[e];
                sb = fmaf(xs, ba[e], sb);
                h[e] = tf32_part(xs);
                l[e] = tf32_part(xs - h[e]);
            }
            const int64_t o = tc::blk_index(r, j, nk);
            *reinterpret_cast<float4*>(Ah + o) = make_float4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<float4*>(Al + o) = make_float4(l[0], l[1], l[2], l[3]);
        }
        spos = warp_sum(spos);
        sneg = warp_sum(sneg);
        sb = warp_sum(sb);
        if (lane == 0) {
            const int t = warp * kChainRowsPerWarp + q;
            sums[0][t] = spos;
            sums[1][t] = sneg;
            sums[2][t] = sb;
        }
    }
    __syncthreads();
    // kappa in FP64, one thread per row of the block (see k_t_chain_init)
    for (int t = threadIdx.x; t < kRowsPerBlock; t += blockDim.x) {
        const int64_t r = rb0 + t;
        if (r >= nrows) break;
        const int dr = (int)(r / rows), ir = (int)(r - (int64_t)dr * rows);
        const float bi = a.b[N.boff[ell - 1] + ir];
        a.khi[(int64_t)dr * N.maxw + ir] = (double)bi + (double)sums[0][t] + (double)sums[2][t];
        a.klo[(int64_t)dr * N.maxw + ir] = (double)bi + (double)sums[1][t] + (double)sums[2][t];
    }
}

// Target 2 on the tensor cores.  Its chain is one level, Lambda_x = W_2 diag(s_1) W_1, with the
// intercepts W_2^+ d_1, W_2^- d_1 and W_2 (s_1 b_1): all are products of the shared W_2 (or its
// positive and negative parts) with per-domain columns.  k_t2_prep writes those columns as TF32 parts,
// B^T [(d*NB + c)][ldk] with NB = n + 1 (c < n: s_1 W_1[:, c]; c = n: s_1 b_1) and D^T [d][ldk] (d_1);
// two GEMMs give C1 = W_2 B [n_2][Dc*NB] and C2 = [W_2^+; W_2^-] D [2 n_2][Dc]; k_t2_finish
// scatters them into Lambda_x rows and kappa.
__global__ void k_t2_prep(const WideArgs a, int ldk, float* __restrict__ Bh, float* __restrict__ Bl, float* __restrict__ Dh,
                          float* __restrict__ Dl) {
    const NetDesc& N = a.net;
    const int n = N.n, K = N.w[1], NB = n + 1;
    const float* W1 = a.W + N.Woff[0];
    const float* b1 = a.b + N.boff[0];
    const int64_t total = (int64_t)a.Dc * ldk;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int d = (int)(idx / ldk), k = (int)(idx - (int64_t)d * ldk);
        const bool in = k < K;
        const float sk = in ? a.hs[(int64_t)d * N.hidden + N.hoff[1] + k] : 0.f;
        for (int c = 0; c <= n; ++c) {
            const float x = !in ? 0.f : (c < n ? sk * W1[(int64_t)k * n + c] : sk * b1[k]);
            const float h = tf32_part(x);
            const int64_t o = ((int64_t)d * NB + c) * ldk + k;
            Bh[o] = h;
            Bl[o] = tf32_part(x - h);
        }
        const float dk = in ? a.hd[(int64_t)d * N.hidden + N.hoff[1] + k] : 0.f;
        const float h = tf32_part(dk);
        Dh[idx] = h;
        Dl[idx] = tf32_part(dk - h);
    }
}

__global__ void k_t2_finish(const WideArgs a, const float* __restrict__ C1, const float* __restrict__ C2,
                            float* __restrict__ Lx) {
    const NetDesc& N = a.net;
    const int n = N.n, rows = N.w[2], NB = n + 1;
    const int64_t ld1 = (int64_t)a.Dc * NB, ld2 = a.Dc;
    const int64_t total = (int64_t)a.Dc * rows;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < total; r += (int64_t)gridDim.x * blockDim.x) {
        const int d = (int)(r / rows), i = (int)(r - (int64_t)d * rows);
        const float* c1 = C1 + i * ld1 + (int64_t)d * NB;
        for (int c = 0; c < n; ++c) Lx[r * n + c] = c1[c];
        const double bi = a.b[N.boff[1] + i], sb = c1[n];
        a.khi[(int64_t)d * N.maxw + i] = bi + (double)C2[i * ld2 + d] + sb;
        a.klo[(int64_t)d * N.maxw + i] = bi + (double)C2[(rows + i) * ld2 + d] + sb;
    }
}

// k_t2_finish through a shared-memory tile of 32 rows x 8 domains (n <= 16): C1 holds row i's
// domains contiguously ([i][d][NB]) while Lambda_x wants each domain's rows contiguously ([d][i][n]),
// so the one-thread-per-(domain, row) form reads or writes with a stride on one side.  Here the
// block reads the tile's C1 rows with consecutive threads on consecutive addresses and writes each
// domain's rows the same way.  Same values and the same FP64 additions for kappa.
constexpr int kT2TileRows = 32, kT2TileDoms = 8, kT2MaxNB = 17;
__global__ void __launch_bounds__(256) k_t2_finish_tiled(const WideArgs a, const float* __restrict__ C1,
                                                         const float* __restrict__ C2, float* __restrict__ Lx) {
    __shared__ float tile[kT2TileRows][kT2TileDoms * kT2MaxNB + 1];
    const NetDesc& N = a.net;
    const int n = N.n, rows = N.w[2], NB = n + 1, W = kT2TileDoms * NB;
    const int64_t ld1 = (int64_t)a.Dc * NB, ld2 = a.Dc;
    const int d0 = blockIdx.x * kT2TileDoms, i0 = blockIdx.y * kT2TileRows;
    const int nd = min(kT2TileDoms, a.Dc - d0), ni = min(kT2TileRows, rows - i0);
    for (int e = threadIdx.x; e < kT2TileRows * W; e += blockDim.x) {
        const int ii = e / W, q = e - ii * W;
        if (ii < ni && q < nd * NB) tile[ii][q] = C1[(int64_t)(i0 + ii) * ld1 + (int64_t)d0 * NB + q];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kT2TileDoms * kT2TileRows * n; e += blockDim.x) {
        const int dd = e / (kT2TileRows * n), rem = e - dd * (kT2TileRows * n), ii = rem / n, c = rem - ii * n;
        if (dd < nd && ii < ni) Lx[((int64_t)(d0 + dd) * rows + i0 + ii) * n + c] = tile[ii][dd * NB + c];
    }
    const int dd = threadIdx.x % kT2TileDoms, ii = threadIdx.x / kT2TileDoms;
    if (dd < nd && ii < ni) {
        const int d = d0 + dd, i = i0 + ii;
        const double bi = a.b[N.boff[1] + i], sb = tile[ii][dd * NB + n];
        a.khi[(int64_t)d * N.maxw + i] = bi + (double)C2[(int64_t)i * ld2 + d] + sb;
        a.klo[(int64_t)d * N.maxw + i] = bi + (double)C2[(int64_t)(rows + i) * ld2 + d] + sb;
    }
}

// Adds the per-column-tile intercept partials of a fused chain level into kappa (fixed order).
__global__ void k_t_partials(const WideArgs a, int ell, const float* __restrict__ part, int ntiles) {
    const NetDesc& N = a.net;
    const int rows = N.w[ell];
    const int64_t R = (int64_t)a.Dc * rows;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
        const int d = (int)(r / rows), i = (int)(r - (int64_t)d * rows);
        F32Pair psp, psn, psb;
        for (int t = 0; t < ntiles; ++t) {
            pair_add(psp, part[((int64_t)t * 3 + 0) * R + r]);
            pair_add(psn, part[((int64_t)t * 3 + 1) * R + r]);
            pair_add(psb, part[((int64_t)t * 3 + 2) * R + r]);
        }
        const double sp = pair_value(psp), sn = pair_value(psn), sb = pair_value(psb);
        a.khi[(int64_t)d * N.maxw + i] += sp + sb;
        a.klo[(int64_t)d * N.maxw + i] += sn + sb;
    }
}

// Concretisation of target ell (n <= 16) with four threads per (domain, row): thread q of a quad
// owns Lambda_x entries j = 4q..4q+3 (summing the partial rows in order) and G's columns
// k = 4q..4q+3.  The quad exchanges the row by shuffles for G = Lambda_x P; the sums over j (the
// centre and remainder terms) and over k (|G|, |G -+ v|) are split by quad and reduced by
// shuffles, so their rounding order differs from k_t_project's; G itself is summed in the same
// order.  With ntiles > 0 the final chain level's intercept partials (k_t_partials' sums) are
// added to kappa here, the tiles split over the quad in the same way.
template <bool VEC>
__global__ void __launch_bounds__(256, 3) k_t_project4(const WideArgs a, int ell, const float* __restrict__ Lxb, int shared_lx,
                                                    int lx_parts, const float* __restrict__ part, int ntiles) {
    const NetDesc& N = a.net;
    const int n = N.n, L = N.L, rows = N.w[ell];
    const int64_t R = (int64_t)a.Dc * rows;
    const int lane = threadIdx.x & 31, q = lane & 3, qb = lane & ~3;
    const int rows_per_block = blockDim.x >> 2;
    const int k0 = 4 * q;
    for (int64_t base = (int64_t)blockIdx.x * rows_per_block; base < R; base += (int64_t)gridDim.x * rows_per_block) {
        // every thread of a block takes the same number of trips, so the quad shuffles stay full-warp
        const int64_t r = base + (threadIdx.x >> 2);
        const bool live = r < R;
        const int64_t rc = live ? r : R - 1;
        const int d = (int)(rc / rows), i = (int)(rc - (int64_t)d * rows);
        const float* Pf = a.Pf + (int64_t)d * n * n;
        const float* vf = a.vf + (int64_t)d * (n + 1);
        // all stores come after the last load, so the loads need not wait for them
        float xl[4], cj[4], lj[4], hj[4], vk[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int j = k0 + e;
            float v = 0.f;
            cj[e] = lj[e] = hj[e] = vk[e] = 0.f;
            if (j < n) {
                if (lx_parts > 0) {
                    for (int t = 0; t < lx_parts; ++t) v += Lxb[((int64_t)t * n + j) * R + rc];
                } else {
                    v = shared_lx ? Lxb[(int64_t)i * n + j] : Lxb[rc * n + j];
                }
                cj[e] = a.cf[(int64_t)d * n + j];
                lj[e] = a.Ilof[(int64_t)d * n + j];
                hj[e] = a.Ihif[(int64_t)d * n + j];
                vk[e] = vf[j];
            }
            xl[e] = v;
        }
        const float wf = vf[n];
        double klo = 0.0, khi = 0.0;
        if (shared_lx) klo = khi = a.b[N.boff[0] + i];
        else {
            klo = a.klo[(int64_t)d * N.maxw + i];
            khi = a.khi[(int64_t)d * N.maxw + i];
        }
        double sp = 0.0, sn = 0.0, sb = 0.0;
        if (!shared_lx && ntiles > 0) {
            F32Pair psp, psn, psb;
            for (int t = q; t < ntiles; t += 4) {
                pair_add(psp, part[((int64_t)t * 3 + 0) * R + rc]);
                pair_add(psn, part[((int64_t)t * 3 + 1) * R + rc]);
                pair_add(psb, part[((int64_t)t * 3 + 2) * R + rc]);
            }
            sp = pair_value(psp);
            sn = pair_value(psn);
            sb = pair_value(psb);
        }
        float av = 0.f, rlo = 0.f, rhi = 0.f;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float v = xl[e];
            av = fmaf(v, cj[e], av);
            rlo = fmaf(posf(v), lj[e], fmaf(negf(v), hj[e], rlo));
            rhi = fmaf(posf(v), hj[e], fmaf(negf(v), lj[e], rhi));
        }
        float gr[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const float xj = __shfl_sync(0xffffffffu, xl[j & 3], qb | (j >> 2));
            if (j < n && k0 < n) {
                float4 pv;
                if constexpr (VEC) {
                    pv = *reinterpret_cast<const float4*>(Pf + j * n + k0);
                } else {
                    pv = make_float4(Pf[j * n + k0], 0.f, 0.f, 0.f);
                    if (k0 + 1 < n) pv.y = Pf[j * n + k0 + 1];
                    if (k0 + 2 < n) pv.z = Pf[j * n + k0 + 2];
                    if (k0 + 3 < n) pv.w = Pf[j * n + k0 + 3];
                }
                gr[0] = fmaf(xj, pv.x, gr[0]);
                gr[1] = fmaf(xj, pv.y, gr[1]);
                gr[2] = fmaf(xj, pv.z, gr[2]);
                gr[3] = fmaf(xj, pv.w, gr[3]);
            }
        }
        float g1 = 0.f, gm = 0.f, gp = 0.f;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (k0 + e < n) {
                g1 += fabsf(gr[e]);
                gm += fabsf(gr[e] - vk[e]);
                gp += fabsf(gr[e] + vk[e]);
            }
        }
        // quad sums (xor 1, then xor 2): every thread of the quad ends with the same totals
#pragma unroll
        for (int o = 1; o <= 2; o <<= 1) {
            av += __shfl_xor_sync(0xffffffffu, av, o);
            rlo += __shfl_xor_sync(0xffffffffu, rlo, o);
            rhi += __shfl_xor_sync(0xffffffffu, rhi, o);
            g1 += __shfl_xor_sync(0xffffffffu, g1, o);
            gm += __shfl_xor_sync(0xffffffffu, gm, o);
            gp += __shfl_xor_sync(0xffffffffu, gp, o);
            sp += __shfl_xor_sync(0xffffffffu, sp, o);
            sn += __shfl_xor_sync(0xffffffffu, sn, o);
            sb += __shfl_xor_sync(0xffffffffu, sb, o);
        }
        if (!live) continue;
        if (a.Gk && k0 < n) {
            const int64_t ko = ((int64_t)d * a.krows + a.koff + i) * n + k0;
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (k0 + e < n) {
                    a.Gk[ko + e] = gr[e];
                    a.LXk[ko + e] = xl[e];
                }
        }
        if (k0 < n && (ell == L || a.sp_row != nullptr)) {  // G rows nobody reads are not stored
            float* G = a.G + ((int64_t)d * N.maxw + i) * n + k0;
            if constexpr (VEC) {
                *reinterpret_cast<float4*>(G) = make_float4(gr[0], gr[1], gr[2], gr[3]);
            } else {
                G[0] = gr[0];
                if (k0 + 1 < n) G[1] = gr[1];
                if (k0 + 2 < n) G[2] = gr[2];
                if (k0 + 3 < n) G[3] = gr[3];
            }
        }
        if (q != 0) continue;
        if (!shared_lx && ntiles > 0) {
            khi += sp + sb;
            klo += sn + sb;
        }
        if (shared_lx || ntiles > 0) {
            a.klo[(int64_t)d * N.maxw + i] = klo;
            a.khi[(int64_t)d * N.maxw + i] = khi;
        }
        concretise(a, ell, d, i, av, rlo, rhi, g1, gm, gp, wf, klo, khi);
    }
}

// Concretisation of target ell with one thread per (domain, row); Lambda_x rows of domain d start at
// Lxb + d * rows * n (ld n), or, with shared_lx, every domain uses the same rows Lxb + i * n (the
// first layer: Lambda_x = W_1 and kappa = b_1).  Same arithmetic as k_w_project.  NMAX >= n is a compile-time bound
// so that the row lives in registers and the loops unroll.
// With lx_parts > 0 the row is the sum, in order, of lx_parts partial rows stored entry-major:
// entry j of part t at Lxb[(t*n + j)*R + r].
// The row's work is a few hundred FP64 and FP32 operations with long FP64 latencies: the launch
// bounds ask for seven resident blocks per SM (72 registers for NMAX = 16, a few spilled bytes),
// which measured faster than 96 registers (five blocks) or 64 (eight blocks, 400 bytes spilled).
template <int NMAX>
__global__ void __launch_bounds__(128, NMAX <= 16 ? 7 : 1) k_t_project(const WideArgs a, int ell, const float* __restrict__ Lxb, int shared_lx,
                                                   int lx_parts, const float* __restrict__ part, int ntiles) {
    const NetDesc& N = a.net;
    const int n = N.n, L = N.L, rows = N.w[ell];
    const int64_t R = (int64_t)a.Dc * rows;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
        const int d = (int)(r / rows), i = (int)(r - (int64_t)d * rows);
        // kappa (and the final chain level's intercept partials, summed as k_t_partials does) is read
        // before anything is stored
        double klo, khi;
        if (shared_lx) {
            klo = khi = a.b[N.boff[0] + i];
        } else {
            klo = a.klo[(int64_t)d * N.maxw + i];
            khi = a.khi[(int64_t)d * N.maxw + i];
            if (ntiles > 0) {
                F32Pair psp, psn, psb;
                for (int t = 0; t < ntiles; ++t) {
                    pair_add(psp, part[((int64_t)t * 3 + 0) * R + r]);
                    pair_add(psn, part[((int64_t)t * 3 + 1) * R + r]);
                    pair_add(psb, part[((int64_t)t * 3 + 2) * R + r]);
                }
                const double sp = pair_value(psp), sn = pair_value(psn), sb = pair_value(psb);
                khi += sp + sb;
                klo += sn + sb;
            }
        }
        const float* Lx = shared_lx ? Lxb + (int64_t)i * n : Lxb + r * n;
        const float* Pf = a.Pf + (int64_t)d * n * n;
        const float* cf = a.cf + (int64_t)d * n;
        const float* Ilof = a.Ilof + (int64_t)d * n;
        const float* Ihif = a.Ihif + (int64_t)d * n;
        const float* vf = a.vf + (int64_t)d * (n + 1);
        float* G = a.G + ((int64_t)d * N.maxw + i) * n;
        // G = Lambda_x P is read back only as a split's constraint row (hidden layers) or as the
        // controller TM's linear part (output layer)
        const bool keepG = ell == L || a.sp_row != nullptr;
        float x[NMAX];
        if (lx_parts > 0) {
#pragma unroll
            for (int j = 0; j < NMAX; ++j) x[j] = 0.f;
            for (int t = 0; t < lx_parts; ++t) {
                const float* q = Lxb + (int64_t)t * n * R + r;
#pragma unroll
                for (int j = 0; j < NMAX; ++j)
                    if (j < n) x[j] += q[(int64_t)j * R];
            }
        } else {
#pragma unroll
            for (int j = 0; j < NMAX; ++j) x[j] = j < n ? Lx[j] : 0.f;
        }
        float av = 0.f, rlo = 0.f, rhi = 0.f;
#pragma unroll
        for (int j = 0; j < NMAX; ++j) {
            if (j < n) {
                av = fmaf(x[j], cf[j], av);
                rlo = fmaf(posf(x[j]), Ilof[j], fmaf(negf(x[j]), Ihif[j], rlo));
                rhi = fmaf(posf(x[j]), Ihif[j], fmaf(negf(x[j]), Ilof[j], rhi));
            }
        }
        float g1 = 0.f, gm = 0.f, gp = 0.f;
        if ((n & 3) == 0) {
            // G = x P with P's rows read as 16-byte vectors (same accumulation order over j)
            float gr[NMAX];
#pragma unroll
            for (int k = 0; k < NMAX; ++k) gr[k] = 0.f;
#pragma unroll
            for (int j = 0; j < NMAX; ++j) {
                if (j < n) {
                    const float4* prow = reinterpret_cast<const float4*>(Pf + j * n);
#pragma unroll
                    for (int q = 0; q < NMAX / 4; ++q) {
                        if (4 * q < n) {
                            const float4 pv = prow[q];
                            gr[4 * q] = fmaf(x[j], pv.x, gr[4 * q]);
                            gr[4 * q + 1] = fmaf(x[j], pv.y, gr[4 * q + 1]);
                            gr[4 * q + 2] = fmaf(x[j], pv.z, gr[4 * q + 2]);
                            gr[4 * q + 3] = fmaf(x[j], pv.w, gr[4 * q + 3]);
                        }
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < NMAX; ++k) {
                if (k < n) {
                    g1 += fabsf(gr[k]);
                    gm += fabsf(gr[k] - vf[k]);
                    gp += fabsf(gr[k] + vf[k]);
                }
            }
            if (keepG) {
#pragma unroll
                for (int q = 0; q < NMAX / 4; ++q)
                    if (4 * q < n) reinterpret_cast<float4*>(G)[q] = make_float4(gr[4 * q], gr[4 * q + 1], gr[4 * q + 2], gr[4 * q + 3]);
            }
        } else {
            for (int k = 0; k < n; ++k) {
                float acc = 0.f;
#pragma unroll
                for (int j = 0; j < NMAX; ++j)
                    if (j < n) acc = fmaf(x[j], Pf[j * n + k], acc);
                if (keepG) G[k] = acc;
                g1 += fabsf(acc);
                gm += fabsf(acc - vf[k]);
                gp += fabsf(acc + vf[k]);
            }
        }
        if (a.Gk) {
            // keep mode: Lambda_x and G of this row (G recomputed in the same order as above)
            const int64_t ko = ((int64_t)d * a.krows + a.koff + i) * n;
#pragma unroll
            for (int j = 0; j < NMAX; ++j)
                if (j < n) a.LXk[ko + j] = x[j];
            for (int k = 0; k < n; ++k) {
                float acc = 0.f;
#pragma unroll
                for (int j = 0; j < NMAX; ++j)
                    if (j < n) acc = fmaf(x[j], Pf[j * n + k], acc);
                a.Gk[ko + k] = acc;
            }
        }
        // layer 1 has no chain: its intercepts are the bias (and kappa is recorded for the splits)
        if (shared_lx || ntiles > 0) {
            a.klo[(int64_t)d * N.maxw + i] = klo;
            a.khi[(int64_t)d * N.maxw + i] = khi;
        }
        concretise(a, ell, d, i, av, rlo, rhi, g1, gm, gp, vf[n], klo, khi);
    }
}
