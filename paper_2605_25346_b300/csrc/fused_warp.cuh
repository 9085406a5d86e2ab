// Fused forward pass with one warp per domain, for controllers with two hidden layers
// (n_0 - n_1 - n_2 - n_3, n, m <= kWarpNX, n_1, n_2 <= kWarpHMAX).
//
// Same method and per-phase arithmetic as k_fused_forward (fused_core.cuh): FP64 TM -> FP32 view
// -> per target layer the back-substitution chain (Thm. 2) and the concretisation over the TM
// input (Thm. 3) with the split dual and the outward margin rho*S -> shared-slope relaxation
// -> controller TM -> FP64 dynamics and EvalInt.  The difference is the schedule:
//   - a warp carries one domain through all H steps; the phases are separated by __syncwarp only,
//     so the warps of an SM (one per resident domain) run their dependent phases independently
//     and hide each other's latencies;
//   - the chain products are reassociated so that no per-domain n_2 x n_1 matrix is formed:
//     target 2's Lambda_x = W_2 (diag(s_1) W_1), its intercepts read W_2 directly, and target 3's
//     level-1 matrix (W_3 diag(s_2)) W_2 is m x n_1.
// Rounding differs from the CTA kernels only in the order of FP32 operations.
#pragma once
#include "fused_multi.cuh"

constexpr int kWarpNX = 8;      // n, m <= 8
constexpr int kWarpHMAX = 128;  // n_1, n_2 <= 128

struct WarpLayout {  // shared: byte offsets from the CTA base; per warp: from the warp's base
    int W1, W2, W3, bs, A, B, e;
    int ld1, ld2;    // row strides (floats) of W1 and W2 in shared memory
    int dom0;        // first warp region
    int stride;      // bytes per warp region
    int c, P, Ilo, Ihi, v, w, cn, Pn, Ilon, Ihin;
    int cf, Pf, Ilof, Ihif, vf;
    int hl, hu, hs, hd;  // [n_1 + n_2]
    int sb1;             // [n_1] s_1 * b_1
    int B1;              // [n_1][4-aligned n] s_1 * W_1
    int W3s;             // [m][n_2] W_3 * s_2
    int L31;             // [m][n_1] (W_3 diag(s_2)) W_2
    int Lx3;             // [m][n]
    int Pu, cu, Iulo, Iuhi;
    int sa, klo, khi, sRlo, sRhi, sS, Gs;  // split data of the current target (with splits only)
    int misc;            // ints: [0] split cursor, [1] status, [2] Taylor-model scale (FP32 bits)
    int total;
};

#define WF(off) reinterpret_cast<float*>(wb + (off))
#define WD(off) reinterpret_cast<double*>(wb + (off))
#define WI(off) reinterpret_cast<int*>(wb + (off))

__device__ __forceinline__ float wsumf(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}
__device__ __forceinline__ double wsumd(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Concretisation of one target row from its Lambda_x row x[0..n) (registers) and intercepts:
// writes the bounds (hidden) or the controller TM (output), and the split data when `keep`.
struct RowOut {
    float av, rlo, rhi, g1, gm, gp;
};
__device__ __forceinline__ RowOut concretise_row(const float* x, int n, const float* Pf, const float* cf, const float* Ilof,
                                                 const float* Ihif, const float* vf, float* G) {
    RowOut o{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < kWarpNX; ++j) {
        if (j < n) {
            o.av = fmaf(x[j], cf[j], o.av);
            o.rlo = fmaf(posf(x[j]), Ilof[j], fmaf(negf(x[j]), Ihif[j], o.rlo));
            o.rhi = fmaf(posf(x[j]), Ihif[j], fmaf(negf(x[j]), Ilof[j], o.rhi));
        }
    }
#pragma unroll
    for (int k = 0; k < kWarpNX; ++k) {
        if (k < n) {
            float acc = 0.f;
#pragma unroll
            for (int j = 0; j < kWarpNX; ++j)
                if (j < n) acc = fmaf(x[j], Pf[j * n + k], acc);
            G[k] = acc;
            o.g1 += fabsf(acc);
            o.gm += fabsf(acc - vf[k]);
            o.gp += fabsf(acc + vf[k]);
        }
    }
    return o;
}

// Register cap: at least 24 resident warps per SM (one domain each) to hide the phases' latencies.
template <int WPC>
__global__ void __launch_bounds__(32 * WPC, (24 + WPC - 1) / WPC) k_fused_warp(const MultiArgs a, const WarpLayout Y, int has_splits) {
    extern __shared__ __align__(16) unsigned char sm[];
    const NetDesc& N = a.net;
    const int n = N.n, m = N.m, H = N.H;
    const int H1 = N.w[1], H2 = N.w[2];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const float rho = a.rho;
    float* W1 = reinterpret_cast<float*>(sm + Y.W1);
    float* W2 = reinterpret_cast<float*>(sm + Y.W2);
    float* W3 = reinterpret_cast<float*>(sm + Y.W3);
    float* bs = reinterpret_cast<float*>(sm + Y.bs);
    double* A = reinterpret_cast<double*>(sm + Y.A);
    double* B = reinterpret_cast<double*>(sm + Y.B);
    double* e = reinterpret_cast<double*>(sm + Y.e);
    // ---- shared parameters (whole CTA)
    for (int idx = threadIdx.x; idx < H1 * n; idx += blockDim.x) {
        const int r = idx / n, q = idx - r * n;
        W1[r * Y.ld1 + q] = a.W[N.Woff[0] + idx];
    }
    for (int idx = threadIdx.x; idx < H2 * H1; idx += blockDim.x) {
        const int r = idx / H1, q = idx - r * H1;
        W2[r * Y.ld2 + q] = a.W[N.Woff[1] + idx];
    }
    for (int idx = threadIdx.x; idx < m * H2; idx += blockDim.x) W3[idx] = a.W[N.Woff[2] + idx];
    for (int idx = threadIdx.x; idx < H1 + H2 + m; idx += blockDim.x) bs[idx] = a.b[idx];
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) A[idx] = a.A[idx];
    for (int idx = threadIdx.x; idx < n * m; idx += blockDim.x) B[idx] = a.B[idx];
    for (int i = threadIdx.x; i < n; i += blockDim.x) e[i] = a.e ? a.e[i] : 0.0;
    __syncthreads();
    const int64_t dom = (int64_t)blockIdx.x * WPC + wid;
    if (dom >= a.D) return;  // no CTA-wide barrier follows
    unsigned char* wb = sm + Y.dom0 + (size_t)wid * Y.stride;
    double *c = WD(Y.c), *P = WD(Y.P), *Ilo = WD(Y.Ilo), *Ihi = WD(Y.Ihi), *v = WD(Y.v), *wv = WD(Y.w);
    double *cn = WD(Y.cn), *Pn = WD(Y.Pn), *Ilon = WD(Y.Ilon), *Ihin = WD(Y.Ihin);
    float *cf = WF(Y.cf), *Pf = WF(Y.Pf), *Ilof = WF(Y.Ilof), *Ihif = WF(Y.Ihif), *vf = WF(Y.vf);
    float *hl = WF(Y.hl), *hu = WF(Y.hu), *hs = WF(Y.hs), *hd = WF(Y.hd);
    float *sb1 = WF(Y.sb1), *B1 = WF(Y.B1), *W3s = WF(Y.W3s), *L31 = WF(Y.L31), *Lx3 = WF(Y.Lx3);
    float *Pu = WF(Y.Pu), *cu = WF(Y.cu), *Iulo = WF(Y.Iulo), *Iuhi = WF(Y.Iuhi);
    float *sa = WF(Y.sa), *sklo = WF(Y.klo), *skhi = WF(Y.khi), *sRlo = WF(Y.sRlo), *sRhi = WF(Y.sRhi), *sS = WF(Y.sS);
    float* Gs = WF(Y.Gs);
    int* misc = WI(Y.misc);
    const int ldb1 = (n + 3) & ~3;
    const float* b1 = bs;
    const float* b2 = bs + H1;
    const float* b3 = bs + H1 + H2;
    const int64_t sp_end = a.sp_row ? a.sp_row[dom + 1] : 0;

    // ---- a1: seed
    for (int idx = lane; idx < n * n; idx += 32) {
        const int i = idx / n, k = idx - i * n;
        P[idx] = (i == k) ? 0.5 * (a.hi0[dom * n + i] - a.lo0[dom * n + i]) : 0.0;
    }
    for (int i = lane; i < n; i += 32) {
        const double lo = a.lo0[dom * n + i], hi = a.hi0[dom * n + i];
        c[i] = 0.5 * (lo + hi);
        Ilo[i] = 0.0;
        Ihi[i] = 0.0;
        v[i] = 0.0;
        if (a.lo) a.lo[(dom * (H + 1)) * n + i] = lo;
        if (a.hi) a.hi[(dom * (H + 1)) * n + i] = hi;
    }
    if (lane == 0) {
        wv[0] = 0.0;
        misc[0] = a.sp_row ? (int)a.sp_row[dom] : 0;
        misc[1] = 0;
    }
    double vacc = 0.0;
    __syncwarp();

    // Split constraints of (t, ell) on the current target's rows (lane 0), as apply_splits.
    auto splits = [&](int t, int ell) {
        if (lane == 0) {
            float* lh = hl + N.hoff[ell];
            float* uh = hu + N.hoff[ell];
            int cpos = misc[0];
            bool changed = false;
            while (cpos < sp_end) {
                const SplitRec r = a.sp[cpos];
                if (r.t > t || (r.t == t && r.layer > ell)) break;
                if (r.t == t && r.layer == ell) {
                    const int j = r.neuron;
                    const float bt = a.beta ? a.beta[cpos] : 0.f;
                    const float hh = r.sign > 0 ? (sa[j] + skhi[j] + sRhi[j] + rho * sS[j])
                                                : (-(sa[j] + sklo[j] + sRlo[j]) + rho * sS[j]);
                    if (r.sign > 0) {
                        if (lh[j] < 0.f) lh[j] = 0.f;
                    } else {
                        if (uh[j] > 0.f) uh[j] = 0.f;
                    }
                    if (bt != 0.f) {
                        for (int k = 0; k < n; ++k) v[k] += (double)bt * (double)r.sign * (double)Gs[j * kWarpNX + k];
                        wv[0] += (double)bt * (double)hh;
                        changed = true;
                    }
                }
                ++cpos;
            }
            misc[0] = cpos;
            if (changed) {
                double dv = 0.0;
                for (int k = 0; k < n; ++k) {
                    vf[k] = (float)v[k];
                    dv += fabs(v[k] - (double)vf[k]);
                }
                vf[n] = __double2float_ru(wv[0] + dv);
            }
        }
        __syncwarp();
    };
    // a3: relaxation of hidden layer ell
    auto relax_layer = [&](int t, int ell) {
        const int rows = N.w[ell], off = N.hoff[ell];
        for (int j = lane; j < rows; j += 32) {
            const float l = hl[off + j], u = hu[off + j];
            if (l > u) atomicOr(reinterpret_cast<unsigned int*>(misc + 1), DR_STATUS_INFEASIBLE_BIT);
            float sl = 0.f, d = 0.f, al = 0.f;
            if (l >= 0.f) {
                sl = 1.f;
            } else if (u > 0.f) {
                const float user = a.mode == DR_SLOPE_USER_K ? a.alpha[(dom * H + t) * (int64_t)N.hidden + off + j] : 0.f;
                al = slope_of(a.mode, l, u, user);
                const float q1 = -al * l, q2 = (1.f - al) * u;
                sl = al;
                d = (q1 >= q2) ? q1 : q2;
            }
            hs[off + j] = sl;
            hd[off + j] = d;
            if (a.alpha_used) a.alpha_used[(dom * H + t) * (int64_t)N.hidden + off + j] = al;
        }
        __syncwarp();
    };
    // bounds of hidden target row i of layer ell from its concretisation
    auto hidden_row = [&](int ell, int i, const RowOut& o, float klo, float khi, const float* G) {
        const float wf = vf[n];
        const float S = fabsf(o.av) + o.g1 + fabsf(klo) + fabsf(khi) + fabsf(o.rlo) + fabsf(o.rhi) + fabsf(wf);
        if (S > DR_MARGIN_RATIO * __int_as_float(misc[2])) atomicOr(reinterpret_cast<unsigned int*>(misc + 1), DR_STATUS_MARGIN_BIT);
        hl[N.hoff[ell] + i] = o.av + klo + o.rlo - o.gm - wf - rho * S;
        hu[N.hoff[ell] + i] = o.av + khi + o.rhi + o.gp + wf + rho * S;
        if (has_splits) {
            sa[i] = o.av;
            sklo[i] = klo;
            skhi[i] = khi;
            sRlo[i] = o.rlo;
            sRhi[i] = o.rhi;
            sS[i] = S;
#pragma unroll
            for (int k = 0; k < kWarpNX; ++k)
                if (k < n) Gs[i * kWarpNX + k] = G[k];
        }
    };

    for (int t = 0; t < H; ++t) {
        // ---- FP32 view of the TM (remainder absorbs the casts of c and P; wf those of v)
        for (int idx = lane; idx < n * n; idx += 32) Pf[idx] = (float)P[idx];
        float rs = 0.f;  // row `lane` of tm_scale (common.cuh) in its order; lanes past n hold 0
        for (int i = lane; i < n; i += 32) {
            const float ci = (float)c[i];
            rs = fabsf(ci) + fmaxf(fabsf((float)Ilo[i]), fabsf((float)Ihi[i]));
            for (int k = 0; k < n; ++k) rs += fabsf((float)P[i * n + k]);
            double dev = 0.0;
            for (int k = 0; k < n; ++k) dev += fabs(P[i * n + k] - (double)(float)P[i * n + k]);
            const double dc = c[i] - (double)ci;
            cf[i] = ci;
            Ilof[i] = __double2float_rd(Ilo[i] + dc - dev);
            Ihif[i] = __double2float_ru(Ihi[i] + dc + dev);
        }
        if (lane == 0) {
            double dv = 0.0;
            for (int k = 0; k < n; ++k) {
                vf[k] = (float)v[k];
                dv += fabs(v[k] - (double)vf[k]);
            }
            vf[n] = __double2float_ru(wv[0] + dv);
        }
        // the rows' maximum (fmaxf skips a NaN row; n <= kWarpNX < 32, so some lane holds 0)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rs = fmaxf(rs, __shfl_xor_sync(0xffffffffu, rs, o));
        if (lane == 0) misc[2] = __float_as_int(rs);
        __syncwarp();

        // ---- target 1: Lambda_x = W_1, kappa = b_1
        for (int i = lane; i < H1; i += 32) {
            float x[kWarpNX], G[kWarpNX];
#pragma unroll
            for (int j = 0; j < kWarpNX; ++j) x[j] = j < n ? W1[i * Y.ld1 + j] : 0.f;
            const RowOut o = concretise_row(x, n, Pf, cf, Ilof, Ihif, vf, G);
            hidden_row(1, i, o, b1[i], b1[i], G);
        }
        __syncwarp();
        if (has_splits) splits(t, 1);
        relax_layer(t, 1);

        // ---- right factors of layer 1: B1 = diag(s_1) W_1, sb1 = s_1 * b_1
        for (int j = lane; j < H1; j += 32) {
            const float sj = hs[j];
            sb1[j] = sj * b1[j];
#pragma unroll
            for (int k = 0; k < kWarpNX; ++k)
                if (k < ldb1) B1[j * ldb1 + k] = k < n ? sj * W1[j * Y.ld1 + k] : 0.f;
        }
        __syncwarp();

        // ---- target 2: intercepts from W_2 with (d_1, s_1 b_1), Lambda_x = W_2 B1
        for (int i = lane; i < H2; i += 32) {
            float spos = 0.f, sneg = 0.f, sb = 0.f;
            float x[kWarpNX];
#pragma unroll
            for (int k = 0; k < kWarpNX; ++k) x[k] = 0.f;
            const float* wr = W2 + i * Y.ld2;
            for (int j = 0; j < H1; ++j) {
                const float w = wr[j];
                const float dj = hd[j];
                spos = fmaf(posf(w), dj, spos);
                sneg = fmaf(negf(w), dj, sneg);
                sb = fmaf(w, sb1[j], sb);
                const float4* b4 = reinterpret_cast<const float4*>(B1 + j * ldb1);
#pragma unroll
                for (int q = 0; q < kWarpNX / 4; ++q) {
                    if (4 * q < ldb1) {
                        const float4 bv = b4[q];
                        x[4 * q] = fmaf(w, bv.x, x[4 * q]);
                        x[4 * q + 1] = fmaf(w, bv.y, x[4 * q + 1]);
                        x[4 * q + 2] = fmaf(w, bv.z, x[4 * q + 2]);
                        x[4 * q + 3] = fmaf(w, bv.w, x[4 * q + 3]);
                    }
                }
            }
            float G[kWarpNX];
            const RowOut o = concretise_row(x, n, Pf, cf, Ilof, Ihif, vf, G);
            hidden_row(2, i, o, b2[i] + sneg + sb, b2[i] + spos + sb, G);
        }
        __syncwarp();
        if (has_splits) splits(t, 2);
        relax_layer(t, 2);

        // ---- target 3, level 2: W3s = W_3 diag(s_2); intercepts with (d_2, s_2 b_2); L31 = W3s W_2
        const float* s2 = hs + H1;
        const float* d2 = hd + H1;
        for (int idx = lane; idx < m * H2; idx += 32) {
            const int i = idx - (idx / H2) * H2;
            W3s[idx] = W3[idx] * s2[i];
        }
        __syncwarp();
        // kappa of output row r is kept by lane r, which concretises that row
        float kl3 = 0.f, kh3 = 0.f;
        for (int r = 0; r < m; ++r) {
            {
                float spos = 0.f, sneg = 0.f, sb = 0.f;
                for (int i = lane; i < H2; i += 32) {
                    const float w = W3[r * H2 + i];
                    spos = fmaf(posf(w), d2[i], spos);
                    sneg = fmaf(negf(w), d2[i], sneg);
                    sb = fmaf(W3s[r * H2 + i], b2[i], sb);
                }
                spos = wsumf(spos);
                sneg = wsumf(sneg);
                sb = wsumf(sb);
                if (lane == r) {
                    kh3 = b3[r] + spos + sb;
                    kl3 = b3[r] + sneg + sb;
                }
            }
        }
        for (int j = lane; j < H1; j += 32) {
            float acc[kWarpNX];
#pragma unroll
            for (int r = 0; r < kWarpNX; ++r) acc[r] = 0.f;
            for (int i = 0; i < H2; ++i) {
                const float w2 = W2[i * Y.ld2 + j];
#pragma unroll
                for (int r = 0; r < kWarpNX; ++r)
                    if (r < m) acc[r] = fmaf(W3s[r * H2 + i], w2, acc[r]);
            }
#pragma unroll
            for (int r = 0; r < kWarpNX; ++r)
                if (r < m) L31[r * H1 + j] = acc[r];
        }
        __syncwarp();
        // ---- target 3, level 1: intercepts with (d_1, s_1 b_1); Lx3 = L31 B1
        for (int r = 0; r < m; ++r) {
            {
                float spos = 0.f, sneg = 0.f, sb = 0.f;
                for (int j = lane; j < H1; j += 32) {
                    const float x = L31[r * H1 + j];
                    spos = fmaf(posf(x), hd[j], spos);
                    sneg = fmaf(negf(x), hd[j], sneg);
                    sb = fmaf(x, sb1[j], sb);
                }
                spos = wsumf(spos);
                sneg = wsumf(sneg);
                sb = wsumf(sb);
                if (lane == r) {
                    kh3 += spos + sb;
                    kl3 += sneg + sb;
                }
            }
        }
        for (int idx = lane; idx < m * n; idx += 32) {
            const int r = idx / n, k = idx - r * n;
            float acc = 0.f;
            for (int j = 0; j < H1; ++j) acc = fmaf(L31[r * H1 + j], B1[j * ldb1 + k], acc);
            Lx3[idx] = acc;
        }
        __syncwarp();
        // ---- controller TM (a6): rows r < m, one lane each
        {
            const int r = lane;
            if (r < m) {
                float x[kWarpNX], G[kWarpNX];
#pragma unroll
                for (int j = 0; j < kWarpNX; ++j) x[j] = j < n ? Lx3[r * n + j] : 0.f;
                const RowOut o = concretise_row(x, n, Pf, cf, Ilof, Ihif, vf, G);
                const float klo = kl3, khi = kh3, wf = vf[n];
                const float S = fabsf(o.av) + o.g1 + fabsf(klo) + fabsf(khi) + fabsf(o.rlo) + fabsf(o.rhi) + fabsf(wf);
                if (S > DR_MARGIN_RATIO * __int_as_float(misc[2]))
                    atomicOr(reinterpret_cast<unsigned int*>(misc + 1), DR_STATUS_MARGIN_BIT);
                cu[r] = o.av + 0.5f * (klo + khi);
                Iulo[r] = 0.5f * (klo - khi) + o.rlo - rho * S;
                Iuhi[r] = 0.5f * (khi - klo) + o.rhi + rho * S;
#pragma unroll
                for (int k = 0; k < kWarpNX; ++k)
                    if (k < n) Pu[r * kWarpNX + k] = G[k];
            }
        }
        __syncwarp();

        // ---- a7 dynamics (FP64)
        for (int idx = lane; idx < n * n; idx += 32) {
            const int i = idx / n, k = idx - i * n;
            double acc = 0.0;
            for (int j = 0; j < n; ++j) acc = fma(A[i * n + j], P[j * n + k], acc);
            for (int j = 0; j < m; ++j) acc = fma(B[i * m + j], (double)Pu[j * kWarpNX + k], acc);
            Pn[idx] = acc;
        }
        for (int i = lane; i < n; i += 32) {
            double acc = e[i] + (a.eoff ? a.eoff[(dom * H + t) * n + i] : 0.0), lo_ = 0.0, hi_ = 0.0;
            for (int j = 0; j < n; ++j) {
                const double x = A[i * n + j];
                acc = fma(x, c[j], acc);
                lo_ += posd(x) * Ilo[j] + negd(x) * Ihi[j];
                hi_ += posd(x) * Ihi[j] + negd(x) * Ilo[j];
            }
            for (int j = 0; j < m; ++j) {
                const double x = B[i * m + j];
                acc = fma(x, (double)cu[j], acc);
                lo_ += posd(x) * (double)Iulo[j] + negd(x) * (double)Iuhi[j];
                hi_ += posd(x) * (double)Iuhi[j] + negd(x) * (double)Iulo[j];
            }
            cn[i] = acc;
            Ilon[i] = lo_;
            Ihin[i] = hi_;
        }
        __syncwarp();
        for (int idx = lane; idx < n * n; idx += 32) P[idx] = Pn[idx];
        for (int i = lane; i < n; i += 32) {
            c[i] = cn[i];
            Ilo[i] = Ilon[i];
            Ihi[i] = Ihin[i];
        }
        __syncwarp();
        // ---- a8 EvalInt
        double wsum = 0.0;
        for (int i = lane; i < n; i += 32) {
            double pm = 0.0, pp = 0.0, mag = fabs(c[i]) + fabs(Ilo[i]) + fabs(Ihi[i]) + fabs(wv[0]);
            for (int k = 0; k < n; ++k) {
                const double x = P[i * n + k];
                pm += fabs(x - v[k]);
                pp += fabs(x + v[k]);
                mag += fabs(x) + fabs(v[k]);
            }
            const double bl = c[i] + Ilo[i] - pm - wv[0] - a.box_margin * mag;
            const double bh = c[i] + Ihi[i] + pp + wv[0] + a.box_margin * mag;
            if (a.lo) a.lo[(dom * (H + 1) + t + 1) * n + i] = bl;
            if (a.hi) a.hi[(dom * (H + 1) + t + 1) * n + i] = bh;
            wsum += bh - bl;
            if (!isfinite(bl) || !isfinite(bh)) atomicOr(reinterpret_cast<unsigned int*>(misc + 1), DR_STATUS_NONFINITE_BIT);
            if (bl > bh) atomicOr(reinterpret_cast<unsigned int*>(misc + 1), DR_STATUS_INFEASIBLE_BIT);
        }
        vacc += wsumd(wsum);
        __syncwarp();
    }
    if (lane == 0) {
        if (a.V) a.V[dom] = vacc;
        if (a.status) a.status[dom] = (uint32_t)misc[1];
    }
}
