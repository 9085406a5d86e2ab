// Fused per-domain forward pass for narrow controllers (all widths fit in shared memory).
//
// One CTA owns one domain for the whole horizon: the controller's weights, the domain's
// Taylor model and every per-domain back-substitution matrix live in shared memory, so
// the pass costs one launch and no global scratch.  Per step (Alg. 2, closed loop of
// Sec. IV-E):
//   FP64 TM -> FP32 view (remainder widened to cover the cast) -> for each layer l:
//   back-substitution chain Lambda <- (Lambda diag(s_m)) W_m with the Lambda^+/- intercepts
//   (Thm. 2), concretisation over the TM input (Thm. 3) with the split dual and the
//   outward margin, shared-slope relaxation (Sec. IV-C) -> controller TM -> FP64 dynamics
//   and EvalInt.
#pragma once
#include "common.cuh"

struct FusedLayout {  // byte offsets into dynamic shared memory
    int Ws[DR_MAXL];
    int bs;
    int A, B, e;
    int c, P, Ilo, Ihi, v, w;
    int cn, Pn, Ilon, Ihin;
    int cf, Pf, Ilof, Ihif, vf;  // vf holds n floats followed by wf
    int hl, hu, hs, hd;
    int klo, khi;
    int lam0, lam1;
    int G;
    int a, Rlo, Rhi, S;
    int cu, Iulo, Iuhi;
    int misc;  // ints: [0] split cursor, [1] status
    int total;
};

struct FusedArgs {
    NetDesc net;
    FusedLayout lay;
    const float* W;
    const float* b;
    const double* A;
    const double* B;
    const double* e;
    const double* lo0;  // [D][n]
    const double* hi0;
    int64_t d0;         // first domain of this launch
    const int64_t* sp_row;  // [D+1] or null
    const SplitRec* sp;     // [nnz]
    const float* beta;      // [nnz] or null
    const float* alpha;     // [D][H][hidden] (USER) or null
    int mode;
    float rho;
    double* lo;  // [D][H+1][n] or null
    double* hi;
    double* V;          // [D] or null
    uint32_t* status;   // [D] or null
    float* alpha_used;  // [D][H][hidden] or null
    double* tape;       // [D][H][tape_stride] or null
    int tape_stride;
};

#define SMF(off) reinterpret_cast<float*>(sm + (off))
#define SMD(off) reinterpret_cast<double*>(sm + (off))
#define SMI(off) reinterpret_cast<int*>(sm + (off))

template <int NT>
__global__ void __launch_bounds__(NT) k_fused_forward(const FusedArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    const NetDesc& N = a.net;
    const FusedLayout& Y = a.lay;
    const int tid = threadIdx.x;
    const int64_t dom = a.d0 + blockIdx.x;
    const int n = N.n, m = N.m, L = N.L, H = N.H;
    const float rho = a.rho;

    double* c = SMD(Y.c);
    double* P = SMD(Y.P);
    double* Ilo = SMD(Y.Ilo);
    double* Ihi = SMD(Y.Ihi);
    double* v = SMD(Y.v);
    double* wv = SMD(Y.w);
    double* cn = SMD(Y.cn);
    double* Pn = SMD(Y.Pn);
    double* Ilon = SMD(Y.Ilon);
    double* Ihin = SMD(Y.Ihin);
    double* A = SMD(Y.A);
    double* B = SMD(Y.B);
    double* e = SMD(Y.e);
    float* cf = SMF(Y.cf);
    float* Pf = SMF(Y.Pf);
    float* Ilof = SMF(Y.Ilof);
    float* Ihif = SMF(Y.Ihif);
    float* vf = SMF(Y.vf);
    float* hl = SMF(Y.hl);
    float* hu = SMF(Y.hu);
    float* hs = SMF(Y.hs);
    float* hd = SMF(Y.hd);
    float* klo = SMF(Y.klo);
    float* khi = SMF(Y.khi);
    float* G = SMF(Y.G);
    float* sa = SMF(Y.a);
    float* sRlo = SMF(Y.Rlo);
    float* sRhi = SMF(Y.Rhi);
    float* sS = SMF(Y.S);
    float* cu = SMF(Y.cu);
    float* Iulo = SMF(Y.Iulo);
    float* Iuhi = SMF(Y.Iuhi);
    float* bs = SMF(Y.bs);
    int* misc = SMI(Y.misc);
    const int gld = odd_ld(n);

    // ---- parameters into shared memory
    for (int l = 0; l < L; ++l) {
        const int rows = N.w[l + 1], cols = N.w[l], ld = odd_ld(cols);
        float* dst = SMF(Y.Ws[l]);
        const float* src = a.W + N.Woff[l];
        for (int idx = tid; idx < rows * cols; idx += NT) {
            const int r = idx / cols, q = idx - r * cols;
            dst[r * ld + q] = src[idx];
        }
    }
    {
        int nb = 0;
        for (int l = 0; l < L; ++l) nb += N.w[l + 1];
        for (int idx = tid; idx < nb; idx += NT) bs[idx] = a.b[idx];
    }
    for (int idx = tid; idx < n * n; idx += NT) A[idx] = a.A[idx];
    for (int idx = tid; idx < n * m; idx += NT) B[idx] = a.B[idx];
    // ---- a1: BuildLinearTM over the normalised box
    const double* lo0 = a.lo0 + dom * n;
    const double* hi0 = a.hi0 + dom * n;
    for (int idx = tid; idx < n * n; idx += NT) {
        const int i = idx / n, k = idx - i * n;
        P[idx] = (i == k) ? 0.5 * (hi0[i] - lo0[i]) : 0.0;
    }
    for (int i = tid; i < n; i += NT) {
        e[i] = a.e ? a.e[i] : 0.0;
        c[i] = 0.5 * (lo0[i] + hi0[i]);
        Ilo[i] = 0.0;
        Ihi[i] = 0.0;
        v[i] = 0.0;
        if (a.lo) a.lo[(dom * (H + 1)) * n + i] = lo0[i];
        if (a.hi) a.hi[(dom * (H + 1)) * n + i] = hi0[i];
    }
    int64_t sp_end = 0;
    if (a.sp_row) sp_end = a.sp_row[dom + 1];
    if (tid == 0) {
        wv[0] = 0.0;
        misc[0] = a.sp_row ? (int)(a.sp_row[dom]) : 0;  // cursor relative to nothing: absolute index fits int
        misc[1] = 0;
    }
    double vacc = 0.0;
    __syncthreads();

    for (int t = 0; t < H; ++t) {
        if (a.tape) {
            double* tp = a.tape + (dom * H + t) * (int64_t)a.tape_stride;
            for (int idx = tid; idx < n * n; idx += NT) tp[idx] = P[idx];
            for (int i = tid; i < n; i += NT) {
                tp[n * n + i] = c[i];
                tp[n * n + n + i] = Ilo[i];
                tp[n * n + 2 * n + i] = Ihi[i];
                tp[n * n + 3 * n + i] = v[i];
            }
            if (tid == 0) {
                tp[n * n + 4 * n] = wv[0];
                tp[n * n + 4 * n + 1] = (double)misc[0];
            }
        }
        // ---- FP32 view of the TM; the remainder absorbs the rounding of c and P
        for (int idx = tid; idx < n * n; idx += NT) Pf[idx] = (float)P[idx];
        for (int i = tid; i < n; i += NT) {
            const float ci = (float)c[i];
            double dev = 0.0;
            for (int k = 0; k < n; ++k) dev += fabs(P[i * n + k] - (double)(float)P[i * n + k]);
            const double dc = c[i] - (double)ci;
            cf[i] = ci;
            Ilof[i] = __double2float_rd(Ilo[i] + dc - dev);
            Ihif[i] = __double2float_ru(Ihi[i] + dc + dev);
        }
        if (tid == 0) {
            double dv = 0.0;
            for (int k = 0; k < n; ++k) {
                vf[k] = (float)v[k];
                dv += fabs(v[k] - (double)vf[k]);
            }
            vf[n] = __double2float_ru(wv[0] + dv);
        }
        __syncthreads();

        for (int ell = 1; ell <= L; ++ell) {
            const int rows = N.w[ell];
            const float* bl = bs + N.boff[ell - 1];
            for (int i = tid; i < rows; i += NT) {
                klo[i] = bl[i];
                khi[i] = bl[i];
            }
            // ---- a4: back-substitution chain from layer ell down to the input
            const float* cur = SMF(Y.Ws[ell - 1]);
            int cur_ld = odd_ld(N.w[ell - 1]);
            int cur_cols = N.w[ell - 1];
            int buf = 0;
            __syncthreads();
            for (int mm = ell - 1; mm >= 1; --mm) {
                const float* s = hs + N.hoff[mm];
                const float* d = hd + N.hoff[mm];
                const float* bm = bs + N.boff[mm - 1];
                for (int i = tid; i < rows; i += NT) {
                    float spos = 0.f, sneg = 0.f, sb = 0.f;
                    const float* row = cur + i * cur_ld;
                    for (int j = 0; j < cur_cols; ++j) {
                        const float x = row[j];
                        spos = fmaf(posf(x), d[j], spos);
                        sneg = fmaf(negf(x), d[j], sneg);
                        sb = fmaf(x * s[j], bm[j], sb);
                    }
                    khi[i] += spos + sb;
                    klo[i] += sneg + sb;
                }
                const int K = N.w[mm], NN = N.w[mm - 1];
                const float* Wm = SMF(Y.Ws[mm - 1]);
                const int wld = odd_ld(NN);
                float* nxt = SMF(buf ? Y.lam1 : Y.lam0);
                const int nld = odd_ld(NN);
                for (int idx = tid; idx < rows * NN; idx += NT) {
                    const int i = idx / NN, k = idx - i * NN;
                    const float* row = cur + i * cur_ld;
                    float acc = 0.f;
                    for (int j = 0; j < K; ++j) acc = fmaf(row[j] * s[j], Wm[j * wld + k], acc);
                    nxt[i * nld + k] = acc;
                }
                __syncthreads();
                cur = nxt;
                cur_ld = nld;
                cur_cols = NN;
                buf ^= 1;
            }
            // ---- a5: concretisation over the TM input: G = Lambda P, a = Lambda c, R = Lambda (x) I
            for (int idx = tid; idx < rows * n; idx += NT) {
                const int i = idx / n, k = idx - i * n;
                const float* row = cur + i * cur_ld;
                float acc = 0.f;
                for (int j = 0; j < n; ++j) acc = fmaf(row[j], Pf[j * n + k], acc);
                G[i * gld + k] = acc;
            }
            __syncthreads();
            for (int i = tid; i < rows; i += NT) {
                const float* row = cur + i * cur_ld;
                float av = 0.f, rlo = 0.f, rhi = 0.f;
                for (int j = 0; j < n; ++j) {
                    const float x = row[j];
                    av = fmaf(x, cf[j], av);
                    rlo = fmaf(posf(x), Ilof[j], fmaf(negf(x), Ihif[j], rlo));
                    rhi = fmaf(posf(x), Ihif[j], fmaf(negf(x), Ilof[j], rhi));
                }
                float g1 = 0.f, gm = 0.f, gp = 0.f;
                for (int k = 0; k < n; ++k) {
                    const float gk = G[i * gld + k];
                    g1 += fabsf(gk);
                    gm += fabsf(gk - vf[k]);
                    gp += fabsf(gk + vf[k]);
                }
                const float wf = vf[n];
                const float S = fabsf(av) + g1 + fabsf(klo[i]) + fabsf(khi[i]) + fabsf(rlo) + fabsf(rhi) + fabsf(wf);
                if (ell < L) {
                    hl[N.hoff[ell] + i] = av + klo[i] + rlo - gm - wf - rho * S;
                    hu[N.hoff[ell] + i] = av + khi[i] + rhi + gp + wf + rho * S;
                    sa[i] = av;
                    sRlo[i] = rlo;
                    sRhi[i] = rhi;
                    sS[i] = S;
                } else {
                    // a6: controller output as a linear TM (P_u = G stays in place)
                    cu[i] = av + 0.5f * (klo[i] + khi[i]);
                    Iulo[i] = 0.5f * (klo[i] - khi[i]) + rlo - rho * S;
                    Iuhi[i] = 0.5f * (khi[i] - klo[i]) + rhi + rho * S;
                }
            }
            __syncthreads();
            if (ell < L) {
                float* lh = hl + N.hoff[ell];
                float* uh = hu + N.hoff[ell];
                // ---- split constraints of (t, ell): clip, record g^T zeta + h >= 0, update the dual
                if (tid == 0 && a.sp_row) {
                    int cpos = misc[0];
                    bool changed = false;
                    while (cpos < sp_end) {
                        const SplitRec r = a.sp[cpos];
                        if (r.t > t || (r.t == t && r.layer > ell)) break;
                        if (r.t == t && r.layer == ell) {
                            const int j = r.neuron;
                            const float bt = a.beta ? a.beta[cpos] : 0.f;
                            const float hh = r.sign > 0 ? (sa[j] + khi[j] + sRhi[j] + rho * sS[j])
                                                        : (-(sa[j] + klo[j] + sRlo[j]) + rho * sS[j]);
                            if (r.sign > 0) {
                                if (lh[j] < 0.f) lh[j] = 0.f;
                            } else {
                                if (uh[j] > 0.f) uh[j] = 0.f;
                            }
                            if (bt != 0.f) {
                                for (int k = 0; k < n; ++k) v[k] += (double)bt * (double)r.sign * (double)G[j * gld + k];
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
                __syncthreads();
                // ---- a3: shared-slope relaxation
                for (int j = tid; j < rows; j += NT) {
                    const float l = lh[j], u = uh[j];
                    if (l > u) atomicOr(reinterpret_cast<unsigned int*>(&misc[1]), DR_STATUS_INFEASIBLE_BIT);
                    float s = 0.f, d = 0.f, al = 0.f;
                    if (l >= 0.f) {
                        s = 1.f;
                    } else if (u <= 0.f) {
                        s = 0.f;
                    } else {
                        if (a.mode == DR_SLOPE_CHORD_K) al = u / (u - l);
                        else if (a.mode == DR_SLOPE_ADAPTIVE_K) al = (u >= -l) ? 1.f : 0.f;
                        else if (a.mode == DR_SLOPE_ZERO_K) al = 0.f;
                        else al = a.alpha[(dom * H + t) * (int64_t)N.hidden + N.hoff[ell] + j];
                        const float b1 = -al * l, b2 = (1.f - al) * u;
                        s = al;
                        d = (b1 >= b2) ? b1 : b2;
                    }
                    hs[N.hoff[ell] + j] = s;
                    hd[N.hoff[ell] + j] = d;
                    if (a.alpha_used) a.alpha_used[(dom * H + t) * (int64_t)N.hidden + N.hoff[ell] + j] = al;
                }
                __syncthreads();
            }
        }
        // ---- a7: dynamics on the TM (FP64)
        for (int idx = tid; idx < n * n; idx += NT) {
            const int i = idx / n, k = idx - i * n;
            double acc = 0.0;
            for (int j = 0; j < n; ++j) acc = fma(A[i * n + j], P[j * n + k], acc);
            for (int j = 0; j < m; ++j) acc = fma(B[i * m + j], (double)G[j * gld + k], acc);
            Pn[idx] = acc;
        }
        for (int i = tid; i < n; i += NT) {
            double acc = e[i], lo_ = 0.0, hi_ = 0.0;
            for (int j = 0; j < n; ++j) {
                const double aij = A[i * n + j];
                acc = fma(aij, c[j], acc);
                lo_ += posd(aij) * Ilo[j] + negd(aij) * Ihi[j];
                hi_ += posd(aij) * Ihi[j] + negd(aij) * Ilo[j];
            }
            for (int j = 0; j < m; ++j) {
                const double bij = B[i * m + j];
                acc = fma(bij, (double)cu[j], acc);
                lo_ += posd(bij) * (double)Iulo[j] + negd(bij) * (double)Iuhi[j];
                hi_ += posd(bij) * (double)Iuhi[j] + negd(bij) * (double)Iulo[j];
            }
            cn[i] = acc;
            Ilon[i] = lo_;
            Ihin[i] = hi_;
        }
        __syncthreads();
        for (int idx = tid; idx < n * n; idx += NT) P[idx] = Pn[idx];
        for (int i = tid; i < n; i += NT) {
            c[i] = cn[i];
            Ilo[i] = Ilon[i];
            Ihi[i] = Ihin[i];
        }
        __syncthreads();
        // ---- a8: EvalInt with the split dual, outward by a few FP64 ulps of the summed magnitude
        for (int i = tid; i < n; i += NT) {
            double pm = 0.0, pp = 0.0, mag = fabs(c[i]) + fabs(Ilo[i]) + fabs(Ihi[i]) + fabs(wv[0]);
            for (int k = 0; k < n; ++k) {
                const double x = P[i * n + k];
                pm += fabs(x - v[k]);
                pp += fabs(x + v[k]);
                mag += fabs(x) + fabs(v[k]);
            }
            const double bl = c[i] + Ilo[i] - pm - wv[0] - 0x1p-50 * mag;
            const double bh = c[i] + Ihi[i] + pp + wv[0] + 0x1p-50 * mag;
            if (a.lo) a.lo[(dom * (H + 1) + t + 1) * n + i] = bl;
            if (a.hi) a.hi[(dom * (H + 1) + t + 1) * n + i] = bh;
            vacc += bh - bl;
            if (!isfinite(bl) || !isfinite(bh)) atomicOr(reinterpret_cast<unsigned int*>(&misc[1]), DR_STATUS_NONFINITE_BIT);
            if (bl > bh) atomicOr(reinterpret_cast<unsigned int*>(&misc[1]), DR_STATUS_INFEASIBLE_BIT);
        }
        __syncthreads();
    }
    // ---- per-domain objective V_d and status
    double* red = Pn;  // reuse
    if (tid < n) red[tid] = vacc;
    __syncthreads();
    if (tid == 0) {
        double sum = 0.0;
        for (int i = 0; i < n; ++i) sum += red[i];
        if (a.V) a.V[dom] = sum;
        if (a.status) a.status[dom] = (uint32_t)misc[1];
    }
}

// a9: hull over the domains that are not infeasible; one block per (t, i).
__global__ void k_hull(const double* __restrict__ lo, const double* __restrict__ hi, const uint32_t* __restrict__ status,
                       int64_t D, int TN, double* __restrict__ hull_lo, double* __restrict__ hull_hi) {
    __shared__ double slo[256], shi[256];
    const int o = blockIdx.x;
    double mn = __longlong_as_double(0x7ff0000000000000ll), mx = -mn;
    for (int64_t d = threadIdx.x; d < D; d += blockDim.x) {
        if (status && (status[d] & DR_STATUS_INFEASIBLE_BIT)) continue;
        mn = fmin(mn, lo[d * TN + o]);
        mx = fmax(mx, hi[d * TN + o]);
    }
    slo[threadIdx.x] = mn;
    shi[threadIdx.x] = mx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            slo[threadIdx.x] = fmin(slo[threadIdx.x], slo[threadIdx.x + s]);
            shi[threadIdx.x] = fmax(shi[threadIdx.x], shi[threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        hull_lo[o] = slo[0];
        hull_hi[o] = shi[0];
    }
}
