// Fused forward pass over a group of G domains per CTA (narrow controllers).
//
// Same per-domain arithmetic as k_fused_forward (fused_core.cuh), but every phase runs over all G
// domains of the CTA at once: the controller weights are loaded once per G domains, and each
// barrier-separated phase (chain levels, concretisation, relaxation, FP64 dynamics and EvalInt)
// has G times more independent work for the CTA's threads.
#pragma once
#include "fused_core.cuh"

struct MultiLayout {  // shared: byte offsets from the CTA base; per domain: from the domain base
    int Ws[DR_MAXL];
    int bs, A, B, e;
    int chA, chB;  // CTA-level chain buffers (all domains of the CTA)
    int Bs, E;     // first-level right operand [K][ldb] and intercept table [K][G] (float2)
    int dom0;    // start of the first domain's region
    int stride;  // bytes per domain region
    // per-domain offsets
    int c, P, Ilo, Ihi, v, w, cn, Pn, Ilon, Ihin;
    int cf, Pf, Ilof, Ihif, vf;
    int hl, hu, hs, hd;
    int klo, khi, lam0, lam1, G, a, Rlo, Rhi, S, cu, Iulo, Iuhi, misc, red;
    int total;
};

struct MultiArgs {
    NetDesc net;
    MultiLayout lay;
    const float* W;
    const float* b;
    const double* A;
    const double* B;
    const double* e;
    const double* eoff;  // [D][H][n] per-step offsets of the dynamics or null
    const double* lo0;
    const double* hi0;
    int64_t D;
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
};

#define MD(g, off) reinterpret_cast<double*>(sm + Y.dom0 + (g) * Y.stride + (off))
#define MF(g, off) reinterpret_cast<float*>(sm + Y.dom0 + (g) * Y.stride + (off))
#define MI(g, off) reinterpret_cast<int*>(sm + Y.dom0 + (g) * Y.stride + (off))
#define SF(off) reinterpret_cast<float*>(sm + (off))
#define SD(off) reinterpret_cast<double*>(sm + (off))

// Lanes per (row, domain) in the intercept sums: the columns are split over JS consecutive lanes
// (a power of two <= 32) when there are fewer rows x domains than threads, then tree-reduced.
template <int NT>
__device__ __forceinline__ int intercept_lanes(int items) {
    int js = 1;
    while (js < 32 && items * js * 2 <= NT) js <<= 1;
    return js;
}
__device__ __forceinline__ float lanes_sum(float x, int js) {
    for (int o = js >> 1; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

template <int NT, int G>
__global__ void __launch_bounds__(NT) k_fused_forward_multi(const MultiArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    const NetDesc& N = a.net;
    const MultiLayout& Y = a.lay;
    const int tid = threadIdx.x;
    const int n = N.n, m = N.m, L = N.L, H = N.H;
    const int gld = odd_ld(n);
    const int64_t dbase = (int64_t)blockIdx.x * G;
    const int gcount = (int)min((int64_t)G, a.D - dbase);
    const float rho = a.rho;
    const double* A = SD(Y.A);
    const double* B = SD(Y.B);
    const double* e = SD(Y.e);
    const float* bs = SF(Y.bs);

    // ---- shared parameters
    for (int l = 0; l < L; ++l) {
        const int rows = N.w[l + 1], cols = N.w[l], ld = odd_ld(cols);
        float* dst = SF(Y.Ws[l]);
        const float* src = a.W + N.Woff[l];
        for (int idx = tid; idx < rows * cols; idx += NT) {
            const int r = idx / cols, q = idx - r * cols;
            dst[r * ld + q] = src[idx];
        }
    }
    {
        int nb = 0;
        for (int l = 0; l < L; ++l) nb += N.w[l + 1];
        for (int idx = tid; idx < nb; idx += NT) SF(Y.bs)[idx] = a.b[idx];
    }
    for (int idx = tid; idx < n * n; idx += NT) SD(Y.A)[idx] = a.A[idx];
    for (int idx = tid; idx < n * m; idx += NT) SD(Y.B)[idx] = a.B[idx];
    for (int i = tid; i < n; i += NT) SD(Y.e)[i] = a.e ? a.e[i] : 0.0;
    // ---- a1: seed every domain's TM
    for (int idx = tid; idx < gcount * n * n; idx += NT) {
        const int g = idx / (n * n), r = idx - g * n * n, i = r / n, k = r - i * n;
        const int64_t dom = dbase + g;
        MD(g, Y.P)[r] = (i == k) ? 0.5 * (a.hi0[dom * n + i] - a.lo0[dom * n + i]) : 0.0;
    }
    for (int idx = tid; idx < gcount * n; idx += NT) {
        const int g = idx / n, i = idx - g * n;
        const int64_t dom = dbase + g;
        const double lo = a.lo0[dom * n + i], hi = a.hi0[dom * n + i];
        MD(g, Y.c)[i] = 0.5 * (lo + hi);
        MD(g, Y.Ilo)[i] = 0.0;
        MD(g, Y.Ihi)[i] = 0.0;
        MD(g, Y.v)[i] = 0.0;
        if (a.lo) a.lo[(dom * (H + 1)) * n + i] = lo;
        if (a.hi) a.hi[(dom * (H + 1)) * n + i] = hi;
    }
    for (int g = tid; g < gcount; g += NT) {
        MD(g, Y.w)[0] = 0.0;
        for (int i = 0; i <= n; ++i) MD(g, Y.red)[i] = 0.0;
        MI(g, Y.misc)[0] = a.sp_row ? (int)a.sp_row[dbase + g] : 0;
        MI(g, Y.misc)[1] = 0;
        MI(g, Y.misc)[2] = 0;  // the TM scale (bits of a non-negative float), built by atomicMax per step
    }
    __syncthreads();

    for (int t = 0; t < H; ++t) {
        // ---- FP32 views
        for (int idx = tid; idx < gcount * n * n; idx += NT) {
            const int g = idx / (n * n), r = idx - g * n * n;
            MF(g, Y.Pf)[r] = (float)MD(g, Y.P)[r];
        }
        for (int idx = tid; idx < gcount * n; idx += NT) {
            const int g = idx / n, i = idx - g * n;
            const double* P = MD(g, Y.P);
            const double ci = MD(g, Y.c)[i];
            const float cf = (float)ci;
            // row i of tm_scale (common.cuh), in its order; the maximum over rows by atomicMax on the
            // float's bits (a NaN row is skipped, as fmaxf skips it).  One thread per domain doing all
            // rows cost 9 % of this kernel: its FP64-to-FP32 conversions each take the FP64 pipe's time
            // of a whole warp instruction
            float rs = fabsf(cf) + fmaxf(fabsf((float)MD(g, Y.Ilo)[i]), fabsf((float)MD(g, Y.Ihi)[i]));
            for (int k = 0; k < n; ++k) rs += fabsf((float)P[i * n + k]);
            if (!isnan(rs)) atomicMax(reinterpret_cast<unsigned int*>(MI(g, Y.misc) + 2), __float_as_uint(rs));
            double dev = 0.0;
            for (int k = 0; k < n; ++k) dev += fabs(P[i * n + k] - (double)(float)P[i * n + k]);
            const double dc = ci - (double)cf;
            MF(g, Y.cf)[i] = cf;
            MF(g, Y.Ilof)[i] = __double2float_rd(MD(g, Y.Ilo)[i] + dc - dev);
            MF(g, Y.Ihif)[i] = __double2float_ru(MD(g, Y.Ihi)[i] + dc + dev);
        }
        for (int g = tid; g < gcount; g += NT) {
            double dv = 0.0;
            float* vf = MF(g, Y.vf);
            const double* v = MD(g, Y.v);
            for (int k = 0; k < n; ++k) {
                vf[k] = (float)v[k];
                dv += fabs(v[k] - (double)vf[k]);
            }
            vf[n] = __double2float_ru(MD(g, Y.w)[0] + dv);
        }
        __syncthreads();

        for (int ell = 1; ell <= L; ++ell) {
            const int rows = N.w[ell];
            const float* bl = bs + N.boff[ell - 1];
            for (int idx = tid; idx < gcount * rows; idx += NT) {
                const int g = idx / rows, i = idx - g * rows;
                MF(g, Y.klo)[i] = bl[i];
                MF(g, Y.khi)[i] = bl[i];
            }
            // ---- a4 chain over all domains of the CTA.  Domain g's current matrix starts at
            // curb + g * cur_gs with row stride cur_ld (cur_gs = 0: the shared W_ell).
            float* curb = SF(Y.Ws[ell - 1]);
            int cur_gs = 0;
            int cur_ld = odd_ld(N.w[ell - 1]);
            int cur_cols = N.w[ell - 1];
            int buf = 0;
            __syncthreads();
            for (int mm = ell - 1; mm >= 1; --mm) {
                const float* bm = bs + N.boff[mm - 1];
                const int K = N.w[mm], NN = N.w[mm - 1];
                const float* Wm = SF(Y.Ws[mm - 1]);
                const int wld = odd_ld(NN);
                float* nxt = SF(buf ? Y.chB : Y.chA);
                const bool first = (cur_gs == 0);
                const bool shared_a = first && NN <= 16;
                float2* E = reinterpret_cast<float2*>(sm + Y.E);
                if (first) {
                    // intercept table E[j][g] = (d_gj, s_gj b_j) for the shared W_ell rows
                    for (int idx = tid; idx < K * G; idx += NT) {
                        const int j = idx / G, g = idx - j * G;
                        float2 ev = make_float2(0.f, 0.f);
                        if (g < gcount) ev = make_float2(MF(g, Y.hd)[N.hoff[mm] + j], MF(g, Y.hs)[N.hoff[mm] + j] * bm[j]);
                        E[idx] = ev;
                    }
                }
                const int ldb = ru4(G * NN);
                if (shared_a) {
                    // right operand [K][g*NN + k] = s_gj W_mm[j][k]; one GEMM with the shared W_ell
                    float* Bs = SF(Y.Bs);
                    for (int idx = tid; idx < K * ldb; idx += NT) {
                        const int j = idx / ldb, col = idx - j * ldb;
                        const int g = col / NN, k = col - g * NN;
                        float val = 0.f;
                        if (g < gcount) val = MF(g, Y.hs)[N.hoff[mm] + j] * Wm[j * wld + k];
                        Bs[idx] = val;
                    }
                }
                if (first) __syncthreads();
                if (first && rows * G < NT) {
                    // intercepts of a short target: (row i, domain g) with the columns split over JS lanes
                    const int items = rows * G, JS = intercept_lanes<NT>(items);
                    for (int base = 0; base < items * JS; base += NT) {
                        const int idx = base + tid;
                        const bool act = idx < items * JS;
                        const int it = idx / JS, jp = idx - it * JS;
                        const int i = act ? it / G : 0, g = act ? it - (it / G) * G : 0;
                        float sp = 0.f, sn = 0.f, sbv = 0.f;
                        if (act && g < gcount) {
                            const float* row = curb + i * cur_ld;
                            for (int j = jp; j < cur_cols; j += JS) {
                                const float x = row[j];
                                const float2 ev = E[j * G + g];
                                sp = fmaf(posf(x), ev.x, sp);
                                sn = fmaf(negf(x), ev.x, sn);
                                sbv = fmaf(x, ev.y, sbv);
                            }
                        }
                        sp = lanes_sum(sp, JS);
                        sn = lanes_sum(sn, JS);
                        sbv = lanes_sum(sbv, JS);
                        if (act && jp == 0 && g < gcount) {
                            MF(g, Y.khi)[i] += sp + sbv;
                            MF(g, Y.klo)[i] += sn + sbv;
                        }
                    }
                } else if (first) {
                    // intercepts: thread = (row i, GQ domains); the W_ell row is loaded once for them
                    constexpr int GQ = G < 4 ? G : 4;
                    const int gq = G / GQ;
                    for (int idx = tid; idx < rows * gq; idx += NT) {
                        const int i = idx / gq, g0 = (idx - i * gq) * GQ;
                        const float* row = curb + i * cur_ld;
                        float sp[GQ], sn[GQ], sbv[GQ];
#pragma unroll
                        for (int q = 0; q < GQ; ++q) sp[q] = sn[q] = sbv[q] = 0.f;
                        for (int j = 0; j < cur_cols; ++j) {
                            const float x = row[j], xp = posf(x), xn = negf(x);
#pragma unroll
                            for (int q = 0; q < GQ; ++q) {
                                const float2 ev = E[j * G + g0 + q];
                                sp[q] = fmaf(xp, ev.x, sp[q]);
                                sn[q] = fmaf(xn, ev.x, sn[q]);
                                sbv[q] = fmaf(x, ev.y, sbv[q]);
                            }
                        }
#pragma unroll
                        for (int q = 0; q < GQ; ++q) {
                            if (g0 + q < gcount) {
                                MF(g0 + q, Y.khi)[i] += sp[q] + sbv[q];
                                MF(g0 + q, Y.klo)[i] += sn[q] + sbv[q];
                            }
                        }
                    }
                } else {
                    // (domain g, row i) with the columns split over JS lanes
                    const int items = gcount * rows, JS = intercept_lanes<NT>(items);
                    for (int base = 0; base < items * JS; base += NT) {
                        const int idx = base + tid;
                        const bool act = idx < items * JS;
                        const int it = idx / JS, jp = idx - it * JS;
                        const int g = act ? it / rows : 0, i = act ? it - (it / rows) * rows : 0;
                        float spos = 0.f, sneg = 0.f, sb = 0.f;
                        if (act) {
                            const float* row = curb + g * cur_gs + i * cur_ld;
                            const float* sl = MF(g, Y.hs) + N.hoff[mm];
                            const float* dl = MF(g, Y.hd) + N.hoff[mm];
                            for (int j = jp; j < cur_cols; j += JS) {
                                const float x = row[j];
                                spos = fmaf(posf(x), dl[j], spos);
                                sneg = fmaf(negf(x), dl[j], sneg);
                                sb = fmaf(x * sl[j], bm[j], sb);
                            }
                        }
                        spos = lanes_sum(spos, JS);
                        sneg = lanes_sum(sneg, JS);
                        sb = lanes_sum(sb, JS);
                        if (act && jp == 0) {
                            MF(g, Y.khi)[i] += spos + sb;
                            MF(g, Y.klo)[i] += sneg + sb;
                        }
                    }
                }
                if (shared_a) {
                    gemm_shared_a<NT>(curb, cur_ld, SF(Y.Bs), ldb, nxt, ldb, rows, K, G * NN);
                    __syncthreads();
                    curb = nxt;
                    cur_gs = NN;
                    cur_ld = ldb;
                } else {
                    const int nld = odd_ld(NN);
                    gemm_stacked_scaled<NT>(curb, cur_gs, cur_ld, MF(0, Y.hs) + N.hoff[mm], Y.stride / 4, Wm, wld, nxt, nld,
                                            gcount, rows, K, NN);
                    __syncthreads();
                    curb = nxt;
                    cur_gs = rows * nld;
                    cur_ld = nld;
                }
                cur_cols = NN;
                buf ^= 1;
            }
            // ---- a5 / a6 concretisation
            for (int idx = tid; idx < gcount * rows * n; idx += NT) {
                const int g = idx / (rows * n), r = idx - g * rows * n, i = r / n, k = r - i * n;
                const float* row = curb + g * cur_gs + i * cur_ld;
                const float* Pf = MF(g, Y.Pf);
                float acc = 0.f;
                for (int j = 0; j < n; ++j) acc = fmaf(row[j], Pf[j * n + k], acc);
                MF(g, Y.G)[i * gld + k] = acc;
            }
            __syncthreads();
            for (int idx = tid; idx < gcount * rows; idx += NT) {
                const int g = idx / rows, i = idx - g * rows;
                const float* row = curb + g * cur_gs + i * cur_ld;
                const float* cf = MF(g, Y.cf);
                const float* Ilof = MF(g, Y.Ilof);
                const float* Ihif = MF(g, Y.Ihif);
                const float* vf = MF(g, Y.vf);
                const float* Gr = MF(g, Y.G) + i * gld;
                float av = 0.f, rlo = 0.f, rhi = 0.f;
                for (int j = 0; j < n; ++j) {
                    const float x = row[j];
                    av = fmaf(x, cf[j], av);
                    rlo = fmaf(posf(x), Ilof[j], fmaf(negf(x), Ihif[j], rlo));
                    rhi = fmaf(posf(x), Ihif[j], fmaf(negf(x), Ilof[j], rhi));
                }
                float g1 = 0.f, gm = 0.f, gp = 0.f;
                for (int k = 0; k < n; ++k) {
                    const float gk = Gr[k];
                    g1 += fabsf(gk);
                    gm += fabsf(gk - vf[k]);
                    gp += fabsf(gk + vf[k]);
                }
                const float klo = MF(g, Y.klo)[i], khi = MF(g, Y.khi)[i];
                const float wf = vf[n];
                const float S = fabsf(av) + g1 + fabsf(klo) + fabsf(khi) + fabsf(rlo) + fabsf(rhi) + fabsf(wf);
                if (S > DR_MARGIN_RATIO * __int_as_float(MI(g, Y.misc)[2]))
                    atomicOr(reinterpret_cast<unsigned int*>(MI(g, Y.misc) + 1), DR_STATUS_MARGIN_BIT);
                if (ell < L) {
                    MF(g, Y.hl)[N.hoff[ell] + i] = av + klo + rlo - gm - wf - rho * S;
                    MF(g, Y.hu)[N.hoff[ell] + i] = av + khi + rhi + gp + wf + rho * S;
                    MF(g, Y.a)[i] = av;
                    MF(g, Y.Rlo)[i] = rlo;
                    MF(g, Y.Rhi)[i] = rhi;
                    MF(g, Y.S)[i] = S;
                } else {
                    MF(g, Y.cu)[i] = av + 0.5f * (klo + khi);
                    MF(g, Y.Iulo)[i] = 0.5f * (klo - khi) + rlo - rho * S;
                    MF(g, Y.Iuhi)[i] = 0.5f * (khi - klo) + rhi + rho * S;
                }
            }
            __syncthreads();
            if (ell < L) {
                // ---- splits of (t, ell): one thread per domain
                if (a.sp_row) {
                    for (int g = tid; g < gcount; g += NT) {
                        const int64_t dom = dbase + g;
                        const int64_t sp_end = a.sp_row[dom + 1];
                        float* lh = MF(g, Y.hl) + N.hoff[ell];
                        float* uh = MF(g, Y.hu) + N.hoff[ell];
                        double* v = MD(g, Y.v);
                        int cpos = MI(g, Y.misc)[0];
                        bool changed = false;
                        while (cpos < sp_end) {
                            const SplitRec r = a.sp[cpos];
                            if (r.t > t || (r.t == t && r.layer > ell)) break;
                            if (r.t == t && r.layer == ell) {
                                const int j = r.neuron;
                                const float bt = a.beta ? a.beta[cpos] : 0.f;
                                const float hh = r.sign > 0 ? (MF(g, Y.a)[j] + MF(g, Y.khi)[j] + MF(g, Y.Rhi)[j] + rho * MF(g, Y.S)[j])
                                                            : (-(MF(g, Y.a)[j] + MF(g, Y.klo)[j] + MF(g, Y.Rlo)[j]) + rho * MF(g, Y.S)[j]);
                                if (r.sign > 0) {
                                    if (lh[j] < 0.f) lh[j] = 0.f;
                                } else {
                                    if (uh[j] > 0.f) uh[j] = 0.f;
                                }
                                if (bt != 0.f) {
                                    const float* Gj = MF(g, Y.G) + j * gld;
                                    for (int k = 0; k < n; ++k) v[k] += (double)bt * (double)r.sign * (double)Gj[k];
                                    MD(g, Y.w)[0] += (double)bt * (double)hh;
                                    changed = true;
                                }
                            }
                            ++cpos;
                        }
                        MI(g, Y.misc)[0] = cpos;
                        if (changed) {
                            double dv = 0.0;
                            float* vf = MF(g, Y.vf);
                            for (int k = 0; k < n; ++k) {
                                vf[k] = (float)v[k];
                                dv += fabs(v[k] - (double)vf[k]);
                            }
                            vf[n] = __double2float_ru(MD(g, Y.w)[0] + dv);
                        }
                    }
                    __syncthreads();
                }
                // ---- a3 relaxation
                for (int idx = tid; idx < gcount * rows; idx += NT) {
                    const int g = idx / rows, j = idx - g * rows;
                    const int64_t dom = dbase + g;
                    const float l = MF(g, Y.hl)[N.hoff[ell] + j], u = MF(g, Y.hu)[N.hoff[ell] + j];
                    if (l > u) atomicOr(reinterpret_cast<unsigned int*>(MI(g, Y.misc) + 1), DR_STATUS_INFEASIBLE_BIT);
                    float sl = 0.f, d = 0.f, al = 0.f;
                    if (l >= 0.f) {
                        sl = 1.f;
                    } else if (u > 0.f) {
                        const float user = a.mode == DR_SLOPE_USER_K ? a.alpha[(dom * H + t) * (int64_t)N.hidden + N.hoff[ell] + j] : 0.f;
                        al = slope_of(a.mode, l, u, user);
                        const float b1 = -al * l, b2 = (1.f - al) * u;
                        sl = al;
                        d = (b1 >= b2) ? b1 : b2;
                    }
                    MF(g, Y.hs)[N.hoff[ell] + j] = sl;
                    MF(g, Y.hd)[N.hoff[ell] + j] = d;
                    if (a.alpha_used) a.alpha_used[(dom * H + t) * (int64_t)N.hidden + N.hoff[ell] + j] = al;
                }
                __syncthreads();
            }
        }
        // ---- a7 dynamics (FP64); the step's projections no longer read the TM scale: reset it
        for (int g = tid; g < gcount; g += NT) MI(g, Y.misc)[2] = 0;
        for (int idx = tid; idx < gcount * n * n; idx += NT) {
            const int g = idx / (n * n), r = idx - g * n * n, i = r / n, k = r - i * n;
            const double* P = MD(g, Y.P);
            const float* Gu = MF(g, Y.G);
            double acc = 0.0;
            for (int j = 0; j < n; ++j) acc = fma(A[i * n + j], P[j * n + k], acc);
            for (int j = 0; j < m; ++j) acc = fma(B[i * m + j], (double)Gu[j * gld + k], acc);
            MD(g, Y.Pn)[r] = acc;
        }
        for (int idx = tid; idx < gcount * n; idx += NT) {
            const int g = idx / n, i = idx - g * n;
            const double* c = MD(g, Y.c);
            const double* Ilo = MD(g, Y.Ilo);
            const double* Ihi = MD(g, Y.Ihi);
            const float* cu = MF(g, Y.cu);
            const float* Iulo = MF(g, Y.Iulo);
            const float* Iuhi = MF(g, Y.Iuhi);
            double acc = e[i] + (a.eoff ? a.eoff[((dbase + g) * H + t) * n + i] : 0.0), lo_ = 0.0, hi_ = 0.0;
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
            MD(g, Y.cn)[i] = acc;
            MD(g, Y.Ilon)[i] = lo_;
            MD(g, Y.Ihin)[i] = hi_;
        }
        __syncthreads();
        for (int idx = tid; idx < gcount * n * n; idx += NT) {
            const int g = idx / (n * n), r = idx - g * n * n;
            MD(g, Y.P)[r] = MD(g, Y.Pn)[r];
        }
        for (int idx = tid; idx < gcount * n; idx += NT) {
            const int g = idx / n, i = idx - g * n;
            MD(g, Y.c)[i] = MD(g, Y.cn)[i];
            MD(g, Y.Ilo)[i] = MD(g, Y.Ilon)[i];
            MD(g, Y.Ihi)[i] = MD(g, Y.Ihin)[i];
        }
        __syncthreads();
        // ---- a8 EvalInt; the width sum goes into red[1 + i]
        for (int idx = tid; idx < gcount * n; idx += NT) {
            const int g = idx / n, i = idx - g * n;
            const int64_t dom = dbase + g;
            const double* P = MD(g, Y.P);
            const double* v = MD(g, Y.v);
            const double c = MD(g, Y.c)[i], Ilo = MD(g, Y.Ilo)[i], Ihi = MD(g, Y.Ihi)[i], wv = MD(g, Y.w)[0];
            double pm = 0.0, pp = 0.0, mag = fabs(c) + fabs(Ilo) + fabs(Ihi) + fabs(wv);
            for (int k = 0; k < n; ++k) {
                const double x = P[i * n + k];
                pm += fabs(x - v[k]);
                pp += fabs(x + v[k]);
                mag += fabs(x) + fabs(v[k]);
            }
            const double bl = c + Ilo - pm - wv - a.box_margin * mag;
            const double bh = c + Ihi + pp + wv + a.box_margin * mag;
            if (a.lo) a.lo[(dom * (H + 1) + t + 1) * n + i] = bl;
            if (a.hi) a.hi[(dom * (H + 1) + t + 1) * n + i] = bh;
            MD(g, Y.red)[1 + i] += bh - bl;
            if (!isfinite(bl) || !isfinite(bh)) atomicOr(reinterpret_cast<unsigned int*>(MI(g, Y.misc) + 1), DR_STATUS_NONFINITE_BIT);
            if (bl > bh) atomicOr(reinterpret_cast<unsigned int*>(MI(g, Y.misc) + 1), DR_STATUS_INFEASIBLE_BIT);
        }
        __syncthreads();
    }
    for (int g = tid; g < gcount; g += NT) {
        double sum = 0.0;
        for (int i = 0; i < n; ++i) sum += MD(g, Y.red)[1 + i];
        if (a.V) a.V[dbase + g] = sum;
        if (a.status) a.status[dbase + g] = (uint32_t)MI(g, Y.misc)[1];
    }
}
