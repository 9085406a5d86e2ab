// Fused reverse sweep (adjoint) of the per-domain forward pass: dV/dalpha and dV/dbeta.
//
// Objective sum_{t,i} (g_lo lo_{t,i} + g_hi hi_{t,i}); the tube-volume proxy of Sec. V-A is
// g_lo = -1, g_hi = +1.  One CTA owns one domain.  Steps are reversed t = H-1..0; each step is recomputed
// from its tape entry (FP64 TM, dual state, split cursor) and then differentiated in exactly
// the reverse order of the forward: EvalInt, dynamics, then for each target layer
// l = L..1 the relaxation, split records, concretisation, input projection and the
// back-substitution chain (Lambda matrices recomputed per target, not stored per step).
// Subgradient conventions: |0|' = 0, Lambda^+/- have zero slope at 0, the intercept
// max(-alpha l, (1-alpha) u) takes the first branch on a tie.  The outward margin is treated
// as a constant.
#pragma once
#include "fused_core.cuh"

// Sums over a target's rows for few outputs (TM adjoints, dual adjoints): each output gets JS
// consecutive lanes (a power of two <= 32) that stride over the rows, then a shuffle tree.
template <int NT>
__device__ __forceinline__ int row_lanes(int items) {
    int js = 1;
    while (js < 32 && items * js * 2 <= NT) js <<= 1;
    return js;
}
__device__ __forceinline__ double lanes_sumd(double x, int js) {
    for (int o = js >> 1; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

template <int NT>
// Two CTAs per SM: narrow controllers fit twice in shared memory, and the register cap keeps that occupancy.
__global__ void __launch_bounds__(NT, 2) k_fused_backward(const FusedArgs a) {
    extern __shared__ __align__(16) unsigned char sm_dyn[];
    unsigned char* sm = a.gslab ? a.gslab + (int64_t)blockIdx.x * a.slab_stride : sm_dyn;
    const NetDesc& N = a.net;
    const FusedLayout& Y = a.lay;
    Dom s = make_dom(sm, Y);
    s.gw = a.gwpad;
    s.tiles = (NT == 256 && a.gslab) ? reinterpret_cast<float*>(sm_dyn) : nullptr;  // slab mode: GEMM tiles
    const int tid = threadIdx.x;
    const int64_t dom = a.d0 + blockIdx.x;
    const int n = N.n, m = N.m, L = N.L, H = N.H, gld = odd_ld(n);
    double* gc = SMD(Y.gc);
    double* gP = SMD(Y.gP);
    double* gIlo = SMD(Y.gIlo);
    double* gIhi = SMD(Y.gIhi);
    double* gcn = SMD(Y.gcn);
    double* gPn = SMD(Y.gPn);
    double* gIlon = SMD(Y.gIlon);
    double* gIhin = SMD(Y.gIhin);
    double* gPu = SMD(Y.gPu);
    double* gcu = SMD(Y.gcu);
    double* gIulo = SMD(Y.gIulo);
    double* gIuhi = SMD(Y.gIuhi);
    double* gv = SMD(Y.gv);
    double* gw = SMD(Y.gw);
    float* gs = SMF(Y.gs);
    float* gd = SMF(Y.gd);
    float* gl = SMF(Y.gl);
    float* gu = SMF(Y.gu);
    float* gG = SMF(Y.gG);
    float* ga = SMF(Y.ga);
    float* gklo = SMF(Y.gklo);
    float* gkhi = SMF(Y.gkhi);
    float* gRlo = SMF(Y.gRlo);
    float* gRhi = SMF(Y.gRhi);
    float* vsnap = SMF(Y.vsnap);
    float* lev = SMF(Y.lev);
    float* levall = Y.levall ? SMF(Y.levall) : nullptr;  // slab mode: every target's levels of the step
    float* kall = Y.kall ? SMF(Y.kall) : nullptr;

    load_params<NT>(s, a);
    for (int idx = tid; idx < n * n; idx += NT) gPn[idx] = 0.0;
    for (int i = tid; i < n; i += NT) {
        gcn[i] = 0.0;
        gIlon[i] = 0.0;
        gIhin[i] = 0.0;
        gv[i] = 0.0;
    }
    if (tid == 0) gw[0] = 0.0;
    const int64_t sp_end = a.sp_row ? a.sp_row[dom + 1] : 0;
    __syncthreads();

    for (int t = H - 1; t >= 0; --t) {
        // ---- recompute step t from its tape entry
        const double* tp = a.tape + (dom * H + t) * (int64_t)a.tape_stride;
        for (int idx = tid; idx < n * n; idx += NT) s.P[idx] = tp[idx];
        for (int i = tid; i < n; i += NT) {
            s.c[i] = tp[n * n + i];
            s.Ilo[i] = tp[n * n + n + i];
            s.Ihi[i] = tp[n * n + 2 * n + i];
            s.v[i] = tp[n * n + 3 * n + i];
        }
        if (tid == 0) {
            s.wv[0] = tp[n * n + 4 * n];
            s.misc[0] = (int)tp[n * n + 4 * n + 1];
            s.misc[1] = 0;
        }
        __syncthreads();
        const int cursor0 = s.misc[0];
        tm_view<NT>(s, n);
        controller_pass<NT>(s, N, a, dom, sp_end, t, vsnap, levall, kall);
        dynamics<NT>(s, N, a.eoff ? a.eoff + (dom * H + t) * (int64_t)n : nullptr);

        // ---- EvalInt of box t+1 (uses the dual state after step t)
        const int64_t wrow = (dom * (H + 1) + t + 1) * n;
        for (int i = tid; i < n; i += NT) {
            const double wl = a.wlo ? a.wlo[wrow + i] : -1.0;
            const double wh = a.whi ? a.whi[wrow + i] : 1.0;
            gcn[i] += wl + wh;
            gIlon[i] += wl;
            gIhin[i] += wh;
            for (int k = 0; k < n; ++k) {
                const double x = s.Pn[i * n + k];
                gPn[i * n + k] += -wl * sgnd(x - s.v[k]) + wh * sgnd(x + s.v[k]);
            }
        }
        for (int k = tid; k < n; k += NT) {
            double acc = 0.0;
            for (int i = 0; i < n; ++i) {
                const double wl = a.wlo ? a.wlo[wrow + i] : -1.0;
                const double wh = a.whi ? a.whi[wrow + i] : 1.0;
                const double x = s.Pn[i * n + k];
                acc += wl * sgnd(x - s.v[k]) + wh * sgnd(x + s.v[k]);
            }
            gv[k] += acc;
        }
        if (tid == 0) {
            double acc = 0.0;
            for (int i = 0; i < n; ++i) {
                const double wl = a.wlo ? a.wlo[wrow + i] : -1.0;
                const double wh = a.whi ? a.whi[wrow + i] : 1.0;
                acc += wh - wl;
            }
            gw[0] += acc;
        }
        __syncthreads();
        // gcn is now the whole adjoint of c_{t+1}: the gradient of a shift added after step t
        if (a.gshift)
            for (int i = tid; i < n; i += NT) a.gshift[(dom * (H + 1) + t + 1) * n + i] = gcn[i];

        // ---- dynamics reverse: TM_t and controller-TM adjoints
        for (int idx = tid; idx < n * n; idx += NT) {
            const int j = idx / n, k = idx - j * n;
            double acc = 0.0;
            for (int i = 0; i < n; ++i) acc += s.A[i * n + j] * gPn[i * n + k];
            gP[idx] = acc;
        }
        for (int idx = tid; idx < m * n; idx += NT) {
            const int j = idx / n, k = idx - j * n;
            double acc = 0.0;
            for (int i = 0; i < n; ++i) acc += s.B[i * m + j] * gPn[i * n + k];
            gPu[idx] = acc;
        }
        for (int j = tid; j < n; j += NT) {
            double c_ = 0.0, lo_ = 0.0, hi_ = 0.0;
            for (int i = 0; i < n; ++i) {
                const double x = s.A[i * n + j];
                c_ += x * gcn[i];
                lo_ += posd(x) * gIlon[i] + negd(x) * gIhin[i];
                hi_ += posd(x) * gIhin[i] + negd(x) * gIlon[i];
            }
            gc[j] = c_;
            gIlo[j] = lo_;
            gIhi[j] = hi_;
        }
        for (int j = tid; j < m; j += NT) {
            double c_ = 0.0, lo_ = 0.0, hi_ = 0.0;
            for (int i = 0; i < n; ++i) {
                const double x = s.B[i * m + j];
                c_ += x * gcn[i];
                lo_ += posd(x) * gIlon[i] + negd(x) * gIhin[i];
                hi_ += posd(x) * gIhin[i] + negd(x) * gIlon[i];
            }
            gcu[j] = c_;
            gIulo[j] = lo_;
            gIuhi[j] = hi_;
        }
        for (int j = tid; j < N.hidden; j += NT) {
            gs[j] = 0.f;
            gd[j] = 0.f;
        }
        __syncthreads();

        // ---- targets in reverse order
        for (int ell = L; ell >= 1; --ell) {
            const int rows = N.w[ell];
            int ld;
            const float* cur;
            float* levp = lev;  // this target's chain levels
            if (levall) {
                // kept by the replayed controller pass: no second evaluation of the chain
                if (ell >= 2) levp = levall + levall_offset(N, ell);
                cur = ell >= 2 ? levp + lev_offset(N, ell, 0) : s.W(0);
                ld = odd_ld(N.w[0]);
                const int ko = kall_offset(N, ell), kt = kall_total(N);
                for (int i = tid; i < rows; i += NT) {
                    s.klo[i] = kall[ko + i];
                    s.khi[i] = kall[kt + ko + i];
                }
                __syncthreads();
            } else {
                cur = chain<NT>(s, N, ell, lev, &ld);
            }
            if (ell < L) {
                for (int k = tid; k <= n; k += NT) s.vf[k] = vsnap[ell * (n + 1) + k];
                __syncthreads();
            }
            project<NT>(s, N, ell, cur, ld, a.rho, false);
            const float* vb = vsnap + ell * (n + 1);
            if (ell == L) {
                for (int i = tid; i < rows; i += NT) {
                    const float c_ = (float)gcu[i], dl = (float)(gIulo[i] - gIuhi[i]);
                    ga[i] = c_;
                    gklo[i] = 0.5f * c_ + 0.5f * dl;
                    gkhi[i] = 0.5f * c_ - 0.5f * dl;
                    gRlo[i] = (float)gIulo[i];
                    gRhi[i] = (float)gIuhi[i];
                    for (int k = 0; k < n; ++k) gG[i * gld + k] = (float)gPu[i * n + k];
                }
                __syncthreads();
            } else {
                const int ho = N.hoff[ell];
                // relaxation reverse (post-clip bounds), then the clip
                for (int j = tid; j < rows; j += NT) {
                    const float l = s.hl[ho + j], u = s.hu[ho + j];
                    const float g_s = gs[ho + j], g_d = gd[ho + j];
                    float g_l = 0.f, g_u = 0.f, g_a = 0.f;
                    if (l < 0.f && u > 0.f) {
                        const float user = a.mode == DR_SLOPE_USER_K ? a.alpha[(dom * H + t) * (int64_t)N.hidden + ho + j] : 0.f;
                        const float al = slope_of(a.mode, l, u, user);
                        const bool br = (-al * l) >= ((1.f - al) * u);
                        g_a = g_s + g_d * (br ? -l : -u);
                        if (br) g_l = g_d * (-al);
                        else g_u = g_d * (1.f - al);
                        if (a.mode == DR_SLOPE_CHORD_K) {
                            const float den = u - l;
                            g_l += g_a * u / (den * den);
                            g_u += g_a * (-l) / (den * den);
                        }
                    }
                    if (a.dalpha) a.dalpha[(dom * H + t) * (int64_t)N.hidden + ho + j] = (a.mode == DR_SLOPE_USER_K) ? g_a : 0.f;
                    if (s.hl0[ho + j] != l) g_l = 0.f;  // clipped by a split
                    if (s.hu0[ho + j] != u) g_u = 0.f;
                    gl[ho + j] = g_l;
                    gu[ho + j] = g_u;
                    ga[j] = 0.f;
                    gklo[j] = 0.f;
                    gkhi[j] = 0.f;
                    gRlo[j] = 0.f;
                    gRhi[j] = 0.f;
                    for (int k = 0; k < n; ++k) gG[j * gld + k] = 0.f;
                }
                __syncthreads();
                // split records of (t, ell): v += beta sign G_j, w += beta h (adjoint of the updated dual)
                if (tid == 0 && a.sp_row) {
                    for (int cpos = cursor0; cpos < sp_end; ++cpos) {
                        const SplitRec r = a.sp[cpos];
                        if (r.t > t) break;
                        if (r.t != t || r.layer != ell) continue;
                        const int j = r.neuron;
                        const float bt = a.beta ? a.beta[cpos] : 0.f;
                        const float hh = split_h(s, j, r.sign, a.rho);
                        double gb = gw[0] * (double)hh;
                        for (int k = 0; k < n; ++k) gb += gv[k] * (double)r.sign * (double)s.G[j * gld + k];
                        if (a.dbeta) a.dbeta[cpos] = (float)gb;
                        if (bt != 0.f) {
                            for (int k = 0; k < n; ++k) gG[j * gld + k] += (float)((double)bt * (double)r.sign * gv[k]);
                            const float hb = (float)((double)bt * gw[0]);
                            if (r.sign > 0) {
                                ga[j] += hb;
                                gkhi[j] += hb;
                                gRhi[j] += hb;
                            } else {
                                ga[j] -= hb;
                                gklo[j] -= hb;
                                gRlo[j] -= hb;
                            }
                        }
                    }
                }
                __syncthreads();
                // concretisation reverse (dual vector as seen by this layer)
                for (int i = tid; i < rows; i += NT) {
                    const float g_l = gl[ho + i], g_u = gu[ho + i];
                    ga[i] += g_l + g_u;
                    gklo[i] += g_l;
                    gkhi[i] += g_u;
                    gRlo[i] += g_l;
                    gRhi[i] += g_u;
                    for (int k = 0; k < n; ++k) {
                        const float x = s.G[i * gld + k];
                        gG[i * gld + k] += -g_l * sgnf(x - vb[k]) + g_u * sgnf(x + vb[k]);
                    }
                }
                {
                    // adjoint of the dual (v: n entries, w: entry n), rows split over JS lanes
                    const int items = n + 1, JS = row_lanes<NT>(items);
                    for (int base = 0; base < items * JS; base += NT) {
                        const int idx = base + tid;
                        const bool act = idx < items * JS;
                        const int k = idx / JS, jp = idx - k * JS;
                        double acc = 0.0;
                        if (act && k < n) {
                            for (int i = jp; i < rows; i += JS) {
                                const float x = s.G[i * gld + k];
                                acc += (double)(gl[ho + i] * sgnf(x - vb[k]) + gu[ho + i] * sgnf(x + vb[k]));
                            }
                        } else if (act) {
                            for (int i = jp; i < rows; i += JS) acc += (double)(gu[ho + i] - gl[ho + i]);
                        }
                        acc = lanes_sumd(acc, JS);
                        if (act && jp == 0) {
                            if (k < n) gv[k] += acc;
                            else gw[0] += acc;
                        }
                    }
                }
                __syncthreads();
            }
            // ---- input projection reverse: TM adjoints and Lambda_x adjoint
            {
                // gP[j][k] += sum_i Lx[i][j] gG[i][k]; gc, gIlo, gIhi likewise; rows split over JS lanes
                const int items = n * n + n, JS = row_lanes<NT>(items);
                for (int base = 0; base < items * JS; base += NT) {
                    const int idx = base + tid;
                    const bool act = idx < items * JS;
                    const int it = idx / JS, jp = idx - it * JS;
                    double acc = 0.0, lo_ = 0.0, hi_ = 0.0;
                    if (act && it < n * n) {
                        const int j = it / n, k = it - j * n;
                        for (int i = jp; i < rows; i += JS) acc += (double)(cur[i * ld + j] * gG[i * gld + k]);
                    } else if (act) {
                        const int j = it - n * n;
                        for (int i = jp; i < rows; i += JS) {
                            const float x = cur[i * ld + j];
                            acc += (double)(x * ga[i]);
                            lo_ += (double)(gRlo[i] * posf(x) + gRhi[i] * negf(x));
                            hi_ += (double)(gRlo[i] * negf(x) + gRhi[i] * posf(x));
                        }
                    }
                    acc = lanes_sumd(acc, JS);
                    lo_ = lanes_sumd(lo_, JS);
                    hi_ = lanes_sumd(hi_, JS);
                    if (act && jp == 0) {
                        if (it < n * n) {
                            gP[it] += acc;
                        } else {
                            const int j = it - n * n;
                            gc[j] += acc;
                            gIlo[j] += lo_;
                            gIhi[j] += hi_;
                        }
                    }
                }
            }
            float* gLprev = SMF(Y.gL0);  // adjoint of Lambda^(0) = Lambda_x
            const int xld = odd_ld(n);
            if (ell > 1 || a.gth) {
                for (int idx = tid; idx < rows * n; idx += NT) {
                    const int i = idx / n, j = idx - i * n;
                    const float x = cur[i * ld + j];
                    float acc = ga[i] * s.cf[j];
                    for (int k = 0; k < n; ++k) acc = fmaf(gG[i * gld + k], s.Pf[j * n + k], acc);
                    acc += gRlo[i] * (x > 0.f ? s.Ilof[j] : (x < 0.f ? s.Ihif[j] : 0.f));
                    acc += gRhi[i] * (x > 0.f ? s.Ihif[j] : (x < 0.f ? s.Ilof[j] : 0.f));
                    gLprev[i * xld + j] = acc;
                }
            }
            __syncthreads();
            // ---- chain reverse, levels mm = 1 .. ell-1
            int prev_ld = xld;
            int buf = 1;
            for (int mm = 1; mm <= ell - 1; ++mm) {
                const int K = N.w[mm], NN = N.w[mm - 1];
                const float* Wm = s.W(mm - 1);
                const int wld = odd_ld(NN);
                const float* Lm = (mm == ell - 1) ? s.W(ell - 1) : (levp + lev_offset(N, ell, mm));
                const int lmld = odd_ld(K);
                const float* sl = s.hs + N.hoff[mm];
                const float* dl = s.hd + N.hoff[mm];
                const float* bm = s.bs + N.boff[mm - 1];
                float* gLnext = SMF(buf ? Y.gL1 : Y.gL0);
                // column j of Lambda_s adjoint: sum_k gLprev[i][k] W_m[j][k] + (gklo_i + gkhi_i) b_m[j]
                const int ncg = (K + 3) >> 2;
                if (NT == 256 && s.tiles && rows >= 32 && K >= 32 && NN >= 32) {
                    // slab mode: the products through shared-memory tiles into gLnext (used as scratch
                    // also on the last level), then per column the same epilogue as below
                    gemm_nt_tiled256(gLprev, prev_ld, Wm, wld, gLnext, lmld, rows, K, NN, gklo, gkhi, bm, s.tiles);
                    for (int j = tid; j < K; j += NT) {
                        float acc_s = 0.f, acc_d = 0.f;
                        for (int i = 0; i < rows; ++i) {
                            const float gls = gLnext[i * lmld + j];
                            const float x = Lm[i * lmld + j];
                            acc_s = fmaf(gls, x, acc_s);
                            acc_d += gkhi[i] * posf(x) + gklo[i] * negf(x);
                            if (mm < ell - 1 || a.gth)
                                gLnext[i * lmld + j] = gls * sl[j] + gkhi[i] * (x > 0.f ? dl[j] : 0.f) + gklo[i] * (x < 0.f ? dl[j] : 0.f);
                        }
                        gs[N.hoff[mm] + j] += acc_s;
                        gd[N.hoff[mm] + j] += acc_d;
                    }
                } else if (ncg * 2 >= NT && rows >= 4) {
                    // wide level: a thread owns 4 columns and walks the rows in blocks of 4 (4 x 4
                    // register tile per block); per element the same operation order as below
                    for (int cg = tid; cg < ncg; cg += NT) {
                        const int j0 = cg << 2;
                        int jj[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) jj[q] = min(j0 + q, K - 1);
                        float acc_s[4] = {0.f, 0.f, 0.f, 0.f}, acc_d[4] = {0.f, 0.f, 0.f, 0.f};
                        for (int i0 = 0; i0 < rows; i0 += 4) {
                            int ii[4];
                            float g[4][4];
#pragma unroll
                            for (int r = 0; r < 4; ++r) {
                                ii[r] = min(i0 + r, rows - 1);
                                const float gk = gklo[ii[r]] + gkhi[ii[r]];
#pragma unroll
                                for (int q = 0; q < 4; ++q) g[r][q] = gk * bm[jj[q]];
                            }
                            for (int k = 0; k < NN; ++k) {
                                float pv[4], wv[4];
#pragma unroll
                                for (int r = 0; r < 4; ++r) pv[r] = gLprev[ii[r] * prev_ld + k];
#pragma unroll
                                for (int q = 0; q < 4; ++q) wv[q] = Wm[jj[q] * wld + k];
#pragma unroll
                                for (int r = 0; r < 4; ++r)
#pragma unroll
                                    for (int q = 0; q < 4; ++q) g[r][q] = fmaf(pv[r], wv[q], g[r][q]);
                            }
#pragma unroll
                            for (int r = 0; r < 4; ++r) {
                                if (i0 + r >= rows) break;
                                const int i = i0 + r;
#pragma unroll
                                for (int q = 0; q < 4; ++q) {
                                    const int j = j0 + q;
                                    if (j >= K) break;
                                    const float x = Lm[i * lmld + j];
                                    acc_s[q] = fmaf(g[r][q], x, acc_s[q]);
                                    acc_d[q] += gkhi[i] * posf(x) + gklo[i] * negf(x);
                                    if (mm < ell - 1 || a.gth)
                                        gLnext[i * lmld + j] = g[r][q] * sl[j] + gkhi[i] * (x > 0.f ? dl[j] : 0.f) +
                                                               gklo[i] * (x < 0.f ? dl[j] : 0.f);
                                }
                            }
                        }
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            if (j0 + q >= K) break;
                            gs[N.hoff[mm] + j0 + q] += acc_s[q];
                            gd[N.hoff[mm] + j0 + q] += acc_d[q];
                        }
                    }
                } else
                for (int j = tid; j < K; j += NT) {
                    float acc_s = 0.f, acc_d = 0.f;
                    for (int i = 0; i < rows; ++i) {
                        float gls = (gklo[i] + gkhi[i]) * bm[j];
                        const float* pr = gLprev + i * prev_ld;
                        for (int k = 0; k < NN; ++k) gls = fmaf(pr[k], Wm[j * wld + k], gls);
                        const float x = Lm[i * lmld + j];
                        acc_s = fmaf(gls, x, acc_s);
                        acc_d += gkhi[i] * posf(x) + gklo[i] * negf(x);
                        if (mm < ell - 1 || a.gth) {
                            gLnext[i * lmld + j] = gls * sl[j] + gkhi[i] * (x > 0.f ? dl[j] : 0.f) + gklo[i] * (x < 0.f ? dl[j] : 0.f);
                        }
                    }
                    gs[N.hoff[mm] + j] += acc_s;
                    gd[N.hoff[mm] + j] += acc_d;
                }
                if (a.gth) {
                    // dV/dW_mm += (Lambda diag(s_mm))^T gLprev and dV/db_mm += (Lambda diag(s_mm))^T (gklo + gkhi):
                    // the level's product Lambda_s W_mm and its intercept Lambda_s b_mm
                    float* th = a.gth + (int64_t)blockIdx.x * a.gth_stride;
                    float* gWm = th + N.Woff[mm - 1];
                    for (int e = tid; e < K * NN; e += NT) {
                        const int j = e / NN, k = e - j * NN;
                        const float sj = sl[j];
                        if (sj == 0.f) continue;
                        float acc = 0.f;
                        for (int i = 0; i < rows; ++i) acc = fmaf(Lm[i * lmld + j], gLprev[i * prev_ld + k], acc);
                        gWm[e] += sj * acc;
                    }
                    float* gbm = th + a.gth_boff + N.boff[mm - 1];
                    for (int j = tid; j < K; j += NT) {
                        float acc = 0.f;
                        for (int i = 0; i < rows; ++i) acc = fmaf(Lm[i * lmld + j], gklo[i] + gkhi[i], acc);
                        gbm[j] += sl[j] * acc;
                    }
                }
                __syncthreads();
                gLprev = gLnext;
                prev_ld = lmld;
                buf ^= 1;
            }
            if (a.gth) {
                // the target's own layer: Lambda starts as W_ell (its adjoint is now gLprev) and kappa as b_ell
                float* th = a.gth + (int64_t)blockIdx.x * a.gth_stride;
                float* gWl = th + N.Woff[ell - 1];
                const int cols = N.w[ell - 1];
                for (int e = tid; e < rows * cols; e += NT) {
                    const int i = e / cols, j = e - i * cols;
                    gWl[e] += gLprev[i * prev_ld + j];
                }
                float* gbl = th + a.gth_boff + N.boff[ell - 1];
                for (int i = tid; i < rows; i += NT) gbl[i] += gklo[i] + gkhi[i];
                __syncthreads();
            }
        }
        // ---- TM_t adjoint becomes the incoming adjoint of the previous step
        for (int idx = tid; idx < n * n; idx += NT) gPn[idx] = gP[idx];
        for (int i = tid; i < n; i += NT) {
            gcn[i] = gc[i];
            gIlon[i] = gIlo[i];
            gIhin[i] = gIhi[i];
        }
        __syncthreads();
    }
    // after step 0: the adjoint of the initial centre c_0
    if (a.gshift)
        for (int i = tid; i < n; i += NT) a.gshift[(dom * (H + 1)) * n + i] = gcn[i];
}

// Keep-best per domain: if V improved, remember the slopes and multipliers.
__global__ void k_keep_best(const double* __restrict__ V, double* __restrict__ bestV, const float* __restrict__ alpha,
                            float* __restrict__ best_alpha, const float* __restrict__ beta, float* __restrict__ best_beta,
                            const int64_t* __restrict__ sp_row, int64_t per_dom) {
    const int64_t d = blockIdx.x;
    __shared__ int better;
    if (threadIdx.x == 0) {
        better = V[d] < bestV[d];
        if (better) bestV[d] = V[d];
    }
    __syncthreads();
    if (!better) return;
    for (int64_t i = threadIdx.x; i < per_dom; i += blockDim.x) best_alpha[d * per_dom + i] = alpha[d * per_dom + i];
    if (sp_row)
        for (int64_t k = sp_row[d] + threadIdx.x; k < sp_row[d + 1]; k += blockDim.x) best_beta[k] = beta[k];
}

// Projected gradient step: x <- clip(x - lr g, lo, hi).
__global__ void k_pgd(float* __restrict__ x, const float* __restrict__ g, int64_t cnt, float lr, float lo, float hi) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = fminf(fmaxf(x[i] - lr * g[i], lo), hi);
}

// Sum of v[0..D) into hist[*slot], then *slot += 1: the slot index lives on the device, so one
// captured refinement step (CUDA graph) writes the next history entry on every replay.
__global__ void k_sum_hist(const double* __restrict__ v, int64_t D, double* __restrict__ hist, int* __restrict__ slot) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < D; i += blockDim.x) acc += v[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int k = *slot;
        hist[k] = red[0];
        *slot = k + 1;
    }
}

// Sum of D values into out[0] (single block, deterministic order per thread then tree).
__global__ void k_sum(const double* __restrict__ v, int64_t D, double* __restrict__ out) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < D; i += blockDim.x) acc += v[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

// Weight gradient, first half of the reduction over the per-domain slices: part[g][e] = sum of
// slice[s][e] over s = g, g + G, ... (G = gridDim.y).  Threads of a warp read consecutive e of one
// slice; the fixed order makes the sum deterministic.
__global__ void k_theta_partial(const float* __restrict__ slices, int64_t nslices, int64_t stride, int64_t count,
                                double* __restrict__ part) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= count) return;
    double acc = 0.0;
    for (int64_t s = blockIdx.y; s < nslices; s += gridDim.y) acc += (double)slices[s * stride + e];
    part[(int64_t)blockIdx.y * count + e] = acc;
}

// Second half: out[e] += sum over the G partial sums (out accumulates over the backward chunks).
__global__ void k_theta_finish(const double* __restrict__ part, int groups, int64_t count, double* __restrict__ out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= count) return;
    double acc = 0.0;
    for (int g = 0; g < groups; ++g) acc += part[(int64_t)g * count + e];
    out[e] += acc;
}
