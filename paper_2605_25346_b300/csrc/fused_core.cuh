// Per-domain phases of one closed-loop step in shared memory, shared by the fused forward
// kernel and the fused reverse (adjoint) kernel.
//
// Step of Alg. 2 for the closed loop of Sec. IV-E:
//   FP64 TM -> FP32 view (remainder widened to cover the cast) -> for each layer l:
//   back-substitution chain Lambda <- (Lambda diag(s_m)) W_m with Lambda^+/- intercepts
//   (Thm. 2), concretisation over the TM input (Thm. 3) with the split dual and the outward
//   margin rho*S, shared-slope relaxation (Sec. IV-C) -> controller TM -> FP64 dynamics and
//   EvalInt.
#pragma once
#include "common.cuh"
#include "tiles.cuh"

struct FusedLayout {  // byte offsets into dynamic shared memory
    int Ws[DR_MAXL];
    int bs;
    int A, B, e;
    int c, P, Ilo, Ihi, v, w;
    int cn, Pn, Ilon, Ihin;
    int cf, Pf, Ilof, Ihif, vf;  // vf holds n floats followed by wf
    int hl, hu, hs, hd;
    int hl0, hu0;                // pre-clip bounds (reverse kernel only; alias hl/hu otherwise)
    int klo, khi;
    int lam0, lam1;              // forward ping-pong chain buffers
    int G;
    int a, Rlo, Rhi, S;
    int cu, Iulo, Iuhi;
    int misc;  // ints: [0] split cursor, [1] status
    // reverse kernel only
    int vsnap;                   // [L][n+1] floats: dual vector seen by each hidden layer
    int lev;                     // chain levels of one target (offsets from lev_offset)
    int levall, kall;            // slab mode: every target's levels and kappa of one step (0: not kept)
    int gc, gP, gIlo, gIhi;      // adjoint of TM_t (double)
    int gcn, gPn, gIlon, gIhin;  // adjoint of TM_{t+1} (double)
    int gPu, gcu, gIulo, gIuhi;  // adjoint of the controller TM (double)
    int gv, gw;                  // adjoint of the dual state (double)
    int gs, gd, gl, gu;          // per hidden neuron (float)
    int gG, ga, gklo, gkhi, gRlo, gRhi;  // adjoint of one target's concretisation (float)
    int gL0, gL1;                // ping-pong Lambda adjoints
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
    const double* eoff;  // [D][H][n] per-step offsets of the dynamics (added after step t) or null
    const double* lo0;  // [D][n]
    const double* hi0;
    int64_t d0;         // first domain of this launch
    const int64_t* sp_row;  // [D+1] or null
    const SplitRec* sp;     // [nnz]
    const float* beta;      // [nnz] or null
    const float* alpha;     // [D][H][hidden] (USER) or null
    int mode;
    float rho;
    double box_margin;
    double* lo;  // [D][H+1][n] or null
    double* hi;
    double* V;          // [D] or null
    uint32_t* status;   // [D] or null
    float* alpha_used;  // [D][H][hidden] or null
    double* tape;       // [D][H][tape_stride] or null
    int tape_stride;
    // wide controllers: the working set lives in a per-CTA slab of global memory instead of
    // dynamic shared memory (slab of CTA b at gslab + b * slab_stride)
    unsigned char* gslab;
    int64_t slab_stride;
    const float* gwpad;  // slab mode: one padded weight copy shared by all CTAs (offsets Ws[l] - Ws[0])
    // reverse kernel
    double* gshift;     // [D][H+1][n] dV/d(shift of the TM centre at step t) or null
    const double* wlo;  // [D][H+1][n] upstream gradient of lo (null: -1 on steps 1..H)
    const double* whi;  // [D][H+1][n] upstream gradient of hi (null: +1 on steps 1..H)
    float* dalpha;      // [D][H][hidden] or null
    float* dbeta;       // [nnz] or null
    // weight gradient: per-CTA slices gth + blockIdx.x * gth_stride of dV/dW (packed as NetDesc::Woff)
    // followed at gth_boff by dV/db (packed as NetDesc::boff), accumulated by the CTA; null = off
    float* gth;
    int64_t gth_stride;
    int64_t gth_boff;
};

#define SMF(off) reinterpret_cast<float*>(sm + (off))
#define SMD(off) reinterpret_cast<double*>(sm + (off))
#define SMI(off) reinterpret_cast<int*>(sm + (off))

// Shared-memory views of one domain's working set.
struct Dom {
    unsigned char* sm;
    const FusedLayout* Y;
    const float* gw;  // shared padded weights in global memory (slab mode), else null
    float* tiles;     // slab mode with 256 threads: shared-memory GEMM tiles (kSlabTileFloats), else null
    double *c, *P, *Ilo, *Ihi, *v, *wv, *cn, *Pn, *Ilon, *Ihin, *A, *B, *e;
    float *cf, *Pf, *Ilof, *Ihif, *vf, *hl, *hu, *hs, *hd, *hl0, *hu0, *klo, *khi, *G, *sa, *sRlo, *sRhi, *sS, *cu,
        *Iulo, *Iuhi, *bs;
    int* misc;
    __device__ float* W(int l) const {
        return gw ? const_cast<float*>(gw) + (Y->Ws[l] - Y->Ws[0]) / 4 : reinterpret_cast<float*>(sm + Y->Ws[l]);
    }
};

__device__ __forceinline__ Dom make_dom(unsigned char* sm, const FusedLayout& Y) {
    Dom s;
    s.sm = sm;
    s.Y = &Y;
    s.gw = nullptr;
    s.tiles = nullptr;
    s.c = SMD(Y.c);
    s.P = SMD(Y.P);
    s.Ilo = SMD(Y.Ilo);
    s.Ihi = SMD(Y.Ihi);
    s.v = SMD(Y.v);
    s.wv = SMD(Y.w);
    s.cn = SMD(Y.cn);
    s.Pn = SMD(Y.Pn);
    s.Ilon = SMD(Y.Ilon);
    s.Ihin = SMD(Y.Ihin);
    s.A = SMD(Y.A);
    s.B = SMD(Y.B);
    s.e = SMD(Y.e);
    s.cf = SMF(Y.cf);
    s.Pf = SMF(Y.Pf);
    s.Ilof = SMF(Y.Ilof);
    s.Ihif = SMF(Y.Ihif);
    s.vf = SMF(Y.vf);
    s.hl = SMF(Y.hl);
    s.hu = SMF(Y.hu);
    s.hs = SMF(Y.hs);
    s.hd = SMF(Y.hd);
    s.hl0 = SMF(Y.hl0);
    s.hu0 = SMF(Y.hu0);
    s.klo = SMF(Y.klo);
    s.khi = SMF(Y.khi);
    s.G = SMF(Y.G);
    s.sa = SMF(Y.a);
    s.sRlo = SMF(Y.Rlo);
    s.sRhi = SMF(Y.Rhi);
    s.sS = SMF(Y.S);
    s.cu = SMF(Y.cu);
    s.Iulo = SMF(Y.Iulo);
    s.Iuhi = SMF(Y.Iuhi);
    s.bs = SMF(Y.bs);
    s.misc = SMI(Y.misc);
    return s;
}

template <int NT>
__device__ void load_params(const Dom& s, const FusedArgs& a) {
    const NetDesc& N = a.net;
    const int tid = threadIdx.x, n = N.n, m = N.m;
    for (int l = 0; l < N.L && !s.gw; ++l) {
        const int rows = N.w[l + 1], cols = N.w[l], ld = odd_ld(cols);
        float* dst = s.W(l);
        const float* src = a.W + N.Woff[l];
        for (int idx = tid; idx < rows * cols; idx += NT) {
            const int r = idx / cols, q = idx - r * cols;
            dst[r * ld + q] = src[idx];
        }
    }
    int nb = 0;
    for (int l = 0; l < N.L; ++l) nb += N.w[l + 1];
    for (int idx = tid; idx < nb; idx += NT) s.bs[idx] = a.b[idx];
    for (int idx = tid; idx < n * n; idx += NT) s.A[idx] = a.A[idx];
    for (int idx = tid; idx < n * m; idx += NT) s.B[idx] = a.B[idx];
    for (int i = tid; i < n; i += NT) s.e[i] = a.e ? a.e[i] : 0.0;
}

// FP32 view of the FP64 TM; the remainder absorbs the rounding of c and P, the dual offset
// absorbs the rounding of v.  Ends with a barrier.
template <int NT>
__device__ void tm_view(const Dom& s, int n) {
    const int tid = threadIdx.x;
    if (tid == 0) s.misc[2] = 0;  // the previous step's projections are done (the step ended with a barrier)
    __syncthreads();
    for (int idx = tid; idx < n * n; idx += NT) s.Pf[idx] = (float)s.P[idx];
    for (int i = tid; i < n; i += NT) {
        const float ci = (float)s.c[i];
        // row i of tm_scale (common.cuh), in its order; the maximum over rows by atomicMax on the
        // float's bits (a NaN row is skipped, as fmaxf skips it), instead of one thread doing all rows
        float rs = fabsf(ci) + fmaxf(fabsf((float)s.Ilo[i]), fabsf((float)s.Ihi[i]));
        for (int k = 0; k < n; ++k) rs += fabsf((float)s.P[i * n + k]);
        if (!isnan(rs)) atomicMax(reinterpret_cast<unsigned int*>(s.misc + 2), __float_as_uint(rs));
        double dev = 0.0;
        for (int k = 0; k < n; ++k) dev += fabs(s.P[i * n + k] - (double)(float)s.P[i * n + k]);
        const double dc = s.c[i] - (double)ci;
        s.cf[i] = ci;
        s.Ilof[i] = __double2float_rd(s.Ilo[i] + dc - dev);
        s.Ihif[i] = __double2float_ru(s.Ihi[i] + dc + dev);
    }
    if (tid == 0) {
        double dv = 0.0;
        for (int k = 0; k < n; ++k) {
            s.vf[k] = (float)s.v[k];
            dv += fabs(s.v[k] - (double)s.vf[k]);
        }
        s.vf[n] = __double2float_ru(s.wv[0] + dv);
    }
    __syncthreads();
}

// Offset (floats) of Lambda^(k) of target ell inside the level store: Lambda^(k) is
// n_ell x odd_ld(n_k), stored for k = 0 .. ell-2.
__host__ __device__ __forceinline__ int lev_offset(const NetDesc& N, int ell, int k) {
    int off = 0;
    for (int q = 0; q < k; ++q) off += N.w[ell] * odd_ld(N.w[q]);
    return off;
}

// Slab mode keeps one step's chain levels of every target (levall) and their kappa (kall), so the
// reverse sweep need not evaluate each chain a second time: target ell's levels start at
// levall_offset(N, ell) floats; its kappa_lo at kall_offset(N, ell), kappa_hi kall_total(N) later.
__host__ __device__ __forceinline__ int levall_offset(const NetDesc& N, int ell) {
    int off = 0;
    for (int l = 2; l < ell; ++l) off += lev_offset(N, l, l - 1);
    return off;
}
__host__ __device__ __forceinline__ int kall_offset(const NetDesc& N, int ell) {
    int off = 0;
    for (int l = 1; l < ell; ++l) off += N.w[l];
    return off;
}
__host__ __device__ __forceinline__ int kall_total(const NetDesc& N) { return kall_offset(N, N.L + 1); }

// a4: back-substitution chain of target layer ell.  Initialises kappa to b_ell, walks the
// levels m = ell-1..1 and returns Lambda_x (rows n_ell, ld *ld) in shared memory.  With
// `lev` non-null every level's matrix Lambda^(m-1) is kept at lev + lev_offset(N, ell, m-1).
template <int NT>
__device__ const float* chain(const Dom& s, const NetDesc& N, int ell, float* lev, int* out_ld) {
    const int tid = threadIdx.x;
    const int rows = N.w[ell];
    const float* bl = s.bs + N.boff[ell - 1];
    for (int i = tid; i < rows; i += NT) {
        s.klo[i] = bl[i];
        s.khi[i] = bl[i];
    }
    const float* cur = s.W(ell - 1);
    int cur_ld = odd_ld(N.w[ell - 1]);
    int cur_cols = N.w[ell - 1];
    int buf = 0;
    __syncthreads();
    for (int mm = ell - 1; mm >= 1; --mm) {
        const float* sl = s.hs + N.hoff[mm];
        const float* dl = s.hd + N.hoff[mm];
        const float* bm = s.bs + N.boff[mm - 1];
        // intercept sums: a short target (fewer rows than threads) splits each row's columns over JS
        // consecutive lanes (a power of two <= 32) and reduces them with shuffles
        int JS = 1;
        while (JS < 32 && rows * JS * 2 <= NT) JS <<= 1;
        for (int base = 0; base < rows * JS; base += NT) {
            const int idx = base + tid;
            const bool act = idx < rows * JS;
            const int i = idx / JS, jp = idx - i * JS;
            float spos = 0.f, sneg = 0.f, sb = 0.f;
            if (act) {
                const float* row = cur + i * cur_ld;
                for (int j = jp; j < cur_cols; j += JS) {
                    const float x = row[j];
                    spos = fmaf(posf(x), dl[j], spos);
                    sneg = fmaf(negf(x), dl[j], sneg);
                    sb = fmaf(x * sl[j], bm[j], sb);
                }
            }
            for (int o = JS >> 1; o > 0; o >>= 1) {
                spos += __shfl_xor_sync(0xffffffffu, spos, o);
                sneg += __shfl_xor_sync(0xffffffffu, sneg, o);
                sb += __shfl_xor_sync(0xffffffffu, sb, o);
            }
            if (act && jp == 0) {
                s.khi[i] += spos + sb;
                s.klo[i] += sneg + sb;
            }
        }
        const int K = N.w[mm], NN = N.w[mm - 1];
        const float* Wm = s.W(mm - 1);
        const int wld = odd_ld(NN);
        float* nxt = lev ? (lev + lev_offset(N, ell, mm - 1)) : reinterpret_cast<float*>(s.sm + (buf ? s.Y->lam1 : s.Y->lam0));
        const int nld = odd_ld(NN);
        // nxt[i][k] = sum_j (row_i[j] s_j) W_m[j][k]: register tiles when they still give every
        // thread of the CTA work (wide levels), one element per thread otherwise
        if (NT == 256 && s.tiles && rows >= 32 && K >= 32 && NN >= 32)
            gemm_nn_scaled_tiled256(cur, cur_ld, sl, Wm, wld, nxt, nld, rows, K, NN, s.tiles);
        else if (((rows + 3) >> 2) * ((NN + 3) >> 2) >= NT)
            gemm_stacked_scaled_t<NT, 4>(cur, 0, cur_ld, sl, 0, Wm, wld, nxt, nld, 1, rows, K, NN);
        else if (rows * ((NN + 3) >> 2) >= NT)
            gemm_stacked_scaled_t<NT, 1>(cur, 0, cur_ld, sl, 0, Wm, wld, nxt, nld, 1, rows, K, NN);
        else
            gemm_stacked_scaled_1<NT>(cur, 0, cur_ld, sl, 0, Wm, wld, nxt, nld, 1, rows, K, NN);
        __syncthreads();
        cur = nxt;
        cur_ld = nld;
        cur_cols = NN;
        buf ^= 1;
    }
    *out_ld = cur_ld;
    return cur;
}

// a5/a6: concretisation of target ell over the TM input.  Hidden targets write the (pre-clip)
// bounds into hl/hu (and hl0/hu0) and keep a, R, S for the split records; the output target
// writes the controller TM (P_u stays in G).  Uses the dual vector vf (wf = vf[n]).
template <int NT>
__device__ void project(const Dom& s, const NetDesc& N, int ell, const float* cur, int cur_ld, float rho,
                        bool write_bounds = true) {
    const int tid = threadIdx.x, n = N.n, L = N.L, rows = N.w[ell];
    const int gld = odd_ld(n);
    for (int idx = tid; idx < rows * n; idx += NT) {
        const int i = idx / n, k = idx - i * n;
        const float* row = cur + i * cur_ld;
        float acc = 0.f;
        for (int j = 0; j < n; ++j) acc = fmaf(row[j], s.Pf[j * n + k], acc);
        s.G[i * gld + k] = acc;
    }
    __syncthreads();
    for (int i = tid; i < rows; i += NT) {
        const float* row = cur + i * cur_ld;
        float av = 0.f, rlo = 0.f, rhi = 0.f;
        for (int j = 0; j < n; ++j) {
            const float x = row[j];
            av = fmaf(x, s.cf[j], av);
            rlo = fmaf(posf(x), s.Ilof[j], fmaf(negf(x), s.Ihif[j], rlo));
            rhi = fmaf(posf(x), s.Ihif[j], fmaf(negf(x), s.Ilof[j], rhi));
        }
        float g1 = 0.f, gm = 0.f, gp = 0.f;
        for (int k = 0; k < n; ++k) {
            const float gk = s.G[i * gld + k];
            g1 += fabsf(gk);
            gm += fabsf(gk - s.vf[k]);
            gp += fabsf(gk + s.vf[k]);
        }
        const float wf = s.vf[n];
        const float S = fabsf(av) + g1 + fabsf(s.klo[i]) + fabsf(s.khi[i]) + fabsf(rlo) + fabsf(rhi) + fabsf(wf);
        if (S > DR_MARGIN_RATIO * __int_as_float(s.misc[2])) atomicOr(reinterpret_cast<unsigned int*>(&s.misc[1]), DR_STATUS_MARGIN_BIT);
        if (ell < L) {
            const float lb = av + s.klo[i] + rlo - gm - wf - rho * S;
            const float ub = av + s.khi[i] + rhi + gp + wf + rho * S;
            if (write_bounds) {
                s.hl[N.hoff[ell] + i] = lb;
                s.hu[N.hoff[ell] + i] = ub;
                s.hl0[N.hoff[ell] + i] = lb;
                s.hu0[N.hoff[ell] + i] = ub;
            }
            s.sa[i] = av;
            s.sRlo[i] = rlo;
            s.sRhi[i] = rhi;
            s.sS[i] = S;
        } else {
            s.cu[i] = av + 0.5f * (s.klo[i] + s.khi[i]);
            s.Iulo[i] = 0.5f * (s.klo[i] - s.khi[i]) + rlo - rho * S;
            s.Iuhi[i] = 0.5f * (s.khi[i] - s.klo[i]) + rhi + rho * S;
        }
    }
    __syncthreads();
}

// The constraint value h of a split at neuron j of the current target (outward by the margin).
__device__ __forceinline__ float split_h(const Dom& s, int j, int sign, float rho) {
    return sign > 0 ? (s.sa[j] + s.khi[j] + s.sRhi[j] + rho * s.sS[j]) : (-(s.sa[j] + s.klo[j] + s.sRlo[j]) + rho * s.sS[j]);
}

// Split constraints of (t, ell): clip the bounds, record g^T zeta + h >= 0 in the dual.
// Thread 0 walks the domain's sorted list from the cursor misc[0].  Ends with a barrier.
__device__ void apply_splits(const Dom& s, const NetDesc& N, const FusedArgs& a, int64_t sp_end, int t, int ell,
                             float rho) {
    const int n = N.n, gld = odd_ld(n);
    if (threadIdx.x == 0 && a.sp_row) {
        float* lh = s.hl + N.hoff[ell];
        float* uh = s.hu + N.hoff[ell];
        int cpos = s.misc[0];
        bool changed = false;
        while (cpos < sp_end) {
            const SplitRec r = a.sp[cpos];
            if (r.t > t || (r.t == t && r.layer > ell)) break;
            if (r.t == t && r.layer == ell) {
                const int j = r.neuron;
                const float bt = a.beta ? a.beta[cpos] : 0.f;
                const float hh = split_h(s, j, r.sign, rho);
                if (r.sign > 0) {
                    if (lh[j] < 0.f) lh[j] = 0.f;
                } else {
                    if (uh[j] > 0.f) uh[j] = 0.f;
                }
                if (bt != 0.f) {
                    for (int k = 0; k < n; ++k) s.v[k] += (double)bt * (double)r.sign * (double)s.G[j * gld + k];
                    s.wv[0] += (double)bt * (double)hh;
                    changed = true;
                }
            }
            ++cpos;
        }
        s.misc[0] = cpos;
        if (changed) {
            double dv = 0.0;
            for (int k = 0; k < n; ++k) {
                s.vf[k] = (float)s.v[k];
                dv += fabs(s.v[k] - (double)s.vf[k]);
            }
            s.vf[n] = __double2float_ru(s.wv[0] + dv);
        }
    }
    __syncthreads();
}

__device__ __forceinline__ float slope_of(int mode, float l, float u, float user) {
    if (mode == DR_SLOPE_CHORD_K) return u / (u - l);
    if (mode == DR_SLOPE_ADAPTIVE_K) return (u >= -l) ? 1.f : 0.f;
    if (mode == DR_SLOPE_ZERO_K) return 0.f;
    return user;
}

// a3: shared-slope relaxation of hidden layer ell (after the splits).  Ends with a barrier.
template <int NT>
__device__ void relax(const Dom& s, const NetDesc& N, const FusedArgs& a, int64_t dom, int t, int ell) {
    const int rows = N.w[ell], H = N.H;
    for (int j = threadIdx.x; j < rows; j += NT) {
        const float l = s.hl[N.hoff[ell] + j], u = s.hu[N.hoff[ell] + j];
        if (l > u) atomicOr(reinterpret_cast<unsigned int*>(&s.misc[1]), DR_STATUS_INFEASIBLE_BIT);
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
        s.hs[N.hoff[ell] + j] = sl;
        s.hd[N.hoff[ell] + j] = d;
        if (a.alpha_used) a.alpha_used[(dom * H + t) * (int64_t)N.hidden + N.hoff[ell] + j] = al;
    }
    __syncthreads();
}

// a7: dynamics on the TM in FP64 into cn/Pn/Ilon/Ihin.  Ends with a barrier.
template <int NT>
__device__ void dynamics(const Dom& s, const NetDesc& N, const double* off) {
    const int tid = threadIdx.x, n = N.n, m = N.m, gld = odd_ld(n);
    for (int idx = tid; idx < n * n; idx += NT) {
        const int i = idx / n, k = idx - i * n;
        double acc = 0.0;
        for (int j = 0; j < n; ++j) acc = fma(s.A[i * n + j], s.P[j * n + k], acc);
        for (int j = 0; j < m; ++j) acc = fma(s.B[i * m + j], (double)s.G[j * gld + k], acc);
        s.Pn[idx] = acc;
    }
    for (int i = tid; i < n; i += NT) {
        double acc = s.e[i] + (off ? off[i] : 0.0), lo_ = 0.0, hi_ = 0.0;
        for (int j = 0; j < n; ++j) {
            const double aij = s.A[i * n + j];
            acc = fma(aij, s.c[j], acc);
            lo_ += posd(aij) * s.Ilo[j] + negd(aij) * s.Ihi[j];
            hi_ += posd(aij) * s.Ihi[j] + negd(aij) * s.Ilo[j];
        }
        for (int j = 0; j < m; ++j) {
            const double bij = s.B[i * m + j];
            acc = fma(bij, (double)s.cu[j], acc);
            lo_ += posd(bij) * (double)s.Iulo[j] + negd(bij) * (double)s.Iuhi[j];
            hi_ += posd(bij) * (double)s.Iuhi[j] + negd(bij) * (double)s.Iulo[j];
        }
        s.cn[i] = acc;
        s.Ilon[i] = lo_;
        s.Ihin[i] = hi_;
    }
    __syncthreads();
}

// a8: EvalInt of the TM in cn/Pn/Ilon/Ihin with the current dual, outward by box_margin times the
// summed magnitude.  Returns this thread's width sum contribution.
template <int NT>
__device__ double eval_box(const Dom& s, const NetDesc& N, const FusedArgs& a, int64_t dom, int t1) {
    const int n = N.n, H = N.H;
    double vsum = 0.0;
    for (int i = threadIdx.x; i < n; i += NT) {
        double pm = 0.0, pp = 0.0, mag = fabs(s.cn[i]) + fabs(s.Ilon[i]) + fabs(s.Ihin[i]) + fabs(s.wv[0]);
        for (int k = 0; k < n; ++k) {
            const double x = s.Pn[i * n + k];
            pm += fabs(x - s.v[k]);
            pp += fabs(x + s.v[k]);
            mag += fabs(x) + fabs(s.v[k]);
        }
        const double bl = s.cn[i] + s.Ilon[i] - pm - s.wv[0] - a.box_margin * mag;
        const double bh = s.cn[i] + s.Ihin[i] + pp + s.wv[0] + a.box_margin * mag;
        if (a.lo) a.lo[(dom * (H + 1) + t1) * n + i] = bl;
        if (a.hi) a.hi[(dom * (H + 1) + t1) * n + i] = bh;
        vsum += bh - bl;
        if (!isfinite(bl) || !isfinite(bh)) atomicOr(reinterpret_cast<unsigned int*>(&s.misc[1]), DR_STATUS_NONFINITE_BIT);
        if (bl > bh) atomicOr(reinterpret_cast<unsigned int*>(&s.misc[1]), DR_STATUS_INFEASIBLE_BIT);
    }
    return vsum;
}

// Slab mode: the padded weight layout of the shared-memory region Ws, written once for all CTAs.
__global__ void k_pad_weights(const NetDesc N, FusedLayout Y, const float* __restrict__ W, float* __restrict__ out) {
    for (int l = 0; l < N.L; ++l) {
        const int rows = N.w[l + 1], cols = N.w[l], ld = odd_ld(cols);
        float* dst = out + (Y.Ws[l] - Y.Ws[0]) / 4;
        for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)rows * ld;
             idx += (int64_t)gridDim.x * blockDim.x) {
            const int r = (int)(idx / ld), q = (int)(idx - (int64_t)r * ld);
            dst[idx] = q < cols ? W[N.Woff[l] + (int64_t)r * cols + q] : 0.f;
        }
    }
}

// One controller pass of step t (all targets) on the current FP32 view.  With `vsnap`
// non-null the dual vector seen by each hidden layer's concretisation is kept.
template <int NT>
__device__ void controller_pass(const Dom& s, const NetDesc& N, const FusedArgs& a, int64_t dom, int64_t sp_end, int t,
                                float* vsnap, float* levall = nullptr, float* kall = nullptr) {
    const int n = N.n, L = N.L;
    for (int ell = 1; ell <= L; ++ell) {
        int ld;
        const float* cur = chain<NT>(s, N, ell, (levall && ell >= 2) ? levall + levall_offset(N, ell) : nullptr, &ld);
        if (kall) {
            const int ko = kall_offset(N, ell), kt = kall_total(N);
            for (int i = threadIdx.x; i < N.w[ell]; i += NT) {
                kall[ko + i] = s.klo[i];
                kall[kt + ko + i] = s.khi[i];
            }
            __syncthreads();
        }
        if (vsnap && ell < L) {
            for (int k = threadIdx.x; k <= n; k += NT) vsnap[ell * (n + 1) + k] = s.vf[k];
        }
        project<NT>(s, N, ell, cur, ld, a.rho);
        if (ell < L) {
            apply_splits(s, N, a, sp_end, t, ell, a.rho);
            relax<NT>(s, N, a, dom, t, ell);
        }
    }
}

template <int NT>
__global__ void __launch_bounds__(NT, 2) k_fused_forward(const FusedArgs a) {
    extern __shared__ __align__(16) unsigned char sm_dyn[];
    unsigned char* sm = a.gslab ? a.gslab + (int64_t)blockIdx.x * a.slab_stride : sm_dyn;
    const NetDesc& N = a.net;
    Dom s = make_dom(sm, a.lay);
    s.gw = a.gwpad;
    s.tiles = (NT == 256 && a.gslab) ? reinterpret_cast<float*>(sm_dyn) : nullptr;  // slab mode: GEMM tiles
    const int tid = threadIdx.x;
    const int64_t dom = a.d0 + blockIdx.x;
    const int n = N.n, H = N.H;

    load_params<NT>(s, a);
    // a1: BuildLinearTM over the normalised box
    const double* lo0 = a.lo0 + dom * n;
    const double* hi0 = a.hi0 + dom * n;
    for (int idx = tid; idx < n * n; idx += NT) {
        const int i = idx / n, k = idx - i * n;
        s.P[idx] = (i == k) ? 0.5 * (hi0[i] - lo0[i]) : 0.0;
    }
    for (int i = tid; i < n; i += NT) {
        s.c[i] = 0.5 * (lo0[i] + hi0[i]);
        s.Ilo[i] = 0.0;
        s.Ihi[i] = 0.0;
        s.v[i] = 0.0;
        if (a.lo) a.lo[(dom * (H + 1)) * n + i] = lo0[i];
        if (a.hi) a.hi[(dom * (H + 1)) * n + i] = hi0[i];
    }
    const int64_t sp_end = a.sp_row ? a.sp_row[dom + 1] : 0;
    if (tid == 0) {
        s.wv[0] = 0.0;
        s.misc[0] = a.sp_row ? (int)a.sp_row[dom] : 0;
        s.misc[1] = 0;
    }
    double vacc = 0.0;
    __syncthreads();

    for (int t = 0; t < H; ++t) {
        if (a.tape) {
            double* tp = a.tape + (dom * H + t) * (int64_t)a.tape_stride;
            for (int idx = tid; idx < n * n; idx += NT) tp[idx] = s.P[idx];
            for (int i = tid; i < n; i += NT) {
                tp[n * n + i] = s.c[i];
                tp[n * n + n + i] = s.Ilo[i];
                tp[n * n + 2 * n + i] = s.Ihi[i];
                tp[n * n + 3 * n + i] = s.v[i];
            }
            if (tid == 0) {
                tp[n * n + 4 * n] = s.wv[0];
                tp[n * n + 4 * n + 1] = (double)s.misc[0];
            }
        }
        tm_view<NT>(s, n);
        controller_pass<NT>(s, N, a, dom, sp_end, t, nullptr);
        dynamics<NT>(s, N, a.eoff ? a.eoff + (dom * H + t) * (int64_t)n : nullptr);
        vacc += eval_box<NT>(s, N, a, dom, t + 1);
        __syncthreads();
        for (int idx = tid; idx < n * n; idx += NT) s.P[idx] = s.Pn[idx];
        for (int i = tid; i < n; i += NT) {
            s.c[i] = s.cn[i];
            s.Ilo[i] = s.Ilon[i];
            s.Ihi[i] = s.Ihin[i];
        }
        __syncthreads();
    }
    // per-domain objective V_d and status
    double* red = s.Pn;
    if (tid < n) red[tid] = vacc;
    __syncthreads();
    if (tid == 0) {
        double sum = 0.0;
        for (int i = 0; i < n; ++i) sum += red[i];
        if (a.V) a.V[dom] = sum;
        if (a.status) a.status[dom] = (uint32_t)s.misc[1];
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
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            slo[threadIdx.x] = fmin(slo[threadIdx.x], slo[threadIdx.x + st]);
            shi[threadIdx.x] = fmax(shi[threadIdx.x], shi[threadIdx.x + st]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        hull_lo[o] = slo[0];
        hull_hi[o] = shi[0];
    }
}
