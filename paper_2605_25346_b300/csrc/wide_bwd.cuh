// Staged reverse sweep for wide controllers: dV/dalpha, dV/dbeta and dV/d(centre shift) of the
// staged forward pass, with the chain's reverse products on the tensor cores.
//
// The forward pass of a chunk of domains runs in keep mode (wide.cuh): every step leaves its FP32
// view of the TM, the dual vector seen by each target, the pre-activation bounds before and after the
// split clipping, the slopes and intercepts, G = Lambda_x P and Lambda_x of every target, the chain
// levels Lambda^(m) before the slopes, the split values h, and the FP64 TM on the chunk's tape.  The
// reverse sweep then walks t = H-1 .. 0 and, inside a step, the targets l = L .. 1, in exactly the
// reverse order of the forward pass (the same order as the fused reverse kernel):
//   k_rv_dyn        EvalInt of box t+1 and the FP64 dynamics, reversed (adjoint of TM_t and of the
//                   controller TM)
//   k_rv_target     per target: the relaxation (slope and intercept adjoints -> bound adjoints and
//                   dV/dalpha), the split records (dV/dbeta), the concretisation with the split dual,
//                   the input projection (TM_t adjoints) and the adjoint of Lambda_x
//   chain reverse   levels m = 1 .. l-1: adjoint of Lambda_s = (adjoint of the level below) W_m^T +
//                   kappa-adjoint b_m^T, the column sums giving the slope and intercept adjoints of
//                   hidden layer m, and the adjoint of Lambda^(m) for the next level; on the tensor
//                   cores (persistent 3xTF32 GEMM, reverse epilogue EPI 3) for targets whose width is
//                   a multiple of 32, else on CUDA cores (k_rv_chain_rows for the few rows of the
//                   output target, k_rv_chain_simt for the rest)
//   k_rv_carry      the adjoint of TM_t becomes the incoming adjoint of step t-1
// Subgradient conventions are the fused reverse kernel's: |0|' = 0, Lambda^+/- have slope 0 at 0,
// the intercept max takes the first branch on a tie; the outward margins are constants.
#pragma once
#include "wide.cuh"

struct RevArgs {
    NetDesc net;  // H set
    const float* W;
    const float* b;
    const double* A;
    const double* B;
    int64_t d0;
    int Dc;
    const int64_t* sp_row;
    const SplitRec* sp;
    const float* beta;
    const float* sph;    // [nnz] split values h of the forward pass
    const float* alpha;  // user slopes (DR_SLOPE_USER) or null
    int mode;
    const double* wlo;  // [D][H+1][n] upstream gradient of lo (null: -1 on steps 1..H)
    const double* whi;  // null: +1
    float* dalpha;      // [D][H][hidden] or null
    float* dbeta;       // [nnz] or null
    double* gshift;     // [D][H+1][n] or null
    const double* tape; // [Dc][H+1][n*n + 4n + 2] chunk tape
    // keep slot of the step being reversed
    const float *Pf, *cf, *Ilof, *Ihif, *vsnap, *hl, *hu, *hs, *hd, *hl0, *hu0, *Gk, *LXk;
    int krows;
    // adjoint state (chunk-local)
    double *gcn, *gPn, *gIlon, *gIhin;  // adjoint of TM_{t+1}
    double *gc, *gP, *gIlo, *gIhi;      // adjoint of TM_t (accumulated over the step)
    double *gcu, *gPu, *gIulo, *gIuhi;  // adjoint of the controller TM
    double *gv, *gw;                    // adjoint of the split dual (carried over the steps)
    float *gs, *gd;                     // [Dc][hidden] adjoints of the slopes and intercepts of the step
    float *ga, *gklo, *gkhi, *gRlo, *gRhi;  // [Dc][maxw] per-row adjoints of the current target
    float* gG;                          // [Dc][maxw][n]
    // adjoint of Lambda_x written by k_rv_target: plain [Dc * rows][n] (gLx) or blocked TF32 parts
    // (gLxh/gLxl, tc::blk_index, ldk = ru32(n)) as the first reverse GEMM's left operand
    float *gLx, *gLxh, *gLxl;
    // CUDA-core chain reverse: the kept levels of the current target (index m; null = the shared
    // W_l at m = l-1) and two adjoint buffers [Dc][rows][ldw]
    const float* tlev[DR_MAXL + 1];
    float *gLa, *gLb;
    int ldw;
};

// Adjoint of EvalInt of box t+1 (from TM_{t+1} and the dual after step t, both on the tape) added to
// the incoming adjoint of TM_{t+1}, then the adjoint of the FP64 dynamics: TM_t and controller TM.
// One block per domain.
__global__ void k_rv_dyn(const RevArgs a, int t) {
    const NetDesc& N = a.net;
    const int n = N.n, m = N.m, H = N.H, d = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const int64_t dom = a.d0 + d;
    const int ts = n * n + 4 * n + 2;
    const double* tp = a.tape + ((int64_t)d * (H + 1) + t + 1) * ts;
    const double* Pn = tp;
    const double* v = tp + n * n + 3 * n;
    double* gcn = a.gcn + (int64_t)d * n;
    double* gPn = a.gPn + (int64_t)d * n * n;
    double* gIlon = a.gIlon + (int64_t)d * n;
    double* gIhin = a.gIhin + (int64_t)d * n;
    const int64_t wrow = (dom * (H + 1) + t + 1) * n;
    for (int i = tid; i < n; i += nt) {
        const double wl = a.wlo ? a.wlo[wrow + i] : -1.0;
        const double wh = a.whi ? a.whi[wrow + i] : 1.0;
        gcn[i] += wl + wh;
        gIlon[i] += wl;
        gIhin[i] += wh;
        for (int k = 0; k < n; ++k) {
            const double x = Pn[i * n + k];
            gPn[i * n + k] += -wl * sgnd(x - v[k]) + wh * sgnd(x + v[k]);
        }
    }
    for (int k = tid; k < n; k += nt) {
        double acc = 0.0;
        for (int i = 0; i < n; ++i) {
            const double wl = a.wlo ? a.wlo[wrow + i] : -1.0;
            const double wh = a.whi ? a.whi[wrow + i] : 1.0;
            const double x = Pn[i * n + k];
            acc += wl * sgnd(x - v[k]) + wh * sgnd(x + v[k]);
        }
        a.gv[(int64_t)d * n + k] += acc;
    }
    if (tid == 0) {
        double acc = 0.0;
        for (int i = 0; i < n; ++i) {
            const double wl = a.wlo ? a.wlo[wrow + i] : -1.0;
            const double wh = a.whi ? a.whi[wrow + i] : 1.0;
            acc += wh - wl;
        }
        a.gw[d] += acc;
    }
    __syncthreads();
    // gcn is now the whole adjoint of c_{t+1}: the gradient of a shift added after step t
    if (a.gshift)
        for (int i = tid; i < n; i += nt) a.gshift[(dom * (H + 1) + t + 1) * n + i] = gcn[i];
    double* gP = a.gP + (int64_t)d * n * n;
    double* gPu = a.gPu + (int64_t)d * m * n;
    for (int idx = tid; idx < n * n; idx += nt) {
        const int j = idx / n, k = idx - j * n;
        double acc = 0.0;
        for (int i = 0; i < n; ++i) acc += a.A[i * n + j] * gPn[i * n + k];
        gP[idx] = acc;
    }
    for (int idx = tid; idx < m * n; idx += nt) {
        const int j = idx / n, k = idx - j * n;
        double acc = 0.0;
        for (int i = 0; i < n; ++i) acc += a.B[i * m + j] * gPn[i * n + k];
        gPu[idx] = acc;
    }
    for (int j = tid; j < n; j += nt) {
        double c_ = 0.0, lo_ = 0.0, hi_ = 0.0;
        for (int i = 0; i < n; ++i) {
            const double x = a.A[i * n + j];
            c_ += x * gcn[i];
            lo_ += posd(x) * gIlon[i] + negd(x) * gIhin[i];
            hi_ += posd(x) * gIhin[i] + negd(x) * gIlon[i];
        }
        a.gc[(int64_t)d * n + j] = c_;
        a.gIlo[(int64_t)d * n + j] = lo_;
        a.gIhi[(int64_t)d * n + j] = hi_;
    }
    for (int j = tid; j < m; j += nt) {
        double c_ = 0.0, lo_ = 0.0, hi_ = 0.0;
        for (int i = 0; i < n; ++i) {
            const double x = a.B[i * m + j];
            c_ += x * gcn[i];
            lo_ += posd(x) * gIlon[i] + negd(x) * gIhin[i];
            hi_ += posd(x) * gIhin[i] + negd(x) * gIlon[i];
        }
        a.gcu[(int64_t)d * m + j] = c_;
        a.gIulo[(int64_t)d * m + j] = lo_;
        a.gIuhi[(int64_t)d * m + j] = hi_;
    }
    for (int j = tid; j < N.hidden; j += nt) {
        a.gs[(int64_t)d * N.hidden + j] = 0.f;
        a.gd[(int64_t)d * N.hidden + j] = 0.f;
    }
}

// Rows per shared-memory chunk of k_rv_target's column reductions, and its dynamic shared memory
// (floats): the bound adjoints of the rows, a chunk of Lambda_x, of G's adjoint, of G and of the rows'
// centre/remainder adjoints, and the FP32 view of TM_t (P padded to n + 1 columns) with the dual.
__host__ __device__ inline int rv_chunk_rows(int n) { return n <= 16 ? 64 : 16; }
__host__ __device__ inline int rv_target_smem_floats(int rows, int n) {
    const int CH = rv_chunk_rows(n);
    return 2 * rows + 3 * CH * n + 3 * CH + n * (n + 1) + 3 * n + n + 1;
}
// Column-reduction outputs per thread (256 threads): n^2 + 4n + 1 items, 2 per thread for n <= 16, at
// most 18 for n <= 64.
__host__ __device__ inline int rv_items_per_thread(int n) { return (n * n + 4 * n + 1 + 255) / 256; }

// Target ell of step t, reversed (one block of 256 threads per domain): for a hidden target the
// relaxation (with dV/dalpha), the split records (dV/dbeta) and the concretisation with the dual; for
// the output target the controller TM's adjoint; then, for every target, the input projection
// (adjoints of the FP32 view of TM_t, which pass to the FP64 TM unchanged), and for ell >= 2 the
// adjoint of Lambda_x for the chain reverse.  Element-wise phases run one thread per (row, column)
// (coalesced); the sums over the rows run per output from chunks of rows staged in shared memory,
// FP32 within a chunk and FP64 across chunks.
template <int kRvMaxItems>
__global__ void __launch_bounds__(256) k_rv_target(const RevArgs a, int ell, int t) {
    extern __shared__ float rsm[];
    const NetDesc& N = a.net;
    const int n = N.n, m = N.m, L = N.L, H = N.H, rows = N.w[ell];
    const int d = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const int64_t dom = a.d0 + d;
    const int CH = rv_chunk_rows(n), pn = n + 1;
    float* sgl = rsm;
    float* sgu = sgl + rows;
    float* cLx = sgu + rows;
    float* cgG = cLx + CH * n;
    float* cG = cgG + CH * n;
    float* cga = cG + CH * n;
    float* cRlo = cga + CH;
    float* cRhi = cRlo + CH;
    float* sPf = cRhi + CH;  // [n][n + 1]
    float* scf = sPf + n * pn;
    float* sIlo = scf + n;
    float* sIhi = sIlo + n;
    float* svb = sIhi + n;  // [n + 1]
    float* ga = a.ga + (int64_t)d * N.maxw;
    float* gklo = a.gklo + (int64_t)d * N.maxw;
    float* gkhi = a.gkhi + (int64_t)d * N.maxw;
    float* gRlo = a.gRlo + (int64_t)d * N.maxw;
    float* gRhi = a.gRhi + (int64_t)d * N.maxw;
    float* gG = a.gG + (int64_t)d * N.maxw * n;
    const int koff = ell < L ? N.hoff[ell] : N.hidden;
    const float* G = a.Gk + ((int64_t)d * a.krows + koff) * n;
    const float* Lx = a.LXk + ((int64_t)d * a.krows + koff) * n;
    const float* vb = a.vsnap + ((int64_t)d * L + ell - 1) * (n + 1);
    double* gv = a.gv + (int64_t)d * n;
    double* gw = a.gw + d;
    for (int idx = tid; idx < n * n; idx += nt) sPf[(idx / n) * pn + idx % n] = a.Pf[(int64_t)d * n * n + idx];
    for (int j = tid; j < n; j += nt) {
        scf[j] = a.cf[(int64_t)d * n + j];
        sIlo[j] = a.Ilof[(int64_t)d * n + j];
        sIhi[j] = a.Ihif[(int64_t)d * n + j];
    }
    for (int k = tid; k <= n; k += nt) svb[k] = vb[k];
    if (ell == L) {
        for (int idx = tid; idx < rows * n; idx += nt) gG[idx] = (float)a.gPu[(int64_t)d * m * n + idx];
        for (int i = tid; i < rows; i += nt) {
            const double c_ = a.gcu[(int64_t)d * m + i], lo = a.gIulo[(int64_t)d * m + i], hi = a.gIuhi[(int64_t)d * m + i];
            const float cf = (float)c_, dl = (float)(lo - hi);
            ga[i] = cf;
            gklo[i] = 0.5f * cf + 0.5f * dl;
            gkhi[i] = 0.5f * cf - 0.5f * dl;
            gRlo[i] = (float)lo;
            gRhi[i] = (float)hi;
        }
    } else {
        const int ho = N.hoff[ell];
        const int64_t hb = (int64_t)d * N.hidden + ho;
        // relaxation reverse (post-clip bounds), then the clip
        for (int j = tid; j < rows; j += nt) {
            const float l = a.hl[hb + j], u = a.hu[hb + j];
            const float g_s = a.gs[hb + j], g_d = a.gd[hb + j];
            float g_l = 0.f, g_u = 0.f, g_a = 0.f;
            if (l < 0.f && u > 0.f) {
                float al;
                if (a.mode == DR_SLOPE_CHORD_K) al = u / (u - l);
                else if (a.mode == DR_SLOPE_ADAPTIVE_K) al = (u >= -l) ? 1.f : 0.f;
                else if (a.mode == DR_SLOPE_ZERO_K) al = 0.f;
                else al = a.alpha[(dom * H + t) * (int64_t)N.hidden + ho + j];
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
            if (a.hl0[hb + j] != l) g_l = 0.f;  // clipped by a split
            if (a.hu0[hb + j] != u) g_u = 0.f;
            sgl[j] = g_l;
            sgu[j] = g_u;
            ga[j] = 0.f;
            gklo[j] = 0.f;
            gkhi[j] = 0.f;
            gRlo[j] = 0.f;
            gRhi[j] = 0.f;
        }
        for (int idx = tid; idx < rows * n; idx += nt) gG[idx] = 0.f;
        __syncthreads();
        // split records of (t, ell): v += beta sign G_j, w += beta h (adjoint of the updated dual)
        if (tid == 0 && a.sp_row) {
            const int ts = n * n + 4 * n + 2;
            const int cursor0 = (int)a.tape[((int64_t)d * (H + 1) + t) * ts + n * n + 4 * n + 1];
            const int64_t sp_end = a.sp_row[dom + 1];
            for (int64_t cpos = cursor0; cpos < sp_end; ++cpos) {
                const SplitRec r = a.sp[cpos];
                if (r.t > t) break;
                if (r.t != t || r.layer != ell) continue;
                const int j = r.neuron;
                const float bt = a.beta ? a.beta[cpos] : 0.f;
                double gbv = gw[0] * (double)a.sph[cpos];
                for (int k = 0; k < n; ++k) gbv += gv[k] * (double)r.sign * (double)G[j * n + k];
                if (a.dbeta) a.dbeta[cpos] = (float)gbv;
                if (bt != 0.f) {
                    for (int k = 0; k < n; ++k) gG[j * n + k] += (float)((double)bt * (double)r.sign * gv[k]);
                    const float hbv = (float)((double)bt * gw[0]);
                    if (r.sign > 0) {
                        ga[j] += hbv;
                        gkhi[j] += hbv;
                        gRhi[j] += hbv;
                    } else {
                        ga[j] -= hbv;
                        gklo[j] -= hbv;
                        gRlo[j] -= hbv;
                    }
                }
            }
        }
        __syncthreads();
        // concretisation reverse with the dual vector this target saw
        for (int idx = tid; idx < rows * n; idx += nt) {
            const int i = idx / n, k = idx - i * n;
            const float x = G[idx];
            gG[idx] += -sgl[i] * sgnf(x - svb[k]) + sgu[i] * sgnf(x + svb[k]);
        }
        for (int i = tid; i < rows; i += nt) {
            const float g_l = sgl[i], g_u = sgu[i];
            ga[i] += g_l + g_u;
            gklo[i] += g_l;
            gkhi[i] += g_u;
            gRlo[i] += g_l;
            gRhi[i] += g_u;
        }
    }
    __syncthreads();
    // sums over the rows, one output per item: q < n^2: gP[j][k] (q = j n + k); then gc[j], gIlo[j],
    // gIhi[j]; for a hidden target also gv[k] and gw (the adjoint of the dual it saw)
    const int nq = n * n + 3 * n + (ell < L ? n + 1 : 0);
    double acc[kRvMaxItems];
#pragma unroll
    for (int u = 0; u < kRvMaxItems; ++u) acc[u] = 0.0;
    for (int i0 = 0; i0 < rows; i0 += CH) {
        const int ch = min(CH, rows - i0);
        for (int idx = tid; idx < ch * n; idx += nt) {
            const int64_t o = (int64_t)i0 * n + idx;
            cLx[idx] = Lx[o];
            cgG[idx] = gG[o];
            if (ell < L) cG[idx] = G[o];
        }
        for (int i = tid; i < ch; i += nt) {
            cga[i] = ga[i0 + i];
            cRlo[i] = gRlo[i0 + i];
            cRhi[i] = gRhi[i0 + i];
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kRvMaxItems; ++u) {
            const int q = tid + u * nt;
            if (q >= nq) break;
            float s = 0.f;
            if (q < n * n) {
                const int j = q / n, k = q - j * n;
                for (int i = 0; i < ch; ++i) s = fmaf(cLx[i * n + j], cgG[i * n + k], s);
            } else if (q < n * n + n) {
                const int j = q - n * n;
                for (int i = 0; i < ch; ++i) s = fmaf(cLx[i * n + j], cga[i], s);
            } else if (q < n * n + 2 * n) {
                const int j = q - n * n - n;
                for (int i = 0; i < ch; ++i) {
                    const float x = cLx[i * n + j];
                    s += cRlo[i] * posf(x) + cRhi[i] * negf(x);
                }
            } else if (q < n * n + 3 * n) {
                const int j = q - n * n - 2 * n;
                for (int i = 0; i < ch; ++i) {
                    const float x = cLx[i * n + j];
                    s += cRlo[i] * negf(x) + cRhi[i] * posf(x);
                }
            } else if (q < n * n + 4 * n) {
                const int k = q - n * n - 3 * n;
                for (int i = 0; i < ch; ++i) {
                    const float x = cG[i * n + k];
                    s += sgl[i0 + i] * sgnf(x - svb[k]) + sgu[i0 + i] * sgnf(x + svb[k]);
                }
            } else {
                for (int i = 0; i < ch; ++i) s += sgu[i0 + i] - sgl[i0 + i];
            }
            acc[u] += (double)s;
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < kRvMaxItems; ++u) {
        const int q = tid + u * nt;
        if (q >= nq) break;
        if (q < n * n) a.gP[(int64_t)d * n * n + q] += acc[u];
        else if (q < n * n + n) a.gc[(int64_t)d * n + q - n * n] += acc[u];
        else if (q < n * n + 2 * n) a.gIlo[(int64_t)d * n + q - n * n - n] += acc[u];
        else if (q < n * n + 3 * n) a.gIhi[(int64_t)d * n + q - n * n - 2 * n] += acc[u];
        else if (q < n * n + 4 * n) gv[q - n * n - 3 * n] += acc[u];
        else gw[0] += acc[u];
    }
    if (ell < 2) return;
    // adjoint of Lambda_x (rows x n): the centre, linear and remainder terms of the concretisation.
    // The blocked operand's padding columns n .. 31 stay zero (cleared once per sweep).
    const int nkx = ((n + 31) & ~31) >> 5;
    for (int idx = tid; idx < rows * n; idx += nt) {
        const int i = idx / n, j = idx - i * n;
        const float x = Lx[idx];
        const float* gr = gG + (int64_t)i * n;
        const float* pr = sPf + j * pn;
        float v = ga[i] * scf[j];
        for (int k = 0; k < n; ++k) v = fmaf(gr[k], pr[k], v);
        v += gRlo[i] * (x > 0.f ? sIlo[j] : (x < 0.f ? sIhi[j] : 0.f));
        v += gRhi[i] * (x > 0.f ? sIhi[j] : (x < 0.f ? sIlo[j] : 0.f));
        const int64_t r = (int64_t)d * rows + i;
        if (a.gLxh) {
            const float h = tf32_part(v);
            const int64_t o = tc::blk_index(r, j, nkx);
            a.gLxh[o] = h;
            a.gLxl[o] = tf32_part(v - h);
        } else {
            a.gLx[r * n + j] = v;
        }
    }
}

// Slope and intercept adjoints of hidden layer mm from the reverse GEMM's column sums per row
// segment (colpart [segments][2][K], K = n_mm; 32-row segments, or one per domain when a domain has
// fewer rows), summed over each domain's segments in order.
__global__ void k_rv_colsum(const RevArgs a, int ell, int mm, const float* __restrict__ colpart) {
    const NetDesc& N = a.net;
    const int K = N.w[mm], nb = max(1, N.w[ell] >> 5);  // one segment per 32 rows, or per domain for fewer rows
    const int64_t total = (int64_t)a.Dc * K;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int d = (int)(idx / K), j = (int)(idx - (int64_t)d * K);
        float s = 0.f, dd = 0.f;
        for (int q = 0; q < nb; ++q) {
            const int64_t o = ((int64_t)d * nb + q) * 2 * K + j;
            s += colpart[o];
            dd += colpart[o + K];
        }
        a.gs[(int64_t)d * N.hidden + N.hoff[mm] + j] += s;
        a.gd[(int64_t)d * N.hidden + N.hoff[mm] + j] += dd;
    }
}

// Chain reverse of target ell on CUDA cores (any row count; the output target and targets whose
// width is not a multiple of 32): levels mm = 1 .. ell-1, one block per domain, a thread per column j
// of the level (neuron j of hidden layer mm).
__global__ void __launch_bounds__(256) k_rv_chain_simt(const RevArgs a, int ell) {
    const NetDesc& N = a.net;
    const int n = N.n, rows = N.w[ell], d = blockIdx.x;
    const float* gklo = a.gklo + (int64_t)d * N.maxw;
    const float* gkhi = a.gkhi + (int64_t)d * N.maxw;
    const float* prev = a.gLx + (int64_t)d * rows * n;
    int pld = n;
    for (int mm = 1; mm <= ell - 1; ++mm) {
        const int K = N.w[mm], NN = N.w[mm - 1];
        const float* Wm = a.W + N.Woff[mm - 1];
        const float* Wl = a.W + N.Woff[ell - 1];
        const float* lev = a.tlev[mm];
        const float* sl = a.hs + (int64_t)d * N.hidden + N.hoff[mm];
        const float* dl = a.hd + (int64_t)d * N.hidden + N.hoff[mm];
        const float* bm = a.b + N.boff[mm - 1];
        float* next = ((mm & 1) ? a.gLa : a.gLb) + (int64_t)d * rows * a.ldw;
        for (int j = threadIdx.x; j < K; j += blockDim.x) {
            float acc_s = 0.f, acc_d = 0.f;
            const float* wrow = Wm + (int64_t)j * NN;
            for (int i = 0; i < rows; ++i) {
                float g = (gklo[i] + gkhi[i]) * bm[j];
                const float* pr = prev + (int64_t)i * pld;
                for (int k = 0; k < NN; ++k) g = fmaf(pr[k], wrow[k], g);
                const float lam = lev ? lev[tc::blk_index((int64_t)d * rows + i, j, (K + 31) >> 5)] : Wl[(int64_t)i * K + j];
                acc_s = fmaf(lam, g, acc_s);
                acc_d += gkhi[i] * posf(lam) + gklo[i] * negf(lam);
                if (mm < ell - 1)
                    next[(int64_t)i * a.ldw + j] = g * sl[j] + gkhi[i] * (lam > 0.f ? dl[j] : 0.f) + gklo[i] * (lam < 0.f ? dl[j] : 0.f);
            }
            a.gs[(int64_t)d * N.hidden + N.hoff[mm] + j] += acc_s;
            a.gd[(int64_t)d * N.hidden + N.hoff[mm] + j] += acc_d;
        }
        __syncthreads();
        prev = next;
        pld = a.ldw;
    }
}

// Chain reverse of a target with few rows (the output target; at most 32 rows) on CUDA cores: one
// block per domain, the adjoint rows of the level below in shared memory (two buffers of
// rows x ldw floats), a warp per column j of the level reading W_m's row j coalesced (lanes over k)
// into row partial sums, which a warp reduction completes; lane r then finishes row r of the column.
__global__ void __launch_bounds__(256) k_rv_chain_rows(const RevArgs a, int ell) {
    extern __shared__ float csm[];
    const NetDesc& N = a.net;
    const int n = N.n, rows = N.w[ell], d = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const float* gklo = a.gklo + (int64_t)d * N.maxw;
    const float* gkhi = a.gkhi + (int64_t)d * N.maxw;
    float* prev = csm;
    float* next = csm + rows * a.ldw;
    for (int idx = threadIdx.x; idx < rows * n; idx += blockDim.x) prev[idx] = a.gLx[(int64_t)d * rows * n + idx];
    __syncthreads();
    int pld = n;
    const float* Wl = a.W + N.Woff[ell - 1];
    for (int mm = 1; mm <= ell - 1; ++mm) {
        const int K = N.w[mm], NN = N.w[mm - 1];
        const bool top = mm == ell - 1;
        const float* Wm = a.W + N.Woff[mm - 1];
        const float* lev = a.tlev[mm];
        const float* sl = a.hs + (int64_t)d * N.hidden + N.hoff[mm];
        const float* dl = a.hd + (int64_t)d * N.hidden + N.hoff[mm];
        const float* bm = a.b + N.boff[mm - 1];
        for (int j = warp; j < K; j += nwarps) {
            const float* wrow = Wm + (int64_t)j * NN;
            const float bj = bm[j], sj = sl[j], dj = dl[j];
            float S = 0.f, Dd = 0.f;
            for (int rb = 0; rb < rows; rb += 8) {
                float acc[8];
#pragma unroll
                for (int r = 0; r < 8; ++r) acc[r] = 0.f;
                for (int k = lane; k < NN; k += 32) {
                    const float w = __ldg(wrow + k);
#pragma unroll
                    for (int r = 0; r < 8; ++r)
                        if (rb + r < rows) acc[r] = fmaf(prev[(rb + r) * pld + k], w, acc[r]);
                }
                float mine = 0.f;
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const float tot = warp_sum(acc[r]);
                    if (lane == r) mine = tot;
                }
                const int i = rb + lane;
                float ps = 0.f, pd = 0.f;
                if (lane < 8 && i < rows) {
                    const float kl = gklo[i], kh = gkhi[i];
                    const float g = fmaf(kl + kh, bj, mine);
                    const float lam = lev ? lev[tc::blk_index((int64_t)d * rows + i, j, (K + 31) >> 5)] : Wl[(int64_t)i * K + j];
                    ps = lam * g;
                    pd = kh * posf(lam) + kl * negf(lam);
                    if (!top) next[i * a.ldw + j] = g * sj + kh * (lam > 0.f ? dj : 0.f) + kl * (lam < 0.f ? dj : 0.f);
                }
                S += warp_sum(ps);
                Dd += warp_sum(pd);
            }
            if (lane == 0) {
                a.gs[(int64_t)d * N.hidden + N.hoff[mm] + j] += S;
                a.gd[(int64_t)d * N.hidden + N.hoff[mm] + j] += Dd;
            }
        }
        __syncthreads();
        float* t = prev;
        prev = next;
        next = t;
        pld = a.ldw;
    }
}

// End of step t: the adjoint of TM_t becomes the incoming adjoint of step t-1; after step 0 the
// adjoint of the initial centre is dV/d(shift at t = 0).
__global__ void k_rv_carry(const RevArgs a, int t) {
    const int n = a.net.n, H = a.net.H;
    const int64_t total = (int64_t)a.Dc * n;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int d = (int)(idx / n), i = (int)(idx - (int64_t)d * n);
        a.gcn[idx] = a.gc[idx];
        a.gIlon[idx] = a.gIlo[idx];
        a.gIhin[idx] = a.gIhi[idx];
        for (int k = 0; k < n; ++k) a.gPn[idx * n + k] = a.gP[idx * n + k];
        if (t == 0 && a.gshift) a.gshift[((a.d0 + d) * (H + 1)) * n + i] = a.gc[idx];
    }
}
